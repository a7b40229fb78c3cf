"""Launch planning on the host (owqs_describe_launches, no GPU): which
measurements run as pass groups, which as single passes, in what order.
These are the decisions the run driver makes; the GPU tests check that a
profiled run launches exactly these kernels."""
import pytest

from owqs_inputs import workloads
from owqs_inputs.rng import SplitMix64


@pytest.fixture(scope="module")
def owqs():
    from paper_1604_05659_gb300 import build, owqs as mod
    build.ensure_built()
    mod.library()
    return mod


def _check_cover(launches, K):
    """Every measurement once, in order; groups of 2..12 measurements; or the
    whole run in one single-block kernel."""
    if launches[0][0] == "small_run":
        assert launches == [("small_run", 0, K)], launches
        return
    at = 0
    for kind, first, n in launches:
        if n:
            assert first == at, (kind, first, at)
            at += n
        if kind == "group_pass":
            assert 2 <= n <= 12
        elif kind in ("fast_pass", "tma_pass", "generic_pass"):
            assert n == 1
        else:
            assert n == 0
    assert at == K
    assert launches[-1][0] == "final"


def test_brickwork_full_size_plan(owqs):
    wl = workloads.brickwork(28, 40)
    h = owqs.load(wl.pattern)
    h.reorder()
    for dtype in ("c64", "c128"):
        lv = h.describe_launches(wl.outcomes, dtype=dtype)        # virtual |+> input
        _check_cover(lv, wl.pattern.K)
        groups = [x for x in lv if x[0] == "group_pass"]
        assert lv[0] == ("group_pass", 0, 12)                    # the first group reads the virtual input
        assert len(lv) <= 120 and sum(x[2] for x in groups) >= 1085, (dtype, len(lv))
        lr = h.describe_launches(wl.outcomes, dtype=dtype, real_input=True)
        assert lr[0] == ("norm", 0, 0)
        _check_cover(lr, wl.pattern.K)


def test_qft_plan_and_small_arrays(owqs):
    wl = workloads.qft(24, with_input=False)
    h = owqs.load(wl.pattern)
    h.reorder()
    lr = h.describe_launches(wl.outcomes, real_input=True)
    _check_cover(lr, wl.pattern.K)
    assert len(lr) <= 260, len(lr)
    # live arrays narrower than one tile (2^9 amplitudes for complex64) never group
    small = workloads.small_random()
    hs = owqs.load(small.pattern)
    hs.reorder()
    ls = hs.describe_launches(small.outcomes, real_input=True)
    _check_cover(ls, small.pattern.K)
    assert not any(k == "group_pass" for k, _, _ in ls)


def test_random_patterns_cover_every_measurement(owqs):
    for wl in workloads.random_batch(12, 10, 16, 5, 20, config_index=4, start=50):
        h = owqs.load(wl.pattern)
        h.reorder()
        for dtype in ("c64", "c128"):
            for real in (False, True):
                _check_cover(h.describe_launches(wl.outcomes, dtype=dtype, real_input=real), wl.pattern.K)


def test_group_eligibility_follows_the_tile_width(owqs):
    """A group needs at least one tile of free indices: 2^9 input amplitudes
    for complex64 (a warp's 4 KB tile), 2^11 for complex128 (a block's 32 KB
    tile).  Brickworks of 7..11 rows have live arrays of rows or rows + 1
    qubits; below the boundary the measurements run as single passes and
    the first one reads the virtual input in the generic kernel (or, with
    every array at most 2^8 amplitudes, the whole run is one single-block
    kernel); from the boundary on the first group reads the virtual input
    itself."""
    first = {"c64": 9, "c128": 11}
    for rows in (7, 8, 9, 10, 11):
        wl = workloads.brickwork(rows, 6)
        h = owqs.load(wl.pattern)
        h.reorder()
        for dtype in ("c64", "c128"):
            for real in (False, True):
                plan = h.describe_launches(wl.outcomes, dtype=dtype, real_input=real)
                _check_cover(plan, wl.pattern.K)
                ngroups = sum(1 for k, _, _ in plan if k == "group_pass")
                assert (ngroups > 0) == (rows >= first[dtype]), (rows, dtype, real, plan[:3])
                if not real:
                    # every array at most 2^8 amplitudes: the whole run is one kernel
                    widest = max(max(d.n_in, d.n_out) for d in h.describe_passes(wl.outcomes))
                    expect = ("group_pass" if rows >= first[dtype] else
                              "small_run" if widest <= 8 else "generic_pass")
                    assert plan[0][0] == expect, (rows, dtype, plan[:2])


def test_small_run_boundary(owqs):
    """The single-block run takes at most 160 passes (its pass table sits in
    shared memory) and arrays of at most 2^8 amplitudes; beyond either the
    run has one kernel per pass."""
    from owqs_inputs.patterns import circuit_to_pattern, random_jcz_circuit
    for depth, small in ((53, True), (54, False)):
        p = circuit_to_pattern(3, random_jcz_circuit(3, depth, SplitMix64(5), cz_per_layer=1), "r3")
        h = owqs.load(p)
        h.reorder()
        assert len(h.describe_passes(None)) == p.K + 1
        plan = h.describe_launches(None, dtype="c64")
        _check_cover(plan, p.K)
        assert (plan[0][0] == "small_run") == small and (p.K + 1 <= 160) == small, (depth, p.K, plan[:2])
    wl = workloads.brickwork(9, 4)   # arrays of 2^9 amplitudes
    h = owqs.load(wl.pattern)
    h.reorder()
    assert h.describe_launches(wl.outcomes, dtype="c128")[0][0] != "small_run"


def test_group_slot_sequences_and_compiled_kernels(owqs):
    """owqs_describe_groups lists the same groups as owqs_describe_launches,
    with valid register-slot sequences (k <= 12 passes, slots below m, the
    first pass on slot 0, a new slot only after every lower one); all but at
    most two of the brickwork's groups run on kernels compiled for their
    sequence, the first one from the virtual |+> input included (a 2-qubit
    register); complex128 groups never do."""
    wl = workloads.brickwork(28, 40)
    h = owqs.load(wl.pattern)
    h.reorder()
    for real in (False, True):
        lv = [x for x in h.describe_launches(wl.outcomes, real_input=real) if x[0] == "group_pass"]
        gs = h.describe_groups(wl.outcomes, real_input=real)
        assert [len(g["slots"]) for g in gs] == [x[2] for x in lv]
        for i, g in enumerate(gs):
            sl = g["slots"]
            assert 2 <= len(sl) <= 12 and 1 <= g["m"] <= 4 and sl[0] == 0
            assert all(s < g["m"] for s in sl) and max(sl) == g["m"] - 1
            for j, s in enumerate(sl):
                assert s <= max(sl[:j], default=-1) + 1
            if not real and i == 0:   # the virtual input, on the sequence kernel of a 2-qubit register
                assert g["m"] == 2 and g["specialised"], g
        spec = [g["specialised"] for g in gs]
        assert sum(spec) >= len(spec) - 2, spec
        assert not any(g["specialised"] for g in h.describe_groups(wl.outcomes, dtype="c128", real_input=real))


def test_exact_half_groups(owqs):
    """A pass group sums no per-pass norms (bit 31 of the sequence code, "half") exactly when every
    pass measures a qubit joined by an odd number of E to the qubit it
    prepares: all groups of the J/CZ families, none of a chain whose
    prepared qubits get E twice (the identity), and all of the same chain
    with one E each."""
    for wl in (workloads.brickwork(12, 8), workloads.qft(12, with_input=False),
               workloads.random_batch(2, 12, 14, 10, 20)[0]):
        h = owqs.load(wl.pattern)
        h.reorder()
        for real in (False, True):
            gs = h.describe_groups(wl.outcomes, real_input=real)
            assert gs and all(g["half"] for g in gs), wl.name
    for joined, half in ((0, False), (1, True)):
        wl = workloads.chain_measurements(14, 9, joined_every=joined)
        h = owqs.load(wl.pattern)
        for dtype in ("c64", "c128"):
            gs = h.describe_groups(wl.outcomes, dtype=dtype, real_input=True)
            # nine passes on 3-qubit registers (arrays below 2^26 amplitudes take no 4-qubit register)
            assert len(gs) == 3 and all(g["m"] == 3 for g in gs), (joined, dtype, gs)
            assert all(g["half"] == half for g in gs), (joined, dtype, gs)


def test_memory_plan_separate_substates(owqs):
    """owqs_plan_memory: two brickwork blocks with |+> inputs stay separate
    sub-states until the joining E (joins, less memory and at most half the
    work of one array, so a default run takes them); with an input vector
    the inputs are one sub-state and the blocks share it from the start; the
    paper's m of the order is the widest sub-state at a measurement."""
    wl = workloads.joined_bricks(12, 8, 2)
    h = owqs.load(wl.pattern)
    order, info = h.reorder()
    plan = h.plan_memory(wl.outcomes)
    assert plan["joins"] >= 1 and plan["components"] >= 2 and plan["uses_substates"] == 1, plan
    assert plan["substate_bytes"] < plan["one_array_bytes"], plan
    assert 2 * plan["substate_work"] <= plan["one_array_work"], plan
    assert plan["peak_m"] <= info["peak_m"]
    one = h.plan_memory(wl.outcomes, real_input=True)
    assert one["joins"] == 0 and one["uses_substates"] == 0, one
    for dtype, amp in (("c64", 8), ("c128", 16)):
        p2 = h.plan_memory(wl.outcomes, dtype=dtype)
        assert p2["one_array_bytes"] % amp == 0 and p2["substate_bytes"] >= amp


def test_four_qubit_registers_from_a_width(owqs):
    """Complex64 groups take a 4-qubit register (at most 8 passes) only on
    arrays of at least 2^26 amplitudes, or from the width the test hook
    sets; complex128 groups never do."""
    wl = workloads.brickwork(14, 8)
    h = owqs.load(wl.pattern)
    h.reorder()
    assert max(g["m"] for g in h.describe_groups(wl.outcomes)) == 3
    try:
        owqs.test_group_m4_width(10)
        gs = h.describe_groups(wl.outcomes)
        assert any(g["m"] == 4 for g in gs) and all(len(g["slots"]) <= 8 for g in gs if g["m"] == 4)
        assert max(g["m"] for g in h.describe_groups(wl.outcomes, dtype="c128")) == 3
    finally:
        owqs.test_group_m4_width(0)
    big = workloads.brickwork(28, 40)
    hb = owqs.load(big.pattern)
    hb.reorder()
    gs = hb.describe_groups(big.outcomes)
    assert sum(g["m"] == 4 for g in gs) >= 30 and len(gs) <= 106


def test_compiled_sequences_cover_the_measured_families(owqs):
    """The compiled register-slot sequences carry the group work (passes x
    2^width) of the measured families: every brickwork 28x40 group, and at
    least 60 % of the recognition set's wide unitaries (13-14 inputs, whose
    arrays take 4-qubit registers: planned here through the test hook)."""
    big = workloads.brickwork(28, 40)
    h = owqs.load(big.pattern)
    h.reorder()
    assert all(g["specialised"] for g in h.describe_groups(big.outcomes))
    wide = [wl for wl in workloads.random_batch(count=256, with_input=False) if len(wl.pattern.inputs) > 12]
    assert len(wide) >= 50
    total = covered = 0.0
    try:
        owqs.test_group_m4_width(10)
        for wl in wide:
            hw = owqs.load(wl.pattern)
            hw.reorder()
            for g in hw.describe_groups(wl.outcomes, real_input=True):
                w = len(g["slots"]) * 2.0 ** g["n_in"]
                total += w
                covered += w if g["specialised"] else 0.0
            hw.close()
    finally:
        owqs.test_group_m4_width(0)
    assert covered >= 0.6 * total, covered / total
