"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Tolerances: complex128 amplitudes and probabilities within 1e-12 max-abs of
the oracle, complex64 amplitudes within 2e-5 max-abs after global-phase
alignment (forced-outcome results carry no phase freedom, so the alignment
is a no-op up to rounding) and complex64 probabilities within 1e-6.  Outcome
bits and index maps are compared exactly.
"""
import math

import numpy as np
import pytest

from oracle import proa, substate
from owqs_inputs import workloads
from owqs_inputs.patterns import E, M, N, Pattern, X, Z, circuit_to_pattern, random_jcz_circuit
from owqs_inputs.rng import SplitMix64, random_state

from helpers import outcomes_by_label, phase_aligned_maxabs
from test_oracle_pins import _wild_patterns, cnot_eq22

pytestmark = pytest.mark.gpu

TOL = {"c128": 1e-12, "c64": 2e-5}
# outcome probabilities: FP64 reductions of the complex64 amplitudes keep them
# within about 1e-7 of the oracle (observed at 2^28 amplitudes); 1e-6 leaves
# headroom for the rounding of the FP32 amplitudes themselves
PROB_TOL = {"c128": 1e-12, "c64": 1e-6}


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1604_05659_gb300 import build, owqs
    build.ensure_built()
    owqs.library()
    return torch, owqs


def _dev(torch, psi, dtype):
    if psi is None:
        return None
    t = torch.complex64 if dtype == "c64" else torch.complex128
    return torch.from_numpy(np.asarray(psi, dtype=np.complex128)).to(t).cuda()


def _oracle_for(h, p):
    order = h.order()
    return proa.reorder_commands(p, order) if p.is_standard() else p


def _compare(env, p, psi, bits, dtype, mode, reorder=True, graph=True, per_pass=False):
    torch, owqs = env
    h = owqs.load(p)
    if reorder and p.is_standard():
        h.reorder()
    op = _oracle_for(h, p) if reorder and p.is_standard() else p
    out, oc, probs, st = h.run(_dev(torch, psi, dtype), dtype=dtype, mode=mode, outcomes=bits, use_graph=graph,
                               per_pass=per_pass)
    torch.cuda.synchronize()
    ref = substate.run(op, psi, outcomes=outcomes_by_label(p, bits), mode=mode)
    got = out.cpu().numpy().astype(np.complex128)
    err = phase_aligned_maxabs(ref.psi_out, got) if dtype == "c64" else float(np.max(np.abs(ref.psi_out - got)))
    assert err <= TOL[dtype], (p.name, dtype, mode, err)
    if mode == "owqs":
        ref_p = np.array([ref.probs[q] for q in p.measured()])
        assert np.max(np.abs(probs - ref_p)) <= PROB_TOL[dtype]
    else:
        assert np.all(probs == 0.5)
    return h, got


def _small_cases():
    cases = [cnot_eq22(), workloads.small_random().pattern, workloads.brickwork(6, 10).pattern,
             workloads.qft(5, with_input=False).pattern]
    cases += [w.pattern for w in workloads.random_batch(count=8, wmin=3, wmax=9, dmin=3, dmax=10)]
    return cases


@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("mode", ["owqs", "eowqs"])
@pytest.mark.parametrize("per_pass", [False, True], ids=["one_kernel", "per_pass"])
def test_small_patterns(env, dtype, mode, per_pass):
    """Patterns whose arrays fit 2^8 amplitudes run in one single-block
    kernel; per_pass forces one kernel per pass.  Both against the oracle."""
    rng = SplitMix64(101)
    for p in _small_cases():
        psi = random_state(rng, len(p.inputs))
        bits = rng.bits(p.K)
        _compare(env, p, psi, bits, dtype, mode, per_pass=per_pass)
        _compare(env, p, None, bits, dtype, mode, per_pass=per_pass)


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_small_run_is_one_launch(env, dtype):
    """The single-block run: one launch where the planner says so, the same
    outputs and probabilities as one kernel per pass, and the same for a
    small unitary (the diagonal virtual input)."""
    torch, owqs = env
    rng = SplitMix64(111)
    tol = 1e-13 if dtype == "c128" else 1e-6
    for p in _small_cases():
        h = owqs.load(p)
        if p.is_standard():
            h.reorder()
        psi = _dev(torch, random_state(rng, len(p.inputs)), dtype)
        bits = rng.bits(p.K)
        plan = h.describe_launches(bits, dtype=dtype, real_input=True)
        ms, _, kd, _ = h.profile(psi, dtype=dtype, outcomes=bits)
        assert [owqs.KERNEL_KIND[int(k)] for k in kd] == [x[0] for x in plan], p.name
        a, _, pa, _ = h.run(psi, dtype=dtype, outcomes=bits)
        b, _, pb, _ = h.run(psi, dtype=dtype, outcomes=bits, per_pass=True)
        assert torch.max(torch.abs(a - b)).item() <= tol and np.max(np.abs(pa - pb)) <= tol, p.name
        if plan[0][0] == "small_run":
            assert len(kd) == 1
    p = circuit_to_pattern(3, random_jcz_circuit(3, 6, rng, cz_per_layer=1), "u3")
    h = owqs.load(p)
    h.reorder()
    bits = rng.bits(p.K)
    assert h.describe_launches(bits, dtype=dtype)[0][0] == "small_run"
    ua, _ = h.unitary(dtype=dtype, outcomes=bits)
    ub, _ = h.unitary(dtype=dtype, outcomes=bits, per_pass=True)
    assert torch.max(torch.abs(ua - ub)).item() <= tol


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_wild_patterns_pattern_order(env, dtype):
    """X/Z between measurements and every E up front (generic kernel, X
    masks, non-star sign functions)."""
    rng = SplitMix64(102)
    for p in _wild_patterns():
        psi = random_state(rng, len(p.inputs))
        for _ in range(2):
            _compare(env, p, psi, rng.bits(p.K), dtype, "owqs", reorder=False)


def dangling_pattern(n: int, m: int, seed: int) -> Pattern:
    """n input/output qubits with m extra qubits, each joined by E to one to
    three random outputs and measured right away: every such measurement is
    of a qubit prepared in the same segment (the fast kernel's new-bit case)."""
    rng = SplitMix64(seed)
    cmds = []
    for i in range(m):
        v = n + i
        cmds.append(N(v))
        nbr = set()
        for _ in range(1 + rng.randint(3)):
            nbr.add(rng.randint(n))
        cmds += [E(u, v) for u in sorted(nbr)]
        cmds.append(M(v, 2 * math.pi * rng.uniform()))
        if i % 3 == 0:
            a = rng.randint(n)
            b = (a + 1 + rng.randint(n - 1)) % n
            cmds.append(E(a, b))
    p = Pattern(n + m, list(range(n)), list(range(n)), cmds, f"dangling{n}+{m}")
    return p


def _medium_cases():
    """Several thread tiles and every fast-kernel case: measured bit 0 and 1,
    a middle bit, a newly prepared bit; widths 10-17."""
    cases = [workloads.brickwork(12, 16).pattern, workloads.qft(11, with_input=False).pattern]
    for i in range(4):
        rng = SplitMix64(900 + i)
        n = 10 + rng.randint(5)
        cases.append(circuit_to_pattern(n, random_jcz_circuit(n, 6, rng, cz_per_layer=3), f"rand{n}"))
    cases.append(dangling_pattern(13, 12, 905))
    cases.append(dangling_pattern(8, 10, 906))          # new-qubit case of the register-tiled pass
    cases.append(workloads.brickwork(16, 5).pattern)   # 2^16 per pass: TMA tiles, measured bit below and above 11
    return cases


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_medium_patterns_tiles(env, dtype):
    torch, owqs = env
    rng = SplitMix64(103)
    kinds = set()
    for p in _medium_cases():
        psi = random_state(rng, len(p.inputs))
        bits = rng.bits(p.K)
        h, _ = _compare(env, p, psi, bits, dtype, "owqs")
        ms, by, kd, _ = h.profile(_dev(torch, psi, dtype), dtype=dtype, outcomes=bits)
        kinds |= set(int(k) for k in kd)
    assert 0 in kinds and 2 in kinds   # fast passes and the final pass ran


def test_fast_kernel_variants_covered(env):
    """The medium cases hit every case of the register-tiled pass (measured
    bit 0, 1, middle, new qubit) and of the complex64 TMA pass (one run with
    the partner 2^b apart inside a 2^11 tile, two runs, new qubit)."""
    torch, owqs = env
    seen = set()
    for p in _medium_cases():
        h = owqs.load(p)
        if p.is_standard():
            h.reorder()
        for d in h.describe_passes(np.zeros(p.K, np.uint8)):
            if d.kind:
                continue
            star = all(d.b in (d.edges[e][0], d.edges[e][1]) for e in range(d.nedges)) and d.xmask == 0
            if not star:
                continue
            new = d.b >= d.n_in
            nlo = d.n_in if new else d.n_in - 1
            if nlo >= 11:
                seen.add(("c64", "tma", "new" if new else ("two_runs" if d.b >= 11 else "one_run")))
            if nlo >= 3 and nlo < 11:
                seen.add(("reg", "new" if new else ("mid" if d.b >= 3 else d.b)))
    want = {("c64", "tma", c) for c in ("one_run", "two_runs", "new")}
    want |= {("reg", 0), ("reg", 1), ("reg", "mid"), ("reg", "new")}
    assert want <= seen, want - seen


def test_graph_replay_matches_direct(env):
    torch, owqs = env
    wl = workloads.brickwork(10, 12)
    h = owqs.load(wl.pattern)
    h.reorder()
    outs = []
    for graph in (False, True, True):
        out, _, probs, _ = h.run(None, dtype="c64", outcomes=wl.outcomes, use_graph=graph)
        torch.cuda.synchronize()
        outs.append((out.cpu().numpy(), probs))
    for o, p in outs[1:]:
        assert np.array_equal(o, outs[0][0]) and np.array_equal(p, outs[0][1])


def test_sampled_outcomes_follow_the_oracle_stream(env):
    torch, owqs = env
    rng = SplitMix64(104)
    for p in _small_cases()[:6]:
        psi = random_state(rng, len(p.inputs))
        h = owqs.load(p)
        h.reorder()
        op = _oracle_for(h, p)
        for seed in (1, 2, 3):
            out, oc, probs, _ = h.run(_dev(torch, psi, "c128"), dtype="c128", policy="sampled", seed=seed)
            ref = substate.run(op, psi, policy="sampled", seed=seed)
            assert [int(oc[k]) for k in range(p.K)] == [ref.outcomes[q] for q in p.measured()]
            assert np.max(np.abs(out.cpu().numpy() - ref.psi_out)) <= 1e-12


def test_sampled_complex64_on_bulk_copy_tiles(env):
    """complex64 sampled runs on arrays wide enough for the bulk-copy pass
    (at least 2^11 live outputs): the outcome probabilities come from that
    kernel's probability mode.  Outcomes follow the oracle's stream, the
    probabilities and the output match within the complex64 tolerance."""
    torch, owqs = env
    rng = SplitMix64(131)
    for p in [workloads.brickwork(13, 6).pattern, workloads.qft(12, with_input=False).pattern]:
        psi = random_state(rng, len(p.inputs))
        h = owqs.load(p)
        h.reorder()
        op = _oracle_for(h, p)
        for seed in (11, 12):
            out, oc, probs, _ = h.run(_dev(torch, psi, "c64"), dtype="c64", policy="sampled", seed=seed,
                                      sequential_sampling=True)
            ref = substate.run(op, psi, policy="sampled", seed=seed)
            assert [int(oc[k]) for k in range(p.K)] == [ref.outcomes[q] for q in p.measured()], (p.name, seed)
            ref_p = np.array([ref.probs[q] for q in p.measured()])
            assert np.max(np.abs(probs - ref_p)) <= PROB_TOL["c64"], p.name
            got = out.cpu().numpy().astype(np.complex128)
            assert phase_aligned_maxabs(ref.psi_out, got) <= TOL["c64"], p.name


def test_eowqs_sampled_is_a_forced_run_of_fair_coins(env):
    """EOWQS with sampled outcomes (Section 4.5: every probability is 1/2):
    the outcomes are the oracle's fair-coin stream, every reported
    probability is 1/2, the output matches the oracle and is bit-identical
    to the forced EOWQS run of the same outcomes, and the run takes the
    forced run's launches (pass groups, no probability sweep)."""
    torch, owqs = env
    rng = SplitMix64(133)
    for p in [workloads.brickwork(13, 6).pattern, workloads.qft(10, with_input=False).pattern]:
        psi = random_state(rng, len(p.inputs))
        h = owqs.load(p)
        h.reorder()
        op = _oracle_for(h, p)
        for dtype in ("c64", "c128"):
            for seed in (21, 22):
                out, oc, probs, _ = h.run(_dev(torch, psi, dtype), dtype=dtype, mode="eowqs", policy="sampled",
                                          seed=seed)
                ref = substate.run(op, psi, mode="eowqs", policy="sampled", seed=seed)
                assert [int(oc[k]) for k in range(p.K)] == [ref.outcomes[q] for q in p.measured()], (p.name, seed)
                assert np.all(probs == 0.5)
                got = out.cpu().numpy().astype(np.complex128)
                assert phase_aligned_maxabs(ref.psi_out, got) <= TOL[dtype], (p.name, dtype)
                fout, _, _, _ = h.run(_dev(torch, psi, dtype), dtype=dtype, mode="eowqs", outcomes=oc)
                assert torch.equal(fout, out), (p.name, dtype, seed)
            _, _, kinds, _ = h.profile(_dev(torch, psi, dtype), dtype=dtype, mode="eowqs", policy="sampled")
            names = {owqs.KERNEL_KIND.get(int(k), str(k)) for k in kinds}
            assert not any("prob" in n or "decide" in n for n in names), names


def test_device_sampling_matches_host_sampling(env):
    """Outcomes drawn on the device (counter-based splitmix64, one graph)
    equal the per-measurement host draws bit for bit: same outcomes, same
    probabilities, same output, for complex64 and complex128, with and
    without a graph; a pattern with X between its measurements takes the
    host path and still follows the oracle's stream."""
    torch, owqs = env
    rng = SplitMix64(106)
    for p in [workloads.brickwork(12, 16).pattern, workloads.qft(11, with_input=False).pattern,
              workloads.small_random().pattern]:
        psi = random_state(rng, len(p.inputs))
        h = owqs.load(p)
        h.reorder()
        for dtype in ("c128", "c64"):
            for seed in (5, 6):
                dev_out, dev_oc, dev_p, _ = h.run(_dev(torch, psi, dtype), dtype=dtype, policy="sampled", seed=seed,
                                                  sequential_sampling=True)
                host_out, host_oc, host_p, _ = h.run(_dev(torch, psi, dtype), dtype=dtype, policy="sampled",
                                                     seed=seed, host_sampling=True)
                ng_out, ng_oc, ng_p, _ = h.run(_dev(torch, psi, dtype), dtype=dtype, policy="sampled", seed=seed,
                                               use_graph=False, sequential_sampling=True)
                assert np.array_equal(dev_oc, host_oc) and np.array_equal(dev_oc, ng_oc)
                assert np.array_equal(dev_p, host_p) and np.array_equal(dev_p, ng_p)
                assert torch.equal(dev_out, host_out) and torch.equal(dev_out, ng_out)
        op = _oracle_for(h, p)
        ref = substate.run(op, psi, policy="sampled", seed=7)
        out, oc, probs, _ = h.run(_dev(torch, psi, "c128"), dtype="c128", policy="sampled", seed=7)
        assert [int(oc[k]) for k in range(p.K)] == [ref.outcomes[q] for q in p.measured()]
        assert np.max(np.abs(out.cpu().numpy() - ref.psi_out)) <= 1e-12
    for p in _wild_patterns()[:2]:
        psi = random_state(rng, len(p.inputs))
        h = owqs.load(p)
        out, oc, _, _ = h.run(_dev(torch, psi, "c128"), dtype="c128", policy="sampled", seed=8)
        ref = substate.run(p, psi, policy="sampled", seed=8)
        assert [int(oc[k]) for k in range(p.K)] == [ref.outcomes[q] for q in p.measured()]
        assert np.max(np.abs(out.cpu().numpy() - ref.psi_out)) <= 1e-12


def test_sampling_by_a_checked_guess(env):
    """Sampled OWQS runs first run the guesses u > 1/2 as forced outcomes and
    keep that run iff every draw u_k <= prob_0 against the probabilities it
    computed reproduces its guess; otherwise they draw one measurement at a
    time.  Either way the outcomes are the one-at-a-time draw's (the oracle's
    stream): on flow patterns, where every probability is 1/2 (Section 4.5);
    on a measured input with prob_0 != 1/2, where the guess fails for u
    between prob_0 and 1/2; and where the guess is a branch of probability 0."""
    torch, owqs = env
    rng = SplitMix64(134)
    for p in [workloads.brickwork(12, 16).pattern, workloads.qft(11, with_input=False).pattern]:
        psi = random_state(rng, len(p.inputs))
        h = owqs.load(p)
        h.reorder()
        for dtype in ("c128", "c64"):
            for seed in (5, 6):
                g_out, g_oc, g_p, _ = h.run(_dev(torch, psi, dtype), dtype=dtype, policy="sampled", seed=seed)
                s_out, s_oc, s_p, _ = h.run(_dev(torch, psi, dtype), dtype=dtype, policy="sampled", seed=seed,
                                            sequential_sampling=True)
                assert np.array_equal(g_oc, s_oc), (p.name, dtype, seed)
                assert np.max(np.abs(g_p - s_p)) <= PROB_TOL[dtype]
                d = phase_aligned_maxabs(s_out.cpu().numpy().astype(np.complex128),
                                         g_out.cpu().numpy().astype(np.complex128))
                assert d <= TOL[dtype], (p.name, dtype, d)
    # one measured input qubit: prob_0 = |<+_a|psi>|^2
    p = Pattern(2, [0], [1], [N(1), M(0, 0.3)])
    h = owqs.load(p)
    psi = np.array([0.8, 0.6j])
    failed = 0
    for seed in range(40):
        ref = substate.run(p, psi, policy="sampled", seed=seed)
        u = SplitMix64(seed).uniform()
        failed += int(ref.outcomes[0] != (0 if u <= 0.5 else 1))
        out, oc, probs, _ = h.run(_dev(torch, psi, "c128"), dtype="c128", policy="sampled", seed=seed)
        assert int(oc[0]) == ref.outcomes[0], seed
        assert abs(probs[0] - ref.probs[0]) <= 1e-12
        assert np.max(np.abs(out.cpu().numpy() - ref.psi_out)) <= 1e-12
    assert failed >= 2   # the failed-guess path ran
    # |+> measured at angle 0: outcome 1 has probability 0
    p = Pattern(2, [0], [1], [N(1), M(0, 0.0)])
    h = owqs.load(p)
    plus = np.array([1, 1]) / math.sqrt(2)
    seeds = [sd for sd in range(16) if SplitMix64(sd).uniform() > 0.5]
    assert seeds
    for seed in seeds:
        out, oc, probs, st = h.run(_dev(torch, plus, "c128"), dtype="c128", policy="sampled", seed=seed)
        assert st == owqs.OK and int(oc[0]) == 0 and abs(probs[0] - 1.0) <= 1e-12


def test_host_io_matches_device_io(env):
    torch, owqs = env
    wl = workloads.qft(8)
    h = owqs.load(wl.pattern)
    h.reorder()
    dev, _, pd, _ = h.run(_dev(torch, wl.psi_in, "c64"), dtype="c64", outcomes=wl.outcomes)
    host_in = torch.from_numpy(wl.psi_in.astype(np.complex64)).pin_memory()
    host_out = torch.empty(1 << 8, dtype=torch.complex64).pin_memory()
    oc, ph = h.run_host(host_in, host_out, dtype="c64", outcomes=wl.outcomes)
    assert np.array_equal(host_out.numpy(), dev.cpu().numpy()) and np.array_equal(ph, pd)


def test_impossible_branch_and_eowqs_check(env):
    torch, owqs = env
    p = Pattern(2, [0], [1], [N(1), M(0, 0.0)])          # |+> measured at angle 0
    plus = np.array([1, 1]) / math.sqrt(2)
    h = owqs.load(p)
    out, _, probs, st = h.run(_dev(torch, plus, "c128"), dtype="c128", outcomes=[1], check=False)
    assert st == owqs.ERR_IMPOSSIBLE_BRANCH and probs[0] < 1e-24
    assert np.all(out.cpu().numpy() == 0)
    out, _, probs, st = h.run(_dev(torch, plus, "c128"), dtype="c128", outcomes=[0], check=False)
    assert st == owqs.OK and abs(probs[0] - 1) < 1e-15
    # EOWQS on a pattern without flow: the output norm is 2, flagged
    out, _, _, st = h.run(_dev(torch, plus, "c128"), dtype="c128", mode="eowqs", outcomes=[0], check=False)
    assert st == owqs.ERR_NOT_DETERMINISTIC
    with pytest.raises(ValueError):
        h.run(_dev(torch, plus, "c64"), dtype="c128", outcomes=[0])   # dtype mismatch caught in the binding


def test_qft24_full_size_closed_form(env):
    """QFT-shaped pattern on 24 logical qubits (2784 measurements, peak 25):
    the output equals the discrete Fourier transform of the bit-reversed
    input (the circuit has no final swaps) up to a global phase."""
    torch, owqs = env
    wl = workloads.qft(24)
    h = owqs.load(wl.pattern)
    _, info = h.reorder()
    assert info["peak_m"] == 25
    n = 24
    idx = np.arange(1 << n, dtype=np.int64)
    rev = np.zeros_like(idx)
    for b in range(n):
        rev |= ((idx >> b) & 1) << (n - 1 - b)
    ref = np.fft.ifft(wl.psi_in[rev]) * math.sqrt(1 << n)     # sum_x e^{+2 pi i x y / N} / sqrt(N)
    for dtype in ("c128", "c64"):
        out, _, probs, _ = h.run(_dev(torch, wl.psi_in, dtype), dtype=dtype, outcomes=wl.outcomes)
        got = out.cpu().numpy().astype(np.complex128)
        err = phase_aligned_maxabs(ref, got)
        assert err <= (1e-11 if dtype == "c128" else 2e-5), (dtype, err)
        assert np.max(np.abs(probs - 0.5)) <= PROB_TOL[dtype]


def test_brickwork_full_size_properties(env):
    """Brickwork 28 x 40 (1092 measurements, 2^28 live amplitudes): every
    branch probability is 1/2 (flow pattern, Section 4.5), the output is
    normalised, complex64 agrees with complex128 and a second outcome branch
    gives the same state up to a global phase."""
    torch, owqs = env
    wl = workloads.brickwork(28, 40)
    h = owqs.load(wl.pattern)
    _, info = h.reorder()
    assert info["peak_m"] == 29 and info["peak_live"] == 29
    o128, _, p128, _ = h.run(None, dtype="c128", outcomes=wl.outcomes)
    assert np.max(np.abs(p128 - 0.5)) <= 1e-12
    o64, _, p64, _ = h.run(None, dtype="c64", outcomes=wl.outcomes)
    assert np.max(np.abs(p64 - 0.5)) <= PROB_TOL["c64"]
    d = (o64.to(torch.complex128) - o128)
    ov = torch.vdot(o64.to(torch.complex128), o128)
    assert abs(abs(ov.item()) - 1) < 1e-5
    assert torch.max(torch.abs(o64.to(torch.complex128) * (ov / abs(ov)) - o128)).item() <= 2e-5
    assert abs(torch.linalg.vector_norm(o128).item() - 1) < 1e-12
    other = SplitMix64(55).bits(wl.pattern.K)
    o2, _, _, _ = h.run(None, dtype="c64", outcomes=other)
    ov2 = torch.vdot(o2, o64)
    assert abs(abs(ov2.item()) - 1) < 1e-4
    del d


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_pass_groups(env, dtype):
    """Up to twelve consecutive measure passes in one sweep: the output and
    every per-measurement probability still match the oracle, in both modes,
    from the virtual |+> input and from a random input; the profile shows the
    group kernel ran and covered most measurements."""
    torch, owqs = env
    rng = SplitMix64(105)
    for wl in (workloads.brickwork(14, 8), workloads.brickwork(13, 10), workloads.qft(12, with_input=False)):
        p = wl.pattern
        bits = rng.bits(p.K)
        h, _ = _compare(env, p, None, bits, dtype, "owqs")
        psi = random_state(rng, len(p.inputs))
        _compare(env, p, psi, bits, dtype, "owqs")
        _compare(env, p, psi, bits, dtype, "eowqs")
        # one array over every live qubit: the launches owqs_describe_launches
        # plans (a default run of a |+>-input pattern may take separate
        # sub-states instead, tests/test_gpu_substates.py)
        ms, by, kd, _ = h.profile(None, dtype=dtype, outcomes=bits, layout="one_array")
        assert (kd == 8).sum() >= 5, sorted(set(kd.tolist()))
        assert len(kd) < 0.6 * p.K, (len(kd), p.K)
        # the run launched exactly what the host planner describes
        plan = h.describe_launches(bits, dtype=dtype)
        assert [owqs.KERNEL_KIND[int(k)] for k in kd] == [x[0] for x in plan]
        assert list(h.profile_meas) == [x[2] for x in plan]


def _degenerate_patterns():
    """No measurement (E only; no command at all with permuted outputs; a
    new qubit entangled and kept), and no input (the first pass has a
    one-amplitude input)."""
    return [Pattern(2, [0, 1], [0, 1], [E(0, 1)], "cz_only"),
            Pattern(3, [0, 1, 2], [2, 0, 1], [], "permutation_only"),
            Pattern(3, [0, 1], [0, 1, 2], [N(2), E(0, 2), E(1, 2)], "prepare_only"),
            Pattern(2, [], [1], [N(0), N(1), E(0, 1), M(0, 0.3)], "no_input"),
            Pattern(3, [], [2], [N(0), N(1), N(2), E(0, 1), E(1, 2), M(0, 1.1), M(1, -0.4, sdom=(0,))],
                    "no_input_two_measurements")]


@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("per_pass", [False, True], ids=["one_kernel", "per_pass"])
def test_degenerate_patterns(env, dtype, per_pass):
    torch, owqs = env
    rng = SplitMix64(121)
    for p in _degenerate_patterns():
        h = owqs.load(p)
        bits = rng.bits(p.K)
        outs = outcomes_by_label(p, bits)
        for psi in (random_state(rng, len(p.inputs)), None):
            ref = substate.run(p, psi, outcomes=outs)
            out, _, probs, st = h.run(_dev(torch, psi, dtype), dtype=dtype, outcomes=bits, per_pass=per_pass)
            assert st == owqs.OK
            got = out.cpu().numpy().astype(np.complex128)
            err = phase_aligned_maxabs(ref.psi_out, got) if dtype == "c64" else float(np.max(np.abs(ref.psi_out - got)))
            assert err <= TOL[dtype], (p.name, dtype, per_pass, err)
            if p.K:
                ref_p = np.array([ref.probs[q] for q in p.measured()])
                assert np.max(np.abs(probs - ref_p)) <= PROB_TOL[dtype], p.name
