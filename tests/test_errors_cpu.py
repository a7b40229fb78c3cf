"""Error paths of the C ABI that are decided on the host (no GPU needed):
live width above the compiler's limit, the EOWQS gflow pre-check (which runs
before any device work), sampled OWQS runs that cannot draw one measurement
at a time, and argument errors of the newer entry points."""
import ctypes as C

import pytest

from owqs_inputs.patterns import E, M, N, Pattern


@pytest.fixture(scope="module")
def owqs():
    from paper_1604_05659_gb300 import build, owqs as mod
    build.ensure_built()
    mod.library()
    return mod


def test_live_width_above_limit_is_oom(owqs):
    p = Pattern(63, list(range(63)), list(range(63)), [], "wide")
    h = owqs.load(p)
    with pytest.raises(owqs.OwqsError) as ei:
        h.describe_passes()
    assert ei.value.status == owqs.ERR_OOM


def test_eowqs_refuses_a_pattern_without_gflow_before_device_work(owqs):
    p = Pattern(2, [0], [1], [N(1), M(0, 0.0)], "no-flow")      # the qubits share no E
    h = owqs.load(p)
    assert h.find_flow("gflow") is None
    opts = owqs.owqs_run_opts(owqs.DTYPE["c128"], owqs.MODE["eowqs"], owqs.POLICY["zero"], 0, 0, None, 0, 0)
    st = owqs.library().owqs_run(h._h, C.byref(opts), None, None, None, None)
    assert st == owqs.ERR_NOT_DETERMINISTIC
    assert "gflow" in owqs.last_error()


def test_argument_errors_of_newer_entry_points(owqs):
    lib = owqs.library()
    p = Pattern(3, [0], [2], [N(1), N(2), E(0, 1), E(1, 2), M(0, 0.3), M(1, 0.2, sdom=(0,))], "chain")
    h = owqs.load(p)
    found = C.c_uint32()
    assert lib.owqs_find_flow(h._h, 7, C.byref(found), None, None, None, 0, None) == owqs.ERR_ARG
    n = C.c_uint32()
    assert lib.owqs_describe_launches(h._h, 5, 0, 0, None, None, None, None, 0, C.byref(n)) == owqs.ERR_ARG
    assert lib.owqs_test_wait_timeout(1, 0) == owqs.ERR_ARG
    assert lib.owqs_test_wait_timeout(0, 0) == owqs.OK
    # product input: every input in exactly one factor, checked before any device work
    opts = owqs.owqs_run_opts(owqs.DTYPE["c128"], owqs.MODE["owqs"], owqs.POLICY["zero"], 0, 0, None, 0, 0)
    sizes = (C.c_uint32 * 1)(1)
    qubits = (C.c_uint32 * 1)(1)                                   # qubit 1 is not an input
    vec = (C.c_double * 8)()
    addr = C.addressof(vec) + (-C.addressof(vec) % 16)          # a 16-byte aligned host address
    vecs = (C.c_void_p * 1)(addr)
    st = lib.owqs_run_product(h._h, C.byref(opts), 1, sizes, qubits, vecs, None, None, None)
    assert st == owqs.ERR_ARG


def test_sampled_owqs_refusals_come_before_device_work(owqs):
    """A sampled OWQS run under an order that measures a qubit before its
    domain (an EOWQS order) cannot draw one measurement at a time, and a
    profile of such a draw is refused; both are ERR_ARG before any device
    work.  The same order runs sampled in EOWQS mode, where every outcome is
    drawn first (not run here: that needs a GPU)."""
    from owqs_inputs import workloads
    p = workloads.brickwork(4, 4).pattern
    h = owqs.load(p)
    order, _ = h.reorder(mode="eowqs")
    pos = {q: i for i, q in enumerate(order)}
    assert any(pos[d] > pos[c.q0] for c in p.cmds if c.kind == "M" for d in list(c.sdom) + list(c.tdom))
    lib = owqs.library()
    for flags in (0, owqs.RUN_SEQUENTIAL_SAMPLING, owqs.RUN_HOST_SAMPLING):
        opts = owqs.owqs_run_opts(owqs.DTYPE["c64"], owqs.MODE["owqs"], owqs.POLICY["sampled"], 0, 7, None, 0, flags)
        assert lib.owqs_run(h._h, C.byref(opts), None, None, None, None) == owqs.ERR_ARG
        assert "domain first" in owqs.last_error()
    h.reset_order()
    opts = owqs.owqs_run_opts(owqs.DTYPE["c64"], owqs.MODE["owqs"], owqs.POLICY["sampled"], 0, 7, None, 0, 0)
    ms = (C.c_float * 64)()
    n = C.c_uint32()
    st = lib.owqs_profile_run(h._h, C.byref(opts), None, None, None, ms, None, None, None, 64, C.byref(n))
    assert st == owqs.ERR_ARG and "profiling" in owqs.last_error()
