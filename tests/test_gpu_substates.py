"""Separate sub-states on the GPU (Section 4.1): components that no E has
joined live in separate arrays, each measure pass reads only its own
component's array, and an E between components joins them by a tensor
product.  The results equal the one-array runs and the oracle (O-A, which
keeps separate sub-states itself) in both precisions and modes; a run of two
brickwork blocks keeps them apart until the joining E, with pass groups
inside each component."""
import numpy as np
import pytest

from oracle import proa, substate, substate_c
from owqs_inputs import workloads
from owqs_inputs.patterns import E, M, N, Pattern
from owqs_inputs.rng import SplitMix64, random_state

from helpers import outcomes_by_label, phase_aligned_maxabs

pytestmark = pytest.mark.gpu

TOL = {"c128": 1e-12, "c64": 2e-5}
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


def _run(env, h, psi, dtype, mode, bits, layout):
    torch, owqs = env
    t = torch.complex64 if dtype == "c64" else torch.complex128
    dev = None if psi is None else torch.from_numpy(np.asarray(psi)).to(t).cuda()
    out, _, probs, _ = h.run(dev, dtype=dtype, mode=mode, outcomes=bits, layout=layout)
    torch.cuda.synchronize()
    return out.cpu().numpy().astype(np.complex128), probs


def _compare(env, wl, psi, dtype, mode, expect_joins=None):
    torch, owqs = env
    p = wl.pattern
    h = owqs.load(p)
    h.reorder()  # an order that measures every domain first, valid in both modes
    op = proa.reorder_commands(p, h.order())
    # the C build of O-A: compensated probability sums, exact enough at the
    # 2^25-amplitude sub-states of the larger cases for the complex128 bound
    ref = substate_c.run(op, psi, outcomes=outcomes_by_label(p, wl.outcomes), mode=mode)
    got, probs = _run(env, h, psi, dtype, mode, wl.outcomes, "substates")
    one, probs1 = _run(env, h, psi, dtype, mode, wl.outcomes, "one_array")
    for x in (got, one):
        err = phase_aligned_maxabs(ref.psi_out, x) if dtype == "c64" else float(np.max(np.abs(ref.psi_out - x)))
        assert err <= TOL[dtype], (p.name, dtype, mode, err)
    if mode == "owqs":
        ref_p = np.array([ref.probs[q] for q in p.measured()])
        assert np.max(np.abs(probs - ref_p)) <= PROB_TOL[dtype], (p.name, dtype)
    else:
        assert np.all(probs == 0.5)
    plan = h.plan_memory(wl.outcomes, dtype=dtype, mode=mode, real_input=psi is not None)
    if expect_joins is not None:
        assert (plan["joins"] > 0) == expect_joins, plan
        kinds = {owqs.KERNEL_KIND[int(k)] for k in h.profile(None if psi is None else
                                                               torch.from_numpy(np.asarray(psi)).to(
                                                                   torch.complex64 if dtype == "c64" else
                                                                   torch.complex128).cuda(),
                                                               dtype=dtype, mode=mode, outcomes=wl.outcomes,
                                                               layout="substates")[2]}
        assert ("factor_join" in kinds) == expect_joins, kinds
    return h, plan


@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("mode", ["owqs", "eowqs"])
def test_joined_blocks(env, dtype, mode):
    for rows, cols in ((3, 4), (4, 6)):
        _compare(env, workloads.joined_bricks(rows, cols, 2), None, dtype, mode, expect_joins=True)
    _compare(env, workloads.joined_bricks(3, 3, 3), None, dtype, mode, expect_joins=True)


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_components_with_pass_groups(env, dtype):
    """Two 12-row blocks: each component reaches 13 live qubits, where pass
    groups form; the one-array run holds up to 25."""
    torch, owqs = env
    wl = workloads.joined_bricks(12, 8, 2)
    h, plan = _compare(env, wl, None, dtype, "owqs", expect_joins=True)
    assert plan["uses_substates"] == 1 and plan["substate_bytes"] < plan["one_array_bytes"], plan
    kinds = {owqs.KERNEL_KIND[int(k)] for k in h.profile(None, dtype=dtype, outcomes=wl.outcomes,
                                                         layout="substates")[2]}
    assert "group_pass" in kinds, kinds


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_random_patterns_and_inputs(env, dtype):
    """Random J/CZ circuits with |+> inputs (each input its own component)
    and with a random input vector (one input component)."""
    rng = SplitMix64(511)
    for wl in workloads.random_batch(count=6, wmin=3, wmax=8, dmin=3, dmax=8):
        _compare(env, wl, None, dtype, "owqs")
        _compare(env, wl, random_state(rng, len(wl.pattern.inputs)), dtype, "owqs")


def test_scalar_component_and_default_choice(env):
    """A component measured away entirely leaves a one-amplitude factor that
    joins the output; a default run takes separate sub-states exactly when
    the plan says so."""
    torch, owqs = env
    p = Pattern(5, [0], [0, 4], [N(1), N(2), E(1, 2), M(1, 0.3), M(2, 0.9, (1,)), N(3), N(4), E(3, 4),
                                 M(3, 1.7), E(0, 4)], "scalar and late join")
    psi = random_state(SplitMix64(512), 1)
    bits = np.array([1, 0, 1], dtype=np.uint8)
    ref = substate.run(p, psi, outcomes=outcomes_by_label(p, bits))
    h = owqs.load(p)
    for dtype in ("c128", "c64"):
        got, _ = _run(env, h, psi, dtype, "owqs", bits, "substates")
        err = float(np.max(np.abs(ref.psi_out - got)))
        assert err <= TOL[dtype], (dtype, err)
    wl = workloads.brickwork(14, 8)
    h = owqs.load(wl.pattern)
    h.reorder()
    plan = h.plan_memory(wl.outcomes, real_input=True)
    assert plan["uses_substates"] == 0 and plan["joins"] == 0, plan
