"""The persistent kernels' shared-memory rings, wrapped many times, against
the oracle.

Every warp of the pass-group kernels (and every block of the bulk-copy pass)
walks its share of tiles through a small ring of stages, reusing a stage
once its data has been read, with mbarrier phases that flip on each round.
At full size every warp loops; in small parity cases the grid covers every
tile at once and no stage is reused.  Here the grid is capped (a test hook)
to one to three blocks, so that a brickwork or QFT pattern of 13-16 live
qubits makes every warp take 4-32 tiles through its ring (from |+>, the
first group's sequence kernel paces its ring without copies); and a brickwork of
23 live qubits runs with the full grid (at least three tiles per warp at the
production grid), checked against the C build of the oracle.  Both
precisions, |+> and random inputs, OWQS probabilities."""
import numpy as np
import pytest

from oracle import proa, substate, substate_c
from owqs_inputs import workloads
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
    yield torch, owqs
    owqs.test_grid_cap(0)


def _check(env, wl, psi, dtype, ref, kinds_expected):
    torch, owqs = env
    p = wl.pattern
    h = owqs.load(p)
    h.reorder()
    t = torch.complex64 if dtype == "c64" else torch.complex128
    dev = None if psi is None else torch.from_numpy(psi).to(t).cuda()
    out, _, probs, _ = h.run(dev, dtype=dtype, outcomes=wl.outcomes)
    got = out.cpu().numpy().astype(np.complex128)
    err = phase_aligned_maxabs(ref.psi_out, got) if dtype == "c64" else float(np.max(np.abs(ref.psi_out - got)))
    assert err <= TOL[dtype], (p.name, dtype, err)
    ref_p = np.array([ref.probs[q] for q in p.measured()])
    assert np.max(np.abs(probs - ref_p)) <= PROB_TOL[dtype], (p.name, dtype)
    kinds = {owqs.KERNEL_KIND[int(k)] for k in h.profile(dev, dtype=dtype, outcomes=wl.outcomes)[2]}
    assert kinds_expected <= kinds, kinds


@pytest.mark.parametrize("blocks", [1, 2, 3])
def test_capped_grid_wraps_the_rings(env, blocks):
    torch, owqs = env
    rng = SplitMix64(401 + blocks)
    cases = [workloads.brickwork(14, 8), workloads.brickwork(13, 10), workloads.qft(12, with_input=False)]
    try:
        owqs.test_grid_cap(blocks)
        for wl in cases:
            p = wl.pattern
            h = owqs.load(p)
            h.reorder()
            op = proa.reorder_commands(p, h.order())
            for psi in (None, random_state(rng, len(p.inputs))):
                if psi is None and p.name.startswith("qft"):
                    continue
                if psi is None:   # the first group paces its ring without copies, on its sequence kernel
                    g0 = h.describe_groups(wl.outcomes, real_input=False)[0]
                    assert g0["m"] == 2 and g0["specialised"], (p.name, g0)
                ref = substate.run(op, psi, outcomes=outcomes_by_label(p, wl.outcomes))
                for dtype in ("c128", "c64"):
                    _check(env, wl, psi, dtype, ref, {"group_pass"})
    finally:
        owqs.test_grid_cap(0)


def test_23_live_qubits_against_the_c_oracle(env):
    """Brickwork 22 x 16 with 11 of its outputs also measured (23 live
    qubits, 2^22-amplitude arrays): at the production grid every warp of the
    complex64 group kernel takes at least three tiles, every block of the
    complex128 one at least three; with the grid capped at three blocks the
    complex64 run's output measurements, bulk-copy single passes (no qubit
    prepared, so no group), also take hundreds of tiles per block through
    their ring."""
    torch, owqs = env
    wl = workloads.brickwork_readout(22, 16, kept=11, with_input=True)
    p = wl.pattern
    h = owqs.load(p)
    h.reorder()
    op = proa.reorder_commands(p, h.order())
    oc = outcomes_by_label(p, wl.outcomes)
    psi = wl.psi_in
    for inp in (None, psi):
        ref = substate_c.run(op, inp, outcomes=oc)
        for dtype in ("c128", "c64"):
            _check(env, wl, inp, dtype, ref, {"group_pass"} | ({"tma_pass"} if dtype == "c64" else set()))
        try:
            owqs.test_grid_cap(3)
            _check(env, wl, inp, "c64", ref, {"group_pass", "tma_pass"})
        finally:
            owqs.test_grid_cap(0)
