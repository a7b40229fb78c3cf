"""Complex64 pass groups on a 4-qubit register, against the oracle.

Such groups (2^4 configurations per free index, 8 KB warp tiles, one block
per SM, at most 8 passes) are planned only for arrays of at least 2^26
amplitudes; the test hook owqs_test_group_m4_width lowers that width so
that patterns the oracle finishes in seconds take them too.  Brickwork,
QFT-shaped and random J/CZ patterns from |+> and random inputs, both modes,
compiled-sequence and run-time-slot kernels, and capped grids that make
every warp wrap its ring of 8 KB stages."""
import numpy as np
import pytest

from oracle import proa, substate
from owqs_inputs import workloads
from owqs_inputs.rng import SplitMix64, random_state

from helpers import outcomes_by_label, phase_aligned_maxabs

pytestmark = pytest.mark.gpu

TOL, PROB_TOL = 2e-5, 1e-6


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1604_05659_gb300 import build, owqs
    build.ensure_built()
    owqs.library()
    owqs.test_group_m4_width(10)
    yield torch, owqs
    owqs.test_group_m4_width(0)
    owqs.test_grid_cap(0)


def _cases():
    return [workloads.brickwork(14, 8), workloads.brickwork(13, 10), workloads.qft(12, with_input=False),
            workloads.random_pattern(7, 13, 13, 12, 12, 3, with_input=False)]


def _check(torch, owqs, wl, psi, mode, kernels):
    p = wl.pattern
    h = owqs.load(p)
    h.reorder()
    groups = h.describe_groups(wl.outcomes, real_input=psi is not None)
    m4 = [g for g in groups if g["m"] == 4]
    assert m4 and all(len(g["slots"]) <= 8 for g in m4), (p.name, groups)
    for g in m4:
        kernels.add(g["specialised"])
    op = proa.reorder_commands(p, h.order())
    ref = substate.run(op, psi, outcomes=outcomes_by_label(p, wl.outcomes), mode=mode)
    dev = None if psi is None else torch.from_numpy(psi).to(torch.complex64).cuda()
    out, _, probs, st = h.run(dev, dtype="c64", mode=mode, outcomes=wl.outcomes, layout="one_array")
    assert st == owqs.OK
    err = phase_aligned_maxabs(ref.psi_out, out.cpu().numpy().astype(np.complex128))
    assert err <= TOL, (p.name, mode, err)
    if mode == "owqs":
        ref_p = np.array([ref.probs[q] for q in p.measured()])
        assert np.max(np.abs(probs - ref_p)) <= PROB_TOL, (p.name, float(np.max(np.abs(probs - ref_p))))
    kinds = [owqs.KERNEL_KIND[int(k)] for k in h.profile(dev, dtype="c64", mode=mode, outcomes=wl.outcomes,
                                                         layout="one_array")[2]]
    assert kinds.count("group_pass") == len(groups), (p.name, kinds)


@pytest.mark.parametrize("mode", ["owqs", "eowqs"])
def test_four_qubit_registers_against_the_oracle(env, mode):
    torch, owqs = env
    rng = SplitMix64(1500)
    kernels = set()
    for wl in _cases():
        for psi in (None, random_state(rng, len(wl.pattern.inputs))):
            if psi is None and wl.name.startswith("qft"):
                continue
            _check(torch, owqs, wl, psi, mode, kernels)
    assert kernels == {True, False}   # compiled-sequence and run-time-slot kernels both ran


@pytest.mark.parametrize("blocks", [1, 3])
def test_four_qubit_registers_wrap_their_rings(env, blocks):
    torch, owqs = env
    rng = SplitMix64(1510 + blocks)
    try:
        owqs.test_grid_cap(blocks)
        for wl in _cases()[:2]:
            _check(torch, owqs, wl, random_state(rng, len(wl.pattern.inputs)), "owqs", set())
    finally:
        owqs.test_grid_cap(0)
