"""The final pass (corrections and the gather to output order) when the
output order moves the array's low bits, against the oracle.

Random J/CZ patterns of 12-13 wires end with the outputs in an order whose
low five bits come from higher array bits, so the final pass reads the array
in tiles through shared memory (k_final_tiled).  Random inputs, both
precisions, sign terms and X masks on the outputs, the full grid and a grid
capped at one block (every block then walks all tiles of the array)."""
import numpy as np
import pytest

from oracle import proa, substate
from owqs_inputs import workloads

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


def _cases():
    return [workloads.random_pattern(i, 12, 13, 10, 14, 9, with_input=True) for i in range(4)]


@pytest.mark.parametrize("blocks", [0, 1])
def test_scrambled_output_order(env, blocks):
    torch, owqs = env
    try:
        owqs.test_grid_cap(blocks)
        for wl in _cases():
            p = wl.pattern
            h = owqs.load(p)
            h.reorder()
            fin = h.describe_passes(wl.outcomes)[-1]
            # the output order takes the low five output bits from higher array bits
            assert fin.n_out >= 11 and any(fin.perm[r] >= 5 for r in range(5)), list(fin.perm[:fin.n_out])
            assert fin.xmask != 0 and fin.nedges > 0
            op = proa.reorder_commands(p, h.order())
            ref = substate.run(op, wl.psi_in, outcomes=outcomes_by_label(p, wl.outcomes))
            ref_p = np.array([ref.probs[q] for q in p.measured()])
            for dtype, tdt in (("c128", torch.complex128), ("c64", torch.complex64)):
                psi = torch.from_numpy(wl.psi_in).to(tdt).cuda()
                out, _, probs, st = h.run(psi, dtype=dtype, outcomes=wl.outcomes)
                assert st == owqs.OK
                got = out.cpu().numpy().astype(np.complex128)
                err = (phase_aligned_maxabs(ref.psi_out, got) if dtype == "c64"
                       else float(np.max(np.abs(ref.psi_out - got))))
                assert err <= TOL[dtype], (p.name, dtype, blocks, err)
                assert np.max(np.abs(probs - ref_p)) <= PROB_TOL[dtype], (p.name, dtype, blocks)
                kinds = [owqs.KERNEL_KIND[int(k)] for k in h.profile(psi, dtype=dtype, outcomes=wl.outcomes)[2]]
                assert kinds[-1] == "final", kinds
    finally:
        owqs.test_grid_cap(0)
