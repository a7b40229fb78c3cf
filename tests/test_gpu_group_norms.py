"""Pass groups of both kinds against the oracle (Eq. 13).

Groups whose passes each measure a qubit joined by E to the qubit the pass
prepares have every probability exactly 1/2 (the projection leaves
|+>phi0 +- e^{-i a}|->phi1, half of phi's squared norm) and sum only the
last pass's norm; every other group sums each pass's squared norm.  The
chain patterns give both kinds on the same measurements: the prepared
qubits get E to the measured one once (exact 1/2) or twice (the identity,
so the prepared qubit stays unentangled and the probabilities differ from
1/2).  Random inputs, complex64 and complex128, forced outcomes."""
import numpy as np
import pytest

from oracle import substate
from owqs_inputs import workloads
from owqs_inputs.rng import SplitMix64

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


@pytest.mark.parametrize("joined", [0, 1, 2])
@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_chain_groups_against_the_oracle(env, joined, dtype):
    torch, owqs = env
    rng = SplitMix64(700 + joined)
    for n, k in ((14, 9), (17, 12)):
        wl = workloads.chain_measurements(n, k, joined_every=joined, pattern_index=n)
        p = wl.pattern
        h = owqs.load(p)
        groups = h.describe_groups(wl.outcomes, dtype=dtype, real_input=True)
        assert groups and all(g["half"] == (joined == 1) for g in groups), groups
        t = torch.complex64 if dtype == "c64" else torch.complex128
        psi = torch.from_numpy(wl.psi_in).to(t).cuda()
        for bits in (wl.outcomes, rng.bits(p.K)):
            out, _, probs, st = h.run(psi, dtype=dtype, outcomes=bits, layout="one_array")
            assert st == owqs.OK
            kinds = [owqs.KERNEL_KIND[int(x)] for x in h.profile(psi, dtype=dtype, outcomes=bits,
                                                                  layout="one_array")[2]]
            assert kinds.count("group_pass") == len(groups), kinds
            ref = substate.run(p, wl.psi_in, outcomes=outcomes_by_label(p, bits))
            ref_p = np.array([ref.probs[q] for q in p.measured()])
            assert np.max(np.abs(probs - ref_p)) <= PROB_TOL[dtype], (p.name, dtype)
            if joined == 0:
                assert np.max(np.abs(ref_p - 0.5)) > 1e-3   # the group really computes them
            got = out.cpu().numpy().astype(np.complex128)
            err = phase_aligned_maxabs(ref.psi_out, got) if dtype == "c64" else float(
                np.max(np.abs(ref.psi_out - got)))
            assert err <= TOL[dtype], (p.name, dtype, err)
