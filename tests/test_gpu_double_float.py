"""complex128 pass groups in double-float arithmetic (OWQS_RUN_DOUBLE_FLOAT):
every real number as the sum of two floats, computed on the FP32 pipes.
The results stay within the complex128 bounds of the parity tests (1e-12
max-abs on amplitudes and probabilities, no phase alignment) against the
oracle, and agree with the plain FP64 groups, with groups that read and
write double-float pairs between them and complex128 at the ends."""
import numpy as np
import pytest

from oracle import proa, substate, substate_c
from owqs_inputs import workloads
from owqs_inputs.rng import SplitMix64, random_state

from helpers import outcomes_by_label

pytestmark = pytest.mark.gpu

TOL = 1e-12


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1604_05659_gb300 import build, owqs
    build.ensure_built()
    owqs.library()
    return torch, owqs


def _check(env, wl, psi, ref, mode="owqs"):
    torch, owqs = env
    p = wl.pattern
    h = owqs.load(p)
    h.reorder()
    dev = None if psi is None else torch.from_numpy(psi).cuda()
    out, _, probs, _ = h.run(dev, dtype="c128", mode=mode, outcomes=wl.outcomes, layout="one_array",
                             double_float=True)
    got = out.cpu().numpy()
    err = float(np.max(np.abs(got - ref.psi_out)))
    assert err <= TOL, (p.name, mode, err)
    if mode == "owqs":
        ref_p = np.array([ref.probs[q] for q in p.measured()])
        assert np.max(np.abs(probs - ref_p)) <= TOL, (p.name, float(np.max(np.abs(probs - ref_p))))
    plain, _, pprobs, _ = h.run(dev, dtype="c128", mode=mode, outcomes=wl.outcomes, layout="one_array")
    assert float(np.max(np.abs(plain.cpu().numpy() - got))) <= TOL
    kinds = [owqs.KERNEL_KIND[int(k)] for k in h.profile(dev, dtype="c128", mode=mode, outcomes=wl.outcomes,
                                                         layout="one_array", double_float=True)[2]]
    assert kinds.count("group_pass") >= 2, kinds
    return h


@pytest.mark.parametrize("mode", ["owqs", "eowqs"])
def test_double_float_groups_against_the_oracle(env, mode):
    rng = SplitMix64(601)
    for wl in (workloads.brickwork(14, 8), workloads.brickwork(13, 10), workloads.qft(12, with_input=False)):
        p = wl.pattern
        h = env[1].load(p)
        h.reorder()   # a PROA order, which the oracle accepts in both modes
        op = proa.reorder_commands(p, h.order())
        for psi in (None, random_state(rng, len(p.inputs))):
            if psi is None and p.name.startswith("qft"):
                continue
            ref = substate.run(op, psi, outcomes=outcomes_by_label(p, wl.outcomes), mode=mode)
            _check(env, wl, psi, ref, mode)


def test_double_float_23_live_qubits(env):
    """Brickwork 22 x 16 from |+> and from a random input: 330 measurements in
    double-float groups, against the C oracle."""
    wl = workloads.brickwork(22, 16)
    p = wl.pattern
    h = env[1].load(p)
    h.reorder()
    op = proa.reorder_commands(p, h.order())
    psi = random_state(SplitMix64(602), len(p.inputs))
    for inp in (None, psi):
        ref = substate_c.run(op, inp, outcomes=outcomes_by_label(p, wl.outcomes))
        _check(env, wl, inp, ref)
