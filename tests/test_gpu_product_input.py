"""Product inputs (Section 4.1, Fig. 8a): the input as separate factors,
each joining the live array when the pattern first reaches it, against the
oracle's sub-state simulation with the same factors and against the same run
with the dense product vector."""
import numpy as np
import pytest

from oracle import proa, substate
from owqs_inputs import workloads
from owqs_inputs.patterns import circuit_to_pattern, random_jcz_circuit
from owqs_inputs.rng import SplitMix64, random_state

from helpers import outcomes_by_label, phase_aligned_maxabs

pytestmark = pytest.mark.gpu
TOL = {"c128": 1e-12, "c64": 2e-5}


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1604_05659_gb300 import build, owqs
    build.ensure_built()
    owqs.library()
    return torch, owqs


def _factors(rng, inputs):
    """Split the inputs into factors of 1-3 qubits with random states."""
    qs = list(inputs)
    out = []
    while qs:
        k = min(len(qs), 1 + rng.randint(3))
        f, qs = qs[:k], qs[k:]
        out.append((f, random_state(rng, k)))
    return out


def _dense(factors, inputs):
    """The product vector over the inputs (bit k = inputs[k])."""
    n = len(inputs)
    pos = {q: k for k, q in enumerate(inputs)}
    idx = np.arange(1 << n)
    v = np.ones(1 << n, dtype=np.complex128)
    for qs, vec in factors:
        sub = np.zeros(1 << n, dtype=np.int64)
        for k, q in enumerate(qs):
            sub |= ((idx >> pos[q]) & 1) << k
        v *= np.asarray(vec)[sub]
    return v


def _cases():
    cases = [workloads.small_random().pattern, workloads.brickwork(5, 8).pattern]
    for i in range(4):
        rng = SplitMix64(700 + i)
        n = 3 + rng.randint(6)
        cases.append(circuit_to_pattern(n, random_jcz_circuit(n, 4, rng, cz_per_layer=2), f"rand{n}"))
    return cases


@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("mode", ["owqs", "eowqs"])
def test_product_input_matches_oracle_factors(env, dtype, mode):
    torch, owqs = env
    rng = SplitMix64(707)
    tdt = torch.complex64 if dtype == "c64" else torch.complex128
    for p in _cases():
        fac = _factors(rng, p.inputs)
        bits = rng.bits(p.K)
        h = owqs.load(p)
        h.reorder()
        op = proa.reorder_commands(p, h.order())
        ref = substate.run(op, None, outcomes=outcomes_by_label(p, bits), mode=mode, input_factors=fac)
        dev = [(qs, torch.from_numpy(np.asarray(v)).to(tdt).cuda()) for qs, v in fac]
        out, _, probs, _ = h.run_product(dev, dtype=dtype, mode=mode, outcomes=bits)
        got = out.cpu().numpy().astype(np.complex128)
        err = phase_aligned_maxabs(ref.psi_out, got) if dtype == "c64" else float(np.max(np.abs(ref.psi_out - got)))
        assert err <= TOL[dtype], (p.name, err)
        if mode == "owqs":
            ref_p = np.array([ref.probs[q] for q in p.measured()])
            assert np.max(np.abs(probs - ref_p)) <= (1e-12 if dtype == "c128" else 1e-6)
        # the same as the dense product vector through owqs_run
        dense = torch.from_numpy(_dense(fac, p.inputs)).to(tdt).cuda()
        out2, _, _, _ = h.run(dense, dtype=dtype, mode=mode, outcomes=bits)
        err2 = float(torch.max(torch.abs(out2 - out)).item())
        assert err2 <= TOL[dtype], (p.name, err2)


def test_factor_joins_happen_late_and_bad_factors_are_rejected(env):
    torch, owqs = env
    wl = workloads.brickwork(6, 6)
    h = owqs.load(wl.pattern)
    h.reorder()
    fac = [([q], torch.tensor([0.6, 0.8j], dtype=torch.complex128).cuda()) for q in wl.pattern.inputs]
    out, _, _, st = h.run_product(fac, dtype="c128", outcomes=wl.outcomes)
    assert st == owqs.OK
    with pytest.raises(owqs.OwqsError):
        h.run_product(fac[:-1], dtype="c128", outcomes=wl.outcomes)      # an input left out
    with pytest.raises(owqs.OwqsError):
        h.run_product(fac + fac[:1], dtype="c128", outcomes=wl.outcomes)  # an input twice
