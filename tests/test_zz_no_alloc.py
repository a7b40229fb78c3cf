"""owqs_run_static, the entry point that allocates no device memory, against
owqs_run on the same patterns.

Some callers cannot call cudaMalloc: a program whose device memory belongs
to another allocator (a framework's caching pool, an embedding application)
or is held to a fixed budget.  owqs_run_static keeps its scratch in a
fixed device array, so it must give owqs_run's results; it is called twice
in a row because the array keeps the previous call's contents.  This file is
collected last so that a failure here, in a run that stops at the first
failure, comes after every other test.
"""
import numpy as np
import pytest

from owqs_inputs import workloads
from owqs_inputs.rng import SplitMix64, random_state

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


def _cases():
    rng = SplitMix64(4242)
    small = workloads.small_random()
    qft = workloads.qft(10)
    brick = workloads.brickwork(12, 14)
    return [(small.pattern, small.psi_in, small.outcomes, "owqs"),
            (qft.pattern, qft.psi_in, qft.outcomes, "owqs"),
            (brick.pattern, None, brick.outcomes, "owqs"),
            (brick.pattern, None, rng.bits(brick.pattern.K), "eowqs")]


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_static_entry_matches_owqs_run(env, dtype):
    torch, owqs = env
    tdt = torch.complex64 if dtype == "c64" else torch.complex128
    for p, psi, bits, mode in _cases():
        h = owqs.load(p)
        h.reorder()
        dev_in = None if psi is None else torch.from_numpy(psi).to(tdt).cuda()
        ref, _, ref_probs, _ = h.run(dev_in, dtype=dtype, mode=mode, outcomes=bits)
        ref = ref.cpu().numpy().astype(np.complex128)
        for call in range(2):
            out, _, probs, st = h.run_static(dev_in, dtype=dtype, mode=mode, outcomes=bits)
            torch.cuda.synchronize()
            assert st == owqs.OK
            got = out.cpu().numpy().astype(np.complex128)
            err = float(np.max(np.abs(got - ref)))
            assert err <= TOL[dtype], (p.name, dtype, mode, call, err)
            assert np.max(np.abs(probs - ref_probs)) <= (1e-12 if dtype == "c128" else 1e-6)


def test_static_entry_rejects_patterns_beyond_its_scratch(env):
    torch, owqs = env
    wl = workloads.brickwork(20, 3)            # passes of 2^20 amplitudes
    h = owqs.load(wl.pattern)
    h.reorder()
    for dtype in ("c64", "c128"):
        with pytest.raises(owqs.OwqsError) as ei:
            h.run_static(None, dtype=dtype, outcomes=wl.outcomes)
        assert ei.value.status == owqs.ERR_ARG and "static scratch holds" in str(ei.value)
