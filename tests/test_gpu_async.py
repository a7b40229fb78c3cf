"""Asynchronous runs (owqs_run_async / owqs_wait).

An asynchronous run launches the same kernels, in the same order, as a
synchronous one-array run with one launch per pass or pass group, so its
output and probabilities are bit-identical to that run's.  Runs complete in
order; with host vectors, consecutive runs overlap their copies with each
other's launches and every run still gets its own input and output.  The
library refuses a third run in flight, a synchronous run while runs are in
flight, a wait with none, and sampled outcomes."""
import numpy as np
import pytest

from owqs_inputs import workloads
from owqs_inputs.rng import SplitMix64, random_state

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1604_05659_gb300 import build, owqs
    build.ensure_built()
    owqs.library()
    return torch, owqs


def _sync(h, torch, psi, bits, dtype):
    t = torch.complex64 if dtype == "c64" else torch.complex128
    x = None if psi is None else torch.from_numpy(psi).to(t).cuda()
    out, _, probs, st = h.run(x, dtype=dtype, outcomes=bits, layout="one_array", per_pass=True)
    assert st == 0
    return out.cpu().numpy(), probs


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_device_vectors_match_the_synchronous_run(env, dtype):
    torch, owqs = env
    rng = SplitMix64(900)
    for wl in (workloads.brickwork(12, 10), workloads.qft(12), workloads.small_random()):
        p = wl.pattern
        h = owqs.load(p)
        h.reorder()
        t = torch.complex64 if dtype == "c64" else torch.complex128
        cases = []
        for _ in range(2):
            psi = random_state(rng, len(p.inputs))
            bits = rng.bits(p.K)
            cases.append((psi, bits, *_sync(h, torch, psi, bits, dtype)))
        outs = []
        for psi, bits, _, _ in cases:   # two runs in flight
            o = torch.empty(1 << len(p.outputs), dtype=t, device="cuda")
            h.run_async(torch.from_numpy(psi).to(t).cuda(), o, dtype=dtype, outcomes=bits)
            outs.append(o)
        for (psi, bits, ref, ref_p), o in zip(cases, outs):
            _, probs, st = h.wait()
            assert st == owqs.OK
            assert np.array_equal(o.cpu().numpy(), ref), (p.name, dtype)
            assert np.array_equal(probs, ref_p), (p.name, dtype)
        h.close()


def test_pipelined_host_vectors(env):
    """Six runs with pinned host vectors, two in flight at a time, each with
    its own input and output buffer: every output equals the synchronous
    run of its input."""
    torch, owqs = env
    wl = workloads.brickwork(16, 8)
    p = wl.pattern
    h = owqs.load(p)
    h.reorder()
    rng = SplitMix64(901)
    ins = [torch.from_numpy(random_state(rng, 16).astype(np.complex64)).pin_memory() for _ in range(6)]
    outs = [torch.empty(1 << 16, dtype=torch.complex64).pin_memory() for _ in range(6)]
    refs = [_sync(h, torch, x.numpy().astype(np.complex128), wl.outcomes, "c64") for x in ins]
    done = []
    for i in range(6):
        h.run_async(ins[i], outs[i], dtype="c64", outcomes=wl.outcomes)
        if i >= 1:
            done.append(h.wait())
    done.append(h.wait())
    for i in range(6):
        assert done[i][2] == owqs.OK
        assert np.array_equal(outs[i].numpy(), refs[i][0]), i
        assert np.array_equal(done[i][1], refs[i][1]), i
    h.close()


def test_refusals(env):
    torch, owqs = env
    wl = workloads.brickwork(10, 6)
    h = owqs.load(wl.pattern)
    h.reorder()
    o = [torch.empty(1 << 10, dtype=torch.complex64, device="cuda") for _ in range(3)]
    with pytest.raises(owqs.OwqsError):
        h.wait()                                            # none in flight
    h.run_async(None, o[0], outcomes=wl.outcomes)
    h.run_async(None, o[1], outcomes=wl.outcomes)
    with pytest.raises(owqs.OwqsError):
        h.run_async(None, o[2], outcomes=wl.outcomes)       # a third
    with pytest.raises(owqs.OwqsError):
        h.run(None, dtype="c64", outcomes=wl.outcomes, out=o[2])   # synchronous while in flight
    h.wait()
    h.wait()
    with pytest.raises(owqs.OwqsError):
        h.run_async(None, o[0], policy="sampled")
    out, _, _, st = h.run(None, dtype="c64", outcomes=wl.outcomes, out=o[2])
    assert st == owqs.OK and torch.equal(o[0], o[1])
    h.close()


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_eowqs_and_zero_policy(env, dtype):
    """EOWQS (every probability reported as 1/2, the output norm checked) and
    the zero policy (all outcomes 0, reported by owqs_wait) give the
    synchronous one-array run's results."""
    torch, owqs = env
    t = torch.complex64 if dtype == "c64" else torch.complex128
    wl = workloads.qft(10)
    p = wl.pattern
    h = owqs.load(p)
    h.reorder()
    psi = torch.from_numpy(wl.psi_in).to(t).cuda()
    for mode, policy in (("eowqs", "forced"), ("owqs", "zero"), ("eowqs", "zero")):
        bits = wl.outcomes if policy == "forced" else None
        ref, ref_oc, ref_p, st = h.run(psi, dtype=dtype, mode=mode, policy=policy, outcomes=bits,
                                       layout="one_array", per_pass=True)
        assert st == owqs.OK
        o = torch.empty(1 << len(p.outputs), dtype=t, device="cuda")
        h.run_async(psi, o, dtype=dtype, mode=mode, policy=policy, outcomes=bits)
        oc, probs, st = h.wait()
        assert st == owqs.OK, (mode, policy)
        assert torch.equal(o, ref), (mode, policy)
        assert np.array_equal(probs, ref_p), (mode, policy)
        if policy == "zero":
            assert not np.any(oc) and np.array_equal(oc, ref_oc)
        if mode == "eowqs":
            assert np.all(probs == 0.5)
    h.close()
