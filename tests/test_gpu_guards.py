"""Guard canaries on the caller's buffers: every entry point writes exactly
its output range and never touches its input.  Each output is a view into a
larger allocation whose head and tail hold a sentinel value; each input is
checked unchanged after the call.  The results equal those of the same call
on plain allocations bit for bit (the same launches run).  This stands in
for a memory checker, which is not available for these runs."""
import numpy as np
import pytest

from owqs_inputs import workloads
from owqs_inputs.patterns import circuit_to_pattern, random_jcz_circuit
from owqs_inputs.rng import SplitMix64, random_state

pytestmark = pytest.mark.gpu
GUARD = 4096  # elements on each side of a guarded view
SENT = complex(-7.25, 3.5)


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1604_05659_gb300 import build, owqs
    build.ensure_built()
    owqs.library()
    return torch, owqs


def _tdt(torch, dtype):
    return torch.complex64 if dtype == "c64" else torch.complex128


def _guarded(torch, n, tdt):
    buf = torch.full((n + 2 * GUARD,), SENT, dtype=tdt, device="cuda")
    return buf, buf[GUARD:GUARD + n]


def _guards_intact(torch, buf, n):
    torch.cuda.synchronize()
    return bool(torch.all(buf[:GUARD] == SENT)) and bool(torch.all(buf[GUARD + n:] == SENT))


def _input(torch, rng, n, tdt):
    return torch.from_numpy(random_state(rng, n)).to(tdt).cuda()


def _patterns():
    """Patterns whose runs take every launch kind: pass groups and single
    bulk-copy passes on a 14-qubit random input, register-tiled and generic
    passes, the final gather."""
    out = [("small", workloads.small_random().pattern, 3),
           ("brickwork14x8", workloads.brickwork(14, 8).pattern, 14)]
    rng = SplitMix64(811)
    out.append(("rand14", circuit_to_pattern(14, random_jcz_circuit(14, 6, rng, cz_per_layer=4), "rand14"), 14))
    return out


@pytest.mark.parametrize("dtype", ["c64", "c128"])
@pytest.mark.parametrize("name,pattern,nin", _patterns(), ids=lambda v: v if isinstance(v, str) else None)
def test_run_writes_only_its_output(env, dtype, name, pattern, nin):
    torch, owqs = env
    tdt = _tdt(torch, dtype)
    h = owqs.load(pattern)
    h.reorder()
    rng = SplitMix64(900 + nin)
    oc = workloads.forced_outcomes(pattern, rng)
    psi = _input(torch, rng, nin, tdt)
    psi_copy = psi.clone()
    nout = 1 << len(pattern.outputs)
    ref, _, ref_p, _ = h.run(psi, dtype=dtype, outcomes=oc)
    buf, view = _guarded(torch, nout, tdt)
    got, _, p, _ = h.run(psi, dtype=dtype, outcomes=oc, out=view)
    assert _guards_intact(torch, buf, nout), name
    assert torch.equal(got, ref) and np.array_equal(p, ref_p)
    assert torch.equal(psi, psi_copy)
    # |+> input (generated in the kernel), and device-sampled outcomes
    buf2, view2 = _guarded(torch, nout, tdt)
    h.run(None, dtype=dtype, outcomes=oc, out=view2)
    assert _guards_intact(torch, buf2, nout)
    for seq in (False, True):  # checked guess, one measurement at a time
        buf3, view3 = _guarded(torch, nout, tdt)
        h.run(psi, dtype=dtype, policy="sampled", seed=5, out=view3, sequential_sampling=seq)
        assert _guards_intact(torch, buf3, nout)
    assert torch.equal(psi, psi_copy)


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_product_static_and_unitary_write_only_their_outputs(env, dtype):
    torch, owqs = env
    tdt = _tdt(torch, dtype)
    rng = SplitMix64(923)
    n = 6
    p = circuit_to_pattern(n, random_jcz_circuit(n, 5, rng, cz_per_layer=2), "rand6")
    h = owqs.load(p)
    h.reorder()
    oc = workloads.forced_outcomes(p, rng)
    nout = 1 << len(p.outputs)
    # product input: three factors of two qubits
    factors = [(p.inputs[2 * f:2 * f + 2], _input(torch, rng, 2, tdt)) for f in range(3)]
    copies = [v.clone() for _, v in factors]
    ref, _, _, _ = h.run_product(factors, dtype=dtype, outcomes=oc)
    buf, view = _guarded(torch, nout, tdt)
    got, _, _, _ = h.run_product(factors, dtype=dtype, outcomes=oc, out=view)
    assert _guards_intact(torch, buf, nout) and torch.equal(got, ref)
    assert all(torch.equal(v, c) for (_, v), c in zip(factors, copies))
    # allocation-free entry point
    psi = _input(torch, rng, n, tdt)
    ref, _, _, _ = h.run_static(psi, dtype=dtype, outcomes=oc)
    buf, view = _guarded(torch, nout, tdt)
    got, _, _, _ = h.run_static(psi, dtype=dtype, outcomes=oc, out=view)
    assert _guards_intact(torch, buf, nout) and torch.equal(got, ref)
    # all basis columns
    nu = 1 << (len(p.outputs) + len(p.inputs))
    ref, _ = h.unitary(dtype=dtype, outcomes=oc)
    buf, view = _guarded(torch, nu, tdt)
    got, _ = h.unitary(dtype=dtype, outcomes=oc, out=view)
    assert _guards_intact(torch, buf, nu) and torch.equal(got, ref)


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_batch_writes_only_its_outputs(env, dtype):
    """Shared-memory items and a wide item that takes the array path, each
    output between guards, and the branch inputs unchanged."""
    torch, owqs = env
    tdt = _tdt(torch, dtype)
    items, bufs, plain = [], [], []
    for i, n in enumerate((5, 7, 13)):
        rng = SplitMix64(940 + i)
        p = circuit_to_pattern(n, random_jcz_circuit(n, 8, rng, cz_per_layer=(n + 3) // 4), f"b{n}")
        h = owqs.load(p)
        h.reorder()
        size = 1 << (2 * n)
        buf, view = _guarded(torch, size, tdt)
        items.append({"handle": h, "outcomes": rng.bits(p.K), "psi_in": None, "out": view, "ref": -1})
        plain.append(dict(items[-1], out=torch.empty(size, dtype=tdt, device="cuda")))
        bufs.append((buf, size))
    psi = _input(torch, SplitMix64(950), 7, tdt)
    psi_copy = psi.clone()
    h7 = items[1]["handle"]
    for b in range(2):
        rng = SplitMix64(960 + b)
        buf, view = _guarded(torch, 1 << 7, tdt)
        items.append({"handle": h7, "outcomes": rng.bits(h7.K), "psi_in": psi, "out": view, "ref": -1})
        plain.append(dict(items[-1], out=torch.empty(1 << 7, dtype=tdt, device="cuda")))
        bufs.append((buf, 1 << 7))
    owqs.run_batch(plain, dtype=dtype)
    owqs.run_batch(items, dtype=dtype)
    for (buf, size), it, ref in zip(bufs, items, plain):
        assert _guards_intact(torch, buf, size)
        assert torch.equal(it["out"], ref["out"])
    assert torch.equal(psi, psi_copy)
