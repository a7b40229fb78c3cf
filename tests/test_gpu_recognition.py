"""Recognition (the unitary a pattern implements) and batched determinism
checks on the GPU, through the C ABI, against the FP64 oracle.

owqs_unitary and owqs_run_batch take every measurement with probability 1/2
(EOWQS scaling), so column c of the result equals the oracle run in EOWQS
mode on the basis input e_c with the same forced outcomes: compared exactly
(complex128 1e-12, complex64 2e-5).  For J/CZ circuits the matrix also equals
the product of the gate matrices up to a global phase."""
import math

import numpy as np
import pytest

from oracle import circuit, proa, substate
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


def _circ(i, n, d):
    rng = SplitMix64(7000 + i)
    return circuit_to_pattern(n, random_jcz_circuit(n, d, rng, cz_per_layer=max(1, n // 3)), f"r{n}x{d}#{i}"), rng


def _oracle_columns(p, order, bits, cols):
    op = proa.reorder_commands(p, order)
    outs = outcomes_by_label(p, bits)
    res = []
    for c in cols:
        e = np.zeros(1 << len(p.inputs), dtype=np.complex128)
        e[c] = 1
        res.append(substate.run(op, e, outcomes=outs, mode="eowqs").psi_out)
    return np.stack(res, axis=1)


def _as_matrix(t, nout, nin):
    return t.cpu().numpy().astype(np.complex128).reshape(1 << nin, 1 << nout).T   # column-major


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_unitary_single_against_oracle_and_circuit(env, dtype):
    torch, owqs = env
    for i, (n, d) in enumerate([(1, 3), (2, 4), (3, 5), (4, 4), (5, 3), (6, 3)]):
        p, rng = _circ(i, n, d)
        h = owqs.load(p)
        order, _ = h.reorder()
        bits = rng.bits(p.K)
        U, f2 = h.unitary(dtype=dtype, outcomes=bits)
        got = _as_matrix(U, n, n)
        ref = _oracle_columns(p, order, bits, range(1 << n))
        assert np.max(np.abs(got - ref)) <= TOL[dtype], (n, d)
        Uc = circuit.circuit_unitary(n, p.circuit)
        ov = np.vdot(got.reshape(-1), Uc.reshape(-1))
        assert np.max(np.abs(got * (ov / abs(ov)) - Uc)) <= (1e-12 if dtype == "c128" else 2e-5)
        assert abs(f2 - 1) < (1e-12 if dtype == "c128" else 1e-5)


def test_unitary_qft_is_dft(env):
    torch, owqs = env
    n = 5
    wl = workloads.qft(n)
    h = owqs.load(wl.pattern)
    h.reorder()
    U, _ = h.unitary(dtype="c128", outcomes=wl.outcomes)
    got = _as_matrix(U, n, n)
    N = 1 << n
    F = np.array([[np.exp(2j * math.pi * j * k / N) for k in range(N)] for j in range(N)]) / math.sqrt(N)
    rev = [int(format(j, f"0{n}b")[::-1], 2) for j in range(N)]
    F = F[:, rev]
    ov = np.vdot(got.reshape(-1), F.reshape(-1))
    assert np.max(np.abs(got * (ov / abs(ov)) - F)) <= 1e-12


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_batch_unitaries_mixed_widths(env, dtype):
    """One call: many small patterns in the persistent shared-memory launch,
    a wider one in the persistent launch with global-memory state buffers,
    and a still wider input-vector item through the pass kernels; each
    result against the single call and, for n <= 8, every column against the
    oracle."""
    torch, owqs = env
    tdt = torch.complex64 if dtype == "c64" else torch.complex128
    # widest arrays: 2^12 fits a block's shared memory in both dtypes; 2^13
    # (c128) and 2^14 (c64) do not and run with global-memory buffers
    wide = (13, 1) if dtype == "c128" else (14, 1)
    specs = [(1 + (i % 8), 3 + (i % 5)) for i in range(20)] + [(11, 3), (12, 2), wide]
    items, meta = [], []
    for i, (n, d) in enumerate(specs):
        p, rng = _circ(100 + i, n, d)
        h = owqs.load(p)
        order, _ = h.reorder()
        bits = rng.bits(p.K)
        out = torch.empty(1 << (2 * n), dtype=tdt, device="cuda")
        items.append({"handle": h, "outcomes": bits, "psi_in": None, "out": out, "ref": -1})
        meta.append((p, order, bits, n))
    # an input-vector item whose arrays exceed 2^18 amplitudes: pass kernels
    pw, rngw = _circ(199, 19, 1)
    hw = owqs.load(pw)
    hw.reorder()
    bw = rngw.bits(pw.K)
    psi_w = torch.from_numpy(random_state(rngw, 19)).to(tdt).cuda()
    out_w = torch.empty(1 << 19, dtype=tdt, device="cuda")
    info, _ = owqs.run_batch(items + [{"handle": hw, "outcomes": bw, "psi_in": psi_w, "out": out_w, "ref": -1}],
                             dtype=dtype)
    assert info["smem_items"] == len(specs) - 1 and info["global_items"] == 1 and info["hbm_items"] == 1, info
    single_w, _, _, _ = hw.run(psi_w, dtype=dtype, mode="eowqs", outcomes=bw, check=False)
    assert torch.max(torch.abs(out_w - single_w)).item() <= TOL[dtype]
    for it, (p, order, bits, n) in zip(items, meta):
        single, _ = it["handle"].unitary(dtype=dtype, outcomes=bits)
        assert torch.max(torch.abs(it["out"] - single)).item() <= TOL[dtype], p.name
        del single
        if n <= 8:
            got = _as_matrix(it["out"], n, n)
            cols = range(1 << n) if n <= 5 else range(0, 1 << n, 7)
            ref = _oracle_columns(p, order, bits, list(cols))
            assert np.max(np.abs(got[:, list(cols)] - ref)) <= TOL[dtype], p.name


def test_batch_fixed_column_blocks_agree(env):
    torch, owqs = env
    p, rng = _circ(300, 6, 4)
    h = owqs.load(p)
    h.reorder()
    bits = rng.bits(p.K)
    res = []
    for cb in (0, 1, 4, 64):
        out = torch.empty(1 << 12, dtype=torch.complex128, device="cuda")
        owqs.run_batch([{"handle": h, "outcomes": bits, "psi_in": None, "out": out, "ref": -1}], column_block=cb)
        res.append(out.cpu().numpy())
    for r in res[1:]:
        assert np.max(np.abs(r - res[0])) <= 1e-14


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_batch_determinism_branches(env, dtype):
    """Every outcome branch of a flow pattern gives the same output up to a
    global phase (Section 4.5): |<out_0|out_b>|^2 = |out_0|^2 |out_b|^2."""
    torch, owqs = env
    tdt = torch.complex64 if dtype == "c64" else torch.complex128
    items = []
    for q, (n, d) in enumerate([(4, 6), (7, 5), (10, 3), (13, 2)]):
        p, rng = _circ(400 + q, n, d)
        h = owqs.load(p)
        h.reorder()
        psi = torch.from_numpy(random_state(rng, n)).to(tdt).cuda()
        first = len(items)
        for b in range(16):
            out = torch.empty(1 << n, dtype=tdt, device="cuda")
            items.append({"handle": h, "outcomes": SplitMix64(50 * q + b).bits(p.K), "psi_in": psi, "out": out,
                          "ref": first if b else -1})
    info, ov = owqs.run_batch(items, dtype=dtype, overlaps=True)
    tol = 1e-12 if dtype == "c128" else 1e-5
    for i, it in enumerate(items):
        if it["ref"] < 0:
            continue
        re, im, nx, na = ov[i]
        assert abs((re * re + im * im) / (nx * na) - 1) <= tol, (i, ov[i])
        assert abs(nx - 1) <= tol and abs(na - 1) <= tol


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_batch_unitaries_full_widths_against_circuits(env, dtype):
    """Recognition at the full widths of the batched configuration (11..14
    logical qubits): eight sampled columns of each matrix equal the J/CZ
    circuit applied to those basis vectors (the textbook reduction), up to
    the branch's global phase, common to all columns."""
    torch, owqs = env
    tdt = torch.complex64 if dtype == "c64" else torch.complex128
    items, meta = [], []
    for i, n in enumerate((11, 12, 13, 14)):
        rng = SplitMix64(600 + i)
        gates = random_jcz_circuit(n, 12, rng, cz_per_layer=(n + 3) // 4)
        p = circuit_to_pattern(n, gates, f"full{n}")
        h = owqs.load(p)
        h.reorder()
        out = torch.empty(1 << (2 * n), dtype=tdt, device="cuda")
        items.append({"handle": h, "outcomes": rng.bits(p.K), "psi_in": None, "out": out, "ref": -1})
        meta.append((n, gates, rng))
    owqs.run_batch(items, dtype=dtype)
    tol = 1e-11 if dtype == "c128" else 2e-5
    for it, (n, gates, rng) in zip(items, meta):
        cols = sorted({rng.randint(1 << n) for _ in range(8)})
        ref = np.stack([circuit.apply_circuit(n, gates, np.eye(1, 1 << n, c, dtype=np.complex128)[0]) for c in cols],
                       axis=1)
        # column c of the column-major matrix is the contiguous slice [c 2^n, (c+1) 2^n)
        sub = np.stack([it["out"][c << n:(c + 1) << n].cpu().numpy().astype(np.complex128) for c in cols], axis=1)
        ov = np.vdot(sub.reshape(-1), ref.reshape(-1))
        assert np.max(np.abs(sub * (ov / abs(ov)) - ref)) <= tol, (n, dtype)

