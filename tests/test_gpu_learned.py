"""The learned reorder proposal on the GPU: the library's forward and
backward kernels against the FP64 reference network (oracle/mlp.py), GPU
training, and what the trained proposal gains over the greedy reordering it
is checked against."""
import json
import os

import numpy as np
import pytest

from oracle import mlp, proa, substate
from owqs_inputs import workloads
from owqs_inputs.rng import SplitMix64

from helpers import outcomes_by_label

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1604_05659_gb300 import build, owqs
    build.ensure_built()
    owqs.library()
    return torch, owqs


def _synthetic(seed, steps=300, width=12):
    """Seeded parameters and feature rows (not produced by the library)."""
    rng = SplitMix64(seed)
    params = ((rng.uniform_block(mlp.NPARAM) * 2 - 1) * 0.25).astype(np.float32)
    first, target = [0], []
    for _ in range(steps):
        n = 1 + rng.randint(width)
        target.append(first[-1] + rng.randint(n))
        first.append(first[-1] + n)
    X = (rng.uniform_block(first[-1] * mlp.NF).reshape(-1, mlp.NF) * 3 - 1).astype(np.float32)
    return params, X, np.array(first, dtype=np.int32), np.array(target, dtype=np.int32)


def _dev(torch, *arrs):
    return [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in arrs]


def test_scores_and_gradient_match_reference(env):
    """Forward scores and the loss gradient of the GPU kernels against the
    FP64 reference with the same bfloat16 rounding points.  Rounding an
    activation to bfloat16 is decided from an FP32 (GPU) or FP64 (reference)
    pre-activation, so a value lying on a rounding boundary may round the
    other way; the tolerances allow for that, not for a wrong term."""
    torch, owqs = env
    params, X, first, target = _synthetic(11)
    m = owqs.Model(weights=params)
    Xd, Fd, Td = _dev(torch, X, first, target)
    s_gpu = m.score(Xd).cpu().numpy().astype(np.float64)
    s_ref, _ = mlp.forward(params.astype(np.float64), X, bf=True)
    err = np.abs(s_gpu - s_ref)
    assert np.median(err) < 1e-5 and np.mean(err > 1e-3) < 0.01, (np.median(err), err.max())
    g_gpu, l_gpu = m.gradient(Xd, Fd, Td)
    l_ref, g_ref = mlp.loss_and_grad(params.astype(np.float64), X, first, target, bf=True)
    assert abs(l_gpu - l_ref) <= 1e-4 * max(1.0, abs(l_ref))
    scale = np.max(np.abs(g_ref))
    assert np.max(np.abs(g_gpu - g_ref)) <= 5e-3 * scale, np.max(np.abs(g_gpu - g_ref)) / scale
    # every parameter group gets its gradient (a dropped term would leave zeros)
    for a, b in ((mlp.P_W1, mlp.P_B1), (mlp.P_B1, mlp.P_W2), (mlp.P_W2, mlp.P_B2), (mlp.P_B2, mlp.P_W3),
                 (mlp.P_W3, mlp.P_B3)):
        ref_norm = np.linalg.norm(g_ref[a:b])
        assert np.linalg.norm(g_gpu[a:b] - g_ref[a:b]) <= 1e-2 * ref_norm + 1e-7


def _small_set(count, start):
    return workloads.random_batch(count, 8, 12, 8, 16, config_index=4, start=start)


def _dataset(owqs, wls, cands=8):
    from paper_1604_05659_gb300.train_reorder import build_dataset
    hs = [owqs.load(w.pattern) for w in wls]
    return build_dataset(hs, cands, seed=3)


def _best_greedy(h):
    """(peak live width, amplitude updates) of the better greedy order: the
    greedy EOWQS order (every qubit ready) and the greedy OWQS sweep order
    (which waits for every domain, so it is valid with preselected outcomes
    too)."""
    k = float(max(1, h.nout))
    _, e = h.reorder(mode="eowqs", sweep=False, weights=(k, k, 0.5, k))
    _, o = h.reorder(mode="owqs", sweep=True)
    return min((e["peak_live"], e["amp_updates"]), (o["peak_live"], o["amp_updates"]))


def _with_proposal(h, m):
    k = float(max(1, h.nout))
    return h.reorder(mode="eowqs", sweep=False, weights=(k, k, 0.5, k), model=m)


def test_training_reduces_loss_and_proposal_is_never_worse(env):
    """Train on small random J/CZ patterns with the library's kernels, then
    reorder held-out patterns in EOWQS mode with the proposal: the kept order
    is never worse, by (peak live width, amplitude updates), than the best
    greedy order, against which the library keeps or drops it; the gain over it is
    reported, not required."""
    torch, owqs = env
    X, first, target = _dataset(owqs, _small_set(40, 0))
    Xd, Fd, Td = _dev(torch, X, first.astype(np.int32), target.astype(np.int32))
    m = owqs.Model(seed=5)
    _, l0 = m.gradient(Xd, Fd, Td)
    losses = m.train(Xd, Fd, Td, epochs=25, batch_steps=512, lr=3e-3, seed=1)
    _, l1 = m.gradient(Xd, Fd, Td)
    assert l1 < 0.5 * l0, (l0, l1, losses)
    gains = []
    for wl in _small_set(10, 10_000):
        h = owqs.load(wl.pattern)
        best = _best_greedy(h)
        order, info = _with_proposal(h, m)
        assert (info["greedy_peak_live"], info["greedy_amp_updates"]) == best, (info, best)
        kept = (info["peak_live"], info["amp_updates"])
        assert kept <= best, (kept, best)
        if info["learned_accepted"]:
            assert kept == (info["learned_peak_live"], info["learned_amp_updates"])
        gains.append(best[1] / max(1, kept[1]))
    print("amplitude-update gain of the kept order over the best greedy order:", gains)


def test_learned_order_simulates_to_the_oracle_state(env):
    """A learned EOWQS order measures qubits out of circuit order; with the
    outcomes fixed the output is the same state (measurements on different
    qubits commute, Eq. 14), exactly, as the oracle computes it in circuit
    order."""
    torch, owqs = env
    X, first, target = _dataset(owqs, _small_set(30, 0))
    Xd, Fd, Td = _dev(torch, X, first.astype(np.int32), target.astype(np.int32))
    m = owqs.Model(seed=9)
    m.train(Xd, Fd, Td, epochs=20, batch_steps=512, lr=3e-3, seed=2)
    wl = _small_set(1, 20_000)[0]
    p = wl.pattern
    h = owqs.load(p)
    order, info = h.reorder(mode="eowqs", model=m)
    psi = torch.from_numpy(wl.psi_in).cuda()
    out, _, _, _ = h.run(psi, dtype="c128", mode="eowqs", outcomes=wl.outcomes)
    ref = substate.run(proa.reorder_commands(p, p.measured()), wl.psi_in, outcomes=outcomes_by_label(p, wl.outcomes),
                       mode="eowqs")
    assert np.max(np.abs(out.cpu().numpy() - ref.psi_out)) <= 1e-12


def test_committed_weights_on_heldout_patterns(env):
    """The committed network (trained by train_reorder.py on 16..30-qubit
    patterns) on held-out patterns of that range: the kept order is never
    worse than the best greedy order; the gain is reported."""
    torch, owqs = env
    path = os.path.join(ROOT, "paper_1604_05659_gb300", "reorder_mlp.json")
    if not os.path.exists(path):
        pytest.skip("no trained weights committed")
    w = np.array(json.load(open(path))["params"], dtype=np.float32)
    m = owqs.Model(weights=w)
    held = workloads.random_batch(6, 16, 30, 20, 60, config_index=4, start=1_000_000, with_input=False)
    for wl in held:
        h = owqs.load(wl.pattern)
        best = _best_greedy(h)
        _, info = _with_proposal(h, m)
        kept = (info["peak_live"], info["amp_updates"])
        assert kept <= best, (kept, best)
        print(wl.pattern.name, "best greedy", best, "kept", kept, "learned", info["learned_peak_live"],
              "accepted", info["learned_accepted"])
