"""Sampled OWQS on patterns without a gflow: checked launches.

The forced run of the current outcome vector (initially the guesses
u_k > 1/2) runs one launch at a time; after each launch that measures, the
host checks its draws u_k <= prob_0 against the probabilities it computed,
and at the first draw that decides the other outcome corrects it and runs
that launch again.  The outcomes must be the one-at-a-time draw's (the
oracle's splitmix64 stream, Fig. 6), the output and probabilities within the
parity bounds, and the run must report that it took checked launches."""
import numpy as np
import pytest

from oracle import proa, substate
from owqs_inputs import workloads
from owqs_inputs.rng import SplitMix64, random_state

from helpers import phase_aligned_maxabs

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


def _dev(torch, psi, dtype):
    if psi is None:
        return None
    t = torch.complex64 if dtype == "c64" else torch.complex128
    return torch.from_numpy(np.asarray(psi, dtype=np.complex128)).to(t).cuda()


def _check_against_oracle(env, wl, seeds, dtypes=("c128", "c64")):
    """Every seed: GPU outcomes == oracle outcomes, output and
    probabilities within the bounds; returns the relaunch count summed over
    the runs."""
    torch, owqs = env
    p = wl.pattern
    h = owqs.load(p)
    if p.is_standard():
        h.reorder()
    op = proa.reorder_commands(p, h.order()) if p.is_standard() else p
    relaunches = 0
    for seed in seeds:
        ref = substate.run(op, wl.psi_in, policy="sampled", seed=seed)
        ref_oc = [ref.outcomes[q] for q in p.measured()]
        ref_p = np.array([ref.probs[q] for q in p.measured()])
        for dtype in dtypes:
            out, oc, probs, st = h.run(_dev(torch, wl.psi_in, dtype), dtype=dtype, policy="sampled", seed=seed)
            assert st == owqs.OK
            info = h.last_sample_info()
            assert info["path"] == "checked_launches" and not info["guessed"], info
            assert info["checks"] >= 1
            relaunches += info["relaunches"]
            got_oc = [int(oc[k]) for k in range(p.K)]
            if dtype == "c64" and got_oc != ref_oc:
                # a draw within complex64 rounding of prob_0 may go the other way
                k = next(i for i in range(p.K) if got_oc[i] != ref_oc[i])
                u = _uniforms(p, h, seed)[k]
                assert abs(u - (ref_p[k] if ref_oc[k] == 0 else 1 - ref_p[k])) <= 1e-6, (p.name, seed, k)
                continue
            assert got_oc == ref_oc, (p.name, dtype, seed)
            # every measurement whose drawn outcome differs from its guess u > 1/2 is corrected once
            u = _uniforms(p, h, seed)
            assert info["relaunches"] == sum(ref_oc[k] != (0 if u[k] <= 0.5 else 1) for k in range(p.K)), info
            assert np.max(np.abs(probs - ref_p)) <= PROB_TOL[dtype], (p.name, dtype, seed)
            got = out.cpu().numpy().astype(np.complex128)
            err = phase_aligned_maxabs(ref.psi_out, got) if dtype == "c64" else float(
                np.max(np.abs(ref.psi_out - got)))
            assert err <= TOL[dtype], (p.name, dtype, seed, err)
    return relaunches


def _uniforms(p, h, seed):
    """u_k per measurement (K-index), drawn in execution order."""
    rng = SplitMix64(seed)
    order = h.order()
    label = {q: k for k, q in enumerate(p.measured())}
    u = [0.0] * p.K
    for q in order:
        u[label[q]] = rng.uniform()
    return u


def test_readout_of_a_brickwork(env):
    """The brickwork with its outputs measured in random bases (no gflow):
    from |+> and from a random input, all outputs measured or three kept."""
    total = 0
    for kept in (0, 3):
        for with_input in (False, True):
            wl = workloads.brickwork_readout(7, 10, kept=kept, with_input=with_input)
            total += _check_against_oracle(env, wl, seeds=(11, 12, 13, 14))
    assert total >= 1   # some guess was corrected and its launch run again


def test_measured_product_input(env):
    """A random product input measured qubit by qubit: every probability is
    far from 1/2, so many guesses are corrected (single measure passes)."""
    wl = workloads.measured_inputs(12)
    assert _check_against_oracle(env, wl, seeds=(1, 2, 3)) >= 6


def test_agrees_with_one_at_a_time(env):
    """The same outcomes, probabilities and output as drawing one
    measurement at a time on the device (OWQS_RUN_SEQUENTIAL_SAMPLING), on a
    readout pattern wide enough for pass groups (2^15 live amplitudes)."""
    torch, owqs = env
    wl = workloads.brickwork_readout(14, 12, kept=4, with_input=True)
    h = owqs.load(wl.pattern)
    h.reorder()
    kinds = [owqs.KERNEL_KIND[int(k)] for k in h.profile(_dev(torch, wl.psi_in, "c64"), dtype="c64",
                                                         outcomes=wl.outcomes)[2]]
    assert "group_pass" in kinds
    for dtype in ("c128", "c64"):
        for seed in (21, 22, 23):
            a, oa, pa, _ = h.run(_dev(torch, wl.psi_in, dtype), dtype=dtype, policy="sampled", seed=seed)
            assert h.last_sample_info()["path"] == "checked_launches"
            b, ob, pb, _ = h.run(_dev(torch, wl.psi_in, dtype), dtype=dtype, policy="sampled", seed=seed,
                                 sequential_sampling=True)
            assert h.last_sample_info()["path"] == "one_at_a_time"
            assert np.array_equal(oa, ob), (dtype, seed)
            assert np.max(np.abs(pa - pb)) <= PROB_TOL[dtype]
            d = phase_aligned_maxabs(b.cpu().numpy().astype(np.complex128), a.cpu().numpy().astype(np.complex128))
            assert d <= TOL[dtype], (dtype, seed, d)


def test_flow_pattern_keeps_the_whole_run_guess(env):
    """On a flow pattern the whole-run guess holds and no launch is checked."""
    torch, owqs = env
    wl = workloads.brickwork(10, 8)
    h = owqs.load(wl.pattern)
    h.reorder()
    for seed in (31, 32):
        h.run(None, dtype="c128", policy="sampled", seed=seed)
        info = h.last_sample_info()
        assert info["path"] == "guess_kept" and info["guessed"] and info["checks"] == 0, info


def test_host_vectors(env):
    """Checked launches with host input and output vectors give the device
    run's result."""
    torch, owqs = env
    wl = workloads.brickwork_readout(8, 6, kept=4, with_input=True)
    h = owqs.load(wl.pattern)
    h.reorder()
    dev, od, pd, _ = h.run(_dev(torch, wl.psi_in, "c128"), dtype="c128", policy="sampled", seed=5)
    host_in = torch.from_numpy(wl.psi_in.astype(np.complex128)).pin_memory()
    host_out = torch.empty(1 << 4, dtype=torch.complex128).pin_memory()
    oc, ph = h.run_host(host_in, host_out, dtype="c128", policy="sampled", seed=5)
    assert h.last_sample_info()["path"] == "checked_launches"
    assert np.array_equal(oc, od) and np.array_equal(ph, pd)
    assert np.array_equal(host_out.numpy(), dev.cpu().numpy())
