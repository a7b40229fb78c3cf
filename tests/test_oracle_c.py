"""The C oracle (oracle/substate_omp.c, O-A with OpenMP loops) against the
numpy O-A (oracle/substate.py) and the brute-force O-B: the same outputs,
probabilities and peak sub-state on every kind of pattern, with one thread
and with all host cores; and planted mistakes in the C file are caught.

The C oracle times the CPU baseline on every host core and serves GPU parity
cases too large for the numpy oracle, so it is pinned to the pinned oracles
here (no GPU)."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import brute, proa, substate, substate_c
from owqs_inputs import workloads
from owqs_inputs.patterns import E, M, N, Pattern, X, Z
from owqs_inputs.rng import SplitMix64, random_state

from helpers import outcomes_by_label, random_proposition_order


def _ordered(p):
    """The pattern under its PROA order (a standard pattern in its written
    order entangles every qubit before the first measurement)."""
    return proa.reorder_commands(p, proa.proa(p)[0])


def _cases():
    cases = []
    wl = workloads.small_random()
    cases.append(("small_random", _ordered(wl.pattern), wl.psi_in, outcomes_by_label(wl.pattern, wl.outcomes)))
    for rows, cols in ((4, 8), (3, 5)):
        wl = workloads.brickwork(rows, cols)
        cases.append((f"brickwork{rows}x{cols}", _ordered(wl.pattern), None,
                      outcomes_by_label(wl.pattern, wl.outcomes)))
    wl = workloads.qft(4)
    cases.append(("qft4", _ordered(wl.pattern), wl.psi_in, outcomes_by_label(wl.pattern, wl.outcomes)))
    for i in range(4):
        wl = workloads.random_pattern(i, 3, 5, 3, 6, 3, True)
        cases.append((f"random{i}", _ordered(wl.pattern), wl.psi_in, outcomes_by_label(wl.pattern, wl.outcomes)))
    # a reordered standard pattern (measurements interleaved with E)
    wl = workloads.small_random(1)
    rp = random_proposition_order(wl.pattern, SplitMix64(7))
    cases.append(("reordered", rp, wl.psi_in, outcomes_by_label(wl.pattern, wl.outcomes)))
    # a wild pattern: X and Z between measurements, a later E joining two sub-states
    wild = Pattern(5, [0], [3, 4], [N(1), N(2), N(3), N(4), E(0, 1), M(0, 0.4), X(1, (0,)), E(1, 2), Z(2, (0,)),
                                     M(1, 1.1, (0,)), E(3, 4), E(2, 3), M(2, -0.7, (1,), (0,)), X(3, (2,)),
                                     Z(4, (1,))], "wild")
    cases.append(("wild", wild, random_state(SplitMix64(3), 1), {0: 1, 1: 0, 2: 1}))
    # a sub-state measured away entirely leaves a scalar factor
    scal = Pattern(3, [0], [0], [N(1), N(2), E(1, 2), M(1, 0.3), M(2, 0.9, (1,))], "scalar")
    cases.append(("scalar", scal, random_state(SplitMix64(4), 1), {1: 1, 2: 0}))
    return cases


@pytest.mark.parametrize("threads", [1, 0])
def test_c_oracle_equals_numpy_oracle(threads):
    for name, p, psi, oc in _cases():
        for mode in ("owqs", "eowqs"):
            if mode == "eowqs" and name in ("wild", "scalar"):
                continue
            ref = substate.run(p, psi, outcomes=oc, mode=mode)
            got = substate_c.run(p, psi, outcomes=oc, mode=mode, threads=threads)
            assert np.max(np.abs(got.psi_out - ref.psi_out)) <= 1e-13, (name, mode)
            for q, pv in ref.probs.items():
                assert abs(got.probs[q] - pv) <= 1e-13, (name, mode, q)
            assert got.peak_substate == ref.peak_substate, (name, mode)


def test_c_oracle_zero_policy_and_no_input():
    wl = workloads.small_random()
    p = _ordered(wl.pattern)
    ref = substate.run(p, None, policy="zero", mode="eowqs")
    got = substate_c.run(p, None, policy="zero", mode="eowqs")
    assert np.max(np.abs(got.psi_out - ref.psi_out)) <= 1e-13
    p = Pattern(2, [], [1], [N(0), N(1), E(0, 1), M(0, 0.5)], "no input")
    for psi in (None, np.array([0.6 - 0.8j])):
        ref = substate.run(p, psi, outcomes={0: 1})
        got = substate_c.run(p, psi, outcomes={0: 1})
        assert np.max(np.abs(got.psi_out - ref.psi_out)) <= 1e-14


def test_c_oracle_equals_brute_force():
    wl = workloads.small_random(0, 2, 4)
    oc = outcomes_by_label(wl.pattern, wl.outcomes)
    ref_psi = brute.run(wl.pattern, wl.psi_in, outcomes=oc)[0]
    got = substate_c.run(_ordered(wl.pattern), wl.psi_in, outcomes=oc)
    assert np.max(np.abs(got.psi_out - ref_psi)) <= 1e-12


def test_c_oracle_prefix_probabilities_match():
    """stop_after: the probabilities of a measured prefix (the CPU baseline
    times such a prefix) equal the full run's."""
    wl = workloads.brickwork(6, 6)
    order = proa.proa(wl.pattern)[0]
    p = proa.reorder_commands(wl.pattern, order)
    oc = outcomes_by_label(wl.pattern, wl.outcomes)
    full = substate.run(p, None, outcomes=oc)
    part = substate_c.run(p, None, outcomes=oc, stop_after=7)
    assert len(part.probs) >= 7
    first7 = [c.q0 for c in p.cmds if c.kind == "M"][:7]
    for q in first7:
        assert abs(part.probs[q] - full.probs[q]) <= 1e-13


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
@pytest.mark.parametrize("mutation", [
    ("if (tg) e = -e;", ""),                                            # t signal dropped
    ("const cplx h0 = (a0 + e * a1) * r2, h1 = (a0 - e * a1) * r2;",
     "const cplx h0 = (a0 + e * a1) * r2, h1 = (a0 + e * a1) * r2;"),   # outcome-1 row wrong
    ("a->t[i] = -a->t[i];", "a->t[i] = a->t[i];"),                      # E does nothing
    ("cos(angle[ci]) - I * sin(angle[ci])", "cos(angle[ci]) + I * sin(angle[ci])"),  # Eq. 1 literal sign
])
def test_planted_mistakes_in_the_c_oracle_are_caught(tmp_path, mutation):
    src = open(substate_c.SRC).read()
    assert mutation[0] in src
    bad = tmp_path / "bad.c"
    bad.write_text(src.replace(mutation[0], mutation[1], 1))
    so = tmp_path / "libbad.so"
    subprocess.run(["gcc", "-O1", "-std=c99", "-fopenmp", "-fPIC", "-shared", str(bad), "-o", str(so), "-lm"],
                   check=True, capture_output=True)
    saved = substate_c._lib, substate_c.LIB, substate_c.SRC
    try:
        substate_c._lib, substate_c.LIB, substate_c.SRC = None, str(so), str(bad)
        os.utime(so)
        caught = False
        for name, p, psi, oc in _cases():
            ref = substate.run(p, psi, outcomes=oc)
            got = substate_c.run(p, psi, outcomes=oc)
            if np.max(np.abs(got.psi_out - ref.psi_out)) > 1e-9:
                caught = True
                break
        assert caught, mutation
    finally:
        substate_c._lib, substate_c.LIB, substate_c.SRC = saved
