"""Pins of the oracle to facts the paper and the mathematics fix (CPU only).

Each test names the passage it checks.  Together they are chosen so that a
dropped term, a wrong sign or index, or a transposed operand in the oracle
fails at least one of them (tests/test_oracle_mutations.py plants such
mistakes and checks that they are caught).
"""
import cmath
import json
import math
import os

import numpy as np
import pytest

from oracle import basis, brute, circuit, counting, proa, substate
from owqs_inputs import workloads
from owqs_inputs.patterns import (E, M, N, Pattern, X, Z, brickwork_circuit,
                                  circuit_to_pattern, qft_circuit, random_jcz_circuit)
from owqs_inputs.rng import SplitMix64, random_state

from helpers import outcomes_by_label, phase_aligned_maxabs, random_proposition_order

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
R2 = 1.0 / math.sqrt(2.0)


def _val(x):
    if isinstance(x, str):
        return {"r2": R2, "-r2": -R2, "0": 0.0, "0.5": 0.5, "-0.5": -0.5}[x]
    return float(x)


# --------------------------------------------------------------------------
# Section 4.2: operators
# --------------------------------------------------------------------------

@pytest.mark.parametrize("alpha", [0.0, 0.3, 1.1, math.pi / 2, 2.5, math.pi, 4.0, 5.9])
def test_measurement_operators_match_eqs_9_to_12(alpha):
    e_m = cmath.exp(-1j * alpha)
    e_p = cmath.exp(1j * alpha)
    # matrices as printed in Eqs. 9-12
    P0 = 0.5 * np.array([[1, e_m], [e_p, 1]])
    P1 = 0.5 * np.array([[1, -e_m], [-e_p, 1]])
    M0 = R2 * np.array([[1, e_m], [0, 0]])
    M1 = R2 * np.array([[0, 0], [1, -e_m]])
    assert np.allclose(basis.projector(alpha, 0), P0, atol=1e-15)
    assert np.allclose(basis.projector(alpha, 1), P1, atol=1e-15)
    assert np.allclose(basis.gen_operator(alpha, 0), M0, atol=1e-15)
    assert np.allclose(basis.gen_operator(alpha, 1), M1, atol=1e-15)
    # M_i^dag M_i = P_i (Section 4.2) and the completeness of Eq. 5
    for s in (0, 1):
        Ms = basis.gen_operator(alpha, s)
        assert np.allclose(Ms.conj().T @ Ms, basis.projector(alpha, s), atol=1e-15)
    tot = sum(basis.gen_operator(alpha, s).conj().T @ basis.gen_operator(alpha, s) for s in (0, 1))
    assert np.allclose(tot, np.eye(2), atol=1e-15)
    # derivation of Section 4.2: M_0 = |0><0| . H . R_z(-alpha)
    Rz = np.diag([1, e_m])
    assert np.allclose(np.diag([1, 0]) @ circuit.H @ Rz, M0, atol=1e-15)
    assert np.allclose(np.diag([0, 1]) @ circuit.H @ Rz, M1, atol=1e-15)


@pytest.mark.parametrize("alpha,s,t", [(0.4, 0, 0), (0.4, 1, 0), (0.4, 0, 1), (0.4, 1, 1), (2.9, 1, 1)])
def test_signal_dependent_angle_eq2(alpha, s, t):
    theta = (-1) ** s * alpha + t * math.pi
    assert abs(basis.resolved_phase(alpha, s, t) - cmath.exp(-1j * theta)) < 1e-15
    assert abs(basis.resolved_angle(alpha, s, t) - theta) < 1e-15


def test_state_layout_eq8():
    """Eq. 8: the ket |b3 b2 b1> sits at index b3*4 + b2*2 + b1 (qubit 1 is
    bit 0); the oracle's flatten follows that order."""
    amps = {"100": (1 - 1j), "101": -(1 + 1j), "110": (1 + 1j), "111": (-1 + 1j)}
    vec = np.zeros(8, dtype=complex)
    for ket, a in amps.items():
        vec[int(ket, 2)] = a / (2 * math.sqrt(2))
    printed = np.array([0, 0, 0, 0, 1 - 1j, -1 - 1j, 1 + 1j, -1 + 1j]) / (2 * math.sqrt(2))
    assert np.allclose(vec, printed)
    sub = substate.from_flat([1, 2, 3], printed)
    assert sub.labels == [1, 2, 3]
    assert np.allclose(sub.flat(), printed)
    # qubit 3 (bit 2) is 1 in every nonzero amplitude
    assert np.allclose(np.take(sub.tensor, 0, axis=2), 0)
    assert abs(np.linalg.norm(printed) - 1) < 1e-15


def test_measurement_compaction_eq21():
    """Eq. 21: measuring the middle qubit (v = 2) of a 3-qubit state with
    outcome 0 gives alpha'_i = (alpha_i + e^{-ia} beta_i)/sqrt(2 prob_0),
    compacted; alpha_i are the v=0 amplitudes in index order, beta_i the v=1."""
    rng = SplitMix64(21)
    psi = random_state(rng, 3)
    a = 0.77
    p = Pattern(3, [0, 1, 2], [0, 2], [M(1, a)])
    r = substate.run(p, psi, outcomes={1: 0})
    al = psi[[0, 1, 4, 5]]
    be = psi[[2, 3, 6, 7]]
    p0 = 0.5 * np.sum(np.abs(al + cmath.exp(-1j * a) * be) ** 2)
    expect = (al + cmath.exp(-1j * a) * be) / math.sqrt(2 * p0)
    assert abs(r.probs[1] - p0) < 1e-15
    assert np.allclose(r.psi_out, expect, atol=1e-15)


# --------------------------------------------------------------------------
# closed forms: J(alpha), CZ, CNOT (Section 2.1, 2.2)
# --------------------------------------------------------------------------

def jpattern(alpha):
    return Pattern(2, [0], [1], [N(1), E(0, 1), M(0, -alpha), X(1, [0])])


@pytest.mark.parametrize("alpha", [k * math.pi / 8 for k in range(16)] + [0.123, 2.71828, 5.5])
def test_j_alpha_closed_form(alpha):
    """N2 E12 M1^{-a} X2^{s1} = (1/sqrt2)[[1, e^{ia}], [1, -e^{ia}]] for both
    outcomes, exactly (no phase freedom)."""
    Jm = R2 * np.array([[1, cmath.exp(1j * alpha)], [1, -cmath.exp(1j * alpha)]])
    rng = SplitMix64(int(alpha * 1000) + 7)
    for psi in [np.array([1, 0]), np.array([0, 1]), random_state(rng, 1), random_state(rng, 1)]:
        for s in (0, 1):
            for mode in ("owqs", "eowqs"):
                r = substate.run(jpattern(alpha), psi, outcomes={0: s}, mode=mode)
                assert np.allclose(r.psi_out, Jm @ psi, atol=1e-15, rtol=0), (alpha, s, mode)
                if mode == "owqs":
                    assert abs(r.probs[0] - 0.5) < 1e-15


def test_cz_pattern():
    """The pattern E12 with I = O = {1, 2} is the CZ matrix (Section 2.1)."""
    p = Pattern(2, [0, 1], [0, 1], [E(0, 1)])
    for k in range(4):
        e = np.zeros(4)
        e[k] = 1
        assert np.allclose(substate.run(p, e).psi_out, circuit.CZ[:, k])


def cnot_eq22():
    # X_4^{s3} Z_4^{s2} Z_1^{s2} M_3^0 M_2^0 E_13 E_23 E_34 (Eq. 22), q_k -> k-1
    return Pattern(4, [0, 1], [0, 3],
                   [E(2, 3), E(1, 2), E(0, 2), M(1, 0.0), M(2, 0.0), Z(0, [1]), Z(3, [1]), X(3, [2])])


def test_cnot_pattern_eq22():
    """Eq. 22 implements CNOT with control q1 (input bit 0) and target q2
    (input bit 1) -> q4 (output bit 1), up to a global phase, on every branch."""
    # input bit0 = q1 (control), bit1 = q2 (target); output bit0 = q1, bit1 = q4
    U = np.zeros((4, 4))
    for x in range(4):
        c, t = x & 1, (x >> 1) & 1
        U[c | ((t ^ c) << 1), x] = 1
    rng = SplitMix64(22)
    inputs = [np.eye(4)[k] for k in range(4)] + [random_state(rng, 2) for _ in range(3)]
    for psi in inputs:
        for s2 in (0, 1):
            for s3 in (0, 1):
                r = substate.run(cnot_eq22(), psi, outcomes={1: s2, 2: s3})
                assert phase_aligned_maxabs(U @ psi, r.psi_out) < 1e-14
                assert abs(r.probs[1] - 0.5) < 1e-14 and abs(r.probs[2] - 0.5) < 1e-14


def test_figure8_cnot_trace():
    """Every intermediate sub-state of Figure 8 (Eq. 23 order, |q2 q1> = |11>,
    s2 = 0, s3 = 1), with the inputs as separate sub-states (Fig. 8a)."""
    g = json.load(open(os.path.join(GOLDEN, "fig8_cnot_trace.json")))
    cmds = []
    for step in g["eq23_execution_order"]:
        k = step[0]
        if k == "E":
            cmds.append(E(step[1] - 1, step[2] - 1))
        elif k == "M":
            cmds.append(M(step[1] - 1, 0.0))
        else:
            dom = [d - 1 for d in step[2]]
            cmds.append(X(step[1] - 1, dom) if k == "X" else Z(step[1] - 1, dom))
    p = Pattern(4, [q - 1 for q in g["inputs"]], [q - 1 for q in g["outputs"]], cmds)
    snaps = {}

    def tr(i, c, subs):
        snaps[i] = {tuple(s.labels): s.flat() for s in subs}

    r = substate.run(p, None, outcomes={int(k) - 1: v for k, v in g["outcomes"].items()},
                     trace=tr, input_factors=[([0], [0, 1]), ([1], [0, 1])])
    after = {"E23": 0, "M2": 1, "E34 E13": 3, "M3": 4, "X4 Z4 Z1": 7}
    for step in g["steps"][1:]:
        snap = snaps[after[step["after"]]]
        for qs, vals in step["substates"]:
            key = tuple(q - 1 for q in qs)
            assert key in snap, (step["figure"], key, list(snap))
            assert np.allclose(snap[key], [_val(x) for x in vals], atol=1e-15), step["figure"]
    assert np.allclose(r.psi_out, [0, 1, 0, 0])
    assert abs(r.probs[1] - 0.5) < 1e-15 and abs(r.probs[2] - 0.5) < 1e-15


# --------------------------------------------------------------------------
# Section 4.3: PROA
# --------------------------------------------------------------------------

def swap_graph_pattern():
    g = json.load(open(os.path.join(GOLDEN, "table1_swap_proa.json")))
    outs = [q - 1 for q in g["outputs"]]
    cmds = [E(a - 1, b - 1) for a, b in g["edges"]]
    cmds += [M(q, 0.0) for q in range(8) if q not in outs]
    return g, Pattern(8, [0, 1], outs, cmds)


def test_table1_proa_trace():
    """Table I: with every qubit its own sub-state, a = b = d = |O| = 2,
    g = 0.5 and SS = 0, PROA measures 2, 3, 1, 4, 5, 7 with the printed
    measurement state-spaces and sub-states; peak 3."""
    g, p = swap_graph_pattern()
    prm = g["params"]
    stages = []
    order, ms = proa.greedy(p, prm["alpha"], prm["beta"], prm["gamma"], prm["delta"],
                            eowqs=True, product_input=True, stages=stages)
    assert [v + 1 for v in order] == [st["measure"] for st in g["stages"]]
    for got, want in zip(stages, g["stages"]):
        assert got["state_space"] == sorted(q - 1 for q in want["state_space"])
        assert got["substates"] == sorted(sorted(q - 1 for q in s) for s in want["substates"])
    assert max(ms) == 3
    order2, ms2, _ = proa.proa(p, eowqs=True, product_input=True)
    assert [v + 1 for v in order2] == [2, 3, 1, 4, 5, 7] and max(ms2) == 3


def test_cnot_reorder_eq23_and_table3():
    """PROA on Eq. 22 measures q2 first (Eq. 23) and reaches m = 3 (Table III)."""
    p = cnot_eq22()
    for eowqs in (False, True):
        order, ms, _ = proa.proa(p, eowqs=eowqs, product_input=True)
        assert order == [1, 2] and max(ms) == 3
    rp = proa.reorder_commands(p, [1, 2])
    kinds = [(c.kind, c.q0, c.q1) for c in rp.cmds]
    assert kinds[:6] == [("N", 2, -1), ("E", 1, 2), ("M", 1, -1), ("N", 3, -1), ("E", 2, 3), ("E", 0, 2)]


@pytest.mark.parametrize("rows,cols", [(1, 6), (2, 5), (3, 6), (4, 7)])
def test_cluster_column_sweep_bound(rows, cols):
    """Section 4.6: measuring an N x M cluster column by column gives
    m = N + 1 (N = rows); a 1-row cluster keeps m = 2."""
    rng = SplitMix64(46 + rows)
    gates = []
    for c in range(cols - 1):
        for r in range(rows - 1):
            gates.append(("CZ", r, r + 1))
        for r in range(rows):
            gates.append(("J", r, 0.1 * rng.randint(60)))
    for r in range(rows - 1):
        gates.append(("CZ", r, r + 1))
    p = circuit_to_pattern(rows, gates)
    column_order = p.measured()      # circuit order = column by column
    stages = []
    _, ms = proa.greedy(p, 1, 1, 0.5, 1, eowqs=True, product_input=True, stages=stages)
    # the column order itself
    pr = proa.reorder_commands(p, column_order)
    assert proa.single_array_peak(pr) == rows + 1
    # PROA reaches the bound too
    order, ms, _ = proa.proa(p, eowqs=False)
    assert max(ms) == rows + 1


def test_brickwork_proa_peak_small():
    """Brickwork clusters: PROA reaches rows + 1 live qubits."""
    for rows, cols in [(4, 9), (6, 12), (8, 17)]:
        gates, _ = brickwork_circuit(rows, cols, SplitMix64(rows * 100 + cols))
        p = circuit_to_pattern(rows, gates)
        order, ms, _ = proa.proa(p)
        assert max(ms) == rows + 1
        assert proa.single_array_peak(proa.reorder_commands(p, order)) == rows + 1


# --------------------------------------------------------------------------
# invariants, textbook reduction, brute force
# --------------------------------------------------------------------------

def _small_circuits():
    res = []
    for i in range(6):
        rng = SplitMix64(1000 + i)
        n = 2 + rng.randint(3)
        d = 2 + rng.randint(4)
        res.append((n, random_jcz_circuit(n, d, rng, cz_per_layer=1), rng))
    return res


def test_textbook_reduction_jcz_circuits():
    """For J/CZ circuits, the pattern output equals the product of the J and
    CZ gate matrices applied to the input, up to a global phase, for every
    branch (determinism of flow patterns, Section 4.5)."""
    for n, gates, rng in _small_circuits():
        p = circuit_to_pattern(n, gates)
        U = circuit.circuit_unitary(n, gates)
        psi = random_state(rng, n)
        ref = U @ psi
        for b in range(3):
            bits = SplitMix64(77 + b).bits(p.K)
            r = substate.run(p, psi, outcomes=outcomes_by_label(p, bits))
            assert phase_aligned_maxabs(ref, r.psi_out) < 1e-12
            assert all(abs(v - 0.5) < 1e-12 for v in r.probs.values())


def test_gate_by_gate_application_equals_the_dense_product():
    """apply_circuit (per-gate updates of one vector, for widths where the
    dense product does not fit) equals circuit_unitary on random J/CZ
    circuits, column by column and on random states, exactly up to rounding;
    a J on the wrong wire or a CZ on the wrong pair is caught."""
    for i in range(6):
        rng = SplitMix64(5100 + i)
        n = 2 + rng.randint(4)
        gates = random_jcz_circuit(n, 3, rng, cz_per_layer=1)
        U = circuit.circuit_unitary(n, gates)
        for c in range(1 << n):
            e = np.zeros(1 << n, dtype=np.complex128)
            e[c] = 1
            assert np.max(np.abs(circuit.apply_circuit(n, gates, e) - U[:, c])) < 1e-13
        psi = random_state(rng, n)
        assert np.max(np.abs(circuit.apply_circuit(n, gates, psi) - U @ psi)) < 1e-13
        wrong = [("J", (g[1] + 1) % n, g[2]) if g[0] == "J" else g for g in gates]
        assert np.max(np.abs(circuit.apply_circuit(n, wrong, psi) - U @ psi)) > 1e-3


def test_qft_small_textbook():
    """QFT-shaped J/CZ pattern (3 wires) against the DFT matrix up to the bit
    reversal the missing final swaps leave and a global phase."""
    n = 3
    p = circuit_to_pattern(n, qft_circuit(n))
    U = circuit.circuit_unitary(n, qft_circuit(n))
    Nn = 1 << n
    F = np.array([[cmath.exp(2j * math.pi * j * k / Nn) for k in range(Nn)] for j in range(Nn)]) / math.sqrt(Nn)
    # wire 0 is processed first, so it plays the most significant input bit;
    # without the final swaps it ends holding the least significant output bit
    rev = [int(format(j, f"0{n}b")[::-1], 2) for j in range(Nn)]
    Frev = F[:, rev]
    for k in range(Nn):
        assert phase_aligned_maxabs(Frev[:, k], U[:, k]) < 1e-12
    psi = random_state(SplitMix64(5), n)
    pr = proa.reorder_commands(p, p.measured())      # standard order would be 50+ qubits wide
    r = substate.run(pr, psi, outcomes=outcomes_by_label(p, SplitMix64(6).bits(p.K)))
    assert phase_aligned_maxabs(Frev @ psi, r.psi_out) < 1e-12


def test_invariants_norm_probs_determinism_order():
    """Norm 1 after every OWQS measurement; p0 + p1 = 1; every branch of a
    flow pattern has p = 1/2 and the same output; with forced outcomes the
    output does not depend on the command order (Proposition, Eqs. 14-17)."""
    wl = workloads.small_random()
    std = wl.pattern
    p = proa.reorder_commands(std, std.measured())   # circuit order; all-E-first is 33 qubits wide
    outs = outcomes_by_label(p, wl.outcomes)
    norms = []

    def tr(i, c, subs):
        if c.kind == "M":
            norms.append(np.prod([np.linalg.norm(s.flat()) for s in subs]))

    base = substate.run(p, wl.psi_in, outcomes=outs, trace=tr)
    assert np.allclose(norms, 1.0, atol=1e-14)
    for v, (p0, p1) in base.pairs.items():
        assert abs(p0 + p1 - 1) < 1e-14 and abs(p0 - 0.5) < 1e-13
    for b in range(4):
        other = substate.run(p, wl.psi_in, outcomes=outcomes_by_label(p, SplitMix64(900 + b).bits(p.K)))
        assert phase_aligned_maxabs(base.psi_out, other.psi_out) < 1e-13
    order, _, _ = proa.proa(std)
    for q in [proa.reorder_commands(std, order)] + [random_proposition_order(std, SplitMix64(40 + k)) for k in range(4)]:
        r = substate.run(q, wl.psi_in, outcomes=outs)
        assert np.allclose(r.psi_out, base.psi_out, atol=1e-13, rtol=0)   # exact, no phase alignment
    # EOWQS: all-zero branch, same output up to phase, norm 1
    ez = substate.run(p, wl.psi_in, policy="zero", mode="eowqs")
    assert abs(np.linalg.norm(ez.psi_out) - 1) < 1e-13
    assert phase_aligned_maxabs(base.psi_out, ez.psi_out) < 1e-13


def _wild_patterns():
    """Small non-standard patterns with corrections between measurements."""
    pats = []
    for i in range(8):
        rng = SplitMix64(3000 + i)
        n = 2 + rng.randint(2)
        gates = random_jcz_circuit(n, 2 + rng.randint(2), rng)
        p = circuit_to_pattern(n, gates)
        # wild form: each measurement followed by its flow corrections
        cmds = [c for c in p.cmds if c.kind in ("N", "E")]
        ms = [c for c in p.cmds if c.kind == "M"]
        from owqs_inputs.patterns import Cmd
        for m in ms:
            cmds.append(Cmd("M", m.q0, -1, m.angle + 0.3 * rng.uniform()))
            tgt = rng.randint(p.nqubits)
            for q in (tgt, rng.randint(p.nqubits)):
                if q not in [x.q0 for x in cmds if x.kind == "M"]:
                    cmds.append(Cmd("X" if rng.randint(2) else "Z", q, -1, 0.0, (m.q0,)))
        cmds += [c for c in p.cmds if c.kind in ("X", "Z")]
        pats.append(p.with_cmds(cmds))
    return pats


def test_bruteforce_agrees_with_substate():
    """O-A (elimination, sub-states) equals O-B (full register, projectors)
    on tiny patterns, exactly including the phase, in both modes."""
    pats = [cnot_eq22(), jpattern(0.9)] + [circuit_to_pattern(n, g) for n, g, _ in _small_circuits()[:4]]
    pats += _wild_patterns()
    for i, p in enumerate(pats):
        if p.nqubits > 14:
            continue
        rng = SplitMix64(500 + i)
        psi = random_state(rng, len(p.inputs))
        bits = rng.bits(p.K)
        outs = outcomes_by_label(p, bits)
        for mode in ("owqs", "eowqs"):
            ra = substate.run(p, psi, outcomes=outs, mode=mode)
            ob, _, probs = brute.run(p, psi, outcomes=outs, mode=mode)
            assert np.allclose(ra.psi_out, ob, atol=1e-13, rtol=0), (i, mode)
            if mode == "owqs":
                for v in probs:
                    assert abs(probs[v] - ra.probs[v]) < 1e-13
        # sampled outcomes follow the same stream on both
        ra = substate.run(p, psi, policy="sampled", seed=17 + i)
        ob, meas, _ = brute.run(p, psi, policy="sampled", seed=17 + i)
        assert meas == ra.outcomes
        assert np.allclose(ra.psi_out, ob, atol=1e-13, rtol=0)


def test_eowqs_sampled_draws_fair_coins():
    """Section 4.5: with a flow every branch has probability 1/2, so EOWQS
    draws a sampled outcome against 1/2 without computing anything.  The
    outcome of the k-th measurement in execution order is then fixed by the
    k-th splitmix64 uniform alone (0 iff u <= 1/2), the output is the OWQS
    output of the same branch, OWQS sampling with the same seed draws the
    same outcomes (its probabilities are 1/2 up to rounding), and the
    brute-force oracle agrees."""
    for n, gates, rng in _small_circuits()[:5]:
        p = circuit_to_pattern(n, gates)
        psi = random_state(rng, n)
        order = [c.q0 for c in p.cmds if c.kind == "M"]
        for seed in (3, 4, 5):
            stream = SplitMix64(seed)
            u = [stream.uniform() for _ in order]
            want = {q: (0 if uk <= 0.5 else 1) for q, uk in zip(order, u)}
            e = substate.run(p, psi, mode="eowqs", policy="sampled", seed=seed)
            assert e.outcomes == want
            assert all(v == 0.5 for v in e.probs.values())
            f = substate.run(p, psi, outcomes=want)
            assert np.allclose(e.psi_out, f.psi_out, atol=1e-13, rtol=0)
            if min(abs(uk - 0.5) for uk in u) > 1e-9:
                o = substate.run(p, psi, policy="sampled", seed=seed)
                assert o.outcomes == want
            if p.nqubits <= 14:
                ob, meas, _ = brute.run(p, psi, mode="eowqs", policy="sampled", seed=seed)
                assert meas == want
                assert np.allclose(ob, e.psi_out, atol=1e-13, rtol=0)
    # where prob_0 is not 1/2 (one measured input, no flow), EOWQS still draws
    # against 1/2 and OWQS against prob_0 = |<+_a|psi>|^2: they differ exactly
    # for u between the two
    p = Pattern(2, [0], [1], [N(1), M(0, 0.3)])
    psi = np.array([0.8, 0.6j])
    p0 = substate.run(p, psi, outcomes={0: 0}).pairs[0][0]
    assert abs(p0 - 0.5) > 0.1
    differ = 0
    for seed in range(40):
        u = SplitMix64(seed).uniform()
        e = substate.run(p, psi, mode="eowqs", policy="sampled", seed=seed)
        o = substate.run(p, psi, policy="sampled", seed=seed)
        _, eb, _ = brute.run(p, psi, mode="eowqs", policy="sampled", seed=seed)
        assert e.outcomes[0] == eb[0] == (0 if u <= 0.5 else 1)
        assert o.outcomes[0] == (0 if u <= p0 else 1)
        differ += int(e.outcomes[0] != o.outcomes[0])
    assert differ >= 2


def test_well_formedness_rules():
    with pytest.raises(basis.PatternError):   # D0: depends on unmeasured
        basis.validate(Pattern(3, [0], [2], [E(0, 1), E(1, 2), M(0, 0.0, [1]), M(1, 0.0)]))
    with pytest.raises(basis.PatternError):   # D1: acts on measured
        basis.validate(Pattern(2, [0], [1], [E(0, 1), M(0, 0.0), Z(0)]))
    with pytest.raises(basis.PatternError):   # D2: before preparation
        basis.validate(Pattern(2, [0], [1], [E(0, 1), N(1), M(0, 0.0)]))
    with pytest.raises(basis.PatternError):   # D3: output measured
        basis.validate(Pattern(2, [0], [1], [E(0, 1), M(0, 0.0), M(1, 0.0)]))
    with pytest.raises(basis.PatternError):   # E on one qubit
        basis.validate(Pattern(2, [0], [1], [E(1, 1), M(0, 0.0)]))
    basis.validate(cnot_eq22())


def test_generated_patterns_are_standard_and_valid():
    for wl in [workloads.small_random(), workloads.brickwork(4, 6), workloads.qft(4)]:
        p = wl.pattern
        basis.validate(p)
        assert p.is_standard()
    p = workloads.small_random().pattern
    assert p.nqubits == 33 and p.K == 30 and len(p.outputs) == 3
    q = workloads.qft(24, with_input=False).pattern
    assert q.K == 24 + 276 * 10
    b = workloads.brickwork(28, 40).pattern
    assert b.K == 28 * 39 and b.nqubits == 28 * 40


def test_amplitude_update_count_closed_form():
    """One wire of L J gates: live widths 1 -> 2 (N, E, M at 2^2 each) per gate,
    then the output corrections at width 1: X always, Z once L >= 2
    (the flow's Z correction from the second-to-last measurement); so
    12 L + 2 + 2 [L >= 2] updates."""
    for L in (1, 2, 3, 7):
        p = circuit_to_pattern(1, [("J", 0, 0.1 * k) for k in range(L)])
        pr = proa.reorder_commands(p, p.measured())
        assert counting.amplitude_updates(pr) == 12 * L + 2 + (2 if L >= 2 else 0)


def test_no_input_qubit_takes_a_one_amplitude_input():
    """A pattern without input qubits: its input is a state over no qubit,
    one amplitude c, and the initial state is c times |+> on every qubit
    (Section 4.1).  Both oracles then give c/|c| (OWQS: the input is
    normalised, Eq. 4) or c (EOWQS) times the result from the default
    input, and agree with each other."""
    p = Pattern(3, [], [2], [N(0), N(1), N(2), E(0, 1), E(1, 2), M(0, 1.1), M(1, -0.4, sdom=(0,))], "no_input")
    c = 0.6 - 0.8j
    for mode in ("owqs", "eowqs"):
        for bits in ([0, 0], [1, 0], [0, 1], [1, 1]):
            outs = outcomes_by_label(p, bits)
            base = substate.run(p, None, outcomes=outs, mode=mode).psi_out
            ra = substate.run(p, np.array([c * 2.5]), outcomes=outs, mode=mode).psi_out
            ob, _, _ = brute.run(p, np.array([c * 2.5]), outcomes=outs, mode=mode)
            factor = c if mode == "owqs" else c * 2.5
            assert np.allclose(ra, factor * base, atol=1e-14, rtol=0), (mode, bits)
            assert np.allclose(ob, ra, atol=1e-13, rtol=0), (mode, bits)
