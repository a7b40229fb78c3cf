"""Pins of the flow oracle (oracle/flow.py) on the CPU: the definitions
against flows known by construction and planted mistakes, the necessary
conditions of a gflow, and the determinism a gflow guarantees (the reason
Section 4.5 asks for one), checked by simulating every branch."""
import itertools
import math

import numpy as np
import pytest

from oracle import flow, substate
from owqs_inputs import workloads
from owqs_inputs.patterns import E, M, N, Pattern, X, Z, circuit_to_pattern, random_jcz_circuit
from owqs_inputs.rng import SplitMix64, random_state

from helpers import phase_aligned_maxabs


def _wire_flow(p):
    """The generator's flow: f(i) is the one qubit whose X correction
    (s-domain, or output X domain) contains i."""
    f = {}
    for c in p.cmds:
        dom = c.sdom if c.kind in ("M", "X") else ()
        for i in dom:
            assert i not in f
            f[i] = c.q0
    return f


def _order_layer(p):
    meas = p.measured()
    layer = {o: 0 for o in p.outputs}
    for k, v in enumerate(meas):
        layer[v] = len(meas) - k
    return layer


def test_generator_flows_satisfy_the_definitions():
    cases = [workloads.small_random().pattern, workloads.brickwork(5, 8).pattern, workloads.qft(4, with_input=False).pattern]
    cases += [w.pattern for w in workloads.random_batch(6, 3, 7, 3, 8)]
    for p in cases:
        adj, I, O = flow.open_graph(p)
        f = _wire_flow(p)
        layer = _order_layer(p)
        assert flow.is_causal_flow(adj, I, O, f, layer), p.name
        assert flow.is_gflow(adj, I, O, {i: {fi} for i, fi in f.items()}, layer), p.name


def test_planted_mistakes_are_rejected():
    p = workloads.random_batch(1, 4, 4, 4, 4, start=3)[0].pattern
    adj, I, O = flow.open_graph(p)
    f = _wire_flow(p)
    layer = _order_layer(p)
    first = p.measured()[0]
    # F1: a non-neighbour as f(i)
    bad = dict(f)
    bad[first] = next(v for v in range(p.nqubits) if v not in adj[first] and v != first and v not in I)
    assert not flow.is_causal_flow(adj, I, O, bad, layer)
    # F2: the order reversed
    rev = {v: (0 if l == 0 else len(f) + 1 - l) for v, l in layer.items()}
    assert not flow.is_causal_flow(adj, I, O, f, rev)
    assert not flow.is_gflow(adj, I, O, {i: {fi} for i, fi in f.items()}, rev)
    # G3: i in g(i); g(i) empty
    g = {i: {fi} for i, fi in f.items()}
    g2 = dict(g)
    g2[first] = {f[first], first}
    assert not flow.is_gflow(adj, I, O, g2, layer)
    g3 = dict(g)
    g3[first] = set()
    assert not flow.is_gflow(adj, I, O, g3, layer)
    # G2: a set whose odd neighbourhood reaches an earlier qubit
    last = p.measured()[-1]
    g4 = dict(g)
    g4[last] = {f[last]} | {f[first]}
    assert not flow.is_gflow(adj, I, O, g4, layer)


def _random_open_graph(rng, nmin=3, nmax=6):
    n = nmin + rng.randint(nmax - nmin + 1)
    adj = [set() for _ in range(n)]
    for a in range(n):
        for b in range(a + 1, n):
            if rng.uniform() < 0.5:
                adj[a].add(b)
                adj[b].add(a)
    perm = list(range(n))
    for k in range(n - 1, 0, -1):
        j = rng.randint(k + 1)
        perm[k], perm[j] = perm[j], perm[k]
    nout = 1 + rng.randint(min(3, n - 1))
    O = sorted(perm[:nout])
    nin = rng.randint(3)
    I = sorted(rng.randint(n) for _ in range(nin))
    I = sorted(set(I))
    return adj, I, O


def test_necessary_conditions_and_causal_implies_gflow():
    rng = SplitMix64(77)
    both = causal_only = gflow_only = 0
    for _ in range(300):
        adj, I, O = _random_open_graph(rng)
        gf = flow.find_gflow_brute(adj, I, O)
        cf = flow.find_causal_flow_brute(adj, I, O)
        if gf is not None:
            assert len(I) <= len(O)            # a deterministic map from I to O is an isometry
            assert flow.is_gflow(adj, I, O, *gf)
        if cf is not None:
            assert flow.is_causal_flow(adj, I, O, *cf)
            f, layer = cf
            assert gf is not None and flow.is_gflow(adj, I, O, {i: {fi} for i, fi in f.items()}, layer)
        both += cf is not None
        gflow_only += gf is not None and cf is None
    assert both > 20 and gflow_only > 0        # the two notions differ
    # no outputs: the last measured qubit has nothing to correct it
    adj = [{1}, {0, 2}, {1}]
    assert flow.find_gflow_brute(adj, [0], []) is None


def _gflow_pattern(adj, I, O, g, layer, angles, drop=None):
    """N on non-inputs, every edge, then each qubit measured from the highest
    layer down followed by X on g(i) and Z on Odd(g(i)) minus i, conditioned
    on s_i (optionally one correction left out)."""
    n = len(adj)
    cmds = [N(v) for v in range(n) if v not in I]
    cmds += [E(a, b) for a in range(n) for b in sorted(adj[a]) if a < b]
    order = sorted((v for v in range(n) if v not in O), key=lambda v: -layer[v])
    for i in order:
        cmds.append(M(i, angles[i]))
        for j in sorted(g[i]):
            if drop != (i, "X", j):
                cmds.append(X(j, (i,)))
        for k in sorted(flow.odd(adj, g[i]) - {i}):
            if drop != (i, "Z", k):
                cmds.append(Z(k, (i,)))
    return Pattern(n, list(I), list(O), cmds, "gflow"), order


def _branches(p, order, psi):
    outs, probs = [], []
    for bits in itertools.product((0, 1), repeat=len(order)):
        r = substate.run(p, psi, outcomes=dict(zip(order, bits)))
        outs.append(r.psi_out)
        probs += [r.probs[q] for q in order]
    return outs, probs


def test_gflow_corrections_make_every_branch_deterministic():
    """Uniform strong determinism from a gflow ([13]; Section 4.5): each
    outcome has probability 1/2 and every branch gives the same output up to
    a global phase.  Leaving out one correction breaks it."""
    rng = SplitMix64(78)
    checked = broken = 0
    while checked < 25:
        adj, I, O = _random_open_graph(rng, 3, 6)
        gf = flow.find_gflow_brute(adj, I, O)
        if gf is None or len(adj) - len(O) == 0:
            continue
        g, layer = gf
        angles = {v: 2 * math.pi * rng.uniform() for v in range(len(adj))}
        psi = random_state(rng, len(I))
        p, order = _gflow_pattern(adj, I, O, g, layer, angles)
        outs, probs = _branches(p, order, psi)
        assert np.max(np.abs(np.array(probs) - 0.5)) < 1e-12
        for o in outs[1:]:
            assert phase_aligned_maxabs(outs[0], o) < 1e-12
        checked += 1
        # plant a mistake: drop the last correction of the first measurement
        i = order[0]
        zs = sorted(flow.odd(adj, g[i]) - {i})
        drop = (i, "Z", zs[-1]) if zs else (i, "X", sorted(g[i])[-1])
        pb, _ = _gflow_pattern(adj, I, O, g, layer, angles, drop=drop)
        outs, probs = _branches(pb, order, psi)
        dev = max(np.max(np.abs(np.array(probs) - 0.5)), max(phase_aligned_maxabs(outs[0], o) for o in outs))
        broken += dev > 1e-6
    assert broken >= 20, broken
