"""The library's flow search (owqs_find_flow, host only) against the flow
oracle: existence decided bit-exactly like the brute force on tiny open
graphs, and every flow it returns satisfies the definitions, also on graphs
large enough to span several 64-bit words of the GF(2) search."""
import math

import pytest

from oracle import flow
from owqs_inputs import workloads
from owqs_inputs.patterns import E, M, N, Pattern
from owqs_inputs.rng import SplitMix64

from test_oracle_flow import _random_open_graph


@pytest.fixture(scope="module")
def owqs():
    from paper_1604_05659_gb300 import build, owqs as mod
    build.ensure_built()
    mod.library()
    return mod


def _pattern(adj, I, O, angle=0.3):
    n = len(adj)
    cmds = [N(v) for v in range(n) if v not in I]
    cmds += [E(a, b) for a in range(n) for b in sorted(adj[a]) if a < b]
    cmds += [M(v, angle) for v in range(n) if v not in O]
    return Pattern(n, list(I), list(O), cmds, "graph")


def _check(owqs, p, expect_causal=None, expect_gflow=None):
    adj, I, O = flow.open_graph(p)
    h = owqs.load(p)
    cf = h.find_flow("causal")
    gf = h.find_flow("gflow")
    if expect_causal is not None:
        assert (cf is not None) == expect_causal
    if expect_gflow is not None:
        assert (gf is not None) == expect_gflow
    if cf is not None:
        layer, g = cf
        lay = {v: layer[v] for v in range(p.nqubits)}
        assert all(len(s) == 1 for s in g.values())
        assert flow.is_causal_flow(adj, I, O, {i: s[0] for i, s in g.items()}, lay)
        assert gf is not None
    if gf is not None:
        layer, g = gf
        lay = {v: layer[v] for v in range(p.nqubits)}
        assert flow.is_gflow(adj, I, O, {i: set(s) for i, s in g.items()}, lay)
    return cf, gf


def test_existence_matches_brute_force(owqs):
    rng = SplitMix64(77)
    for _ in range(300):
        adj, I, O = _random_open_graph(rng)
        ecf = flow.find_causal_flow_brute(adj, I, O) is not None
        egf = flow.find_gflow_brute(adj, I, O) is not None
        _check(owqs, _pattern(adj, I, O), ecf, egf)


def test_generator_patterns_have_causal_flow(owqs):
    cases = [workloads.brickwork(6, 10).pattern, workloads.qft(6, with_input=False).pattern,
             workloads.small_random().pattern]
    cases += [w.pattern for w in workloads.random_batch(6, 4, 12, 5, 20)]
    for p in cases:
        _check(owqs, p, True, True)


def test_gflow_without_causal_flow_on_a_wide_graph(owqs):
    """A tiny component with gflow and no causal flow beside a brickwork
    component: the whole graph has no causal flow, so the GF(2) layered
    search runs over more than 64 unplaced qubits."""
    rng = SplitMix64(79)
    while True:
        adj, I, O = _random_open_graph(rng)
        if flow.find_gflow_brute(adj, I, O) is not None and flow.find_causal_flow_brute(adj, I, O) is None:
            break
    big = workloads.brickwork(5, 16).pattern
    badj, bI, bO = flow.open_graph(big)
    off = len(badj)
    uadj = [set(s) for s in badj] + [{v + off for v in s} for s in adj]
    p = _pattern(uadj, bI + [v + off for v in I], bO + [v + off for v in O])
    assert p.nqubits - len(p.outputs) > 64
    _check(owqs, p, False, True)


def test_no_flow_cases(owqs):
    # more inputs than outputs, and a measured qubit without neighbours
    _check(owqs, _pattern([{2}, {2}, {0, 1}], [0, 1], [2]), False, False)
    _check(owqs, _pattern([set(), {2}, {1}], [1], [2]), False, False)
