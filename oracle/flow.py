"""Causal flow and gflow of a pattern's open graph -- oracle; test
infrastructure only.

Section 4.5: EOWQS simulates only patterns whose open graph (G, I, O) has a
generalized flow (gflow, ref. [13]); a gflow is sought before each pattern is
simulated, and a pattern without one is reported as incorrect.  The paper
gives neither the definition nor the finding algorithm (ref. [25]); this file
writes out the published definitions and decides existence by brute force
over measurement orders, with no search strategy of its own.

Open graph: V = every qubit label of the pattern, I and O as given, and an
edge u-v iff the pattern has an odd number of E commands on {u, v} (two CZ on
the same pair cancel).  Odd(K) is the set of vertices with an odd number of
neighbours in K.

Causal flow (f, <): f maps each measured qubit i (i not in O) to a non-input
f(i) with
  (F1) f(i) adjacent to i,
  (F2) i < f(i),
  (F3) i < k for every neighbour k of f(i) other than i.
Gflow (g, <), every measurement in the XY plane (the paper's M^alpha): g maps
each measured i to a set of non-inputs with
  (G1) i < j for every j in g(i),
  (G2) i < j for every j in Odd(g(i)) other than i,
  (G3) i not in g(i) and i in Odd(g(i)).
Here < is given by layers: layer 0 holds the outputs, measured qubits have
layers >= 1, and i < j iff layer(i) > layer(j) (a higher layer is measured
earlier).  A flow of either kind exists iff one exists with respect to some
total order of the measured qubits, which is what the brute force enumerates.

Parity pinned by tests/test_oracle_flow.py: flows known by construction (the
circuit generator's wire successor), mutated flows rejected, the necessary
conditions |I| <= |O| and O non-empty, causal flow implying gflow, a graph
with gflow and no causal flow, and the determinism the flow guarantees: a
pattern built from a brute-force gflow with the corrections X on g(i) and Z
on Odd(g(i)) minus i gives probability 1/2 at every measurement and the same
output on every branch (simulated by substate.run).
"""
from __future__ import annotations

import itertools
from typing import Dict, List, Optional, Sequence, Set, Tuple


def open_graph(pattern) -> Tuple[List[Set[int]], List[int], List[int]]:
    """Adjacency sets over labels 0..nqubits-1 from the E commands (odd
    multiplicity), and the input and output lists."""
    adj = [set() for _ in range(pattern.nqubits)]
    for c in pattern.cmds:
        if c.kind == "E":
            u, v = c.q0, c.q1
            if v in adj[u]:
                adj[u].discard(v)
                adj[v].discard(u)
            else:
                adj[u].add(v)
                adj[v].add(u)
    return adj, list(pattern.inputs), list(pattern.outputs)


def odd(adj: Sequence[Set[int]], K) -> Set[int]:
    """Vertices with an odd number of neighbours in K."""
    count: Dict[int, int] = {}
    for k in K:
        for v in adj[k]:
            count[v] = count.get(v, 0) ^ 1
    return {v for v, c in count.items() if c}


def before(layer: Dict[int, int], i: int, j: int) -> bool:
    """i < j: i is measured strictly before j (outputs are at layer 0)."""
    return layer[i] > layer[j]


def is_causal_flow(adj, inputs, outputs, f: Dict[int, int], layer: Dict[int, int]) -> bool:
    """(F1)-(F3) with the layer order; f must cover exactly the measured qubits."""
    V = set(range(len(adj)))
    O, I = set(outputs), set(inputs)
    measured = V - O
    if set(f) != measured or any(layer.get(o, -1) != 0 for o in O):
        return False
    if any(layer.get(i, 0) < 1 for i in measured):
        return False
    for i, fi in f.items():
        if fi in I or fi not in V:
            return False
        if fi not in adj[i]:                               # F1
            return False
        if not before(layer, i, fi):                       # F2
            return False
        for k in adj[fi]:                                  # F3
            if k != i and not before(layer, i, k):
                return False
    return True


def is_gflow(adj, inputs, outputs, g: Dict[int, Set[int]], layer: Dict[int, int]) -> bool:
    """(G1)-(G3) with the layer order; g must cover exactly the measured qubits."""
    V = set(range(len(adj)))
    O, I = set(outputs), set(inputs)
    measured = V - O
    if set(g) != measured or any(layer.get(o, -1) != 0 for o in O):
        return False
    if any(layer.get(i, 0) < 1 for i in measured):
        return False
    for i, gi in g.items():
        gi = set(gi)
        if not gi <= V or gi & I:
            return False
        if any(not before(layer, i, j) for j in gi):        # G1
            return False
        oi = odd(adj, gi)
        if any(j != i and not before(layer, i, j) for j in oi):   # G2
            return False
        if i in gi or i not in oi:                          # G3
            return False
    return True


def _order_layers(order: Sequence[int], outputs) -> Dict[int, int]:
    """Layers of a total order: the first measured qubit gets the highest."""
    layer = {o: 0 for o in outputs}
    for pos, v in enumerate(order):
        layer[v] = len(order) - pos
    return layer


def find_gflow_brute(adj, inputs, outputs, max_measured: int = 7) -> Optional[Tuple[Dict[int, Set[int]], Dict[int, int]]]:
    """A gflow by brute force: every order of the measured qubits and, at
    each position, every subset of the later non-input qubits; None if no
    gflow exists.  Tiny graphs only."""
    V = list(range(len(adj)))
    O, I = set(outputs), set(inputs)
    measured = [v for v in V if v not in O]
    if len(measured) > max_measured:
        raise ValueError("brute force is for tiny graphs")
    for order in itertools.permutations(measured):
        g: Dict[int, Set[int]] = {}
        ok = True
        for pos, i in enumerate(order):
            later = set(order[pos + 1:]) | O
            cands = sorted(later - I)
            earlier_or_self = set(order[:pos + 1])
            found = None
            for r in range(len(cands) + 1):
                for K in itertools.combinations(cands, r):
                    oi = odd(adj, K)
                    if i in oi and not ((oi - {i}) & earlier_or_self):
                        found = set(K)
                        break
                if found is not None:
                    break
            if found is None:
                ok = False
                break
            g[i] = found
        if ok:
            return g, _order_layers(order, outputs)
    return None


def find_causal_flow_brute(adj, inputs, outputs, max_measured: int = 7) -> Optional[Tuple[Dict[int, int], Dict[int, int]]]:
    """A causal flow by brute force: every order of the measured qubits and,
    at each position, every later non-input neighbour as f(i); None if no
    causal flow exists.  Tiny graphs only."""
    V = list(range(len(adj)))
    O, I = set(outputs), set(inputs)
    measured = [v for v in V if v not in O]
    if len(measured) > max_measured:
        raise ValueError("brute force is for tiny graphs")
    for order in itertools.permutations(measured):
        layer = _order_layers(order, outputs)
        f: Dict[int, int] = {}
        ok = True
        for i in order:
            choice = None
            for fi in sorted(adj[i]):
                if fi in I or not before(layer, i, fi):
                    continue
                if all(k == i or before(layer, i, k) for k in adj[fi]):
                    choice = fi
                    break
            if choice is None:
                ok = False
                break
            f[i] = choice
        if ok:
            return f, layer
    return None


def gflow_exists(pattern) -> bool:
    adj, I, O = open_graph(pattern)
    return find_gflow_brute(adj, I, O) is not None
