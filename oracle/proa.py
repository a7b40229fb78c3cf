"""Greedy pattern reordering, PROA (Section 4.3) -- oracle; test
infrastructure only.

The Proposition of Section 4.3 (Eqs. 14-17): before measuring a qubit v whose
dependencies are resolved, only the E commands on v are needed.  PROA picks
the measurement order greedily; each step it scores every ready qubit with the
Eq. 18 cost and takes the cheapest:

    Cost(v) = a*MS(v) + b*OS(v) - g*SS(v)              if flag(v) = 1
              a*((MS(v)+1)*d) + b*OS(v) - g*SS(v)      if flag(v) = 0

Readings of the criteria (the paper defines them in words):
  MS(v)  size of the sub-state created by measuring v: the union of v's
         sub-state and the sub-states of every neighbour joined to v by an E
         not yet applied (counting v);
  OS(v)  number of output qubits adjacent to v in the entanglement graph;
  SS(v)  |S(v)|, the number of qubits whose measurement domains or
         correction domains contain v; 0 in EOWQS mode (no dependencies);
  flag   1 iff v is adjacent to a qubit already selected.
Ready list: qubits whose s- and t-domains are all measured; in EOWQS mode
every qubit is ready from the start (Section 4.5).  Ties go to the lowest
qubit label.  Parameters follow Section 5: a = b = d = |O|, g = 0.5, and a is
swept |O|, |O|-1, ..., 1; the best run has the smallest peak MS, then the
smallest sum over steps of 2^MS, then comes first.
Sub-states: the input qubits start as one sub-state (the input vector may be
entangled); with product_input=True every qubit starts alone, as in Table I.
"""
from __future__ import annotations

from typing import Dict, List, Tuple


class _DSU:
    def __init__(self, n):
        self.parent = list(range(n))

    def find(self, x):
        while self.parent[x] != x:
            self.parent[x] = self.parent[self.parent[x]]
            x = self.parent[x]
        return x

    def union(self, a, b):
        ra, rb = self.find(a), self.find(b)
        if ra != rb:
            self.parent[max(ra, rb)] = min(ra, rb)


def _dependents(pattern) -> Dict[int, set]:
    dep = {q: set() for q in range(pattern.nqubits)}
    for c in pattern.cmds:
        if c.kind in ("M", "X", "Z"):
            for d in tuple(c.sdom) + tuple(c.tdom):
                dep[d].add(c.q0)
    return dep


def greedy(pattern, a: float, b: float, g: float, d: float, eowqs: bool = False,
           product_input: bool = False, stages: list | None = None) -> Tuple[List[int], List[int]]:
    """One greedy run; returns (measurement order, MS at each step).  If
    `stages` is a list, one record per step is appended: the measured qubit,
    its measurement state-space and the sub-states left afterwards."""
    n = pattern.nqubits
    outputs = set(pattern.outputs)
    measured_q = [c.q0 for c in pattern.cmds if c.kind == "M"]
    adj = [set() for _ in range(n)]
    pending = [set() for _ in range(n)]
    for c in pattern.cmds:
        if c.kind == "E":
            adj[c.q0].add(c.q1)
            adj[c.q1].add(c.q0)
            pending[c.q0] ^= {c.q1}
            pending[c.q1] ^= {c.q0}
    deps = {c.q0: set(c.sdom) | set(c.tdom) for c in pattern.cmds if c.kind == "M"}
    dependents = _dependents(pattern)
    ss = {v: (0 if eowqs else len(dependents[v])) for v in measured_q}
    os_ = {v: len(adj[v] & outputs) for v in measured_q}

    dsu = _DSU(n)
    members: Dict[int, set] = {q: {q} for q in range(n)}

    def merge(x, y):
        ra, rb = dsu.find(x), dsu.find(y)
        if ra != rb:
            dsu.union(ra, rb)
            root = dsu.find(ra)
            other = rb if root == ra else ra
            members[root] |= members.pop(other)

    if not product_input:
        for q in pattern.inputs[1:]:
            merge(pattern.inputs[0], q)

    def sub(q):
        return members[dsu.find(q)]

    done = set()
    selected = set()
    order, ms_list = [], []
    remaining = set(measured_q)
    while remaining:
        best_v, best_cost, best_ms = None, None, None
        for v in sorted(remaining):
            if not eowqs and not deps[v] <= done:
                continue
            ms = set(sub(v))
            for u in pending[v]:
                ms |= sub(u)
            msz = len(ms)
            flag = any(u in selected for u in adj[v])
            if flag:
                cost = a * msz + b * os_[v] - g * ss[v]
            else:
                cost = a * ((msz + 1) * d) + b * os_[v] - g * ss[v]
            if best_cost is None or cost < best_cost:
                best_v, best_cost, best_ms, best_set = v, cost, msz, ms
        if best_v is None:
            raise ValueError("no ready qubit: dependency cycle")
        v = best_v
        # apply v's pending E commands: merge sub-states, then eliminate v
        for u in list(pending[v]):
            merge(v, u)
            pending[u].discard(v)
        pending[v] = set()
        members[dsu.find(v)].discard(v)
        order.append(v)
        ms_list.append(best_ms)
        if stages is not None:
            subs = sorted(sorted(m) for m in members.values() if m)
            stages.append({"measure": v, "state_space": sorted(best_set), "substates": subs})
        selected.add(v)
        done.add(v)
        remaining.discard(v)
    return order, ms_list


def proa(pattern, eowqs: bool = False, product_input: bool = False):
    """Parameter sweep of Section 5; returns (order, ms_list, alpha)."""
    k = len(pattern.outputs)
    best = None
    for a in range(k, 0, -1) if k > 0 else [1]:
        kk = max(k, 1)
        order, ms = greedy(pattern, float(a), float(kk), 0.5, float(kk), eowqs, product_input)
        key = (max(ms) if ms else 0, sum(2 ** m for m in ms))
        if best is None or key < best[0]:
            best = (key, order, ms, a)
    return best[1], best[2], best[3]


def reorder_commands(pattern, order: List[int]):
    """Command list for a measurement order (Eq. 17): for each v in order,
    the E commands on v not yet applied (original order), each preceded by N
    for endpoints not yet prepared, then M_v; afterwards the remaining E
    commands, N for outputs never touched, and the corrections in their
    original order.  Requires a standard-form pattern."""
    from owqs_inputs.patterns import Cmd
    if not pattern.is_standard():
        raise ValueError("PROA needs a standard-form pattern")
    inputs = set(pattern.inputs)
    prepared = set(inputs)
    e_cmds = [c for c in pattern.cmds if c.kind == "E"]
    m_by_q = {c.q0: c for c in pattern.cmds if c.kind == "M"}
    corr = [c for c in pattern.cmds if c.kind in ("X", "Z")]
    used = [False] * len(e_cmds)
    e_of = {}
    for i, c in enumerate(e_cmds):
        e_of.setdefault(c.q0, []).append(i)
        e_of.setdefault(c.q1, []).append(i)
    out = []

    def prep(q):
        if q not in prepared:
            out.append(Cmd("N", q))
            prepared.add(q)

    for v in order:
        for i in e_of.get(v, []):
            c = e_cmds[i]
            if not used[i]:
                prep(c.q0)
                prep(c.q1)
                out.append(c)
                used[i] = True
        prep(v)
        out.append(m_by_q[v])
    for i, c in enumerate(e_cmds):
        if not used[i]:
            prep(c.q0)
            prep(c.q1)
            out.append(c)
    for o in pattern.outputs:
        prep(o)
    out.extend(corr)
    return pattern.with_cmds(out)


def single_array_peak(pattern) -> int:
    """Peak number of live qubits (prepared and not yet measured) over the
    command sequence, with each qubit prepared just before the first command
    that touches it; this is the width of one state array holding every live
    qubit, counted at each command after any preparation it needs."""
    live = set(pattern.inputs)
    peak = len(live)
    for c in pattern.cmds:
        if c.kind == "N":
            continue
        qs = [c.q0] + ([c.q1] if c.kind == "E" else [])
        live.update(qs)
        peak = max(peak, len(live))
        if c.kind == "M":
            live.discard(c.q0)
    live.update(pattern.outputs)
    return max(peak, len(live))
