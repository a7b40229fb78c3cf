"""Measurement-pattern data model and J/CZ circuit-to-pattern generator.

A pattern is P = (V, I, O, A) (Section 2.2): qubits V = {0, ..., nqubits-1},
inputs I, outputs O and the command sequence A.  Here `cmds` lists the
commands in EXECUTION order (cmds[0] acts first), i.e. the paper's
right-to-left notation read from the right.

Command kinds (Section 2.2):
  N v          prepare v in |+>
  E u v        CZ on u and v
  M v a s t    measure v at angle a with signal domains s (s-signal) and
               t (t-signal): the actual angle is (-1)^s a + t pi (Eq. 2)
  X v s        Pauli X on v if the parity of outcomes in s is 1
  Z v s        Pauli Z on v if the parity of outcomes in s is 1

The generator turns a circuit of J(alpha) and CZ gates into the standard-form
(CME) pattern given by the causal flow f(i) = next qubit on the same wire: the
J(alpha) gate on a wire is the pattern N_j E_ij M_i^{-alpha} X_j^{s_i}, and the
corrections of a flow pattern, pushed through to the measurements, become the
s- and t-domains (the pattern used in Eqs. 22-23 is of this family).  The
paper extracts its benchmark patterns the same way from J/CZ circuits
(Section 5); the extraction references are not reproduced, only the flow
construction.  This module builds inputs; it does not simulate anything.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Sequence, Tuple

from .rng import SplitMix64

KINDS = ("N", "E", "M", "X", "Z")


@dataclass
class Cmd:
    kind: str
    q0: int
    q1: int = -1
    angle: float = 0.0
    sdom: Tuple[int, ...] = ()
    tdom: Tuple[int, ...] = ()

    def __post_init__(self):
        if self.kind not in KINDS:
            raise ValueError(f"bad command kind {self.kind!r}")
        self.sdom = tuple(int(x) for x in self.sdom)
        self.tdom = tuple(int(x) for x in self.tdom)


def N(v):
    return Cmd("N", v)


def E(u, v):
    return Cmd("E", u, v)


def M(v, angle, sdom=(), tdom=()):
    return Cmd("M", v, -1, float(angle), tuple(sdom), tuple(tdom))


def X(v, dom=()):
    return Cmd("X", v, -1, 0.0, tuple(dom))


def Z(v, dom=()):
    return Cmd("Z", v, -1, 0.0, tuple(dom))


@dataclass
class Pattern:
    nqubits: int
    inputs: List[int]
    outputs: List[int]
    cmds: List[Cmd]
    name: str = ""
    # optional circuit the pattern was built from (for textbook checks)
    circuit: list = field(default_factory=list)
    nwires: int = 0

    def measured(self) -> List[int]:
        """Measured qubits in command order."""
        return [c.q0 for c in self.cmds if c.kind == "M"]

    @property
    def K(self) -> int:
        return sum(1 for c in self.cmds if c.kind == "M")

    def edges(self) -> List[Tuple[int, int]]:
        return [(c.q0, c.q1) for c in self.cmds if c.kind == "E"]

    def with_cmds(self, cmds: Sequence[Cmd], name: str | None = None) -> "Pattern":
        return Pattern(self.nqubits, list(self.inputs), list(self.outputs), list(cmds),
                       self.name if name is None else name, list(self.circuit), self.nwires)

    def is_standard(self) -> bool:
        """True if the execution order is N*, E*, M*, then X/Z (CME form)."""
        rank = {"N": 0, "E": 0, "M": 1, "X": 2, "Z": 2}
        last = 0
        for c in self.cmds:
            r = rank[c.kind]
            if r < last:
                return False
            last = r
        return True


# ---------------------------------------------------------------------------
# circuits of J(alpha) and CZ gates
#   gate ("J", wire, alpha) applies J(alpha) = (1/sqrt2)[[1, e^{i alpha}],
#   [1, -e^{i alpha}]]; gate ("CZ", a, b) applies CZ.  Listed in time order.
# ---------------------------------------------------------------------------

def circuit_to_pattern(nwires: int, gates: Sequence[tuple], name: str = "") -> Pattern:
    """Standard-form flow pattern of a J/CZ circuit.

    Input qubit k is wire k; output qubit k is the last qubit of wire k, so
    bit k of the input and output vectors is wire k.
    """
    cur = list(range(nwires))
    nxt = nwires
    edge_set: dict = {}
    flow: dict = {}
    meas_angle: dict = {}
    order: List[int] = []

    def toggle(a, b):
        key = (min(a, b), max(a, b))
        if key in edge_set:
            del edge_set[key]
        else:
            edge_set[key] = True

    for g in gates:
        if g[0] == "J":
            w, alpha = int(g[1]), float(g[2])
            i, j = cur[w], nxt
            nxt += 1
            toggle(i, j)
            flow[i] = j
            meas_angle[i] = -alpha
            order.append(i)
            cur[w] = j
        elif g[0] == "CZ":
            a, b = int(g[1]), int(g[2])
            if a == b:
                raise ValueError("CZ needs two different wires")
            toggle(cur[a], cur[b])
        else:
            raise ValueError(f"unknown gate {g[0]!r}")

    nq = nxt
    adj = [set() for _ in range(nq)]
    for (a, b) in edge_set:
        adj[a].add(b)
        adj[b].add(a)
    pos = {q: k for k, q in enumerate(order)}
    sdom = {q: [] for q in range(nq)}
    tdom = {q: [] for q in range(nq)}
    for i in order:
        fi = flow[i]
        sdom[fi].append(i)
        for k in sorted(adj[fi]):
            if k != i:
                tdom[k].append(i)
    for q in range(nq):
        for d in sdom[q] + tdom[q]:
            if q in pos and pos[d] >= pos[q]:
                raise AssertionError("flow order violated")  # cannot happen for circuits

    inputs = list(range(nwires))
    outputs = list(cur)
    cmds: List[Cmd] = [N(v) for v in range(nwires, nq)]
    cmds += [E(a, b) for (a, b) in edge_set]
    cmds += [M(i, meas_angle[i], sorted(sdom[i], key=pos.get), sorted(tdom[i], key=pos.get)) for i in order]
    for o in outputs:
        if tdom[o]:
            cmds.append(Z(o, sorted(tdom[o], key=pos.get)))
    for o in outputs:
        if sdom[o]:
            cmds.append(X(o, sorted(sdom[o], key=pos.get)))
    p = Pattern(nq, inputs, outputs, cmds, name, list(gates), nwires)
    return p


def random_jcz_circuit(nwires: int, depth: int, rng: SplitMix64, cz_per_layer: int = 1) -> list:
    """Each layer: J(alpha) on every wire, alpha uniform in [0, 2pi), then CZ
    on `cz_per_layer` disjoint wire pairs chosen uniformly."""
    gates = []
    for _ in range(depth):
        for w in range(nwires):
            gates.append(("J", w, 2.0 * math.pi * rng.uniform()))
        free = list(range(nwires))
        for _ in range(min(cz_per_layer, nwires // 2)):
            a = free.pop(rng.randint(len(free)))
            b = free.pop(rng.randint(len(free)))
            gates.append(("CZ", a, b))
    return gates


def brickwork_vertical(r: int, c: int) -> bool:
    """Vertical edge (r,c)-(r+1,c) of this project's brickwork layout."""
    m = c % 8
    if m in (2, 4) and r % 2 == 0:
        return True
    if m in (6, 0) and c > 0 and r % 2 == 1:
        return True
    return False


def brickwork_circuit(rows: int, cols: int, rng: SplitMix64) -> Tuple[list, dict]:
    """Brickwork cluster of rows x cols qubits as a J/CZ circuit.

    Qubit (r, c) has measurement angle k*pi/4, k uniform in 0..7; measuring it
    at angle beta is J(-beta) on wire r.  Vertical edges of column c are the
    CZ gates applied while column c is current.  Returns (gates, angles).
    """
    gates = []
    angles = {}
    for c in range(cols):
        for r in range(rows - 1):
            if brickwork_vertical(r, c):
                gates.append(("CZ", r, r + 1))
        if c == cols - 1:
            break
        for r in range(rows):
            k = rng.randint(8)
            beta = k * math.pi / 4.0
            angles[(r, c)] = beta
            gates.append(("J", r, -beta))
    return gates, angles


def qft_circuit(n: int) -> list:
    """Quantum Fourier transform on n wires (no final swaps) in J/CZ gates.

    H = J(0); CP(phi) = P_c(phi/2) CNOT P_t(-phi/2) CNOT P_t(phi/2) with
    P(phi) = J(0) J(phi) and CNOT = (I x J(0)) CZ (I x J(0)).
    """
    gates = []

    def P(w, phi):
        gates.append(("J", w, phi))
        gates.append(("J", w, 0.0))

    def CNOT(c, t):
        gates.append(("J", t, 0.0))
        gates.append(("CZ", c, t))
        gates.append(("J", t, 0.0))

    for i in range(n):
        gates.append(("J", i, 0.0))
        for j in range(i + 1, n):
            phi = math.pi / (1 << (j - i))
            c, t = j, i
            P(t, phi / 2)
            CNOT(c, t)
            P(t, -phi / 2)
            CNOT(c, t)
            P(c, phi / 2)
    return gates
