"""Seeded synthetic workloads (the paper's benchmark circuits are not
available; these stand in for them with the same structure).

  small_random      random 3-wire J/CZ circuit of depth 10 (30 J + 10 CZ,
                    33 pattern qubits), random normalised input, forced
                    seeded outcomes.  Stands in for the small circuits of
                    Table II.
  brickwork         brickwork cluster rows x cols (28 x 40 at full size),
                    angles k pi/4, |+>^rows input, forced seeded outcomes.
                    Stands in for the cluster-state case of Section 4.6.
  qft               QFT-shaped J/CZ pattern on n logical qubits (24 at full
                    size), random normalised input.  Stands in for the QFT
                    rows of Table II.
  random_batch      uneven random J/CZ patterns for batched recognition.
  brickwork_readout the brickwork with (some of) its outputs measured in
                    seeded random bases: no gflow, sampled-outcome workloads.
  measured_inputs   a random product input measured qubit by qubit.
  chain_measurements inputs measured one by one, each pass preparing a qubit
                    that is (mostly) not joined to the measured one: pass
                    groups whose probabilities are not 1/2.
"""
from __future__ import annotations

import math

from dataclasses import dataclass
from typing import List, Optional

import numpy as np

from .patterns import (E, M, N, Pattern, brickwork_circuit, circuit_to_pattern, qft_circuit,
                       random_jcz_circuit)
from .rng import SplitMix64, pattern_rng, random_state


@dataclass
class Workload:
    pattern: Pattern
    psi_in: Optional[np.ndarray]      # None means |+> on every input
    outcomes: np.ndarray              # forced outcome per M command (command order)
    name: str


def forced_outcomes(pattern: Pattern, rng: SplitMix64) -> np.ndarray:
    return rng.bits(pattern.K)


def small_random(pattern_index: int = 0, nwires: int = 3, depth: int = 10) -> Workload:
    rng = pattern_rng(0, pattern_index)
    gates = random_jcz_circuit(nwires, depth, rng, cz_per_layer=1)
    p = circuit_to_pattern(nwires, gates, f"random{nwires}x{depth}")
    psi = random_state(rng, nwires)
    out = forced_outcomes(p, rng)
    return Workload(p, psi, out, p.name)


def brickwork(rows: int = 28, cols: int = 40, pattern_index: int = 0) -> Workload:
    rng = pattern_rng(1, pattern_index)
    gates, _ = brickwork_circuit(rows, cols, rng)
    p = circuit_to_pattern(rows, gates, f"brickwork{rows}x{cols}")
    out = forced_outcomes(p, rng)
    return Workload(p, None, out, p.name)


def joined_bricks(rows: int, cols: int, copies: int = 2, pattern_index: int = 0) -> Workload:
    """`copies` brickwork circuits of rows x cols on disjoint blocks of wires,
    then one CZ joining the last wire of each block to the first wire of the
    next and a J layer on those wires: |+> inputs, so the blocks stay
    separate sub-states (Section 4.1) until the joining E.  Forced seeded
    outcomes."""
    rng = pattern_rng(5, pattern_index)
    gates = []
    for b in range(copies):
        g, _ = brickwork_circuit(rows, cols, rng)
        for gate in g:
            if gate[0] == "CZ":
                gates.append(("CZ", gate[1] + b * rows, gate[2] + b * rows))
            else:
                gates.append(("J", gate[1] + b * rows, gate[2]))
    for b in range(copies - 1):
        u, v = b * rows + rows - 1, (b + 1) * rows
        gates.append(("CZ", u, v))
        gates.append(("J", u, 2.0 * math.pi * rng.uniform()))
        gates.append(("J", v, 2.0 * math.pi * rng.uniform()))
    p = circuit_to_pattern(rows * copies, gates, f"joined_bricks{copies}x{rows}x{cols}")
    out = forced_outcomes(p, rng)
    return Workload(p, None, out, p.name)


def brickwork_readout(rows: int, cols: int, kept: int = 0, pattern_index: int = 0,
                      with_input: bool = False) -> Workload:
    """The brickwork rows x cols with its output wires kept..rows-1 measured
    as well, each at a seeded random angle in [0, 2 pi): the corrections X^s
    Z^t the flow pattern puts on such an output become that measurement's s-
    and t-domains (X^s before M_a gives the angle (-1)^s a, Z^t gives a + t pi,
    Eq. 2), and the measurements follow all the others.  Outputs: wires
    0..kept-1.  With fewer outputs than inputs the open graph has no gflow,
    so these last measurements' probabilities are not 1/2 (Section 4.5); the
    rest of the pattern is the flow pattern, whose probabilities are 1/2.
    |+> inputs unless with_input (a random normalised state)."""
    if not 0 <= kept <= rows:
        raise ValueError("kept must lie in [0, rows]")
    rng = pattern_rng(6, pattern_index)
    gates, _ = brickwork_circuit(rows, cols, rng)
    base = circuit_to_pattern(rows, gates, "")
    measured_out = set(base.outputs[kept:])
    xdom = {c.q0: c.sdom for c in base.cmds if c.kind == "X"}
    zdom = {c.q0: c.sdom for c in base.cmds if c.kind == "Z"}
    cmds = [c for c in base.cmds if c.kind in ("N", "E", "M")]
    for q in base.outputs[kept:]:
        cmds.append(M(q, 2.0 * math.pi * rng.uniform(), xdom.get(q, ()), zdom.get(q, ())))
    cmds += [c for c in base.cmds if c.kind in ("X", "Z") and c.q0 not in measured_out]
    p = Pattern(base.nqubits, list(base.inputs), base.outputs[:kept], cmds, f"brickwork_readout{rows}x{cols}k{kept}",
                list(gates), rows)
    psi = random_state(rng, rows) if with_input else None
    out = forced_outcomes(p, rng)
    return Workload(p, psi, out, p.name)


def measured_inputs(n: int, kept: int = 2, pattern_index: int = 0) -> Workload:
    """n input qubits, every one but the last `kept` measured directly at a
    seeded random angle (no E, no N): with a random product input, each
    probability is |<+_a|psi_q>|^2, far from 1/2 in general.  Outputs: the
    last `kept` inputs."""
    rng = pattern_rng(7, pattern_index)
    cmds = [M(q, 2.0 * math.pi * rng.uniform()) for q in range(n - kept)]
    p = Pattern(n, list(range(n)), list(range(n - kept, n)), cmds, f"measured_inputs{n}k{kept}")
    psi = np.ones(1, dtype=np.complex128)
    for q in range(n):   # bit q of the index is qubit q: kron puts the last factor lowest
        v = random_state(rng, 1)
        psi = np.kron(v, psi)
    out = forced_outcomes(p, rng)
    return Workload(p, psi, out, p.name)


def chain_measurements(n: int, k: int, joined_every: int = 0, pattern_index: int = 0) -> Workload:
    """n input qubits in a random normalised state; k passes, pass j measuring
    input j (at a seeded random angle) after E(j, j+1) and preparing qubit
    n + j.  The prepared qubit gets E(j, n + j) once where joined_every > 0
    and j % joined_every == 0, and twice (the identity: an E is its own
    inverse) elsewhere, so most passes prepare a qubit that stays unentangled
    and their probabilities are not 1/2 (Section 4.5 does not apply).
    Outputs: inputs k..n-1 and the prepared qubits."""
    if not 1 <= k < n:
        raise ValueError("need 1 <= k < n")
    rng = pattern_rng(8, pattern_index)
    cmds = []
    for j in range(k):
        cmds.append(N(n + j))
        cmds.append(E(j, j + 1))
        cmds.append(E(j, n + j))
        if not (joined_every and j % joined_every == 0):
            cmds.append(E(j, n + j))
        cmds.append(M(j, 2.0 * math.pi * rng.uniform()))
    p = Pattern(n + k, list(range(n)), list(range(k, n)) + [n + j for j in range(k)], cmds,
                f"chain{n}x{k}j{joined_every}")
    psi = random_state(rng, n)
    out = forced_outcomes(p, rng)
    return Workload(p, psi, out, p.name)


def qft(n: int = 24, pattern_index: int = 0, with_input: bool = True) -> Workload:
    rng = pattern_rng(2, pattern_index)
    p = circuit_to_pattern(n, qft_circuit(n), f"qft{n}")
    psi = random_state(rng, n) if with_input else None
    out = forced_outcomes(p, rng)
    return Workload(p, psi, out, p.name)


def random_pattern(i: int, wmin: int, wmax: int, dmin: int, dmax: int, config_index: int,
                   with_input: bool = True) -> Workload:
    """Pattern i of an uneven random J/CZ set (seeded from config seed XOR i):
    width uniform in [wmin, wmax], depth uniform in [dmin, dmax], ceil(width/4)
    CZ pairs per layer; the random input state is drawn only if asked for."""
    rng = pattern_rng(config_index, i)
    n = wmin + rng.randint(wmax - wmin + 1)
    d = dmin + rng.randint(dmax - dmin + 1)
    gates = random_jcz_circuit(n, d, rng, cz_per_layer=max(1, (n + 3) // 4))
    p = circuit_to_pattern(n, gates, f"rand{n}x{d}#{i}")
    psi = random_state(rng, n) if with_input else None
    out = forced_outcomes(p, rng)
    return Workload(p, psi, out, p.name)


def random_batch(count: int = 256, wmin: int = 6, wmax: int = 14, dmin: int = 10, dmax: int = 40,
                 config_index: int = 3, start: int = 0, with_input: bool = True) -> List[Workload]:
    """Patterns start .. start+count-1 of the uneven random J/CZ set."""
    return [random_pattern(i, wmin, wmax, dmin, dmax, config_index, with_input)
            for i in range(start, start + count)]
