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
"""
from __future__ import annotations

import math

from dataclasses import dataclass
from typing import List, Optional

import numpy as np

from .patterns import (Pattern, brickwork_circuit, circuit_to_pattern, qft_circuit,
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
