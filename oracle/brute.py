"""O-B: brute-force full-register simulation (oracle; test infrastructure
only).  For tiny patterns (|V| up to about 14).

No qubit elimination and no reordering: one 2^|V| tensor with an axis per
qubit label.  Every non-input qubit starts in |+> (N commutes with every
command on other qubits, and D2 forbids acting on v before N_v).  Commands run
in the given order:
  E      CZ: negate where both bits are 1;
  X, Z   Pauli when the signal parity is 1;
  M      the projective measurement of Section 2.3 with
         P_s = |+-theta><+-theta| (Eqs. 9-10), theta from Eq. 2:
         prob_s = <psi|P_s|psi> (Eq. 3), psi -> P_s psi / sqrt(prob_s) (Eq. 4).
         In EOWQS mode the probability is taken as 1/2, also for a sampled
         outcome.
The measured qubit stays in the register in state |+-theta>; at the end it is
contracted with <+-theta| to read the state of the outputs.
"""
from __future__ import annotations

import math
from typing import Dict, Optional

import numpy as np

from owqs_inputs.rng import SplitMix64

from .basis import PatternError, ket_pm, resolved_angle, signal_parity, validate


def run(pattern, psi_in: Optional[np.ndarray] = None, outcomes=None, mode: str = "owqs",
        policy: str = "forced", seed: int = 0, max_qubits: int = 16):
    validate(pattern)
    n = pattern.nqubits
    if n > max_qubits:
        raise ValueError(f"brute force limited to {max_qubits} qubits")
    I = list(pattern.inputs)
    # state over the inputs: C-order axis a is bit |I|-1-a
    if I:
        if psi_in is None:
            vin = np.full(1 << len(I), 2.0 ** (-len(I) / 2.0), dtype=np.complex128)
        else:
            vin = np.array(psi_in, dtype=np.complex128).reshape(-1)
            if mode == "owqs":
                vin = vin / np.linalg.norm(vin)
        tin = vin.reshape([2] * len(I))
        in_axes = [I[len(I) - 1 - a] for a in range(len(I))]
    else:
        # no input qubit: a one-amplitude input multiplies the whole state
        tin = np.array(1.0 + 0j)
        if psi_in is not None:
            c = complex(np.asarray(psi_in, dtype=np.complex128).reshape(-1)[0])
            tin = np.array(c / abs(c) if mode == "owqs" else c)
        in_axes = []
    # full register: axis q <-> label q
    others = [q for q in range(n) if q not in I]
    plus = np.array([1.0, 1.0], dtype=np.complex128) / math.sqrt(2.0)
    t = tin
    axes = list(in_axes)
    for q in others:
        t = np.multiply.outer(t, plus)
        axes.append(q)
    perm = [axes.index(q) for q in range(n)]
    T = np.transpose(t, perm).copy()

    rng = SplitMix64(seed)
    meas: Dict[int, int] = {}
    theta: Dict[int, float] = {}
    probs: Dict[int, float] = {}
    for c in pattern.cmds:
        if c.kind == "N":
            continue
        if c.kind == "E":
            idx = [slice(None)] * n
            idx[c.q0] = 1
            idx[c.q1] = 1
            T[tuple(idx)] *= -1.0
        elif c.kind in ("X", "Z"):
            if signal_parity(meas, c.sdom):
                if c.kind == "X":
                    T = np.flip(T, axis=c.q0).copy()
                else:
                    idx = [slice(None)] * n
                    idx[c.q0] = 1
                    T[tuple(idx)] *= -1.0
        else:
            v = c.q0
            th = resolved_angle(c.angle, signal_parity(meas, c.sdom), signal_parity(meas, c.tdom))
            norm2 = float(np.vdot(T, T).real)
            proj = []
            p = []
            for s in (0, 1):
                k = ket_pm(th, s)
                P = np.outer(k, k.conj())
                Ts = np.moveaxis(np.tensordot(P, T, axes=([1], [v])), 0, v)
                proj.append(Ts)
                p.append(float(np.vdot(Ts, Ts).real) / norm2)
            if policy == "forced":
                s = int(outcomes[v]) & 1
            elif policy == "zero":
                s = 0
            else:  # EOWQS draws against the 1/2 of Section 4.5
                s = 0 if rng.uniform() <= (p[0] if mode == "owqs" else 0.5) else 1
            if mode == "owqs":
                if p[s] <= 0.0:
                    raise PatternError("forced outcome has probability 0")
                T = proj[s] / math.sqrt(p[s])
            else:
                T = proj[s] * math.sqrt(2.0)
            meas[v] = s
            theta[v] = th
            probs[v] = p[s]
    # contract measured qubits with <+-theta|, highest label first so the
    # remaining axes keep their relative order
    labels = list(range(n))
    for v in sorted(meas, reverse=True):
        bra = ket_pm(theta[v], meas[v]).conj()
        T = np.tensordot(bra, T, axes=([0], [labels.index(v)]))
        labels.remove(v)
    O = list(pattern.outputs)
    if not O:
        return np.array([complex(T)]), meas, probs
    perm = [labels.index(O[len(O) - 1 - a]) for a in range(len(O))]
    return np.transpose(T, perm).reshape(-1).copy(), meas, probs
