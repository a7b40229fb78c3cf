"""Measurement basis, measurement operators, signal-dependent angles and
well-formedness rules of a one-way-QC pattern (oracle; test infrastructure).

Reading of Eq. 1: the paper prints |+-a> = (|0> +- e^{-ia}|1>)/sqrt2, but its
projectors (Eqs. 9-10), its generalised operators (Eqs. 11-12) and the
R_z(-a)-then-H derivation (Section 4.2) all need |+-a> = (|0> +- e^{+ia}|1>)/sqrt2.
The oracle uses e^{+ia}; then <+a|psi> = (psi0 + e^{-ia} psi1)/sqrt2.
"""
from __future__ import annotations

import math

import numpy as np

SQRT2 = math.sqrt(2.0)


def ket_pm(alpha: float, s: int) -> np.ndarray:
    """|+alpha> (s=0) or |-alpha> (s=1) as a length-2 vector."""
    sign = 1.0 if s == 0 else -1.0
    return np.array([1.0, sign * np.exp(1j * alpha)], dtype=np.complex128) / SQRT2


def projector(alpha: float, s: int) -> np.ndarray:
    """P_s = |+-alpha><+-alpha| (Eqs. 9-10)."""
    k = ket_pm(alpha, s)
    return np.outer(k, k.conj())


def gen_operator(alpha: float, s: int) -> np.ndarray:
    """M_0 = |0><+alpha|, M_1 = |1><-alpha| (Eqs. 11-12): the measured qubit
    collapses to |s> so it can be dropped (Section 4.2)."""
    ket_s = np.zeros(2, dtype=np.complex128)
    ket_s[s] = 1.0
    return np.outer(ket_s, ket_pm(alpha, s).conj())


def signal_parity(outcomes, domain) -> int:
    """Sum modulo 2 of the outcomes of the qubits in `domain` (Section 2.2)."""
    p = 0
    for q in domain:
        p ^= int(outcomes[q])
    return p


def resolved_phase(alpha: float, s: int, t: int) -> complex:
    """e^{-i theta} for theta = (-1)^s alpha + t pi (Eq. 2).

    The t pi part is applied as an exact sign rather than by adding pi in
    floating point: e^{-i theta} = (-1)^t (cos a - i (-1)^s sin a).
    """
    c, sn = math.cos(alpha), math.sin(alpha)
    e = complex(c, -sn) if s == 0 else complex(c, sn)
    return -e if t else e


def resolved_angle(alpha: float, s: int, t: int) -> float:
    """theta itself, (-1)^s alpha + t pi (Eq. 2)."""
    return (-alpha if s else alpha) + (math.pi if t else 0.0)


class PatternError(ValueError):
    pass


def validate(pattern) -> None:
    """Well-formedness rules D0-D3 (Section 2.2) plus basic sanity.

    Non-input qubits without an explicit N are taken as prepared before the
    first command (N commutes with every command on other qubits).
    """
    n = pattern.nqubits
    I, O = list(pattern.inputs), list(pattern.outputs)
    for q in I + O:
        if not (0 <= q < n):
            raise PatternError(f"qubit {q} out of range")
    if len(set(I)) != len(I) or len(set(O)) != len(O):
        raise PatternError("duplicate input or output qubit")
    explicit_n = {c.q0 for c in pattern.cmds if c.kind == "N"}
    prepared = set(I) | (set(range(n)) - set(I) - explicit_n)
    measured = set()
    seen_n = set()
    for idx, c in enumerate(pattern.cmds):
        qs = [c.q0] + ([c.q1] if c.kind == "E" else [])
        for q in qs:
            if not (0 <= q < n):
                raise PatternError(f"command {idx}: qubit {q} out of range")
        if c.kind == "E" and c.q0 == c.q1:
            raise PatternError(f"command {idx}: E on a single qubit")
        for q in tuple(c.sdom) + tuple(c.tdom):
            if not (0 <= q < n):
                raise PatternError(f"command {idx}: domain qubit {q} out of range")
            if q not in measured:                                    # D0
                raise PatternError(f"command {idx}: depends on unmeasured qubit {q}")
        for q in qs:
            if q in measured:                                        # D1
                raise PatternError(f"command {idx}: acts on measured qubit {q}")
        if c.kind == "N":
            if c.q0 in I or c.q0 in seen_n:
                raise PatternError(f"command {idx}: N on an input or prepared qubit")
            seen_n.add(c.q0)
            prepared.add(c.q0)
            continue
        for q in qs:
            if q not in prepared:                                    # D2
                raise PatternError(f"command {idx}: acts on unprepared qubit {q}")
        if c.kind == "M":
            measured.add(c.q0)
    for q in range(n):                                               # D3
        if (q in measured) == (q in O):
            raise PatternError(f"qubit {q}: measured iff not an output is violated")
