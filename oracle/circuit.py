"""Textbook unitaries of J(alpha)/CZ circuits by dense matrix products
(oracle; test infrastructure only).

J(alpha) = (1/sqrt2) [[1, e^{i alpha}], [1, -e^{i alpha}]] is the gate the
one-qubit pattern N_2 E_12 M_1^{-alpha} X_2^{s_1} implements; CZ and CNOT are
the matrices printed in Section 2.1.  Bit k of a basis index is wire k.
"""
from __future__ import annotations

import cmath
import math

import numpy as np

CZ = np.diag([1, 1, 1, -1]).astype(np.complex128)
CNOT = np.array([[1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 0, 1], [0, 0, 1, 0]], dtype=np.complex128)
H = np.array([[1, 1], [1, -1]], dtype=np.complex128) / math.sqrt(2.0)


def J(alpha: float) -> np.ndarray:
    e = cmath.exp(1j * alpha)
    return np.array([[1, e], [1, -e]], dtype=np.complex128) / math.sqrt(2.0)


def embed_1q(g: np.ndarray, wire: int, n: int) -> np.ndarray:
    """Full 2^n matrix of a one-qubit gate on `wire` (bit `wire` of the index)."""
    m = np.array([[1.0 + 0j]])
    for w in range(n - 1, -1, -1):          # kron: leftmost factor is the top bit
        m = np.kron(m, g if w == wire else np.eye(2))
    return m


def embed_cz(a: int, b: int, n: int) -> np.ndarray:
    d = np.ones(1 << n, dtype=np.complex128)
    for x in range(1 << n):
        if (x >> a) & 1 and (x >> b) & 1:
            d[x] = -1
    return np.diag(d)


def circuit_unitary(nwires: int, gates) -> np.ndarray:
    """Product of the gate matrices, first gate rightmost."""
    U = np.eye(1 << nwires, dtype=np.complex128)
    for g in gates:
        if g[0] == "J":
            U = embed_1q(J(g[2]), g[1], nwires) @ U
        elif g[0] == "CZ":
            U = embed_cz(g[1], g[2], nwires) @ U
        else:
            raise ValueError(g[0])
    return U


def apply_circuit(nwires: int, gates, vec: np.ndarray) -> np.ndarray:
    """The circuit applied to one state vector, gate by gate (first gate
    first), without forming any 2^n x 2^n matrix: a J on wire w mixes the
    amplitude pairs that differ in bit w with the 2x2 matrix; a CZ negates
    the amplitudes whose two bits are 1.  For widths where the dense product
    is too large."""
    v = np.asarray(vec, dtype=np.complex128).copy()
    idx = np.arange(1 << nwires)
    for g in gates:
        if g[0] == "J":
            w = g[1]
            m = J(g[2])
            lo = idx[((idx >> w) & 1) == 0]
            hi = lo | (1 << w)
            a, b = v[lo].copy(), v[hi].copy()
            v[lo] = m[0, 0] * a + m[0, 1] * b
            v[hi] = m[1, 0] * a + m[1, 1] * b
        elif g[0] == "CZ":
            both = ((idx >> g[1]) & 1) & ((idx >> g[2]) & 1)
            v[both == 1] *= -1
        else:
            raise ValueError(g[0])
    return v


def align_phase(ref: np.ndarray, x: np.ndarray) -> np.ndarray:
    """x multiplied by the unit phase that best aligns it with ref."""
    ov = np.vdot(x, ref)
    if abs(ov) == 0:
        return x
    return x * (ov / abs(ov))
