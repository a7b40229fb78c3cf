"""CPU model of the documented pass contract, used to check the host schedule
compiler without a GPU (test infrastructure; the product never calls it).

A measure pass over extended index k (bits [0, n_in) read from the input,
bits [n_in, n_in + r) new |+> qubits) computes
    x(k)   = (-1)^q(k) in[(k ^ xmask) & (2^n_in - 1)]
    q(k)   = c0 ^ parity(k & zmask) ^ XOR over edges (u, v) of k_u k_v
    out[j] = s_c (x(ins(j, b, 0)) + w1 x(ins(j, b, 1)))
and the final pass out[u] = s_c x(sum_k u_k 2^perm[k]); s_c = scale /
sqrt(norm of the previous array) in OWQS mode, scale in EOWQS mode.
"""
from __future__ import annotations

import math

import numpy as np


def _parity(a: np.ndarray) -> np.ndarray:
    a = a.copy()
    p = np.zeros_like(a)
    while np.any(a):
        p ^= a & np.uint64(1)
        a >>= np.uint64(1)
    return p


def _x(d, vin, k, n_in, virt):
    k = k.astype(np.uint64)
    q = np.full(k.shape, np.uint64(d.c0), dtype=np.uint64)
    q ^= _parity(k & np.uint64(d.zmask))
    for e in range(d.nedges):
        u, v = d.edges[e][0], d.edges[e][1]
        q ^= ((k >> np.uint64(u)) & (k >> np.uint64(v)) & np.uint64(1))
    if virt:
        val = np.full(k.shape, 2.0 ** (-n_in / 2.0), dtype=np.complex128)
    else:
        idx = (k ^ np.uint64(d.xmask)) & np.uint64((1 << n_in) - 1)
        val = vin[idx.astype(np.int64)]
    return np.where(q.astype(bool), -val, val)


def emulate(descs, psi_in, mode="owqs"):
    """Returns (psi_out, probs per measure pass in execution order)."""
    virt = psi_in is None
    cur = None if virt else np.asarray(psi_in, dtype=np.complex128)
    norm_prev = None if virt else float(np.vdot(cur, cur).real)
    probs = []
    for d in descs:
        sc = d.scale
        if mode == "owqs" and norm_prev is not None:
            sc = sc / math.sqrt(norm_prev)
        if d.kind == 0:
            j = np.arange(1 << d.n_out, dtype=np.uint64)
            b = np.uint64(d.b)
            k0 = ((j >> b) << (b + np.uint64(1))) | (j & ((np.uint64(1) << b) - np.uint64(1)))
            k1 = k0 | (np.uint64(1) << b)
            w1 = complex(d.w1re, d.w1im)
            out = sc * (_x(d, cur, k0, d.n_in, virt) + w1 * _x(d, cur, k1, d.n_in, virt))
            norm_prev = float(np.vdot(out, out).real)
            probs.append(norm_prev)
            cur, virt = out, False
        else:
            u = np.arange(1 << d.n_out, dtype=np.uint64)
            k = np.zeros_like(u)
            for i in range(d.n_out):
                k |= ((u >> np.uint64(i)) & np.uint64(1)) << np.uint64(d.perm[i])
            return sc * _x(d, cur, k, d.n_in, virt), probs
    raise ValueError("no final pass")
