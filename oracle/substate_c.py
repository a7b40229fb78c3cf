"""ctypes front end of oracle/substate_omp.c: O-A in plain C, its loops over
the amplitude index shared among the host cores by OpenMP (oracle; test
infrastructure only, like the rest of this package).

The C file is the same algorithm as oracle/substate.py, step for step
(Section 4: sub-states merged only by E, N as |+>, E/X/Z as sign flips and
half exchanges, M with Eqs. 2 and 11-13 and elimination); this module only
builds it (gcc -fopenmp) and passes a pattern to it as flat arrays.  It is
what times the CPU baseline on every host core, and it serves GPU parity
tests at sizes where the numpy oracle takes minutes.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from typing import Dict, Optional

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "substate_omp.c")
LIB = os.path.join(HERE, "libsubstate_omp.so")
KIND = {"N": 0, "E": 1, "M": 2, "X": 3, "Z": 4}
STATUS = {0: "ok", 1: "pattern error", 2: "out of memory", 3: "forced outcome of probability 0",
          4: "sub-state wider than 62 qubits"}

_lib = None


def build() -> str:
    """Compile the C oracle (host code only: no GPU, no CUDA)."""
    tmp = LIB + ".tmp"
    subprocess.run(["gcc", "-O2", "-std=c99", "-fopenmp", "-fPIC", "-shared", SRC, "-o", tmp, "-lm"],
                   check=True, capture_output=True, text=True)
    os.replace(tmp, LIB)
    return LIB


def library():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
            build()
        lib = C.CDLL(LIB)
        i32p = C.POINTER(C.c_int32)
        dp = C.POINTER(C.c_double)
        lib.oa_run.restype = C.c_int
        lib.oa_run.argtypes = [C.c_int, i32p, C.c_int, i32p, C.c_int, C.c_int, i32p, i32p, i32p, dp,
                               i32p, i32p, i32p, i32p, i32p, dp, C.POINTER(C.c_uint8), C.c_int, C.c_int,
                               dp, dp, C.c_int, C.POINTER(C.c_int)]
        lib.oa_max_threads.restype = C.c_int
        _lib = lib
    return _lib


def max_threads() -> int:
    """Threads an OpenMP region gets by default (the host cores)."""
    return int(library().oa_max_threads())


class Result:
    def __init__(self):
        self.psi_out: Optional[np.ndarray] = None
        self.probs: Dict[int, float] = {}
        self.peak_substate = 0


def _i32(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.int32).reshape(-1)) if len(a) else np.zeros(1, np.int32)


def run(pattern, psi_in: Optional[np.ndarray] = None, outcomes=None, mode: str = "owqs", policy: str = "forced",
        stop_after: int = 0, threads: int = 0, want_output: bool = True) -> Result:
    """As oracle.substate.run for forced and zero outcomes.  outcomes:
    forced outcome per qubit label (indexable by label).  stop_after > 0
    returns after that many measurements, without an output."""
    if mode not in ("owqs", "eowqs") or policy not in ("forced", "zero"):
        raise ValueError("the C oracle takes OWQS or EOWQS with forced or zero outcomes")
    n = pattern.nqubits
    cmds = pattern.cmds
    kind = _i32([KIND[c.kind] for c in cmds])
    q0 = _i32([c.q0 for c in cmds])
    q1 = _i32([c.q1 for c in cmds])
    angle = np.ascontiguousarray([float(c.angle) for c in cmds] or [0.0], dtype=np.float64)
    dom, soff, slen, toff, tlen = [], [], [], [], []
    for c in cmds:
        soff.append(len(dom)); slen.append(len(c.sdom)); dom += list(c.sdom)
        toff.append(len(dom)); tlen.append(len(c.tdom)); dom += list(c.tdom)
    dom, soff, slen, toff, tlen = _i32(dom), _i32(soff), _i32(slen), _i32(toff), _i32(tlen)
    ins, outs = _i32(pattern.inputs), _i32(pattern.outputs)
    pin = None
    if psi_in is not None:
        pin = np.ascontiguousarray(np.asarray(psi_in, dtype=np.complex128).reshape(-1)).view(np.float64)
    oc = None
    if policy == "forced":
        oc = np.zeros(max(1, n), dtype=np.uint8)
        for q in range(n):
            try:
                oc[q] = int(outcomes[q]) & 1
            except (KeyError, IndexError, TypeError):
                oc[q] = 0
    nout = len(pattern.outputs)
    pout = np.zeros(2 << nout, dtype=np.float64) if (want_output and stop_after <= 0) else None
    probs = np.zeros(max(1, n), dtype=np.float64)
    peak = C.c_int(0)
    P = lambda a: a.ctypes.data_as(C.POINTER(C.c_int32))  # noqa: E731
    D = lambda a: a.ctypes.data_as(C.POINTER(C.c_double)) if a is not None else None  # noqa: E731
    st = library().oa_run(n, P(ins), len(pattern.inputs), P(outs), nout, len(cmds), P(kind), P(q0), P(q1),
                          D(angle), P(soff), P(slen), P(toff), P(tlen), P(dom), D(pin),
                          oc.ctypes.data_as(C.POINTER(C.c_uint8)) if oc is not None else None,
                          0 if mode == "owqs" else 1, int(stop_after), D(pout), D(probs), int(threads),
                          C.byref(peak))
    if st != 0:
        raise RuntimeError(f"C oracle: {STATUS.get(st, st)}")
    res = Result()
    if pout is not None:
        res.psi_out = pout.view(np.complex128).copy()
    measured = {c.q0 for c in cmds if c.kind == "M"}
    res.probs = {q: float(probs[q]) for q in measured}
    res.peak_substate = peak.value
    return res
