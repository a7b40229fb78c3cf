"""O-A: direct sub-state simulator with qubit elimination (oracle; test
infrastructure only).

Follows Section 4 of the paper step by step, in FP64:
  * state representation (Section 4.1): separate sub-states, merged by a
    tensor product only when an E joins them; the input qubits form one
    sub-state (the caller's vector may be entangled);
  * N_v (Section 2.2): a new sub-state |+> = (1, 1)/sqrt2;
  * E_uv (Section 4.4.1, Fig. 5): merge the two sub-states if needed, then
    negate every amplitude whose u and v bits are both 1;
  * X_v^s, Z_v^s (Section 4.4.1): exchange the v=0 and v=1 halves, or negate
    the v=1 half, when the signal is 1;
  * ^t[M_v^a]^s (Eq. 2, Section 4.2, Eqs. 11-13, Fig. 6): with
    theta = (-1)^s a + t pi, the outcome-0 and outcome-1 rows of the
    generalised operators give (psi0 + e^{-i theta} psi1)/sqrt2 and
    (psi0 - e^{-i theta} psi1)/sqrt2 over every pair of amplitudes that differ
    only in bit v; prob_s is the squared norm of that half (Eq. 13); the
    kept half is divided by sqrt(prob_s) (Eq. 7) and qubit v is dropped.
    In EOWQS mode (Section 4.5) every probability is taken as 1/2, so the
    kept half is multiplied by sqrt2 instead and no probability is computed.
A sub-state is a numpy tensor with one axis per qubit, axis k holding the
k-th qubit in ascending label order; flattened, bit k of the index is that
qubit, which is the ordering Fig. 8 prints (|q3 q2>, |q4 q3 q1>).

Probabilities: a sampled outcome is 0 iff u <= prob_0 with u uniform in
[0, 1) from a splitmix64 stream (reading of the `rand(0,1) <= prob` test of
Fig. 6); in EOWQS mode prob_0 is the 1/2 of Section 4.5 there too, so the
draws do not depend on the state.  A scalar left over when a whole sub-state is measured away is a
global factor; it is kept, so results carry the exact branch phase.
"""
from __future__ import annotations

import math
from typing import Callable, Dict, List, Optional

import numpy as np

from owqs_inputs.rng import SplitMix64

from .basis import SQRT2, PatternError, resolved_phase, signal_parity, validate


class SubState:
    __slots__ = ("labels", "tensor")

    def __init__(self, labels: List[int], tensor: np.ndarray):
        self.labels = list(labels)
        self.tensor = tensor

    def axis(self, q: int) -> int:
        return self.labels.index(q)

    def flat(self) -> np.ndarray:
        """Vector with bit k = k-th qubit in ascending label order."""
        n = len(self.labels)
        if n == 0:
            return self.tensor.reshape(1)
        return np.transpose(self.tensor, list(range(n - 1, -1, -1))).reshape(-1).copy()


def plus_substate(v: int) -> SubState:
    return SubState([v], np.array([1.0, 1.0], dtype=np.complex128) / SQRT2)


def from_flat(labels_lsb_first: List[int], vec: np.ndarray) -> SubState:
    """Sub-state from a vector whose bit k is qubit labels_lsb_first[k]."""
    n = len(labels_lsb_first)
    t = np.array(vec, dtype=np.complex128, copy=True).reshape([2] * n if n else ())
    # C order: axis a is bit n-1-a
    axis_qubits = [labels_lsb_first[n - 1 - a] for a in range(n)]
    order = sorted(range(n), key=lambda a: axis_qubits[a])
    return SubState([axis_qubits[a] for a in order], np.transpose(t, order) if n else t)


def kron(a: SubState, b: SubState) -> SubState:
    """Tensor product of two sub-states (Section 4.1)."""
    labels = a.labels + b.labels
    t = np.multiply.outer(a.tensor, b.tensor)
    order = sorted(range(len(labels)), key=lambda k: labels[k])
    return SubState([labels[k] for k in order], np.transpose(t, order))


def to_output(sub: SubState, outputs: List[int]) -> np.ndarray:
    """Vector with bit k = outputs[k]."""
    n = len(outputs)
    if n == 0:
        return sub.tensor.reshape(1).copy()
    # want C-order axes: axis a <-> outputs[n-1-a]
    perm = [sub.labels.index(outputs[n - 1 - a]) for a in range(n)]
    return np.transpose(sub.tensor, perm).reshape(-1).copy()


class Result:
    def __init__(self):
        self.psi_out: Optional[np.ndarray] = None
        self.outcomes: Dict[int, int] = {}
        self.probs: Dict[int, float] = {}
        self.pairs: Dict[int, tuple] = {}
        self.peak_substate = 0
        self.measurements_done = 0


def outcome_probabilities(mode: str, tensor: np.ndarray, half) -> List[float]:
    """[prob_0, prob_1] of a measurement: the squared norms of the two halves
    over the sub-state's (Eq. 13) in OWQS mode; 1/2 each in EOWQS mode
    (Section 4.5), which computes nothing."""
    if mode == "owqs":
        norm2 = float(np.vdot(tensor, tensor).real)
        return [float(np.vdot(h, h).real) / norm2 for h in half]
    return [0.5, 0.5]


def run(pattern, psi_in: Optional[np.ndarray] = None, outcomes=None, mode: str = "owqs",
        policy: str = "forced", seed: int = 0,
        trace: Optional[Callable[[int, object, List[SubState]], None]] = None,
        stop_after: Optional[int] = None, input_factors=None) -> Result:
    """Simulate `pattern` (commands in execution order).

    psi_in   vector over the inputs, bit k = inputs[k]; None = |+> on each.
    outcomes forced outcome per qubit label (indexable by label) when
             policy == "forced"; policy "zero" preselects 0 for every
             measurement (EOWQS, Section 4.5); "sampled" draws them.
    mode     "owqs" (probabilities computed, branch renormalised) or
             "eowqs" (probabilities taken as 1/2).
    input_factors  optional product form of the input: a list of
             (qubits, vector) pairs, vector bit k = qubits[k]; each factor
             starts as its own sub-state (Fig. 8a).  Replaces psi_in.
    Returns a Result with psi_out (bit k = outputs[k]), outcomes and
    probabilities keyed by qubit label.
    """
    if mode not in ("owqs", "eowqs"):
        raise ValueError("mode must be owqs or eowqs")
    if policy not in ("forced", "zero", "sampled"):
        raise ValueError("bad outcome policy")
    validate(pattern)
    res = Result()
    rng = SplitMix64(seed)
    owner: Dict[int, SubState] = {}
    gfactor = complex(1.0)
    I = list(pattern.inputs)
    explicit_n = {c.q0 for c in pattern.cmds if c.kind == "N"}

    if input_factors is not None:
        covered = sorted(q for qs, _ in input_factors for q in qs)
        if covered != sorted(I):
            raise ValueError("input factors must cover the inputs exactly once")
        for qs, vec in input_factors:
            f = from_flat(list(qs), np.asarray(vec, dtype=np.complex128))
            for q in qs:
                owner[q] = f
    elif I:
        if psi_in is None:
            vec = np.full(1 << len(I), 2.0 ** (-len(I) / 2.0), dtype=np.complex128)
        else:
            vec = np.asarray(psi_in, dtype=np.complex128).reshape(-1)
            if vec.size != (1 << len(I)):
                raise ValueError("psi_in has the wrong length")
            if mode == "owqs":
                vec = vec / np.linalg.norm(vec)
        s = from_flat(I, vec)
        for q in I:
            owner[q] = s
    elif psi_in is not None:
        # no input qubit: the input is a state over no qubit, one amplitude,
        # and the initial state is that amplitude times |+> on every qubit
        # (Section 4.1); normalised in OWQS like any input
        vec = np.asarray(psi_in, dtype=np.complex128).reshape(-1)
        if vec.size != 1:
            raise ValueError("psi_in has the wrong length")
        gfactor *= vec[0] / abs(vec[0]) if mode == "owqs" else vec[0]

    def ensure(q):
        if q not in owner:
            if q in explicit_n:
                raise PatternError(f"qubit {q} used before its N")
            owner[q] = plus_substate(q)

    def live_substates() -> List[SubState]:
        seen, out = set(), []
        for sub in owner.values():
            if id(sub) not in seen:
                seen.add(id(sub))
                out.append(sub)
        return out

    meas_outcomes: Dict[int, int] = {}
    for idx, c in enumerate(pattern.cmds):
        k = c.kind
        if k == "N":
            owner[c.q0] = plus_substate(c.q0)
        elif k == "E":
            ensure(c.q0)
            ensure(c.q1)
            a, b = owner[c.q0], owner[c.q1]
            if a is not b:
                m = kron(a, b)
                for q in m.labels:
                    owner[q] = m
                a = m
            res.peak_substate = max(res.peak_substate, len(a.labels))
            idx_t = [slice(None)] * len(a.labels)
            idx_t[a.axis(c.q0)] = 1
            idx_t[a.axis(c.q1)] = 1
            a.tensor[tuple(idx_t)] *= -1.0
        elif k in ("X", "Z"):
            ensure(c.q0)
            if signal_parity(meas_outcomes, c.sdom):
                sub = owner[c.q0]
                ax = sub.axis(c.q0)
                if k == "X":
                    sub.tensor = np.flip(sub.tensor, axis=ax).copy()
                else:
                    idx_t = [slice(None)] * len(sub.labels)
                    idx_t[ax] = 1
                    sub.tensor[tuple(idx_t)] *= -1.0
        else:  # M
            v = c.q0
            ensure(v)
            sub = owner[v]
            res.peak_substate = max(res.peak_substate, len(sub.labels))
            ax = sub.axis(v)
            s_sig = signal_parity(meas_outcomes, c.sdom)
            t_sig = signal_parity(meas_outcomes, c.tdom)
            e = resolved_phase(c.angle, s_sig, t_sig)
            a0 = np.take(sub.tensor, 0, axis=ax)
            a1 = np.take(sub.tensor, 1, axis=ax)
            half = [(a0 + e * a1) / SQRT2, (a0 - e * a1) / SQRT2]   # rows of M_0, M_1
            p = outcome_probabilities(mode, sub.tensor, half)
            if policy == "forced":
                s = int(outcomes[v]) & 1
            elif policy == "zero":
                s = 0
            else:
                u = rng.uniform()
                s = 0 if u <= p[0] else 1
            if mode == "owqs":
                if p[s] <= 0.0:
                    raise PatternError(f"forced outcome {s} on qubit {v} has probability 0")
                kept = half[s] / math.sqrt(p[s])
            else:
                kept = half[s] * SQRT2
            meas_outcomes[v] = s
            res.outcomes[v] = s
            res.probs[v] = p[s]
            res.pairs[v] = (p[0], p[1])
            labels = [q for q in sub.labels if q != v]
            del owner[v]
            if labels:
                new = SubState(labels, kept)
                for q in labels:
                    owner[q] = new
            else:
                gfactor *= complex(kept.reshape(()))
            res.measurements_done += 1
            if stop_after is not None and res.measurements_done >= stop_after:
                return res
        if trace is not None:
            trace(idx, c, live_substates())

    for o in pattern.outputs:
        ensure(o)
    subs = live_substates()
    if subs:
        total = subs[0]
        for s2 in subs[1:]:
            total = kron(total, s2)
        if sorted(total.labels) != sorted(pattern.outputs):
            raise PatternError("live qubits at the end are not the outputs")
        res.psi_out = to_output(total, list(pattern.outputs)) * gfactor
    else:
        res.psi_out = np.array([gfactor], dtype=np.complex128)
    return res
