"""Test helpers: random valid command orders and comparisons."""
from __future__ import annotations

import numpy as np

from owqs_inputs.patterns import Cmd
from owqs_inputs.rng import SplitMix64


def random_proposition_order(pattern, rng: SplitMix64):
    """A random command order that the Proposition of Section 4.3 allows for
    a standard-form pattern: repeatedly take a random ready qubit, apply its
    E commands not yet applied, measure it; then the remaining E commands and
    the corrections.  Forced-outcome results must not depend on the order."""
    assert pattern.is_standard()
    e_cmds = [c for c in pattern.cmds if c.kind == "E"]
    m_cmds = {c.q0: c for c in pattern.cmds if c.kind == "M"}
    corr = [c for c in pattern.cmds if c.kind in ("X", "Z")]
    used = [False] * len(e_cmds)
    done = set()
    out = []
    remaining = sorted(m_cmds)
    while remaining:
        ready = [v for v in remaining if set(m_cmds[v].sdom) | set(m_cmds[v].tdom) <= done]
        v = ready[rng.randint(len(ready))]
        for i, c in enumerate(e_cmds):
            if not used[i] and v in (c.q0, c.q1):
                out.append(c)
                used[i] = True
        out.append(m_cmds[v])
        done.add(v)
        remaining.remove(v)
    out += [c for i, c in enumerate(e_cmds) if not used[i]]
    out += corr
    return pattern.with_cmds(out)


def outcomes_by_label(pattern, bits):
    """Forced outcome per qubit label from bits listed in M-command order."""
    res = {}
    for k, q in enumerate(pattern.measured()):
        res[q] = int(bits[k])
    return res


def phase_aligned_maxabs(ref: np.ndarray, x: np.ndarray) -> float:
    ov = np.vdot(x, ref)
    if abs(ov) > 0:
        x = x * (ov / abs(ov))
    return float(np.max(np.abs(ref - x)))


def cmd(kind, *args, angle=0.0, sdom=(), tdom=()):
    if kind == "E":
        return Cmd("E", args[0], args[1])
    return Cmd(kind, args[0], -1, angle, sdom, tdom)
