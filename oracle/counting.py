"""Amplitude-update count of a command sequence (oracle; test
infrastructure only).

Each command updates every amplitude of the array holding all live qubits
(prepared and not yet measured): a command acting at live width w counts 2^w.
N counts the width after the new qubit is added, M the width before the
measured qubit is eliminated; a qubit without an explicit N is prepared just
before the first command that touches it and that implicit N is counted too.
"""
from __future__ import annotations


def amplitude_updates(pattern) -> int:
    live = set(pattern.inputs)
    total = 0
    for c in pattern.cmds:
        if c.kind == "N":
            live.add(c.q0)
            total += 1 << len(live)
            continue
        qs = [c.q0] + ([c.q1] if c.kind == "E" else [])
        for q in qs:
            if q not in live:
                live.add(q)
                total += 1 << len(live)
        total += 1 << len(live)
        if c.kind == "M":
            live.discard(c.q0)
    return total
