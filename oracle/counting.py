"""Amplitude-update count of a command sequence (oracle; test
infrastructure only).

Each command updates every amplitude of the array holding all live qubits
(prepared and not yet measured): a command acting at live width w counts 2^w.
N counts the width after the new qubit is added, M the width before the
measured qubit is eliminated.  N commutes with every command on other qubits
(Section 2.2), so every qubit is prepared just before the first command that
touches it, wherever its N command is listed; that preparation is the N that
is counted.
"""
from __future__ import annotations


def amplitude_updates(pattern) -> int:
    live = set(pattern.inputs)
    total = 0
    for c in pattern.cmds:
        if c.kind == "N":
            continue
        qs = [c.q0] + ([c.q1] if c.kind == "E" else [])
        for q in qs:
            if q not in live:
                live.add(q)
                total += 1 << len(live)
        total += 1 << len(live)
        if c.kind == "M":
            live.discard(c.q0)
    for o in pattern.outputs:          # outputs no command touched
        if o not in live:
            live.add(o)
            total += 1 << len(live)
    return total
