"""Rebuild csrc/owqs_group_sequences.inc: the register-slot sequences of the
complex64 pass groups that get a kernel compiled for them.

A pass group runs k consecutive measurements on an M-qubit register; pass j
measures the register slot slots[j].  The table lists the sequences that
carry the most work, measurements x 2^(live width), in the brickwork and
QFT-shaped J/CZ patterns and in random J/CZ circuits (the library's own
host planner under the greedy PROA order, read through
owqs_describe_groups; each family weighted equally), until the listed
sequences cover at least `coverage` of that work or `limit` of them are
listed.  Every other sequence runs on the kernel that reads the slots at run
time.

  python -m paper_1604_05659_gb300.gen_group_sequences [--limit 320] [--coverage 0.999]
"""
from __future__ import annotations

import argparse
import collections
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))
OUT = os.path.join(HERE, "csrc", "owqs_group_sequences.inc")


def workload_families():
    """Brickwork clusters of 16-28 rows, QFT-shaped patterns of 12-24 wires,
    random J/CZ circuits of 16-24 wires, and the wide items (13-14 inputs)
    of the recognition set, whose unitaries run on arrays of 2^27-2^29
    amplitudes and so take 4-qubit registers (the synthetic families the
    library is measured on), each family weighted equally."""
    from owqs_inputs import workloads
    return {
        "brickwork": [workloads.brickwork(r, 24) for r in range(16, 29)] + [workloads.brickwork(28, 40)],
        "qft": [workloads.qft(n, with_input=False) for n in range(12, 25, 2)],
        "random": workloads.random_batch(8, 16, 24, 20, 40, config_index=4, start=2000, with_input=False),
        "recognition_wide": [wl for wl in workloads.random_batch(count=256, with_input=False)
                             if len(wl.pattern.inputs) > 12],
    }


# families planned as on arrays of at least 2^26 amplitudes (4-qubit registers)
WIDE_FAMILIES = ("recognition_wide",)


def sequence_work(families):
    """Share of each (m, slots, half) in the group work of each family (work =
    passes x 2^(input width)), summed over the families."""
    from paper_1604_05659_gb300 import owqs
    owqs.library()
    share = collections.Counter()
    for name, wls in families.items():
        work = collections.Counter()
        # a unitary's array carries one reference qubit per input: plan these
        # patterns with the 4-qubit registers such arrays get
        owqs.test_group_m4_width(10 if name in WIDE_FAMILIES else 0)
        for wl in wls:
            h = owqs.load(wl.pattern)
            h.reorder()
            for real in (False, True):
                for g in h.describe_groups(wl.outcomes, dtype="c64", real_input=real):
                    work[(g["m"], g["slots"], g["half"])] += len(g["slots"]) * 2.0 ** g["n_in"]
            h.close()
        owqs.test_group_m4_width(0)
        total = sum(work.values())
        for key, w in work.items():
            share[key] += w / total
    return share


def code(m: int, slots, half: bool) -> int:
    c = (int(half) << 31) | (m << 28) | (len(slots) << 24)
    for j, s in enumerate(slots):
        c |= s << (2 * j)
    return c


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--limit", type=int, default=320)
    ap.add_argument("--coverage", type=float, default=0.999)
    a = ap.parse_args(argv)
    work = sequence_work(workload_families())
    total = sum(work.values())
    rows, acc = [], 0.0
    for (m, slots, half), w in work.most_common():
        if len(rows) >= a.limit or acc >= a.coverage * total:
            break
        rows.append(f"    0x{code(m, slots, half):08x}u,  // M={m} {' '.join(str(s) for s in slots)}"
                    f"{' (every probability 1/2)' if half else ''}")
        acc += w
    with open(OUT, "w") as f:
        f.write("// generated by gen_group_sequences.py: register-slot sequences of the complex64\n")
        f.write(f"// pass groups compiled as their own kernels ({len(rows)} sequences, "
                f"{100.0 * acc / total:.2f} % of the group work of brickwork, QFT and random J/CZ patterns\n"
                f"// and of the recognition set's wide unitaries)\n")
        f.write("\n".join(rows) + "\n")
    print(f"{len(rows)} sequences, {100.0 * acc / total:.2f} % of the work -> {OUT}")


if __name__ == "__main__":
    main()
