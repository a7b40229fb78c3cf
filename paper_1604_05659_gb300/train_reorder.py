"""Train the learned reorder proposal on the GPU and save its weights.

  python -m paper_1604_05659_gb300.train_reorder [--train 2000] [--heldout 200]

Training patterns are random J/CZ circuits of 16..30 logical qubits and depth
20..60 (seeded).  For each one the target order is the cheaper of the two
greedy orders the library builds, PROA with every qubit ready (EOWQS) and
PROA with measurement dependencies (OWQS), ranked by (peak live width,
amplitude updates) -- the quantities that set GPU memory and time.  The
network learns to score the target's choice lowest among the ready
candidates at every step (features from owqs_reorder_features, training by
owqs_model_train: the library's own forward and backward kernels).  For a
seeded subset the target is instead the fastest of the library's candidate
orders as simulated and timed on the GPU.  The held-out patterns are then
reordered in EOWQS mode with the proposal, which is kept only if no worse than the greedy order,
the kept orders of a subset are timed against the greedy orders that fit the
device, and the comparison is stored next to the weights.
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))
DEFAULT_OUT = os.path.join(HERE, "reorder_mlp.json")


def target_order(h):
    """Cheaper of the EOWQS and OWQS greedy orders by (peak live, updates)."""
    best = None
    for mode in ("eowqs", "owqs"):
        order, info = h.reorder(mode=mode, sweep=(mode == "owqs"),
                                weights=(float(max(1, h.nout)), float(max(1, h.nout)), 0.5, float(max(1, h.nout))))
        key = (info["peak_live"], info["amp_updates"])
        if best is None or key < best[0]:
            best = (key, order)
    return best[1]


def gpu_seconds(h, reps: int = 3) -> float:
    """Median CUDA-event time of one EOWQS run (complex64, all-zero branch,
    one array, graph replay) under the handle's active order."""
    import torch
    out = torch.empty(1 << h.nout, dtype=torch.complex64, device="cuda")
    h.run(None, dtype="c64", mode="eowqs", policy="zero", out=out, layout="one_array")
    ts = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        h.run(None, dtype="c64", mode="eowqs", policy="zero", out=out, layout="one_array")
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1) / 1e3)
    del out
    return sorted(ts)[len(ts) // 2]


def timed_target(h, max_live: int = 24):
    """Candidate orders generated by the library (greedy OWQS sweep, greedy
    EOWQS, the circuit's own order), each simulated and timed on the GPU when
    its widest array fits max_live qubits; returns the fastest among those of
    the smallest peak, and whether the modelled choice (peak, then amplitude
    updates) agrees with the measured one."""
    k = float(max(1, h.nout))
    w = (k, k, 0.5, k)
    cands = []
    for label in ("owqs_sweep", "eowqs_greedy", "circuit"):
        if label == "owqs_sweep":
            order, info = h.reorder(mode="owqs", sweep=True, weights=w)
        elif label == "eowqs_greedy":
            order, info = h.reorder(mode="eowqs", sweep=False, weights=w)
        else:
            order = h.pattern.measured()
            h.set_order(order)
            info = h.info()
        if info["peak_live"] > max_live:
            continue
        cands.append({"label": label, "order": list(order), "peak": info["peak_live"],
                      "updates": info["amp_updates"], "seconds": gpu_seconds(h)})
    if not cands:
        return None
    best = min(cands, key=lambda c: (c["peak"], c["seconds"]))
    modelled = min(cands, key=lambda c: (c["peak"], c["updates"]))
    return best, modelled


def build_dataset(handles, cands, seed, timed: int = 0, timed_width: int = 22):
    """handles: iterable of loaded patterns (consumed one at a time).  The
    first `timed` patterns of at most timed_width inputs take their target
    from GPU timings (timed_target); the others from the modelled cost."""
    feats, firsts, targets = [], [0], []
    row = 0
    stats = {"timed": 0, "agree": 0, "modelled_over_measured": []}
    for i, h in enumerate(handles):
        order = None
        if stats["timed"] < timed and h.nin <= timed_width:
            tt = timed_target(h)
            if tt is not None:
                best, modelled = tt
                order = best["order"]
                stats["timed"] += 1
                stats["agree"] += best["label"] == modelled["label"]
                stats["modelled_over_measured"].append(modelled["seconds"] / best["seconds"])
        if order is None:
            order = target_order(h)
        f, first, tgt = h.features(order, mode="eowqs", max_cands=cands, seed=seed + i)
        feats.append(f)
        firsts.extend((first[1:] + row).tolist())
        targets.extend((tgt + row).tolist())
        row += f.shape[0]
    X = (np.concatenate(feats).astype(np.float32), np.array(firsts, dtype=np.uint32),
         np.array(targets, dtype=np.uint32))
    return X if timed == 0 else (X, stats)


def evaluate(handles, model, sweep, timed: int = 0, timed_width: int = 30):
    """EOWQS reordering of each held-out pattern with the proposal, checked against
    the best greedy order: the greedy EOWQS order (without the sweep the
    Eq. 18 weights are Section 5's first run, a = b = d = |O|, g = 0.5) and
    the greedy OWQS sweep order, which waits for every domain and so is
    valid with preselected outcomes too; the library keeps the proposal only
    if it is no worse by (peak live width, amplitude updates).  For the first
    `timed` patterns of at most timed_width inputs, the kept order and the
    best greedy order are simulated on the GPU (EOWQS, complex64, all-zero
    branch) when they fit the device."""
    rows = []
    ntimed = 0
    for h in handles:
        k = float(max(1, h.nout))
        w = (k, k, 0.5, k)
        _, e = h.reorder(mode="eowqs", sweep=sweep, weights=w)
        _, o = h.reorder(mode="owqs", sweep=True)
        greedy_seconds = gpu_seconds(h) if ntimed < timed and h.nin <= timed_width and o["peak_live"] <= 31 else None
        _, l = h.reorder(mode="eowqs", sweep=sweep, weights=w, model=model)
        row = {"n": h.nin, "K": h.K, "eowqs_greedy_peak": e["peak_live"], "owqs_greedy_peak": o["peak_live"],
               "greedy_peak": l["greedy_peak_live"], "greedy_updates": l["greedy_amp_updates"],
               "greedy_best": "owqs" if l["greedy_best_owqs"] else "eowqs",
               "learned_peak": l["learned_peak_live"], "learned_updates": l["learned_amp_updates"],
               "accepted": l["learned_accepted"], "kept_peak": l["peak_live"], "kept_updates": l["amp_updates"]}
        if greedy_seconds is not None and l["peak_live"] <= 31:
            row["kept_seconds"] = gpu_seconds(h) if l["learned_accepted"] else greedy_seconds
            if l["greedy_best_owqs"]:
                row["greedy_seconds"] = greedy_seconds
            ntimed += 1
        rows.append(row)
    return rows


SATURATED = (1 << 64) - 1  # the library's update count saturates here (64+ live qubits)


def summary(rows):
    """Held-out comparison against the best greedy order.  The update ratio is
    a geometric mean over the patterns whose greedy count did not saturate."""
    acc = sum(r["accepted"] for r in rows)
    exact = [r for r in rows if r["greedy_updates"] < SATURATED]
    ratio = (float(np.exp(np.mean([np.log(r["greedy_updates"] / r["kept_updates"]) for r in exact])))
             if exact else None)
    tr = [r for r in rows if "greedy_seconds" in r and "kept_seconds" in r]
    timing = None
    if tr:
        timing = {"patterns": len(tr),
                  "geomean_best_greedy_over_kept_seconds": float(np.exp(np.mean(
                      [np.log(r["greedy_seconds"] / r["kept_seconds"]) for r in tr]))),
                  "kept_seconds_total": float(sum(r["kept_seconds"] for r in tr)),
                  "best_greedy_seconds_total": float(sum(r["greedy_seconds"] for r in tr))}
    return {"patterns": len(rows), "accepted": acc,
            "compared_with": "the better of the greedy EOWQS order and the greedy OWQS sweep order",
            "best_greedy_is_owqs_sweep": sum(r["greedy_best"] == "owqs" for r in rows),
            "kept_never_worse": all((r["kept_peak"], r["kept_updates"]) <= (r["greedy_peak"], r["greedy_updates"])
                                    for r in rows),
            "mean_peak_live": {"eowqs_greedy": float(np.mean([r["eowqs_greedy_peak"] for r in rows])),
                               "owqs_greedy": float(np.mean([r["owqs_greedy_peak"] for r in rows])),
                               "best_greedy": float(np.mean([r["greedy_peak"] for r in rows])),
                               "learned": float(np.mean([r["learned_peak"] for r in rows])),
                               "kept": float(np.mean([r["kept_peak"] for r in rows]))},
            "gpu_time": timing,
            "geomean_update_ratio_best_greedy_over_kept": ratio,
            "learned_peak_equals_n_plus_1": sum(r["learned_peak"] == r["n"] + 1 for r in rows)}


def main(argv=None):
    import torch
    from owqs_inputs import workloads
    from paper_1604_05659_gb300 import owqs

    ap = argparse.ArgumentParser()
    ap.add_argument("--train", type=int, default=2000)
    ap.add_argument("--heldout", type=int, default=200)
    ap.add_argument("--wmin", type=int, default=16)
    ap.add_argument("--wmax", type=int, default=30)
    ap.add_argument("--dmin", type=int, default=20)
    ap.add_argument("--dmax", type=int, default=60)
    ap.add_argument("--cands", type=int, default=8)
    ap.add_argument("--epochs", type=int, default=6)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--batch-steps", type=int, default=2048)
    ap.add_argument("--eval-sweep", action="store_true", help="compare with the full Section 5 sweep")
    ap.add_argument("--out", default=DEFAULT_OUT)
    ap.add_argument("--timed", type=int, default=64, help="training patterns labelled by GPU timings")
    ap.add_argument("--timed-eval", type=int, default=200, help="held-out patterns whose orders are GPU-timed")
    ap.add_argument("--eval-only", action="store_true",
                    help="re-evaluate the weights already in --out on the held-out set and rewrite its summary")
    a = ap.parse_args(argv)

    t0 = time.time()

    def handles(count, start):
        for i in range(start, start + count):  # one pattern in memory at a time
            w = workloads.random_pattern(i, a.wmin, a.wmax, a.dmin, a.dmax, 4, with_input=False)
            yield owqs.load(w.pattern)

    if a.eval_only:
        res = json.load(open(a.out))
        model = owqs.Model(weights=np.array(res["params"], dtype=np.float32))
        rows = evaluate(handles(a.heldout, 1_000_000), model, a.eval_sweep, timed=a.timed_eval)
        res["heldout"] = summary(rows)
        res.setdefault("seconds", {})["eval"] = time.time() - t0
        with open(a.out, "w") as f:
            json.dump(res, f)
        print(json.dumps({k: v for k, v in res.items() if k != "params"}))
        return

    (X, first, target), tstats = build_dataset(handles(a.train, 0), a.cands, seed=4, timed=a.timed)
    t_data = time.time() - t0
    Xd = torch.from_numpy(X).cuda()
    Fd = torch.from_numpy(first.astype(np.int32)).cuda()
    Td = torch.from_numpy(target.astype(np.int32)).cuda()
    model = owqs.Model(seed=1604)
    t1 = time.time()
    losses = model.train(Xd, Fd, Td, epochs=a.epochs, batch_steps=a.batch_steps, lr=a.lr, seed=7)
    torch.cuda.synchronize()
    t_train = time.time() - t1
    t2 = time.time()
    rows = evaluate(handles(a.heldout, 1_000_000), model, a.eval_sweep, timed=a.timed_eval)
    t_eval = time.time() - t2
    res = {"params": [float(x) for x in model.weights()],
           "trained_on": {"patterns": a.train, "widths": [a.wmin, a.wmax], "depths": [a.dmin, a.dmax],
                          "candidates_per_step": a.cands, "rows": int(X.shape[0]), "steps": int(len(target)),
                          "epochs": a.epochs, "lr": a.lr, "batch_steps": a.batch_steps,
                          "epoch_losses": [float(x) for x in losses],
                          "gpu_timed_targets": {"patterns": tstats["timed"], "measured_equals_modelled": tstats["agree"],
                                                "geomean_modelled_over_measured_seconds": float(np.exp(np.mean(
                                                    np.log(tstats["modelled_over_measured"]))))
                                                if tstats["modelled_over_measured"] else None}},
           "heldout": summary(rows),
           "seconds": {"data": t_data, "train": t_train, "eval": t_eval}}
    with open(a.out, "w") as f:
        json.dump(res, f)
    print(json.dumps({k: v for k, v in res.items() if k != "params"}))


if __name__ == "__main__":
    main()
