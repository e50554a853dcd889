"""Train and evaluate the learned merge scorer (AJF_PLANNER_LEARNED).

    python -m paper_2103_11595_gb300.learned_planner train [--circuits 2000] [--out MODEL.npy]
    python -m paper_2103_11595_gb300.learned_planner eval  [--model MODEL.npy] [--held-out 200]

train: for circuits of the learned-planner workload (n ~ U{10..24}, 100-400 gates of U3 / CX / CZ
on random pairs, 5-40 mixed noises; seeds 0..N-1), the Alg. II network is planned by the greedy and
min-fill planners with restarts, the best path is replayed into ranking pairs (taken merge vs
other candidates; at most --pairs-per-circuit kept per circuit), and the MLP is trained on the GPU
with the library's CUDA kernels (ajf_learned_train).

eval: on held-out circuits (seeds 10000..) it compares the planned cost (complex multiply-adds) of
the learned planner against the greedy planner (one pass each, and with restarts), the planning
time, and -- for the circuits whose plan fits the device -- checks that F_J is unchanged.
All of it goes through the C ABI; the dataset is built on host-only contexts in parallel processes.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
DEFAULT_MODEL = os.path.join(os.path.dirname(os.path.abspath(__file__)), "data", "merge_scorer.npy")


def _dataset_worker(args):
    seeds, trials, per_circuit = args
    sys.path.insert(0, ROOT)
    from paper_2103_11595_gb300 import ajf
    from paper_2103_11595_gb300 import workloads as W
    c = ajf.Context(-1)
    chunks = []
    for s in seeds:
        inst = W.random_pairs_circuit(s)
        ajf.load_instance(c.handle, inst)
        try:
            d = ajf.ajf_learned_dataset(c.handle, 2, trials=trials, seed=s, negatives=4)
        except ajf.AjfError:
            continue
        if d.shape[0] > per_circuit:
            idx = np.random.default_rng(s).choice(d.shape[0], size=per_circuit, replace=False)
            d = d[np.sort(idx)]
        chunks.append(d)
    c.close()
    return np.concatenate(chunks) if chunks else np.zeros((0, 2, 16), np.float32)


def build_dataset(n_circuits: int, trials: int, per_circuit: int, procs: int) -> np.ndarray:
    import multiprocessing as mp
    seeds = list(range(n_circuits))
    parts = [seeds[i::procs] for i in range(procs)]
    with mp.get_context("spawn").Pool(procs) as pool:
        outs = pool.map(_dataset_worker, [(p, trials, per_circuit) for p in parts])
    return np.concatenate(outs)


def cmd_train(a):
    sys.path.insert(0, ROOT)
    import __graft_entry__
    __graft_entry__.build()
    from paper_2103_11595_gb300 import ajf
    t0 = time.time()
    data = build_dataset(a.circuits, a.trials, a.pairs_per_circuit, a.procs)
    t1 = time.time()
    w, loss = ajf.ajf_learned_train(a.device, data, epochs=a.epochs, batch=a.batch, lr=a.lr, seed=a.seed)
    t2 = time.time()
    os.makedirs(os.path.dirname(os.path.abspath(a.out)), exist_ok=True)
    np.save(a.out, w)
    print(json.dumps({"pairs": int(data.shape[0]), "circuits": a.circuits, "dataset_s": round(t1 - t0, 1),
                      "train_s": round(t2 - t1, 1), "final_loss": loss, "epochs": a.epochs, "model": a.out}))


def cmd_eval(a):
    sys.path.insert(0, ROOT)
    import __graft_entry__
    __graft_entry__.build()
    from paper_2103_11595_gb300 import ajf
    from paper_2103_11595_gb300 import workloads as W
    w = np.load(a.model)
    dev = a.device
    rows = []
    c = ajf.Context(dev)
    ajf.ajf_set_learned_model(c.handle, w)
    for i in range(a.held_out):
        inst = W.random_pairs_circuit(10000 + i)
        ajf.load_instance(c.handle, inst)
        row = {"seed": 10000 + i, "n": inst.n, "gates": len(inst.ideal), "noises": len(inst.noises)}
        runs = [("greedy1", "greedy", 1), ("learned1", "learned", 1)]
        if i < a.restart_subset:
            runs += [("greedy8", "greedy", 8), ("auto8", "auto", 8), ("learned8", "learned", 8)]
        for name, planner, trials in runs:
            t0 = time.time()
            try:
                info = ajf.ajf_plan(c.handle, 2, planner=planner, trials=trials, mem_budget_bytes=1e18)
            except ajf.AjfError as e:
                info = getattr(e, "info", {"cmacs": float("nan"), "width": -1, "arena_bytes": float("inf")})
                info["planner_used"] = -1
            row[name] = {"cmacs": info["cmacs"], "width": info["width"], "s": time.time() - t0,
                         "used": info.get("planner_used", -1), "arena": info.get("arena_bytes", 0.0)}
        # the learned planner alone (without the greedy judge) for the comparison of proposals
        rows.append(row)
    # F_J unchanged where the plans fit: learned vs greedy path, FP64
    checked = 0
    for row in rows:
        if checked >= a.fj_checks or row["learned1"]["arena"] > a.fj_budget or row["greedy1"]["arena"] > a.fj_budget:
            continue
        inst = W.random_pairs_circuit(row["seed"])
        ajf.load_instance(c.handle, inst)
        f = {}
        for planner in ("greedy", "learned"):
            ajf.ajf_plan(c.handle, 2, planner=planner, trials=1, precision="f64")
            f[planner] = ajf.ajf_fidelity_alg2(c.handle)["F"]
        row["F_greedy"], row["F_learned"] = f["greedy"], f["learned"]
        checked += 1
    # the held-out learned-family circuits are far too wide to execute; the executable n=16 line
    # circuits (mid workload, seeds 0..9) check that the learned path leaves F_J unchanged
    mid = []
    for s in range(a.mid_checks):
        inst = W.mid(s)
        ajf.load_instance(c.handle, inst)
        f, cm = {}, {}
        for planner in ("greedy", "learned"):
            info = ajf.ajf_plan(c.handle, 2, planner=planner, trials=1, precision="f64")
            f[planner] = ajf.ajf_fidelity_alg2(c.handle)["F"]
            cm[planner] = info["cmacs"]
        mid.append({"seed": s, "dF": abs(f["greedy"] - f["learned"]), "cmacs_greedy1": cm["greedy"],
                    "cmacs_learned1": cm["learned"]})
    c.close()

    def geo(key_a, key_b):
        r = [row[key_a]["cmacs"] / row[key_b]["cmacs"] for row in rows if key_a in row and key_b in row
             and math.isfinite(row[key_a]["cmacs"]) and math.isfinite(row[key_b]["cmacs"])]
        return float(np.exp(np.mean(np.log(r)))) if r else float("nan")

    fj = [abs(r["F_greedy"] - r["F_learned"]) for r in rows if "F_greedy" in r]
    summary = {
        "held_out": len(rows),
        "geomean_cmacs_learned1_over_greedy1": geo("learned1", "greedy1"),
        "geomean_cmacs_learned8_over_greedy8": geo("learned8", "greedy8"),
        "geomean_cmacs_learned8_over_auto8": geo("learned8", "auto8"),
        "learned_path_kept_1": sum(1 for r in rows if r["learned1"]["used"] == 3),
        "learned_path_kept_8": sum(1 for r in rows if "learned8" in r and r["learned8"]["used"] == 3),
        "restart_subset": min(a.restart_subset, len(rows)),
        "mean_plan_s": {k: float(np.mean([r[k]["s"] for r in rows if k in r]))
                        for k in ("greedy1", "learned1", "greedy8", "auto8", "learned8")},
        "fj_checked": len(fj), "max_abs_dF_learned_vs_greedy": max(fj) if fj else None,
        "executable_held_out": sum(1 for r in rows if r["learned1"]["arena"] <= a.fj_budget),
        "mid_fj_checked": len(mid), "mid_max_abs_dF_learned_vs_greedy": max((m["dF"] for m in mid), default=None),
        "mid_geomean_cmacs_learned1_over_greedy1": float(np.exp(np.mean(
            [np.log(m["cmacs_learned1"] / m["cmacs_greedy1"]) for m in mid]))) if mid else None,
    }
    if a.out:
        with open(a.out, "w") as f:
            json.dump({"summary": summary, "rows": rows, "mid": mid}, f)
    print(json.dumps(summary))


def main():
    ap = argparse.ArgumentParser()
    sub = ap.add_subparsers(dest="cmd", required=True)
    t = sub.add_parser("train")
    t.add_argument("--circuits", type=int, default=2000)
    t.add_argument("--trials", type=int, default=4)
    t.add_argument("--pairs-per-circuit", type=int, default=256)
    t.add_argument("--procs", type=int, default=os.cpu_count() or 4)
    t.add_argument("--epochs", type=int, default=20)
    t.add_argument("--batch", type=int, default=1024)
    t.add_argument("--lr", type=float, default=1e-3)
    t.add_argument("--seed", type=int, default=0)
    t.add_argument("--device", type=int, default=0)
    t.add_argument("--out", default=DEFAULT_MODEL)
    e = sub.add_parser("eval")
    e.add_argument("--model", default=DEFAULT_MODEL)
    e.add_argument("--held-out", type=int, default=200)
    e.add_argument("--device", type=int, default=0)
    e.add_argument("--fj-checks", type=int, default=20)
    e.add_argument("--restart-subset", type=int, default=40)
    e.add_argument("--mid-checks", type=int, default=10)
    e.add_argument("--fj-budget", type=float, default=4e9)
    e.add_argument("--out", default="")
    a = ap.parse_args()
    cmd_train(a) if a.cmd == "train" else cmd_eval(a)


if __name__ == "__main__":
    main()
