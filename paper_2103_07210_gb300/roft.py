"""Fault-tolerance statistics of FT-GCR(k) under the paper's data-loss model
(Section 3, Table 2, Figs. 1-3), on the GPU.

For each data-loss fraction q the study runs `runs` solves with fault
injection and `runs` without protection, each solve drawing its own plan: at
every executed step, with probability `prob`, one event (at most
`max_events` per solve) flips one bit in each of round(q N) entries of e,
chosen inside the block of one of `nranks` "processes" (the paper's MPI
ranks).  Solves in which no event fired are left out, as in the paper.
Reported per q, with iterations counted as executed inner steps:

  baseline      steps of the fault-free solve
  ftgcr, gcr    mean steps to convergence of the protected / unprotected runs
                (a run that does not converge counts max_steps)
  converged     fraction of runs that converged, per mode
  detection     detected faults / data-loss events that fired (protected)
  roft          (gcr - ftgcr) / baseline, the Return on Fault Tolerance
                score of Section 3

All runs of one (q, mode) go to the GPU as one batched persistent launch.

    python -m paper_2103_07210_gb300.roft [--nlon 512 --nlat 256 --runs 100]
"""
from __future__ import annotations

import argparse
import json

import numpy as np

from . import ftgcr, inputs

FRACTIONS = (4e-6, 4e-4, 2e-3, 1e-2, 5e-2, 2e-1)  # the paper's data-loss sizes (0.0004 % .. 20 %)


def loss_plan(seed: int, run: int, max_steps: int, prob: float, max_events: int, q: float, N: int, nranks: int):
    """Data-loss events (step, rank, nranks, count, seed) of one run: a
    Bernoulli(prob) draw per executed step, at most max_events events."""
    g = inputs.SplitMix64((seed << 20) + run)
    count = max(1, int(round(q * N)))
    ev = []
    for t in range(1, max_steps + 1):
        if len(ev) >= max_events:
            break
        if g.uniform() < prob:
            ev.append((t, g.below(nranks), nranks, count, g.next()))
    return ev


def study(nlon=512, nlat=256, k=5, tol=1e-10, runs=100, prob=0.02, max_events=10, nranks=72,
          fractions=FRACTIONS, precision="fp64", seed=2021, max_steps=None):
    import torch

    p = inputs.hill_problem(nlon, nlat)
    N = p.R.size
    R = torch.from_numpy(p.R).cuda()
    with ftgcr.Solver(p.D, p.mu, k=k, tol=tol, precision=precision) as s:
        x = torch.zeros_like(R)
        s.solve(R, x)
        base = s.stats()["steps"]
    cap = max_steps or 4 * base + 50
    out = {"grid": f"{nlon}x{nlat}", "k": k, "tol": tol, "runs": runs, "prob": prob, "max_events": max_events,
           "nranks": nranks, "precision": precision, "baseline": base, "max_steps": cap, "rows": []}
    for q in fractions:
        plans = [loss_plan(seed, i, cap, prob, max_events, q, N, nranks) for i in range(runs)]
        row = {"fraction": q}
        for mode, protect in (("ftgcr", True), ("gcr", False)):
            solvers = [ftgcr.Solver(p.D, p.mu, k=k, tol=tol, precision=precision, protect=protect, max_steps=cap)
                       for _ in range(runs)]
            xs = [torch.zeros_like(R) for _ in range(runs)]
            ftgcr.solve_batch(solvers, [R] * runs, xs, losses=plans)
            torch.cuda.synchronize()
            st = [s.stats() for s in solvers]
            for s in solvers:
                s.close()
            faulty = [t for t in st if t["loss_events"] > 0]
            steps = [t["steps"] if t["converged"] else cap for t in faulty]
            row[mode] = float(np.mean(steps)) if steps else float("nan")
            row[mode + "_converged"] = float(np.mean([t["converged"] for t in faulty])) if faulty else float("nan")
            row[mode + "_faulty_runs"] = len(faulty)
            if protect:
                fired = sum(t["loss_events"] for t in faulty)
                row["detection"] = sum(t["faults_detected"] for t in faulty) / fired if fired else float("nan")
        row["roft"] = (row["gcr"] - row["ftgcr"]) / base
        out["rows"].append(row)
    return out


def format_table(res) -> str:
    lines = [f"grid {res['grid']}, k = {res['k']}, tol {res['tol']:g}, {res['runs']} runs per mode, "
             f"p = {res['prob']:g} per step, <= {res['max_events']} events, {res['nranks']} blocks, "
             f"{res['precision']}; baseline {res['baseline']} steps",
             "data loss | GCR steps | FT-GCR steps | GCR conv | FT-GCR conv | detection | RoFT",
             "---|---|---|---|---|---|---"]
    for r in res["rows"]:
        lines.append(f"{100 * r['fraction']:.4g} % | {r['gcr']:.2f} | {r['ftgcr']:.2f} | {r['gcr_converged']:.2f} | "
                     f"{r['ftgcr_converged']:.2f} | {r['detection']:.2f} | {r['roft']:.3f}")
    return "\n".join(lines)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--nlon", type=int, default=512)
    ap.add_argument("--nlat", type=int, default=256)
    ap.add_argument("--k", type=int, default=5)
    ap.add_argument("--tol", type=float, default=1e-10)
    ap.add_argument("--runs", type=int, default=100)
    ap.add_argument("--prob", type=float, default=0.02)
    ap.add_argument("--precision", default="fp64")
    ap.add_argument("--json", action="store_true")
    a = ap.parse_args()
    res = study(a.nlon, a.nlat, a.k, a.tol, a.runs, a.prob, precision=a.precision)
    print(json.dumps(res) if a.json else format_table(res))


if __name__ == "__main__":
    main()
