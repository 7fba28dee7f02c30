"""Solve the seeded hill problem once (or a few times) on the current GPU and
print the solver's statistics as JSON:

    python -m paper_2103_07210_gb300 --nlon 1024 --nlat 512 --precision mixed

Each solve is one persistent launch of the library's kernel; the first
solve of a handle is no different from the others, so --repeat 2 gives a
profiler one launch to skip and one to capture."""
import argparse
import json
import time

from . import ftgcr, inputs


def main(argv=None):
    ap = argparse.ArgumentParser(prog="python -m paper_2103_07210_gb300")
    ap.add_argument("--nlon", type=int, default=1024)
    ap.add_argument("--nlat", type=int, default=512)
    ap.add_argument("--k", type=int, default=4)
    ap.add_argument("--tol", type=float, default=1e-10)
    ap.add_argument("--precision", choices=["mixed", "fp64"], default="mixed")
    ap.add_argument("--rounds", choices=list(ftgcr.ROUNDS), default="auto")
    ap.add_argument("--rhs", choices=["flow", "random"], default="flow")
    ap.add_argument("--repeat", type=int, default=1)
    ap.add_argument("--zero-guess", action="store_true",
                    help="declare x = 0 on entry (FTGCR_FLAG_ZERO_GUESS), as the benchmark's solves do")
    a = ap.parse_args(argv)
    import torch

    p = inputs.hill_problem(a.nlon, a.nlat, rhs=a.rhs)
    R = torch.from_numpy(p.R).cuda()
    with ftgcr.Solver(p.D, p.mu, k=a.k, tol=a.tol, precision=a.precision, rounds=a.rounds,
                      zero_guess=a.zero_guess) as s:
        times = []
        for _ in range(max(1, a.repeat)):
            x = torch.zeros_like(R)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            status = s.solve(R, x)
            torch.cuda.synchronize()
            times.append(1e3 * (time.perf_counter() - t0))
        st = s.stats()
    keep = ("steps", "outer", "converged", "tiles", "split_rounds", "streamed_rounds", "res_final_true", "norm_R")
    print(json.dumps({"status": status, "host_ms": times, **{k: st[k] for k in keep if k in st}}))
    return 0 if status == ftgcr.OK else 1


if __name__ == "__main__":
    raise SystemExit(main())
