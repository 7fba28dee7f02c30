"""Tile autotuner (ftgcr_tune): the chosen layout is the fastest of those it
timed (never slower than the layout ftgcr_create picks by itself, which is
among them), a repeated call is answered from the cache, and a solve with
the tuned layout matches the oracle like any other (mixed: rel <= 1e-10 at
tol 1e-13; FP64: the oracle's decisions, rel <= 1e-10)."""
import pytest

import oracle
from paper_2103_07210_gb300 import ftgcr, inputs
from tests.gpu_util import rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _solve(p, k, tol, precision, tiles, rounds):
    with ftgcr.Solver(p.D, p.mu, k=k, tol=tol, precision=precision, tiles=tiles, rounds=rounds) as s:
        R = torch.from_numpy(p.R).cuda()
        x = torch.zeros_like(R)
        st = s.solve(R, x)
        return st, x.cpu().numpy(), s.stats()


def test_mixed_tuning_is_the_fastest_timed_layout_and_is_cached():
    p = inputs.hill_problem(256, 128, **inputs.random_hill(11))
    t = ftgcr.tune(p.D, p.mu, k=4, tol=1e-10, precision="mixed", concurrency=4)
    assert 1 <= t["tiles"] <= 128 and t["rounds"] in ("fused", "split") and t["candidates"] >= 4
    assert not t["cached"] and 0 < t["ms"] <= t["default_ms"]
    again = ftgcr.tune(p.D, p.mu, k=4, tol=1e-10, precision="mixed", concurrency=4)
    assert again["cached"] and (again["tiles"], again["rounds"], again["ms"]) == (t["tiles"], t["rounds"], t["ms"])
    ref = oracle.ftgcr(p.D, p.R, p.mu, 4, 1e-13)
    st, x, s = _solve(p, 4, 1e-13, "mixed", t["tiles"], t["rounds"])
    assert st == ftgcr.OK and s["tiles"] == t["tiles"] and s["split_rounds"] == (t["rounds"] == "split")
    assert rel_err(x, ref["x"]) <= 1e-10


def test_fp64_tuning_keeps_the_oracle_decisions():
    p = inputs.hill_problem(128, 64, rhs="random", seed=3)
    t = ftgcr.tune(p.D, p.mu, k=4, tol=1e-10, precision="fp64", concurrency=2)
    assert t["rounds"] == "auto" and 0 < t["ms"] <= t["default_ms"]
    ref = oracle.ftgcr(p.D, p.R, p.mu, 4, 1e-10)
    st, x, s = _solve(p, 4, 1e-10, "fp64", t["tiles"], "auto")
    assert st == ftgcr.OK and s["tiles"] == t["tiles"]
    assert s["steps"] == ref["steps"] and s["detect_steps"] == ref["detect_steps"]
    assert rel_err(x, ref["x"]) <= 1e-10


def test_fp64_wide_rows_tuning_reaches_global_factor_layouts():
    # 2048 columns: staged factors allow 1-row bands only; thicker bands read
    # the factors from global memory, and the tuner times both kinds
    p = inputs.hill_problem(2048, 48, rhs="random", seed=5)
    t = ftgcr.tune(p.D, p.mu, k=4, tol=1e-10, precision="fp64", concurrency=1)
    assert 0 < t["ms"] <= t["default_ms"] and t["candidates"] >= 3
    ref = oracle.ftgcr(p.D, p.R, p.mu, 4, 1e-10)
    st, x, s = _solve(p, 4, 1e-10, "fp64", t["tiles"], "auto")
    assert st == ftgcr.OK and s["tiles"] == t["tiles"]
    assert s["global_factors"] == (-(-48 // t["tiles"]) > 1)
    assert s["steps"] == ref["steps"] and s["detect_steps"] == ref["detect_steps"]
    assert rel_err(x, ref["x"]) <= 1e-10
