"""The data-loss study runs end to end on the GPU (small grid, few runs):
every row has its statistics, detection is a rate, and a protected solve never
needs more steps on average than the baseline plus k + 1 per detected fault
when all faults are detected."""
import math

import pytest

from paper_2103_07210_gb300 import roft

pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_study_small():
    res = roft.study(nlon=128, nlat=64, k=5, runs=12, prob=0.1, fractions=(1e-3, 0.2))
    assert res["baseline"] > 0 and len(res["rows"]) == 2
    for r in res["rows"]:
        for key in ("ftgcr", "gcr", "roft", "detection", "ftgcr_converged", "gcr_converged"):
            assert key in r
        if r["ftgcr_faulty_runs"]:
            assert 0.0 <= r["detection"] <= 1.0
            assert math.isfinite(r["roft"])
            assert r["ftgcr"] >= res["baseline"] - 1e-9 or r["detection"] < 1.0
    print(roft.format_table(res))
