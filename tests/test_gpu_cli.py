"""The package's command line (python -m paper_2103_07210_gb300) solves the
seeded hill problem and prints its statistics as one JSON object."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.parametrize("args", [["--nlon", "64", "--nlat", "32", "--precision", "fp64"],
                                  ["--nlon", "256", "--nlat", "128", "--repeat", "2"],
                                  ["--nlon", "256", "--nlat", "128", "--zero-guess"]])
def test_command_line_solves_and_reports(args):
    r = subprocess.run([sys.executable, "-m", "paper_2103_07210_gb300"] + args, cwd=ROOT, capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    out = json.loads(r.stdout.strip().splitlines()[-1])
    assert out["status"] == 0 and out["converged"] and out["steps"] > 0
    assert out["res_final_true"] <= 1e-10 * out["norm_R"]
