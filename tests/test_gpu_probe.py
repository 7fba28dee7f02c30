"""The FP64 FMA-rate probe (ftgcr_fp64_fma_rate) on the device: a positive
rate, below what the FP64 pipe of any GB300 can issue (nominal 1.25 TFLOP/s
dense FP64), and proportional work: four times the iterations take about
four times as long, so the figure is a rate and not a launch overhead."""
import pytest

from paper_2103_07210_gb300 import ftgcr

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_fp64_fma_rate_is_a_plausible_rate():
    r1 = ftgcr.fp64_fma_rate(1024)
    r4 = ftgcr.fp64_fma_rate(4096)
    assert 0.05 < r4 < 4.0, r4
    # the same rate at four times the work (launch overhead amortised)
    assert 0.5 < r4 / r1 < 2.0, (r1, r4)
