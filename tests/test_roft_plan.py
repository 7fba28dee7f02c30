"""Host logic of the data-loss study (Section 3's fault model): the per-run
plans are deterministic, respect the event cap, draw ranks inside [0,
nranks), size every event as round(q N) flips, and fire at the per-step rate
asked for."""
import numpy as np

from paper_2103_07210_gb300 import roft


def test_plans_are_deterministic_and_bounded():
    a = roft.loss_plan(7, 3, 200, 0.05, 10, 1e-2, 131072, 72)
    b = roft.loss_plan(7, 3, 200, 0.05, 10, 1e-2, 131072, 72)
    assert a == b and 0 < len(a) <= 10
    steps = [e[0] for e in a]
    assert steps == sorted(steps) and len(set(steps)) == len(steps) and steps[0] >= 1
    for step, rank, nranks, count, seed in a:
        assert nranks == 72 and 0 <= rank < 72 and count == 1311 and 0 <= seed < 2 ** 64
    assert roft.loss_plan(7, 4, 200, 0.05, 10, 1e-2, 131072, 72) != a


def test_tiny_fractions_still_flip_one_entry_and_the_cap_holds():
    ev = roft.loss_plan(1, 0, 10000, 0.5, 10, 4e-6, 1000, 8)
    assert len(ev) == 10 and all(e[3] == 1 for e in ev)


def test_event_rate_matches_the_probability():
    hits = sum(len(roft.loss_plan(11, r, 50, 0.02, 1000, 1e-3, 4096, 4)) for r in range(2000))
    rate = hits / (2000 * 50)
    assert abs(rate - 0.02) < 0.003
