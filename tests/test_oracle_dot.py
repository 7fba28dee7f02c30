"""Pin of the oracle's inner product: accumulated in twice the working
precision (Dot2, Ogita-Rump-Oishi) and rounded once, so it agrees with the
exactly rounded sum of the exact products (computed here with rationals)
except within its error bound, and survives cancellation that destroys the
naive sum."""
from fractions import Fraction

import numpy as np

import oracle
from paper_2103_07210_gb300 import inputs


def exact_dot(a, b):
    return float(sum(Fraction(float(x)) * Fraction(float(y)) for x, y in zip(a, b)))


def test_dot_is_exactly_rounded_on_random_data():
    hits = 0
    for seed in range(60):
        a = inputs.uniform_pm1(1000 + seed, (700,)) * 10.0 ** (seed % 7 - 3)
        b = inputs.uniform_pm1(2000 + seed, (700,))
        got, ref = oracle.dot(a, b), exact_dot(a, b)
        # Dot2 bound: |got - exact| <= eps |exact| + gamma_{n-1}^2 sum |a b|
        eps = 2.0 ** -53
        gam = 699 * eps / (1 - 699 * eps)
        assert abs(got - ref) <= 2 * eps * abs(ref) + gam * gam * float(np.abs(a * b).sum())
        hits += got == ref
    assert hits >= 58


def test_dot_survives_cancellation():
    a = np.array([1e16, 1.0, -1e16, 3.0, 1e-20])
    b = np.ones(5)
    assert oracle.dot(a, b) == exact_dot(a, b) == 4.0
    assert float(np.sum(a)) != 4.0  # what plain summation loses
    g = inputs.SplitMix64(9)
    for _ in range(50):
        x = inputs.uniform_pm1(g.next() & 0xFFFF, (200,))
        a = np.concatenate([x * 1e10, -x * 1e10, x[:3]])
        b = np.ones_like(a)
        assert oracle.dot(a, b) == exact_dot(a, b)


def test_dot_propagates_non_finite():
    assert np.isnan(oracle.dot(np.array([np.inf, 1.0]), np.array([0.0, 1.0])))
    # an overflowing product makes the result non-finite (the exact split of an
    # infinite product is Inf - Inf), which the fault test treats as a fault
    assert not np.isfinite(oracle.dot(np.array([1e300, 1e300]), np.array([1e300, 1.0])))
