"""Seeded synthetic inputs for FT-GCR(k) runs: coefficient fields, right-hand
sides and fault plans.

This module holds no arithmetic of the solver (no operator, preconditioner or
iteration).  It is shared by the tests, ``bench.py`` and the smoke check; both
the CUDA library and the CPU oracle receive its arrays as plain inputs.

Workload recipe (stand-in for the paper's potential flow over an isolated hill
on the sphere, Section 3, whose octahedral 3-D Atlas problem is not available):
  * grid: regular latitude-longitude, nlon x nlat cells on the unit sphere;
  * coefficient D = 1 - h, h a Gaussian hill h0 exp(-(d/w)^2) of great-circle
    distance d from its centre (h0 = 0.1 ~ the paper's h/H = 4000/40800,
    e-folding width w, default 20 degrees, centre (pi, 0));
  * right-hand side: either seeded uniform noise U[-1, 1) or the divergence
    of the ambient zonal flow over the hill, div(D v_a) with v_a = (cos theta, 0)
    integrated over each cell (sums to zero over every latitude row);
  * faults: single-bit flips {step, vector, index, bit} drawn from SplitMix64.

Random numbers come from SplitMix64 (S. Vigna's published 64-bit generator:
add the golden-ratio increment, then two xor-shift-multiply rounds and a
final xor-shift).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

VEC_CODES = {"x": 0, "r": 1, "p": 2, "ap": 3, "e": 4}


def splitmix64(seed: int, n: int) -> np.ndarray:
    """The first n outputs of SplitMix64 started at state `seed`."""
    with np.errstate(over="ignore"):
        k = np.arange(1, n + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + k * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


class SplitMix64:
    """Sequential SplitMix64 stream (for small draws such as fault plans)."""

    def __init__(self, seed: int):
        self.state = seed & 0xFFFFFFFFFFFFFFFF

    def next(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & 0xFFFFFFFFFFFFFFFF
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & 0xFFFFFFFFFFFFFFFF
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & 0xFFFFFFFFFFFFFFFF
        return z ^ (z >> 31)

    def uniform(self) -> float:
        return (self.next() >> 11) * (1.0 / 9007199254740992.0)

    def below(self, n: int) -> int:
        return self.next() % n


def uniform_pm1(seed: int, shape) -> np.ndarray:
    """U[-1, 1) in FP64 from the top 53 bits of SplitMix64(seed)."""
    n = int(np.prod(shape))
    u = (splitmix64(seed, n) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
    return (2.0 * u - 1.0).reshape(shape)


def cell_centres(nlon: int, nlat: int):
    lam = (np.arange(nlon) + 0.5) * (2.0 * math.pi / nlon)
    th = -0.5 * math.pi + (np.arange(nlat) + 0.5) * (math.pi / nlat)
    return lam, th


def hill_depth(nlon: int, nlat: int, h0: float = 0.1, width: float = math.radians(20.0),
               centre=(math.pi, 0.0)) -> np.ndarray:
    """D = 1 - h0 exp(-(d/w)^2), d the great-circle distance (haversine form)."""
    lam, th = cell_centres(nlon, nlat)
    lc, tc = centre
    L, TH = np.meshgrid(lam, th)
    s = np.sin(0.5 * (TH - tc)) ** 2 + np.cos(TH) * math.cos(tc) * np.sin(0.5 * (L - lc)) ** 2
    d = 2.0 * np.arcsin(np.sqrt(np.clip(s, 0.0, 1.0)))
    return 1.0 - h0 * np.exp(-(d / width) ** 2)


def flow_rhs(D: np.ndarray) -> np.ndarray:
    """Cell-integrated div(D v_a) for the solid-body zonal wind v_a = (cos theta, 0):
    east-face flux D_face * cos(theta_j) * dtheta, differenced across the cell."""
    nlat, nlon = D.shape
    _, th = cell_centres(nlon, nlat)
    dth = math.pi / nlat
    Dx = 0.5 * (D + np.roll(D, -1, axis=1))
    flux = Dx * (np.cos(th) * dth)[:, None]
    return flux - np.roll(flux, 1, axis=1)


def random_hill(seed: int):
    """Hill parameters of the batched / serving mixes: centre lambda ~ U[0, 2pi),
    theta = asin(U[-1, 1)); h0 ~ U[0.05, 0.2]; w ~ U[10, 30] degrees."""
    g = SplitMix64(seed)
    lc = 2.0 * math.pi * g.uniform()
    tc = math.asin(2.0 * g.uniform() - 1.0)
    h0 = 0.05 + 0.15 * g.uniform()
    w = math.radians(10.0 + 20.0 * g.uniform())
    return dict(h0=h0, width=w, centre=(lc, tc))


@dataclass
class Problem:
    nlon: int
    nlat: int
    D: np.ndarray
    R: np.ndarray
    mu: float


def mu_for(nlat: int, mu_hat: float) -> float:
    """Helmholtz coefficient mu = mu_hat / dtheta^2 (a fixed Courant-like number
    on every grid)."""
    dth = math.pi / nlat
    return mu_hat / (dth * dth)


# Calibrated once with the oracle so that the fault-free FP64 FT-GCR(4) solve
# of the 512 x 256 hill problem at tol 1e-10 takes a number of steps in the
# 17-21 range of the paper's fault-free runs (Table 2 baselines).
MU_HAT = 0.3


def hill_problem(nlon: int, nlat: int, rhs: str = "flow", seed: int = 1, mu_hat: float = MU_HAT, **hill) -> Problem:
    D = hill_depth(nlon, nlat, **hill)
    R = uniform_pm1(seed, (nlat, nlon)) if rhs == "random" else flow_rhs(D)
    return Problem(nlon, nlat, D, R, mu_for(nlat, mu_hat))


def single_flip(seed: int, step: int, vec: str, N: int, nbits: int = 64):
    """One flip at `step` on `vec`; index and bit from SplitMix64(seed)."""
    g = SplitMix64(seed)
    return (int(step), VEC_CODES[vec], g.below(N), g.below(nbits))


def sweep_flip(seed: int, trial: int, n_steps: int, N: int, nbits: int = 64, vecs=("x", "r", "p", "ap")):
    """Fault-sweep trial: step ~ U{1..n_steps}, vec ~ U(vecs), index ~ U{0..N-1},
    bit ~ U{0..nbits-1}, from SplitMix64(seed + trial)."""
    g = SplitMix64(seed + trial)
    step = 1 + g.below(n_steps)
    vec = VEC_CODES[vecs[g.below(len(vecs))]]
    return (step, vec, g.below(N), g.below(nbits))


def batch_sizes(seed: int, n: int, choices=((128, 64), (256, 128), (512, 256), (1024, 512))):
    g = SplitMix64(seed)
    return [choices[g.below(len(choices))] for _ in range(n)]


def poisson_arrivals(seed: int, n: int, rate: float) -> np.ndarray:
    """Arrival times (s) of a Poisson stream of the given rate."""
    g = SplitMix64(seed)
    t, out = 0.0, np.empty(n)
    for i in range(n):
        u = g.uniform()
        t += -math.log(1.0 - u) / rate
        out[i] = t
    return out
