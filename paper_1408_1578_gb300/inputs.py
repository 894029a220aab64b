"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle's
callers.  This module draws random numbers and fixes workload shapes only; it
holds none of the CFIE arithmetic.

Workloads (synthetic stand-ins for the ellipse / bean experiments of Section 3,
which the paper runs at p = 8 points per wavelength):

* ``disk``      unit circle, omega = 64, n = 1024, one plane wave d = (1, 0)
* ``star``      r = 1 + 0.3 cos 5t, omega = 256, n = 4096, 16 directions
* ``kite``      kite curve, omega = 2048, n = 32768, 64 directions
* ``stars``     256 random stars r = 1 + sum_{k<=8} a_k cos kt + b_k sin kt,
                a_k, b_k ~ U(-0.05, 0.05), n log-uniform in [512, 16384] (even),
                omega at 10 points per wavelength, 32 directions
* ``requests``  Poisson arrivals (rate 200/s) of sound-soft / sound-hard solves
                on random stars, n log-uniform in [1024, 65536] (even), 1..64
                directions, 10 points per wavelength
"""
import math

import numpy as np


def directions(count):
    """Incidence angles theta_k = 2 pi k / count."""
    return 2.0 * np.pi * np.arange(count) / count


def random_density(n, nrhs, seed):
    """Complex vectors with unit-variance real and imaginary parts, shape
    (nrhs, n): row k is right-hand side k (column-major n x nrhs)."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal((nrhs, n)) + 1j * rng.standard_normal((nrhs, n))


def star_perimeter(a, b, samples=4096):
    """Perimeter of r(t) = 1 + sum a_k cos kt + b_k sin kt (trapezoid rule,
    spectrally accurate for the periodic integrand); used to set omega."""
    t = 2.0 * np.pi * np.arange(samples) / samples
    k = np.arange(1, len(a) + 1)
    r = 1.0 + np.cos(np.outer(t, k)) @ np.asarray(a) + np.sin(np.outer(t, k)) @ np.asarray(b)
    dr = (-np.sin(np.outer(t, k)) * k) @ np.asarray(a) + (np.cos(np.outer(t, k)) * k) @ np.asarray(b)
    return float(np.sum(np.hypot(r, dr)) * 2.0 * np.pi / samples)


def omega_for_ppw(n, perimeter, ppw=10.0):
    """Frequency that puts `ppw` nodes on each wavelength: n = ppw L omega / (2 pi)."""
    return 2.0 * math.pi * n / (ppw * perimeter)


def _log_uniform_even(rng, lo, hi):
    return int(2 * round(math.exp(rng.uniform(math.log(lo), math.log(hi))) / 2))


def random_stars(count=256, seed=1408, n_lo=512, n_hi=16384, nrhs=32):
    """The batched workload: list of dicts with a, b, n, omega, nrhs."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        a = rng.uniform(-0.05, 0.05, 8)
        b = rng.uniform(-0.05, 0.05, 8)
        n = _log_uniform_even(rng, n_lo, n_hi)
        omega = omega_for_ppw(n, star_perimeter(a, b))
        out.append({"a": a, "b": b, "n": n, "omega": omega, "nrhs": nrhs})
    return out


def poisson_requests(count=2000, rate=200.0, seed=1578, n_lo=1024, n_hi=65536):
    """The served workload: arrival time, boundary condition, obstacle, n, omega, nrhs."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, count))
    out = []
    for i in range(count):
        a = rng.uniform(-0.05, 0.05, 8)
        b = rng.uniform(-0.05, 0.05, 8)
        n = _log_uniform_even(rng, n_lo, n_hi)
        out.append({
            "arrival": float(t[i]),
            "bc": "soft" if rng.uniform() < 0.5 else "hard",
            "a": a, "b": b, "n": n,
            "omega": omega_for_ppw(n, star_perimeter(a, b)),
            "nrhs": int(rng.integers(1, 65)),
        })
    return out


WORKLOADS = {
    "disk": {"curve": "circle", "params": {}, "n": 1024, "omega": 64.0, "nrhs": 1, "bc": "soft"},
    "star": {"curve": "star", "params": {"a": [0, 0, 0, 0, 0.3], "b": [0, 0, 0, 0, 0]},
             "n": 4096, "omega": 256.0, "nrhs": 16, "bc": "hard"},
    "kite": {"curve": "kite", "params": {}, "n": 32768, "omega": 2048.0, "nrhs": 64, "bc": "soft"},
    # the paper's ellipse experiments (Section 3, Tables 1 and 3, first rows):
    # semi-axes (1, 0.5), p = 8 points per wavelength (omega = 2 pi n / (8 L),
    # L = 4.8442 the perimeter), one plane wave along +x, GMRES(80) to 1e-6
    "ellipse": {"curve": "ellipse", "params": {"a": 1.0, "b": 0.5}, "n": 32768, "omega": 5313.0,
                "nrhs": 1, "bc": "soft", "rtol": 1e-6},
    "ellipse-hard": {"curve": "ellipse", "params": {"a": 1.0, "b": 0.5}, "n": 32768,
                     "omega": 5313.0, "nrhs": 1, "bc": "hard", "rtol": 1e-6},
}
