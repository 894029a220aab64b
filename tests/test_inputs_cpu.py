"""The seeded input generators shared by the tests, the benchmark and the oracle's
callers: shapes, ranges, determinism, and the frequencies they derive, each
checked against an independent computation.  CPU only."""
import math

import numpy as np
import pytest
import scipy.integrate as si
import scipy.special as sp

from paper_1408_1578_gb300 import inputs


def test_directions():
    th = inputs.directions(64)
    assert th.shape == (64,) and th[0] == 0.0
    assert np.allclose(np.diff(th), 2 * np.pi / 64, rtol=0, atol=1e-15)


def test_random_density_is_seeded_and_standard():
    x = inputs.random_density(5000, 3, seed=7)
    assert x.shape == (3, 5000) and x.dtype == np.complex128
    assert np.array_equal(x, inputs.random_density(5000, 3, seed=7))
    assert not np.array_equal(x, inputs.random_density(5000, 3, seed=8))
    assert abs(np.var(x.real) - 1) < 0.05 and abs(np.var(x.imag) - 1) < 0.05
    assert abs(np.mean(x)) < 0.05


def test_star_perimeter_against_adaptive_quadrature():
    assert abs(inputs.star_perimeter([0.0], [0.0]) - 2 * np.pi) < 1e-13
    a, b = [0, 0, 0, 0, 0.3], [0.02, 0, -0.04, 0, 0]
    k = np.arange(1, 6)

    def speed(t):
        r = 1 + np.dot(a, np.cos(k * t)) + np.dot(b, np.sin(k * t))
        dr = np.dot(a, -k * np.sin(k * t)) + np.dot(b, k * np.cos(k * t))
        return math.hypot(r, dr)

    want, _ = si.quad(speed, 0, 2 * np.pi, limit=400, epsabs=1e-13, epsrel=1e-13)
    assert abs(inputs.star_perimeter(a, b) - want) < 1e-11


def test_points_per_wavelength_round_trip():
    L = 7.3
    w = inputs.omega_for_ppw(4096, L, ppw=10.0)
    assert abs(4096 / (L / (2 * np.pi / w)) - 10.0) < 1e-12


def test_random_stars_workload():
    stars = inputs.random_stars()
    assert len(stars) == 256
    again = inputs.random_stars()
    assert all(np.array_equal(s["a"], t["a"]) and s["n"] == t["n"] for s, t in zip(stars, again))
    for s in stars:
        assert s["n"] % 2 == 0 and 512 <= s["n"] <= 16384 and s["nrhs"] == 32
        assert np.all(np.abs(s["a"]) <= 0.05) and np.all(np.abs(s["b"]) <= 0.05)
        L = inputs.star_perimeter(s["a"], s["b"])
        assert abs(2 * np.pi * s["n"] / (s["omega"] * L) - 10.0) < 1e-9
    ns = np.array([s["n"] for s in stars])
    # log-uniform: the median sits near the geometric mean of the range
    assert 0.6 < np.median(ns) / math.sqrt(512 * 16384) < 1.6


def test_poisson_requests():
    reqs = inputs.poisson_requests(count=2000)
    t = np.array([r["arrival"] for r in reqs])
    assert np.all(np.diff(t) > 0)
    assert abs(np.mean(np.diff(t)) - 1 / 200.0) < 0.1 / 200.0
    assert {r["bc"] for r in reqs} == {"soft", "hard"}
    assert all(1 <= r["nrhs"] <= 64 and r["n"] % 2 == 0 and 1024 <= r["n"] <= 65536 for r in reqs)
    soft = sum(r["bc"] == "soft" for r in reqs) / len(reqs)
    assert 0.45 < soft < 0.55


@pytest.mark.parametrize("name", ["ellipse", "ellipse-hard"])
def test_ellipse_workload_is_the_papers(name):
    """Section 3 at p = 8 points per wavelength on the (1, 0.5) ellipse: omega =
    2 pi n / (8 L) with L the perimeter from the complete elliptic integral,
    5313 at n = 32768 (Table 1, first row: 5.3e3, 3.3e4)."""
    spec = inputs.WORKLOADS[name]
    L = 4.0 * sp.ellipe(1.0 - 0.25)
    assert spec["n"] == 32768
    assert abs(spec["omega"] - 2 * np.pi * spec["n"] / (8 * L)) < 0.5
    assert spec["rtol"] == 1e-6 and spec["nrhs"] == 1
