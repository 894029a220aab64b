"""Pins of the oracle's building blocks: Bessel values, curves, Kress weights,
spectral derivative (CPU only)."""
import numpy as np
import pytest
import scipy.integrate as si
import scipy.special as sp

from oracle import geometry, kress, operators


# --- Bessel values (G = (i/4) H0^(1), Section 1) ---------------------------------

def test_bessel_against_mpmath():
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 40
    xs = np.concatenate([np.geomspace(1e-3, 1e4, 60), [7.9, 8.0, 8.1, 25.0, 6143.7]])
    j0, y0, j1, y1 = operators.bessel01(xs)
    for x, a, b, c, d in zip(xs, j0, y0, j1, y1):
        ref = [float(mpmath.besselj(0, x)), float(mpmath.bessely(0, x)),
               float(mpmath.besselj(1, x)), float(mpmath.bessely(1, x))]
        amp = max(1.0, abs(complex(mpmath.hankel1(0, x))))
        amp = min(amp, 1.0) if x > 1 else amp
        scale = np.sqrt(2 / (np.pi * x)) if x > 1 else 1.0
        # absolute error relative to the envelope sqrt(2/(pi x)) of the oscillation
        for got, want in zip([a, b, c, d], ref):
            tol = 3e-15 * max(scale, abs(want)) + 1e-16 * x * scale
            assert abs(got - want) <= max(tol, 1e-15 * abs(want)), (x, got, want)


def test_bessel_wronskian():
    xs = np.geomspace(1e-2, 5e3, 500)
    j0, y0, j1, y1 = operators.bessel01(xs)
    lhs = j1 * y0 - j0 * y1
    np.testing.assert_allclose(lhs, 2.0 / (np.pi * xs), rtol=1e-12)


def test_hankel_matches_amos():
    xs = np.geomspace(1e-2, 3e3, 200)
    h0, h1 = operators.hankel01(xs)
    # a phase error of one ulp of x is inherent at large x: allow ~x * eps relative
    for got, want in [(h0, sp.hankel1(0, xs)), (h1, sp.hankel1(1, xs))]:
        assert np.all(np.abs(got - want) <= (1e-13 + 2e-16 * xs) * np.abs(want))


# --- curves -------------------------------------------------------------------------

CURVES = [
    ("circle", {}),
    ("ellipse", {"a": 1.0, "b": 0.5}),
    ("star", {"a": [0, 0, 0, 0, 0.3], "b": [0] * 5}),
    ("star", {"a": [0.03, -0.02, 0.01], "b": [0.04, 0.0, -0.05]}),
    ("kite", {}),
]


@pytest.mark.parametrize("kind,params", CURVES)
def test_curve_derivatives_by_finite_differences(kind, params):
    n = 64
    eps = 1e-5
    c = geometry.make(kind, n, **params)
    # shift the nodes by +-eps through a phase-shifted evaluation on a fine grid
    big = 64 * 1000
    fine = geometry.make(kind, big, **params)
    # derivative through the fine grid's neighbours (step 2 pi / big)
    step = 2 * np.pi / big
    idx = np.arange(n) * 1000
    dz_fd = (fine.z[(idx + 1) % big] - fine.z[idx - 1]) / (2 * step)
    ddz_fd = (fine.z[(idx + 1) % big] - 2 * fine.z[idx] + fine.z[idx - 1]) / step**2
    np.testing.assert_allclose(c.dz, dz_fd, atol=1e-7)
    np.testing.assert_allclose(c.ddz, ddz_fd, atol=2e-4)
    assert eps > 0


@pytest.mark.parametrize("kind,params", CURVES)
def test_curve_is_counterclockwise(kind, params):
    c = geometry.make(kind, 256, **params)
    h = 2 * np.pi / c.n
    area = 0.5 * h * np.sum(c.z[:, 0] * c.dz[:, 1] - c.z[:, 1] * c.dz[:, 0])
    assert area > 0
    # outward normal: (z - centroid) . n > 0 for star-shaped curves about the centroid
    if kind != "kite":
        assert np.all(np.sum(c.z * c.normal, axis=1) > 0)


def test_perimeters():
    c = geometry.circle(64, radius=2.5)
    assert abs(np.sum(c.speed) * 2 * np.pi / 64 - 2 * np.pi * 2.5) < 1e-12
    # ellipse (1, 0.5): perimeter 4 E(e^2) with the complete elliptic integral
    e = geometry.ellipse(512, 1.0, 0.5)
    per = np.sum(e.speed) * 2 * np.pi / 512
    assert abs(per - 4.0 * sp.ellipe(1 - 0.25)) < 1e-12
    k = geometry.kite(2048)
    per_k = np.sum(k.speed) * 2 * np.pi / 2048
    ref, _ = si.quad(lambda t: np.hypot(-np.sin(t) - 1.3 * np.sin(2 * t), 1.5 * np.cos(t)),
                     0, 2 * np.pi, limit=200, epsabs=1e-13, epsrel=1e-13)
    assert abs(per_k - ref) < 1e-10


# --- Kress weights ------------------------------------------------------------------

@pytest.mark.parametrize("n", [8, 16, 64, 250])
def test_kress_weights_exact_on_trig_polynomials(n):
    R = kress.kress_weights(n)
    t = geometry.nodes(n)
    i = np.arange(n)
    for m in range(-(n // 2) + 1, n // 2):
        for ti in [0, 1, n // 3]:
            s = np.sum(R[(ti - i) % n] * np.exp(1j * m * t))
            want = 0.0 if m == 0 else -(2 * np.pi / abs(m)) * np.exp(1j * m * t[ti])
            assert abs(s - want) < 1e-12, (n, m, ti)


def test_kress_rule_on_analytic_density():
    # int_0^{2pi} ln(4 sin^2(tau/2)) exp(cos tau) dtau = -4 pi sum_{m>=1} I_m(1)/m
    want = -4 * np.pi * sum(sp.iv(m, 1.0) / m for m in range(1, 40))
    errs = {}
    for n in [16, 32, 64]:
        R = kress.kress_weights(n)
        t = geometry.nodes(n)
        errs[n] = abs(np.sum(R[(-np.arange(n)) % n] * np.exp(np.cos(t))) - want)
    # exact up to the interpolation error of exp(cos t), ~ I_{n/2}(1)
    assert 1e-11 < errs[16] < 1e-8
    assert errs[32] < 1e-13 and errs[64] < 1e-13


def test_kress_weights_odd_n_rejected():
    with pytest.raises(ValueError):
        kress.kress_weights(9)


# --- spectral derivative ------------------------------------------------------------

def test_spectral_derivative_exact_and_nyquist():
    n = 32
    t = geometry.nodes(n)
    f = 1 + np.cos(3 * t) - 2j * np.sin(7 * t) + 0.5 * np.exp(-15j * t)
    df = -3 * np.sin(3 * t) - 14j * np.cos(7 * t) + 0.5 * (-15j) * np.exp(-15j * t)
    np.testing.assert_allclose(operators.spectral_derivative(f), df, atol=1e-12)
    # the Nyquist mode cos(n t / 2) has zero derivative at the nodes and is zeroed
    nyq = np.cos(n / 2 * t)
    np.testing.assert_allclose(operators.spectral_derivative(nyq), 0, atol=1e-12)
    # along axis 1 of a matrix
    M = np.stack([f, 2 * f])
    np.testing.assert_allclose(operators.spectral_derivative(M, axis=1), np.stack([df, 2 * df]),
                               atol=1e-12)
