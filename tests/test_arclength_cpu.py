"""Parity of the library's arclength sampling (cfie_arclength_samples, host
code) with the oracle's (geometry.Arclength, a different construction: Fourier
integration of the speed), and with closed forms.  CPU only: the call needs no
GPU.

Section 2 samples the boundary at points equispaced in arclength; the returned
derivatives are with respect to sigma = 2 pi s / L, so the speed is L / (2 pi)."""
import numpy as np
import pytest
import scipy.special as sp

from oracle import geometry
from paper_1408_1578_gb300 import build, cfie

CURVES = [
    ("circle", {"radius": 1.3}),
    ("ellipse", {"a": 1.0, "b": 0.5}),
    ("kite", {}),
    ("star", {"a": [0, 0, 0, 0, 0.3], "b": [0.02, 0, -0.04, 0, 0]}),
    ("star", {"a": [0.03, -0.02, 0.04], "b": [0.01, 0.05, -0.03]}),
]


@pytest.fixture(scope="module", autouse=True)
def lib():
    build.build()
    return cfie.load()


@pytest.mark.parametrize("n", [512, 1002])
@pytest.mark.parametrize("kind,params", CURVES)
def test_matches_the_oracle(kind, params, n):
    z, dz, ddz, L = cfie.arclength_samples(kind, n, **params)
    arc = geometry.Arclength(kind, **params)
    c = arc.curve(n)
    assert abs(L - arc.L) < 1e-13 * arc.L
    for got, want, tol in [(z, c.z, 1e-13), (dz, c.dz, 1e-12), (ddz, c.ddz, 1e-11)]:
        assert np.max(np.abs(got - want)) < tol * np.max(np.abs(want))


@pytest.mark.parametrize("kind,params", CURVES)
def test_constant_speed(kind, params):
    _, dz, _, L = cfie.arclength_samples(kind, 256, **params)
    assert np.max(np.abs(np.hypot(dz[:, 0], dz[:, 1]) - L / (2 * np.pi))) < 1e-12 * L


def test_closed_forms():
    # circle: arclength is the angle times the radius
    R, n = 1.3, 64
    z, dz, ddz, L = cfie.arclength_samples("circle", n, radius=R)
    s = 2 * np.pi * np.arange(n) / n
    assert abs(L - 2 * np.pi * R) < 1e-13
    assert np.max(np.abs(z - R * np.stack([np.cos(s), np.sin(s)], 1))) < 1e-14
    assert np.max(np.abs(dz - R * np.stack([-np.sin(s), np.cos(s)], 1))) < 1e-14
    assert np.max(np.abs(ddz + z)) < 1e-14
    # ellipse perimeter: complete elliptic integral of the second kind
    L = cfie.arclength_samples("ellipse", 64, a=1.0, b=0.5)[3]
    assert abs(L - 4 * sp.ellipe(0.75)) < 1e-13
    # equal arcs: a chord of an arc ds with curvature k is ds (1 - (k ds)^2 / 24 + ...)
    z, dz, ddz, L = cfie.arclength_samples("kite", 4096)
    ds = L / 4096
    chords = np.hypot(*np.diff(np.vstack([z, z[:1]]), axis=0).T)
    kappa = np.abs(dz[:, 0] * ddz[:, 1] - dz[:, 1] * ddz[:, 0]) / (L / (2 * np.pi))**3
    assert np.max(np.abs(chords / ds - 1)) < 1.1 * (kappa.max() * ds)**2 / 24


@pytest.mark.parametrize("args", [
    (cfie.CFIE_CURVE_CIRCLE, [1.0], 7),           # odd n
    (cfie.CFIE_CURVE_CIRCLE, [1.0], 6),           # n < 8
    (cfie.CFIE_CURVE_CIRCLE, [0.0], 64),          # radius 0
    (cfie.CFIE_CURVE_ELLIPSE, [1.0, -0.5], 64),   # negative axis
    (cfie.CFIE_CURVE_ELLIPSE, [1.0], 64),         # missing axis
    (cfie.CFIE_CURVE_STAR, [0.1], 64),            # odd parameter count
    (cfie.CFIE_CURVE_STAR, [1.2, 0.0], 64),       # r = 1 + 1.2 cos t reaches 0
    (cfie.CFIE_CURVE_KITE, [1.0], 64),            # the kite takes none
    (cfie.CFIE_CURVE_CIRCLE, [float("nan")], 64),
    (7, [1.0], 64),                               # unknown curve
])
def test_invalid_arguments(lib, args):
    kind, params, n = args
    import ctypes
    par = np.ascontiguousarray(params, dtype=np.float64)
    out = [np.empty((max(n, 1), 2)) for _ in range(3)]
    dp = ctypes.POINTER(ctypes.c_double)
    st = lib.cfie_arclength_samples(kind, par.ctypes.data_as(dp), par.size, n,
                                    *[o.ctypes.data_as(dp) for o in out], None)
    assert st == cfie.CFIE_EINVAL


def test_null_outputs(lib):
    assert lib.cfie_arclength_samples(cfie.CFIE_CURVE_KITE, None, 0, 64, None, None, None,
                                      None) == cfie.CFIE_EINVAL
