"""Pins of the oracle's CFIE operators and solves against closed forms
(unit disk eigenvalues, Fourier-Bessel series, interior point source,
spectral convergence).  CPU only."""
import numpy as np
import pytest

from oracle import field, geometry, kress, operators, solvers
from tests import closed_forms as cf


def _circulant_eigs(row, t, ms):
    return np.array([np.sum(row * np.exp(1j * m * t)) for m in ms])


@pytest.mark.parametrize("w,n", [(64.0, 1024), (10.0, 128)])
def test_disk_layer_eigenvalues(w, n):
    """S, D, D', N on the unit circle against the addition-theorem eigenvalues."""
    c = geometry.circle(n)
    R = kress.kress_weights(n)
    rows = np.array([0])
    ms = np.arange(-int(w) - 30, int(w) + 31)
    S_ex, D_ex, N_ex = cf.disk_layer_eigenvalues(ms, w)
    S = operators.layer_rows(c, w, rows, "S", R)[0]
    D = operators.layer_rows(c, w, rows, "D", R)[0]
    Dp = operators.layer_rows(c, w, rows, "Dp", R)[0]
    for got, want in [(S, S_ex), (D, D_ex), (Dp, D_ex)]:
        lam = _circulant_eigs(got, c.t, ms)
        assert np.max(np.abs(lam - want)) < 1e-12 * max(1.0, np.max(np.abs(want)))
    if n <= 1024:
        Sfull = operators._blocked(c, w, "S", R)
        N = operators.hypersingular_matrix(c, w, Sfull)
        lam = _circulant_eigs(N[0], c.t, ms)
        assert np.max(np.abs(lam - N_ex) / np.abs(N_ex)) < 1e-11


@pytest.mark.parametrize("bc", ["soft", "hard"])
def test_disk_cfie_eigenvalues(bc):
    w, n = 64.0, 1024
    c = geometry.circle(n)
    A = operators.cfie_matrix(c, w, w, bc)
    ms = np.arange(-94, 95)
    lam = _circulant_eigs(A[0], c.t, ms)
    want = cf.disk_soft_eigenvalue(ms, w, w) if bc == "soft" else cf.disk_hard_eigenvalue(ms, w, w)
    assert np.max(np.abs(lam - want) / np.abs(want)) < 1e-12
    # circulant: every row is the first row shifted
    np.testing.assert_allclose(A[5], np.roll(A[0], 5), atol=1e-13)


@pytest.mark.parametrize("bc", ["soft", "hard"])
def test_disk_plane_wave_series(bc):
    """Unit circle, w = 64, n = 1024, d = (1, 0): LU solution and field at r = 2."""
    w, n = 64.0, 1024
    c = geometry.circle(n)
    A = operators.cfie_matrix(c, w, w, bc)
    f = operators.plane_wave_rhs(c, w, [0.0], bc)
    q = solvers.lu_solve(A, f)[:, 0]
    pts = cf.ring(2.0, 24)
    u = field.scattered_field(c, w, w, bc, q, pts)
    u_ex = cf.disk_scattered(w, 0.0, pts, bc)
    assert cf.rel(u, u_ex) < 1e-11
    # boundary density against the modal solution q_m = f_m / lambda_m
    fm = np.fft.fft(f[:, 0]) / n
    ms = np.fft.fftfreq(n, 1.0 / n)
    lam = cf.disk_soft_eigenvalue(ms, w, w) if bc == "soft" else cf.disk_hard_eigenvalue(ms, w, w)
    keep = np.abs(ms) <= w + 30
    qm = np.fft.fft(q) / n
    assert np.max(np.abs(qm[keep] - fm[keep] / lam[keep])) < 1e-12 * np.max(np.abs(qm))


@pytest.mark.parametrize("bc", ["soft", "hard"])
@pytest.mark.parametrize("kind,params,w,n", [
    ("star", {"a": [0, 0, 0, 0, 0.3], "b": [0] * 5}, 16.0, 512),
    ("kite", {}, 16.0, 512),
    ("ellipse", {"a": 1.0, "b": 0.5}, 20.0, 400),
])
def test_interior_point_source(bc, kind, params, w, n):
    """Boundary data -G(., x0), x0 inside: the scattered field is -G(x, x0)."""
    x0 = np.array([0.1, 0.05])
    c = geometry.make(kind, n, **params)
    A = operators.cfie_matrix(c, w, w, bc)
    f = operators.point_source_rhs(c, w, x0, bc)
    q = solvers.lu_solve(A, f)
    pts = cf.ring(3.0, 32)
    u = field.scattered_field(c, w, w, bc, q, pts)
    assert cf.rel(u, -cf.green(w, pts, x0)) < 1e-10


def test_spectral_convergence_star():
    """Error against the point-source field drops geometrically as n doubles."""
    w = 32.0
    x0 = np.array([0.1, 0.05])
    pts = cf.ring(3.0, 16)
    errs = []
    for n in [96, 128, 192, 256, 384]:
        c = geometry.fourier_star(n, [0, 0, 0, 0, 0.3], [0] * 5)
        A = operators.soft_matrix(c, w, w)
        q = solvers.lu_solve(A, operators.point_source_rhs(c, w, x0, "soft"))
        errs.append(cf.rel(field.scattered_field(c, w, w, "soft", q, pts), -cf.green(w, pts, x0)))
    errs = np.array(errs)
    assert errs[0] > 1e-5                       # under-resolved start
    assert np.all(np.diff(np.log(errs[:4])) < -1.0)   # geometric decrease
    assert errs[-1] < 1e-11


def test_row_sampling_matches_full_matrix():
    c = geometry.kite(256)
    A = operators.soft_matrix(c, 12.0, 12.0)
    rows = np.array([0, 17, 255])
    np.testing.assert_allclose(operators.soft_rows(c, 12.0, 12.0, rows), A[rows], atol=1e-15)


def test_hard_plane_wave_rhs_is_normal_derivative():
    c = geometry.kite(64)
    w, th = 5.0, 0.7
    f = operators.plane_wave_rhs(c, w, [th], "hard")[:, 0]
    eps = 1e-6
    d = np.array([np.cos(th), np.sin(th)])
    p = c.z + eps * c.normal
    m = c.z - eps * c.normal
    fd = (np.exp(1j * w * p @ d) - np.exp(1j * w * m @ d)) / (2 * eps)
    np.testing.assert_allclose(f, -fd, atol=1e-7)
