"""Pins of the oracle's directional preconditioner (Section 2) and of the
arclength sampling it needs.  CPU only.

What fixes each part independently of the code under test:
* arclength sampling: the ellipse perimeter is a complete elliptic integral;
  the circle's arclength parametrisation is its usual one; the Kress-Nystrom
  CFIE on the resampled ellipse reproduces the interior point-source field
  (which checks z, z' and z'' of the reparametrisation);
* the entry function: on the nodes it equals the oracle's matrix entries;
* the flat block B_l: on the straight sides of a stadium it is the oracle's
  CFIE matrix (itself pinned by closed forms), diagonal included;
* Chebyshev interpolation: exact on polynomials of degree < m_c;
* eq. (aug) / (fac) / (esol): with the exact T and W the five factors solve
  (B + U E U^t) q = f exactly, and so does the augmented 3 x 3 block system;
* the block coefficients e_ij: the Chebyshev route of eq. (entry) agrees with
  the least-squares constant over the block's own nodes, which it approximates;
* the preconditioner's effect: GMRES iterations drop on the p = 8 ellipse, as
  in Table 1 (n_n 47 -> n_p 14 at n = 32768; the size here is 2048) and Table 3
  (sound hard, 38 -> 15).
"""
import numpy as np
import pytest
import scipy.special as sp

from oracle import directional, field, geometry, operators, solvers
from tests import closed_forms as cf


@pytest.fixture(scope="module")
def ellipse_arc():
    return geometry.Arclength("ellipse", a=1.0, b=0.5)


def test_arclength_perimeter_and_speed(ellipse_arc):
    assert abs(ellipse_arc.L - 4.0 * sp.ellipe(1.0 - 0.25)) < 1e-13
    c = ellipse_arc.curve(512)
    assert np.ptp(c.speed) < 1e-12
    assert abs(c.speed[0] - ellipse_arc.L / (2 * np.pi)) < 1e-12
    circ = geometry.Arclength("circle").curve(64)
    ref = geometry.circle(64)
    for a, b in [(circ.z, ref.z), (circ.dz, ref.dz), (circ.ddz, ref.ddz)]:
        assert np.max(np.abs(a - b)) < 1e-13


@pytest.mark.parametrize("bc", ["soft", "hard"])
def test_arclength_curve_point_source(ellipse_arc, bc):
    """The CFIE on the arclength-sampled ellipse: interior point source."""
    w, n = 20.0, 400
    c = ellipse_arc.curve(n)
    x0 = np.array([0.1, 0.05])
    A = operators.cfie_matrix(c, w, w, bc)
    q = solvers.lu_solve(A, operators.point_source_rhs(c, w, x0, bc))
    pts = cf.ring(3.0, 32)
    u = field.scattered_field(c, w, w, bc, q, pts)
    assert cf.rel(u, -cf.green(w, pts, x0)) < 1e-10


def test_curvature_of_the_ellipse(ellipse_arc):
    """kappa = a b / (a^2 sin^2 t + b^2 cos^2 t)^(3/2) at the arclength nodes."""
    n = 256
    c = ellipse_arc.curve(n)
    t = ellipse_arc.t_of_s(ellipse_arc.L * np.arange(n) / n)
    want = 0.5 / (np.sin(t) ** 2 + 0.25 * np.cos(t) ** 2) ** 1.5
    assert np.max(np.abs(directional.curvature(c) - want)) < 1e-12


def test_partition_rules(ellipse_arc):
    q, p = 4, 8
    c = ellipse_arc.curve(4**q * p)
    segs = directional.partition(c, q, p, m_leaf=2)
    firsts = np.array([f for f, _ in segs])
    counts = np.array([2**l * p for _, l in segs])
    assert counts.sum() == c.n and firsts[0] == 0
    assert np.all(firsts[1:] == np.cumsum(counts)[:-1])        # ordered, contiguous
    kappa = np.abs(directional.curvature(c))
    for f, l in segs:
        cmax = kappa[f:f + 2**l * p].max()
        assert 2.0**l <= 2.0**q / np.sqrt(cmax) or 2.0**l <= 2   # each leaf stops
    # the ellipse (curvature 0.5 .. 4) is split once near its tips only
    assert {l for _, l in segs} == {q - 1, q}


def test_frequency_grid_rounding():
    w, l = 100.0, 2
    K = directional.frequency_grid(l, w)
    assert K.size == 9 and K[0] == -w and K[-1] == w
    for i, k in enumerate(K):
        assert directional.round_to_grid(k, l, w) == i
    step = K[1] - K[0]
    # ties go away from zero
    assert directional.round_to_grid(0.5 * step, l, w) == 5
    assert directional.round_to_grid(-0.5 * step, l, w) == 3
    assert directional.round_to_grid(0.49 * step, l, w) == 4


def test_chebyshev_interpolation_exact_on_polynomials():
    m = 10
    xc, wc = directional.chebyshev_points(m, 0.3, 1.7)
    x = np.linspace(0.3, 1.7, 57)
    I = directional.interpolation_matrix(xc, wc, x)
    assert np.allclose(I.sum(axis=1), 1.0, atol=1e-14)      # constants: e_ij of a constant
    for deg in range(m):
        assert np.max(np.abs(I @ xc**deg - x**deg)) < 1e-11 * max(1.0, 1.7**deg)


def test_entry_function_matches_matrix(ellipse_arc):
    n, w = 512, 40.0
    c = ellipse_arc.curve(n)
    A = operators.soft_matrix(c, w, w)
    rows = np.arange(0, n, 7)
    cols = (rows + 3 + rows // 5) % n
    with np.errstate(invalid="ignore", divide="ignore"):     # only the paired entries are used
        got = directional.soft_entries(n, w, w, c.z[rows], c.z[cols], c.normal_unscaled[cols],
                                       c.speed[cols], c.t[rows], c.t[cols])
    assert np.max(np.abs(np.diag(got) - A[rows, cols])) < 1e-13 * np.max(np.abs(A))
    # the flat block: its off-diagonal entries are the entry function on a line
    B = directional.flat_block(n, 2, 8, w, w, ellipse_arc.L)
    g = ellipse_arc.L / (2 * np.pi)
    s = np.arange(32) * ellipse_arc.L / n
    zl = np.stack([s, np.zeros_like(s)], axis=1)
    nul = np.tile([0.0, -g], (32, 1))
    tl = 2 * np.pi * np.arange(32) / n
    a, b = np.array([0, 5, 31]), np.array([9, 4, 0])
    with np.errstate(invalid="ignore", divide="ignore"):
        ref = directional.soft_entries(n, w, w, zl[a], zl[b], nul[b], np.full(3, g), tl[a], tl[b])
    assert np.max(np.abs(np.diag(ref) - B[a, b])) < 1e-13 * np.max(np.abs(B))


@pytest.fixture(scope="module")
def small_precond(ellipse_arc):
    q, p = 3, 8
    n = 4**q * p
    w = 2 * np.pi * (n / p) / ellipse_arc.L
    return directional.Directional(ellipse_arc, q, p, w)


def test_exact_factorisation_solves_the_approximation(small_precond):
    """Eq. (esol) with the exact T and W = E + T: q = (B + U E U^t)^-1 f."""
    P = small_precond
    rng = np.random.default_rng(5)
    f = rng.standard_normal(P.n) + 1j * rng.standard_normal(P.n)
    T, Ws = P.exact_solver()
    q = P.apply(f, T=T, W_solve=Ws)
    ref = np.linalg.solve(P.approximation(), f)
    assert np.linalg.norm(q - ref) < 1e-10 * np.linalg.norm(ref)
    # the augmented system (eq. aug) has the same first component
    U, B, E = P.dense_U(), P.dense_B(), P.E.toarray()
    nk = E.shape[0]
    Z = np.zeros
    aug = np.block([[B, U, Z((P.n, nk))],
                    [U.T, Z((nk, nk)), np.eye(nk)],
                    [Z((nk, P.n)), np.eye(nk), E]])
    sol = np.linalg.solve(aug, np.concatenate([f, np.zeros(2 * nk)]))
    assert np.linalg.norm(sol[:P.n] - ref) < 1e-9 * np.linalg.norm(ref)


def test_approximation_captures_the_operator(small_precond, ellipse_arc):
    """M ~ B + U E U^t (eq. Mapp): an aggressive rank-1-per-block form, but
    far closer to M than B alone."""
    P = small_precond
    A = operators.soft_matrix(P.curve, P.omega, P.eta)
    e_full = np.linalg.norm(A - P.approximation(), 2) / np.linalg.norm(A, 2)
    e_diag = np.linalg.norm(A - P.dense_B(), 2) / np.linalg.norm(A, 2)
    assert e_full < 0.5 * e_diag


def test_preconditioner_cuts_gmres_iterations(ellipse_arc):
    """Table 1 (p = 8, ellipse): the directional preconditioner cuts the GMRES
    iteration count several-fold; here n = 2048 (q = 4)."""
    q, p = 4, 8
    n = 4**q * p
    w = 2 * np.pi * (n / p) / ellipse_arc.L
    P = directional.Directional(ellipse_arc, q, p, w)
    A = operators.soft_matrix(P.curve, w, w)
    f = operators.plane_wave_rhs(P.curve, w, [0.0], "soft")[:, 0]
    _, it0, r0 = directional.preconditioned_gmres(A, None, f, rtol=1e-6)
    x, it1, r1 = directional.preconditioned_gmres(A, P.apply, f, rtol=1e-6)
    assert r0 <= 1e-6 and r1 <= 1e-6
    assert it1 <= 0.6 * it0
    assert np.linalg.norm(x - np.linalg.solve(A, f)) < 1e-5 * np.linalg.norm(x)


def test_chebyshev_coefficients_match_the_nodal_least_squares(ellipse_arc):
    """e_ij of eq. (entry) (m_c^2 Chebyshev samples) against the least-squares
    constant over the nodes of the block (the mean of M~_ij)."""
    q, p = 3, 8
    n = 4**q * p
    w = 2 * np.pi * (n / p) / ellipse_arc.L
    A = operators.soft_matrix(ellipse_arc.curve(n), w, w)
    Pc = directional.Directional(ellipse_arc, q, p, w)
    Pn = directional.Directional(ellipse_arc, q, p, w, A=A, e_from="nodes")
    ec, en = Pc.E.toarray(), Pn.E.toarray()
    nz = np.abs(en) > 0
    assert np.array_equal(nz, np.abs(ec) > 0)                  # same wave-number pairs
    rel = np.abs(ec[nz] - en[nz]) / np.abs(en[nz])
    assert np.median(rel) < 1e-3 and rel.max() < 5e-2         # worst: adjacent segments


def test_hard_preconditioner(ellipse_arc):
    """Sound hard (eq. 2): the factors solve B + U E U^t exactly, and GMRES
    needs fewer iterations with the preconditioner (Table 3)."""
    q, p = 4, 8
    n = 4**q * p
    w = 2 * np.pi * (n / p) / ellipse_arc.L
    c = ellipse_arc.curve(n)
    A = operators.hard_matrix(c, w, w)
    P = directional.Directional(ellipse_arc, q, p, w, bc="hard", A=A)
    f = operators.plane_wave_rhs(c, w, [0.0], "hard")[:, 0]
    T, Ws = P.exact_solver()
    ref = np.linalg.solve(P.approximation(), f)
    assert np.linalg.norm(P.apply(f, T=T, W_solve=Ws) - ref) < 1e-10 * np.linalg.norm(ref)
    _, it0, r0 = directional.preconditioned_gmres(A, None, f, rtol=1e-6)
    x, it1, r1 = directional.preconditioned_gmres(A, P.apply, f, rtol=1e-6)
    assert r0 <= 1e-6 and r1 <= 1e-6 and it1 < it0


def _stadium(n, ell, rho):
    """A stadium (straight sides of length ell joined by half circles of radius
    rho), counter-clockwise, sampled equispaced in arclength with speed
    L / (2 pi); its first side runs along y = -rho from x = -ell / 2."""
    L = 2 * ell + 2 * np.pi * rho
    g = L / (2 * np.pi)
    s = L * np.arange(n) / n
    z, tan, curv = np.zeros((n, 2)), np.zeros((n, 2)), np.zeros((n, 2))
    for k, sk in enumerate(s):
        if sk < ell:
            z[k], tan[k] = (-ell / 2 + sk, -rho), (1.0, 0.0)
        elif sk < ell + np.pi * rho:
            f = (sk - ell) / rho
            z[k] = (ell / 2 + rho * np.sin(f), -rho * np.cos(f))
            tan[k], curv[k] = (np.cos(f), np.sin(f)), (-np.sin(f) / rho, np.cos(f) / rho)
        elif sk < 2 * ell + np.pi * rho:
            z[k], tan[k] = (ell / 2 - (sk - ell - np.pi * rho), rho), (-1.0, 0.0)
        else:
            f = (sk - 2 * ell - np.pi * rho) / rho
            z[k] = (-ell / 2 - rho * np.sin(f), rho * np.cos(f))
            tan[k], curv[k] = (-np.cos(f), -np.sin(f)), (np.sin(f) / rho, -np.cos(f) / rho)
    return geometry.from_samples(z, g * tan, g * g * curv), L


@pytest.mark.parametrize("level", [2, 4])
def test_flat_block_is_the_operator_on_a_straight_side(level):
    """B_l of the soft operator is the CFIE matrix of a boundary that really is
    straight there: on a stadium sampled in arclength, the rows and columns of
    the nodes of one straight side give the whole flat block, diagonal included
    (the matrix of operators.soft_matrix is pinned on its own by closed forms)."""
    p, n = 8, 512
    c, L = _stadium(n, 1.0, 1.0 / np.pi)       # sides of n / 4 nodes, L = 4
    w = 2 * np.pi * (n / p) / L
    A = operators.soft_matrix(c, w, w)
    m = 2**level * p
    assert m <= n // 4
    B = directional.flat_block(n, level, p, w, w, L)
    blk = A[:m, :m]
    assert np.max(np.abs(B - blk)) < 1e-13 * np.max(np.abs(blk))
    # the same block further along the side (Toeplitz) and on the other side
    for o in sorted({n // 4 - m, n // 2, 3 * n // 4 - m}):
        assert np.max(np.abs(B - A[o:o + m, o:o + m])) < 1e-13 * np.max(np.abs(blk))


@pytest.mark.parametrize("bc", ["soft", "hard"])
def test_iteration_count_script(bc):
    """oracle.iteration_counts at the smallest size: the setting of Section 3
    (omega from p = 8 points per wavelength) and fewer iterations with the
    preconditioner than without."""
    from oracle import iteration_counts
    n, omega, n_n, n_p = iteration_counts.counts(3, bc, eta_factor=0.5)
    L = geometry.Arclength("ellipse", a=1.0, b=0.5).L
    assert n == 512 and abs(omega - 2 * np.pi * 64 / L) < 1e-9
    assert 0 < n_p <= n_n


def test_preconditioner_on_a_curve_with_non_planar_leaves():
    """The kite's tip (curvature up to ~11.7) forces segments down to level 1,
    the non-planar leaves of Section 2.1 (m_leaf = 2); the preconditioner still
    solves its approximation exactly and cuts the GMRES iterations."""
    arc = geometry.Arclength("kite")
    q, p = 3, 8
    n = 4**q * p
    w = 2 * np.pi * (n / p) / arc.L
    P = directional.Directional(arc, q, p, w, eta=0.5 * w)
    assert P.level.min() <= 1 and P.level.max() == q
    A = operators.soft_matrix(P.curve, w, 0.5 * w)
    f = operators.plane_wave_rhs(P.curve, w, [0.0], "soft")[:, 0]
    T, Ws = P.exact_solver()
    ref = np.linalg.solve(P.approximation(), f)
    assert np.linalg.norm(P.apply(f, T=T, W_solve=Ws) - ref) < 1e-10 * np.linalg.norm(ref)
    _, it0, _ = directional.preconditioned_gmres(A, None, f, rtol=1e-6)
    _, it1, r1 = directional.preconditioned_gmres(A, P.apply, f, rtol=1e-6)
    assert r1 <= 1e-6 and it1 < it0
