"""Pins of the oracle's GMRES against LU and against brute-force facts."""
import numpy as np

from oracle import geometry, operators, solvers


def test_gmres_finite_termination_distinct_eigenvalues():
    """A diagonalisable matrix with k distinct eigenvalues: GMRES ends in k steps."""
    rng = np.random.default_rng(0)
    n, k = 40, 5
    lam = np.array([1.0, 2.0 + 1j, -0.5j, 3.0, 0.7 - 0.2j])
    d = lam[rng.integers(0, k, n)]
    d[:k] = lam
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))
    A = Q @ np.diag(d) @ Q.conj().T
    f = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    x, its, rel = solvers.gmres(lambda v: A @ v, f, rtol=1e-12, restart=0, maxit=n)
    assert its == k
    assert rel < 1e-12
    np.testing.assert_allclose(x, np.linalg.solve(A, f), rtol=1e-10)


def test_gmres_matches_lu_on_cfie():
    c = geometry.kite(256)
    w = 20.0
    A = operators.soft_matrix(c, w, w)
    f = operators.plane_wave_rhs(c, w, [0.0, 1.0], "soft")
    X, its, rel = solvers.gmres_columns(lambda v: A @ v, f, rtol=1e-13, restart=0, maxit=256)
    ref = solvers.lu_solve(A, f)
    assert np.all(rel <= 1e-13)
    assert np.linalg.norm(X - ref) / np.linalg.norm(ref) < 1e-12


def test_gmres_restarted_converges_and_counts():
    c = geometry.fourier_star(200, [0, 0, 0, 0, 0.3], [0] * 5)
    w = 30.0
    A = operators.hard_matrix(c, w, w)
    f = operators.plane_wave_rhs(c, w, [0.3], "hard")[:, 0]
    x_full, its_full, _ = solvers.gmres(lambda v: A @ v, f, rtol=1e-8, restart=0, maxit=400)
    x_r, its_r, rel_r = solvers.gmres(lambda v: A @ v, f, rtol=1e-8, restart=10, maxit=400)
    assert rel_r <= 1e-8
    assert its_r >= its_full          # restarting never helps GMRES's residual
    ref = np.linalg.solve(A, f)
    assert np.linalg.norm(x_r - ref) / np.linalg.norm(ref) < 1e-6


def test_gmres_zero_rhs():
    x, its, rel = solvers.gmres(lambda v: v, np.zeros(5, complex))
    assert its == 0 and rel == 0.0 and not np.any(x)


def test_block_gmres_one_column_is_gmres():
    """With one right-hand side the block Krylov space is the ordinary one:
    the same iteration count and solution as GMRES."""
    n, w = 256, 12.0
    c = geometry.make("kite", n)
    A = operators.soft_matrix(c, w, w)
    f = operators.plane_wave_rhs(c, w, [0.3], "soft")
    x1, it1, _ = solvers.gmres(lambda v: A @ v, f[:, 0], rtol=1e-10, restart=100)
    X2, it2, rel2 = solvers.block_gmres(lambda V: A @ V, f, rtol=1e-10, restart=100)
    assert it2 == it1 and rel2[0] <= 1e-10
    assert np.linalg.norm(X2[:, 0] - x1) < 1e-8 * np.linalg.norm(x1)


def test_block_gmres_many_columns_against_lu():
    """64 plane waves on one kite: every column meets rtol, the solutions equal
    LU, and the shared space needs no more block steps than the slowest
    column needs alone (it contains each column's Krylov space)."""
    n, w, s = 512, 30.0, 64
    c = geometry.make("kite", n)
    A = operators.soft_matrix(c, w, w)
    F = operators.plane_wave_rhs(c, w, 2 * np.pi * np.arange(s) / s, "soft")
    X, its, rel = solvers.block_gmres(lambda V: A @ V, F, rtol=1e-10, restart=60)
    assert np.all(rel <= 1e-10)
    ref = solvers.lu_solve(A, F)
    assert np.max(np.abs(X - ref)) < 1e-8 * np.max(np.abs(ref))
    _, its1, _ = solvers.gmres_columns(lambda v: A @ v, F, rtol=1e-10, restart=200)
    assert its <= its1.max()


def test_block_gmres_rank_deficient_block():
    """Repeated directions and a zero right-hand side make the residual block
    rank deficient: every column still converges, equal columns give equal
    solutions and the zero column gives zero."""
    n, w = 512, 32.0
    c = geometry.make("kite", n)
    A = operators.soft_matrix(c, w, w)
    F = operators.plane_wave_rhs(c, w, [0.0, 0.0, 1.0, 2.0, 1.0], "soft")
    F[:, 4] = 0.0
    X, its, rel = solvers.block_gmres(lambda V: A @ V, F, rtol=1e-10, restart=60)
    assert np.all(rel <= 1e-10)
    assert np.array_equal(X[:, 0], X[:, 1]) or np.max(np.abs(X[:, 0] - X[:, 1])) < 1e-12
    assert not np.any(X[:, 4])
    ref = solvers.lu_solve(A, F)
    assert np.max(np.abs(X - ref)) < 1e-8 * np.max(np.abs(ref))
