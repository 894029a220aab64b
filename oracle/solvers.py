"""Direct and Krylov solves of the discrete CFIE (oracle, test infrastructure only).

Section 1 of the paper: a direct LU solve costs O(n^3); the experiments of
Section 3 use GMRES with relative tolerance 1e-6 and restart 80, zero initial
guess.  The oracle provides both:

* ``lu_solve``  -- numpy.linalg.solve (LAPACK LU with partial pivoting);
* ``gmres``     -- restarted GMRES (Saad & Schultz): Arnoldi with modified
  Gram-Schmidt, Givens rotations on the Hessenberg matrix, the residual norm
  read from the rotated right-hand side, x updated at the end of every cycle
  and the true residual f - A x recomputed at each restart.  Each right-hand
  side is solved independently.
"""
import numpy as np


def lu_solve(A, f):
    return np.linalg.solve(A, f)


def _givens(a, b):
    """Complex Givens rotation (c real, s complex) with
    [c, s; -conj(s), c] [a; b] = [rho; 0]."""
    if b == 0:
        return 1.0, 0.0 + 0.0j
    if a == 0:
        return 0.0, np.conj(b) / abs(b)
    t = np.hypot(abs(a), abs(b))
    c = abs(a) / t
    s = (a / abs(a)) * np.conj(b) / t
    return c, s


def gmres(matvec, f, rtol=1e-6, restart=80, maxit=1000, x0=None):
    """Solve A x = f for one right-hand side.

    matvec(v) returns A v.  restart=0 means unrestarted (one cycle of up to
    maxit steps).  Returns (x, iterations, relative residual ||f - A x|| / ||f||
    computed from the final x).
    """
    f = np.asarray(f, dtype=np.complex128)
    n = f.shape[0]
    x = np.zeros(n, dtype=np.complex128) if x0 is None else np.array(x0, dtype=np.complex128)
    fnorm = np.linalg.norm(f)
    if fnorm == 0.0:
        return np.zeros_like(f), 0, 0.0
    m = maxit if restart in (0, None) else restart
    its = 0
    while True:
        r = f - matvec(x)
        beta = np.linalg.norm(r)
        if beta / fnorm <= rtol or its >= maxit:
            return x, its, beta / fnorm
        V = np.zeros((n, m + 1), dtype=np.complex128)
        H = np.zeros((m + 1, m), dtype=np.complex128)
        cs = np.zeros(m)
        sn = np.zeros(m, dtype=np.complex128)
        g = np.zeros(m + 1, dtype=np.complex128)
        g[0] = beta
        V[:, 0] = r / beta
        k_done = 0
        for k in range(m):
            w = matvec(V[:, k])
            for j in range(k + 1):          # modified Gram-Schmidt
                H[j, k] = np.vdot(V[:, j], w)
                w = w - H[j, k] * V[:, j]
            H[k + 1, k] = np.linalg.norm(w)
            if H[k + 1, k] != 0.0:
                V[:, k + 1] = w / H[k + 1, k]
            for j in range(k):              # earlier rotations
                a, b = H[j, k], H[j + 1, k]
                H[j, k] = cs[j] * a + sn[j] * b
                H[j + 1, k] = -np.conj(sn[j]) * a + cs[j] * b
            cs[k], sn[k] = _givens(H[k, k], H[k + 1, k])
            H[k, k] = cs[k] * H[k, k] + sn[k] * H[k + 1, k]
            H[k + 1, k] = 0.0
            g[k + 1] = -np.conj(sn[k]) * g[k]
            g[k] = cs[k] * g[k]
            its += 1
            k_done = k + 1
            if abs(g[k + 1]) / fnorm <= rtol or its >= maxit:
                break
        # back substitution on the k_done x k_done triangle
        y = np.zeros(k_done, dtype=np.complex128)
        for i in range(k_done - 1, -1, -1):
            y[i] = (g[i] - H[i, i + 1:k_done] @ y[i + 1:]) / H[i, i]
        x = x + V[:, :k_done] @ y


def gmres_columns(matvec, F, rtol=1e-6, restart=80, maxit=1000):
    """GMRES on each column of F independently.  matvec acts on one column."""
    F = np.atleast_2d(np.asarray(F, dtype=np.complex128).T).T
    X = np.zeros_like(F)
    its = np.zeros(F.shape[1], dtype=np.int64)
    rel = np.zeros(F.shape[1])
    for k in range(F.shape[1]):
        X[:, k], its[k], rel[k] = gmres(matvec, F[:, k], rtol, restart, maxit)
    return X, its, rel
