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
* ``block_gmres`` -- block GMRES over all right-hand sides at once (one
  shared Krylov space; block Gram-Schmidt twice, QR of each new block, the
  block Hessenberg least-squares problem solved directly).
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


def block_gmres(matmat, F, rtol=1e-6, restart=40, maxit=500):
    """Block GMRES over all columns of F at once: one Krylov space
    span{R, A R, A^2 R, ...} shared by the s right-hand sides (the variant of
    the Arnoldi step listed after the preconditioner among the next steps).

    Block Arnoldi with block classical Gram-Schmidt applied twice and a QR of
    each new block; the (m+1)s x ms block Hessenberg least-squares problem
    min ||E1 B - Hbar Y||_F is solved directly each step, its column residuals
    giving the convergence test ||f_k - A x_k|| <= rtol ||f_k|| for every k.
    matmat(V) returns A V.  Returns (X, block iterations, relative residuals
    computed from the final X).  Restarted every `restart` block steps.
    """
    F = np.asarray(F, dtype=np.complex128)
    n, s = F.shape
    X = np.zeros_like(F)
    fn = np.linalg.norm(F, axis=0)
    fn[fn == 0.0] = 1.0
    its = 0
    while True:
        R = F - matmat(X)
        if np.all(np.linalg.norm(R, axis=0) <= rtol * fn) or its >= maxit:
            return X, its, np.linalg.norm(R, axis=0) / fn
        V0, B = np.linalg.qr(R)
        Vs = [V0]
        Hcols = []                                      # block columns of Hbar
        Y = None
        for k in range(restart):
            W = matmat(Vs[-1])
            Vk = np.concatenate(Vs, axis=1)
            h = Vk.conj().T @ W
            W = W - Vk @ h
            h2 = Vk.conj().T @ W                        # second pass (CGS2)
            W = W - Vk @ h2
            h = h + h2
            Q, Rk = np.linalg.qr(W)
            Vs.append(Q)
            col = np.zeros(((k + 2) * s, s), dtype=np.complex128)
            col[:(k + 1) * s] = h
            col[(k + 1) * s:] = Rk
            Hcols.append(col)
            its += 1
            Hbar = np.zeros(((k + 2) * s, (k + 1) * s), dtype=np.complex128)
            for j, c in enumerate(Hcols):
                Hbar[:c.shape[0], j * s:(j + 1) * s] = c
            G = np.zeros(((k + 2) * s, s), dtype=np.complex128)
            G[:s] = B
            Y = np.linalg.lstsq(Hbar, G, rcond=None)[0]
            res = np.linalg.norm(G - Hbar @ Y, axis=0)
            if np.all(res <= rtol * fn) or its >= maxit:
                break
        X = X + np.concatenate(Vs[:len(Hcols)], axis=1) @ Y
