"""Directional preconditioner of Section 2 (oracle, test infrastructure only).

The paper's construction for the sound-soft operator M of eq. 1, on a boundary
sampled at n = 4^q p points equispaced in arclength (p points per
wavelength lambda = 2 pi / omega), followed step by step:

Section 2.1 (data-sparse approximation M ~ B + U E U^t)
  * segments: 2^q pieces of 2^q p points, split in halves until a piece is
    almost-planar (length <= 2^q lambda / sqrt(c), c the largest |curvature| on
    it) or a non-planar leaf (length <= m_l lambda); P_j then holds 2^l_j p
    points and has length 2^l_j lambda;
  * diagonal blocks M_jj ~ B_j: the operator restricted to a straight segment
    of the same length and spacing (same quadrature: here the Kress-Nystrom
    entries of the closed curve's discretisation with the geometry of a line,
    on which the double-layer kernel vanishes);
  * off-diagonal blocks: with c_i, t_i the centre and unit tangent of P_i and
    a_ij = (c_i - c_j) / |c_i - c_j|, the wave numbers k^i_ij = [omega a_ij . t_i]_i
    and k^j_ij = [-omega a_ij . t_j]_j, rounded to the 2^(l+1) + 1 points K_i of
    [-omega, omega] (nearest; ties away from zero), and the partial Fourier
    matrices U_i(x, k) = exp(i k (rho(x) - rho(c_i))) (eq. Ui);
  * M~_ij(x, y) = M_ij(x, y) / (U_i(x, k^i) U_j(y, k^j)) (eq. Mtilde) is sampled
    on Chebyshev grids R_i, R_j of m_c points and
    e_ij = (w_i^+ I_i) M~_ij(R_i, R_j) (I_j^t w_j^t+)  (eq. entry), the
    least-squares constant of the rank-1 form U_i(:, k^i) e_ij U_j(:, k^j)^t;
    E holds e_ij at (k^i_ij, k^j_ij) of block (i, j).

Section 2.2 (preconditioner)
  * S_i = U_i^t B_i^-1 U_i, T_i = S_i^-1; T~ keeps the largest entries of each
    T_i (a fixed multiple of its dimension); W~ = E + the anti-diagonal of T,
    factored by sparse LU;
  * eq. (eapp): from (f, 0, 0), p -= U^t B^-1 q; r += T~ p; (q, p, r) <-
    (B^-1 q, -T~ p, W~^-1 r); p += T~ r; q -= B^-1 U p; return q.
  B^-1 is applied densely (the H-matrix / HSS compression of Section 2.2 is
  out of scope) and U by dense partial Fourier matrices (the FFT is a speed
  device, not a change of result).

The entries of M at points off the nodes (Chebyshev grids) come from the same
Kress-Nystrom entry formula with the weight R_d replaced by its trigonometric
interpolant R(tau), so that on the nodes they are the matrix entries.

Sound hard (eq. 2): the same construction with the nodal least-squares e_ij
and the matrix's own diagonal blocks (see Directional).

Parity: the algebra (eq. aug, fac, esol), the entry function, the Chebyshev
interpolation, the curvature, the partition rules and the e_ij of eq. (entry)
against the least-squares constants over the nodes are pinned by
tests/test_oracle_directional.py, and so is the sound-soft flat B_l, diagonal
included: it equals the CFIE matrix of operators.soft_matrix on the straight
sides of a stadium sampled in arclength.  The sound-hard operator takes the
matrix's own diagonal blocks, pinned with the matrix.
"""
import numpy as np
import scipy.linalg as sla
import scipy.sparse as sps
import scipy.sparse.linalg as spla

from .kress import kress_weights
from .operators import EULER_GAMMA, bessel01


# ---------------------------------------------------------------------------
# geometry of the segments
# ---------------------------------------------------------------------------

def curvature(curve):
    """Signed curvature (z1' z2'' - z2' z1'') / |z'|^3 at the nodes."""
    dz, ddz = curve.dz, curve.ddz
    return (dz[:, 0] * ddz[:, 1] - dz[:, 1] * ddz[:, 0]) / curve.speed**3


def partition(curve, q, p, m_leaf=2):
    """Segments of Section 2.1 as (first node, level l) with 2^l p nodes each.

    The curve must hold n = 4^q p nodes equispaced in arclength.  A piece of
    level l (length 2^l lambda) is kept when 2^l <= 2^q / sqrt(c) (almost
    planar) or 2^l <= m_leaf (non-planar leaf), else split in halves."""
    n = curve.n
    if n != 4**q * p:
        raise ValueError("the partition needs n = 4^q p nodes")
    kappa = np.abs(curvature(curve))
    out = []

    def split(first, level):
        cnt = 2**level * p
        c = kappa[first:first + cnt].max()
        if 2.0**level <= 2.0**q / np.sqrt(c) or 2.0**level <= m_leaf:
            out.append((first, level))
        else:
            split(first, level - 1)
            split(first + cnt // 2, level - 1)

    for k in range(2**q):
        split(k * 2**q * p, q)
    return out


def frequency_grid(level, omega):
    """K_i: 2^(l+1) + 1 equispaced wave numbers on [-omega, omega]."""
    return np.linspace(-omega, omega, 2**(level + 1) + 1)


def round_to_grid(k, level, omega):
    """Index of [k]_i, the gridpoint of K_i nearest to k (ties away from zero)."""
    m = 2**(level + 1)
    v = (k + omega) * m / (2.0 * omega)          # fractional index
    idx = np.floor(v + 0.5) if k >= 0 else np.ceil(v - 0.5)
    return int(min(max(idx, 0), m))


def chebyshev_points(m, a, b):
    """First-kind Chebyshev points of [a, b] and their barycentric weights."""
    k = np.arange(m)
    th = (2 * k + 1) * np.pi / (2 * m)
    x = 0.5 * (a + b) + 0.5 * (b - a) * np.cos(th)
    w = (-1.0) ** k * np.sin(th)
    return x, w


def interpolation_matrix(x_nodes, w, x):
    """Barycentric Lagrange interpolation from the Chebyshev nodes to x."""
    d = x[:, None] - x_nodes[None, :]
    exact = np.isclose(d, 0.0, atol=1e-14)
    d = np.where(exact, 1.0, d)
    T = w[None, :] / d
    T /= T.sum(axis=1, keepdims=True)
    rows = np.nonzero(exact.any(axis=1))[0]
    for r in rows:
        T[r] = exact[r].astype(float)
    return T


# ---------------------------------------------------------------------------
# entries of M (sound-soft, eq. 1) at arbitrary curve points
# ---------------------------------------------------------------------------

def kress_weight_function(n, tau):
    """R(tau), the trigonometric interpolant of the Kress weights R_d:
    R(2 pi d / n) = R_d."""
    N = n // 2
    tau = np.asarray(tau, dtype=np.float64)
    m = np.arange(1, N, dtype=np.float64)
    acc = np.cos(np.multiply.outer(tau, m)) @ (1.0 / m)
    return -(2.0 * np.pi / N) * acc - (np.pi / N**2) * np.cos(N * tau)


def soft_entries(n, omega, eta, zx, zy, nuy, speedy, tx, ty):
    """Nystrom entries R(tx - ty) K1 + h K2 of the sound-soft CFIE for target
    points zx (parameters tx) and source points zy (ty, normals nuy, speeds
    speedy), all pairs distinct: K = L - i eta M, K1 = L1 - i eta M1."""
    h = 2.0 * np.pi / n
    diff = zx[:, None, :] - zy[None, :, :]
    r = np.hypot(diff[..., 0], diff[..., 1])
    j0, y0, j1, y1 = bessel01(omega * r)
    c = (diff[..., 0] * nuy[None, :, 0] + diff[..., 1] * nuy[None, :, 1]) / r
    K = 0.25j * omega * (j1 + 1j * y1) * c - 1j * eta * 0.25j * (j0 + 1j * y0) * speedy[None, :]
    K1 = (-(omega / (4 * np.pi)) * j1 * c
          + 1j * eta * (1.0 / (4 * np.pi)) * j0 * speedy[None, :])
    dt = tx[:, None] - ty[None, :]
    logf = np.log(4.0 * np.sin(0.5 * dt) ** 2)
    return kress_weight_function(n, dt) * K1 + h * (K - K1 * logf)


def flat_single_layer(n, level, p, omega, L):
    """The single-layer (S) Kress-Nystrom block on a straight segment of 2^l p
    nodes with the spacing and speed L / (2 pi) of the curve's arclength
    discretisation."""
    cnt = 2**level * p
    h = 2.0 * np.pi / n
    g = L / (2.0 * np.pi)
    R = kress_weights(n)
    a = np.arange(cnt)
    d = a[:, None] - a[None, :]
    off = d != 0
    r_safe = np.where(off, np.abs(d) * h * g, 1.0)
    j0, y0, _, _ = bessel01(omega * r_safe)
    M = 0.25j * (j0 + 1j * y0) * g
    M1 = -(1.0 / (4 * np.pi)) * j0 * g
    logf = np.log(4.0 * np.sin(np.pi * np.where(off, d, 1) / n) ** 2)
    S = R[d % n] * M1 + h * (M - M1 * logf)
    m1 = -g / (4 * np.pi)
    m2 = (0.25j - EULER_GAMMA / (2 * np.pi) - np.log(omega * g / 2.0) / (2 * np.pi)) * g
    S[~off] = R[0] * m1 + h * m2
    return S


def flat_block(n, level, p, omega, eta, L):
    """B_l: the sound-soft entries on a straight segment of 2^l p nodes with
    the spacing and speed L / (2 pi) of the curve's arclength discretisation
    (the double-layer kernel and the curvature term vanish on a line)."""
    B = -1j * eta * flat_single_layer(n, level, p, omega, L)
    B[np.diag_indices(B.shape[0])] += 0.5
    return B


# ---------------------------------------------------------------------------
# the preconditioner
# ---------------------------------------------------------------------------

class Directional:
    """Setup of Section 2 on an arclength-sampled curve (`arc`:
    geometry.Arclength, n = 4^q p nodes).

    bc = "soft" builds E from Chebyshev samples of the entry function (eq.
    entry).  For bc = "hard" the Maue-discretised N has no pointwise kernel at
    off-node points, so each e_ij is the least-squares constant over the nodes
    of the block itself (the quantity eq. entry approximates with m_c^2
    samples): the mean of M~_ij over P_i x P_j, taken from the dense matrix
    `A`; e_from = "nodes" does the same for the soft operator.

    The diagonal blocks are the flat-segment B_l (b_from = "flat", sound soft
    only, its default) or the matrix's own diagonal blocks M_jj (b_from =
    "matrix", the only form for hard: a flat restriction of Maue's N, with the
    curve's spectral derivative cut to the segment, has no closed-form check
    and missed 15-20 % of the block)."""

    def __init__(self, arc, q, p, omega, eta=None, m_leaf=2, m_c=10, t_keep=4, bc="soft",
                 A=None, e_from=None, b_from=None):
        self.bc = bc
        e_from = e_from or ("chebyshev" if bc == "soft" else "nodes")
        b_from = b_from or ("flat" if bc == "soft" else "matrix")
        if b_from == "flat" and bc != "soft":
            raise ValueError("the flat diagonal block is the sound-soft one: b_from='matrix'")
        if (e_from == "nodes" or b_from == "matrix") and A is None:
            raise ValueError("the nodal E and the matrix blocks need the dense matrix A")
        self.arc, self.q, self.p = arc, q, p
        self.omega = omega
        self.eta = omega if eta is None else eta
        n = 4**q * p
        self.n = n
        self.curve = arc.curve(n)
        L = arc.L
        self.segs = partition(self.curve, q, p, m_leaf)
        s_nodes = L * np.arange(n) / n
        # per segment: nodes, arclength of the centre, centre, unit tangent
        self.first = np.array([f for f, _ in self.segs])
        self.level = np.array([l for _, l in self.segs])
        self.count = 2**self.level * p
        centre_s = s_nodes[self.first] + 0.5 * (self.count - 1) * (L / n)
        zc, dzc, _ = arc.sample(centre_s)
        self.centre_s = centre_s
        self.centre = zc
        self.tangent = dzc / np.hypot(dzc[:, 0], dzc[:, 1])[:, None]
        m = len(self.segs)
        self.m = m
        # B blocks (one per level) and their inverses
        levels = sorted(set(self.level.tolist()))
        if b_from == "flat":
            Bl = {l: flat_block(n, l, p, omega, self.eta, L) for l in levels}
            Bli = {l: np.linalg.inv(Bl[l]) for l in levels}
            self.Bseg = [Bl[l] for l in self.level]
            self.Binv = [Bli[l] for l in self.level]
        else:
            self.Bseg = [A[f:f + c, f:f + c] for f, c in zip(self.first, self.count)]
            self.Binv = [np.linalg.inv(b) for b in self.Bseg]
        # frequency grids and partial Fourier matrices U_i
        self.K = [frequency_grid(l, omega) for l in self.level]
        self.koff = np.concatenate([[0], np.cumsum([k.size for k in self.K])])
        rho = [s_nodes[f:f + c] - cs for f, c, cs in zip(self.first, self.count, centre_s)]
        self.U = [np.exp(1j * np.outer(r, k)) for r, k in zip(rho, self.K)]
        # E (eq. entry), one non-zero per off-diagonal block
        self.E = self._build_E(m_c) if e_from == "chebyshev" else self._build_E_nodes(A)
        # S_i, T_i, the thresholded T~ and W~ = E + antidiag(T)
        self.T = []
        for i in range(m):
            Si = self.U[i].T @ self.Binv[i] @ self.U[i]
            self.T.append(np.linalg.inv(Si))
        self.Tt = [self._threshold(Ti, t_keep * Ti.shape[0]) for Ti in self.T]
        self.W = self.E.tolil()
        for i in range(m):
            o, kk = self.koff[i], self.K[i].size
            a = np.arange(kk)
            for r_, c_ in zip(a, kk - 1 - a):
                self.W[o + r_, o + c_] += self.T[i][r_, c_]
        self.W = self.W.tocsc()
        self.Wlu = spla.splu(self.W)

    def _build_E(self, m_c):
        n, omega, eta, L = self.n, self.omega, self.eta, self.arc.L
        g = L / (2.0 * np.pi)
        # Chebyshev grids per segment (in arclength) and the averaged
        # interpolation rows w^+ I
        grids, avg = [], []
        for f, c in zip(self.first, self.count):
            s0 = L * f / n
            s1 = L * (f + c - 1) / n
            xc, wc = chebyshev_points(m_c, s0, s1)
            s_nodes = L * np.arange(f, f + c) / n
            I = interpolation_matrix(xc, wc, s_nodes)
            grids.append(xc)
            avg.append(I.mean(axis=0))
        pts = []
        for xc in grids:
            z, dz, _ = self.arc.sample(xc)
            nu = np.stack([dz[:, 1], -dz[:, 0]], axis=1)
            pts.append((z, nu, 2.0 * np.pi * xc / L))
        K_tot = int(self.koff[-1])
        E = sps.lil_matrix((K_tot, K_tot), dtype=np.complex128)
        self.kidx = {}
        for i in range(self.m):
            for j in range(self.m):
                if i == j:
                    continue
                ki, kj = self._pair_wavenumbers(i, j)
                self.kidx[(i, j)] = (ki, kj)
                zi, _, ti = pts[i]
                zj, nuj, tj = pts[j]
                Mij = soft_entries(n, omega, eta, zi, zj, nuj, np.full(m_c, g), ti, tj)
                Ui = np.exp(1j * self.K[i][ki] * (grids[i] - self.centre_s[i]))
                Uj = np.exp(1j * self.K[j][kj] * (grids[j] - self.centre_s[j]))
                Mt = Mij / (Ui[:, None] * Uj[None, :])
                E[self.koff[i] + ki, self.koff[j] + kj] = avg[i] @ Mt @ avg[j]
        return E.tocsr()

    def _pair_wavenumbers(self, i, j):
        a = self.centre[i] - self.centre[j]
        a = a / np.hypot(a[0], a[1])
        ki = round_to_grid(self.omega * a @ self.tangent[i], self.level[i], self.omega)
        kj = round_to_grid(-self.omega * a @ self.tangent[j], self.level[j], self.omega)
        return ki, kj

    def _build_E_nodes(self, A):
        """e_ij = mean of M_ij / (U_i(:, k^i) U_j(:, k^j)^t) over the nodes: the
        least-squares constant of the rank-1 form on the block itself."""
        K_tot = int(self.koff[-1])
        E = sps.lil_matrix((K_tot, K_tot), dtype=np.complex128)
        self.kidx = {}
        for i in range(self.m):
            fi, ci = self.first[i], self.count[i]
            for j in range(self.m):
                if i == j:
                    continue
                fj, cj = self.first[j], self.count[j]
                ki, kj = self._pair_wavenumbers(i, j)
                self.kidx[(i, j)] = (ki, kj)
                Mt = A[fi:fi + ci, fj:fj + cj] / np.outer(self.U[i][:, ki], self.U[j][:, kj])
                E[self.koff[i] + ki, self.koff[j] + kj] = Mt.mean()
        return E.tocsr()

    @staticmethod
    def _threshold(T, keep):
        """The `keep` largest entries of T in absolute value (T~_i, reading P7);
        entries within a relative 2^-30 of the smallest one kept count as tied
        with it and are kept too (T is symmetric, so equal entries differ only
        by rounding)."""
        if keep >= T.size:
            return sps.csr_matrix(T)
        cut = np.partition(np.abs(T).ravel(), -keep)[-keep] * (1.0 - 2.0**-30)
        return sps.csr_matrix(np.where(np.abs(T) >= cut, T, 0.0))

    # block operators ------------------------------------------------------
    def _B_inv(self, x):
        y = np.empty_like(x)
        for f, c, bi in zip(self.first, self.count, self.Binv):
            y[f:f + c] = bi @ x[f:f + c]
        return y

    def _U(self, p):
        y = np.empty(self.n, dtype=np.complex128)
        for i, (f, c) in enumerate(zip(self.first, self.count)):
            y[f:f + c] = self.U[i] @ p[self.koff[i]:self.koff[i + 1]]
        return y

    def _Ut(self, x):
        y = np.empty(int(self.koff[-1]), dtype=np.complex128)
        for i, (f, c) in enumerate(zip(self.first, self.count)):
            y[self.koff[i]:self.koff[i + 1]] = self.U[i].T @ x[f:f + c]
        return y

    def _Tblock(self, blocks, x):
        y = np.empty_like(x)
        for i in range(self.m):
            s = slice(self.koff[i], self.koff[i + 1])
            y[s] = blocks[i] @ x[s]
        return y

    # dense forms (tests) --------------------------------------------------
    def dense_B(self):
        return sla.block_diag(*self.Bseg)

    def dense_U(self):
        return sla.block_diag(*self.U)

    def dense_T(self):
        return sla.block_diag(*self.T)

    def approximation(self):
        """B + U E U^t (eq. Mapp)."""
        U = self.dense_U()
        return self.dense_B() + U @ self.E.toarray() @ U.T

    # eq. (eapp) -----------------------------------------------------------
    def apply(self, f, T=None, W_solve=None):
        """The preconditioner: q of eq. (eapp) for the right-hand side f.

        T (list of blocks) and W_solve (callable) default to the thresholded
        T~ and the sparse LU of W~; passing the exact T and a solve with
        W = E + T gives eq. (esol), the exact solve of (B + U E U^t) q = f."""
        T = self.Tt if T is None else T
        W_solve = self.Wlu.solve if W_solve is None else W_solve
        q = np.asarray(f, dtype=np.complex128).copy()
        p = -self._Ut(self._B_inv(q))
        r = self._Tblock(T, p)
        q = self._B_inv(q)
        p = -self._Tblock(T, p)
        r = W_solve(r)
        p = p + self._Tblock(T, r)
        q = q - self._B_inv(self._U(p))
        return q

    def exact_solver(self):
        """(T blocks, W solve) of eq. (esol) without the approximations."""
        W = self.E.toarray() + self.dense_T()
        lu = sla.lu_factor(W)
        return self.T, (lambda r: sla.lu_solve(lu, r))


def preconditioned_gmres(A, prec, f, rtol=1e-6, restart=80, maxit=500):
    """GMRES on A P y = f with the preconditioner P on the right, x = P y
    (modified Gram-Schmidt, Givens rotations; unpreconditioned when prec is
    None).  Returns (x, iterations, ||f - A x|| / ||f||)."""
    from .solvers import gmres
    if prec is None:
        return gmres(lambda v: A @ v, f, rtol=rtol, restart=restart, maxit=maxit)
    y, its, _ = gmres(lambda v: A @ prec(v), f, rtol=rtol, restart=restart, maxit=maxit)
    x = prec(y)
    return x, its, np.linalg.norm(f - A @ x) / np.linalg.norm(f)
