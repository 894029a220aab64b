"""Nystrom discretisation of S, D, D', N and the two CFIE operators
(oracle, test infrastructure only).

Paper, Section 1: G(x, y) = (i/4) H0^(1)(omega |x - y|) and

    (S q)(x)  = int G(x, y) q(y) ds(y)           (D q)(x)  = int dG/dn(y) q(y) ds(y)
    (D' q)(x) = int dG/dn(x) q(y) ds(y)          (N q)(x)  = f.p. int d2G/dn(x)dn(y) q(y) ds(y)

    sound soft  (eq. 1):  (1/2 I + D - i eta S) q = -u_I
    sound hard  (eq. 2):  (1/2 I - D' + N/(i eta)) q = -du_I/dn

Eq. 2 is used for the sound-hard operator; the operator form printed after it
(dis2) carries the opposite sign on D' and N, which on the unit disk makes the
operator nearly singular for every propagating mode at eta = omega, so it is
read as a sign slip.

Parametric kernels (x = z(t), y = z(tau), r = |z(t) - z(tau)|, nu~ = (z2', -z1')):

    M(t, tau)  = (i/4) H0(omega r) |z'(tau)|                               -> S
    L(t, tau)  = (i omega/4) H1(omega r) (z(t) - z(tau)) . nu~(tau) / r     -> D
    L'(t, tau) = (i omega/4) H1(omega r) (z(tau) - z(t)) . nu~(t) / r
                 * |z'(tau)| / |z'(t)|                                        -> D'

Each splits as K = K1 ln(4 sin^2((t - tau)/2)) + K2 with
M1 = -(1/4pi) J0(omega r) |z'(tau)| and L1 = -(omega/4pi) J1(omega r) (...) / r
(from the (2/pi) ln(x/2) J_nu(x) term of Y_nu).  The Nystrom entry is
R_{(i-j) mod n} K1(t_i, t_j) + h K2(t_i, t_j), h = 2 pi / n, with the diagonal
limits

    M1(t, t) = -|z'| / (4 pi)
    M2(t, t) = [ i/4 - C_E/(2 pi) - ln(omega |z'| / 2) / (2 pi) ] |z'|
    L1(t, t) = 0,   L2(t, t) = (z2' z1'' - z1' z2'') / (4 pi |z'|^2)   (same for L')

N follows Maue's identity  N = d/ds S d/ds + omega^2 (n1 S n1 + n2 S n2), with
d/ds = |z'|^{-1} d/dt and d/dt the spectral derivative of the trigonometric
interpolant (Nyquist mode set to zero).
"""
import numpy as np
import scipy.special as sp

from .kress import kress_weights

EULER_GAMMA = 0.57721566490153286061


def bessel01(x):
    """J0, Y0, J1, Y1 at x > 0 (scipy.special, Cephes)."""
    return sp.j0(x), sp.y0(x), sp.j1(x), sp.y1(x)


def hankel01(x):
    """H0^(1)(x), H1^(1)(x)."""
    j0, y0, j1, y1 = bessel01(x)
    return j0 + 1j * y0, j1 + 1j * y1


def log_factor(n, d):
    """ln(4 sin^2(pi d / n)) for integer d not divisible by n."""
    return np.log(4.0 * np.sin(np.pi * d / n) ** 2)


def layer_rows(curve, omega, rows, which, R=None):
    """Rows `rows` of the Kress-Nystrom matrix of S ('S'), D ('D') or D' ('Dp').

    No identity term is included.  `R` are the Kress weights (computed if None).
    """
    n = curve.n
    h = 2.0 * np.pi / n
    if R is None:
        R = kress_weights(n)
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.arange(n, dtype=np.int64)
    z, dz, ddz = curve.z, curve.dz, curve.ddz
    speed = curve.speed
    nu = curve.normal_unscaled

    diff = z[rows][:, None, :] - z[None, :, :]          # z(t_i) - z(t_j)
    r = np.hypot(diff[..., 0], diff[..., 1])
    d = (rows[:, None] - cols[None, :]) % n
    on_diag = d == 0
    r_safe = np.where(on_diag, 1.0, r)
    x = omega * r_safe
    j0, y0, j1, y1 = bessel01(x)
    h0 = j0 + 1j * y0
    h1 = j1 + 1j * y1

    if which == "S":
        K = 0.25j * h0 * speed[None, :]
        K1 = -(1.0 / (4.0 * np.pi)) * j0 * speed[None, :]
    elif which == "D":
        c = (diff[..., 0] * nu[None, :, 0] + diff[..., 1] * nu[None, :, 1]) / r_safe
        K = 0.25j * omega * h1 * c
        K1 = -(omega / (4.0 * np.pi)) * j1 * c
    elif which == "Dp":
        c = -(diff[..., 0] * nu[rows][:, None, 0] + diff[..., 1] * nu[rows][:, None, 1]) / r_safe
        c = c * speed[None, :] / speed[rows][:, None]
        K = 0.25j * omega * h1 * c
        K1 = -(omega / (4.0 * np.pi)) * j1 * c
    else:
        raise ValueError(which)

    logf = log_factor(n, np.where(on_diag, 1, d))
    K2 = K - K1 * logf
    A = R[d] * K1 + h * K2

    # diagonal limits
    ii = np.nonzero(on_diag)
    ri = rows[ii[0]]
    s_i = speed[ri]
    if which == "S":
        m1 = -s_i / (4.0 * np.pi)
        m2 = (0.25j - EULER_GAMMA / (2.0 * np.pi)
              - np.log(omega * s_i / 2.0) / (2.0 * np.pi)) * s_i
        A[ii] = R[0] * m1 + h * m2
    else:
        l2 = (dz[ri, 1] * ddz[ri, 0] - dz[ri, 0] * ddz[ri, 1]) / (4.0 * np.pi * s_i**2)
        A[ii] = h * l2
    return A


def soft_rows(curve, omega, eta, rows, R=None):
    """Rows of the sound-soft CFIE matrix 1/2 I + D - i eta S (eq. 1)."""
    if R is None:
        R = kress_weights(curve.n)
    rows = np.asarray(rows, dtype=np.int64)
    A = layer_rows(curve, omega, rows, "D", R) - 1j * eta * layer_rows(curve, omega, rows, "S", R)
    A[np.arange(rows.size), rows] += 0.5
    return A


def _blocked(curve, omega, which, R, block=512):
    n = curve.n
    out = np.empty((n, n), dtype=np.complex128)
    for s in range(0, n, block):
        rows = np.arange(s, min(n, s + block))
        out[rows] = layer_rows(curve, omega, rows, which, R)
    return out


def soft_matrix(curve, omega, eta, R=None):
    """Full sound-soft CFIE matrix (eq. 1)."""
    if R is None:
        R = kress_weights(curve.n)
    A = _blocked(curve, omega, "D", R) - 1j * eta * _blocked(curve, omega, "S", R)
    A[np.diag_indices(curve.n)] += 0.5
    return A


def spectral_derivative(x, axis=0):
    """d/dt of the trigonometric interpolant of samples on t_j = 2 pi j / n,
    Nyquist mode set to zero (n even)."""
    x = np.asarray(x)
    n = x.shape[axis]
    m = np.fft.fftfreq(n, d=1.0 / n)          # integer frequencies
    factor = 1j * m
    factor[n // 2] = 0.0
    shape = [1] * x.ndim
    shape[axis] = n
    return np.fft.ifft(np.fft.fft(x, axis=axis) * factor.reshape(shape), axis=axis)


def hypersingular_matrix(curve, omega, S):
    """N by Maue's identity from the single-layer matrix S:
    N = diag(1/|z'|) Dt S diag(1/|z'|) Dt + omega^2 (N1 S N1 + N2 S N2)."""
    inv_speed = 1.0 / curve.speed
    nrm = curve.normal
    T = S * inv_speed[None, :]
    T = -spectral_derivative(T, axis=1)      # (S diag) Dt, since Dt^T = -Dt
    T = spectral_derivative(T, axis=0)       # Dt (...)
    tangential = inv_speed[:, None] * T
    normal = (nrm[:, 0, None] * S * nrm[None, :, 0]
              + nrm[:, 1, None] * S * nrm[None, :, 1])
    return tangential + omega**2 * normal


def hard_matrix(curve, omega, eta, R=None):
    """Full sound-hard CFIE matrix 1/2 I - D' + N/(i eta) (eq. 2)."""
    if R is None:
        R = kress_weights(curve.n)
    S = _blocked(curve, omega, "S", R)
    Dp = _blocked(curve, omega, "Dp", R)
    A = -Dp + hypersingular_matrix(curve, omega, S) / (1j * eta)
    A[np.diag_indices(curve.n)] += 0.5
    return A


def cfie_matrix(curve, omega, eta, bc, R=None):
    if bc == "soft":
        return soft_matrix(curve, omega, eta, R)
    if bc == "hard":
        return hard_matrix(curve, omega, eta, R)
    raise ValueError(bc)


def plane_wave_rhs(curve, omega, theta, bc):
    """Right-hand sides for incident plane waves u_I = exp(i omega d . x),
    d = (cos theta_k, sin theta_k): soft -u_I, hard -du_I/dn (Section 1)."""
    theta = np.atleast_1d(np.asarray(theta, dtype=np.float64))
    dvec = np.stack([np.cos(theta), np.sin(theta)], axis=0)       # (2, K)
    phase = np.exp(1j * omega * (curve.z @ dvec))                  # (n, K)
    if bc == "soft":
        return -phase
    if bc == "hard":
        dn = curve.normal @ dvec
        return -1j * omega * dn * phase
    raise ValueError(bc)


def point_source_rhs(curve, omega, x0, bc):
    """Boundary data of the radiating field G(., x0) with x0 inside the
    obstacle: soft -G(z_j, x0), hard -dG(z_j, x0)/dn(z_j)."""
    diff = curve.z - np.asarray(x0, dtype=np.float64)[None, :]
    r = np.hypot(diff[:, 0], diff[:, 1])
    h0, h1 = hankel01(omega * r)
    if bc == "soft":
        return -0.25j * h0
    if bc == "hard":
        dn = (diff * curve.normal).sum(axis=1) / r
        return 0.25j * omega * h1 * dn
    raise ValueError(bc)
