"""Closed forms that pin the oracle (tests only).

Everything here follows from the mathematics of Section 1 of the paper on the
unit disk, written independently of the Nystrom code:

* Graf/Fourier-Bessel addition theorem on |x| = |y| = 1 gives, for the density
  e^{i m theta},
      S_m  = (i pi / 2) J_m(w) H_m(w)
      D_m  = D'_m = (i pi w / 2) J_m(w) H_m'(w) + 1/2
      N_m  = (i pi w^2 / 2) J_m'(w) H_m'(w)
  so the sound-soft operator has eigenvalue (pi/2) H_m [i w J_m' + eta J_m] and
  the sound-hard operator (eq. 2) (pi w/2) H_m' [-i J_m + (w/eta) J_m'].
* Plane wave e^{i w x . d} = sum_m i^m J_m(w r) e^{i m (theta - theta_d)}
  (Jacobi-Anger), so the radiating field scattered by the unit disk is
      soft:  -sum_m i^m J_m(w) H_m(w r) / H_m(w) e^{i m (theta - theta_d)}
      hard:  -sum_m i^m J_m'(w) H_m(w r) / H_m'(w) e^{i m (theta - theta_d)}
* The field of a point source x0 inside the obstacle is itself a radiating
  solution outside, so boundary data -G(., x0) gives u = -G(x, x0).
"""
import numpy as np
import scipy.special as sp


def disk_layer_eigenvalues(m, w):
    J = sp.jv(m, w)
    H = sp.hankel1(m, w)
    Jp = sp.jvp(m, w)
    Hp = sp.h1vp(m, w)
    S = 0.5j * np.pi * J * H
    D = 0.5j * np.pi * w * J * Hp + 0.5
    N = 0.5j * np.pi * w**2 * Jp * Hp
    return S, D, N


def disk_soft_eigenvalue(m, w, eta):
    return 0.5 * np.pi * sp.hankel1(m, w) * (1j * w * sp.jvp(m, w) + eta * sp.jv(m, w))


def disk_hard_eigenvalue(m, w, eta):
    return 0.5 * np.pi * w * sp.h1vp(m, w) * (-1j * sp.jv(m, w) + (w / eta) * sp.jvp(m, w))


def disk_scattered(w, theta_d, pts, bc, mmax=None):
    pts = np.asarray(pts, dtype=np.float64)
    r = np.hypot(pts[:, 0], pts[:, 1])
    th = np.arctan2(pts[:, 1], pts[:, 0])
    if mmax is None:
        mmax = int(w + 40)
    u = np.zeros(pts.shape[0], dtype=np.complex128)
    for m in range(-mmax, mmax + 1):
        if bc == "soft":
            coef = sp.jv(m, w) / sp.hankel1(m, w)
        else:
            coef = sp.jvp(m, w) / sp.h1vp(m, w)
        u -= (1j ** (m % 4)) * coef * sp.hankel1(m, w * r) * np.exp(1j * m * (th - theta_d))
    return u


def green(w, pts, x0):
    pts = np.asarray(pts, dtype=np.float64)
    r = np.hypot(pts[:, 0] - x0[0], pts[:, 1] - x0[1])
    return 0.25j * sp.hankel1(0, w * r)


def ring(radius, count):
    th = 2 * np.pi * (np.arange(count) + 0.37) / count
    return np.stack([radius * np.cos(th), radius * np.sin(th)], axis=1)


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b))
