"""Off-surface scattered field from a boundary density (oracle, test
infrastructure only).

Section 1 of the paper says that once q is known the scattered field is
evaluated through a boundary integral, without writing it out.  The oracle
uses the representations that produce eq. 1 and eq. 2 through the jump
relations of the layer potentials (outward normal):

    sound soft:  u(x) = (D q)(x) - i eta (S q)(x)
    sound hard:  u(x) = -(S q)(x) + (D q)(x) / (i eta)

discretised by the plain trapezoidal rule, which is spectrally accurate for
points a few node spacings away from the boundary.
"""
import numpy as np

from .operators import hankel01


def layer_potentials(curve, omega, q, pts):
    """Return (S q)(x), (D q)(x) at off-surface points pts (m, 2)."""
    pts = np.asarray(pts, dtype=np.float64)
    n = curve.n
    h = 2.0 * np.pi / n
    diff = pts[:, None, :] - curve.z[None, :, :]
    r = np.hypot(diff[..., 0], diff[..., 1])
    h0, h1 = hankel01(omega * r)
    nu = curve.normal_unscaled
    c = (diff[..., 0] * nu[None, :, 0] + diff[..., 1] * nu[None, :, 1]) / r
    Sk = 0.25j * h0 * curve.speed[None, :]
    Dk = 0.25j * omega * h1 * c
    q = np.asarray(q, dtype=np.complex128)
    return h * (Sk @ q), h * (Dk @ q)


def scattered_field(curve, omega, eta, bc, q, pts):
    Sq, Dq = layer_potentials(curve, omega, q, pts)
    if bc == "soft":
        return Dq - 1j * eta * Sq
    if bc == "hard":
        return -Sq + Dq / (1j * eta)
    raise ValueError(bc)
