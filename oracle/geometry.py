"""Curve sampling for the oracle (test infrastructure only).

Section 1 of the paper asks for a smooth boundary; Section 2 samples it at n
equispaced points.  The oracle samples a counter-clockwise, 2*pi-periodic
parametrisation z(t) at t_j = 2 pi j / n (equispaced in the parameter, the
Nystrom nodes of Kress's rule) and returns z, z' and z'' from their closed-form
derivatives.  The unnormalised outward normal is nu~ = (z2', -z1'), with
|nu~| = |z'|.
"""
from dataclasses import dataclass

import numpy as np


@dataclass
class Curve:
    t: np.ndarray      # (n,) nodes
    z: np.ndarray      # (n, 2) points
    dz: np.ndarray     # (n, 2) z'(t)
    ddz: np.ndarray    # (n, 2) z''(t)

    @property
    def n(self):
        return self.t.shape[0]

    @property
    def speed(self):
        """|z'(t_j)|."""
        return np.hypot(self.dz[:, 0], self.dz[:, 1])

    @property
    def normal_unscaled(self):
        """nu~(t_j) = (z2', -z1'), outward for a counter-clockwise curve."""
        return np.stack([self.dz[:, 1], -self.dz[:, 0]], axis=1)

    @property
    def normal(self):
        """Unit outward normal n(z(t_j))."""
        return self.normal_unscaled / self.speed[:, None]


def nodes(n):
    return 2.0 * np.pi * np.arange(n) / n


def circle(n, radius=1.0, center=(0.0, 0.0), t=None):
    t = nodes(n) if t is None else np.asarray(t, dtype=np.float64)
    c, s = np.cos(t), np.sin(t)
    z = np.stack([center[0] + radius * c, center[1] + radius * s], axis=1)
    dz = radius * np.stack([-s, c], axis=1)
    ddz = radius * np.stack([-c, -s], axis=1)
    return Curve(t, z, dz, ddz)


def ellipse(n, a, b, t=None):
    t = nodes(n) if t is None else np.asarray(t, dtype=np.float64)
    c, s = np.cos(t), np.sin(t)
    z = np.stack([a * c, b * s], axis=1)
    dz = np.stack([-a * s, b * c], axis=1)
    ddz = np.stack([-a * c, -b * s], axis=1)
    return Curve(t, z, dz, ddz)


def fourier_star(n, a, b, t=None):
    """Star-shaped curve z(t) = r(t) (cos t, sin t) with
    r(t) = 1 + sum_{k=1..K} a_k cos(k t) + b_k sin(k t)."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    t = nodes(n) if t is None else np.asarray(t, dtype=np.float64)
    k = np.arange(1, a.shape[0] + 1, dtype=np.float64)
    kt = np.outer(t, k)
    ck, sk = np.cos(kt), np.sin(kt)
    r = 1.0 + ck @ a + sk @ b
    dr = (-sk * k) @ a + (ck * k) @ b
    ddr = (-ck * k * k) @ a + (-sk * k * k) @ b
    c, s = np.cos(t), np.sin(t)
    z = np.stack([r * c, r * s], axis=1)
    dz = np.stack([dr * c - r * s, dr * s + r * c], axis=1)
    ddz = np.stack([ddr * c - 2.0 * dr * s - r * c,
                    ddr * s + 2.0 * dr * c - r * s], axis=1)
    return Curve(t, z, dz, ddz)


def kite(n, t=None):
    """Kite z(t) = (cos t + 0.65 cos 2t - 0.65, 1.5 sin t)."""
    t = nodes(n) if t is None else np.asarray(t, dtype=np.float64)
    z = np.stack([np.cos(t) + 0.65 * np.cos(2 * t) - 0.65, 1.5 * np.sin(t)], axis=1)
    dz = np.stack([-np.sin(t) - 1.3 * np.sin(2 * t), 1.5 * np.cos(t)], axis=1)
    ddz = np.stack([-np.cos(t) - 2.6 * np.cos(2 * t), -1.5 * np.sin(t)], axis=1)
    return Curve(t, z, dz, ddz)


def from_samples(z, dz, ddz):
    z = np.asarray(z, dtype=np.float64)
    return Curve(nodes(z.shape[0]), z, np.asarray(dz, np.float64),
                 np.asarray(ddz, np.float64))


def make(kind, n, t=None, **params):
    """Build a curve by name: 'circle', 'ellipse', 'star' (Fourier star), 'kite';
    sampled at the nodes t_j, or at the parameters `t` when given."""
    if kind == "circle":
        return circle(n, params.get("radius", 1.0), t=t)
    if kind == "ellipse":
        return ellipse(n, params["a"], params["b"], t=t)
    if kind == "star":
        return fourier_star(n, params["a"], params["b"], t=t)
    if kind == "kite":
        return kite(n, t=t)
    raise ValueError(f"unknown curve kind {kind!r}")


class Arclength:
    """Arclength reparametrisation of a named curve (Section 2 samples the
    boundary at points equispaced in arclength, rho = arclength coordinate).

    s(t) = int_0^t |z'| is integrated term by term from the Fourier series of
    |z'| on a fine grid (spectrally accurate for these analytic curves) and
    inverted by Newton's method.  With sigma = 2 pi s / L the curve
    z~(sigma) = z(t(sigma)) has constant speed L / (2 pi), and

        dz~/dsigma   = z' dt/dsigma,           dt/dsigma = (L / 2 pi) / |z'|
        d2z~/dsigma2 = z'' (dt/dsigma)^2 - z' (L / 2 pi)^2 (z' . z'') / |z'|^4.
    """

    def __init__(self, kind, fine=4096, **params):
        self.kind, self.params = kind, params
        tf = nodes(fine)
        c = make(kind, fine, t=tf, **params)
        speed = c.speed
        coef = np.fft.fft(speed) / fine
        m = np.fft.fftfreq(fine, d=1.0 / fine)
        # the coefficients decay geometrically: keep those above 1e-17 |c_0|
        # (the dropped ones change s(t) by less than that)
        keep = np.abs(coef) > 1e-17 * abs(coef[0])
        keep[0] = True
        self._m = m[keep]
        self._c = coef[keep]
        self.L = 2.0 * np.pi * coef[0].real

    def s_of_t(self, t):
        """Arclength from t = 0 (the Fourier series of |z'| integrated)."""
        t = np.atleast_1d(np.asarray(t, dtype=np.float64))
        m = self._m[1:]            # self._m[0] is the zero mode
        c = self._c[1:]
        e = (np.exp(1j * np.outer(t, m)) - 1.0) / (1j * m)
        return self._c[0].real * t + (e @ c).real

    def t_of_s(self, s):
        """Parameter t with s(t) = s (Newton's method from t = 2 pi s / L)."""
        s = np.atleast_1d(np.asarray(s, dtype=np.float64))
        t = 2.0 * np.pi * s / self.L
        for _ in range(30):
            c = make(self.kind, 1, t=t, **self.params)
            step = (self.s_of_t(t) - s) / c.speed
            t = t - step
            if np.max(np.abs(step)) < 1e-15:
                break
        return t

    def sample(self, s):
        """Points, d/dsigma and d2/dsigma2 at arclengths s (sigma = 2 pi s / L)."""
        t = self.t_of_s(s)
        c = make(self.kind, 1, t=t, **self.params)
        g = self.L / (2.0 * np.pi)
        sp = c.speed
        dt = g / sp
        zz = np.sum(c.dz * c.ddz, axis=1)
        dz = c.dz * dt[:, None]
        ddz = c.ddz * (dt**2)[:, None] - c.dz * (g**2 * zz / sp**4)[:, None]
        return c.z, dz, ddz

    def curve(self, n):
        """The curve at n points equispaced in arclength, as a Curve in the
        parameter sigma (nodes 2 pi j / n)."""
        z, dz, ddz = self.sample(self.L * np.arange(n) / n)
        return Curve(nodes(n), z, dz, ddz)
