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


def circle(n, radius=1.0, center=(0.0, 0.0)):
    t = nodes(n)
    c, s = np.cos(t), np.sin(t)
    z = np.stack([center[0] + radius * c, center[1] + radius * s], axis=1)
    dz = radius * np.stack([-s, c], axis=1)
    ddz = radius * np.stack([-c, -s], axis=1)
    return Curve(t, z, dz, ddz)


def ellipse(n, a, b):
    t = nodes(n)
    c, s = np.cos(t), np.sin(t)
    z = np.stack([a * c, b * s], axis=1)
    dz = np.stack([-a * s, b * c], axis=1)
    ddz = np.stack([-a * c, -b * s], axis=1)
    return Curve(t, z, dz, ddz)


def fourier_star(n, a, b):
    """Star-shaped curve z(t) = r(t) (cos t, sin t) with
    r(t) = 1 + sum_{k=1..K} a_k cos(k t) + b_k sin(k t)."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    t = nodes(n)
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


def kite(n):
    """Kite z(t) = (cos t + 0.65 cos 2t - 0.65, 1.5 sin t)."""
    t = nodes(n)
    z = np.stack([np.cos(t) + 0.65 * np.cos(2 * t) - 0.65, 1.5 * np.sin(t)], axis=1)
    dz = np.stack([-np.sin(t) - 1.3 * np.sin(2 * t), 1.5 * np.cos(t)], axis=1)
    ddz = np.stack([-np.cos(t) - 2.6 * np.cos(2 * t), -1.5 * np.sin(t)], axis=1)
    return Curve(t, z, dz, ddz)


def from_samples(z, dz, ddz):
    z = np.asarray(z, dtype=np.float64)
    return Curve(nodes(z.shape[0]), z, np.asarray(dz, np.float64),
                 np.asarray(ddz, np.float64))


def make(kind, n, **params):
    """Build a curve by name: 'circle', 'ellipse', 'star' (Fourier star), 'kite'."""
    if kind == "circle":
        return circle(n, params.get("radius", 1.0))
    if kind == "ellipse":
        return ellipse(n, params["a"], params["b"])
    if kind == "star":
        return fourier_star(n, params["a"], params["b"])
    if kind == "kite":
        return kite(n)
    raise ValueError(f"unknown curve kind {kind!r}")
