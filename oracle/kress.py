"""Kress log-split quadrature weights (oracle, test infrastructure only).

The paper discretises the CFIE with a Nystrom method (Section 1) but states no
quadrature rule.  The oracle uses Kress's rule for kernels of the form
K(t, tau) = K1(t, tau) ln(4 sin^2((t - tau)/2)) + K2(t, tau) with K1, K2 smooth
(Colton & Kress, Section 3.5).  The logarithmic factor is integrated exactly
against the trigonometric interpolant of K1(t, .) phi(.) on the n = 2N nodes,
using the closed form

    int_0^{2pi} ln(4 sin^2((t - tau)/2)) e^{i m tau} dtau = -(2 pi/|m|) e^{i m t}   (m != 0),
                                                          = 0                       (m = 0).

With the interpolant's Nyquist term taken as cos(N tau), this gives weights
that depend only on d = (i - j) mod n:

    R_d = -(2 pi / N) sum_{m=1}^{N-1} cos(m d pi / N) / m  -  (pi / N^2) cos(d pi).
"""
import numpy as np


def kress_weights(n):
    """R_d, d = 0..n-1, by the direct sum above (n even)."""
    if n % 2:
        raise ValueError("Kress weights need an even number of nodes")
    N = n // 2
    d = np.arange(n, dtype=np.int64)
    acc = np.zeros(n)
    for m in range(1, N):
        # the integer reduction (m d) mod n keeps each cosine argument in [0, 2 pi)
        acc += np.cos(2.0 * np.pi * ((m * d) % n) / n) / m
    sign = np.where(d % 2 == 0, 1.0, -1.0)
    return -(2.0 * np.pi / N) * acc - (np.pi / N**2) * sign
