"""Parity of the library's level blocks of the directional preconditioner
(cfie_dirprec_level, host code: the flat block B_l, its inverse, the partial
Fourier matrix U_l and T_l = (U^t B^-1 U)^-1) with the oracle's
directional.Directional / flat_block.  CPU only: the call needs no GPU.

The two sides share no code: the library sums its own Kress weights and takes
J0, Y0 from the C++17 special functions; the oracle uses scipy.  Tolerance
1e-12 relative to each block's largest entry (the agreement is ~1e-14)."""
import numpy as np
import pytest

from oracle import directional, geometry
from paper_1408_1578_gb300 import build, cfie


@pytest.fixture(scope="module", autouse=True)
def lib():
    build.build()
    return cfie.load()


def _rel(a, b):
    return np.max(np.abs(a - b)) / np.max(np.abs(b))


@pytest.mark.parametrize("kind,params,q,eta_factor", [
    ("ellipse", {"a": 1.0, "b": 0.5}, 3, 1.0),
    ("ellipse", {"a": 1.0, "b": 0.5}, 4, 0.5),
    ("kite", {}, 4, 1.0),
])
def test_level_blocks_match_the_oracle(kind, params, q, eta_factor):
    p = 8
    arc = geometry.Arclength(kind, **params)
    n = 4**q * p
    w = 2 * np.pi * (n / p) / arc.L
    P = directional.Directional(arc, q, p, w, eta=eta_factor * w)
    for level in sorted(set(P.level.tolist())):
        B, Binv, U, T = cfie.dirprec_level(n, p, level, w, eta_factor * w, arc.L)
        i = int(np.nonzero(P.level == level)[0][0])        # any segment of this level
        assert _rel(B, P.Bseg[i]) < 1e-12
        assert _rel(Binv, P.Binv[i]) < 1e-12
        assert _rel(U, P.U[i]) < 1e-12
        assert _rel(T, P.T[i]) < 1e-12


def test_blocks_are_consistent():
    """B Binv = I, the anti-diagonal of T dominates it (Section 2.2: T
    concentrates on its anti-diagonal), U has unit-modulus entries."""
    n, p, level, w = 2048, 8, 4, 400.0
    B, Binv, U, T = cfie.dirprec_level(n, p, level, w, w, 4.0)
    assert np.max(np.abs(B @ Binv - np.eye(B.shape[0]))) < 1e-12
    assert np.max(np.abs(np.abs(U) - 1)) < 1e-14
    K = T.shape[0]
    anti = np.abs(T[np.arange(K), K - 1 - np.arange(K)])
    off = np.abs(T).copy()
    off[np.arange(K), K - 1 - np.arange(K)] = 0
    assert np.median(anti) > 3 * np.median(off.max(axis=1))


@pytest.mark.parametrize("args", [
    (7, 8, 2, 10.0, 10.0, 1.0),          # odd n
    (64, 8, 3, 10.0, 10.0, 1.0),         # 2^l p = 64 > n / 2
    (2048, 8, 2, 0.0, 10.0, 1.0),        # omega
    (2048, 8, 2, 10.0, -1.0, 1.0),       # eta
    (2048, 8, 2, 10.0, 10.0, float("nan")),
    (2048, 0, 2, 10.0, 10.0, 1.0),       # p
    (2048, 8, -1, 10.0, 10.0, 1.0),      # level
    (65536, 8, 8, 10.0, 10.0, 1.0),      # 2^l p = 2048 > 1024
])
def test_invalid_arguments(lib, args):
    assert lib.cfie_dirprec_level(*args, None, None, None, None) == cfie.CFIE_EINVAL


def test_threshold_matches_the_oracle():
    """T~ keeps the 4 K largest entries of T (reading P7, entries within a
    relative 2^-30 of the cut counted as tied): identical to the oracle's on
    the same T, and from the library's own T_l the same entries are kept."""
    arc = geometry.Arclength("ellipse", a=1.0, b=0.5)
    q, p = 4, 8
    n = 4**q * p
    w = 2 * np.pi * (n / p) / arc.L
    P = directional.Directional(arc, q, p, w)
    for level in sorted(set(P.level.tolist())):
        i = int(np.nonzero(P.level == level)[0][0])
        T = P.T[i]
        K = T.shape[0]
        assert np.array_equal(cfie.dirprec_threshold(T, 4 * K), P.Tt[i].toarray())
        mine = cfie.dirprec_threshold(cfie.dirprec_level(n, p, level, w, w, arc.L)[3], 4 * K)
        ref = P.Tt[i].toarray()
        assert np.array_equal(mine != 0, ref != 0)
        assert np.max(np.abs(mine - ref)) < 1e-12 * np.max(np.abs(T))


def test_threshold_edges(lib):
    T = np.arange(9, dtype=float).reshape(3, 3) * (1 + 1j)
    assert not np.any(cfie.dirprec_threshold(T, 0))
    assert np.array_equal(cfie.dirprec_threshold(T, 9), T)
    assert np.array_equal(cfie.dirprec_threshold(T, 100), T)
    kept = cfie.dirprec_threshold(T, 2)
    assert np.count_nonzero(kept) == 2 and kept[2, 2] == T[2, 2] and kept[2, 1] == T[2, 1]
    import ctypes
    buf = np.zeros(18)
    dp = ctypes.POINTER(ctypes.c_double)
    assert lib.cfie_dirprec_threshold(0, buf.ctypes.data_as(dp), 1,
                                      buf.ctypes.data_as(dp)) == cfie.CFIE_EINVAL
    assert lib.cfie_dirprec_threshold(3, buf.ctypes.data_as(dp), -1,
                                      buf.ctypes.data_as(dp)) == cfie.CFIE_EINVAL
    assert lib.cfie_dirprec_threshold(3, None, 1, buf.ctypes.data_as(dp)) == cfie.CFIE_EINVAL
