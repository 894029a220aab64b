"""Parity of the library's preconditioner structure (cfie_dirprec_plan, host
code) with the oracle's directional.Directional: the segments of Section 2.1
and, for every ordered pair of segments, the wave-number indices k^i_ij and
k^j_ij.  Index work: bit-exact.  CPU only: the call needs no GPU."""
import ctypes

import numpy as np
import pytest

from oracle import directional, geometry
from paper_1408_1578_gb300 import build, cfie


@pytest.fixture(scope="module", autouse=True)
def lib():
    build.build()
    return cfie.load()


@pytest.mark.parametrize("kind,params,q,m_leaf", [
    ("ellipse", {"a": 1.0, "b": 0.5}, 3, 2),
    ("ellipse", {"a": 1.0, "b": 0.5}, 4, 2),
    ("ellipse", {"a": 1.0, "b": 0.25}, 4, 4),
    ("kite", {}, 4, 2),
    ("star", {"a": [0, 0, 0, 0, 0.3], "b": [0.02, 0, -0.04, 0, 0]}, 3, 2),
    # radius 1.3: curvature 1/1.3, away from the threshold 2^l = 2^q / sqrt(c);
    # at radius 1 every level-q piece sits exactly on it and the last bit of the
    # computed curvature decides (on either side)
    ("circle", {"radius": 1.3}, 3, 2),
])
def test_plan_matches_the_oracle(kind, params, q, m_leaf):
    p = 8
    arc = geometry.Arclength(kind, **params)
    n = 4**q * p
    w = 2 * np.pi * (n / p) / arc.L
    first, level, kpair = cfie.dirprec_plan(kind, q, p, w, m_leaf=m_leaf, **params)
    P = directional.Directional(arc, q, p, w, m_leaf=m_leaf)
    assert np.array_equal(first, P.first) and np.array_equal(level, P.level)
    assert len(P.kidx) == P.m * (P.m - 1)
    for (i, j), (ki, kj) in P.kidx.items():
        assert (kpair[i, j, 0], kpair[i, j, 1]) == (ki, kj), (i, j)
    assert not np.any(kpair[np.arange(P.m), np.arange(P.m)])
    # the indices address each segment's grid of 2^(l+1) + 1 wave numbers
    assert np.all(kpair[..., 0] <= 2 ** (level[:, None] + 1))
    assert np.all(kpair[..., 1] <= 2 ** (level[None, :] + 1))


def test_sizing_call_and_capacity(lib):
    m = ctypes.c_int()
    par = np.array([1.0, 0.5])
    dp = ctypes.POINTER(ctypes.c_double)
    ip = ctypes.POINTER(ctypes.c_int)
    args = (cfie.CFIE_CURVE_ELLIPSE, par.ctypes.data_as(dp), 2, 3, 8, 80.0, 2)
    assert lib.cfie_dirprec_plan(*args, 0, ctypes.byref(m), None, None, None) == cfie.CFIE_OK
    k = m.value
    assert k > 4
    small = k - 1
    f = np.zeros(small, dtype=np.int32)
    lv = np.zeros(small, dtype=np.int32)
    kp = np.zeros(2 * small * small, dtype=np.int32)
    st = lib.cfie_dirprec_plan(*args, small, ctypes.byref(m), f.ctypes.data_as(ip),
                               lv.ctypes.data_as(ip), kp.ctypes.data_as(ip))
    assert st == cfie.CFIE_EINVAL and m.value == k
    # one output array without the others
    assert lib.cfie_dirprec_plan(*args, k, ctypes.byref(m), f.ctypes.data_as(ip), None,
                                 None) == cfie.CFIE_EINVAL


@pytest.mark.parametrize("q,p,omega,m_leaf", [
    (0, 8, 10.0, 2), (10, 8, 10.0, 2), (3, 0, 10.0, 2),
    (9, 8, 10.0, 2),                                   # n = 2^21 > 2^20
    (3, 8, 0.0, 2), (3, 8, float("inf"), 2), (3, 8, 10.0, 0),
])
def test_invalid_sizes(lib, q, p, omega, m_leaf):
    m = ctypes.c_int()
    assert lib.cfie_dirprec_plan(cfie.CFIE_CURVE_KITE, None, 0, q, p, omega, m_leaf, 0,
                                 ctypes.byref(m), None, None, None) == cfie.CFIE_EINVAL


@pytest.mark.parametrize("kind,params", [("ellipse", {"a": 1.0, "b": 0.5}), ("kite", {})])
def test_w_pattern_matches_the_oracle(kind, params):
    """Positions of W~ = E + antidiag(T): the oracle's sparse W~ has exactly
    these non-zeros, one per ordered segment pair plus every anti-diagonal."""
    p, q = 8, 4
    arc = geometry.Arclength(kind, **params)
    n = 4**q * p
    w = 2 * np.pi * (n / p) / arc.L
    first, level, kpair = cfie.dirprec_plan(kind, q, p, w, **params)
    koff, row, col = cfie.dirprec_w_pattern(level, kpair)
    P = directional.Directional(arc, q, p, w)
    assert np.array_equal(koff, P.koff)
    W = P.W.tocoo()
    assert len(row) == W.nnz
    assert set(zip(row.tolist(), col.tolist())) == set(zip(W.row.tolist(), W.col.tolist()))


def test_w_pattern_rejects_bad_indices(lib):
    level = np.array([1, 1], dtype=np.int32)
    kpair = np.zeros((2, 2, 2), dtype=np.int32)
    kpair[0, 1] = (5, 0)                 # K = 5: index 5 is out of range
    koff = np.zeros(3, dtype=np.int32)
    nnz = ctypes.c_int()
    ip = ctypes.POINTER(ctypes.c_int)
    row = np.zeros(16, dtype=np.int32)
    col = np.zeros(16, dtype=np.int32)
    st = lib.cfie_dirprec_w_pattern(2, level.ctypes.data_as(ip), kpair.ctypes.data_as(ip), 16,
                                    koff.ctypes.data_as(ip), ctypes.byref(nnz),
                                    row.ctypes.data_as(ip), col.ctypes.data_as(ip))
    # rejected before any output is written
    assert st == cfie.CFIE_EINVAL and nnz.value == 0 and not koff.any() and not row.any()
