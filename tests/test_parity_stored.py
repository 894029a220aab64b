"""GPU parity of the stored-matrix tensor-core path (bf16 hi/lo split-complex
matrix, TMA + tcgen05 contraction) and of its refined solve, through the C ABI.

Tolerances: raw stored matvec <= 1e-4 relative per right-hand side (the bf16
hi/lo split keeps ~16 bits per component, ~1e-5 in practice); refined solve
<= 1e-6 relative error against the oracle's LU solution at residual 1e-8."""
import numpy as np
import pytest

from oracle import geometry, operators, solvers
from paper_1408_1578_gb300 import inputs
from tests.gpu_util import col_rel, empty, to_dev, to_host, zeros

pytestmark = pytest.mark.gpu

TOL_STORED = 1e-4
TOL_REFINED = 1e-6


@pytest.fixture(scope="module")
def ctx():
    from paper_1408_1578_gb300 import cfie
    c = cfie.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("kind,params,n,omega,nrhs", [
    ("kite", {}, 256, 24.0, 1),
    ("kite", {}, 2000, 200.0, 5),
    ("kite", {}, 2000, 200.0, 32),
    ("kite", {}, 2000, 200.0, 33),
    ("star", {"a": [0, 0, 0, 0, 0.3], "b": [0] * 5}, 1502, 120.0, 64),
    ("ellipse", {"a": 1.0, "b": 0.5}, 1000, 90.0, 7),
    ("circle", {}, 8, 1.0, 2),
])
def test_stored_matvec_parity(ctx, kind, params, n, omega, nrhs):
    c = geometry.make(kind, n, **params)
    A = operators.soft_matrix(c, omega, omega)
    X = inputs.random_density(n, nrhs, seed=3 * n + nrhs)
    op = ctx.geometry(kind, **params).discretise(n, omega, bc="soft", precision="tensor",
                                                 layout="stored")
    y = empty(nrhs, n)
    op.apply(to_dev(X), y)
    err = np.max(col_rel(to_host(y), (A @ X.T).T))
    assert err < TOL_STORED, err


def test_stored_matches_fp32_matrix_free(ctx):
    """Same entries (up to the bf16 split) as the FP32 fused kernel."""
    n, w, nrhs = 3000, 450.0, 16
    X = inputs.random_density(n, nrhs, seed=5)
    opt = ctx.kite().discretise(n, w, precision="tensor", layout="stored")
    opf = ctx.kite().discretise(n, w, precision="fp32")
    y1 = empty(nrhs, n)
    y2 = empty(nrhs, n)
    opt.apply(to_dev(X), y1)
    opf.apply(to_dev(X), y2)
    assert np.max(col_rel(to_host(y1), to_host(y2))) < TOL_STORED


def test_stored_refined_solve(ctx):
    n, w, nrhs = 2000, 200.0, 6
    c = geometry.kite(n)
    A = operators.soft_matrix(c, w, w)
    F = operators.plane_wave_rhs(c, w, inputs.directions(nrhs), "soft")
    Q = solvers.lu_solve(A, F).T
    op = ctx.kite().discretise(n, w, precision="tensor", layout="stored")
    x = zeros(nrhs, n)
    its, rel, _ = op.gmres_solve(to_dev(F.T), x, rtol=1e-8, restart=80, maxit=3000)
    stats = op.last_stats()
    assert np.all(rel <= 1e-8)
    assert stats["refinements"] >= 1 and stats["inner_matvecs"] > 0
    assert np.max(col_rel(to_host(x), Q)) < TOL_REFINED


def test_stored_layout_arguments(ctx):
    from paper_1408_1578_gb300 import cfie
    g = ctx.kite()
    with pytest.raises(cfie.CfieError) as e:
        g.discretise(256, 20.0, bc="hard", precision="tensor", layout="stored")
    assert e.value.status == cfie.CFIE_EINVAL
    with pytest.raises(cfie.CfieError):
        g.discretise(256, 20.0, precision="fp32", layout="stored")
    with pytest.raises(cfie.CfieError):
        g.discretise(256, 20.0, precision="tensor", layout="matrix_free")
