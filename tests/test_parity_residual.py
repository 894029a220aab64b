"""GPU parity of the FP64-accurate residual matvec evaluated in double-float
arithmetic on the FP32 pipe (cfie_apply_residual), against the oracle and
against the FP64 kernel.  Tolerance 1e-11 relative per right-hand side (the
kernel lands near 1e-13; at omega r ~ 6e3 the double-float phase carries
~2e-11 rad, hence the looser full-size bound)."""
import numpy as np
import pytest

from oracle import geometry, kress, operators
from paper_1408_1578_gb300 import inputs
from tests.gpu_util import col_rel, empty, to_dev, to_host

pytestmark = pytest.mark.gpu

TOL_RES = 1e-11


@pytest.fixture(scope="module")
def ctx():
    from paper_1408_1578_gb300 import cfie
    c = cfie.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("kind,params,n,omega,nrhs,prec", [
    ("kite", {}, 2000, 200.0, 5, "fp32"),
    ("kite", {}, 2000, 200.0, 64, "fp32"),
    ("star", {"a": [0.03, -0.02, 0.04], "b": [0.01, 0.05, -0.03]}, 3000, 450.0, 17, "tensor"),
    ("ellipse", {"a": 1.0, "b": 0.5}, 1000, 90.0, 3, "fp32"),
    ("circle", {}, 64, 2.0, 2, "fp32"),
])
def test_residual_matvec_parity(ctx, kind, params, n, omega, nrhs, prec):
    c = geometry.make(kind, n, **params)
    A = operators.soft_matrix(c, omega, omega)
    X = inputs.random_density(n, nrhs, seed=9 * n + nrhs)
    layout = "stored" if prec == "tensor" else "matrix_free"
    op = ctx.geometry(kind, **params).discretise(n, omega, precision=prec, layout=layout)
    y = empty(nrhs, n)
    op.apply_residual(to_dev(X), y)
    assert np.max(col_rel(to_host(y), (A @ X.T).T)) < TOL_RES
    y64 = empty(nrhs, n)
    op.apply_fp64(to_dev(X), y64)
    assert np.max(col_rel(to_host(y), to_host(y64))) < TOL_RES


@pytest.mark.parametrize("kind,params,n,omega,nrhs", [
    ("kite", {}, 2000, 200.0, 8),
    ("kite", {}, 2000, 200.0, 64),
    ("kite", {}, 1000, 120.0, 70),                    # two passes (64 + 6)
    ("star", {"a": [0.03, -0.02, 0.04], "b": [0.01, 0.05, -0.03]}, 3002, 450.0, 17),
    ("ellipse", {"a": 1.0, "b": 0.5}, 1000, 90.0, 33),
    ("circle", {}, 64, 2.0, 9),                       # every pair in the band
])
def test_tensor_core_residual_parity(ctx, kind, params, n, omega, nrhs):
    """Sliced tensor-core residual (variant 2) against the oracle and against
    the CUDA-core double-float residual (variant 1)."""
    c = geometry.make(kind, n, **params)
    A = operators.soft_matrix(c, omega, omega)
    X = inputs.random_density(n, nrhs, seed=3 * n + nrhs)
    op = ctx.geometry(kind, **params).discretise(n, omega, precision="fp32")
    y2, y1 = empty(nrhs, n), empty(nrhs, n)
    op.set_residual_variant(2)
    op.apply_residual(to_dev(X), y2)
    op.set_residual_variant(1)
    op.apply_residual(to_dev(X), y1)
    assert np.max(col_rel(to_host(y2), (A @ X.T).T)) < TOL_RES
    assert np.max(col_rel(to_host(y2), to_host(y1))) < TOL_RES


def test_residual_variant_arguments(ctx):
    from paper_1408_1578_gb300 import cfie
    op = ctx.kite().discretise(256, 20.0, bc="hard", precision="fp32")
    op.set_residual_variant(2)
    op.set_residual_variant(1)
    with pytest.raises(cfie.CfieError):
        op.set_residual_variant(3)
    op64 = ctx.kite().discretise(256, 20.0, precision="fp64")
    with pytest.raises(cfie.CfieError):
        op64.set_residual_variant(1)


@pytest.mark.parametrize("kind,params,n,omega,nrhs", [
    ("kite", {}, 2000, 200.0, 8),
    ("star", {"a": [0, 0, 0, 0, 0.3], "b": [0] * 5}, 1502, 120.0, 30),   # S passes of 64 + 26
    ("ellipse", {"a": 1.0, "b": 0.5}, 1000, 90.0, 3),
])
def test_tensor_core_residual_parity_hard(ctx, kind, params, n, omega, nrhs):
    """Sound-hard residual with the S and D' sums sliced on the tensor cores,
    against the oracle and the CUDA-core double-float residual, at the same
    1e-11 as the other residuals (the slice levels joined in double-float,
    passes of at most 32 right-hand sides with an exact accumulator per level;
    the star's S takes 90 columns in three passes)."""
    c = geometry.make(kind, n, **params)
    A = operators.cfie_matrix(c, omega, omega, "hard")
    X = inputs.random_density(n, nrhs, seed=11 * n + nrhs)
    op = ctx.geometry(kind, **params).discretise(n, omega, bc="hard", precision="fp32")
    y2, y1 = empty(nrhs, n), empty(nrhs, n)
    op.set_residual_variant(2)
    op.apply_residual(to_dev(X), y2)
    op.set_residual_variant(1)
    op.apply_residual(to_dev(X), y1)
    assert np.max(col_rel(to_host(y2), (A @ X.T).T)) < TOL_RES
    assert np.max(col_rel(to_host(y2), to_host(y1))) < TOL_RES


@pytest.mark.parametrize("kind,params,n,omega,nrhs", [
    ("kite", {}, 600, 30.0, 3),
    ("kite", {}, 2000, 200.0, 17),
    ("star", {"a": [0, 0, 0, 0, 0.3], "b": [0] * 5}, 1502, 120.0, 1),
    ("ellipse", {"a": 1.0, "b": 0.5}, 1000, 90.0, 5),
])
def test_hard_residual_matvec_parity(ctx, kind, params, n, omega, nrhs):
    """Sound-hard operator (eq. 2, N by Maue's identity): the double-float
    sums of S and D' with the FP64 spectral derivatives."""
    c = geometry.make(kind, n, **params)
    A = operators.cfie_matrix(c, omega, omega, "hard")
    X = inputs.random_density(n, nrhs, seed=5 * n + nrhs)
    op = ctx.geometry(kind, **params).discretise(n, omega, bc="hard", precision="fp32")
    op.set_residual_variant(1)
    y = empty(nrhs, n)
    op.apply_residual(to_dev(X), y)
    assert np.max(col_rel(to_host(y), (A @ X.T).T)) < TOL_RES
    y64 = empty(nrhs, n)
    op.apply_fp64(to_dev(X), y64)
    assert np.max(col_rel(to_host(y), to_host(y64))) < TOL_RES


def test_residual_of_fp64_operators_is_the_fp64_kernel(ctx):
    n, w = 600, 30.0
    X = to_dev(inputs.random_density(n, 3, seed=2))
    for bc in ("soft", "hard"):
        op = ctx.kite().discretise(n, w, bc=bc, precision="fp64")
        y1, y2 = empty(3, n), empty(3, n)
        op.apply_residual(X, y1)
        op.apply_fp64(X, y2)
        assert np.array_equal(to_host(y1), to_host(y2))


@pytest.mark.slow
def test_kite_n32768_residual_rows(ctx):
    spec = inputs.WORKLOADS["kite"]
    n, w, nrhs = spec["n"], spec["omega"], spec["nrhs"]
    c = geometry.kite(n)
    rows = np.array([0, 3, 777, 8192, 16384, 24000, n - 1])
    Arows = operators.soft_rows(c, w, w, rows, kress.kress_weights(n))
    X = inputs.random_density(n, nrhs, seed=23)
    op = ctx.kite().discretise(n, w, precision="fp32")
    y = empty(nrhs, n)
    op.apply_residual(to_dev(X), y)
    got = to_host(y)[:, rows]
    want = (Arows @ X.T).T
    assert np.linalg.norm(got - want) / np.linalg.norm(want) < 1e-10
