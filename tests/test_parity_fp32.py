"""GPU parity of the FP32 fused matrix-free matvec and of the mixed-precision
refined GMRES against the FP64 oracle, through the C ABI.

Tolerances: raw FP32 matvec <= 1e-4 relative per right-hand side (the
implementation lands near 1e-6); refined solve <= 1e-6 relative error against
the oracle's FP64 (LU) solution when driven to a residual of 1e-8."""
import numpy as np
import pytest

from oracle import geometry, kress, operators, solvers
from paper_1408_1578_gb300 import inputs
from tests.gpu_util import col_rel, empty, to_dev, to_host, zeros

pytestmark = pytest.mark.gpu

TOL_FP32 = 1e-4
TOL_REFINED = 1e-6


@pytest.fixture(scope="module")
def ctx():
    from paper_1408_1578_gb300 import cfie
    c = cfie.Context(0)
    yield c
    c.close()


CASES = [
    # omega large enough that most pairs take the on-the-fly asymptotic path
    ("kite", {}, 2000, 200.0, "soft", 3),
    ("kite", {}, 2000, 200.0, "soft", 17),
    ("kite", {}, 2000, 200.0, "hard", 5),
    ("star", {"a": [0, 0, 0, 0, 0.3], "b": [0] * 5}, 1502, 120.0, "hard", 16),
    ("star", {"a": [0.03, -0.02, 0.04], "b": [0.01, 0.05, -0.03]}, 3000, 450.0, "soft", 64),
    ("ellipse", {"a": 1.0, "b": 0.5}, 1000, 90.0, "soft", 9),
    # large scaled coordinates: omega |z| up to 2^14 (coarse coordinate grid,
    # phase error ~2e-6 rad), both summation forms, both conditions
    ("circle", {}, 2048, 12000.0, "soft", 3),
    ("circle", {}, 2048, 12000.0, "soft", 12),
    ("circle", {}, 2048, 12000.0, "hard", 8),
    # small problems: the near band covers every pair
    ("circle", {}, 64, 2.0, "soft", 2),
    ("circle", {}, 64, 2.0, "hard", 2),
]


@pytest.mark.parametrize("kind,params,n,omega,bc,nrhs", CASES)
def test_fp32_matvec_parity(ctx, kind, params, n, omega, bc, nrhs):
    c = geometry.make(kind, n, **params)
    A = operators.cfie_matrix(c, omega, omega, bc)
    X = inputs.random_density(n, nrhs, seed=n + 7 * nrhs)
    op = ctx.geometry(kind, **params).discretise(n, omega, bc=bc, precision="fp32")
    y = empty(nrhs, n)
    op.apply(to_dev(X), y)
    err = np.max(col_rel(to_host(y), (A @ X.T).T))
    assert err < TOL_FP32, err
    # the same operator's FP64 matvec (used for true residuals) stays FP64-exact:
    # 1e-12, or the FP64 resolution of the phase omega r when that is coarser
    # (a few roundings of 2^-53 relative on omega r up to omega x diameter:
    # ~1e-11 for the omega = 12000 circle)
    y64 = empty(nrhs, n)
    op.apply_fp64(to_dev(X), y64)
    diam = np.hypot(*np.ptp(c.z, axis=0))      # bounding-box diagonal >= diameter
    tol64 = max(1e-12, 4e-16 * omega * diam)
    assert np.max(col_rel(to_host(y64), (A @ X.T).T)) < tol64


def test_fp32_matvec_plane_wave_data(ctx):
    """Smooth data (the right-hand sides themselves) through the FP32 matvec."""
    n, w = 2000, 200.0
    c = geometry.kite(n)
    A = operators.soft_matrix(c, w, w)
    F = operators.plane_wave_rhs(c, w, inputs.directions(4), "soft").T
    op = ctx.kite().discretise(n, w, precision="fp32")
    y = empty(4, n)
    op.apply(to_dev(F), y)
    assert np.max(col_rel(to_host(y), (A @ F.T).T)) < TOL_FP32


@pytest.mark.parametrize("bc", ["soft", "hard"])
def test_refined_solve_matches_fp64_solution(ctx, bc):
    n, w, nrhs = 2000, 200.0, 4
    c = geometry.kite(n)
    A = operators.cfie_matrix(c, w, w, bc)
    F = operators.plane_wave_rhs(c, w, inputs.directions(nrhs), bc)
    Q = solvers.lu_solve(A, F).T
    op = ctx.kite().discretise(n, w, bc=bc, precision="fp32")
    f = to_dev(F.T)
    x = zeros(nrhs, n)
    its, rel, _ = op.gmres_solve(f, x, rtol=1e-8, restart=80, maxit=3000)
    stats = op.last_stats()
    assert np.all(rel <= 1e-8)
    assert stats["refinements"] >= 1 and stats["fp64_matvecs"] >= 2
    assert np.max(col_rel(to_host(x), Q)) < TOL_REFINED


@pytest.mark.slow
def test_kite_n32768_fp32_sampled_rows(ctx):
    """Kite, omega = 2048, n = 32768, 64 right-hand sides (the precision
    workload): FP32 matvec rows sampled against the oracle's FP64 rows."""
    spec = inputs.WORKLOADS["kite"]
    n, w, nrhs = spec["n"], spec["omega"], spec["nrhs"]
    c = geometry.kite(n)
    R = kress.kress_weights(n)
    rows = np.array([0, 1, 2, 100, 8191, 8192, 16384, 16390, 24576, 30000, n - 2, n - 1])
    Arows = operators.soft_rows(c, w, w, rows, R)
    X = inputs.random_density(n, nrhs, seed=19)
    op = ctx.kite().discretise(n, w, precision="fp32")
    y = empty(nrhs, n)
    op.apply(to_dev(X), y)
    got = to_host(y)[:, rows]
    want = (Arows @ X.T).T
    assert np.linalg.norm(got - want) / np.linalg.norm(want) < TOL_FP32


@pytest.mark.slow
def test_kite_n32768_refined_residual_rows(ctx):
    """Full-size refined solve: the returned FP64 residual meets 1e-8, and the
    oracle's rows of f - A x agree with it (sampled property at full size)."""
    spec = inputs.WORKLOADS["kite"]
    n, w = spec["n"], spec["omega"]
    nrhs = 8
    theta = inputs.directions(nrhs)
    op = ctx.kite().discretise(n, w, precision="fp32")
    f = empty(nrhs, n)
    op.rhs_plane_waves(theta, f)
    x = zeros(nrhs, n)
    its, rel, _ = op.gmres_solve(f, x, rtol=1e-8, restart=80, maxit=4000)
    assert np.all(rel <= 1e-8)
    c = geometry.kite(n)
    rows = np.array([0, 5000, 12345, 20000, 32767])
    Arows = operators.soft_rows(c, w, w, rows, kress.kress_weights(n))
    F = operators.plane_wave_rhs(c, w, theta, "soft")
    res = F[rows, :] - Arows @ to_host(x).T
    # per-row residual relative to the data scale (|f| = 1 pointwise)
    assert np.max(np.abs(res)) < 1e-6


def test_band_too_wide_is_rejected_or_served(ctx):
    """A tiny problem: the band covers every pair.  The CUDA-core sums of its
    FP64-evaluated entries stay within FP32 rounding (1e-6); the tensor-core
    sums within their bf16 hi + lo operands (1e-4, the raw FP32 bound)."""
    n, w = 16, 0.5
    c = geometry.circle(n)
    A = operators.soft_matrix(c, w, w)
    X = inputs.random_density(n, 1, seed=1)
    op = ctx.circle().discretise(n, w, precision="fp32")
    y = empty(1, n)
    for variant, tol in ((1, 1e-6), (2, TOL_FP32)):
        op.set_variant(variant)
        op.apply(to_dev(X), y)
        assert np.max(col_rel(to_host(y), (A @ X.T).T)) < tol, variant


# ---------------------------------------------------------------------------
# the same FP32 entries summed on the tensor cores (cfie_op_set_variant(op, 2))
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("kind,params,n,omega,nrhs", [
    ("kite", {}, 2000, 200.0, 1),
    ("kite", {}, 2000, 200.0, 3),
    ("kite", {}, 2000, 200.0, 8),
    ("kite", {}, 2000, 200.0, 33),
    ("star", {"a": [0.03, -0.02, 0.04], "b": [0.01, 0.05, -0.03]}, 3000, 450.0, 64),
    ("ellipse", {"a": 1.0, "b": 0.5}, 1000, 90.0, 32),
    ("circle", {}, 64, 2.0, 9),
])
def test_fp32_tensor_core_sums(ctx, kind, params, n, omega, nrhs):
    c = geometry.make(kind, n, **params)
    A = operators.soft_matrix(c, omega, omega)
    X = inputs.random_density(n, nrhs, seed=4 * n + nrhs)
    op = ctx.geometry(kind, **params).discretise(n, omega, precision="fp32")
    op.set_variant(2)
    y = empty(nrhs, n)
    op.apply(to_dev(X), y)
    assert np.max(col_rel(to_host(y), (A @ X.T).T)) < TOL_FP32
    op.set_variant(1)
    y1 = empty(nrhs, n)
    op.apply(to_dev(X), y1)
    assert np.max(col_rel(to_host(y), to_host(y1))) < TOL_FP32


def test_fp32_tensor_core_refined_solve(ctx):
    n, w, nrhs = 2000, 200.0, 40
    c = geometry.kite(n)
    A = operators.soft_matrix(c, w, w)
    F = operators.plane_wave_rhs(c, w, inputs.directions(nrhs), "soft")
    Q = solvers.lu_solve(A, F).T
    op = ctx.kite().discretise(n, w, precision="fp32")
    op.set_variant(2)
    x = zeros(nrhs, n)
    its, rel, _ = op.gmres_solve(to_dev(F.T), x, rtol=1e-8, restart=80, maxit=3000)
    assert np.all(rel <= 1e-8)
    assert np.max(col_rel(to_host(x), Q)) < TOL_REFINED


def test_tensor_core_variant_arguments(ctx):
    from paper_1408_1578_gb300 import cfie
    op64 = ctx.kite().discretise(256, 20.0, precision="fp64")
    with pytest.raises(cfie.CfieError):
        op64.set_variant(2)
    op = ctx.kite().discretise(256, 20.0, precision="fp32")
    with pytest.raises(cfie.CfieError):
        op.set_variant(3)


@pytest.mark.parametrize("kind,params,n,omega,nrhs", [
    ("kite", {}, 2000, 200.0, 1),
    ("kite", {}, 2000, 200.0, 5),
    ("kite", {}, 2000, 200.0, 8),
    ("kite", {}, 2000, 200.0, 30),                    # S pass of 90 right-hand sides
    ("star", {"a": [0, 0, 0, 0, 0.3], "b": [0] * 5}, 1502, 120.0, 16),
    ("ellipse", {"a": 1.0, "b": 0.5}, 1000, 90.0, 64),
])
def test_fp32_tensor_core_sums_hard(ctx, kind, params, n, omega, nrhs):
    """Sound-hard operator (eq. 2, N by Maue's identity) with the source sums of
    S and D' on the tensor cores."""
    c = geometry.make(kind, n, **params)
    A = operators.cfie_matrix(c, omega, omega, "hard")
    X = inputs.random_density(n, nrhs, seed=7 * n + nrhs)
    op = ctx.geometry(kind, **params).discretise(n, omega, bc="hard", precision="fp32")
    op.set_variant(2)
    y = empty(nrhs, n)
    op.apply(to_dev(X), y)
    assert np.max(col_rel(to_host(y), (A @ X.T).T)) < TOL_FP32
    op.set_variant(1)
    y1 = empty(nrhs, n)
    op.apply(to_dev(X), y1)
    assert np.max(col_rel(to_host(y), to_host(y1))) < TOL_FP32


def test_fp32_tensor_core_refined_solve_hard(ctx):
    n, w, nrhs = 1502, 120.0, 12
    params = {"a": [0, 0, 0, 0, 0.3], "b": [0] * 5}
    c = geometry.fourier_star(n, params["a"], params["b"])
    A = operators.cfie_matrix(c, w, w, "hard")
    F = operators.plane_wave_rhs(c, w, inputs.directions(nrhs), "hard")
    Q = solvers.lu_solve(A, F).T
    op = ctx.fourier_star(params["a"], params["b"]).discretise(n, w, bc="hard", precision="fp32")
    op.set_variant(2)
    x = zeros(nrhs, n)
    its, rel, _ = op.gmres_solve(to_dev(F.T), x, rtol=1e-8, restart=80, maxit=3000)
    assert np.all(rel <= 1e-8)
    assert op.last_stats()["matvec_variant"] == 2
    assert np.max(col_rel(to_host(x), Q)) < TOL_REFINED


@pytest.mark.parametrize("bc", ["soft", "hard"])
def test_refined_solve_basis_precisions(ctx, bc):
    """The inner Krylov basis in FP32 (default) and in FP64 reach the same
    FP64 solution; the counters say which basis ran."""
    n, w, nrhs = 1500, 150.0, 6
    c = geometry.kite(n)
    A = operators.cfie_matrix(c, w, w, bc)
    F = operators.plane_wave_rhs(c, w, inputs.directions(nrhs), bc)
    Q = solvers.lu_solve(A, F).T
    op = ctx.kite().discretise(n, w, bc=bc, precision="fp32")
    got = {}
    for fp32 in (True, False):
        op.set_inner_basis(fp32)
        x = zeros(nrhs, n)
        its, rel, _ = op.gmres_solve(to_dev(F.T), x, rtol=1e-8, restart=40, maxit=3000)
        st = op.last_stats()
        assert st["basis_fp32"] == int(fp32)
        assert st["arnoldi_elems"] > 0
        assert np.all(rel <= 1e-8)
        got[fp32] = to_host(x)
        assert np.max(col_rel(got[fp32], Q)) < TOL_REFINED
    assert np.max(col_rel(got[True], got[False])) < TOL_REFINED
    op64 = ctx.kite().discretise(n, w, bc=bc, precision="fp64")
    x = zeros(nrhs, n)
    op64.gmres_solve(to_dev(F.T), x, rtol=1e-10, restart=40, maxit=3000)
    assert op64.last_stats()["basis_fp32"] == 0 and op64.last_stats()["matvec_variant"] == 0
