"""GPU parity of the FP64 path (geometry, Kress tables, matvec, spectral
derivative, GMRES) against the FP64 oracle, through the C ABI.

Tolerance: 1e-12 relative per right-hand side for the FP64 matvec and for
solves driven to rtol 1e-14 (the FP64 path must match the oracle to 1e-12)."""
import numpy as np
import pytest

from oracle import geometry, kress, operators, solvers
from paper_1408_1578_gb300 import inputs
from tests.gpu_util import col_rel, empty, to_dev, to_host, zeros

pytestmark = pytest.mark.gpu

TOL_FP64 = 1e-12


@pytest.fixture(scope="module")
def ctx():
    from paper_1408_1578_gb300 import cfie
    c = cfie.Context(0)
    yield c
    c.close()


CASES = [
    # kind, params, n, omega, bc, nrhs   (n spans several 64-row tiles with a ragged tail)
    ("kite", {}, 1000, 40.0, "soft", 5),
    ("kite", {}, 1000, 40.0, "hard", 5),
    ("star", {"a": [0, 0, 0, 0, 0.3], "b": [0] * 5}, 600, 30.0, "hard", 17),
    ("ellipse", {"a": 1.0, "b": 0.5}, 514, 25.0, "soft", 17),
    ("circle", {}, 8, 1.5, "soft", 1),
    ("circle", {}, 8, 1.5, "hard", 2),
]


def _oracle_matrix(kind, params, n, omega, bc):
    c = geometry.make(kind, n, **params)
    return c, operators.cfie_matrix(c, omega, omega, bc)


@pytest.mark.parametrize("kind,params,n,omega,bc,nrhs", CASES)
def test_fp64_matvec_parity(ctx, kind, params, n, omega, bc, nrhs):
    _, A = _oracle_matrix(kind, params, n, omega, bc)
    X = inputs.random_density(n, nrhs, seed=n + nrhs)
    op = ctx.geometry(kind, **params).discretise(n, omega, bc=bc, precision="fp64")
    x = to_dev(X)
    y = empty(nrhs, n)
    op.apply(x, y)
    want = (A @ X.T).T
    assert np.max(col_rel(to_host(y), want)) < TOL_FP64


@pytest.mark.parametrize("bc", ["soft", "hard"])
def test_fp64_matrix_columns(ctx, bc):
    """Individual entries: A e_j against the oracle's columns."""
    n, omega = 256, 20.0
    _, A = _oracle_matrix("kite", {}, n, omega, bc)
    cols = [0, 1, 37, 128, 255]
    E = np.zeros((len(cols), n), dtype=complex)
    for k, j in enumerate(cols):
        E[k, j] = 1.0
    op = ctx.kite().discretise(n, omega, bc=bc)
    y = empty(len(cols), n)
    op.apply(to_dev(E), y)
    got = to_host(y)
    for k, j in enumerate(cols):
        err = np.abs(got[k] - A[:, j]) / np.max(np.abs(A[:, j]))
        assert np.max(err) < 1e-13, (j, np.argmax(err))


@pytest.mark.parametrize("bc", ["soft", "hard"])
def test_plane_wave_rhs_parity(ctx, bc):
    n, omega = 1000, 40.0
    c = geometry.kite(n)
    theta = inputs.directions(7)
    op = ctx.kite().discretise(n, omega, bc=bc)
    f = empty(7, n)
    op.rhs_plane_waves(theta, f)
    want = operators.plane_wave_rhs(c, omega, theta, bc).T
    # the phase omega d.z carries ~omega |z| eps of rounding on either side
    assert np.max(col_rel(to_host(f), want)) < 8 * omega * 2.2e-16


def test_disk_n1024_unrestarted_gmres(ctx):
    """Unit circle, omega = eta = 64, n = 1024, d = (1, 0), unrestarted GMRES to 1e-8."""
    w, n = 64.0, 1024
    c = geometry.circle(n)
    A = operators.soft_matrix(c, w, w)
    f_np = operators.plane_wave_rhs(c, w, [0.0], "soft")[:, 0]
    q_lu = solvers.lu_solve(A, f_np)
    x_or, its_or, _ = solvers.gmres(lambda v: A @ v, f_np, rtol=1e-8, restart=0, maxit=400)
    op = ctx.circle().discretise(n, w, bc="soft")
    f = empty(1, n)
    op.rhs_plane_waves([0.0], f)
    x = zeros(1, n)
    its, rel, _ = op.gmres_solve(f, x, rtol=1e-8, restart=0, maxit=400)
    assert rel[0] <= 1e-8
    assert abs(int(its[0]) - its_or) <= 1
    xs = to_host(x)[0]
    assert np.linalg.norm(xs - x_or) / np.linalg.norm(x_or) < 1e-7
    assert np.linalg.norm(xs - q_lu) / np.linalg.norm(q_lu) < 1e-7


@pytest.mark.parametrize("bc,restart", [("soft", 0), ("hard", 10)])
def test_fp64_solve_matches_lu(ctx, bc, restart):
    """Driven to rtol 1e-14 the FP64 GMRES reaches the LU solution to 1e-12."""
    n, w, nrhs = 800, 30.0, 3
    c = geometry.fourier_star(n, [0, 0, 0, 0, 0.3], [0] * 5)
    A = operators.cfie_matrix(c, w, w, bc)
    F = operators.plane_wave_rhs(c, w, inputs.directions(nrhs), bc)
    Q = solvers.lu_solve(A, F).T
    op = ctx.fourier_star([0, 0, 0, 0, 0.3], [0] * 5).discretise(n, w, bc=bc)
    f = to_dev(F.T)
    x = zeros(nrhs, n)
    its, rel, _ = op.gmres_solve(f, x, rtol=1e-14, restart=restart, maxit=500)
    assert np.all(rel <= 1e-14)
    assert np.max(col_rel(to_host(x), Q)) < TOL_FP64


def test_initial_guess_is_used(ctx):
    n, w = 400, 12.0
    c = geometry.kite(n)
    A = operators.soft_matrix(c, w, w)
    F = operators.plane_wave_rhs(c, w, [0.3], "soft").T
    Q = solvers.lu_solve(A, F.T).T
    op = ctx.kite().discretise(n, w)
    x = to_dev(Q)
    its, rel, _ = op.gmres_solve(to_dev(F), x, rtol=1e-10, restart=20, maxit=50)
    assert its[0] == 0 and rel[0] <= 1e-10


@pytest.mark.slow
def test_star_n4096_full_size(ctx):
    """Sound-hard star r = 1 + 0.3 cos 5t, omega = 256, n = 4096, 16 directions:
    FP64 matvec and solve against the oracle's assembled matrix and LU."""
    spec = inputs.WORKLOADS["star"]
    n, w, nrhs = spec["n"], spec["omega"], spec["nrhs"]
    c = geometry.make("star", n, **spec["params"])
    A = operators.hard_matrix(c, w, w)
    theta = inputs.directions(nrhs)
    F = operators.plane_wave_rhs(c, w, theta, "hard")
    op = ctx.geometry("star", **spec["params"]).discretise(n, w, bc="hard")
    X = inputs.random_density(n, 4, seed=3)
    y = empty(4, n)
    op.apply(to_dev(X), y)
    assert np.max(col_rel(to_host(y), (A @ X.T).T)) < TOL_FP64
    f = empty(nrhs, n)
    op.rhs_plane_waves(theta, f)
    assert np.max(col_rel(to_host(f), F.T)) < 8 * w * 2.2e-16
    x = zeros(nrhs, n)
    its, rel, _ = op.gmres_solve(f, x, rtol=1e-13, restart=80, maxit=2000)
    Q = solvers.lu_solve(A, F).T
    assert np.all(rel <= 1e-13)
    assert np.max(col_rel(to_host(x), Q)) < 1e-11


@pytest.mark.slow
def test_kite_n32768_sampled_rows(ctx):
    """Kite, omega = 2048, n = 32768, 64 right-hand sides: FP64 matvec rows
    sampled against the oracle's rows (the full oracle matvec is too slow)."""
    spec = inputs.WORKLOADS["kite"]
    n, w = spec["n"], spec["omega"]
    nrhs = 8
    c = geometry.kite(n)
    R = kress.kress_weights(n)
    rows = np.array([0, 1, 4095, 8192, 16384, 16385, 30000, n - 1])
    Arows = operators.soft_rows(c, w, w, rows, R)
    X = inputs.random_density(n, nrhs, seed=11)
    op = ctx.kite().discretise(n, w)
    y = empty(nrhs, n)
    op.apply(to_dev(X), y)
    got = to_host(y)[:, rows]
    want = (Arows @ X.T).T
    # the phase omega r is only known to ~omega r * eps ~ 1e-12 at this size
    assert np.max(np.abs(got - want) / np.abs(want)) < 5e-11


def test_invalid_arguments(ctx):
    from paper_1408_1578_gb300 import cfie
    g = ctx.circle()
    for bad in [dict(n=7), dict(n=6), dict(n=1001), dict(omega=-1.0), dict(omega=float("nan"))]:
        kw = dict(n=64, omega=5.0)
        kw.update(bad)
        with pytest.raises(cfie.CfieError) as e:
            g.discretise(kw["n"], kw["omega"])
        assert e.value.status == cfie.CFIE_EINVAL
    op = g.discretise(64, 5.0)
    x = zeros(1, 64)
    with pytest.raises(cfie.CfieError):
        op.apply(x, x)                            # overlapping buffers
    with pytest.raises(cfie.CfieError):
        op.apply(x, x.data_ptr() + 8, nrhs=1)     # misaligned output
    st = ctx.lib.cfie_apply(op.h, x.data_ptr(), empty(1, 64).data_ptr(), 0)
    assert st == cfie.CFIE_EINVAL
    with pytest.raises(cfie.CfieError):
        ctx.fourier_star([0.7], [0.5])            # r(t) would change sign
