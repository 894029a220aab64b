"""GPU parity of the directional preconditioner of Section 2 against the
oracle's construction (oracle.directional.Directional), through the C ABI.

The operator is the sound-soft CFIE of eq. 1 on a curve sampled at
n = 4^q p points equispaced in arclength (the library's samples on the GPU,
the oracle's own arclength map on the CPU), p = 8 points per wavelength and
eta = omega / 2, the setting of Table 1.  Checked:

* the block coefficients e_ij (the nodal least-squares constants of the
  rank-1 forms, the oracle's e_from="nodes"): from FP64 entries within 1e-9
  of the largest, from a refined operator's FP32 entries within 1e-5;
* P v of eq. (eapp) for random right-hand sides against the oracle's apply
  with its sparse LU of W~: the GPU applies in complex64, within 1e-5;
* GMRES(80) to 1e-6 with P on the right (FP64 operator): the iteration count
  within one of the oracle's preconditioned GMRES on the same problem, and
  far below the unpreconditioned count; the refined FP32 solve with P reaches
  1e-8 and the oracle's LU solution within 1e-6;
* invalid uses: a sound-hard operator, nodes that are not the arclength
  samples, n != 4^q p."""
import numpy as np
import pytest

from oracle import directional, geometry, operators, solvers
from paper_1408_1578_gb300 import inputs
from tests.gpu_util import col_rel, empty, to_dev, to_host, zeros

pytestmark = pytest.mark.gpu

P_PPW = 8


@pytest.fixture(scope="module")
def ctx():
    from paper_1408_1578_gb300 import cfie
    c = cfie.Context(0)
    yield c
    c.close()


def _setup(kind, q, params):
    arc = geometry.Arclength(kind, **params)
    n = 4**q * P_PPW
    omega = 2.0 * np.pi * (n / P_PPW) / arc.L
    return arc, n, omega, 0.5 * omega


@pytest.fixture(scope="module", params=[("ellipse", 4, {"a": 1.0, "b": 0.5}),
                                        ("kite", 4, {})],
                ids=["ellipse-q4", "kite-q4"])
def case(request, ctx):
    from paper_1408_1578_gb300 import cfie
    kind, q, params = request.param
    arc, n, omega, eta = _setup(kind, q, params)
    A = operators.soft_matrix(arc.curve(n), omega, eta)
    ref = directional.Directional(arc, q, P_PPW, omega, eta=eta, A=A, e_from="nodes")
    z, dz, ddz, _ = cfie.arclength_samples(kind, n, **params)
    op = ctx.samples(z, dz, ddz).discretise(n, omega, eta=eta, precision="fp64")
    prec = op.dirprec(kind, q, P_PPW, **params)
    return dict(kind=kind, q=q, params=params, arc=arc, n=n, omega=omega, eta=eta, A=A, ref=ref,
                op=op, prec=prec, z=z, dz=dz, ddz=ddz)


def test_block_coefficients(case):
    ref, e = case["ref"], case["prec"].coefficients()
    m = ref.m
    assert e.shape == (m, m)
    want = np.zeros((m, m), dtype=np.complex128)
    E = ref.E.toarray()
    for (i, j), (ki, kj) in ref.kidx.items():
        want[i, j] = E[ref.koff[i] + ki, ref.koff[j] + kj]
    assert np.all(np.diag(e) == 0)
    assert np.max(np.abs(e - want)) < 1e-9 * np.max(np.abs(want))


def test_block_coefficients_from_fp32_entries(ctx, case):
    """A refined (FP32) operator builds E from its FP32 entries: within 1e-5
    of the largest e_ij."""
    ref = case["ref"]
    op32 = ctx.samples(case["z"], case["dz"], case["ddz"]).discretise(
        case["n"], case["omega"], eta=case["eta"], precision="fp32")
    prec = op32.dirprec(case["kind"], case["q"], P_PPW, **case["params"])
    e = prec.coefficients()
    want = np.zeros_like(e)
    E = ref.E.toarray()
    for (i, j), (ki, kj) in ref.kidx.items():
        want[i, j] = E[ref.koff[i] + ki, ref.koff[j] + kj]
    assert np.max(np.abs(e - want)) < 1e-5 * np.max(np.abs(want))
    prec.close()
    op32.close()


def test_apply_matches_oracle(case):
    n, ref = case["n"], case["ref"]
    X = inputs.random_density(n, 5, seed=17)
    y = empty(5, n)
    case["prec"].apply(to_dev(X), y)
    want = np.stack([ref.apply(X[k]) for k in range(5)])
    assert np.max(col_rel(to_host(y), want)) < 1e-5


def test_apply_ragged_right_hand_sides(case):
    """17 right-hand sides (a ragged tile of the batched products): each
    column equals the apply of that column alone."""
    n = case["n"]
    X = inputs.random_density(n, 17, seed=23)
    y = empty(17, n)
    case["prec"].apply(to_dev(X), y)
    y1 = empty(1, n)
    case["prec"].apply(to_dev(X[16:17]), y1)
    assert np.max(col_rel(to_host(y)[16:17], to_host(y1))) < 1e-6


def test_preconditioned_gmres_iterations(case):
    n, omega, A, ref, op = case["n"], case["omega"], case["A"], case["ref"], case["op"]
    c = case["arc"].curve(n)
    f = operators.plane_wave_rhs(c, omega, [0.0], "soft")[:, 0]
    _, nn_ref, _ = directional.preconditioned_gmres(A, None, f, rtol=1e-6, restart=80)
    _, np_ref, _ = directional.preconditioned_gmres(A, ref.apply, f, rtol=1e-6, restart=80)
    fd = to_dev(f[None, :])
    x = zeros(1, n)
    op.set_preconditioner(None)
    its_n, rel_n, _ = op.gmres_solve(fd, x, rtol=1e-6, restart=80, maxit=500)
    op.set_preconditioner(case["prec"])
    x = zeros(1, n)
    its_p, rel_p, _ = op.gmres_solve(fd, x, rtol=1e-6, restart=80, maxit=500)
    op.set_preconditioner(None)
    assert rel_n[0] <= 1e-6 and rel_p[0] <= 1e-6
    assert abs(int(its_n[0]) - nn_ref) <= 1
    assert abs(int(its_p[0]) - np_ref) <= 1
    assert its_p[0] < its_n[0]


def test_refined_solve_with_preconditioner(ctx, case):
    n, omega, eta, A = case["n"], case["omega"], case["eta"], case["A"]
    c = case["arc"].curve(n)
    theta = inputs.directions(4)
    F = operators.plane_wave_rhs(c, omega, theta, "soft")
    Q = solvers.lu_solve(A, F).T
    op32 = ctx.samples(case["z"], case["dz"], case["ddz"]).discretise(n, omega, eta=eta,
                                                                       precision="fp32")
    prec = op32.dirprec(case["kind"], case["q"], P_PPW, **case["params"])
    op32.set_preconditioner(prec)
    x = zeros(4, n)
    its, rel, _ = op32.gmres_solve(to_dev(F.T), x, rtol=1e-8, restart=80, maxit=2000)
    assert np.all(rel <= 1e-8)
    assert np.max(col_rel(to_host(x), Q)) < 1e-6
    op32.set_preconditioner(None)
    x0 = zeros(4, n)
    its0, _, _ = op32.gmres_solve(to_dev(F.T), x0, rtol=1e-8, restart=80, maxit=2000)
    assert np.max(its) < np.max(its0)
    prec.close()
    op32.close()


def test_invalid_uses(ctx):
    from paper_1408_1578_gb300 import cfie
    kind, q, params = "ellipse", 3, {"a": 1.0, "b": 0.5}
    arc, n, omega, eta = _setup(kind, q, params)
    z, dz, ddz, _ = cfie.arclength_samples(kind, n, **params)
    hard = ctx.samples(z, dz, ddz).discretise(n, omega, eta=eta, bc="hard", precision="fp64")
    with pytest.raises(cfie.CfieError):
        hard.dirprec(kind, q, P_PPW, **params)
    para = ctx.ellipse(1.0, 0.5).discretise(n, omega, eta=eta, precision="fp64")   # parameter nodes
    with pytest.raises(cfie.CfieError):
        para.dirprec(kind, q, P_PPW, **params)
    z2, dz2, ddz2, _ = cfie.arclength_samples(kind, 2 * n, **params)
    wrong = ctx.samples(z2, dz2, ddz2).discretise(2 * n, omega, eta=eta, precision="fp64")
    with pytest.raises(cfie.CfieError):
        wrong.dirprec(kind, q, P_PPW, **params)
    soft = ctx.samples(z, dz, ddz).discretise(n, omega, eta=eta, precision="fp64")
    prec = soft.dirprec(kind, q, P_PPW, **params)
    with pytest.raises(cfie.CfieError):
        wrong.set_preconditioner(prec)            # built for another size
    prec.close()
