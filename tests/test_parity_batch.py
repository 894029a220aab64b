"""GPU parity of batches: many stored operators contracted by one persistent
stream-K tensor-core launch (CUDA graph), lockstep GMRES over all their
right-hand sides, and the same result alone and in the mix.

Tolerances as for one operator: batched stored matvec <= 1e-4 relative per
right-hand side against the oracle; refined solves <= 1e-6 against LU; a
solve alone and inside the batch agree to 1e-6."""
import numpy as np
import pytest

from oracle import geometry, operators, solvers
from paper_1408_1578_gb300 import inputs
from tests.gpu_util import col_rel, empty, to_dev, to_host

pytestmark = pytest.mark.gpu

TOL_STORED = 1e-4
TOL_REFINED = 1e-6


@pytest.fixture(scope="module")
def ctx():
    from paper_1408_1578_gb300 import cfie
    c = cfie.Context(0)
    yield c
    c.close()


def _stars(count, seed, n_lo, n_hi, nrhs):
    return inputs.random_stars(count=count, seed=seed, n_lo=n_lo, n_hi=n_hi, nrhs=nrhs)


def _flat(blocks):
    import torch
    return torch.cat([b.reshape(-1) for b in blocks]).contiguous()


@pytest.fixture(scope="module")
def small_batch(ctx):
    specs = _stars(5, seed=7, n_lo=300, n_hi=1600, nrhs=32)
    specs[1]["nrhs"] = 5
    specs[3]["nrhs"] = 40          # two 32-column jobs
    ops = [ctx.fourier_star(s["a"], s["b"]).discretise(s["n"], s["omega"], precision="tensor",
                                                        layout="stored") for s in specs]
    return specs, ops


def test_batched_stored_matvec(ctx, small_batch):
    from paper_1408_1578_gb300 import cfie
    specs, ops = small_batch
    b = cfie.Batch(ctx, ops, [s["nrhs"] for s in specs])
    Xs = [inputs.random_density(s["n"], s["nrhs"], seed=11 + k) for k, s in enumerate(specs)]
    x = _flat([to_dev(X) for X in Xs])
    y = x.clone()
    b.apply(x, y)
    for k, s in enumerate(specs):
        c = geometry.fourier_star(s["n"], s["a"], s["b"])
        A = operators.soft_matrix(c, s["omega"], s["omega"])
        got = to_host(b.block(y, k))
        assert np.max(col_rel(got, (A @ Xs[k].T).T)) < TOL_STORED
        # the operator on its own: same kernel, but another stream-K split of the
        # source range, so only the FP32 summation order differs
        yk = b.block(y, k).clone()
        ops[k].apply(b.block(x, k).contiguous(), yk)
        assert np.max(col_rel(to_host(yk), got)) < 1e-5
    b.close()


def test_batched_refined_solve_alone_and_in_the_mix(ctx, small_batch):
    from paper_1408_1578_gb300 import cfie
    specs, ops = small_batch
    nr = [s["nrhs"] for s in specs]
    b = cfie.Batch(ctx, ops, nr)
    fs = []
    for k, s in enumerate(specs):
        f = to_dev(np.zeros((s["nrhs"], s["n"]), complex))
        ops[k].rhs_plane_waves(inputs.directions(s["nrhs"]), f)
        fs.append(f)
    f = _flat(fs)
    x = f.clone().zero_()
    its, rel, _ = b.gmres_solve(f, x, rtol=1e-8, restart=60, maxit=3000)
    assert np.all(rel <= 1e-8)
    for k, s in enumerate(specs):
        c = geometry.fourier_star(s["n"], s["a"], s["b"])
        A = operators.soft_matrix(c, s["omega"], s["omega"])
        Q = solvers.lu_solve(A, to_host(fs[k]).T).T
        xk = to_host(b.block(x, k))
        assert np.max(col_rel(xk, Q)) < TOL_REFINED
        alone = fs[k].clone().zero_()
        its_a, rel_a, _ = ops[k].gmres_solve(fs[k], alone, rtol=1e-8, restart=60, maxit=3000)
        assert np.all(rel_a <= 1e-8)
        assert np.max(col_rel(to_host(alone), xk)) < TOL_REFINED
    b.close()


@pytest.mark.parametrize("basis32", [True, False])
def test_batch_of_matrix_free_fp32_operators(ctx, basis32):
    from paper_1408_1578_gb300 import cfie
    specs = _stars(3, seed=9, n_lo=400, n_hi=1200, nrhs=4)
    ops = [ctx.fourier_star(s["a"], s["b"]).discretise(s["n"], s["omega"], precision="fp32")
           for s in specs]
    b = cfie.Batch(ctx, ops, [4, 4, 4])
    fs = []
    for k, s in enumerate(specs):
        f = to_dev(np.zeros((4, s["n"]), complex))
        ops[k].rhs_plane_waves(inputs.directions(4), f)
        fs.append(f)
    f = _flat(fs)
    x = f.clone().zero_()
    b.set_inner_basis(basis32)
    its, rel, _ = b.gmres_solve(f, x, rtol=1e-8, restart=40, maxit=2000)
    assert np.all(rel <= 1e-8)
    assert b.last_stats()["basis_fp32"] == int(basis32)
    for k, s in enumerate(specs):
        c = geometry.fourier_star(s["n"], s["a"], s["b"])
        A = operators.soft_matrix(c, s["omega"], s["omega"])
        Q = solvers.lu_solve(A, to_host(fs[k]).T).T
        assert np.max(col_rel(to_host(b.block(x, k)), Q)) < TOL_REFINED
    b.close()


def test_batch_arguments(ctx, small_batch):
    from paper_1408_1578_gb300 import cfie
    specs, ops = small_batch
    op64 = ctx.kite().discretise(256, 20.0, precision="fp64")
    with pytest.raises(cfie.CfieError):
        cfie.Batch(ctx, [ops[0], op64], [1, 1])      # mixed precisions
    with pytest.raises(cfie.CfieError):
        cfie.Batch(ctx, [ops[0]], [0])               # no right-hand side


def test_contraction_dealings_and_tuning(ctx, small_batch):
    """The autotuner times every dealing of the persistent contraction once and
    keeps one; each dealing gives the oracle's product (they differ only in the
    order of the FP32 partial sums)."""
    from paper_1408_1578_gb300 import cfie
    specs, ops = small_batch
    b = cfie.Batch(ctx, ops, [s["nrhs"] for s in specs])
    d, ms = b.tuning()
    assert d in (0, 1, 2)
    Xs = [inputs.random_density(s["n"], s["nrhs"], seed=31 + k) for k, s in enumerate(specs)]
    x = _flat([to_dev(X) for X in Xs])
    want = []
    for k, s in enumerate(specs):
        c = geometry.fourier_star(s["n"], s["a"], s["b"])
        A = operators.soft_matrix(c, s["omega"], s["omega"])
        want.append((A @ Xs[k].T).T)
    outs = []
    for deal in (0, 1, 2):
        b.set_dealing(deal)
        assert b.tuning()[0] == deal
        y = x.clone()
        b.apply(x, y)
        outs.append(to_host(y))
        for k in range(len(specs)):
            assert np.max(col_rel(to_host(b.block(y, k)), want[k])) < TOL_STORED
    assert np.max(np.abs(outs[0] - outs[1])) <= 1e-6 * np.max(np.abs(outs[0]))
    assert np.max(np.abs(outs[0] - outs[2])) <= 1e-5 * np.max(np.abs(outs[0]))
    # the same shape again: the choice comes from the process's memory
    b2 = cfie.Batch(ctx, ops, [s["nrhs"] for s in specs])
    d2, ms2 = b2.tuning()
    assert d2 == d and not any(ms2)
    assert ctx.lib.cfie_batch_set_dealing(b2.h, 3) == cfie.CFIE_EINVAL
    b2.close()
    b.close()


def test_discretise_many_equals_one_by_one(ctx):
    """cfie_discretise_many sets operators up on worker streams; each one is
    the operator cfie_discretise makes (the same products, bit for bit), for
    the stored and the matrix-free forms; geometries of two contexts are
    refused."""
    from paper_1408_1578_gb300 import cfie
    specs = inputs.random_stars(count=5, seed=33, n_lo=300, n_hi=900, nrhs=3)
    for prec, layout in (("tensor", "stored"), ("fp32", "matrix_free")):
        geoms = [ctx.fourier_star(s["a"], s["b"]) for s in specs]
        many = ctx.discretise_many(geoms, [s["n"] for s in specs], [s["omega"] for s in specs],
                                   precision=prec, layout=layout)
        for k, s in enumerate(specs):
            one = geoms[k].discretise(s["n"], s["omega"], precision=prec, layout=layout)
            X = to_dev(inputs.random_density(s["n"], 3, seed=40 + k))
            y1, y2 = empty(3, s["n"]), empty(3, s["n"])
            many[k].apply(X, y1)
            one.apply(X, y2)
            assert np.array_equal(to_host(y1), to_host(y2))
            one.close()
            many[k].close()
        for g in geoms:
            g.close()
    other = cfie.Context(0)
    g1 = ctx.fourier_star(specs[0]["a"], specs[0]["b"])
    g2 = other.fourier_star(specs[1]["a"], specs[1]["b"])
    with pytest.raises(cfie.CfieError):
        ctx.discretise_many([g1, g2], [specs[0]["n"], specs[1]["n"]],
                            [specs[0]["omega"], specs[1]["omega"]], precision="fp32")
    g1.close()
    g2.close()
    other.close()
