"""GPU tests of the request server: results of concurrently served requests
equal the same solves run alone (and the oracle's LU solutions), admission by
HBM footprint limits how many run at once, bad requests are refused."""
import time

import numpy as np
import pytest

from oracle import geometry, operators, solvers
from paper_1408_1578_gb300 import inputs
from tests.gpu_util import col_rel, to_dev, to_host, zeros

pytestmark = pytest.mark.gpu

TOL_REFINED = 1e-6


def _requests():
    reqs = inputs.poisson_requests(count=8, rate=200.0, seed=77, n_lo=600, n_hi=2400)
    for k, r in enumerate(reqs):
        r["nrhs"] = 1 + (k * 5) % 6
    return reqs


def test_served_results_equal_alone_and_oracle():
    from paper_1408_1578_gb300 import cfie
    reqs = _requests()
    srv = cfie.Server(0, hbm_budget_bytes=48 << 30, slots=4)
    tickets = []
    for r in reqs:
        tickets.append(srv.submit(r["a"], r["b"], r["n"], r["omega"], nrhs=r["nrhs"], bc=r["bc"],
                                  rtol=1e-8, restart=60))
    assert srv.wait_all(300)
    stats = srv.stats()
    assert stats["completed"] == len(reqs)
    assert stats["peak_running"] >= 2          # work overlapped on the device
    ctx = cfie.Context(0)
    for r, t in zip(reqs, tickets):
        out = srv.poll(t, want_x=True)
        assert out["done"] and out["status"] == cfie.CFIE_OK, out.get("error")
        assert out["relres_max"] <= 1e-8
        assert out["latency_s"] >= out["service_s"] > 0
        # the same solve alone, through the operator API
        op = ctx.fourier_star(r["a"], r["b"]).discretise(r["n"], r["omega"], bc=r["bc"],
                                                          precision="fp32")
        f = zeros(r["nrhs"], r["n"])
        op.rhs_plane_waves(inputs.directions(r["nrhs"]), f)
        x = zeros(r["nrhs"], r["n"])
        op.gmres_solve(f, x, rtol=1e-8, restart=60, maxit=4000)
        assert np.max(col_rel(out["x"], to_host(x))) < TOL_REFINED
        # and the oracle's LU solution
        c = geometry.fourier_star(r["n"], r["a"], r["b"])
        A = operators.cfie_matrix(c, r["omega"], r["omega"], r["bc"])
        Q = solvers.lu_solve(A, to_host(f).T).T
        assert np.max(col_rel(out["x"], Q)) < TOL_REFINED
        op.close()
        srv.release(t)
    ctx.close()
    srv.close()


def test_admission_by_footprint():
    from paper_1408_1578_gb300 import cfie
    reqs = _requests()[:4]
    # a budget below two requests' footprints: one solve at a time
    srv = cfie.Server(0, hbm_budget_bytes=1, slots=4)
    for r in reqs:
        srv.submit(r["a"], r["b"], r["n"], r["omega"], nrhs=r["nrhs"], bc=r["bc"], rtol=1e-6)
    assert srv.wait_all(300)
    assert srv.stats()["peak_running"] == 1
    srv.close()


def test_bad_requests_are_refused():
    from paper_1408_1578_gb300 import cfie
    srv = cfie.Server(0, hbm_budget_bytes=1 << 30, slots=1)
    with pytest.raises(cfie.CfieError):
        srv.submit([0.1], [0.0], 1001, 10.0)             # odd n
    with pytest.raises(cfie.CfieError):
        srv.submit([0.1], [0.0], 1000, -1.0)             # omega <= 0
    with pytest.raises(cfie.CfieError):
        srv.submit([0.1], [0.0], 1000, 10.0, bc="hard", precision="tensor")   # stored: soft only
    srv.close()


def test_failed_request_reports_its_error():
    """A request the FP32 form refuses (omega so low that every pair is in the
    near band) finishes with that status and its message, not a crash."""
    from paper_1408_1578_gb300 import cfie
    srv = cfie.Server(0, hbm_budget_bytes=8 << 30, slots=1)
    t = srv.submit([0.1], [0.0], 65536, 0.01)
    assert srv.wait_all(300)
    out = srv.poll(t)
    assert out["done"] and out["status"] == cfie.CFIE_EINVAL
    assert "band" in out["error"]
    srv.release(t)
    srv.close()


def test_batched_slots_equal_alone_and_oracle():
    """With batching on, a slot takes several compatible queued requests and
    solves them as one lockstep batch; each request's result equals its solve
    alone and the oracle's LU solution (<= 1e-6), and its own residual meets
    rtol.  Sizes within a factor of two (so that they group), hard and soft
    mixed, ragged directions."""
    from paper_1408_1578_gb300 import cfie
    reqs = inputs.poisson_requests(count=10, rate=200.0, seed=91, n_lo=1000, n_hi=1900)
    for k, r in enumerate(reqs):
        r["nrhs"] = 1 + (k * 7) % 9
    srv = cfie.Server(0, hbm_budget_bytes=48 << 30, slots=2, batch=6)
    tickets = [srv.submit(r["a"], r["b"], r["n"], r["omega"], nrhs=r["nrhs"], bc=r["bc"],
                          rtol=1e-8, restart=60) for r in reqs]
    assert srv.wait_all(300)
    stats = srv.stats()
    assert stats["completed"] == len(reqs)
    outs = [srv.poll(t, want_x=True) for t in tickets]
    ctx = cfie.Context(0)
    for r, t, out in zip(reqs, tickets, outs):
        assert out["done"] and out["status"] == cfie.CFIE_OK, out.get("error")
        assert out["relres_max"] <= 1e-8
        op = ctx.fourier_star(r["a"], r["b"]).discretise(r["n"], r["omega"], bc=r["bc"],
                                                          precision="fp32")
        f = zeros(r["nrhs"], r["n"])
        op.rhs_plane_waves(inputs.directions(r["nrhs"]), f)
        x = zeros(r["nrhs"], r["n"])
        op.gmres_solve(f, x, rtol=1e-8, restart=60, maxit=4000)
        assert np.max(col_rel(out["x"], to_host(x))) < TOL_REFINED
        c = geometry.fourier_star(r["n"], r["a"], r["b"])
        A = operators.cfie_matrix(c, r["omega"], r["omega"], r["bc"])
        Q = solvers.lu_solve(A, to_host(f).T).T
        assert np.max(col_rel(out["x"], Q)) < TOL_REFINED
        op.close()
        srv.release(t)
    ctx.close()
    srv.close()
    assert stats["peak_running"] >= 3          # a slot ran several requests at once


def test_batching_setting_is_checked():
    from paper_1408_1578_gb300 import cfie
    srv = cfie.Server(0, hbm_budget_bytes=1 << 30, slots=1)
    for bad in (0, 257, -1):
        with pytest.raises(cfie.CfieError):
            srv.set_batching(bad)
    srv.set_batching(256)
    srv.close()


def test_batched_stored_form_equals_alone_and_oracle():
    """Sound-soft requests in the stored tensor-core form, batched by a slot
    (one persistent contraction launch per matvec for the group): each result
    equals the same request's solve alone and the oracle's LU solution
    (<= 1e-6).  The stored form refuses sound-hard requests."""
    from paper_1408_1578_gb300 import cfie
    reqs = inputs.poisson_requests(count=7, rate=200.0, seed=93, n_lo=700, n_hi=1300)
    for k, r in enumerate(reqs):
        r["nrhs"] = 1 + (k * 11) % 40
        r["bc"] = "soft"
    srv = cfie.Server(0, hbm_budget_bytes=48 << 30, slots=1, batch=8)
    with pytest.raises(cfie.CfieError):
        srv.submit(reqs[0]["a"], reqs[0]["b"], 800, 10.0, bc="hard", precision="tensor")
    tickets = [srv.submit(r["a"], r["b"], r["n"], r["omega"], nrhs=r["nrhs"], bc="soft",
                          rtol=1e-8, restart=60, precision="tensor") for r in reqs]
    assert srv.wait_all(300)
    assert srv.stats()["peak_running"] >= 3
    ctx = cfie.Context(0)
    for r, t in zip(reqs, tickets):
        out = srv.poll(t, want_x=True)
        assert out["done"] and out["status"] == cfie.CFIE_OK, out.get("error")
        assert out["relres_max"] <= 1e-8
        op = ctx.fourier_star(r["a"], r["b"]).discretise(r["n"], r["omega"], precision="tensor",
                                                          layout="stored")
        f = zeros(r["nrhs"], r["n"])
        op.rhs_plane_waves(inputs.directions(r["nrhs"]), f)
        x = zeros(r["nrhs"], r["n"])
        op.gmres_solve(f, x, rtol=1e-8, restart=60, maxit=4000)
        assert np.max(col_rel(out["x"], to_host(x))) < TOL_REFINED
        c = geometry.fourier_star(r["n"], r["a"], r["b"])
        A = operators.cfie_matrix(c, r["omega"], r["omega"], "soft")
        Q = solvers.lu_solve(A, to_host(f).T).T
        assert np.max(col_rel(out["x"], Q)) < TOL_REFINED
        op.close()
        srv.release(t)
    ctx.close()
    srv.close()


def test_block_gmres_requests_equal_alone_and_oracle():
    """Requests with at least block_min_rhs directions run alone with block
    GMRES over their directions; the others still batch.  Every result equals
    the per-direction solve alone and the oracle's LU solution (<= 1e-6)."""
    from paper_1408_1578_gb300 import cfie
    reqs = inputs.poisson_requests(count=5, rate=200.0, seed=95, n_lo=800, n_hi=1500)
    for k, r in enumerate(reqs):
        r["nrhs"] = (12, 2, 9, 1, 16)[k]
    srv = cfie.Server(0, hbm_budget_bytes=48 << 30, slots=2, batch=4, block_min_rhs=8)
    tickets = [srv.submit(r["a"], r["b"], r["n"], r["omega"], nrhs=r["nrhs"], bc=r["bc"],
                          rtol=1e-8, restart=60) for r in reqs]
    assert srv.wait_all(300)
    ctx = cfie.Context(0)
    for r, t in zip(reqs, tickets):
        out = srv.poll(t, want_x=True)
        assert out["done"] and out["status"] == cfie.CFIE_OK, out.get("error")
        assert out["relres_max"] <= 1e-8
        op = ctx.fourier_star(r["a"], r["b"]).discretise(r["n"], r["omega"], bc=r["bc"],
                                                          precision="fp32")
        f = zeros(r["nrhs"], r["n"])
        op.rhs_plane_waves(inputs.directions(r["nrhs"]), f)
        x = zeros(r["nrhs"], r["n"])
        its, _, _ = op.gmres_solve(f, x, rtol=1e-8, restart=60, maxit=4000)
        assert np.max(col_rel(out["x"], to_host(x))) < TOL_REFINED
        if r["nrhs"] >= 8:                 # block steps: fewer than the per-direction steps
            assert out["iters_max"] < int(np.max(its))
        c = geometry.fourier_star(r["n"], r["a"], r["b"])
        A = operators.cfie_matrix(c, r["omega"], r["omega"], r["bc"])
        Q = solvers.lu_solve(A, to_host(f).T).T
        assert np.max(col_rel(out["x"], Q)) < TOL_REFINED
        op.close()
        srv.release(t)
    with pytest.raises(cfie.CfieError):
        srv.set_block_gmres(-1)
    with pytest.raises(cfie.CfieError):
        srv.set_block_gmres(8, -1)
    ctx.close()
    srv.close()


def test_batched_fp64_requests_equal_alone_and_oracle():
    """The plain FP64 form batches too (lockstep FP64 GMRES over the group):
    each request's solution equals its FP64 solve alone and the oracle's LU
    solution within 1e-8 (both driven to residual 1e-10)."""
    from paper_1408_1578_gb300 import cfie
    reqs = inputs.poisson_requests(count=4, rate=200.0, seed=97, n_lo=500, n_hi=900)
    for k, r in enumerate(reqs):
        r["nrhs"] = 1 + 2 * k
    srv = cfie.Server(0, hbm_budget_bytes=16 << 30, slots=1, batch=4)
    tickets = [srv.submit(r["a"], r["b"], r["n"], r["omega"], nrhs=r["nrhs"], bc=r["bc"],
                          rtol=1e-10, restart=60, precision="fp64") for r in reqs]
    assert srv.wait_all(300)
    ctx = cfie.Context(0)
    for r, t in zip(reqs, tickets):
        out = srv.poll(t, want_x=True)
        assert out["done"] and out["status"] == cfie.CFIE_OK, out.get("error")
        assert out["relres_max"] <= 1e-10
        op = ctx.fourier_star(r["a"], r["b"]).discretise(r["n"], r["omega"], bc=r["bc"],
                                                          precision="fp64")
        f = zeros(r["nrhs"], r["n"])
        op.rhs_plane_waves(inputs.directions(r["nrhs"]), f)
        x = zeros(r["nrhs"], r["n"])
        op.gmres_solve(f, x, rtol=1e-10, restart=60, maxit=4000)
        assert np.max(col_rel(out["x"], to_host(x))) < 1e-8
        c = geometry.fourier_star(r["n"], r["a"], r["b"])
        A = operators.cfie_matrix(c, r["omega"], r["omega"], r["bc"])
        Q = solvers.lu_solve(A, to_host(f).T).T
        assert np.max(col_rel(out["x"], Q)) < 1e-8
        op.close()
        srv.release(t)
    ctx.close()
    srv.close()
