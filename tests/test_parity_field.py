"""GPU parity of the off-surface field evaluation (cfie_field_eval) against the
oracle's trapezoidal layer potentials, and end to end (GPU solve, GPU field)
against closed forms: the Fourier-Bessel series for the disk and the field of
an interior point source."""
import numpy as np
import pytest
import torch

from oracle import field, geometry, operators
from paper_1408_1578_gb300 import inputs
from tests import closed_forms as cf
from tests.gpu_util import to_dev, to_host, zeros

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_1408_1578_gb300 import cfie
    c = cfie.Context(0)
    yield c
    c.close()


def _pts(p):
    """(m, 2) points as the complex128 device vector x + i y."""
    p = np.asarray(p, dtype=np.float64)
    return torch.from_numpy(np.ascontiguousarray(p[:, 0] + 1j * p[:, 1])).cuda()


@pytest.mark.parametrize("bc", ["soft", "hard"])
@pytest.mark.parametrize("npts,nrhs", [(1, 1), (100, 9), (64, 8), (257, 17)])
def test_field_matches_oracle_elementwise(ctx, bc, npts, nrhs):
    n, w = 600, 30.0                                   # ragged over the 128-source tiles
    c = geometry.kite(n)
    rng = np.random.default_rng(npts + nrhs)
    q = inputs.random_density(n, nrhs, seed=npts)
    ang = rng.uniform(0, 2 * np.pi, npts)
    rad = rng.uniform(2.2, 4.0, npts)                  # outside the kite (|z| < 2)
    pts = np.stack([rad * np.cos(ang), rad * np.sin(ang)], axis=1)
    op = ctx.kite().discretise(n, w, bc=bc, precision="fp64")
    u = zeros(nrhs, npts)
    op.field_eval(to_dev(q), _pts(pts), u)
    want = np.stack([field.scattered_field(c, w, w, bc, q[k], pts) for k in range(nrhs)])
    got = to_host(u)
    assert np.max(np.abs(got - want)) <= 1e-12 * np.max(np.abs(want))


@pytest.mark.parametrize("bc", ["soft", "hard"])
def test_disk_series_end_to_end(ctx, bc):
    """Unit circle, omega = 64, n = 1024, d = (1, 0); the GPU
    solution's field at r = 2 against the Fourier-Bessel series."""
    n, w = 1024, 64.0
    op = ctx.circle().discretise(n, w, bc=bc, precision="fp64")
    f = zeros(1, n)
    op.rhs_plane_waves([0.0], f)
    q = zeros(1, n)
    its, rel, _ = op.gmres_solve(f, q, rtol=1e-13, restart=0, maxit=500)
    pts = cf.ring(2.0, 24)
    u = zeros(1, len(pts))
    op.field_eval(q, _pts(pts), u)
    assert cf.rel(to_host(u)[0], cf.disk_scattered(w, 0.0, pts, bc)) < 1e-10


@pytest.mark.parametrize("bc", ["soft", "hard"])
def test_point_source_refined_end_to_end(ctx, bc):
    """Star r = 1 + 0.3 cos 5t at omega = 64: boundary data -G(., x0) with x0
    inside, FP32-refined GPU solve, GPU field on the radius-3 circle = -G."""
    n, w = 1024, 64.0
    x0 = np.array([0.1, 0.05])
    params = {"a": [0, 0, 0, 0, 0.3], "b": [0] * 5}
    c = geometry.fourier_star(n, params["a"], params["b"])
    F = operators.point_source_rhs(c, w, x0, bc)
    op = ctx.fourier_star(params["a"], params["b"]).discretise(n, w, bc=bc, precision="fp32")
    q = zeros(1, n)
    its, rel, _ = op.gmres_solve(to_dev(F.T), q, rtol=1e-10, restart=80, maxit=2000)
    pts = cf.ring(3.0, 32)
    u = zeros(1, len(pts))
    op.field_eval(q, _pts(pts), u)
    assert cf.rel(to_host(u)[0], -cf.green(w, pts, x0)) < 1e-7


def test_field_arguments(ctx):
    from paper_1408_1578_gb300 import cfie
    op = ctx.kite().discretise(64, 4.0, precision="fp64")
    q = zeros(1, 64)
    u = zeros(1, 4)
    pts = _pts(np.full((4, 2), 3.0))
    lib = ctx.lib
    from paper_1408_1578_gb300.cfie import _addr
    assert lib.cfie_field_eval(op.h, _addr(q), 1, 0, _addr(pts), _addr(u)) == cfie.CFIE_EINVAL
    assert lib.cfie_field_eval(op.h, None, 1, 4, _addr(pts), _addr(u)) == cfie.CFIE_EINVAL
    assert lib.cfie_field_eval(op.h, _addr(q), 0, 4, _addr(pts), _addr(u)) == cfie.CFIE_EINVAL
    assert lib.cfie_field_eval(op.h, _addr(q), 1, 4, _addr(pts), _addr(q)) == cfie.CFIE_EINVAL
