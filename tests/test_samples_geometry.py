"""GPU parity of operators built from caller samples (cfie_geometry_samples),
through the C ABI.

* Closed-form samples of the ellipse (a cos t, b sin t) at t_j = 2 pi j / n,
  written out here, against the oracle's ellipse: the same operator as the
  library's own ellipse, so FP64 <= 1e-12 and FP32 <= 1e-4.
* The node set of Section 2, end to end: the library's arclength samples
  (cfie_arclength_samples) discretised on the GPU, against the oracle's own
  arclength samples (geometry.Arclength) discretised by the oracle.  The two
  sample sets agree to ~1e-12 (checked on the CPU), hence FP64 <= 1e-11."""
import numpy as np
import pytest

from oracle import geometry, operators
from paper_1408_1578_gb300 import cfie, inputs
from tests.gpu_util import col_rel, empty, to_dev, to_host

pytestmark = pytest.mark.gpu

N, OMEGA, NRHS = 1000, 90.0, 5


@pytest.fixture(scope="module")
def ctx():
    c = cfie.Context(0)
    yield c
    c.close()


def _ellipse_samples(n, a, b):
    t = 2 * np.pi * np.arange(n) / n
    c, s = np.cos(t), np.sin(t)
    return (np.stack([a * c, b * s], 1), np.stack([-a * s, b * c], 1),
            np.stack([-a * c, -b * s], 1))


@pytest.mark.parametrize("bc", ["soft", "hard"])
def test_closed_form_samples(ctx, bc):
    A = operators.cfie_matrix(geometry.ellipse(N, 1.0, 0.5), OMEGA, OMEGA, bc)
    X = inputs.random_density(N, NRHS, seed=61)
    want = (A @ X.T).T
    g = ctx.samples(*_ellipse_samples(N, 1.0, 0.5))
    for prec, tol in (("fp64", 1e-12), ("fp32", 1e-4)):
        op = g.discretise(N, OMEGA, bc=bc, precision=prec)
        y = empty(NRHS, N)
        op.apply(to_dev(X), y)
        assert np.max(col_rel(to_host(y), want)) < tol, prec


@pytest.mark.parametrize("bc", ["soft", "hard"])
def test_arclength_nodes_end_to_end(ctx, bc):
    c = geometry.Arclength("ellipse", a=1.0, b=0.5).curve(N)
    A = operators.cfie_matrix(c, OMEGA, OMEGA, bc)
    X = inputs.random_density(N, NRHS, seed=62)
    z, dz, ddz, _ = cfie.arclength_samples("ellipse", N, a=1.0, b=0.5)
    op = ctx.samples(z, dz, ddz).discretise(N, OMEGA, bc=bc, precision="fp64")
    y = empty(NRHS, N)
    op.apply(to_dev(X), y)
    assert np.max(col_rel(to_host(y), (A @ X.T).T)) < 1e-11


def test_sample_count_must_match(ctx):
    g = ctx.samples(*_ellipse_samples(64, 1.0, 0.5))
    with pytest.raises(cfie.CfieError):
        g.discretise(128, 4.0)
