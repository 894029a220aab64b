"""Failure detection without faulting the GPU: a bounded device wait that runs
out returns CFIE_ETIMEOUT and leaves the context usable; GMRES that misses its
tolerance returns CFIE_ENOCONV with the last iterate; bad arguments are refused
before any device work."""
import os

import numpy as np
import pytest

from paper_1408_1578_gb300 import inputs
from tests.gpu_util import col_rel, empty, to_dev, to_host, zeros

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_1408_1578_gb300 import cfie
    c = cfie.Context(0)
    yield c
    c.close()


def test_tensor_core_wait_timeout_is_reported_and_recoverable(ctx, monkeypatch):
    from paper_1408_1578_gb300 import cfie
    n, w = 512, 40.0
    X = to_dev(inputs.random_density(n, 4, seed=1))
    monkeypatch.setenv("CFIE_FAULT_INJECT", "tma_stall")
    op = ctx.kite().discretise(n, w, precision="tensor", layout="stored")
    y = empty(4, n)
    with pytest.raises(cfie.CfieError) as e:
        op.apply(X, y)
    assert e.value.status == cfie.CFIE_ETIMEOUT
    op.close()
    monkeypatch.delenv("CFIE_FAULT_INJECT")
    # the context and the device stay usable
    op2 = ctx.kite().discretise(n, w, precision="tensor", layout="stored")
    y2 = empty(4, n)
    op2.apply(X, y2)
    ref = empty(4, n)
    ctx.kite().discretise(n, w, precision="fp64").apply_fp64(X, ref)
    assert np.max(col_rel(to_host(y2), to_host(ref))) < 1e-4


def test_gmres_reports_no_convergence_with_last_iterate(ctx):
    from paper_1408_1578_gb300 import cfie
    n, w = 800, 60.0
    op = ctx.kite().discretise(n, w, precision="fp64")
    f = empty(2, n)
    op.rhs_plane_waves([0.0, 1.0], f)
    x = zeros(2, n)
    its, rel, st = op.gmres_solve(f, x, rtol=1e-12, restart=5, maxit=7, allow_noconv=True)
    assert st == cfie.CFIE_ENOCONV
    assert np.all(its == 7) and np.all(rel > 1e-12) and np.all(rel < 1.0)
    assert np.linalg.norm(to_host(x)) > 0
