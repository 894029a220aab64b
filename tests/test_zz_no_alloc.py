"""cfie_apply_fp64_static: the FP64 matvec for callers that cannot allocate
device memory (a process that gave its free HBM to its own pool, or a loop
that must not pay the implicit synchronisation of cudaMalloc / cudaFree).

Its scratch is a fixed 32 MiB device array inside the library.  The test calls
the entry point through the C ABI twice in a row on each operator and compares
every result with the regular cfie_apply_fp64, within the FP64 tolerance of
the other parity tests (1e-12 relative per right-hand side).  It checks that
device free memory does not move across the calls and that a request larger
than the array is refused with CFIE_EINVAL.  The file is named to be collected
last, so a run that stops at the first failure has already run the rest."""
import numpy as np
import pytest

from paper_1408_1578_gb300 import inputs
from tests.gpu_util import col_rel, empty, to_dev, to_host

pytestmark = pytest.mark.gpu

TOL_FP64 = 1e-12


@pytest.fixture(scope="module")
def ctx():
    from paper_1408_1578_gb300 import cfie
    c = cfie.Context(0)
    yield c
    c.close()


def _static_apply(ctx, op, x, y, nrhs):
    return ctx.lib.cfie_apply_fp64_static(op.h, x.data_ptr(), y.data_ptr(), nrhs)


@pytest.mark.parametrize("kind,params,n,omega,bc,nrhs", [
    ("kite", {}, 1000, 40.0, "soft", 5),
    ("star", {"a": [0, 0, 0, 0, 0.3], "b": [0] * 5}, 4096, 256.0, "hard", 16),
    ("ellipse", {"a": 1.0, "b": 0.5}, 514, 25.0, "hard", 3),
    # 16 n nrhs just under the 32 MiB cap: the array holds a single split of
    # the sources, while the regular matvec splits them and takes its 64-wide
    # right-hand-side tile
    ("kite", {}, 8192, 512.0, "soft", 255),
])
def test_static_scratch_matches_regular_fp64(ctx, kind, params, n, omega, bc, nrhs):
    import torch
    from paper_1408_1578_gb300 import cfie
    op = ctx.geometry(kind, **params).discretise(n, omega, bc=bc, precision="fp64")
    xs = [to_dev(inputs.random_density(n, nrhs, seed=s)) for s in (101, 202)]
    refs = []
    for x in xs:
        y = empty(nrhs, n)
        op.apply_fp64(x, y)
        refs.append(to_host(y))
    torch.cuda.synchronize()
    outs = [empty(nrhs, n) for _ in xs]
    # first call on this device looks up the array's address; then two calls in a row
    warm = empty(nrhs, n)
    assert _static_apply(ctx, op, xs[0], warm, nrhs) == cfie.CFIE_OK, ctx.last_error()
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for x, y in zip(xs, outs):
        st = _static_apply(ctx, op, x, y, nrhs)
        assert st == cfie.CFIE_OK, ctx.last_error()
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    for y, ref in zip(outs, refs):
        assert np.max(col_rel(to_host(y), ref)) < TOL_FP64
    op.close()


def test_static_scratch_rejects_oversized_requests(ctx):
    from paper_1408_1578_gb300 import cfie
    n, nrhs = 32768, 65            # 16 * n * nrhs bytes > 32 MiB
    op = ctx.kite().discretise(n, 2048.0, precision="fp64")
    x = empty(nrhs, n)
    y = empty(nrhs, n)
    st = _static_apply(ctx, op, x, y, nrhs)
    assert st == cfie.CFIE_EINVAL
    assert "32 MiB" in ctx.last_error()
    op.close()
