"""Run one small, fixed case of one kernel path through the public API, for
profilers (ncu) and quick timing.  Prints the per-class kernel times.

    python -m paper_1408_1578_gb300.profile_case --path fused    [--n 8192] [--nrhs 64]
    python -m paper_1408_1578_gb300.profile_case --path residual [--n 8192] [--nrhs 64] [--variant 1|2]
    python -m paper_1408_1578_gb300.profile_case --path fp64     [--n 4096] [--nrhs 16] [--bc hard]
    python -m paper_1408_1578_gb300.profile_case --path stored   [--n 8192] [--nrhs 32]
    python -m paper_1408_1578_gb300.profile_case --path batch    [--count 16]
    python -m paper_1408_1578_gb300.profile_case --path solve    [--n 8192] [--nrhs 64]

Curves are the kite (fused, residual, stored, solve) and the five-lobed star
r = 1 + 0.3 cos 5t (fp64), with omega = n / 16 (the kite workload's ratio,
about 10 points per wavelength); batches are the seeded random stars of the
batched workload; inputs are seeded random densities.
"""
import argparse
import json

import numpy as np
import torch

from . import cfie, inputs


def main():
    p = argparse.ArgumentParser()
    p.add_argument("--path", required=True,
                   choices=["fused", "residual", "fp64", "stored", "batch", "solve"])
    p.add_argument("--n", type=int, default=8192)
    p.add_argument("--nrhs", type=int, default=None)
    p.add_argument("--bc", default="soft", choices=["soft", "hard"])
    p.add_argument("--variant", type=int, default=0,
                   help="fused: summation variant (0 autotuned, 1, 2); residual: 1 CUDA-core "
                        "Dot2 sums, 2 sliced tensor-core sums (0 automatic)")
    p.add_argument("--count", type=int, default=16, help="batch: operators")
    p.add_argument("--repeat", type=int, default=5)
    a = p.parse_args()

    ctx = cfie.Context(0)
    n = a.n
    w = n / 16.0
    out = {"path": a.path, "n": n}
    if a.path == "batch":
        specs = inputs.random_stars(count=a.count, seed=1408, n_lo=512, n_hi=16384, nrhs=32)
        ops = [ctx.fourier_star(s["a"], s["b"]).discretise(s["n"], s["omega"], precision="tensor",
                                                            layout="stored") for s in specs]
        b = cfie.Batch(ctx, ops, [s["nrhs"] for s in specs])
        L = b.length
        rng = np.random.default_rng(3)
        x = torch.from_numpy(rng.standard_normal(L) + 1j * rng.standard_normal(L)).cuda()
        y = torch.empty_like(x)
        b.apply(x, y)
        torch.cuda.synchronize()
        ctx.set_profiling(True)
        for _ in range(a.repeat):
            b.apply(x, y)
        out.update(count=a.count, sum_n2=sum(s["n"] ** 2 for s in specs))
    else:
        nrhs = a.nrhs or {"fused": 64, "residual": 64, "fp64": 16, "stored": 32, "solve": 64}[a.path]
        if a.path == "fp64":
            geom = ctx.fourier_star([0, 0, 0, 0, 0.3], [0, 0, 0, 0, 0])
        else:
            geom = ctx.kite()
        prec = {"fused": "fp32", "residual": "fp32", "fp64": "fp64", "stored": "tensor",
                "solve": "fp32"}[a.path]
        op = geom.discretise(n, w, bc=a.bc, precision=prec,
                             layout="stored" if prec == "tensor" else "matrix_free")
        if a.variant and a.path == "fused":
            op.set_variant(a.variant)
        if a.variant and a.path == "residual":
            op.set_residual_variant(a.variant)
        X = torch.from_numpy(inputs.random_density(n, nrhs, seed=1)).cuda()
        Y = torch.empty_like(X)
        if a.path == "solve":
            f = torch.empty_like(X)
            op.rhs_plane_waves(inputs.directions(nrhs), f)
            x = torch.zeros_like(X)
            ctx.set_profiling(True)
            its, rel, _ = op.gmres_solve(f, x, rtol=1e-8, restart=80, maxit=4000)
            out.update(iterations=int(its.max()), relres=float(rel.max()), stats=op.last_stats())
        else:
            run = {"fused": op.apply, "residual": op.apply_residual, "fp64": op.apply_fp64,
                   "stored": op.apply}[a.path]
            run(X, Y)
            torch.cuda.synchronize()
            ctx.set_profiling(True)
            for _ in range(a.repeat):
                run(X, Y)
        out.update(nrhs=nrhs, omega=w, bc=a.bc)
    torch.cuda.synchronize()
    out["kernel_ms"] = {k: [round(v[0], 4), v[1]] for k, v in ctx.kernel_times().items()}
    ctx.set_profiling(False)
    print(json.dumps(out))
    ctx.close()


if __name__ == "__main__":
    main()
