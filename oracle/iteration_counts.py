"""The paper's GMRES iteration counts on its ellipse (Section 3, Tables 1 and 3),
recomputed with the oracle (test infrastructure only; no GPU).

Setting of Section 3: ellipse with semi-axes (1, 0.5) (inferred from the
omega / n pairs of Table 1), p = 8 points per wavelength equispaced in
arclength, n = 4^q p, omega = 2 pi (n / p) / L, one plane wave towards +x,
GMRES with relative tolerance 1e-6, restart 80, zero initial guess; n_n without
and n_p with the directional preconditioner of Section 2 (applied on the
right).  The coupling is eta = f omega (Section 1 fixes only eta = O(omega)).

    python -m oracle.iteration_counts --q 3 4 5 --bc soft hard --eta-factor 0.5 1

The dense matrix is assembled in row blocks by a pool of worker processes
(16 n^2 bytes: 17 GB at q = 6, the paper's n = 32768; the sound-hard matrix
needs several such arrays while it is built, so q = 6 is practical for the
sound-soft operator only on a 64 GB host).
"""
import argparse
import multiprocessing as mp
import os
import time

import numpy as np

from . import directional, geometry, operators
from .kress import kress_weights

_W = {}


def _setup(a, b, q, p, eta_factor):
    arc = geometry.Arclength("ellipse", a=a, b=b)
    n = 4**q * p
    omega = 2.0 * np.pi * (n / p) / arc.L
    return arc, n, omega, eta_factor * omega


def _init(a, b, q, p, eta_factor):
    arc, n, omega, eta = _setup(a, b, q, p, eta_factor)
    _W.update(curve=arc.curve(n), n=n, omega=omega, eta=eta, R=kress_weights(n))


def _soft_rows(start):
    n = _W["n"]
    rows = np.arange(start, min(n, start + 128))
    return start, operators.soft_rows(_W["curve"], _W["omega"], _W["eta"], rows, _W["R"])


def soft_matrix_parallel(q, p=8, eta_factor=1.0, a=1.0, b=0.5, workers=None):
    """The sound-soft CFIE matrix of eq. 1 on the arclength-sampled ellipse,
    row blocks computed by `workers` processes (spawned: a calling script must
    keep its own work under `if __name__ == "__main__":`, since each worker
    imports it)."""
    _, n, _, _ = _setup(a, b, q, p, eta_factor)
    workers = workers or os.cpu_count() or 1
    A = np.empty((n, n), dtype=np.complex128)
    with mp.get_context("spawn").Pool(workers, initializer=_init,
                                      initargs=(a, b, q, p, eta_factor)) as pool:
        for start, blk in pool.imap_unordered(_soft_rows, range(0, n, 128)):
            A[start:start + blk.shape[0]] = blk
    return A


def counts(q, bc="soft", eta_factor=1.0, p=8, a=1.0, b=0.5, workers=None):
    """(n, omega, n_n, n_p) for one row of Tables 1 / 3."""
    arc, n, omega, eta = _setup(a, b, q, p, eta_factor)
    c = arc.curve(n)
    if bc == "soft":
        A = soft_matrix_parallel(q, p, eta_factor, a, b, workers) if q >= 5 else \
            operators.soft_matrix(c, omega, eta)
    else:
        A = operators.hard_matrix(c, omega, eta)
    f = operators.plane_wave_rhs(c, omega, [0.0], bc)[:, 0]
    _, n_n, _ = directional.preconditioned_gmres(A, None, f, rtol=1e-6, restart=80)
    P = directional.Directional(arc, q, p, omega, eta=eta, bc=bc, A=A if bc == "hard" else None)
    _, n_p, _ = directional.preconditioned_gmres(A, P.apply, f, rtol=1e-6, restart=80)
    return n, omega, n_n, n_p


def main():
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--q", type=int, nargs="+", default=[3, 4])
    ap.add_argument("--bc", nargs="+", default=["soft"], choices=["soft", "hard"])
    ap.add_argument("--eta-factor", type=float, nargs="+", default=[0.5])
    ap.add_argument("--workers", type=int, default=None)
    args = ap.parse_args()
    print("bc    eta/omega      n    omega   n_n  n_p  seconds")
    for bc in args.bc:
        for fac in args.eta_factor:
            for q in args.q:
                t0 = time.time()
                n, omega, n_n, n_p = counts(q, bc, fac, workers=args.workers)
                print(f"{bc:5s} {fac:9.2f} {n:6d} {omega:8.1f} {n_n:5d} {n_p:4d} "
                      f"{time.time() - t0:8.0f}", flush=True)


if __name__ == "__main__":
    main()
