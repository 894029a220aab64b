"""FP64 CPU oracle for the combined-field integral equation (CFIE) hot path.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or link
this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.  It shares
no code with the CUDA library: it has its own curve formulas, its own Kress
weights, its own operator assembly (Bessel values from ``scipy.special``), its
own GMRES and a direct LU solve (``numpy.linalg.solve``).

What it computes (paper: Ying, "Directional preconditioner for high frequency
obstacle scattering", Section 1):

* the sound-soft CFIE ``(1/2 I + D - i eta S) q = -u_I``          (eq. 1 / dis1)
* the sound-hard CFIE ``(1/2 I - D' + N/(i eta)) q = -du_I/dn``   (eq. 2)
  with ``G(x, y) = (i/4) H0^(1)(omega |x - y|)`` and the operators S, D, D', N
  of Section 1.

The paper names the Nystrom method but not its quadrature; the oracle uses
Kress's logarithmic-split trapezoidal rule on smooth 2*pi-periodic
parametrisations (Colton & Kress, Inverse Acoustic and Electromagnetic
Scattering Theory, Section 3.5) and Maue's identity for the hypersingular N.
Every function names the passage it follows.

Parity status: every function here is pinned by ``tests/test_oracle_*.py``
against closed forms (disk eigenvalues, Fourier-Bessel series, interior point
source identity, trigonometric exactness, Wronskian, brute force).

Modules
-------
geometry   curve samples z, z', z'' at the nodes t_j = 2 pi j / n
kress      the Kress log-split weights R_d
operators  Bessel values, S / D / D' / N Nystrom matrices, CFIE matrices,
           row-sampled operators, spectral derivative, plane-wave data
solvers    LU solve, restarted GMRES (modified Gram-Schmidt, Givens) and block
           GMRES over all right-hand sides (one shared Krylov space)
field      off-surface representation formulas for the scattered field
directional  the directional preconditioner of Section 2 (sound soft and sound
           hard): segment partition, flat diagonal blocks B, partial Fourier
           matrices U, the sparse E of rank-1 block coefficients, eq. (eapp);
           with the arclength sampling it needs (geometry.Arclength).  Its
           algebra (eq. aug / fac / esol), entry function, interpolation,
           arclength map and sound-soft flat blocks are pinned by
           tests/test_oracle_directional.py; the quality of the data-sparse
           approximation is checked through its effect on GMRES iteration
           counts (Tables 1 and 3 give no entries).
iteration_counts  the GMRES iteration counts of Tables 1 and 3 (n_n without,
           n_p with the preconditioner) on the paper's ellipse, recomputed
           (python -m oracle.iteration_counts).
"""
