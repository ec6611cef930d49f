"""Reference oracle for the batched Shen wall-normal solves (test infrastructure only).

This package is NOT part of the product.  Only ``tests/``, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it.
The CUDA path never calls into it and it never calls into the CUDA path; the two
share no code, tables, constants or helpers.

What it computes, from Mortensen, "A spectral-Galerkin turbulent channel flow solver
for large-scale simulations" (arXiv:1701.03787):

* ``chebyshev``  exact Chebyshev-coefficient algebra for the bases of Sec. 2
  (Eqs. Tk, phiD, phiN) and the Chebyshev-Gauss weighted scalar product
  (Eq. quadrature with the GC weights of Sec. 2).
* ``matrices``   dense Galerkin matrices B, A, Q of Sec. 3 (Table tab:matrices,
  Eqs. N_Q, pk, rk), assembled from exact inner products and rounded once to
  float64, plus the Helmholtz / biharmonic systems (Eqs. Biharmonic_matrix,
  Helmholtz_matrix) and the right-hand-side operators of Eqs. ufin / gfin.
* ``solve``      the definition of every solve: dense LU with partial pivoting
  (LAPACK) on those matrices, a 50-digit mpmath brute force for small N, the
  Fourier mode layout (Sec. 2, wavenumber mesh K^p) and the error metrics.
* ``shen_on.c``  the paper's O(N) algorithms written plainly in C (Sec. 4: the
  odd/even Helmholtz LU, Algorithms LUbiharmonic, ReduceAB, LUSolveBiharmonic),
  pinned against the dense definition; also timed as the CPU baseline.

All floating point is IEEE float64 unless a function says otherwise.
"""
