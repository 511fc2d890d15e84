"""CPU FP64 oracle for the FEM-NFFT fast summation (test infrastructure only).

This package is the plain, slow reference the CUDA library is checked against.
Only the tests, the smoke check of ``__graft_entry__`` and the CPU-baseline leg
of ``bench.py`` may import it; the library itself never does, and it shares
no code, tables or constants with the CUDA path.

Contents, each following the paper (Kritsikis, Toussaint, Fruchart, "Fast
computation of magnetostatic fields by Non-uniform Fast Fourier Transforms"):

* ``kernel``  the log Green function G of Eq. (1), its regularisation near the
  origin (the smoothing step of the NFFT paragraph) and at the torus boundary,
  the Fourier coefficients b_l of the regularised kernel, and the
  Kaiser-Bessel window pair used to spread ("diffuse") the charges.
* ``direct``  O1: the plain O(N M) sum of Eq. (2) ("FEM-direct") and its
  gradient, in C with OpenMP (``direct.c``), plus the Hessian used by the
  adjoint.
* ``fastsum`` O2 (exact trigonometric sums over the frequency set, i.e. the
  NDFT) and O3 (the spread / FFT / divide / inverse steps of the NFFT
  paragraph as plain numpy loops over taps), both followed by the near-field
  correction and the rescale to physical units.
* ``fem``     P1 charge assembly of Eq. (2): rho = -div M at triangle
  quadrature points and sigma = M.n at boundary-edge Gauss points.
* ``fastsum3`` the paper's stated next step, the 3D kernel G = 1/(4 pi r):
  O1 direct sum, O2 and O3 fast sums and the near field with the same
  regularisation and window steps in three dimensions.
* ``fem3``    the 3D charge assembly: P1 tetrahedra (rho = -div M, 4 points
  each) and boundary triangles (sigma = M.n, 3 points each).

Readings of points the paper leaves open are listed in the repository's
design notes; each function's docstring states the one it uses.
"""
