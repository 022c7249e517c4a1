"""CPU FP64 oracle for the integral-equation (IE) forward model with domain decomposition.

TEST INFRASTRUCTURE ONLY. Only the test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may import this package. The library itself (the CUDA path behind the C ABI)
never calls it, and this package never imports the library: the two share no code. The only
module both sides use is the seeded input generator ``paper_2306_17537_gb300.inputs``, which
holds none of the method's arithmetic.

Everything here is plain, slow and written for checking by eye against the paper
(Saputera et al., "3D induction log modelling with integral equation method and domain
decomposition preconditioning"):

  physics.py   Section 2.1, eqs. 1-7: k0, scalar Green's function, electric Green's dyadic,
               equal-volume-sphere self term (Section 2.2), magnetic-dipole incident fields,
               scattered magnetic field (eq. 4 with eq. 6).
  operator.py  Section 2.2, eqs. 8-10: tabulated Green kernel, direct-summation operator, FFT
               operator with 2x zero padding, dense matrix for tiny grids.
  gmres.py     restarted GMRES (Saad & Schultz) with the relative-residual rule of eq. 9.
  dd.py        Section 2.3, eqs. 11-23 and Algorithm 1: block Gauss-Seidel / block Jacobi sweeps
               with adaptive sub-domain tolerance and warm starts; flexible GMRES over one sweep
               (the Krylov outer iteration of the paper's conclusion).
  solve.py     the full forward model: incident field, solve, receiver fields.
  contraction.py  the contraction form of the operator (named at the end of Section 2.3).
  fno.py       the warm-start network (not in the paper): forward and analytic backward.

Readings where the paper is silent or garbled are marked "Reading:" in the docstrings.
Every function here is pinned by the ``-m "not gpu"`` tests against closed forms, finite differences,
brute force or the LU solution. The contraction form is parity unpinned against the paper itself
(the paper prints no formula for it); it is pinned by its equivalence with the conventional solution
and by the contraction property of the discrete operator.
"""
