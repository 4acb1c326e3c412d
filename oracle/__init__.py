"""Plain, slow FP64 CPU oracle for the implicit-Coriolis shell-convection step.

This package is TEST INFRASTRUCTURE, not part of the product.  Only the test
suite (``tests/``), ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import it.  The CUDA library never calls into it and the two
share no code: the oracle builds its own tables, transforms, operators and
solvers from the paper's equations, with numpy/scipy primitives (matmul, LU,
least squares) as the only building blocks.

Modules
-------
basis   Chebyshev radial tables, Gauss-Legendre nodes, associated Legendre
        functions with the paper's normalisation (Sec. 3.1, Eq. Ylm_norm).
sht     scalar / vector spherical-harmonic synthesis and analysis by direct
        sums, and the azimuthal DFT (Sec. 3.1).
shell   the discretised Boussinesq model: explicit terms, implicit operator
        with Coriolis (Sec. 3.2, Eqs. impcor_e_final / impcor_f_final), the
        IMEX Euler step (Eq. discrete), the Jacobian action with the phase
        trick (Secs. 3.3-3.4).
krylov  MGS-GMRES and the Newton iteration for rotating waves (Secs. 3.3-3.4).
onset   the linear onset of convection about the conductive state: the pencil of the
        linearised operator per (m, symmetry class), its rightmost eigenvalue, and the
        critical Rayleigh number and drift of each mode (Secs. 2.2, 4.4).
continuation  natural-parameter continuation in Ra and in log10 Ek, spectral-tail
        refinement and zero-fill regridding (Secs. 4.3-4.4).

Parity status of each function is stated in its docstring; functions without
an independent pin say "parity unpinned".
"""
