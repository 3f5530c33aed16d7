"""FP64 CPU oracle for the implicit radiation / ionization / gas-energy step.

TEST INFRASTRUCTURE ONLY.  This package is the slow, plain reference that the CUDA path is
checked against.  Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import it.  The product path (the C-ABI library
and its Python binding) never imports, links or runs anything in here, and this package never
imports the product path: the two share no code.

Modules
-------
closure  physical constants, the tabulated rate/cooling closure, the equation of state and
         the grey spectral constants (Sec. 2.1-2.2, eqs. eos, temperature, grey_definition,
         adaptive_spectrum).
model    the theta-scheme operators, the nonlinear residual and its analytic Jacobian
         (Sec. 3.2, eqs. energy/chemistry/radiation_simplified, mDE, mLe, mLn, mLE,
         nonlinear_residual, jacobian_matrix, jacobian_submatrices, limiter, rmsnorm).
solve    the globalised Newton iteration with either an unreduced sparse direct solve or the
         Schur-complement reduction (eqs. newton_system2, schur_components, step_ia) followed
         by an unpreconditioned CG solve; the explicit predictor (eq. explicit_predictor).
mlp      FP64 forward/backward of the per-cell MLP used as a learned Newton initial guess
         (not in the paper; an added form).

Every stored constant and formula here is written from the paper and from the published
closure forms named in ``closure``; nothing in here is produced by the CUDA path.
"""
