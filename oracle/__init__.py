"""Oracle — TEST INFRASTRUCTURE ONLY.

A plain, slow, FP64 NumPy restatement of what the GSIS method of
"Accelerated simulation of multiscale gas-radiation coupling flows via a general
synthetic iterative scheme" computes.  Only ``tests/``, ``__graft_entry__.smoke()``
and ``bench.py``'s CPU-baseline leg may import it.  It shares no code with the
CUDA library; both consume the seeded inputs of ``gsis_inputs``.

Modules:
  model    -- Section 2.1: relaxation-rate matrix A, auxiliary heat fluxes,
              mode temperatures, tau, k_eff, NSF transport coefficients
  kinetic  -- Eqs. (kinetic_equation), (reference_distribution), (getmoment),
              (dis_micro): reference distributions, moments, the implicit
              finite-volume kinetic sweep for gas and photons
  macro    -- Eqs. (macroscopic_equation), (NSF_constitutive), (getHoTs),
              (delta_macro), Appendix A: HoT and the synthetic-equation solver
  gsis     -- Section 3 and Section 6: CIS/GSIS outer iterations, sync, epsilon
  fourier  -- Section 4: CIS and GSIS Fourier stability matrices
  mlp      -- warm-start network forward/backward/Adam (not in the paper)
"""
