"""FP64 CPU oracle for the FFT multipole estimators (Xie et al., power spectrum and bispectrum
multipole measurements).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the CUDA library and its Python binding)
may import this package.  Only the test suite, ``__graft_entry__.smoke()`` and the benchmark's CPU
baseline leg use it.  It shares no code with the GPU path: it is plain NumPy/SciPy in float64,
written to follow the paper's definitions term by term, and is slow on purpose.

Modules
  harmonics  Legendre / associated Legendre / Y_lm (Appendix A), Wigner 3j (Appendix F),
             g_l(t) closed and integral forms (Lemma 2, Appendix H).
  mesh       mass assignment (CIC/TSC), interlacing, window compensation (Sec. 3.1).
  power      catalogue scalars, Yamamoto multipoles in the Hand+17 form (Eq. hand) and the
             symmetry-reduced form (Eqs. new_F_ell, pk_final), two-index P_ll' and the modified
             multipoles P_4b, P_6b, P_8b (Eqs. Plnew, Pllp).
  bispec     Scoccimarro B_l (Eq. bi_sco), brute-force triangle sums, the compressed TripoSH
             estimator B_l0l (Eq. new_bispec) in its collapsed and explicit-3j forms, odd B_1, B_3,
             multi-tracer bispectra.
  sugiyama   Sugiyama TripoSH B_l1l2L (Eq. sugi_estimator) with every sub-configuration, its
             analytic (Lemma 1) and FFT-method shot noise.
  shot       analytic and FFT-method bispectrum shot noise (Sec. 5.4).
  adjoint    gradients of P_l and equilateral B_0 with respect to the density mesh.

Each module's header names the tests that pin its functions and what they check, and a function's
docstring does so where its pins differ from its module's; a function with no pin would say
"parity unpinned" (none does: the analytic shot-noise forms, thin-shell approximations with no exact
reference, are pinned statistically and against the exact FFT-method sums, as their headers say).
"""
