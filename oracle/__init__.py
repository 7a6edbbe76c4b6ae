"""CPU oracle for the shifted Krylov solver.  TEST INFRASTRUCTURE ONLY.

Plain, slow, FP64 implementations of what the GPU path computes, written from
the Komega paper (arXiv:2001.08707):

* ``dense``: the plain definitions x_k = (z_k I - H)^{-1} b (Eq. 4-5) and the
  spectral (Lehmann) sum of Eq. 3, for small M.
* ``shifted_cocg``: the shifted COCG iteration step by step (Sec. 2.2,
  Appendix A), full and projected modes, seed switching; with ``log=True`` it
  also keeps the per-iteration record used for recalculation.
* ``shifted_bicg``: the other solvers of Table 1 (Appendix B): shifted BiCG
  with a shadow residual, and shifted CG for Hermitian A with real shifts.
* ``recalc``: projections at new shifts replayed from that record without
  matrix-vector products (Sec. 3.3 (iv); Eqs. 20-22, 25-26).
* ``adjoint``: the gradient of the spectrum with respect to the Hamiltonian's
  parameters.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA path
and never imports it.  Every function is pinned by CPU tests against values
fixed by the paper or by mathematics (tests/test_oracle_*.py).
"""
