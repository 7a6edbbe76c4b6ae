"""CPU oracle for the shifted Krylov solver.  TEST INFRASTRUCTURE ONLY.

Plain, slow, FP64 implementations of what the GPU path computes, written from
the Komega paper (arXiv:2001.08707):

* ``dense``: the plain definitions x_k = (z_k I - H)^{-1} b (Eq. 4-5) and the
  spectral (Lehmann) sum of Eq. 3, for small M.
* ``shifted_cocg``: the shifted COCG iteration step by step (Sec. 2.2,
  Appendix A), full and projected modes, seed switching.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA path
and never imports it.  Every function is pinned by CPU tests against values
fixed by the paper or by mathematics (tests/test_oracle_*.py).
"""
