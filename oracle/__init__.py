"""FP64 CPU oracle for sketched ANLS (SANLS / DSANLS, arXiv 2009.02845).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package.  The GPU
library under ``paper_2009_02845_gb300`` never imports, links or runs any of
it, and it imports nothing from the GPU library: the two share no code.

Layout:
  rng.c / rng.py   -- Philox4x32-10 field, uniforms, Gaussian transform and
                      Feistel subsampling (plain C, exact binary32 steps).
  method.py        -- the method itself in FP64 numpy, step by step in the
                      paper's order and notation (Section 3.2-3.5, Alg. 1-3).
  nnls.py          -- exact nonnegative least squares by brute-force support
                      enumeration and by active set, plus a KKT checker.

Parity status of each function is recorded in its docstring; everything
here is pinned by ``tests/test_oracle_*.py``.
"""
