"""FP64 CPU oracle for the two-fluid Yee scheme (arXiv 2305.13419).

TEST INFRASTRUCTURE: only `tests/`, `__graft_entry__.smoke()` and the CPU
baseline leg of `bench.py` may import this package.  The CUDA product path
never does, and the two share no code.

Contents
  stepper.py  -- ctypes wrapper of twofluid_oracle.c (Algorithm 1, Sec. 3)
  theory.py   -- closed forms of Sec. 4: complex wavenumber, skin depth,
                 reflection coefficient, cut-off; discrete dispersion
  qfit.py     -- Q-factor from a windowed probe DFT (exact finite-sum model)
  esprit.py   -- damped-mode poles of a probe time series (ESPRIT), the
                 estimator Sec. 5 names, as an independent Q check
  build.py    -- compiles the C stepper with gcc (no GPU needed)
"""
