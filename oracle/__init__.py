"""CPU oracle for the JaxWildfire stochastic cellular automaton (arXiv 2512.06102).

TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the benchmark's
CPU-baseline leg may import anything here; the CUDA library and its Python
binding share no code with it.

  oracle.discrete   ctypes access to jwf_oracle.c (Philox4x32-10, the discrete
                    step and rollout; Section 3 "Stochastic update")
  oracle.prob       FP64 rates and thresholds (Eqs. 1-4)
  oracle.relaxed    FP64 raw-probabilities update (Eqs. 5-10) and the
                    calibration loss (Section 4)

Parity pins live in tests/test_oracle_*.py.  Parity unpinned: the absolute
parameter values and the per-class modifier tables (the paper prints none).
"""
