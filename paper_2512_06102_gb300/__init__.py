"""jwf: GB300-native engine for the stochastic cellular-automaton wildfire model
of JaxWildfire (arXiv 2512.06102).

  paper_2512_06102_gb300.jwf        ctypes binding of libjwf (the C-ABI library)
  paper_2512_06102_gb300.relaxed    autograd.Function and checkpointed rollout of
                                    the relaxed (raw-probabilities) step
  paper_2512_06102_gb300.scenarios  seeded synthetic inputs
  paper_2512_06102_gb300.build      nvcc build of libjwf for sm_103a

Importing the package loads nothing; the binding loads libjwf on first use and
raises if it is missing (there is no CPU fallback).
"""
__all__ = ["jwf", "relaxed", "scenarios", "build"]
