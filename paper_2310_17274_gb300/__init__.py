"""GB300-native batched cost-and-gradient evaluation, L-BFGS step and parallel
noisy line search for collision-free motion optimisation (arXiv 2310.17274).

The compute path is the C-ABI library ``libcrgb.so`` (hand-written CUDA for
sm_103a, see ``include/crgb.h``); ``paper_2310_17274_gb300.crgb`` is its thin
ctypes binding.  Nothing here falls back to the CPU: every entry point raises
if the library is missing.
"""
__all__ = ["synth"]
