"""GB300-native mixed-precision iterative refinement for LSE and GLS problems.

The compute path is the C-ABI library ``libmpir.so`` (hand-written CUDA for
sm_103a); ``paper_2406_16499_gb300.mpir`` is its thin ctypes binding.
``paper_2406_16499_gb300.inputs`` holds the seeded synthetic workloads.
"""
__all__ = ["inputs", "mpir"]
