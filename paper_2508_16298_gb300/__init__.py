"""GB300-native hybrid quantum Monte Carlo hot path (arXiv 2508.16298).

The compute lives in the CUDA library ``libhqmc.so`` built from ``csrc/`` for
sm_103a and exposed through a C ABI (``include/hqmc.h``).  ``hqmc`` is the thin
ctypes binding with the same entry-point names; importing it loads the library
and fails loudly if it has not been built.  ``inputs`` holds the seeded
synthetic input generators and no arithmetic of the method.
"""

__all__ = ["hqmc", "inputs", "build"]
