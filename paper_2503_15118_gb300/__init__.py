"""GB300-native sparse register-level quantum-state simulation.

The hot path of the sparse-state simulator of SparQSim (arXiv 2503.15118):
applying operations to a state stored only as its nonzero branches (packed
64/128-bit basis keys with complex amplitudes), as hand-written CUDA for
sm_103a behind the C ABI of ``include/sqs.h``.

* ``paper_2503_15118_gb300.sqs``       -- ctypes binding of the C ABI
* ``paper_2503_15118_gb300.build``     -- nvcc build of ``_build/libsqs.so``
* ``paper_2503_15118_gb300.workloads`` -- seeded synthetic gate lists
"""
from . import workloads  # noqa: F401

__all__ = ["workloads", "sqs", "build"]
