"""GB300-native mixed-precision iterative-refinement linear solver.

Baboulin et al., "Accelerating Scientific Computations with Mixed Precision
Algorithms": factor PA = LU in low precision on the tensor cores, refine the
solution to FP64 accuracy with FP64 residuals (Algorithm 1, Section 2.1).

Submodules:
  solver  -- ctypes binding of the C ABI (include/mpsolve.h); needs a GPU
  build   -- nvcc build of csrc/*.cu into _build/libmpsolve.so (sm_103a)
  inputs  -- seeded synthetic workloads (no solver arithmetic)

Importing the package does not load the CUDA library; the first call into
``solver`` does, and raises if it cannot.
"""

__all__ = ["solver", "build", "inputs"]
