"""aewave: autoencoder-compressed adjoint gradients and Gauss-Newton Hessian-vector
products for the 3-D acoustic velocity-strain wave equation on GB300 (sm_103a).

The computation lives in the C-ABI library libaewave.so (include/aewave.h); the
Python layer (``aewave``) only marshals arguments.  Importing this package does not
load the library; ``from paper_2304_04781_gb300 import aewave`` does, on first use.
"""

__all__ = ["aewave", "inputs", "build"]
