"""GB300-native variable-density pressure projection (multigrid Poisson solve + velocity correction).

The compute path is the CUDA library ``libmgproj.so`` built from ``csrc/`` and reached
through the C ABI declared in ``include/mgproj.h``; ``mgproj`` is its ctypes binding and
``autograd`` wraps the projection as a ``torch.autograd.Function``.  Importing this
package does not load the library; importing ``mgproj`` does, and fails loudly if the
library has not been built.
"""
