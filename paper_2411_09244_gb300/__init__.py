"""GB300-native parareal all-at-once partially explicit splitting for high
contrast multiscale diffusion (Wang, Yang, Leung, arXiv:2411.09244).

The numerical work runs in libpint.so (CUDA, sm_103a), reached through the C
ABI of include/pint.h.  `api.Pint` is the Python front end; `inputs` holds the
seeded synthetic problems.  Importing this package does not load the CUDA
library; the first call does, and fails loudly if it has not been built.
"""

__all__ = ["api", "inputs"]
