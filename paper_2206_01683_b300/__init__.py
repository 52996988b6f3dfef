"""B300 (sm_103a) implementation of FishGym's moving-frame IB-LBM time step
(arXiv 2206.01683, Sec. III-B).  The compute path is the CUDA library
libfishlbm.so behind the C ABI of include/fishlbm.h; ``fishlbm`` is its thin
Python binding and ``inputs`` holds the seeded synthetic workloads."""
from . import fishlbm  # noqa: F401  (loads the library lazily, fails loudly if absent)
