"""GB300-native (sm_103a) hot path of the optical-flow video stabiliser of
arXiv 1701.03572: Gaussian pyramid, Shi-Tomasi corners, pyramidal
Lucas-Kanade with a forward-backward check, robust rigid / similarity fit,
averaging-window smoothing and the compensating warp, as hand-written CUDA
kernels behind the C ABI in include/stab.h.  `stab` is the Python binding.
"""
from .build import LIB, build  # noqa: F401
