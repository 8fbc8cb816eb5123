"""GB300-native push-pull BFS: the Boolean masked matvec of direction-optimized
BFS (arXiv 1804.03327) as hand-written sm_103a CUDA kernels behind a C ABI
(include/gbx.h).  ``gbx`` is the Python binding; ``roofline`` holds the
algorithmic byte model used to report achieved bandwidth."""
from . import gbx  # noqa: F401
