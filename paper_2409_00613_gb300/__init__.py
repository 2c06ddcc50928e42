"""GB300-native BWT build / merge / search (the method of H. Li, arXiv 2409.00613).

The compute lives in librb3.so (CUDA, sm_103a; C ABI in include/rb3.h); this
package is its thin Python binding (``rb3``) and the in-tree build script
(``build``).  There is no CPU fallback: without the compiled library or a CUDA
device every call raises ``RB3Error``."""
from .rb3 import *  # noqa: F401,F403
from .rb3 import COMPLETION_DTYPE, Index, RB3Error, SMEM_DTYPE, Server, lib, rb3_opts, rb3_server_opts  # noqa: F401
