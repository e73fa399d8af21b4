"""GB300-native domain-decomposition Helmholtz solver (WaveHoltz subdomain
solves, every subdomain of a sweep in one CUDA kernel launch).

The compute path is the CUDA library ``_lib/libhz.so`` (C ABI in
``include/hz.h``); this package is its ctypes binding.  Importing it loads
the library and raises ImportError if it has not been built -- there is no
CPU fallback.
"""

from ._binding import *  # noqa: F401,F403
from ._binding import HzError, load, library_path, exported_names  # noqa: F401

load()
