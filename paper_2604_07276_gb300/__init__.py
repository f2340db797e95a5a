"""GB300-native DPA-1 (se_atten) energy / force / virial engine.

The compute path lives in ``lib/libdpa1.so`` (hand-written CUDA for sm_103a
behind the C ABI of ``include/dpa1.h``); this package is its thin Python
binding.  Importing the package loads the library and fails loudly if it
has not been built.
"""

from .binding import DPA1, DPError, inspect_weights, kernel_launches, load_library, LIB_PATH, EXPORTS, box9

load_library()

__all__ = ["DPA1", "DPError", "inspect_weights", "kernel_launches", "load_library", "LIB_PATH", "EXPORTS", "box9"]
