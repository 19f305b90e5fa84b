"""GB300-native exchange-correlation integration (E_xc, V_xc, N_el) in a Gaussian basis.

The computation lives in the CUDA library ``_lib/libgbxc.so`` (sources in
``csrc/``, C-ABI in ``include/gbxc.h``); ``binding`` is its ctypes binding.
"""
from .binding import *  # noqa: F401,F403
from .binding import Context, GbxcError, LibraryMissing, lib  # noqa: F401
