"""One-level FETI for nonlocal diffusion and peridynamics on a GB300 (sm_103a).

The computation lives in the CUDA library ``libnlfeti.so`` (``csrc/``, C ABI in
``include/nlfeti.h``); ``binding`` is its ctypes front end.
"""
from .binding import (Context, NlfetiError, Options, Problem, Server, default_options, load,  # noqa: F401
                      library_path)
