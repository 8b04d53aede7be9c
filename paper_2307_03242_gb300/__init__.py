"""GB300-native matrix-free multigrid for the elastic Helmholtz equation (arXiv 2307.03242).

The compute path is libemg.so (hand-written sm_103a CUDA behind a C ABI, include/emg.h);
`emg` is its ctypes binding. Build with __graft_entry__.build()."""
from .build import build_library, LIB as LIB_PATH

__all__ = ["build_library", "LIB_PATH"]
