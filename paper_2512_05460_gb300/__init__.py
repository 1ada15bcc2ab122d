"""GB300-native ProbeWalk: probe-driven random-walk estimation of the squared
biharmonic distance beta(s,t) = ||L^+(e_s - e_t)||^2 (arXiv 2512.05460).

The computation lives in libprobewalk.so (hand-written CUDA for sm_103a behind
the C ABI of include/probewalk.h).  :mod:`paper_2512_05460_gb300.probewalk`
is the ctypes binding with the same function names; :mod:`.build` compiles
the library in-tree.  Importing this package does not load the library.
"""

import importlib

__all__ = ["probewalk", "build"]


def __getattr__(name):
    if name in __all__:
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
