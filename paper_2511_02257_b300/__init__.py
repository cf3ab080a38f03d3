"""B300-native executor for lattice-QCD correlation-function contraction DAGs.

The compute path is the native library ``_lib/liblqc.so`` (C++ host runtime +
CUDA kernels for sm_103a) behind the C ABI declared in ``include/lqc.h``;
this package is the thin ctypes binding.  Importing it loads the library and
raises ImportError when it is missing: there is no fallback implementation.
"""
from .lqc import *  # noqa: F401,F403
from .lqc import Dag, LqcError, library_path  # noqa: F401
