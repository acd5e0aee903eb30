"""GB300-native projection-based RCA 3D ULM (arXiv 2511.21647).

The compute path is librca (CUDA C++, sm_103a) behind the C ABI in
include/rca.h; ``rca`` is its Python binding with the same names and
``pipeline`` a torch-side session helper.  There is no CPU fallback.
"""
from . import _lib  # noqa: F401
from .build import build, LIB as LIB_PATH  # noqa: F401
