"""GB300-native matched-filter search of arXiv:1708.01609 (libbege).

The compute path is the C-ABI library ``libbege.so`` (include/bege.h) built
from ``csrc/`` for sm_103a; ``binding`` is its ctypes binding.
"""
from .build import build  # noqa: F401
