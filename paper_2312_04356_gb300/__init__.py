"""GB300 RNS-CKKS library for CinS conv2d fused with bootstrapping (NeuJeans, arXiv 2312.04356).

The compute path is the CUDA shared library built from csrc/ (C ABI in
include/ckks.h); `ckks` is its Python binding.
"""
from . import ckks  # noqa: F401
