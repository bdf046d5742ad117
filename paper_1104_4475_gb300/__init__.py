"""Tiled Householder QR on one GB300 (sm_103a): the elimination trees of
"Tiled QR factorization algorithms" (Bouwmeester, Jacquelin, Langou, Robert,
2011) executed as a task graph by a persistent CUDA kernel.

The C ABI is include/tqr.h (library ``libtqr.so``, built by
:func:`paper_1104_4475_gb300.build.build`); :mod:`paper_1104_4475_gb300.tqr`
is its Python binding.
"""

from .tqr import *  # noqa: F401,F403
from .tqr import lib, colmajor, to_numpy, Factors, TqrError  # noqa: F401
