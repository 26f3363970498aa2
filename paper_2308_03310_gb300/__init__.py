"""GB300-native LBM-LETKF hot path (arXiv 2308.03310): CUDA library + thin Python binding.

``letkf`` mirrors the C ABI of ``include/letkf.h`` (libletkf.so, built in tree for
sm_103a by ``_build.build()``).  The package holds no CPU implementation of the
method.
"""
from . import letkf  # noqa: F401
from ._build import build, LIB  # noqa: F401
