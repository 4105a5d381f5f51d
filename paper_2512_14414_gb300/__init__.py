"""GB300-native nested single-layer CTMRG energy and gradient (arXiv:2512.14414).

The compute path is libctm.so (hand-written sm_103a CUDA behind the C ABI of
include/ctm.h); ``api`` marshals torch device memory into it.  Build with
``paper_2512_14414_gb300.build.build()``.
"""
from .api import CTM, CTMEnergy, CTMError  # noqa: F401
