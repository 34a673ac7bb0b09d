"""GB300-native Newton step of the fully implicit polymer-flooding model
(arXiv 1807.05298): hand-written CUDA kernels for sm_103a behind the C ABI of
include/polyflood.h, with a thin ctypes binding (``binding``).

Build in-tree with ``python -m paper_1807_05298_gb300.build``.
"""

__all__ = ["binding", "build"]
