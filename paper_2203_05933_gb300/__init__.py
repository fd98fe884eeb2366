"""GB300-native evaluation of the FMM-accelerated volume potential with sparse
singular/near-singular corrections (Anderson, Zhu, Veerapaneni, arXiv 2203.05933).

The compute path lives in ``libvp.so`` (hand-written CUDA for sm_103a behind a
C ABI declared in ``include/vp.h``); :mod:`.vp` is the thin ctypes binding and
:mod:`.autograd` the differentiable wrapper. Nothing here falls back to a CPU
implementation: if the library is missing, the binding raises.
"""

__all__ = ["inputs"]
