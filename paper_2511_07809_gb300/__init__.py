"""GB300-native online Tensor LDA: the streaming whiten + CP-gradient + SGD
hot path as hand-written sm_103a CUDA behind a C ABI (include/tlda.h).

``tlda`` is the thin Python binding of that ABI (ctypes; torch tensors supply
device memory and streams)."""
from . import _build  # noqa: F401

__all__ = ["tlda", "_build"]
