"""GB300-native (sm_103a) sparse FFT by downsampling in time (sFFT-DT).

The transform runs in the CUDA library built from ``csrc/`` behind the C ABI
of ``include/sft.h``; ``sft`` is its thin ctypes binding.
"""
from ._build_lib import build as _build


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile libsft.so for sm_103a in-tree and return its path."""
    return _build(force=force, verbose=verbose)


from . import sft  # noqa: E402
from .sft import Batch, Mlp, Plan, Result, SftError  # noqa: E402

__all__ = ["build", "sft", "Batch", "Mlp", "Plan", "Result", "SftError"]
