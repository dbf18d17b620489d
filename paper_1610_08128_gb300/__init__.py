"""GB300-native Reverse Cuthill-McKee ordering (Azad, Jacquelin, Buluc, Ng; arXiv:1610.08128).

The ordering runs in librcm_gb300.so (hand-written sm_103a CUDA kernels behind the C ABI of
include/rcm.h); :mod:`.rcm` is the thin ctypes binding, :mod:`.synth` the seeded input generators,
:mod:`.build` the in-tree nvcc build.
"""
from . import build, synth  # noqa: F401

LIB_PATH = build.LIB_PATH


def build_library(**kw) -> str:
    return build.build(**kw)
