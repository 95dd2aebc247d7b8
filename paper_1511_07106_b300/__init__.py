"""B300-native multi-volume TSDF integration and raycasting.

Hot path of Salvato, Finman, Leonard, "Multi-Volume High Resolution RGB-D
Mapping with Dynamic Volume Placement" (arXiv 1511.07106): per-frame
projective TSDF + colour integration into every active subvolume and the
per-pixel multi-volume raycast, as hand-written sm_103a CUDA behind the C ABI
of ``include/mvtsdf.h`` (``libmvtsdf.so``, built in-tree by
``python -m paper_1511_07106_b300.build``).

``synth`` (seeded synthetic scenes) is importable without the CUDA library;
``Mapper`` and friends load it on first use and raise if it is missing.
"""
from . import synth  # noqa: F401

_LAZY = {"Mapper", "Placer", "Config", "MVError", "decode", "encode", "intrinsics"}


def __getattr__(name):
    if name in _LAZY:
        from . import mapper
        return getattr(mapper, name)
    raise AttributeError(name)
