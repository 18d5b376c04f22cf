"""GB300-native (sm_103a) implementation of the excursion-set 21-cm likelihood hot path of
21CMMC (Greig & Mesinger 2015, arXiv:1501.06576).

- ``eor21``: ctypes binding of the C ABI in ``include/eor21.h`` (libeor21.so, CUDA);
- ``synth``: seeded synthetic inputs (density boxes, walker parameters);
- ``build``: in-tree nvcc build of libeor21.so.

Submodules load lazily so that ``synth`` works without the CUDA library.
"""
__all__ = ["eor21", "synth", "build"]
