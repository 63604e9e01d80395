"""GB300-native TV-Stokes denoising hot path.

The compute path is libtvs.so (hand-written sm_103a CUDA behind the C ABI of
include/tvs.h); ``binding`` marshals torch CUDA tensors into it.  Import the
binding explicitly (``from paper_2602_17494_gb300 import binding``): it loads
the library and raises if it has not been built.
"""

__all__ = ["binding", "build"]
