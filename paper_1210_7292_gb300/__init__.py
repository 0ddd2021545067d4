"""GB300 (sm_103a) M2L translation of the black-box Chebyshev FMM.

The computation lives in libm2l.so (CUDA kernels behind the C ABI of
include/m2l.h); `m2l` is its thin ctypes binding, `autograd` wraps the
forward/adjoint pair as a torch.autograd.Function, `synth` draws seeded
synthetic inputs.
"""
from . import m2l  # noqa: F401
