"""CPU FP64 oracle of the Chebyshev-FMM M2L translation.

TEST INFRASTRUCTURE ONLY: imported by the tests, by the smoke check and by the
CPU-baseline leg of the benchmark; never by the library or its binding.  It
shares no code with the CUDA path.
"""
from .m2l_oracle import *  # noqa: F401,F403
from .m2l_oracle import build_c  # noqa: F401
from . import dfmm_oracle as dfmm  # noqa: F401,E402
