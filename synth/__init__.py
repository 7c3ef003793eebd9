"""Seeded synthetic inputs shared by the oracle and the CUDA path.

Random draws and index bookkeeping only (Philox-4x32-10, complex normals,
stencil geometry, Hermitian pairing of hop matrices); no solver arithmetic.
"""
from .philox import philox4x32_10, complex_normal  # noqa: F401
from .coarse import (BASE_SEED, STREAM_B, STREAM_HOP, STREAM_SELF, STREAM_U,  # noqa: F401
                     STREAM_W, STREAM_X0, coarse_op, load_shift, stencil, vectors, volume)
from .workloads import BATCH, WORKLOADS  # noqa: F401
