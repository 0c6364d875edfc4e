"""Seeded synthetic inputs shared by the GPU path's tests/benchmark and the CPU oracle.

This module draws interferogram frames only. It contains none of the
demodulation arithmetic (no Fresnel transform, no covariance, no
eigendecomposition, no projection), so both sides can consume the same
frames without sharing any of the method's code.
"""

from .speckle import (  # noqa: F401
    SpeckleParams,
    SpeckleStream,
    speckle_window,
    known_rank_frames,
    hadamard_rows,
)
from .uneven import SizeGroup, uneven_batch  # noqa: F401
