"""Seeded synthetic inputs shaped like VLA fast-sampled visibility segments.

This package only *generates inputs*: antenna positions and their uvw, channel
frequencies, DM trial lists and complex visibilities (noise plus injected
dispersed pulses or a continuum source).  It holds none of the search's own
arithmetic (no delay table, no uv-cell rounding, no gridding, no imaging), so
both the FP64 oracle and the CUDA engine can take its output without sharing
any of the method with each other.
"""

from .segments import (  # noqa: F401
    SegmentSpec,
    array_uvw,
    channel_freqs,
    config,
    dm_grid_linear,
    dm_grid_smearing,
    make_segment,
    serving_shapes,
    CONFIG_NAMES,
)
