"""FP64 CPU oracle for the realfast search hot path.

TEST INFRASTRUCTURE ONLY: imported by the tests, by the smoke check and by
the CPU-baseline leg of the benchmark, never by the engine itself.
"""

from .realfast_oracle import (  # noqa: F401
    CLIP_SIGMA,
    C_LIGHT,
    DISP_CONST,
    EDGE_FULL,
    EDGE_PARTIAL,
    ImageStats,
    OraclePlan,
    baseline_uvw,
    candidate_features,
    candidate_spectrum,
    cell_table,
    dedisperse_resample,
    delay_table,
    dirty_image_complex,
    dirty_image_dft,
    dirty_image_fft,
    grid_full_plane,
    image_stats,
    moments,
    n_valid_times,
    periodic_dm_trials,
    periodic_image,
    periodic_series_transform,
    periodic_stats,
    round_half_away,
    search_periodic,
    search_segment,
    search_stream,
    stream_overlap,
    stokes_i,
    subtract_mean,
)
