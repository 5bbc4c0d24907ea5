"""Pins for the oracle's overlapping-segment stream search (Sec. 3.2).

Without mean subtraction, cutting a run of integrations into segments that
overlap by the longest sweep, each searching t' < stride / dt, and searching
the remainder under the plan's edge rule must give exactly the images of one
search over the whole run: the same (DM, dt, t') set, each start time once,
and the same statistics.  With mean subtraction each segment takes its own
mean, so a steady source vanishes from every segment.
"""

import numpy as np
import pytest

import oracle
import synth


def _small_spec(edge="full", mean_subtract=False, continuum=False):
    spec = synth.SegmentSpec(name="stream-small", nchan=16, f_lo_hz=1.0e9, bw_hz=0.5e9, nint=220,
                             inttime_s=5e-3, npix=32, dm_list=np.linspace(0.0, 150.0, 5),
                             dt_list=[1, 2, 4], threshold=5.0, nant=6, edge=edge,
                             mean_subtract=mean_subtract, cell_rad=26.0 * synth.segments.ARCSEC, seed=7)
    # a pulse whose sweep straddles the boundary between the first two segments
    spec.pulses = [dict(dm=150.0, t0_s=40 * 5e-3, width_s=10e-3, amp=3.0, x=20, y=13)]
    if continuum:
        spec.continuum = [dict(amp=4.0, x=9, y=22)]
    return spec


def _plan(spec, seg):
    return oracle.OraclePlan(seg["ant_uvw"], seg["freq_hz"], spec.inttime_s, spec.npix, spec.cell_rad,
                             spec.dm_list, spec.dt_list, spec.threshold, edge=spec.edge,
                             npol=spec.npol, mean_subtract=spec.mean_subtract)


@pytest.mark.parametrize("edge", ["full", "partial"])
@pytest.mark.parametrize("stride", [4, 16, 40])
def test_stream_equals_one_search_over_the_run(edge, stride):
    spec = _small_spec(edge)
    seg = synth.make_segment(spec)
    op = _plan(spec, seg)
    overlap = oracle.stream_overlap(op)
    assert 0 < overlap < 100
    c1, s1 = oracle.search_segment(op, seg["vis"], with_stats=True)
    c2, s2 = oracle.search_stream(op, seg["vis"], stride, with_stats=True)
    assert sorted(s1) == sorted(s2)
    for k, a in s1.items():
        b = s2[k]
        assert (a.x, a.y) == (b.x, b.y), k
        assert abs(a.peak - b.peak) <= 1e-12 * abs(a.peak) + 1e-15
        assert abs(a.sigma - b.sigma) <= 1e-12 * a.sigma
    assert [(c["dm_idx"], c["dt_idx"], c["t_idx"]) for c in c1] == \
           [(c["dm_idx"], c["dt_idx"], c["t_idx"]) for c in c2]
    assert len(c1) > 0


def test_stream_covers_each_start_time_once():
    spec = _small_spec()
    seg = synth.make_segment(spec)
    op = _plan(spec, seg)
    _, st = oracle.search_stream(op, seg["vis"], 8, with_stats=True)
    total = seg["vis"].shape[0]
    for d in range(len(spec.dm_list)):
        for s, dt in enumerate(spec.dt_list):
            ts = sorted(t for (dd, ss, t) in st if (dd, ss) == (d, s))
            n = oracle.n_valid_times(total, int(op.max_delay[d]), dt, "full")
            assert ts == list(range(n)), (d, s)


def test_stream_rejects_a_stride_that_is_not_a_multiple_of_dt():
    spec = _small_spec()
    seg = synth.make_segment(spec, nint=40)
    with pytest.raises(ValueError):
        oracle.search_stream(_plan(spec, seg), seg["vis"], 6)


def test_stream_mean_subtraction_is_per_segment():
    spec = _small_spec(mean_subtract=True, continuum=True)
    seg = synth.make_segment(spec)
    op = _plan(spec, seg)
    stride = 16
    _, st = oracle.search_stream(op, seg["vis"], stride, with_stats=True)
    # the steady source at (9, 22) is gone from every segment: its pixel is
    # the peak of a noise image's share of the images, not of most of them
    at_src = np.mean([(v.x, v.y) == (9, 22) for v in st.values()])
    assert at_src < 0.02
    spec0 = _small_spec(continuum=True)
    _, st0 = oracle.search_stream(_plan(spec0, seg), seg["vis"], stride, with_stats=True)
    assert np.mean([(v.x, v.y) == (9, 22) for v in st0.values()]) > 0.5
    # and segment k's images equal a one-shot mean-subtracted search of its window
    overlap = oracle.stream_overlap(op)
    w = seg["vis"][2 * stride: 2 * stride + stride + overlap]
    _, sw = oracle.search_segment(op, w, with_stats=True)
    for (d, s, t), a in sw.items():
        dt = spec.dt_list[s]
        if t < stride // dt:
            b = st[(d, s, 2 * stride // dt + t)]
            assert abs(a.peak - b.peak) <= 1e-12 * abs(a.peak) + 1e-15
            assert (a.x, a.y) == (b.x, b.y)
