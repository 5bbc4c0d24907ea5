"""C-ABI checks that need no GPU: symbols, validation, host tables vs the oracle."""

import ctypes

import numpy as np
import pytest

import oracle
import synth
import paper_1802_03084_gb300 as rf


@pytest.fixture(scope="module")
def L():
    from paper_1802_03084_gb300.build import build
    build()
    return rf.lib()


def test_every_declared_symbol_is_exported(L):
    names = rf.declared_symbols()
    assert {"rf_plan_create", "rf_search_segment", "rf_plan_destroy"} <= set(names)
    for n in names:
        assert hasattr(L, n), n
    assert rf.rf_version().startswith("realfast_gb300")


def _host_plan(spec, **kw):
    ant = synth.array_uvw(spec.seed, spec.nant, spec.dec_deg)
    f = synth.channel_freqs(spec.f_lo_hz, spec.bw_hz, spec.nchan)
    flags = rf.RF_HOST_ONLY | (rf.RF_EDGE_PARTIAL if spec.edge == "partial" else 0)
    p = rf.Plan(ant, f, spec.inttime_s, spec.npix, spec.cell_rad, spec.dm_list, spec.dt_list,
                spec.threshold, flags=flags, max_nint=spec.nint, **kw)
    op = oracle.OraclePlan(ant, f, spec.inttime_s, spec.npix, spec.cell_rad, spec.dm_list, spec.dt_list,
                           spec.threshold, edge=spec.edge)
    return p, op


@pytest.mark.parametrize("name", ["tiny", "realtime", "batching", "stress"])
def test_host_tables_bit_exact_vs_oracle(L, name):
    spec = synth.config(name)
    p, op = _host_plan(spec)
    with p:
        np.testing.assert_array_equal(p.delays(), op.delays)
        iu, iv, on = p.cells()
        np.testing.assert_array_equal(on, op.ongrid)
        np.testing.assert_array_equal(iu[on], op.iu[op.ongrid])
        np.testing.assert_array_equal(iv[on], op.iv[op.ongrid])
        info = p.info()
        assert info.nbl == 351
        assert info.iu_max == np.abs(op.iu[op.ongrid]).max()
        assert info.max_delay == op.delays.max()
        assert info.n_offgrid == (~op.ongrid).sum()
        n_zero_col = int(((op.iu == 0) & op.ongrid).sum())
        assert info.n_entries == int(op.ongrid.sum()) + n_zero_col
        for nint in (1, 17, spec.nint // 2, spec.nint):
            assert p.count_images(nint) == op.count_images(nint)


def test_count_images_matches_known_totals(L):
    for name, n in [("tiny", 1024), ("realtime", 177521), ("batching", 553095)]:
        spec = synth.config(name)
        p, _ = _host_plan(spec)
        with p:
            assert p.count_images(spec.nint) == n


def test_host_only_plan_rejects_search(L):
    spec = synth.config("tiny")
    p, _ = _host_plan(spec)
    with p:
        vis = np.zeros((4, 351, spec.nchan, 2), dtype=np.complex64)
        with pytest.raises(rf.RfError) as e:
            p.search(vis)
        assert e.value.status == rf.RF_ERR_INVALID_ARG


def _desc_kwargs(spec):
    ant = synth.array_uvw(spec.seed)
    f = synth.channel_freqs(spec.f_lo_hz, spec.bw_hz, spec.nchan)
    return dict(ant_uvw=ant, freq_hz=f, inttime_s=spec.inttime_s, npix=spec.npix, cell_rad=spec.cell_rad,
                dm_list=spec.dm_list, dt_list=spec.dt_list, threshold=spec.threshold, flags=rf.RF_HOST_ONLY,
                max_nint=spec.nint)


@pytest.mark.parametrize("field,value", [
    ("npix", 100), ("npix", 8), ("npix", 16384), ("npol", 3), ("inttime_s", 0.0), ("cell_rad", -1.0),
    ("threshold", 0.0), ("max_nint", 0), ("flags", rf.RF_HOST_ONLY | 0x80),
])
def test_invalid_desc_rejected(L, field, value):
    kw = _desc_kwargs(synth.config("tiny"))
    kw[field] = value
    d = rf.make_desc(**kw)
    with pytest.raises(rf.RfError) as e:
        rf.rf_plan_create(d)
    assert e.value.status == rf.RF_ERR_INVALID_ARG
    assert rf.rf_last_error()


def test_invalid_lists_rejected(L):
    kw = _desc_kwargs(synth.config("tiny"))
    for key, val in [("dm_list", [-1.0]), ("dt_list", [0]), ("dt_list", [2000]),
                     ("freq_hz", [0.0, 1e9]), ("dm_list", [float("nan")])]:
        k2 = dict(kw)
        k2[key] = val
        with pytest.raises(rf.RfError) as e:
            rf.rf_plan_create(rf.make_desc(**k2))
        assert e.value.status == rf.RF_ERR_INVALID_ARG


def test_null_arguments(L):
    P = ctypes.c_void_p
    assert L.rf_plan_create(None, ctypes.byref(P())) == rf.RF_ERR_INVALID_ARG
    assert L.rf_plan_destroy(None) == 0
    n = ctypes.c_size_t()
    assert L.rf_search_segment(None, None, 1, None, None, 0, ctypes.byref(n)) == rf.RF_ERR_INVALID_ARG
    assert L.rf_plan_get_info(None, None) == rf.RF_ERR_INVALID_ARG


def test_no_device_error_without_gpu(L):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    kw = _desc_kwargs(synth.config("tiny"))
    kw["flags"] = 0
    with pytest.raises(rf.RfError) as e:
        rf.rf_plan_create(rf.make_desc(**kw))
    assert e.value.status == rf.RF_ERR_NO_DEVICE


def test_zero_images_when_segment_shorter_than_sweep(L):
    spec = synth.config("realtime")
    kw = _desc_kwargs(spec)
    with rf.Plan(**kw) as p:
        assert p.count_images(900) > 0
        # FULL edge rule: DM trials whose sweep exceeds nint search nothing
        d = p.delays().max(axis=1)
        n = sum(max(0, (300 - m) // dt) if 300 - m > 0 else 0 for m in d for dt in spec.dt_list)
        assert p.count_images(300) == n


def test_estimate_bytes_without_device(L):
    spec = synth.config("realtime")
    kw = _desc_kwargs(spec)
    kw["flags"] = 0
    b = rf.rf_plan_estimate_bytes(rf.make_desc(**kw))
    # Stokes I (FP32) alone is 351 x 256 x 1024 x 8 bytes
    assert b > 351 * 256 * 1024 * 8
    b_small = rf.rf_plan_estimate_bytes(rf.make_desc(**kw), wave_images=64)
    assert b_small < b


def test_stream_rejects_bad_arguments(L):
    spec = synth.config("tiny")
    p, _ = _host_plan(spec)
    P = ctypes.c_void_p
    with p:
        h = P()
        # a host-only plan cannot stream
        assert L.rf_stream_create(p.handle, 64, 0, ctypes.byref(h)) == rf.RF_ERR_INVALID_ARG
        assert "HOST_ONLY" in rf.rf_last_error()
        assert not h.value
    assert L.rf_stream_create(None, 64, 0, ctypes.byref(P())) == rf.RF_ERR_INVALID_ARG
    assert L.rf_stream_create(None, 64, 0, None) == rf.RF_ERR_INVALID_ARG
    assert L.rf_stream_destroy(None) == 0
    n = ctypes.c_int32()
    assert L.rf_stream_push(None, None, 1, None, ctypes.byref(n)) == rf.RF_ERR_INVALID_ARG
    assert L.rf_stream_flush(None, None, ctypes.byref(n)) == rf.RF_ERR_INVALID_ARG
    m = ctypes.c_size_t()
    assert L.rf_stream_pop(None, None, 0, ctypes.byref(m)) == rf.RF_ERR_INVALID_ARG
    assert L.rf_stream_get_info(None, None) == rf.RF_ERR_INVALID_ARG


def test_clipped_noise_flag_accepted_and_sized(L):
    spec = synth.config("realtime")
    kw = _desc_kwargs(spec)
    kw["flags"] = rf.RF_HOST_ONLY | rf.RF_NOISE_CLIPPED
    with rf.Plan(**kw) as p:
        assert p.count_images(spec.nint) == 177521
    kw["flags"] = 0
    b0 = rf.rf_plan_estimate_bytes(rf.make_desc(**kw), wave_images=1024)
    kw["flags"] = rf.RF_NOISE_CLIPPED
    b1 = rf.rf_plan_estimate_bytes(rf.make_desc(**kw), wave_images=1024)
    # one clipping window (two floats) per image slot of a wave
    assert b1 - b0 == 1024 * 8


def test_plan_whose_column_overflows_shared_memory_is_rejected(L):
    # one north-south baseline: every channel lands in column u = 0, spread over
    # more than two thousand v cells at npix 8192 -- more than the column pass
    # can stage in a block's shared memory
    ant = np.array([[0.0, 0.0, 0.0], [0.0, 1000.0, 0.0]])
    f = np.linspace(1.0e9, 3.0e9, 2048)
    cell = 4000.0 * 299792458.0 / (1000.0 * 3.0e9 * 8192)
    kw = dict(ant_uvw=ant, freq_hz=f, inttime_s=5e-3, npix=8192, cell_rad=cell, dm_list=[0.0], dt_list=[1],
              threshold=6.0, flags=rf.RF_HOST_ONLY, max_nint=16)
    with pytest.raises(rf.RfError) as e:
        rf.rf_plan_create(rf.make_desc(**kw))
    assert e.value.status == rf.RF_ERR_INVALID_ARG
    assert "column" in rf.rf_last_error()
    # the same geometry with 64 channels fits
    kw["freq_hz"] = np.linspace(1.0e9, 3.0e9, 64)
    with rf.Plan(**kw) as p:
        assert p.info().n_cells > 0


def test_wide_index_tuning_key(L):
    kw = _desc_kwargs(synth.config("tiny"))
    with rf.Plan(**kw) as p:
        assert rf.rf_plan_get_tuning(p.handle, rf.RF_TUNE_WIDE_INDEX) == 0
        p.set_wide_index(True)
        assert rf.rf_plan_get_tuning(p.handle, rf.RF_TUNE_WIDE_INDEX) == 1
        with pytest.raises(rf.RfError) as e:
            rf.rf_plan_set_tuning(p.handle, rf.RF_TUNE_WIDE_INDEX, 2)
        assert e.value.status == rf.RF_ERR_INVALID_ARG


def test_fused_and_ring_tuning_keys(L):
    kw = _desc_kwargs(synth.config("tiny"))
    with rf.Plan(**kw) as p:
        assert rf.rf_plan_get_tuning(p.handle, rf.RF_TUNE_FUSED) == 0
        assert rf.rf_plan_get_tuning(p.handle, rf.RF_TUNE_RING) == 3
        p.set_fused(True)
        assert rf.rf_plan_get_tuning(p.handle, rf.RF_TUNE_FUSED) == 1
        for bad_key, bad in ((rf.RF_TUNE_FUSED, 2), (rf.RF_TUNE_RING, 1), (rf.RF_TUNE_RING, 9)):
            with pytest.raises(rf.RfError) as e:
                rf.rf_plan_set_tuning(p.handle, bad_key, bad)
            assert e.value.status == rf.RF_ERR_INVALID_ARG


def test_overlap_tuning_key(L):
    kw = _desc_kwargs(synth.config("tiny"))
    with rf.Plan(**kw) as p:
        assert rf.rf_plan_get_tuning(p.handle, rf.RF_TUNE_OVERLAP) == 0
        p.set_overlap(True)
        assert rf.rf_plan_get_tuning(p.handle, rf.RF_TUNE_OVERLAP) == 1
        p.set_overlap(False)
        assert rf.rf_plan_get_tuning(p.handle, rf.RF_TUNE_OVERLAP) == 0
        for bad in (2, -1):
            with pytest.raises(rf.RfError) as e:
                rf.rf_plan_set_tuning(p.handle, rf.RF_TUNE_OVERLAP, bad)
            assert e.value.status == rf.RF_ERR_INVALID_ARG


def test_noalloc_rejects_host_memory(L):
    # a host (numpy) buffer is not device memory of a current device: the call
    # rejects it before any launch (on a machine without a GPU as on one with)
    import numpy as np
    grid = np.zeros((256, 129), dtype=np.complex64)
    stat = np.zeros(rf.STAT_DTYPE.itemsize, dtype=np.uint8)
    with pytest.raises(rf.RfError) as e:
        rf.rf_image_stats_noalloc(grid, 256, 1.0, stat)
    assert e.value.status == rf.RF_ERR_INVALID_ARG
    assert "device memory" in e.value.message
