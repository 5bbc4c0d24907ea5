"""GPU parity: the CUDA engine (through the C ABI) against the FP64 oracle."""

import numpy as np
import pytest

import oracle
import synth
import paper_1802_03084_gb300 as rf
from gpu_common import (IMG_RMS_FP16, IMG_RMS_FP32, compare_candidates, compare_stats, oracle_images,
                        plans_for, rel_rms, small_random_segment)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def engine():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1802_03084_gb300.build import build
    build()
    rf.lib()
    torch.cuda.init()
    yield


@pytest.fixture(scope="module")
def tiny():
    spec = synth.config("tiny")
    seg = synth.make_segment(spec)
    gp, op = plans_for(spec, seg)
    cands, ost = oracle.search_segment(op, seg["vis"], with_stats=True)
    yield spec, seg, gp, op, cands, ost
    gp.close()


def test_tiny_every_image_stat_and_candidates(tiny):
    spec, seg, gp, op, ocands, ost = tiny
    gc, gst = gp.search_stats(seg["vis"])
    assert len(gst) == 1024
    disagree = [(int(r["dm_idx"]), int(r["dt_idx"]), int(r["t_idx"])) for r in gst
                if (int(r["x"]), int(r["y"])) != (ost[(int(r["dm_idx"]), int(r["dt_idx"]), int(r["t_idx"]))].x,
                                                   ost[(int(r["dm_idx"]), int(r["dt_idx"]), int(r["t_idx"]))].y)]
    oim = oracle_images(op, seg["vis"], disagree) if disagree else None
    compare_stats(gst, ost, oim)
    compare_candidates(gc, ocands, spec.threshold, ost)
    assert len(gc) > 0
    # the injected pulse: DM 300 trial, its time, its pixel
    best = gc[np.argmax(gc["snr"])]
    p = spec.pulses[0]
    assert int(best["dm_idx"]) == int(np.argmin(np.abs(spec.dm_list - p["dm"])))
    assert abs(int(best["t_idx"]) - p["t0_s"] / spec.inttime_s) <= 1
    assert (int(best["x"]), int(best["y"])) == (p["x"], p["y"])


def test_tiny_images_elementwise(tiny):
    spec, seg, gp, op, _, _ = tiny
    trials = [(0, 0, 0), (3, 0, 27), (3, 0, 28), (7, 0, 127), (5, 0, 64), (1, 0, 100)]
    g = gp.render(seg["vis"], trials)
    o = oracle_images(op, seg["vis"], trials)
    for k, tr in enumerate(trials):
        assert rel_rms(g[k], o[tr]) < IMG_RMS_FP32, tr


def test_search_matches_stats_candidates_and_is_deterministic(tiny):
    spec, seg, gp, op, _, _ = tiny
    c1 = gp.search(seg["vis"])
    c2, s2 = gp.search_stats(seg["vis"])
    c3, s3 = gp.search_stats(seg["vis"])
    assert np.array_equal(c1, c2) and np.array_equal(c2, c3)
    assert np.array_equal(s2, s3)


def test_host_and_device_inputs_agree(tiny):
    import torch
    spec, seg, gp, op, _, _ = tiny
    dev = torch.from_numpy(seg["vis"]).cuda()
    pinned = torch.from_numpy(seg["vis"]).pin_memory()
    _, sa = gp.search_stats(seg["vis"])
    _, sb = gp.search_stats(dev)
    _, sc = gp.search_stats(pinned)
    assert np.array_equal(sa, sb) and np.array_equal(sa, sc)


def test_full_edge_rule_counts_and_parity():
    spec = synth.config("tiny")
    spec.edge = "full"
    seg = synth.make_segment(spec)
    gp, op = plans_for(spec, seg)
    with gp:
        gc, gst = gp.search_stats(seg["vis"])
        oc, ost = oracle.search_segment(op, seg["vis"], with_stats=True)
        assert len(gst) == 201
        compare_stats(gst, ost, oracle_images(op, seg["vis"], list(ost)))
        compare_candidates(gc, oc, spec.threshold, ost)
        # a segment shorter than every sweep but DM 0 searches only DM 0
        n = gp.count_images(40)
        _, s40 = gp.search_stats(seg["vis"][:40].copy())
        assert len(s40) == n == 40
        with pytest.raises(rf.RfError) as e:
            gp.search(np.zeros((129, 351, 64, 2), np.complex64))
        assert e.value.status == rf.RF_ERR_SHAPE


@pytest.mark.parametrize("case", [
    # npix, nant, nchan, nint, dt_list, partial, ndm
    (16, 4, 3, 9, [1, 2], False, 3),
    (32, 5, 7, 23, [1, 3], True, 4),
    (64, 6, 12, 40, [1, 2, 4], False, 5),
    (128, 7, 5, 31, [3], True, 3),
    (256, 8, 9, 50, [1, 5], False, 4),
    (512, 9, 6, 19, [1, 2], True, 3),
    # tensor-copy tiles in the row pass (N >= 1024): 128- and 64-byte swizzles, two and more boxes
    (1024, 10, 4, 12, [1, 2], True, 3),
    (2048, 6, 3, 6, [1], False, 2),
])
def test_random_shapes(case):
    npix, nant, nchan, nint, dts, partial, ndm = case
    rng = np.random.default_rng(npix * 7 + nant)
    seg = small_random_segment(rng, nant, nchan, nint, npix)
    # cell so that the longest baselines at the top channel fall just off the grid
    umax = 600.0 * seg["freq_hz"].max() / oracle.C_LIGHT
    cell = 0.47 / umax
    spec = synth.SegmentSpec(name="rand", nchan=nchan, f_lo_hz=1e9, bw_hz=1e9, nint=nint, inttime_s=2e-3,
                             npix=npix, dm_list=np.linspace(0, 25.0, ndm), dt_list=dts, threshold=3.0,
                             nant=nant, cell_rad=cell, edge="partial" if partial else "full")
    gp, op = plans_for(spec, seg)
    with gp:
        gc, gst = gp.search_stats(seg["vis"])
        oc, ost = oracle.search_segment(op, seg["vis"], with_stats=True)
        ok = {k: v for k, v in ost.items()}
        gst = gst[gst["weight"] > 0]
        assert len(gst) == len(ok)
        compare_stats(gst, ok, oracle_images(op, seg["vis"], list(ok)))
        compare_candidates(gc, oc, spec.threshold, ok)
        keys = list(ok)[:: max(1, len(ok) // 6)]
        g = gp.render(seg["vis"], keys)
        o = oracle_images(op, seg["vis"], keys)
        for i, k in enumerate(keys):
            assert rel_rms(g[i], o[k]) < IMG_RMS_FP32, (case, k)


@pytest.mark.parametrize("npix,width", [(2048, "wide"), (2048, "narrow"), (1024, "wide")])
def test_row_transform_edge_columns(npix, width):
    """The row transform's inputs at the edges of the half-plane grid.

    "wide": the cell is set so that the longest baseline at the top channel
    lands on the last on-grid column, |iu| = N/2 - 1, whose Hermitian mirror
    is the row input next to the middle (at N = 2048 the split transform's
    odd-pixel half reads it at u' = 1).  "narrow": a few dozen columns, so
    most row inputs are zero.  Every image's statistics and candidates, and
    a few rendered images, against the oracle.
    """
    rng = np.random.default_rng(4242 + npix + len(width))
    nant, nchan, nint = 12, 6, 6
    seg = small_random_segment(rng, nant, nchan, nint, npix)
    seg["ant_uvw"][:, 1] *= 0.25                 # east-west: |v| well below |u|
    bl = oracle.baseline_uvw(seg["ant_uvw"])
    s_top = seg["freq_hz"].max() / oracle.C_LIGHT
    k = int(np.argmax(np.abs(bl[:, 0])))
    target = npix // 2 - 1 if width == "wide" else 24
    cell = target / (abs(bl[k, 0]) * s_top * npix)
    spec = synth.SegmentSpec(name="edge", nchan=nchan, f_lo_hz=1e9, bw_hz=1e9, nint=nint, inttime_s=2e-3,
                             npix=npix, dm_list=np.linspace(0, 20.0, 2), dt_list=[1, 2], threshold=3.0,
                             nant=nant, cell_rad=cell, edge="partial")
    gp, op = plans_for(spec, seg)
    iu_max = int(np.abs(op.iu[op.ongrid]).max())
    assert iu_max == target, (iu_max, target)
    with gp:
        gc, gst = gp.search_stats(seg["vis"])
        oc, ost = oracle.search_segment(op, seg["vis"], with_stats=True)
        ok = {k: v for k, v in ost.items()}
        gst = gst[gst["weight"] > 0]
        assert len(gst) == len(ok)
        compare_stats(gst, ok, oracle_images(op, seg["vis"], list(ok)))
        compare_candidates(gc, oc, spec.threshold, ok)
        keys = list(ok)[:: max(1, len(ok) // 4)]
        g = gp.render(seg["vis"], keys)
        o = oracle_images(op, seg["vis"], keys)
        for i, key in enumerate(keys):
            assert rel_rms(g[i], o[key]) < IMG_RMS_FP32, (npix, width, key)


def test_fp16_storage_precision(tiny):
    spec, seg, _, op, ocands, ost = tiny
    spec16 = synth.config("tiny")
    spec16.store = "fp16"
    gp, _ = plans_for(spec16, seg)
    with gp:
        trials = [(3, 0, 27), (0, 0, 5), (7, 0, 120)]
        g = gp.render(seg["vis"], trials)
        o = oracle_images(op, seg["vis"], trials)
        errs = [rel_rms(g[k], o[t]) for k, t in enumerate(trials)]
        assert max(errs) < IMG_RMS_FP16, errs
        gc, gst = gp.search_stats(seg["vis"])
        oim = oracle_images(op, seg["vis"], [(int(r["dm_idx"]), int(r["dt_idx"]), int(r["t_idx"]))
                                              for r in gst if (int(r["x"]), int(r["y"])) !=
                                              (ost[(int(r["dm_idx"]), int(r["dt_idx"]), int(r["t_idx"]))].x,
                                               ost[(int(r["dm_idx"]), int(r["dt_idx"]), int(r["t_idx"]))].y)])
        compare_stats(gst, ost, oim, rtol=1e-2)
        compare_candidates(gc, ocands, spec.threshold, ost)


def test_single_channel_single_integration():
    rng = np.random.default_rng(3)
    seg = small_random_segment(rng, 5, 1, 1, 64)
    spec = synth.SegmentSpec(name="one", nchan=1, f_lo_hz=1.4e9, bw_hz=1e6, nint=1, inttime_s=1e-3, npix=64,
                             dm_list=np.array([0.0, 10.0]), dt_list=[1], threshold=2.0, nant=5,
                             cell_rad=0.3 / (600 * 1.4e9 / oracle.C_LIGHT))
    gp, op = plans_for(spec, seg)
    with gp:
        gc, gst = gp.search_stats(seg["vis"])
        oc, ost = oracle.search_segment(op, seg["vis"], with_stats=True)
        compare_stats(gst, ost, oracle_images(op, seg["vis"], list(ost)))
        compare_candidates(gc, oc, spec.threshold, ost)


def _disagreeing(gst, ost):
    return [(int(r["dm_idx"]), int(r["dt_idx"]), int(r["t_idx"])) for r in gst
            if (int(r["x"]), int(r["y"])) != (ost[(int(r["dm_idx"]), int(r["dt_idx"]), int(r["t_idx"]))].x,
                                               ost[(int(r["dm_idx"]), int(r["dt_idx"]), int(r["t_idx"]))].y)]


def test_plain_form_matches_oracle(tiny):
    spec, seg, _, op, ocands, ost = tiny
    gp, _ = plans_for(spec, seg)
    with gp:
        gp.set_form(rf.RF_FORM_PLAIN)
        gc, gst = gp.search_stats(seg["vis"])
        dis = _disagreeing(gst, ost)
        compare_stats(gst, ost, oracle_images(op, seg["vis"], dis) if dis else None)
        compare_candidates(gc, ocands, spec.threshold, ost)


def test_plain_form_random_shape():
    rng = np.random.default_rng(77)
    seg = small_random_segment(rng, 7, 9, 37, 128)
    umax = 600.0 * seg["freq_hz"].max() / oracle.C_LIGHT
    spec = synth.SegmentSpec(name="rand", nchan=9, f_lo_hz=1e9, bw_hz=1e9, nint=37, inttime_s=2e-3, npix=128,
                             dm_list=np.linspace(0, 30.0, 4), dt_list=[1, 3], threshold=3.0, nant=7,
                             cell_rad=0.45 / umax, edge="partial")
    gp, op = plans_for(spec, seg)
    with gp:
        gp.set_form(rf.RF_FORM_PLAIN)
        gc, gst = gp.search_stats(seg["vis"])
        oc, ost = oracle.search_segment(op, seg["vis"], with_stats=True)
        gst = gst[gst["weight"] > 0]
        compare_stats(gst, ost, oracle_images(op, seg["vis"], list(ost)))
        compare_candidates(gc, oc, spec.threshold, ost)


def test_graph_replay_equals_direct_launches(tiny):
    spec, seg, _, op, _, _ = tiny
    gp, _ = plans_for(spec, seg)
    with gp:
        c_graph, s_graph = gp.search_stats(seg["vis"])
        c_graph2, s_graph2 = gp.search_stats(seg["vis"])        # replay
        _, s_short = gp.search_stats(seg["vis"][:64].copy())     # new image list: re-captured
        c_graph3, s_graph3 = gp.search_stats(seg["vis"])
        gp.set_graphs(False)
        c_direct, s_direct = gp.search_stats(seg["vis"])
        for s_ in (s_graph2, s_graph3, s_direct):
            assert np.array_equal(s_graph, s_)
        for c_ in (c_graph2, c_graph3, c_direct):
            assert np.array_equal(c_graph, c_)
        assert len(s_short) == 8 * 64


def test_autotune_keeps_results(tiny, tmp_path):
    spec, seg, _, op, _, _ = tiny
    gp, _ = plans_for(spec, seg)
    with gp:
        c0, s0 = gp.search_stats(seg["vis"])
        cache = str(tmp_path / "tune.json")
        res = gp.autotune(seg["vis"], cache_path=cache)
        assert res["cached"] is False and res["wave_images"] >= 32 and len(res["tried"]) >= 2
        c1, s1 = gp.search_stats(seg["vis"])
        assert np.array_equal(s0, s1) and np.array_equal(c0, c1)
        again = gp.autotune(seg["vis"], cache_path=cache)
        assert again["cached"] is True and again["wave_images"] == res["wave_images"]


def test_maximum_image_size():
    # npix 8192: one transform per block in the column pass, row-pass tiles of
    # one 16-byte chunk per column in several tensor-copy boxes
    rng = np.random.default_rng(8192)
    seg = small_random_segment(rng, 5, 2, 2, 8192)
    umax = 600.0 * seg["freq_hz"].max() / oracle.C_LIGHT
    spec = synth.SegmentSpec(name="max", nchan=2, f_lo_hz=1e9, bw_hz=1e9, nint=2, inttime_s=2e-3, npix=8192,
                             dm_list=np.array([0.0]), dt_list=[1], threshold=3.0, nant=5, cell_rad=0.47 / umax,
                             edge="full")
    gp, op = plans_for(spec, seg)
    with gp:
        assert gp.info().iu_max > 1024          # many columns: several tensor-copy boxes
        gc, gst = gp.search_stats(seg["vis"])
        oc, ost = oracle.search_segment(op, seg["vis"], with_stats=True)
        assert len(gst) == len(ost) == 2
        oim = oracle_images(op, seg["vis"], list(ost))
        compare_stats(gst, ost, oim)
        compare_candidates(gc, oc, spec.threshold, ost)
        g = gp.render(seg["vis"], [(0, 0, 1)])
        assert rel_rms(g[0], oim[(0, 0, 1)]) < IMG_RMS_FP32


@pytest.mark.parametrize("edge,store", [("partial", "fp32"), ("full", "fp16")])
def test_wide_sample_offsets_give_the_same_images(tiny, edge, store):
    # the gridding kernel's 64-bit offset variant (for series of 2^32 samples
    # and more) on a small plan: bit-identical to the 32-bit one
    spec, seg, _, _, _, _ = tiny
    s2 = synth.config("tiny")
    s2.edge = edge
    s2.store = store
    gp, _ = plans_for(s2, seg)
    with gp:
        gp.set_graphs(False)
        c0, s0 = gp.search_stats(seg["vis"])
        gp.set_wide_index(True)
        assert rf.rf_plan_get_tuning(gp.handle, rf.RF_TUNE_WIDE_INDEX) == 1
        c1, s1 = gp.search_stats(seg["vis"])
        assert np.array_equal(s0, s1) and np.array_equal(c0, c1)


def test_registered_and_misaligned_pinned_host_inputs(tiny):
    # page-locked memory registered by cudaHostRegister is read in place by the
    # ingest kernel; a pinned buffer that starts off a 16-byte boundary goes
    # through the staging copies; both give the device input's results bit for bit
    import torch
    spec, seg, gp, op, _, _ = tiny
    c_dev, s_dev = gp.search_stats(torch.from_numpy(seg["vis"]).cuda())
    arr = np.ascontiguousarray(seg["vis"]).copy()
    cudart = torch.cuda.cudart()
    if hasattr(cudart, "cudaHostRegister"):
        ptr = arr.ctypes.data
        assert int(cudart.cudaHostRegister(ptr, arr.nbytes, 0)) == 0
        try:
            c_reg, s_reg = gp.search_stats(arr)
        finally:
            cudart.cudaHostUnregister(ptr)
        assert np.array_equal(s_reg, s_dev) and np.array_equal(c_reg, c_dev)
    big = torch.empty(arr.size + 1, dtype=torch.complex64).pin_memory()
    off = big[1:].view(arr.shape)            # 8 bytes past the pinned allocation's start
    off.copy_(torch.from_numpy(arr))
    assert off.data_ptr() % 16 == 8
    c_off, s_off = gp.search_stats(off)
    assert np.array_equal(s_off, s_dev) and np.array_equal(c_off, c_dev)
