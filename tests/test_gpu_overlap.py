"""Overlapped waves (RF_TUNE_OVERLAP) against one wave after another.

With overlap on, waves take alternate halves of the column-FFT scratch and a
wave's row pass and finalize run on the plan's second stream beside the next
wave's column pass.  Every image goes through the same column and row
transforms, and the finalizes run in wave order, so every image's statistics
and the candidate list must agree bit for bit with the serial order.
Covered: sizes with and without tensor-copy tiles (256, 1024, 2048 with the
split row transform), FP16 storage and the PARTIAL edge rule, waves of one
group and of many, an odd number of waves, graph capture and replay, direct
launches, profiling events on both streams, and switching back and forth on
one plan; and a few images of each size against the FP64 oracle.
"""

import numpy as np
import pytest

import oracle
import synth
import paper_1802_03084_gb300 as rf
from gpu_common import STAT_RTOL, compare_stats, plans_for

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


def _spec(npix, store="fp32", edge="full", nchan=24, nint=112):
    spec = synth.SegmentSpec(name=f"overlap-{npix}", nchan=nchan, f_lo_hz=1.0e9, bw_hz=1.0e9, nint=nint,
                             inttime_s=5e-3, npix=npix, dm_list=synth.dm_grid_linear(240.0, 5), dt_list=[1, 2, 3],
                             threshold=6.0, seed=700 + npix // 256, store=store, edge=edge)
    spec.pulses = [dict(dm=120.0, t0_s=0.12, width_s=10e-3, amp=0.9, x=npix // 2 + npix // 16,
                        y=npix // 2 - npix // 32)]
    return spec


def _run(gp, vis, overlap, graphs=True):
    gp.set_overlap(overlap)
    gp.set_graphs(graphs)
    c, st = gp.search_stats(vis)
    c2 = gp.search(vis)       # graph capture (or direct launches)
    c3 = gp.search(vis)       # and replay
    assert np.array_equal(c, c2) and np.array_equal(c, c3)
    return c, st


@pytest.mark.parametrize("npix,store,edge", [(256, "fp32", "full"), (1024, "fp32", "partial"),
                                             (2048, "fp16", "partial")])
def test_overlap_equals_serial_waves(npix, store, edge):
    import torch
    spec = _spec(npix, store, edge)
    seg = synth.make_segment(spec)
    gp, op = plans_for(spec, seg)
    vis = torch.from_numpy(seg["vis"]).cuda()
    B = gp.info().images_per_group
    n = gp.count_images(spec.nint)
    with gp:
        c0, s0 = _run(gp, vis, False)
        assert len(c0) > 0
        # waves of one group, of three groups (an odd count of waves), of many
        for wave in (2 * B, 6 * B, 1024):
            gp.set_wave_images(wave)
            for graphs in (True, False):
                c1, s1 = _run(gp, vis, True, graphs)
                assert s0.tobytes() == s1.tobytes(), (npix, wave, graphs)
                assert np.array_equal(c0, c1), (npix, wave, graphs)
            if wave >= n:
                break
        # profiling events on both streams; then back to serial waves on the same plan
        gp.set_wave_images(2 * B)
        gp.set_overlap(True)
        gp.set_profiling(True)
        c1, s1 = gp.search_stats(vis)
        prof = gp.profile()
        gp.set_profiling(False)
        assert s0.tobytes() == s1.tobytes() and np.array_equal(c0, c1)
        assert prof["rowfft_stats"][0] > 0 and prof["grid_colfft"][0] > 0
        c2, s2 = _run(gp, vis, False)
        assert s0.tobytes() == s2.tobytes() and np.array_equal(c0, c2)
        # a few images against the FP64 oracle
        keys = [(int(r["dm_idx"]), int(r["dt_idx"]), int(r["t_idx"])) for r in s1]
        rng = np.random.default_rng(npix)
        pick = sorted(set(rng.choice(len(keys), 3, replace=False).tolist()) | {int(np.argmax(s1["snr"]))})
        S = op.stokes(seg["vis"])
        ost, oim = {}, {}
        for i in pick:
            I, W = op.image(S, *keys[i], nint=spec.nint)
            ost[keys[i]] = oracle.image_stats(I)
            oim[keys[i]] = I
        rtol = 1e-2 if store == "fp16" else STAT_RTOL
        compare_stats(s1[pick], ost, oim, rtol=rtol)


def test_autotuner_times_overlap():
    import torch
    spec = _spec(256, nint=512)
    seg = synth.make_segment(spec)
    gp, _ = plans_for(spec, seg)
    vis = torch.from_numpy(seg["vis"]).cuda()
    with gp:
        c0, s0 = _run(gp, vis, False)
        res = gp.autotune(vis)
        tried = res["tried"]
        assert all(len(t) == 6 for t in tried)
        assert any(t[4] == 1 for t in tried) and any(t[4] == 0 for t in tried)
        assert res["overlap"] == rf.rf_plan_get_tuning(gp.handle, rf.RF_TUNE_OVERLAP)
        c1, s1 = gp.search_stats(vis)
        assert s0.tobytes() == s1.tobytes() and np.array_equal(c0, c1)
