"""The fused column + row pass (npix 1024 .. 4096) against the separate
column and row launches.

Both paths run the same column transforms (gathered from the staged cells,
split R = npix / 1024 ways for npix >= 2048) and the same row transforms in
the same order, so every image's statistics and every candidate must agree
bit for bit.  Covered: the three fused sizes, groups whose image count is not
a multiple of the chunk, waves of a few chunks and of many, ring depths 2 and
3, FP16 storage and the PARTIAL edge rule, graph capture and replay; and a
few images of each size against the FP64 oracle.
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
    spec = synth.SegmentSpec(name=f"fused-{npix}", nchan=nchan, f_lo_hz=1.0e9, bw_hz=1.0e9, nint=nint,
                             inttime_s=5e-3, npix=npix, dm_list=synth.dm_grid_linear(240.0, 5), dt_list=[1, 2, 3],
                             threshold=6.0, seed=900 + npix // 1024, store=store, edge=edge)
    spec.pulses = [dict(dm=120.0, t0_s=0.12, width_s=10e-3, amp=0.9, x=npix // 2 + 17, y=npix // 2 - 29)]
    return spec


def _stats(gp, vis, fused, wave=None, ring=None):
    gp.set_fused(fused)
    if wave:
        gp.set_wave_images(wave)
    if ring:
        gp.set_ring(ring)
    c, st = gp.search_stats(vis)
    c2 = gp.search(vis)       # graph capture
    c3 = gp.search(vis)       # and replay
    assert np.array_equal(c, c2) and np.array_equal(c, c3)
    return c, st


@pytest.mark.parametrize("npix,store,edge", [(1024, "fp32", "full"), (2048, "fp16", "partial"),
                                             (4096, "fp32", "partial")])
def test_fused_equals_separate_launches(npix, store, edge):
    import torch
    spec = _spec(npix, store, edge)
    seg = synth.make_segment(spec)
    gp, op = plans_for(spec, seg)
    vis = torch.from_numpy(seg["vis"]).cuda()
    with gp:
        c0, s0 = _stats(gp, vis, False)
        for wave, ring in ((None, None), (64, 2), (32, 3), (4096, 2)):
            c1, s1 = _stats(gp, vis, True, wave, ring)
            assert s0.tobytes() == s1.tobytes(), (npix, wave, ring)
            assert np.array_equal(c0, c1), (npix, wave, ring)
        assert len(c0) > 0
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
