"""The full `realtime` segment (177,521 images of 1024^2) in the launch
configuration the benchmark times (waves of 8192 images under a CUDA graph),
checked against the FP64 oracle on sampled images computed one by one, and by
properties that hold at any size (image count, order, graph replay)."""

import numpy as np
import pytest

import oracle
import synth
import paper_1802_03084_gb300 as rf
from gpu_common import SNR_GUARD, compare_stats, plans_for

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


def _key(r):
    return (int(r["dm_idx"]), int(r["dt_idx"]), int(r["t_idx"]))


def test_realtime_full_segment_sampled_against_oracle():
    import torch
    spec = synth.config("realtime")
    seg = synth.make_segment(spec)
    gp, op = plans_for(spec, seg)
    with gp:
        gp.set_wave_images(8192)
        vis = torch.from_numpy(seg["vis"]).cuda()
        gc, gst = gp.search_stats(vis)
        gc2 = gp.search(vis)                      # captures the search's graph
        gc3 = gp.search(vis)                      # and replays it
    assert len(gst) == len(op.image_list(spec.nint)) == 177521
    assert np.array_equal(gc, gc2) and np.array_equal(gc, gc3)
    keys = [_key(r) for r in gc]
    assert keys == sorted(keys) and len(gc) > 0
    # sampled images: uniformly drawn, plus the brightest and images near the threshold
    rng = np.random.default_rng(7)
    pick = set(rng.choice(len(gst), 12, replace=False).tolist())
    pick |= set(np.argsort(-gst["snr"])[:3].tolist())
    near = np.where(np.abs(gst["snr"] - spec.threshold) < 0.5)[0]
    pick |= set(near[:: max(1, len(near) // 3)][:3].tolist())
    idx = np.array(sorted(pick))
    S = op.stokes(seg["vis"], spec.nint)
    ost, oim = {}, {}
    for i in idx:
        k = _key(gst[i])
        I, W = op.image(S, *k, nint=spec.nint)
        ost[k] = oracle.image_stats(I)
        oim[k] = I
    compare_stats(gst[idx], ost, oim)
    cand = {_key(c): c for c in gc}
    for k, o in ost.items():
        if o.snr >= spec.threshold + SNR_GUARD:
            assert k in cand and (int(cand[k]["x"]), int(cand[k]["y"])) == (o.x, o.y), k
        elif o.snr < spec.threshold - SNR_GUARD:
            assert k not in cand, k
