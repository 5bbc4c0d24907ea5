"""GPU stream search over overlapping segments (Sec. 3.2) against one search
over the whole run and against the oracle's stream."""

import numpy as np
import pytest

import oracle
import synth
import paper_1802_03084_gb300 as rf
from gpu_common import compare_candidates, compare_stats, oracle_images, plans_for

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


def _push_in_chunks(stream, vis, sizes, device_every=2):
    import torch
    t = 0
    k = 0
    while t < len(vis):
        n = min(sizes[k % len(sizes)], len(vis) - t)
        chunk = np.ascontiguousarray(vis[t:t + n])
        if k % device_every == 1:
            stream.push(torch.from_numpy(chunk).cuda(), n)
        else:
            stream.push(chunk, n)
        t += n
        k += 1
    stream.flush()


def _key(r):
    return (int(r["dm_idx"]), int(r["dt_idx"]), int(r["t_idx"]))


@pytest.mark.parametrize("edge,clipped", [("full", False), ("partial", False), ("full", True)])
def test_stream_equals_one_search_bit_for_bit(edge, clipped):
    spec = synth.config("tiny")
    spec.edge = edge
    spec.noise_clipped = clipped
    spec.dt_list = [1, 2, 4]
    seg = synth.make_segment(spec, nint=900)
    gp, _ = plans_for(spec, seg)
    with gp:
        gc1, gst1 = gp.search_stats(seg["vis"])
        with rf.Stream(gp, 64, keep_stats=True) as s:
            info = s.info()
            assert info["overlap"] == int(gp.delays().max())
            assert info["segment_nint"] == 64 + info["overlap"]
            _push_in_chunks(s, seg["vis"], [1, 37, 100, 5, 260])
            gst2 = s.pop_stats()
            gc2 = s.pop()
            assert s.info()["pending_stats"] == 0
    a = {_key(r): r for r in gst1}
    b = {_key(r): r for r in gst2}
    assert len(b) == len(gst2)            # each image once
    assert sorted(a) == sorted(b)
    for k, r in a.items():
        q = b[k]
        assert (int(r["x"]), int(r["y"])) == (int(q["x"]), int(q["y"])), k
        assert r["peak"] == q["peak"] and r["sigma"] == q["sigma"] and r["weight"] == q["weight"], k
    assert [_key(c) for c in gc1] == sorted(_key(c) for c in gc2)
    assert len(gc1) > 0


@pytest.mark.parametrize("mean_subtract", [False, True])
def test_stream_matches_oracle_stream(mean_subtract):
    spec = synth.config("tiny")
    spec.edge = "full"
    spec.dm_list = np.linspace(0.0, 300.0, 4)
    spec.mean_subtract = mean_subtract
    p = spec.pulses[0]
    spec.continuum = [dict(amp=6.0, x=(p["x"] + 70) % spec.npix, y=(p["y"] + 50) % spec.npix)]
    seg = synth.make_segment(spec, nint=420)
    gp, op = plans_for(spec, seg)
    stride = 96
    with gp:
        with rf.Stream(gp, stride, keep_stats=True) as s:
            _push_in_chunks(s, seg["vis"], [50, 200, 13])
            gst = s.pop_stats()
            gc = s.pop()
    oc, ost = oracle.search_stream(op, seg["vis"], stride, with_stats=True)
    assert sorted(_key(r) for r in gst) == sorted(ost)
    compare_stats(np.sort(gst, order=["dm_idx", "dt_idx", "t_idx"]), ost, _stream_images(op, seg, stride, gst, ost))
    gc = np.sort(gc, order=["dm_idx", "dt_idx", "t_idx"])
    compare_candidates(gc, oc, spec.threshold, ost)
    src = spec.continuum[0]
    at_src = np.mean([(int(r["x"]), int(r["y"])) == (src["x"], src["y"]) for r in gst])
    assert (at_src < 0.05) if mean_subtract else (at_src > 0.5)


def _stream_images(op, seg, stride, gst, ost):
    """FP64 images of the stream images whose peak pixel differs (ties)."""
    bad = [_key(r) for r in gst if (int(r["x"]), int(r["y"])) != (ost[_key(r)].x, ost[_key(r)].y)]
    if not bad:
        return None
    total = seg["vis"].shape[0]
    nseg = stride + oracle.stream_overlap(op)
    n_full = (total - nseg) // stride + 1 if total >= nseg else 0
    out = {}
    for (d, s, t) in bad:
        dt = int(op.dt_list[s])
        k = min(t * dt // stride, n_full)
        start = k * stride
        n = nseg if k < n_full else total - start
        S = op.stokes(seg["vis"][start:start + n], n)
        out[(d, s, t)] = op.image(S, d, s, t - start // dt, n)[0]
    return out


def test_stream_rejects_a_stride_that_is_not_a_multiple_of_dt_or_too_long():
    spec = synth.config("tiny")
    spec.dt_list = [1, 4]
    seg = synth.make_segment(spec, nint=600)
    gp, _ = plans_for(spec, seg)
    with gp:
        with pytest.raises(rf.RfError) as e:
            rf.Stream(gp, 6)
        assert e.value.status == rf.RF_ERR_INVALID_ARG
        with pytest.raises(rf.RfError):
            rf.Stream(gp, 600)          # stride + overlap > max_nint
