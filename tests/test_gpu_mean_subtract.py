"""GPU parity of mean-visibility subtraction (Sec. 3.1) against the FP64 oracle."""

import numpy as np
import pytest

import oracle
import synth
import paper_1802_03084_gb300 as rf
from gpu_common import (IMG_RMS_FP16, IMG_RMS_FP32, compare_candidates, compare_stats, oracle_images,
                        plans_for, rel_rms)

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


def _spec_with_continuum(store="fp32", edge="full", amp=20.0):
    spec = synth.config("tiny")
    spec.store = store
    spec.edge = edge
    spec.mean_subtract = True
    # a bright steady source well away from the pulse's pixel
    p = spec.pulses[0]
    spec.continuum = [dict(amp=amp, x=(p["x"] + spec.npix // 3) % spec.npix, y=(p["y"] + spec.npix // 4) % spec.npix)]
    return spec


def _disagreeing(gst, ost):
    return [(int(r["dm_idx"]), int(r["dt_idx"]), int(r["t_idx"])) for r in gst
            if (int(r["x"]), int(r["y"])) != (ost[(int(r["dm_idx"]), int(r["dt_idx"]), int(r["t_idx"]))].x,
                                               ost[(int(r["dm_idx"]), int(r["dt_idx"]), int(r["t_idx"]))].y)]


@pytest.mark.parametrize("store,edge", [("fp32", "full"), ("fp32", "partial"), ("fp16", "full")])
def test_mean_subtract_every_image_matches_oracle(store, edge):
    spec = _spec_with_continuum(store, edge)
    seg = synth.make_segment(spec)
    gp, op = plans_for(spec, seg)
    assert op.mean_subtract
    with gp:
        oc, ost = oracle.search_segment(op, seg["vis"], with_stats=True)
        gc, gst = gp.search_stats(seg["vis"])
        assert len(gst) == len(ost) == op.count_images(seg["vis"].shape[0])
        bad = _disagreeing(gst, ost)
        compare_stats(gst, ost, oracle_images(op, seg["vis"], bad) if bad else None,
                      rtol=1e-4 if store == "fp32" else 1e-2)
        compare_candidates(gc, oc, spec.threshold, ost)
        # the steady source is gone: the brightest candidate is the pulse
        best = gc[np.argmax(gc["snr"])]
        p = spec.pulses[0]
        assert (int(best["x"]), int(best["y"])) == (p["x"], p["y"])
        src = spec.continuum[0]
        assert not any((int(c["x"]), int(c["y"])) == (src["x"], src["y"]) for c in gc)
        trials = [(0, 0, 0), (3, 0, 27), (7, 0, 64)]
        trials = [t for t in trials if t in ost]
        g = gp.render(seg["vis"], trials)
        o = oracle_images(op, seg["vis"], trials)
        tol = IMG_RMS_FP32 if store == "fp32" else IMG_RMS_FP16
        errs = [rel_rms(g[k], o[t]) for k, t in enumerate(trials)]
        assert max(errs) < tol, errs


def test_without_the_flag_the_steady_source_dominates():
    spec = _spec_with_continuum()
    seg = synth.make_segment(spec)
    spec.mean_subtract = False
    gp, op = plans_for(spec, seg)
    assert not op.mean_subtract
    with gp:
        gc, gst = gp.search_stats(seg["vis"])
        src = spec.continuum[0]
        at_src = np.mean([(int(r["x"]), int(r["y"])) == (src["x"], src["y"]) for r in gst])
        assert at_src > 0.9
        _, ost = oracle.search_segment(op, seg["vis"], with_stats=True)
        bad = _disagreeing(gst, ost)
        compare_stats(gst, ost, oracle_images(op, seg["vis"], bad) if bad else None)


def test_mean_subtract_host_chunks_equal_one_device_ingest():
    # 800 integrations of 351 baselines x 64 channels x 2 pols are 288 MB:
    # from host memory they arrive in two staging chunks (two ingest
    # launches), from device memory in one; the mean is taken once over the
    # whole segment either way.
    import torch
    spec = _spec_with_continuum()
    seg = synth.make_segment(spec, nint=800)
    assert seg["vis"].nbytes > 256 * 2 ** 20
    gp, _ = plans_for(spec, seg)
    with gp:
        gc1, gst1 = gp.search_stats(seg["vis"])
        gc2, gst2 = gp.search_stats(torch.from_numpy(seg["vis"]).cuda())
        np.testing.assert_array_equal(gst1, gst2)
        np.testing.assert_array_equal(gc1, gc2)
        assert len(gst1) == gp.count_images(800)
