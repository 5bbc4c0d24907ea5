"""GPU parity of the clipped noise (RF_NOISE_CLIPPED) against the FP64 oracle.

With mu0 and sigma0 over all pixels, the noise is recomputed over the pixels
with |I - mu0| <= 5 sigma0.  Whether a pixel lying on that boundary within
rounding is kept is not fixed by the arithmetic, so such pixels are compared
both ways: the engine's sigma must lie between the oracle's sigma with all
of them dropped and with all of them kept (each kept boundary pixel raises
the variance, since its squared deviation is about 25 sigma0^2), and its mean
within one boundary pixel's weight of the oracle's.
"""

import numpy as np
import pytest

import oracle
import synth
import paper_1802_03084_gb300 as rf
from gpu_common import STAT_RTOL, compare_candidates, plans_for, small_random_segment

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


def _kept_stats(flat, keep):
    k = flat[keep]
    mu = k.mean()
    return mu, float(np.sqrt(np.mean((k - mu) ** 2))), int(keep.sum())


def compare_clipped(gst, op, vis, ost, rtol=STAT_RTOL, band=1e-4, nint=None):
    """Engine stats vs the oracle's clipped stats; returns the number of images
    in which the clipping dropped at least one pixel."""
    S = op.stokes(vis, nint or vis.shape[0])
    bad = []
    nclipped = 0
    for r in gst:
        key = (int(r["dm_idx"]), int(r["dt_idx"]), int(r["t_idx"]))
        o = ost[key]
        I, W = op.image(S, *key, nint=nint or vis.shape[0])
        flat = I.ravel()
        mu0 = flat.mean()
        s0 = float(np.sqrt(np.mean((flat - mu0) ** 2)))
        dist = np.abs(flat - mu0) - oracle.CLIP_SIGMA * s0
        sure = dist < -band * s0
        maybe = dist <= band * s0
        nclipped += int(maybe.sum() < flat.size)
        if (maybe != sure).any():
            _, s_lo, n_lo = _kept_stats(flat, sure)
            _, s_hi, _ = _kept_stats(flat, maybe)
            lo, hi = min(s_lo, s_hi), max(s_lo, s_hi)
            namb = int((maybe != sure).sum())
        else:
            lo = hi = o.sigma
            namb, n_lo = 0, int(sure.sum())
        g_sigma = float(r["sigma"])
        if not (lo * (1 - rtol) <= g_sigma <= hi * (1 + rtol)):
            bad.append(("sigma", key, g_sigma, lo, hi))
        mean_tol = rtol * o.sigma + namb * (oracle.CLIP_SIGMA + 1) * s0 / max(n_lo, 1)
        if abs(float(r["mean"]) - o.mean) > mean_tol:
            bad.append(("mean", key, float(r["mean"]), o.mean))
        if abs(r["peak"] - o.peak) > rtol * abs(o.peak) + 1e-7 * o.sigma:
            bad.append(("peak", key, float(r["peak"]), o.peak))
        if (int(r["x"]), int(r["y"])) != (o.x, o.y):
            if o.peak - I[int(r["y"]), int(r["x"])] > rtol * abs(o.peak):
                bad.append(("argmax", key, (int(r["x"]), int(r["y"])), (o.x, o.y)))
        g_snr = float(r["snr"])
        if abs(g_snr - o.snr) > 2 * rtol * abs(o.snr) + abs(o.peak) * (1 / max(lo, 1e-300) - 1 / max(hi, 1e-300)):
            bad.append(("snr", key, g_snr, o.snr))
    assert not bad, bad[:10]
    return nclipped


@pytest.fixture(scope="module")
def tiny_clip():
    spec = synth.config("tiny")
    seg = synth.make_segment(spec)
    flags = rf.RF_EDGE_PARTIAL | rf.RF_NOISE_CLIPPED
    gp, op = plans_for(spec, seg, flags=flags)
    cands, ost = oracle.search_segment(op, seg["vis"], with_stats=True)
    yield spec, seg, gp, op, cands, ost
    gp.close()


def test_tiny_clipped_every_image_and_candidates(tiny_clip):
    spec, seg, gp, op, ocands, ost = tiny_clip
    gc, gst = gp.search_stats(seg["vis"])
    assert len(gst) == 1024
    nclipped = compare_clipped(gst, op, seg["vis"], ost)
    assert nclipped > 0          # the pulse images lose their brightest pixels
    compare_candidates(gc, ocands, spec.threshold, ost)
    # against the plain noise of the same images: the pulse's S/N rises
    gp0, _ = plans_for(spec, seg, flags=rf.RF_EDGE_PARTIAL)
    with gp0:
        c0, s0 = gp0.search_stats(seg["vis"])
    # (clipping never raises sigma: the kept pixels' squared deviations from
    # mu0 sum to at most (N^2 - 25 n_dropped) sigma0^2), so no candidate of
    # the plain noise is lost
    i = int(np.argmax(gst["snr"]))
    assert gst["snr"][i] > s0["snr"][i] and gst["sigma"][i] < s0["sigma"][i]
    assert np.allclose(gst["peak"], s0["peak"], rtol=1e-6, atol=0)
    assert np.all(gst["sigma"] <= s0["sigma"] * (1 + 1e-5))
    kept = {(int(c["dm_idx"]), int(c["dt_idx"]), int(c["t_idx"])) for c in gc}
    for c in c0:
        if c["snr"] > spec.threshold * (1 + 1e-4):
            assert (int(c["dm_idx"]), int(c["dt_idx"]), int(c["t_idx"])) in kept


def test_clipped_search_deterministic_and_graph_equals_direct(tiny_clip):
    spec, seg, gp, op, _, _ = tiny_clip
    c1, s1 = gp.search_stats(seg["vis"])
    c2, s2 = gp.search_stats(seg["vis"])
    gp.set_graphs(False)
    c3, s3 = gp.search_stats(seg["vis"])
    gp.set_graphs(True)
    assert np.array_equal(s1, s2) and np.array_equal(s1, s3)
    assert np.array_equal(c1, c2) and np.array_equal(c1, c3)
    assert np.array_equal(gp.search(seg["vis"]), c1)


def test_clipped_plain_form(tiny_clip):
    spec, seg, _, op, ocands, ost = tiny_clip
    gp, _ = plans_for(spec, seg, flags=rf.RF_EDGE_PARTIAL | rf.RF_NOISE_CLIPPED)
    with gp:
        gp.set_form(rf.RF_FORM_PLAIN)
        gc, gst = gp.search_stats(seg["vis"])
        assert compare_clipped(gst, op, seg["vis"], ost) > 0
        compare_candidates(gc, ocands, spec.threshold, ost)


def test_clipped_fp16_storage(tiny_clip):
    spec, seg, _, op, ocands, ost = tiny_clip
    gp, _ = plans_for(spec, seg, flags=rf.RF_EDGE_PARTIAL | rf.RF_NOISE_CLIPPED | rf.RF_STORE_FP16)
    with gp:
        gc, gst = gp.search_stats(seg["vis"])
        compare_clipped(gst, op, seg["vis"], ost, rtol=1e-2, band=1e-2)
        compare_candidates(gc, ocands, spec.threshold, ost)


@pytest.mark.parametrize("case", [
    # npix, nant, nchan, nint, dt_list, partial, ndm
    (16, 4, 3, 9, [1, 2], False, 3),
    (64, 6, 12, 40, [1, 2, 4], True, 4),
    (256, 8, 9, 50, [1, 5], False, 3),
    (1024, 10, 4, 12, [1, 2], True, 2),   # tensor-copy tiles
    (2048, 6, 3, 6, [1], False, 2),       # transforms wider than a warp
])
def test_clipped_random_shapes(case):
    npix, nant, nchan, nint, dts, partial, ndm = case
    rng = np.random.default_rng(npix * 11 + nant)
    seg = small_random_segment(rng, nant, nchan, nint, npix)
    umax = 600.0 * seg["freq_hz"].max() / oracle.C_LIGHT
    spec = synth.SegmentSpec(name="rand", nchan=nchan, f_lo_hz=1e9, bw_hz=1e9, nint=nint, inttime_s=2e-3,
                             npix=npix, dm_list=np.linspace(0, 25.0, ndm), dt_list=dts, threshold=3.0,
                             nant=nant, cell_rad=0.47 / umax, edge="partial" if partial else "full")
    flags = (rf.RF_EDGE_PARTIAL if partial else 0) | rf.RF_NOISE_CLIPPED
    gp, op = plans_for(spec, seg, flags=flags)
    with gp:
        gc, gst = gp.search_stats(seg["vis"])
        oc, ost = oracle.search_segment(op, seg["vis"], with_stats=True)
        gst = gst[gst["weight"] > 0]
        assert len(gst) == len(ost)
        nclipped = compare_clipped(gst, op, seg["vis"], ost)
        if npix >= 64:
            assert nclipped > 0   # the bright source is clipped
        compare_candidates(gc, oc, spec.threshold, ost)
