"""Precision of the engine's images and statistics against the FP64 oracle.

Storage is FP16 or FP32; dedispersion sums, gridding and FFTs are FP32 and
the noise reduction is FP64 (Parseval's identity over the grid).  For sampled
images of two large workloads the relative RMS image error, the peak error in
units of the image sigma and the S/N error are measured and bounded:

* 2048^2 images, 1024 channels, 256 DM trials, dt 1..16 (the batching
  workload), first 64 integrations around its first pulse, PARTIAL edge rule;
* 4096^2 images, 2048 channels over 1-3 GHz, 512 DM trials, dt 1..32 with a
  continuum source at 100 times the per-visibility noise (the stress
  workload), first 64 integrations, PARTIAL edge rule.

Run with ``-s`` to print the measured errors.
"""

import numpy as np
import pytest

import oracle
import synth
import paper_1802_03084_gb300 as rf
from gpu_common import IMG_RMS_FP16, IMG_RMS_FP32, SNR_GUARD, STAT_RTOL, plans_for, rel_rms

pytestmark = pytest.mark.gpu

NINT = 64


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


def _window(name):
    spec = synth.config(name)
    spec.edge = "partial"
    p = spec.pulses[0]
    t_pulse = int(p["t0_s"] / spec.inttime_s)
    t_start = max(0, t_pulse - 8)
    seg = synth.make_segment(spec, nint=NINT, t_start=t_start)
    d_pulse = int(np.argmin(np.abs(np.asarray(spec.dm_list) - p["dm"])))
    ndm = len(spec.dm_list)
    trials = [(0, 0, 0), (d_pulse, 0, t_pulse - t_start), (ndm // 2, 2, 3), (ndm - 1, len(spec.dt_list) - 1, 1)]
    return spec, seg, trials


@pytest.fixture(scope="module", params=["batching", "stress"])
def workload(request):
    spec, seg, trials = _window(request.param)
    op = oracle.OraclePlan(seg["ant_uvw"], seg["freq_hz"], spec.inttime_s, spec.npix, spec.cell_rad,
                           spec.dm_list, spec.dt_list, spec.threshold, edge="partial", npol=spec.npol)
    S = op.stokes(seg["vis"], NINT)
    oim = {k: op.image(S, *k, nint=NINT)[0] for k in trials}
    ost = {k: oracle.image_stats(I) for k, I in oim.items()}
    return request.param, spec, seg, trials, oim, ost


@pytest.mark.parametrize("store", ["fp16", "fp32"])
def test_image_and_snr_error_vs_fp64(workload, store):
    name, spec, seg, trials, oim, ost = workload
    flags = rf.RF_EDGE_PARTIAL | (rf.RF_STORE_FP16 if store == "fp16" else 0)
    gp, _ = plans_for(spec, seg, flags=flags, max_nint=NINT)
    with gp:
        g = gp.render(seg["vis"], trials)
        _, gst = gp.search_stats(seg["vis"])
    assert len(gst) == gp_count(spec, NINT)
    by_key = {(int(r["dm_idx"]), int(r["dt_idx"]), int(r["t_idx"])): r for r in gst}
    img_err, peak_err, snr_err = [], [], []
    for k, key in enumerate(trials):
        o = ost[key]
        img_err.append(rel_rms(g[k], oim[key]))
        r = by_key[key]
        peak_err.append(abs(float(r["peak"]) - o.peak) / o.sigma)
        snr_err.append(abs(float(r["snr"]) - o.snr))
        # the engine's peak pixel is a maximum of the FP64 image within its error
        v = oim[key][int(r["y"]), int(r["x"])]
        assert o.peak - v <= 4 * peak_err[-1] * o.sigma + 1e-6 * o.sigma, (key, o.peak, v)
    print(f"\nprecision {name} {spec.npix}^2 store={store}: image rel RMS max {max(img_err):.2e}, "
          f"|d peak|/sigma max {max(peak_err):.2e}, |d snr| max {max(snr_err):.2e}, "
          f"snr of sampled images {[round(ost[k].snr, 2) for k in trials]}")
    tol = IMG_RMS_FP16 if store == "fp16" else IMG_RMS_FP32
    assert max(img_err) < tol, img_err
    # near the threshold the S/N must agree to the guard band; bright images
    # to the storage precision's relative tolerance
    rtol = 1e-2 if store == "fp16" else STAT_RTOL
    for key, e in zip(trials, snr_err):
        assert e < SNR_GUARD + rtol * ost[key].snr, (key, e, ost[key].snr)


def gp_count(spec, nint):
    return sum(len(spec.dm_list) * (nint // dt) for dt in spec.dt_list)
