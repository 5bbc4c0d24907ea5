"""Precision of the engine's images and statistics against the FP64 oracle.

Storage is FP16 or FP32; dedispersion sums (FP32, stored FP32 for dt > 1),
gridding and FFTs are FP32 and the noise reduction is FP64 (Parseval's
identity over the grid).

* The stress subset (4096^2 images, 2048 channels over 1-3 GHz, a continuum
  source at 100 times the per-visibility noise): 8 DM trials spread over the
  grid of 512, every t' < 64 at dt = 1 and t' in {0, 1} at dt = 32, under
  the FULL edge rule from the segment start -- 528 images.  Every image's
  peak, sigma, S/N, pixel and candidate is compared with the oracle in both
  storage modes; the relative RMS image error is measured on ten of them.
* The batching workload (2048^2, 1024 channels, FP16 storage): rendered
  images at dt = 1, 2 and 16 against the oracle, so the boxcar sums of dt > 1
  are seen to keep FP32 precision (an FP16-rounded sum would cost about
  2^-11 relative per sample sum).

Run with ``-s`` to print the per-image errors.
"""

import numpy as np
import pytest

import oracle
import synth
import paper_1802_03084_gb300 as rf
from gpu_common import IMG_RMS_FP16, IMG_RMS_FP32, SNR_GUARD, STAT_RTOL, rel_rms
from oracle_pool import OraclePool, plan_kwargs

pytestmark = pytest.mark.gpu

NSUB = 64


@pytest.fixture(scope="module")
def pool():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    p = OraclePool()
    from paper_1802_03084_gb300.build import build
    build()
    rf.lib()
    torch.cuda.init()
    yield p
    p.close()


def _key(r):
    return (int(r["dm_idx"]), int(r["dt_idx"]), int(r["t_idx"]))


@pytest.fixture(scope="module")
def stress_subset(pool):
    spec = synth.config("stress")
    ndm = len(spec.dm_list)
    dsel = np.linspace(0, ndm - 1, 8).round().astype(int)
    spec.dm_list = np.asarray(spec.dm_list)[dsel]
    spec.dt_list = [1, 32]
    spec.edge = "full"
    freq = synth.channel_freqs(spec.f_lo_hz, spec.bw_hz, spec.nchan)
    maxd = oracle.delay_table(spec.dm_list, freq, spec.inttime_s).max(axis=1)
    nwin = NSUB + int(maxd.max())
    spec.nint = nwin
    seg = synth.make_segment(spec, nint=nwin)
    keys = [(d, 0, t) for d in range(8) for t in range(NSUB)] + [(d, 1, t) for d in range(8) for t in (0, 1)]
    ores = pool.stats(seg["vis"], plan_kwargs(spec, seg), keys)
    assert len(ores) == 528
    op = oracle.OraclePlan(**plan_kwargs(spec, seg))
    S = op.stokes(seg["vis"])
    rms_keys = [(d, 0, 8 * d) for d in range(8)] + [(0, 1, 0), (7, 1, 1)]
    oim = {k: op.image(S, *k, nint=nwin)[0] for k in rms_keys}
    del S
    return spec, seg, ores, oim


@pytest.mark.parametrize("store", ["fp16", "fp32"])
def test_stress_subset_every_image_vs_fp64(stress_subset, store):
    import torch
    spec, seg, ores, oim = stress_subset
    flags = rf.RF_STORE_FP16 if store == "fp16" else 0
    vis = torch.from_numpy(seg["vis"]).cuda()
    with rf.Plan(seg["ant_uvw"], seg["freq_hz"], spec.inttime_s, spec.npix, spec.cell_rad, spec.dm_list,
                 spec.dt_list, spec.threshold, npol=spec.npol, flags=flags, max_nint=spec.nint) as gp:
        gc, gst = gp.search_stats(vis)
        keys = list(oim)
        g = gp.render(vis, keys)
    del vis
    torch.cuda.empty_cache()
    by = {_key(r): r for r in gst}
    cand = {_key(c): c for c in gc}
    rtol = 1e-2 if store == "fp16" else STAT_RTOL
    peak_err, sig_err, snr_err, bad = [], [], [], []
    for key, (o, _, W) in ores.items():
        r = by[key]
        peak_err.append(abs(float(r["peak"]) - o.peak) / o.sigma)
        sig_err.append(abs(float(r["sigma"]) - o.sigma) / o.sigma)
        snr_err.append(abs(float(r["snr"]) - o.snr))
        if abs(float(r["peak"]) - o.peak) > rtol * abs(o.peak):
            bad.append(("peak", key))
        if sig_err[-1] > rtol:
            bad.append(("sigma", key))
        if (int(r["x"]), int(r["y"])) != (o.x, o.y):
            bad.append(("pixel", key, (int(r["x"]), int(r["y"])), (o.x, o.y)))
        if o.snr >= spec.threshold + SNR_GUARD and (key not in cand or
                                                    (int(cand[key]["x"]), int(cand[key]["y"])) != (o.x, o.y)):
            bad.append(("candidate", key))
        if o.snr < spec.threshold - SNR_GUARD and key in cand:
            bad.append(("extra candidate", key))
    img_err = [rel_rms(g[k], oim[key]) for k, key in enumerate(keys)]
    snrs = np.array([o.snr for (o, _, _) in ores.values()])
    print(f"\nprecision stress subset 4096^2 store={store}: {len(ores)} images (S/N {snrs.min():.1f}-{snrs.max():.1f}); "
          f"image rel RMS (10 images) max {max(img_err):.2e} median {np.median(img_err):.2e}; "
          f"|d peak|/sigma max {max(peak_err):.2e} median {np.median(peak_err):.2e}; "
          f"|d sigma|/sigma max {max(sig_err):.2e}; |d snr| max {max(snr_err):.2e} median {np.median(snr_err):.2e}")
    assert not bad, bad[:10]
    tol = IMG_RMS_FP16 if store == "fp16" else IMG_RMS_FP32
    assert max(img_err) < tol, img_err
    for (key, (o, _, _)), e in zip(ores.items(), snr_err):
        assert e < SNR_GUARD + rtol * o.snr, (key, e, o.snr)


def _image_from(op, Sx, key, nint, round_sum=False):
    """Oracle image of trial key from the Stokes series Sx; with round_sum
    the boxcar sums are rounded to FP16 before gridding (the storage the
    engine must not use for them)."""
    d, s, t = key
    R, n = oracle.dedisperse_resample(Sx, op.delays[d], int(op.dt_list[s]), t, nint)
    if round_sum:
        R = R.real.astype(np.float16).astype(np.float64) + 1j * R.imag.astype(np.float16).astype(np.float64)
    G = oracle.grid_full_plane(R, op.iu, op.iv, op.ongrid, op.npix)
    return oracle.dirty_image_fft(G, op.weight(n))


def test_batching_fp16_boxcar_sums_keep_fp32_precision(pool):
    """dt = 1, 2 and 16 at the first pulse of the batching workload, FP16
    storage: the engine's image error must be that of FP16 samples summed
    exactly (computed here from the FP64 Stokes series rounded to FP16), and
    well below that of sums rounded to FP16 again, which adds 2^-12 relative
    per sum (about 1.5 times the error at dt = 2 and 16 on this segment)."""
    spec = synth.config("batching")
    spec.edge = "partial"
    p = spec.pulses[0]
    t_pulse = int(p["t0_s"] / spec.inttime_s)
    t_start = max(0, t_pulse - 8) // 16 * 16
    seg = synth.make_segment(spec, nint=NSUB, t_start=t_start)
    d_pulse = int(np.argmin(np.abs(np.asarray(spec.dm_list) - p["dm"])))
    tp = t_pulse - t_start
    trials = [(d_pulse, 0, tp), (d_pulse, 1, tp // 2), (d_pulse, 4, tp // 16)]
    op = oracle.OraclePlan(**plan_kwargs(spec, seg, edge="partial"))
    S = op.stokes(seg["vis"], NSUB)
    S16 = S.real.astype(np.float16).astype(np.float64) + 1j * S.imag.astype(np.float16).astype(np.float64)
    oim = {k: _image_from(op, S, k, NSUB) for k in trials}
    exact = [rel_rms(_image_from(op, S16, k, NSUB), oim[k]) for k in trials]
    rounded = [rel_rms(_image_from(op, S16, k, NSUB, True), oim[k]) for k in trials]
    del S, S16
    errs = {}
    for store in ("fp16", "fp32"):
        flags = rf.RF_EDGE_PARTIAL | (rf.RF_STORE_FP16 if store == "fp16" else 0)
        with rf.Plan(seg["ant_uvw"], seg["freq_hz"], spec.inttime_s, spec.npix, spec.cell_rad, spec.dm_list,
                     spec.dt_list, spec.threshold, npol=spec.npol, flags=flags, max_nint=NSUB) as gp:
            g = gp.render(seg["vis"], trials)
        errs[store] = [rel_rms(g[k], oim[key]) for k, key in enumerate(trials)]
    print(f"\nbatching 2048^2 image rel RMS at dt 1, 2, 16: engine FP16 {['%.2e' % e for e in errs['fp16']]}, "
          f"FP32 {['%.2e' % e for e in errs['fp32']]}; FP16 samples summed exactly {['%.2e' % e for e in exact]}, "
          f"sums rounded to FP16 {['%.2e' % e for e in rounded]}")
    assert max(errs["fp32"]) < IMG_RMS_FP32
    assert max(errs["fp16"]) < IMG_RMS_FP16
    for k in range(3):
        assert errs["fp16"][k] <= 1.1 * exact[k] + 1e-6, (trials[k], errs["fp16"][k], exact[k])
    for k in (1, 2):
        assert errs["fp16"][k] <= 0.8 * rounded[k], (trials[k], errs["fp16"][k], rounded[k])
