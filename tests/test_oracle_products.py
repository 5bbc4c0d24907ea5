"""Pins for the oracle's candidate products (Sec. 3.3): image and spectrum
statistics and the phased spectrum."""

import numpy as np
import pytest

import oracle
import synth


def test_moments_match_library_routines():
    stats = pytest.importorskip("scipy.stats")
    rng = np.random.default_rng(5)
    for v in (rng.standard_normal(1000), rng.exponential(size=777), rng.uniform(size=64) ** 3):
        mu, sd, sk, ku = oracle.moments(v)
        assert abs(mu - np.mean(v)) < 1e-12
        assert abs(sd - np.std(v)) < 1e-12
        assert abs(sk - stats.skew(v, bias=True)) < 1e-10
        assert abs(ku - stats.kurtosis(v, fisher=True, bias=True)) < 1e-10


def test_moments_of_a_sampled_cosine():
    # over whole periods mean(cos^2) = 1/2, mean(cos^4) = 3/8: kurtosis 3/2, excess -3/2
    x = np.arange(64)
    mu, sd, sk, ku = oracle.moments(np.cos(2 * np.pi * 3 * x / 64))
    assert abs(mu) < 1e-14 and abs(sd - np.sqrt(0.5)) < 1e-14
    assert abs(sk) < 1e-12 and abs(ku + 1.5) < 1e-12
    assert oracle.moments(np.full(5, 2.0)) == (2.0, 0.0, 0.0, 0.0)


def _tiny():
    spec = synth.config("tiny")
    seg = synth.make_segment(spec)
    op = oracle.OraclePlan(seg["ant_uvw"], seg["freq_hz"], spec.inttime_s, spec.npix, spec.cell_rad,
                           spec.dm_list, spec.dt_list, spec.threshold, edge=spec.edge)
    return spec, seg, op


def test_spectrum_mean_is_the_fft_image_pixel():
    spec, seg, op = _tiny()
    S = op.stokes(seg["vis"])
    for (d, s, t) in [(3, 0, 27), (0, 0, 5), (7, 0, 100)]:
        f = oracle.candidate_features(op, S, d, s, t)
        I = f["image"]
        assert abs(f["peak_from_spectrum"] - I[f["y"], f["x"]]) <= 1e-12 * abs(I).max()
        # and at any other pixel the same identity holds
        sp, w = oracle.candidate_spectrum(op, S, d, s, t, 17, 200)
        assert abs((w * sp.real).sum() / w.sum() - I[200, 17]) <= 1e-12 * abs(I).max()
        assert f["nchan_used"] == int((w > 0).sum())


def test_point_source_on_its_cells_gives_a_flat_spectrum():
    spec, seg, op = _tiny()
    N = spec.npix
    x0, y0, A = 70, 181, 2.5
    # visibilities of a source exactly on the image's own cell phases
    k = op.iu * (x0 - N // 2) + op.iv * (y0 - N // 2)
    v = A * np.exp(-2j * np.pi * (k % N) / N)
    vis = np.broadcast_to(v[None, :, :, None], (16,) + v.shape + (2,)).astype(np.complex128)
    S = oracle.stokes_i(vis)
    f = oracle.candidate_features(op, S, 0, 0, 4)
    assert (f["x"], f["y"]) == (x0, y0)
    assert abs(f["spec_mean"] - A) < 1e-12 and f["spec_std"] < 1e-12
    assert abs(f["peak_from_spectrum"] - A) < 1e-12
    assert np.allclose(f["spectrum"][op.ongrid.any(axis=0)], A, atol=1e-12)
    # phased one pixel away the spectrum is no longer flat
    sp, w = oracle.candidate_spectrum(op, S, 0, 0, 4, x0 + 1, y0)
    assert np.std(sp.real[w > 0]) > 1e-3


def test_features_of_the_injected_pulse():
    spec, seg, op = _tiny()
    S = op.stokes(seg["vis"])
    cands = oracle.search_segment(op, seg["vis"])
    best = max(cands, key=lambda c: c["snr"])
    f = oracle.candidate_features(op, S, best["dm_idx"], best["dt_idx"], best["t_idx"])
    assert (f["x"], f["y"]) == (best["x"], best["y"])
    assert abs(f["snr"] - best["snr"]) < 1e-12
    # a bright point source makes the pixel distribution skewed to the right
    assert f["image_skew"] > 0
    assert abs(f["image_sigma"] * f["snr"] - f["peak_from_spectrum"]) < 1e-9
