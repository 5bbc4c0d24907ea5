"""GPU candidate products (Sec. 3.3) against the FP64 oracle."""

import numpy as np
import pytest

import oracle
import synth
import paper_1802_03084_gb300 as rf
from gpu_common import plans_for, rel_rms

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


def _records(trials_xy):
    c = np.zeros(len(trials_xy), dtype=rf.CANDIDATE_DTYPE)
    for k, (d, s, t, x, y) in enumerate(trials_xy):
        c[k]["dm_idx"], c[k]["dt_idx"], c[k]["t_idx"], c[k]["x"], c[k]["y"] = d, s, t, x, y
    return c


def _check_against_oracle(op, S, nint, cands, feats, spectra, images, tol_spec, tol_img):
    for k, c in enumerate(cands):
        d, s, t, x, y = (int(c[f]) for f in ("dm_idx", "dt_idx", "t_idx", "x", "y"))
        sp, w = oracle.candidate_spectrum(op, S, d, s, t, x, y, nint)
        I, _ = op.image(S, d, s, t, nint)
        f = feats[k]
        assert (int(f["dm_idx"]), int(f["dt_idx"]), int(f["t_idx"]), int(f["x"]), int(f["y"])) == (d, s, t, x, y)
        assert int(f["nchan_used"]) == int((w > 0).sum())
        scale = np.sqrt(np.mean(np.abs(sp[w > 0]) ** 2))
        assert np.max(np.abs(spectra[k] - sp)) <= tol_spec * scale, k
        assert abs(f["peak_from_spectrum"] - I[y, x]) <= tol_spec * scale
        mu, sd, sk, ku = oracle.moments(I)
        assert abs(f["image_mean"] - mu) <= tol_img * sd
        assert abs(f["image_sigma"] - sd) <= tol_img * sd
        assert abs(f["image_skew"] - sk) <= 1e3 * tol_img * max(1.0, abs(sk))
        assert abs(f["image_kurtosis"] - ku) <= 1e3 * tol_img * max(1.0, abs(ku))
        smu, ssd, ssk, sku = oracle.moments(sp.real[w > 0])
        assert abs(f["spec_mean"] - smu) <= tol_spec * scale
        assert abs(f["spec_std"] - ssd) <= tol_spec * scale
        if ssd > 1e-3 * scale:
            assert abs(f["spec_skew"] - ssk) <= 1e2 * tol_spec * max(1.0, abs(ssk))
            assert abs(f["spec_kurtosis"] - sku) <= 1e2 * tol_spec * max(1.0, abs(sku))
        assert rel_rms(images[k], I) < tol_img


@pytest.mark.parametrize("store", ["fp32", "fp16"])
def test_products_of_candidates_and_chosen_trials(store):
    spec = synth.config("tiny")
    spec.store = store
    seg = synth.make_segment(spec)
    gp, op = plans_for(spec, seg)
    nint = seg["vis"].shape[0]
    S = op.stokes(seg["vis"], nint)
    with gp:
        gc = gp.search(seg["vis"])
        assert len(gc) > 0
        # the candidates at their peaks, plus trials at the segment's end
        # (PARTIAL: channels whose delayed sample is past the end drop out)
        extra = _records([(7, 0, 127, 5, 9), (4, 0, 120, 200, 31), (0, 0, 0, 128, 128)])
        cands = np.concatenate([gc, extra])
        feats, spectra, images = gp.candidate_products(seg["vis"], cands)
        assert feats.shape == (len(cands),) and spectra.shape == (len(cands), spec.nchan)
        tol_spec, tol_img = (1e-5, 1e-4) if store == "fp32" else (2e-3, 1e-2)
        _check_against_oracle(op, S, nint, cands, feats, spectra, images, tol_spec, tol_img)
        # the engine's own peak equals the spectrum's weighted mean
        for k in range(len(gc)):
            assert abs(feats[k]["peak_from_spectrum"] - gc[k]["peak"]) <= 10 * tol_spec * abs(gc[k]["peak"])
        assert int(feats[-3]["nchan_used"]) < spec.nchan
        # repeatable
        f2, s2, i2 = gp.candidate_products(seg["vis"], cands)
        assert np.array_equal(f2, feats) and np.array_equal(s2, spectra) and np.array_equal(i2, images)


def test_candidate_tiers():
    spec = synth.config("tiny")
    seg = synth.make_segment(spec)
    gp, _ = plans_for(spec, seg)
    with gp:
        gc = gp.search(seg["vis"])
        feats, idx, sp, im = gp.candidate_tiers(seg["vis"], gc, stats_sigma=6.0, plot_sigma=6.5)
        assert len(feats) == int((gc["snr"] >= 6.0).sum())
        assert list(idx) == list(np.nonzero(gc[gc["snr"] >= 6.0]["snr"] >= 6.5)[0])
        if len(idx):
            assert sp.shape == (len(idx), spec.nchan) and im.shape == (len(idx), spec.npix, spec.npix)


def test_products_reject_bad_candidates():
    spec = synth.config("tiny")
    seg = synth.make_segment(spec)
    gp, _ = plans_for(spec, seg)
    with gp:
        for bad in ([(0, 0, 0, spec.npix, 3)], [(0, 0, 10_000, 1, 1)], [(99, 0, 0, 1, 1)]):
            with pytest.raises(rf.RfError) as e:
                gp.candidate_products(seg["vis"], _records(bad))
            assert e.value.status == rf.RF_ERR_INVALID_ARG
