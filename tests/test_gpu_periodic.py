"""GPU periodicity search (Sec. 3.1 footnote) against the FP64 oracle."""

import numpy as np
import pytest

import oracle
import synth
import paper_1802_03084_gb300 as rf
from gpu_common import SNR_GUARD, plans_for

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


def _train_spec(store="fp32", nint=160, npix=None):
    spec = synth.config("tiny")
    if npix:
        spec.npix = npix
    spec.store = store
    spec.edge = "full"
    spec.nint = nint
    spec.dm_list = np.array([0.0, 50.0, 100.0, 150.0])
    # a dispersed pulse every 8 integrations: power at k = L/8 and harmonics
    spec.pulses = [dict(dm=100.0, t0_s=(3 + 8 * n) * spec.inttime_s, width_s=spec.inttime_s, amp=0.6,
                        x=90, y=170) for n in range(nint // 8)]
    return spec


def _compare(gst, ost, op, S, L, rtol):
    assert len(gst) == len(ost)
    for r in gst:
        key = (int(r["dm_idx"]), int(r["k"]))
        o = ost[key]
        assert abs(r["sigma"] - o.sigma) <= rtol * o.sigma, key
        assert abs(r["amplitude"] - o.amplitude) <= rtol * o.amplitude + 1e-6 * o.sigma, key
        assert abs(r["snr"] - o.snr) <= SNR_GUARD + rtol * o.snr, key
        if (int(r["x"]), int(r["y"])) != (o.x, o.y):
            # a tie within rounding: the engine's pixel is a maximum of the FP64 power image
            U, Q = oracle.periodic_series_transform(op, S, key[0], L, [key[1]])
            _, _, P = oracle.periodic_image(op, U[0], Q[0])
            assert o.amplitude ** 2 - P[int(r["y"]), int(r["x"])] <= 4 * rtol * o.amplitude ** 2, key


@pytest.mark.parametrize("store,L,kmin,kmax,nint,npix", [
    ("fp32", 64, 1, 32, 160, None), ("fp32", 128, 3, 40, 224, None), ("fp16", 64, 1, 32, 160, None),
    # 1024^2: the row pass's tiles by tensor copies, warps without block barriers
    ("fp32", 64, 1, 32, 160, 1024), ("fp16", 64, 5, 12, 160, 1024),
    # 2048^2: cp.async tiles, transforms of two warps
    ("fp32", 64, 7, 10, 160, 2048)])
def test_periodicity_search_matches_oracle(store, L, kmin, kmax, nint, npix):
    spec = _train_spec(store, nint, npix)
    seg = synth.make_segment(spec)
    gp, op = plans_for(spec, seg)
    nint = seg["vis"].shape[0]
    with gp:
        gc, gst = gp.periodicity_search(seg["vis"], L, kmin, kmax, 6.0, with_stats=True)
    oc, ost = oracle.search_periodic(op, seg["vis"], L, kmin, kmax, 6.0, with_stats=True)
    fits = oracle.periodic_dm_trials(op, nint, L)
    assert 2 in fits
    assert [int(r["dm_idx"]) for r in gst[::kmax - kmin + 1]] == fits
    S = op.stokes(seg["vis"], nint)
    _compare(gst, ost, op, S, L, 1e-4 if store == "fp32" else 1e-2)
    # candidates: equal outside the guard band around the threshold
    g = {(int(c["dm_idx"]), int(c["k"])): c for c in gc}
    o = {(c["dm_idx"], c["k"]): c for c in oc}
    for k, c in o.items():
        if abs(c["snr"] - 6.0) > SNR_GUARD:
            assert k in g, k
    for k, c in g.items():
        if k not in o:
            assert abs(ost[k].snr - 6.0) <= SNR_GUARD, k
    # the pulse train: its DM trial, harmonic L/8, its pixel
    best = gc[np.argmax(gc["snr"])]
    assert int(best["dm_idx"]) == 2 and (int(best["x"]), int(best["y"])) == (90, 170)
    assert int(best["k"]) % (L // 8) == 0
    assert abs(best["freq_hz"] - best["k"] / (L * spec.inttime_s)) < 1e-9


def test_periodicity_search_rejects_bad_arguments():
    spec = _train_spec()
    seg = synth.make_segment(spec, nint=64)
    gp, _ = plans_for(spec, seg)
    with gp:
        for L, kmin, kmax in [(48, 1, 4), (64, 0, 4), (64, 5, 4), (64, 1, 33), (128, 1, 4)]:
            with pytest.raises(rf.RfError) as e:
                gp.periodicity_search(seg["vis"], L, kmin, kmax, 6.0)
            assert e.value.status == rf.RF_ERR_INVALID_ARG
