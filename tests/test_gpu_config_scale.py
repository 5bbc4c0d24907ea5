"""Candidate lists at configuration scale against the FP64 oracle.

The engine searches whole segments of the measured workloads in the launch
configuration the benchmark times (waves of thousands of images under a CUDA
graph).  Around every injected pulse the oracle then images every (DM, dt,
t') of a window one by one, over a spawn pool of the host cores, and the
engine's statistics and candidates in that window are compared with it:

* realtime (1024^2, FP32): every DM trial, t' dt within 8 integrations of
  each of the five pulses' arrival, all four dt;
* batching (2048^2, FP16 storage): the nine DM trials nearest each pulse's
  DM, the same time window, all five dt;
* a serving-shaped segment (1024 channels, 2048^2 images, the smearing DM
  grid to 1500): a 64-integration window around its pulse under the
  PARTIAL edge rule, the 13 DM trials nearest the pulse plus 32 drawn at
  random, every dt.

Candidates are compared as (DM, dt, t', x, y) tuples for images more than
0.05 sigma from the threshold; a pixel may differ only where the oracle's
image holds the same maximum within the storage precision there.
"""

import numpy as np
import pytest

import synth
import paper_1802_03084_gb300 as rf
from gpu_common import SNR_GUARD, STAT_RTOL
from oracle_pool import OraclePool, plan_kwargs

pytestmark = pytest.mark.gpu

FP16_RTOL = 1e-2


@pytest.fixture(scope="module")
def pool():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    p = OraclePool()               # spawned workers: no CUDA state is inherited
    from paper_1802_03084_gb300.build import build
    build()
    rf.lib()
    torch.cuda.init()
    yield p
    p.close()


def _key(r):
    return (int(r["dm_idx"]), int(r["dt_idx"]), int(r["t_idx"]))


def _compare(gst, gc, ores, threshold, rtol, guard=SNR_GUARD):
    """Engine statistics and candidates of the oracle-checked images."""
    by = {_key(r): r for r in gst}
    cand = {_key(c): c for c in gc}
    bad = []
    for key, (o, v_eng, W) in ores.items():
        r = by[key]
        if abs(float(r["weight"]) - W) > 0:
            bad.append(("weight", key, float(r["weight"]), W))
        if abs(float(r["peak"]) - o.peak) > rtol * abs(o.peak) + 1e-7 * o.sigma:
            bad.append(("peak", key, float(r["peak"]), o.peak))
        if abs(float(r["sigma"]) - o.sigma) > rtol * o.sigma:
            bad.append(("sigma", key, float(r["sigma"]), o.sigma))
        tie_ok = o.peak - v_eng <= rtol * abs(o.peak) + 1e-7 * o.sigma
        if (int(r["x"]), int(r["y"])) != (o.x, o.y) and not tie_ok:
            bad.append(("pixel", key, (int(r["x"]), int(r["y"])), (o.x, o.y)))
        if o.snr >= threshold + guard:
            if key not in cand:
                bad.append(("missing candidate", key, o.snr))
            elif (int(cand[key]["x"]), int(cand[key]["y"])) != (o.x, o.y) and not tie_ok:
                bad.append(("candidate pixel", key))
        elif o.snr < threshold - guard and key in cand:
            bad.append(("extra candidate", key, float(cand[key]["snr"]), o.snr))
    assert not bad, (len(bad), bad[:10])
    n_c = sum(1 for k in ores if k in cand)
    return n_c


def _window_keys(gst, dms, s_dt, t_lo, t_hi):
    """Searched images (d, s, t') with d in dms and t' dt in [t_lo, t_hi]."""
    keys = []
    dm_set = set(dms)
    for r in gst:
        d, s, t = _key(r)
        if d in dm_set and t_lo <= t * s_dt[s] <= t_hi:
            keys.append((d, s, t, int(r["x"]), int(r["y"])))
    return keys


def _search(spec, seg, wave=8192):
    import torch
    flags = (rf.RF_EDGE_PARTIAL if spec.edge == "partial" else 0) | (rf.RF_STORE_FP16 if spec.store == "fp16" else 0)
    vis = torch.from_numpy(seg["vis"]).cuda()
    with rf.Plan(seg["ant_uvw"], seg["freq_hz"], spec.inttime_s, spec.npix, spec.cell_rad, spec.dm_list,
                 spec.dt_list, spec.threshold, npol=spec.npol, flags=flags, max_nint=seg["vis"].shape[0]) as gp:
        gp.set_wave_images(wave)
        gc, gst = gp.search_stats(vis)
        gc2 = gp.search(vis)                      # graph capture, then replay
        gc3 = gp.search(vis)
        n = gp.count_images(seg["vis"].shape[0])
    del vis
    torch.cuda.empty_cache()
    assert np.array_equal(gc, gc2) and np.array_equal(gc, gc3)
    assert len(gst) == n
    keys = [_key(c) for c in gc]
    assert keys == sorted(keys)
    return gc, gst


def _pulse_t(spec, p):
    return int(p["t0_s"] / spec.inttime_s)


def test_realtime_every_dm_around_every_pulse(pool):
    spec = synth.config("realtime")
    seg = synth.make_segment(spec)
    gc, gst = _search(spec, seg)
    assert len(gst) == 177521
    items = []
    for p in spec.pulses:
        tp = _pulse_t(spec, p)
        items += _window_keys(gst, range(len(spec.dm_list)), spec.dt_list, tp - 8, tp + 8)
    items = sorted(set(items))
    ores = pool.stats(seg["vis"], plan_kwargs(spec, seg), items)
    n_c = _compare(gst, gc, ores, spec.threshold, STAT_RTOL)
    print(f"\nrealtime: {len(ores)} images around 5 pulses against the oracle, {n_c} candidates among them")
    assert n_c > 100


def test_batching_fp16_around_every_pulse(pool):
    spec = synth.config("batching")
    seg = synth.make_segment(spec)
    gc, gst = _search(spec, seg)
    assert len(gst) == 553095
    kw = plan_kwargs(spec, seg)
    from oracle import delay_table
    maxd = delay_table(spec.dm_list, seg["freq_hz"], spec.inttime_s).max(axis=1)
    total, n_c = 0, 0
    for p in spec.pulses:
        tp = _pulse_t(spec, p)
        d0 = int(np.argmin(np.abs(np.asarray(spec.dm_list) - p["dm"])))
        dms = [d for d in range(d0 - 4, d0 + 5) if 0 <= d < len(spec.dm_list)]
        items = _window_keys(gst, dms, spec.dt_list, tp - 8, tp + 8)
        if not items:
            continue
        a = max(0, (tp - 8) // 16 * 16)
        b = tp + 8 + 16 + int(maxd[max(dms)]) + 1
        ores = pool.stats(seg["vis"], kw, items, a=a, b=b)
        n_c += _compare(gst, gc, ores, spec.threshold, FP16_RTOL)
        total += len(ores)
    print(f"\nbatching (FP16 storage): {total} images around 5 pulses against the oracle, {n_c} candidates")
    assert total > 500 and n_c > 20


def test_serving_shape_1024_channels_2048_pixels(pool):
    spec = synth.SegmentSpec(name="serving-1024ch-2048px", nchan=1024, f_lo_hz=1.0e9, bw_hz=1.0e9, nint=2048,
                             inttime_s=5e-3, npix=2048,
                             dm_list=synth.dm_grid_smearing(1500.0, None, 1.0e9, 1.0e9, 1024, 5e-3),
                             dt_list=[1, 2, 4], threshold=7.0, seed=104017, edge="partial")
    prng = np.random.Generator(np.random.PCG64(spec.seed + 7919))
    spec.pulses = synth.segments._random_pulses(prng, spec, 1, (200.0, 600.0), (5e-3, 20e-3), (0.5, 1.0))
    p = spec.pulses[0]
    tp = _pulse_t(spec, p)
    t_start = max(0, (tp - 8) // 4 * 4)
    seg = synth.make_segment(spec, nint=64, t_start=t_start)
    spec.nint = 64
    gc, gst = _search(spec, seg, wave=4096)
    ndm = len(spec.dm_list)
    assert ndm > 500 and len(gst) == ndm * (64 + 32 + 16)
    d0 = int(np.argmin(np.abs(np.asarray(spec.dm_list) - p["dm"])))
    near = [d for d in range(d0 - 6, d0 + 7) if 0 <= d < ndm]
    rng = np.random.default_rng(3)
    far = rng.choice([d for d in range(ndm) if d not in near], 32, replace=False).tolist()
    items = _window_keys(gst, near, spec.dt_list, 0, 63)
    items += [it for it in _window_keys(gst, far, spec.dt_list, 0, 63) if rng.random() < 0.15]
    ores = pool.stats(seg["vis"], plan_kwargs(spec, seg), items)
    n_c = _compare(gst, gc, ores, spec.threshold, STAT_RTOL)
    print(f"\nserving shape 1024 ch, 2048^2, {ndm} DM trials: {len(ores)} images against the oracle, "
          f"{n_c} candidates among them")
    assert n_c > 5
