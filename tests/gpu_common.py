"""Shared helpers for the GPU parity tests (engine vs FP64 oracle)."""

import numpy as np

import oracle
import synth
import paper_1802_03084_gb300 as rf

# Tolerances (stated by the engine's precision contract):
IMG_RMS_FP32 = 1e-4     # image relative RMS error, FP32 storage
IMG_RMS_FP16 = 1e-2     # image relative RMS error, FP16 storage
STAT_RTOL = 1e-4        # peak and sigma relative error vs FP64
SNR_GUARD = 0.05        # candidates closer than this to the threshold are not compared


def rel_rms(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.sqrt(np.mean((a - b) ** 2)) / np.sqrt(np.mean(b ** 2)))


def plans_for(spec, seg, flags=None, max_nint=None, dt_list=None):
    dts = spec.dt_list if dt_list is None else dt_list
    edge = spec.edge
    mean = bool(getattr(spec, "mean_subtract", False))
    clip = bool(getattr(spec, "noise_clipped", False))
    if flags is not None:
        edge = "partial" if flags & rf.RF_EDGE_PARTIAL else "full"
        mean = bool(flags & rf.RF_MEAN_SUBTRACT)
        clip = bool(flags & rf.RF_NOISE_CLIPPED)
    op = oracle.OraclePlan(seg["ant_uvw"], seg["freq_hz"], spec.inttime_s, spec.npix, spec.cell_rad,
                           spec.dm_list, dts, spec.threshold, edge=edge, npol=spec.npol, mean_subtract=mean,
                           noise_clipped=clip)
    if flags is None:
        flags = (rf.RF_EDGE_PARTIAL if spec.edge == "partial" else 0) | \
                (rf.RF_STORE_FP16 if spec.store == "fp16" else 0) | \
                (rf.RF_MEAN_SUBTRACT if mean else 0) | \
                (rf.RF_NOISE_CLIPPED if clip else 0)
    gp = rf.Plan(seg["ant_uvw"], seg["freq_hz"], spec.inttime_s, spec.npix, spec.cell_rad, spec.dm_list, dts,
                 spec.threshold, npol=spec.npol, flags=flags, max_nint=max_nint or seg["vis"].shape[0])
    return gp, op


def compare_stats(gst, ost, oimages=None, rtol=STAT_RTOL):
    """gst: engine stats array; ost: dict (d,s,t) -> oracle ImageStats."""
    assert len(gst) == len(ost)
    bad = []
    for r in gst:
        key = (int(r["dm_idx"]), int(r["dt_idx"]), int(r["t_idx"]))
        o = ost[key]
        if abs(r["peak"] - o.peak) > rtol * abs(o.peak) + 1e-7 * o.sigma:
            bad.append(("peak", key, float(r["peak"]), o.peak))
        if abs(r["sigma"] - o.sigma) > rtol * o.sigma:
            bad.append(("sigma", key, float(r["sigma"]), o.sigma))
        if (int(r["x"]), int(r["y"])) != (o.x, o.y):
            # several maxima within rounding: the engine's pixel must be a maximum too
            if oimages is None or key not in oimages:
                bad.append(("argmax", key, (int(r["x"]), int(r["y"])), (o.x, o.y)))
            else:
                v = oimages[key][int(r["y"]), int(r["x"])]
                if o.peak - v > rtol * abs(o.peak):
                    bad.append(("argmax", key, (int(r["x"]), int(r["y"])), (o.x, o.y)))
    assert not bad, bad[:10]


def compare_candidates(gc, oc, threshold, ost=None, guard=SNR_GUARD):
    """Candidate (dm, dt, t, x, y) tuples equal outside the guard band around the threshold."""
    def far(snr):
        return abs(snr - threshold) > guard
    g = {(int(c["dm_idx"]), int(c["dt_idx"]), int(c["t_idx"])): c for c in gc}
    o = {(c["dm_idx"], c["dt_idx"], c["t_idx"]): c for c in oc}
    for k, c in o.items():
        if far(c["snr"]):
            assert k in g, ("missing", k, c["snr"])
            assert (int(g[k]["x"]), int(g[k]["y"])) == (c["x"], c["y"]), ("pixel", k)
    for k, c in g.items():
        if k not in o:
            osnr = ost[k].snr if ost is not None else None
            ref = osnr if osnr is not None else float(c["snr"])
            assert not far(ref), ("extra", k, float(c["snr"]), osnr)
    # sorted by (dm, dt, t)
    keys = [(int(c["dm_idx"]), int(c["dt_idx"]), int(c["t_idx"])) for c in gc]
    assert keys == sorted(keys)


def oracle_images(op, vis, keys, nint=None):
    S = op.stokes(vis, nint or vis.shape[0])
    out = {}
    for k in keys:
        I, W = op.image(S, *k, nint=nint or vis.shape[0])
        out[k] = I
    return out


def small_random_segment(rng, nant, nchan, nint, npix, npol=2, extent=None):
    """Random array/visibilities for shape sweeps (noise plus a random point source)."""
    ant = np.zeros((nant, 3))
    R = extent or 300.0
    ant[:, 0] = rng.uniform(-R, R, nant)
    ant[:, 1] = rng.uniform(-R, R, nant)
    f = np.sort(rng.uniform(1.0e9, 2.0e9, nchan))[::-1].copy() if nchan > 1 else np.array([1.4e9])
    nbl = nant * (nant - 1) // 2
    vis = (rng.standard_normal((nint, nbl, nchan, npol)) + 1j * rng.standard_normal((nint, nbl, nchan, npol)))
    vis = (vis * np.sqrt(0.5)).astype(np.complex64)
    vis += (0.8 * np.exp(1j * rng.uniform(0, 2 * np.pi))).astype(np.complex64)
    return dict(ant_uvw=ant, freq_hz=f, vis=vis)
