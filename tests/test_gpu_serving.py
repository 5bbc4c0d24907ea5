"""Serving: segments of mixed shapes in flight together give the same
candidates as each searched alone; admission respects the HBM budget."""

import numpy as np
import pytest

import oracle
import synth
import paper_1802_03084_gb300 as rf

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


def _serving_shaped_segment():
    """A segment of the serving workload's largest shape class (1024
    channels over 1-2 GHz, 2048^2 images, dt {1, 2, 4}), cut to 128
    integrations and the 16 smearing-grid DM trials around its pulse, under
    the PARTIAL edge rule."""
    dms = synth.dm_grid_smearing(1500.0, None, 1.0e9, 1.0e9, 1024, 5e-3)
    d0 = int(np.argmin(np.abs(dms - 300.0)))
    spec = synth.SegmentSpec(name="mix-1024ch-2048px", nchan=1024, f_lo_hz=1.0e9, bw_hz=1.0e9, nint=128,
                             inttime_s=5e-3, npix=2048, dm_list=dms[d0 - 8:d0 + 8], dt_list=[1, 2, 4],
                             threshold=7.0, seed=311, edge="partial")
    spec.pulses = [dict(dm=300.0, t0_s=0.1, width_s=10e-3, amp=0.6, x=1024 + 40, y=1024 - 25)]
    seg = synth.make_segment(spec)
    desc = rf.make_desc(seg["ant_uvw"], seg["freq_hz"], spec.inttime_s, spec.npix, spec.cell_rad, spec.dm_list,
                        spec.dt_list, spec.threshold, flags=rf.RF_EDGE_PARTIAL, max_nint=spec.nint)
    return spec, seg, desc


def _mixed_segments():
    """Small segments of several shapes (channels, integrations, image size)."""
    out = []
    for k, (nchan, nint, npix) in enumerate([(32, 96, 128), (64, 128, 256), (32, 64, 256), (16, 128, 128),
                                              (64, 128, 256), (32, 96, 128), (48, 80, 512)]):
        spec = synth.SegmentSpec(name=f"mix{k}", nchan=nchan, f_lo_hz=1.0e9, bw_hz=1.0e9, nint=nint,
                                 inttime_s=5e-3, npix=npix, dm_list=synth.dm_grid_linear(200.0, 6),
                                 dt_list=[1, 2], threshold=6.0, seed=300 + (k % 5), edge="partial")
        spec.pulses = [dict(dm=100.0, t0_s=0.05, width_s=10e-3, amp=0.8, x=npix // 2 + 7, y=npix // 2 - 5)]
        seg = synth.make_segment(spec)
        # two clipped-noise plans; segments 0 and 5 keep identical descriptions (a resident plan is reused)
        flags = rf.RF_EDGE_PARTIAL | (rf.RF_NOISE_CLIPPED if k in (2, 6) else 0)
        desc = rf.make_desc(seg["ant_uvw"], seg["freq_hz"], spec.inttime_s, npix, spec.cell_rad, spec.dm_list,
                            spec.dt_list, spec.threshold, flags=flags, max_nint=nint)
        out.append((spec, seg, desc))
    return out


def test_results_same_alone_and_in_the_mix():
    segs = _mixed_segments()
    segs.insert(3, _serving_shaped_segment())
    alone = []
    for spec, seg, desc in segs:
        h = rf.rf_plan_create(desc)
        try:
            alone.append(rf.rf_search_segment(h, seg["vis"], spec.nint))
        finally:
            rf.rf_plan_destroy(h)
    with rf.Server(slots=3, hbm_budget_bytes=16 << 30) as sv:
        tickets = [sv.submit(desc, seg["vis"], spec.nint) for spec, seg, desc in segs]
        infos = [sv.wait(t) for t in tickets]
        mixed = [sv.results(t) for t in tickets]
    for a, m, info in zip(alone, mixed, infos):
        assert info["done"] == 1 and info["status"] == 0
        assert info["submit_s"] <= info["start_s"] <= info["done_s"]
        assert np.array_equal(a, m)
        assert len(a) > 0
    # repeated shapes reuse a resident plan at least once
    assert any(i["plan_reused"] for i in infos)
    # the serving-shaped segment's candidates against the FP64 oracle, image by image
    spec, seg, desc = segs[3]
    cands = mixed[3]
    op = oracle.OraclePlan(seg["ant_uvw"], seg["freq_hz"], spec.inttime_s, spec.npix, spec.cell_rad,
                           spec.dm_list, spec.dt_list, spec.threshold, edge="partial")
    S = op.stokes(seg["vis"])
    pick = np.concatenate([cands[np.argsort(-cands["snr"])[:4]], cands[:: max(1, len(cands) // 4)][:4]])
    for c in pick:
        key = (int(c["dm_idx"]), int(c["dt_idx"]), int(c["t_idx"]))
        I, W = op.image(S, *key, nint=spec.nint)
        o = oracle.image_stats(I)
        assert (int(c["x"]), int(c["y"])) == (o.x, o.y), key
        assert abs(float(c["snr"]) - o.snr) <= 1e-4 * o.snr + 1e-3, (key, float(c["snr"]), o.snr)


def test_budget_admission_and_eviction():
    segs = _mixed_segments()
    need = [rf.rf_plan_estimate_bytes(desc) for _, _, desc in segs]
    alone = []
    for spec, seg, desc in segs:
        h = rf.rf_plan_create(desc)
        try:
            alone.append(rf.rf_search_segment(h, seg["vis"], spec.nint))
        finally:
            rf.rf_plan_destroy(h)
    # a budget that holds only the largest plan: segments that arrive while
    # it is full wait, and are admitted when an earlier segment's plan goes
    # idle and can be evicted; all finish with their results alone
    budget = max(need) + (1 << 20)
    with rf.Server(slots=2, hbm_budget_bytes=budget) as sv:
        tickets = [sv.submit(desc, seg["vis"], spec.nint) for spec, seg, desc in segs]
        infos = [sv.wait(t) for t in tickets]
        res = [sv.results(t) for t in tickets]
    assert all(len(r) > 0 for r in res)
    for a, r in zip(alone, res):
        assert np.array_equal(a, r)
    # with two slots but room for one plan, a segment of another plan starts
    # only after a segment in flight has finished
    waited = 0
    for k in range(1, len(segs)):
        if any(infos[j]["start_s"] < infos[k]["start_s"] for j in range(k)) and \
                infos[k]["start_s"] >= min(infos[j]["done_s"] for j in range(k)) - 1e-6:
            waited += 1
    assert waited >= 1
    starts = sorted((i["start_s"], i["done_s"]) for i in infos)
    for (s0, d0), (s1, d1) in zip(starts, starts[1:]):
        assert s1 >= s0
    with rf.Server(slots=1, hbm_budget_bytes=min(need) // 2) as sv:
        spec, seg, desc = segs[0]
        with pytest.raises(rf.RfError) as e:
            sv.submit(desc, seg["vis"], spec.nint)
        assert e.value.status == rf.RF_ERR_NO_MEMORY


def test_estimate_covers_actual_device_bytes():
    for spec, seg, desc in _mixed_segments()[:3]:
        est = rf.rf_plan_estimate_bytes(desc)
        h = rf.rf_plan_create(desc)
        try:
            actual = rf.rf_plan_get_info(h).device_bytes
        finally:
            rf.rf_plan_destroy(h)
        assert est >= actual and est <= actual * 1.05 + (4 << 20), (est, actual)
