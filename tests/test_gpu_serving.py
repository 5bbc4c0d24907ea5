"""Serving: segments of mixed shapes in flight together give the same
candidates as each searched alone; admission respects the HBM budget."""

import numpy as np
import pytest

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


def test_budget_admission_and_eviction():
    segs = _mixed_segments()
    need = [rf.rf_plan_estimate_bytes(desc) for _, _, desc in segs]
    # a budget that holds only the largest plan: segments run one plan at a time,
    # evicting idle plans, and still all finish with the same results
    budget = max(need) + (1 << 20)
    with rf.Server(slots=2, hbm_budget_bytes=budget) as sv:
        tickets = [sv.submit(desc, seg["vis"], spec.nint) for spec, seg, desc in segs]
        res = [sv.results(t) for t in tickets]
    assert all(len(r) > 0 for r in res)
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
