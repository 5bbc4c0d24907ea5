"""rf_image_stats_noalloc against the search entry point's own image statistics.

Callers that cannot allocate device memory where they image (a CUDA graph
being recorded, a real-time loop, a host framework that owns the memory pool)
use rf_image_stats_noalloc, whose scratch is a static device array.  This
checks, on two calls in a row (and a repeat of the first), that it reports
the same peak pixel, peak, sigma and S/N as rf_search_segment_stats does for
the same images, within the tolerance the parity tests use.
"""

import numpy as np
import pytest

import oracle
import synth
import paper_1802_03084_gb300 as rf
from gpu_common import STAT_RTOL, plans_for

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1802_03084_gb300.build import build
    build()
    rf.lib()
    torch.cuda.init()
    return torch


def _half_plane(op, S, key, spec):
    d, s, t = key
    R, n = oracle.dedisperse_resample(S, op.delays[d], spec.dt_list[s], t, spec.nint)
    G = oracle.grid_full_plane(R, op.iu, op.iv, op.ongrid, spec.npix)
    return np.ascontiguousarray(G[:, : spec.npix // 2 + 1]).astype(np.complex64), op.weight(n)


def test_noalloc_matches_search_stats_on_consecutive_calls(torch_cuda):
    torch = torch_cuda
    spec = synth.config("tiny")
    seg = synth.make_segment(spec)
    gp, op = plans_for(spec, seg)
    N = spec.npix
    with gp:
        _, gst = gp.search_stats(seg["vis"])
    S = oracle.stokes_i(seg["vis"])
    stat = torch.zeros(rf.STAT_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    results = {}
    for key in [(3, 0, 27), (0, 0, 5), (3, 0, 27)]:
        H, W = _half_plane(op, S, key, spec)
        Hd = torch.from_numpy(H).cuda()
        rf.rf_image_stats_noalloc(Hd, N, W, stat)
        torch.cuda.synchronize()
        got = np.frombuffer(stat.cpu().numpy().tobytes(), dtype=rf.STAT_DTYPE)[0]
        sel = (gst["dm_idx"] == key[0]) & (gst["dt_idx"] == key[1]) & (gst["t_idx"] == key[2])
        ref = gst[sel][0]
        assert (int(got["x"]), int(got["y"])) == (int(ref["x"]), int(ref["y"])), key
        for f in ("peak", "sigma", "snr"):
            assert abs(float(got[f]) - float(ref[f])) <= STAT_RTOL * abs(float(ref[f])), (key, f)
        assert float(got["weight"]) == float(ref["weight"])
        if key in results:
            # the static scratch keeps the previous call's contents: a repeat
            # after another image must give the identical answer
            assert results[key].tobytes() == got.tobytes()
        results[key] = got.copy()


def test_noalloc_rejects_images_beyond_its_scratch(torch_cuda):
    torch = torch_cuda
    big = rf.RF_NOALLOC_MAX_NPIX * 2 if hasattr(rf, "RF_NOALLOC_MAX_NPIX") else 2048
    grid = torch.zeros((big, big // 2 + 1), dtype=torch.complex64, device="cuda")
    stat = torch.zeros(rf.STAT_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    with pytest.raises(rf.RfError) as e:
        rf.rf_image_stats_noalloc(grid, big, 1.0, stat)
    assert e.value.status == rf.RF_ERR_INVALID_ARG
    assert "1024" in e.value.message


def _random_half_plane(npix, seed):
    """A half plane gridded by the oracle from a random segment whose longest
    baseline lands near the edge of an npix grid, with its weight W."""
    from gpu_common import small_random_segment
    rng = np.random.default_rng(seed)
    seg = small_random_segment(rng, nant=10, nchan=6, nint=3, npix=npix)
    bl = oracle.baseline_uvw(seg["ant_uvw"])
    umax = np.abs(bl[:, :2]).max() * seg["freq_hz"].max() / oracle.C_LIGHT
    cell = 1.0 / (umax * 2.2)                 # the longest baseline at about N/2.2 cells
    op = oracle.OraclePlan(seg["ant_uvw"], seg["freq_hz"], 5e-3, npix, cell, [0.0], [1], 6.0, edge="full")
    S = op.stokes(seg["vis"])
    R, n = oracle.dedisperse_resample(S, op.delays[0], 1, 1, S.shape[0])
    G = oracle.grid_full_plane(R, op.iu, op.iv, op.ongrid, npix)
    W = op.weight(n)
    I = oracle.dirty_image_fft(G, W)
    return np.ascontiguousarray(G[:, : npix // 2 + 1]).astype(np.complex64), W, I


@pytest.mark.parametrize("npix", [16, 512, 1024])
def test_noalloc_against_the_oracle_at_its_size_limits(torch_cuda, npix):
    # 16: one transform per warp part, no cross-lane Parseval shuffle beyond
    # it; 512 and 1024 need more than 48 KB of dynamic shared memory, and
    # 1024 is the largest image the static scratch holds
    torch = torch_cuda
    stat = torch.zeros(rf.STAT_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    for seed in (1, 2):
        H, W, I = _random_half_plane(npix, seed)
        o = oracle.image_stats(I)
        Hd = torch.from_numpy(H).cuda()
        for _ in range(2):                       # two calls in a row on the shared scratch
            rf.rf_image_stats_noalloc(Hd, npix, W, stat)
            torch.cuda.synchronize()
            got = np.frombuffer(stat.cpu().numpy().tobytes(), dtype=rf.STAT_DTYPE)[0]
            x, y = int(got["x"]), int(got["y"])
            if (x, y) != (o.x, o.y):             # a tie within rounding: the pixel must be a maximum too
                assert o.peak - I[y, x] <= STAT_RTOL * abs(o.peak), ((x, y), (o.x, o.y))
            assert abs(float(got["peak"]) - o.peak) <= STAT_RTOL * abs(o.peak), (npix, seed)
            assert abs(float(got["sigma"]) - o.sigma) <= STAT_RTOL * o.sigma, (npix, seed)
            assert abs(float(got["snr"]) - o.snr) <= 2 * STAT_RTOL * abs(o.snr), (npix, seed)
            assert float(got["weight"]) == W


def test_noalloc_rejects_host_pointers(torch_cuda):
    torch = torch_cuda
    grid = torch.zeros((256, 129), dtype=torch.complex64)
    stat_dev = torch.zeros(rf.STAT_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    for g, s in ((grid, stat_dev), (grid.pin_memory(), stat_dev),
                 (grid.cuda(), torch.zeros(rf.STAT_DTYPE.itemsize, dtype=torch.uint8).pin_memory())):
        with pytest.raises(rf.RfError) as e:
            rf.rf_image_stats_noalloc(g, 256, 1.0, s)
        assert e.value.status == rf.RF_ERR_INVALID_ARG
        assert "device memory" in e.value.message
