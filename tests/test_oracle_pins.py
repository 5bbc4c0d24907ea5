"""Pins for the FP64 oracle against what the paper and mathematics fix.

Every check here is independent of the oracle's own code path: exact rational
re-evaluation of the formulas, closed forms, brute-force DFTs, Parseval's
identity, linearity, the paper's printed numbers, and recovery of an injected
signal built by the separate input generator.
"""

import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _paper():
    with open(os.path.join(GOLDEN, "paper_numbers.json")) as f:
        return json.load(f)


def _plan(spec, edge=None):
    ant = synth.array_uvw(spec.seed, spec.nant, spec.dec_deg)
    f = synth.channel_freqs(spec.f_lo_hz, spec.bw_hz, spec.nchan)
    return oracle.OraclePlan(ant, f, spec.inttime_s, spec.npix, spec.cell_rad, spec.dm_list,
                             spec.dt_list, spec.threshold, edge=edge or spec.edge)


# ---------------------------------------------------------------- delays ----

def _exact_delay(dm, f_hz, ftop_hz, tint):
    """Exact rational tau / t_int (Sec. 2.1 footnote, K = 4.1488 ms)."""
    K = Fraction(41488, 10 ** 7)
    f = Fraction(f_hz) / 10 ** 9
    ft = Fraction(ftop_hz) / 10 ** 9
    return K * Fraction(dm) * (1 / (f * f) - 1 / (ft * ft)) / Fraction(tint)


@pytest.mark.parametrize("name", ["tiny", "realtime"])
def test_delay_table_exact_rational(name):
    spec = synth.config(name)
    f = synth.channel_freqs(spec.f_lo_hz, spec.bw_hz, spec.nchan)
    d = oracle.delay_table(spec.dm_list, f, spec.inttime_s)
    ftop = float(np.max(f))
    ambiguous = 0
    step_d = max(1, len(spec.dm_list) // 16)
    step_c = max(1, spec.nchan // 32)
    for i in range(0, len(spec.dm_list), step_d):
        for c in range(0, spec.nchan, step_c):
            x = _exact_delay(spec.dm_list[i], f[c], ftop, spec.inttime_s)
            frac = x - math.floor(x)
            if abs(frac - Fraction(1, 2)) < Fraction(1, 10 ** 9):
                ambiguous += 1
                continue
            assert d[i, c] == math.floor(x + Fraction(1, 2)), (i, c, float(x))
    assert ambiguous == 0
    assert (d >= 0).all()
    # the highest channel is the reference: zero delay at every DM
    assert (d[:, int(np.argmax(f))] == 0).all()


def test_delay_spot_values_tiny():
    # 64 channels over 1-2 GHz, 5 ms: hand-evaluated tau = 4.1488 ms DM (f_lo^-2 - f_top^-2)
    spec = synth.config("tiny")
    f = synth.channel_freqs(spec.f_lo_hz, spec.bw_hz, spec.nchan)
    d = oracle.delay_table([100.0, 200.0, 300.0, 700.0], f, 5e-3)
    assert list(d[:, 0]) == [61, 122, 182, 426]
    # monotone in DM and decreasing with frequency
    assert (np.diff(d, axis=0) >= 0).all()
    assert (np.diff(d, axis=1) <= 0).all()


def test_dispersion_constant_matches_paper():
    p = _paper()
    assert abs(oracle.DISP_CONST * 1e3 - p["dispersion_constant_ms"]["value"]) < 0.01


def test_sweep_example_sec32():
    # DM 2000 over 256 MHz centred at 1.4 GHz: "roughly 2 seconds" (Sec. 3.2)
    p = _paper()["sweep_example"]
    lo = (p["f_center_ghz"] - p["bw_mhz"] / 2000.0) * 1e9
    hi = (p["f_center_ghz"] + p["bw_mhz"] / 2000.0) * 1e9
    tint = 1e-3
    d = oracle.delay_table([p["dm"]], [lo, hi], tint)
    sweep = d[0, 0] * tint
    assert 1.0 < sweep < 2.5
    assert abs(sweep - p["sweep_s_roughly"]) / p["sweep_s_roughly"] < 0.3


# ----------------------------------------------------------- baselines ----

def test_baseline_count_and_order():
    p = _paper()
    ant = synth.array_uvw(101)
    bl = oracle.baseline_uvw(ant)
    assert bl.shape == (p["baselines"]["value"], 3)
    assert ant.shape[0] == p["antennas"]["value"]
    # three antennas by hand: (0,1), (0,2), (1,2), uvw_j - uvw_i
    a = np.array([[0.0, 0, 0], [1.0, 2, 3], [10.0, 20, 30]])
    np.testing.assert_array_equal(oracle.baseline_uvw(a), [[1, 2, 3], [10, 20, 30], [9, 18, 27]])


def test_table1_data_rates():
    # 351 baselines x channels x 2 pols x 8 B (complex64) per integration
    p = _paper()
    nbl = p["baselines"]["value"]
    for row in p["table1_modes"]["rows"]:
        rate = nbl * row["channels"] * 2 * 8 / (row["tint_ms"] * 1e-3) / 1e6
        assert abs(rate - row["rate_MBps"]) / row["rate_MBps"] < 0.05, row
    spec = synth.config("realtime")
    rate = spec.input_bytes() / (spec.nint * spec.inttime_s) / 1e6
    assert abs(rate - 290) / 290 < 0.02


# ---------------------------------------------------------------- cells ----

def test_cell_table_exact_rational():
    spec = synth.config("tiny")
    ant = synth.array_uvw(spec.seed)
    bl = oracle.baseline_uvw(ant)
    f = synth.channel_freqs(spec.f_lo_hz, spec.bw_hz, spec.nchan)
    iu, iv, on = oracle.cell_table(bl, f, spec.npix, spec.cell_rad)
    fov = Fraction(spec.npix) * Fraction(spec.cell_rad)
    rng = np.random.default_rng(0)
    for _ in range(400):
        b = int(rng.integers(bl.shape[0]))
        c = int(rng.integers(spec.nchan))
        for comp, got in ((0, iu[b, c]), (1, iv[b, c])):
            x = Fraction(bl[b, comp]) * Fraction(f[c]) / Fraction(299792458) * fov
            ax = abs(x)
            assert abs(ax - math.floor(ax) - Fraction(1, 2)) > Fraction(1, 10 ** 9)
            want = math.floor(ax + Fraction(1, 2)) * (1 if x >= 0 else -1)
            assert got == want
    # cell(-u) = -cell(u): the rounding is odd-symmetric
    iu2, iv2, _ = oracle.cell_table(-bl, f, spec.npix, spec.cell_rad)
    np.testing.assert_array_equal(iu2, -iu)
    np.testing.assert_array_equal(iv2, -iv)


def test_ongrid_rule():
    bl = np.array([[100.0, 0, 0], [0, 100.0, 0]])
    f = np.array([1e9])
    N = 16
    # choose cell so that u maps to exactly 7.4 and 8.4 cells
    lam = 299792458.0 / 1e9
    cell7 = 7.4 / (100.0 / lam * N)
    iu, iv, on = oracle.cell_table(bl, f, N, cell7)
    assert iu[0, 0] == 7 and on[0, 0]
    cell8 = 8.4 / (100.0 / lam * N)
    iu, iv, on = oracle.cell_table(bl, f, N, cell8)
    assert iu[0, 0] == 8 and not on[0, 0]        # |iu| must be < N/2
    assert iv[1, 0] == 8 and not on[1, 0]


# -------------------------------------------------------------- imaging ----

def _random_vis(rng, nvis, N):
    iu = rng.integers(-(N // 2) + 1, N // 2, size=(nvis, 1))
    iv = rng.integers(-(N // 2) + 1, N // 2, size=(nvis, 1))
    R = rng.standard_normal((nvis, 1)) + 1j * rng.standard_normal((nvis, 1))
    on = np.ones((nvis, 1), dtype=bool)
    return R, iu, iv, on


@pytest.mark.parametrize("N", [16, 32])
def test_fft_image_equals_bruteforce_dft(N):
    rng = np.random.default_rng(N)
    R, iu, iv, on = _random_vis(rng, 40, N)
    W = 40.0
    G = oracle.grid_full_plane(R, iu, iv, on, N)
    a = oracle.dirty_image_fft(G, W)
    # brute force written directly from the definition, pixel by pixel
    b = np.zeros((N, N))
    for y in range(N):
        for x in range(N):
            acc = 0.0
            for k in range(R.shape[0]):
                ph = 2 * np.pi * (iu[k, 0] * (x - N // 2) + iv[k, 0] * (y - N // 2)) / N
                acc += (R[k, 0] * complex(math.cos(ph), math.sin(ph))).real
            b[y, x] = acc / W
    assert np.max(np.abs(a - b)) <= 1e-12 * np.max(np.abs(b))
    c = oracle.dirty_image_dft(R, iu, iv, on, N, W)
    assert np.max(np.abs(a - c)) <= 1e-12 * np.max(np.abs(b))


def test_single_visibility_is_a_fringe():
    # one unit visibility at (iu, iv) = (3, 0): I = cos(2 pi 3 (x - N/2) / N) / W
    N = 32
    R = np.array([[1.0 + 0j]])
    iu = np.array([[3]])
    iv = np.array([[0]])
    on = np.array([[True]])
    I = oracle.dirty_image_fft(oracle.grid_full_plane(R, iu, iv, on, N), 1.0)
    x = np.arange(N) - N // 2
    np.testing.assert_allclose(I, np.tile(np.cos(2 * np.pi * 3 * x / N), (N, 1)), atol=1e-12)
    # the v axis maps to rows (y), the u axis to columns (x)
    I2 = oracle.dirty_image_fft(oracle.grid_full_plane(R, iv, iu, on, N), 1.0)
    np.testing.assert_allclose(I2, I.T, atol=1e-12)


def test_phase_centre_point_source_peak_is_mean_visibility():
    spec = synth.config("tiny")
    plan = _plan(spec)
    A = 0.37
    nint = 4
    S = np.full((nint, plan.nbl, len(plan.freq_hz)), A, dtype=np.complex128)
    I, W = plan.image(S, 0, 0, 0, nint)
    N = spec.npix
    assert abs(I[N // 2, N // 2] - A) < 1e-12
    st = oracle.image_stats(I)
    assert (st.x, st.y) == (N // 2, N // 2)
    assert abs(st.peak - A) < 1e-12


def test_point_source_at_pixel_with_exact_cells():
    # visibilities phased to pixel (x0, y0) using integer cells reproduce a
    # peak of exactly A at (x0, y0): sign and axis convention of the image.
    N = 64
    rng = np.random.default_rng(5)
    R0, iu, iv, on = _random_vis(rng, 300, N)
    x0, y0, A = 40, 21, 2.5
    R = A * np.exp(-2j * np.pi * (iu * (x0 - N // 2) + iv * (y0 - N // 2)) / N)
    I = oracle.dirty_image_fft(oracle.grid_full_plane(R, iu, iv, on, N), 300.0)
    st = oracle.image_stats(I)
    assert (st.x, st.y) == (x0, y0)
    assert abs(st.peak - A) < 1e-12


def test_parseval_and_hermitian():
    spec = synth.config("tiny")
    plan = _plan(spec)
    seg = synth.make_segment(spec, nint=8)
    S = oracle.stokes_i(seg["vis"])
    R, n = oracle.dedisperse_resample(S, plan.delays[2], 1, 3, 8)
    W = plan.weight(n)
    G = oracle.grid_full_plane(R, plan.iu, plan.iv, plan.ongrid, spec.npix)
    N = spec.npix
    # Hermitian grid -> real image
    Z = oracle.dirty_image_complex(G)
    assert np.max(np.abs(Z.imag)) <= 1e-9 * np.max(np.abs(Z.real))
    I = oracle.dirty_image_fft(G, W)
    lhs = np.sum(I * I)
    rhs = N * N / (4.0 * W * W) * np.sum(np.abs(G) ** 2)
    assert abs(lhs - rhs) <= 1e-10 * rhs


def test_linearity_dt2_is_mean_of_dt1():
    spec = synth.config("tiny")
    ant = synth.array_uvw(spec.seed)
    f = synth.channel_freqs(spec.f_lo_hz, spec.bw_hz, spec.nchan)
    plan = oracle.OraclePlan(ant, f, spec.inttime_s, spec.npix, spec.cell_rad, spec.dm_list,
                             [1, 2], spec.threshold, edge=oracle.EDGE_FULL)
    seg = synth.make_segment(spec)
    S = oracle.stokes_i(seg["vis"])
    for d, t in [(0, 0), (1, 5), (1, 30)]:
        I2, _ = plan.image(S, d, 1, t)
        Ia, _ = plan.image(S, d, 0, 2 * t)
        Ib, _ = plan.image(S, d, 0, 2 * t + 1)
        np.testing.assert_allclose(I2, 0.5 * (Ia + Ib), atol=1e-12)


def test_dedispersion_aligns_a_dispersed_impulse():
    # put one unit sample per channel at t0 + delta[d][c]: trial d gathers all of
    # them at t' = t0 (index direction and per-channel delay), others do not.
    spec = synth.config("tiny")
    plan = _plan(spec)
    nint = 128
    t0 = 5
    d = 1
    S = np.zeros((nint, plan.nbl, len(plan.freq_hz)), dtype=np.complex128)
    for c in range(len(plan.freq_hz)):
        S[t0 + plan.delays[d, c], :, c] = 1.0
    R, n = oracle.dedisperse_resample(S, plan.delays[d], 1, t0, nint)
    assert np.all(R == 1.0) and np.all(n == 1)
    R0, _ = oracle.dedisperse_resample(S, plan.delays[0], 1, t0, nint)
    assert np.abs(R0).sum() < R.size / 4


def test_partial_edge_weights():
    spec = synth.config("tiny")
    plan = _plan(spec, edge=oracle.EDGE_PARTIAL)
    nint = 128
    S = np.ones((nint, plan.nbl, len(plan.freq_hz)), dtype=np.complex128)
    d = 7
    t = 100
    R, n = oracle.dedisperse_resample(S, plan.delays[d], 1, t, nint)
    want = (t + plan.delays[d] < nint).astype(int)
    np.testing.assert_array_equal(n, want)
    np.testing.assert_array_equal(R.real, np.broadcast_to(want, R.shape))
    # flat visibilities still image to A at the centre with partial weights
    I, W = plan.image(S, d, 0, t, nint)
    assert W == plan.ongrid.sum(axis=0) @ want
    assert abs(I[spec.npix // 2, spec.npix // 2] - 1.0) < 1e-12


def test_valid_time_counts():
    # hand count for 'tiny' (64 ch, 1-2 GHz, 5 ms, 128 integrations, DM 0..700
    # step 100): max delays 0, 61, 122, 182, ... so FULL searches
    # 128 + 67 + 6 = 201 images and PARTIAL searches 8 x 128.
    spec = synth.config("tiny")
    assert _plan(spec, edge=oracle.EDGE_FULL).count_images(128) == 201
    assert _plan(spec, edge=oracle.EDGE_PARTIAL).count_images(128) == 1024
    assert oracle.n_valid_times(100, 30, 4, oracle.EDGE_FULL) == 17
    assert oracle.n_valid_times(100, 100, 1, oracle.EDGE_FULL) == 0
    assert oracle.n_valid_times(100, 130, 1, oracle.EDGE_FULL) == 0
    assert oracle.n_valid_times(101, 0, 4, oracle.EDGE_PARTIAL) == 25


def test_image_stats_definition():
    I = np.zeros((4, 4))
    I[1, 2] = 3.0
    I[2, 1] = 3.0                        # tie: lowest y*N + x wins -> (x=2, y=1)
    I[3, 3] = -1.0
    st = oracle.image_stats(I)
    assert (st.x, st.y, st.peak) == (2, 1, 3.0)
    mu = 5.0 / 16
    var = (2 * (3 - mu) ** 2 + (1 + mu) ** 2 + 13 * mu ** 2) / 16
    assert abs(st.mean - mu) < 1e-15 and abs(st.sigma - math.sqrt(var)) < 1e-15
    assert abs(st.snr - 3.0 / math.sqrt(var)) < 1e-12


def test_stokes_i_is_pol_mean():
    v = np.zeros((1, 1, 1, 2), dtype=np.complex64)
    v[..., 0] = 1 + 2j
    v[..., 1] = 3 - 4j
    assert oracle.stokes_i(v)[0, 0, 0] == (2 - 1j)


# ------------------------------------------------------ injected pulse ----

def test_injected_pulse_recovered_tiny():
    spec = synth.config("tiny")
    plan = _plan(spec)
    seg = synth.make_segment(spec)
    p = spec.pulses[0]
    d_true = int(np.argmin(np.abs(spec.dm_list - p["dm"])))
    cands = oracle.search_segment(plan, seg["vis"])
    best = max(cands, key=lambda c: c["snr"])
    assert best["dm_idx"] == d_true
    assert abs(best["t_idx"] - p["t0_s"] / spec.inttime_s) <= 1.0
    assert (best["x"], best["y"]) == (p["x"], p["y"])
    assert best["snr"] > 20


def test_noise_only_image_statistics():
    # pure noise: sigma of the image ~ 0.5 / sqrt(N_vis) for Stokes-I noise 0.5 per component
    spec = synth.config("tiny")
    spec.pulses = []
    plan = _plan(spec)
    seg = synth.make_segment(spec, nint=4)
    S = oracle.stokes_i(seg["vis"])
    I, W = plan.image(S, 0, 0, 1, 4)
    st = oracle.image_stats(I)
    expect = 0.5 / math.sqrt(W)
    assert 0.8 < st.sigma / expect < 1.2
    assert abs(st.mean) < 1e-12          # no visibility on the (0,0) cell
    assert st.snr < 6.0


def test_mean_subtraction_removes_a_constant_source_and_keeps_a_pulse():
    # Sec. 3.1: a source constant over the segment vanishes; a pulse keeps all
    # but 1/nint of its amplitude per sample it occupies.
    spec = synth.config("tiny")
    spec.pulses = []
    spec.continuum = [dict(amp=5.0, x=100, y=150)]
    seg = synth.make_segment(spec, nint=16)
    ant = seg["ant_uvw"]
    op = oracle.OraclePlan(ant, seg["freq_hz"], spec.inttime_s, spec.npix, spec.cell_rad, spec.dm_list,
                           spec.dt_list, spec.threshold, edge="partial", mean_subtract=True)
    S = op.stokes(seg["vis"], 16)
    np.testing.assert_allclose(S.mean(axis=0), 0, atol=1e-12)
    I, _ = op.image(S, 0, 0, 3, 16)
    st = oracle.image_stats(I)
    assert st.peak < 0.3          # the 5.0 continuum is gone, noise-level image remains
    raw = oracle.stokes_i(seg["vis"])
    I_raw, _ = op.image(raw, 0, 0, 3, 16)
    assert oracle.image_stats(I_raw).peak > 4.0
    # an impulse at one integration keeps (1 - 1/nint) of its height
    X = np.zeros((16, 3, 2), dtype=np.complex128)
    X[5] = 1.0
    np.testing.assert_allclose(oracle.subtract_mean(X)[5], 1.0 - 1.0 / 16)
    np.testing.assert_allclose(oracle.subtract_mean(X)[4], -1.0 / 16)


def test_clipped_noise_excludes_a_bright_source():
    # one clipping pass at 5 sigma: a spike far above the noise is excluded,
    # so sigma becomes the noise pixels' own population std
    rng = np.random.default_rng(9)
    I = rng.standard_normal((64, 64)) * 0.1
    I = np.clip(I, -0.45, 0.45)             # every noise pixel within 4.5 of its own sigma
    I[10, 20] = 50.0
    noise = np.delete(I.ravel(), 10 * 64 + 20)
    st = oracle.image_stats(I, clip=True)
    assert abs(st.sigma - noise.std()) < 1e-12
    assert abs(st.mean - noise.mean()) < 1e-12
    assert (st.x, st.y, st.peak) == (20, 10, 50.0)
    full = oracle.image_stats(I)
    assert full.sigma > 5 * st.sigma and st.snr > 5 * full.snr
    # nothing beyond 5 sigma: clipping changes nothing
    J = np.clip(rng.standard_normal((32, 32)), -3, 3)
    a, b = oracle.image_stats(J), oracle.image_stats(J, clip=True)
    assert (a.sigma, a.mean, a.snr) == (b.sigma, b.mean, b.snr)


def test_clipped_noise_raises_a_pulse_snr():
    spec = synth.config("tiny")
    seg = synth.make_segment(spec)
    kw = dict(edge=spec.edge)
    op = oracle.OraclePlan(seg["ant_uvw"], seg["freq_hz"], spec.inttime_s, spec.npix, spec.cell_rad, spec.dm_list,
                           spec.dt_list, spec.threshold, **kw)
    opc = oracle.OraclePlan(seg["ant_uvw"], seg["freq_hz"], spec.inttime_s, spec.npix, spec.cell_rad, spec.dm_list,
                            spec.dt_list, spec.threshold, noise_clipped=True, **kw)
    c0 = max(oracle.search_segment(op, seg["vis"]), key=lambda c: c["snr"])
    c1 = max(oracle.search_segment(opc, seg["vis"]), key=lambda c: c["snr"])
    assert (c0["x"], c0["y"], c0["t_idx"]) == (c1["x"], c1["y"], c1["t_idx"])
    assert c1["snr"] >= c0["snr"] and c1["sigma"] <= c0["sigma"]
