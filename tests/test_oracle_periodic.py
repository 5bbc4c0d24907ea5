"""Pins for the oracle's periodicity search (Sec. 3.1 footnote)."""

import numpy as np
import pytest

import oracle
import synth


def _small(nchan=8, npix=32, L=16, dm=(0.0, 40.0, 120.0)):
    spec = synth.SegmentSpec(name="periodic-small", nchan=nchan, f_lo_hz=1.0e9, bw_hz=0.5e9, nint=96,
                             inttime_s=5e-3, npix=npix, dm_list=np.asarray(dm), dt_list=[1], threshold=5.0,
                             nant=6, cell_rad=26.0 * synth.segments.ARCSEC, seed=11)
    seg = synth.make_segment(spec)
    op = oracle.OraclePlan(seg["ant_uvw"], seg["freq_hz"], spec.inttime_s, spec.npix, spec.cell_rad,
                           spec.dm_list, spec.dt_list, spec.threshold, edge="full", npol=spec.npol)
    return spec, seg, op


def test_series_transform_matches_numpy_fft():
    spec, seg, op = _small()
    S = op.stokes(seg["vis"])
    L = 16
    for d in (0, 2):
        ks = list(range(L))
        U, Q = oracle.periodic_series_transform(op, S, d, L, ks)
        x = np.stack([S[t + op.delays[d][None, :], np.arange(S.shape[1])[:, None], np.arange(S.shape[2])[None, :]]
                      for t in range(L)])
        F = np.fft.fft(x, axis=0)
        for k in ks:
            np.testing.assert_allclose(U[k], (F[k] + F[-k % L]) / (2 * L), atol=1e-12)
            np.testing.assert_allclose(Q[k], (F[-k % L] - F[k]) / (2j * L), atol=1e-12)


def test_modulated_point_source_closed_form():
    spec, seg, op = _small()
    N, L = spec.npix, 16
    x0, y0, A0, A1, k0, psi = 21, 9, 3.0, 1.4, 3, 0.7
    kc = op.iu * (x0 - N // 2) + op.iv * (y0 - N // 2)
    ph = np.exp(-2j * np.pi * (kc % N) / N)
    t = np.arange(L + int(op.delays.max()) + 1)
    A = A0 + A1 * np.cos(2 * np.pi * k0 * t / L + psi)
    vis = (A[:, None, None] * ph[None])[..., None].repeat(2, axis=3)   # DM 0 data: no delays
    S = oracle.stokes_i(vis)
    U, Q = oracle.periodic_series_transform(op, S, 0, L, [k0, k0 + 1, L - k0])
    IU, IQ, P = oracle.periodic_image(op, U[0], Q[0])
    st = oracle.periodic_stats(IU, IQ)
    assert (st.x, st.y) == (x0, y0)
    assert abs(st.amplitude - A1 / 2) < 1e-12
    # the quadratures carry the phase: I_U = A1 cos(psi) / 2, I_Q = -A1 sin(psi) / 2
    assert abs(IU[y0, x0] - A1 * np.cos(psi) / 2) < 1e-12
    assert abs(IQ[y0, x0] + A1 * np.sin(psi) / 2) < 1e-12
    _, _, P1 = oracle.periodic_image(op, U[1], Q[1])
    assert np.abs(P1).max() < 1e-24                      # no power at k0 + 1
    _, _, P2 = oracle.periodic_image(op, U[2], Q[2])
    np.testing.assert_allclose(P2, P, atol=1e-12)        # L - k0 mirrors k0


def test_parseval_over_fluctuation_frequency():
    # sum over all k of I_U^2 + I_Q^2 = (1/L) sum_t I_t^2 per pixel, with I_t
    # the ordinary dt = 1 image of the same DM trial at t
    spec, seg, op = _small()
    S = op.stokes(seg["vis"])
    L = 8
    for d in (1, 2):
        U, Q = oracle.periodic_series_transform(op, S, d, L, list(range(L)))
        lhs = sum(oracle.periodic_image(op, U[k], Q[k])[2] for k in range(L))
        rhs = sum(op.image(S, d, 0, t)[0] ** 2 for t in range(L)) / L
        np.testing.assert_allclose(lhs, rhs, rtol=1e-10, atol=1e-14)


def test_dm_trials_whose_window_fits():
    spec, seg, op = _small()
    n = seg["vis"].shape[0]
    for L in (8, 16, 64):
        want = [d for d in range(3) if op.delays[d].max() + L <= n]
        assert oracle.periodic_dm_trials(op, n, L) == want


def test_injected_pulse_train_is_found_at_its_harmonics():
    spec, seg, op = _small(L=32)
    L, period = 32, 8                       # a pulse every 8 integrations: power at k = 4, 8, 12, 16
    spec.pulses = [dict(dm=120.0, t0_s=(2 + period * n) * spec.inttime_s, width_s=spec.inttime_s,
                        amp=1.5, x=12, y=20) for n in range(12)]
    seg = synth.make_segment(spec)
    cands, stats = oracle.search_periodic(op, seg["vis"], L, 1, L // 2, 6.0, with_stats=True)
    assert cands
    hits = {(c["dm_idx"], c["k"]) for c in cands if (c["x"], c["y"]) == (12, 20)}
    assert (2, 4) in hits and (2, 8) in hits
    assert stats[(2, 4)].snr > stats[(2, 5)].snr


def test_periodic_noise_of_a_hand_built_quadrature_pair():
    # I_U: 1 everywhere but 5 at (x=2, y=1) and -3 at (x=0, y=3): mean 1,
    # population variance (16 + 16) / 16 = 2.  I_Q: +-2 at four pixels, 0
    # elsewhere: mean 0, variance 4 * 4 / 16 = 1.  The per-quadrature noise is
    # sqrt((2 + 1) / 2) = sqrt(1.5); the power peaks at (2, 1) with
    # 5^2 + 0^2 = 25, so the amplitude is 5.  (A max of the two variances
    # would give sqrt(2), their sum sqrt(3), a mean square in place of the
    # variance sqrt(2).)
    IU = np.ones((4, 4))
    IU[1, 2] = 5.0
    IU[3, 0] = -3.0
    IQ = np.zeros((4, 4))
    IQ[0, 0], IQ[0, 1], IQ[2, 3], IQ[3, 3] = 2.0, -2.0, 2.0, -2.0
    st = oracle.periodic_stats(IU, IQ)
    assert (st.x, st.y) == (2, 1)
    assert st.amplitude == 5.0
    assert abs(st.sigma - np.sqrt(1.5)) < 1e-15
    assert abs(st.snr - 5.0 / np.sqrt(1.5)) < 1e-14


def test_periodic_noise_matches_the_closed_form_on_noise():
    """Per-quadrature noise of a noise-only segment against its expectation.

    Stokes I of one (b, c) sample is complex with independent real and
    imaginary parts of variance 1/4 (each polarisation has E|n|^2 = 1, and
    the two are averaged).  With U_k = (1/L) sum_t x_t cos(2 pi k t / L) and
    sum_t cos^2 = L/2 for 1 <= k < L/2 (L at k = L/2, where the sine sum
    vanishes), Re U_k and Im U_k have variance 1/(8L), and so do those of
    Q_k; at k = L/2, U carries 1/(4L) and Q nothing.  A pixel of I_U is
    (1/W) sum over the W on-grid pairs of Re(U e^{i phi}), whose variance is
    W / (8 L W^2) = 1/(8 L W) (twice that for U at k = L/2, with I_Q = 0).
    Either way (var I_U + var I_Q) / 2 has expectation 1/(8 L W), and the
    population variance over the pixels estimates it (the mean term of the
    (0, 0) cell is negligible).  The spread between (DM, k) cases comes from
    the finite number of occupied cells (a few per cent at this size).
    """
    spec = synth.SegmentSpec(name="periodic-noise", nchan=16, f_lo_hz=1.0e9, bw_hz=1.0e9, nint=120,
                             inttime_s=5e-3, npix=128, dm_list=np.array([0.0, 150.0]), dt_list=[1],
                             threshold=7.0, seed=5)
    seg = synth.make_segment(spec)
    op = oracle.OraclePlan(seg["ant_uvw"], seg["freq_hz"], spec.inttime_s, spec.npix, spec.cell_rad,
                           spec.dm_list, spec.dt_list, spec.threshold, edge="full", npol=spec.npol)
    S = op.stokes(seg["vis"])
    W = float(op.ongrid.sum())
    assert W > 5000
    ratios = []
    for L in (16, 32):
        expect = 1.0 / (8.0 * L * W)
        ks = list(range(1, L // 2 + 1))
        for d in (0, 1):
            U, Q = oracle.periodic_series_transform(op, S, d, L, ks)
            for j in range(len(ks)):
                IU, IQ, _ = oracle.periodic_image(op, U[j], Q[j])
                ratios.append(oracle.periodic_stats(IU, IQ).sigma ** 2 / expect)
    ratios = np.asarray(ratios)
    assert np.all(np.abs(ratios - 1.0) < 0.10), ratios
    assert abs(ratios.mean() - 1.0) < 0.03, ratios.mean()
