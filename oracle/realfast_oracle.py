"""Plain FP64 CPU oracle of the realfast search hot path.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path imports this module:
only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` call it.  It shares no code with the CUDA engine.

What it computes (Law et al. 2018, "realfast", Sec. 2.2 and Sec. 3.1): for a
segment of visibilities, for every DM trial, every boxcar width dt and every
output integration t', a dedispersed, resampled Stokes-I visibility set is
imaged by nearest-neighbour gridding and a 2D inverse DFT; each dirty image's
peak is compared with the image noise and images whose peak S/N reaches the
threshold emit one candidate.

The paper states the pipeline in words only.  The readings taken where it is
silent are listed with each function; in short:

* delay  delta[d][c] = floor(4.1488e-3 DM_d (f_c^-2 - f_top^-2) / t_int + 1/2)
  with f in GHz (dispersion law, Sec. 2.1 footnote), evaluated in the fixed
  FP64 order of :func:`delay_table`.
* resample  R[d,s,t'][b,c] = sum_{j<dt_s} S[t' dt_s + j + delta[d][c]][b,c],
  S = mean of the two polarisations (Stokes I, Sec. 3.1).  FULL edge rule
  t' < floor((nint - max_c delta[d][c]) / dt_s); PARTIAL edge rule
  t' < floor(nint / dt_s) with samples past the segment given weight 0.
* grid  (iu, iv) = round-half-away(u_m f_c / c * N cell), same for v; a
  visibility is on the grid iff |iu| < N/2 and |iv| < N/2; w is ignored.
* image  I[y][x] = (1/W) sum_{on-grid b,c} Re(R_bc exp(+2 pi i (iu (x - N/2) +
  iv (y - N/2)) / N)),  W = sum_{on-grid b,c} n_c (samples summed).
* stats  mu = mean(I), sigma = population std of all N^2 pixels, peak = max I
  (lowest y N + x on ties), snr = peak / sigma, candidate iff snr >= threshold.
  Optionally (clipped noise) mu and sigma are recomputed once over the pixels
  within 5 sigma of mu.

Around the search (their docstrings give the readings): mean-visibility
subtraction over the segment, a stream of segments overlapping by the longest
sweep, candidate spectra and moments, and the periodicity search (a time
Fourier transform of dedispersed windows, each frequency imaged).
"""

from __future__ import annotations

import dataclasses
from typing import Dict, List, Optional, Sequence

import numpy as np

C_LIGHT = 299792458.0
DISP_CONST = 4.1488e-3          # s GHz^2 per pc cm^-3 (Sec. 2.1 footnote, refined constant)

EDGE_FULL = "full"
EDGE_PARTIAL = "partial"


# ----------------------------------------------------------------------------
# Geometry and tables
# ----------------------------------------------------------------------------

def baseline_uvw(ant_uvw: np.ndarray) -> np.ndarray:
    """Baseline uvw for every antenna pair (Sec. 2.2: N_bl = N_ant (N_ant - 1) / 2).

    Order: (i, j) with i < j, i outer; uvw_b = uvw_j - uvw_i.
    """
    ant = np.asarray(ant_uvw, dtype=np.float64)
    n = ant.shape[0]
    rows = []
    for i in range(n):
        for j in range(i + 1, n):
            rows.append(ant[j] - ant[i])
    return np.array(rows, dtype=np.float64).reshape(-1, 3)


def delay_table(dm_list: Sequence[float], freq_hz: Sequence[float], inttime_s: float) -> np.ndarray:
    """Integer-sample dispersion delays delta[d][c] (Sec. 2.1 footnote).

    tau = 4.1488 ms * DM * (f^-2 - f_top^-2), f in GHz, referenced to the
    highest channel so that every delay is >= 0, in units of the integration
    time and rounded half up.  FP64 evaluation order:
    ((K * dm) * (1/(f*f) - 1/(ft*ft))) / tint with f = f_hz * 1e-9.
    """
    f = np.asarray(freq_hz, dtype=np.float64) * 1e-9
    ft = np.float64(np.max(np.asarray(freq_hz, dtype=np.float64))) * 1e-9
    dm = np.asarray(dm_list, dtype=np.float64)
    dinv = (1.0 / (f * f)) - (1.0 / (ft * ft))
    d = ((DISP_CONST * dm)[:, None] * dinv[None, :]) / np.float64(inttime_s)
    return np.floor(d + 0.5).astype(np.int64)


def round_half_away(x: np.ndarray) -> np.ndarray:
    """Nearest integer, ties away from zero: sign(x) * floor(|x| + 1/2)."""
    x = np.asarray(x, dtype=np.float64)
    return np.where(x >= 0, np.floor(x + 0.5), -np.floor(-x + 0.5)).astype(np.int64)


def cell_table(bl_uvw: np.ndarray, freq_hz: Sequence[float], npix: int, cell_rad: float):
    """Nearest uv cell of every (baseline, channel) and its on-grid flag.

    u in wavelengths is u_m f / c; the cell size is du = 1 / (N cell), so the
    cell index is round(u_m f / c * N cell).  FP64 order:
    (u_m * (f / c)) * (N * cell).  Returns iu, iv [nbl, nchan] int64 and
    ongrid [nbl, nchan] bool (|iu| < N/2 and |iv| < N/2).
    """
    f = np.asarray(freq_hz, dtype=np.float64)
    s = f / C_LIGHT
    fov = np.float64(npix) * np.float64(cell_rad)
    u = np.asarray(bl_uvw, dtype=np.float64)[:, 0]
    v = np.asarray(bl_uvw, dtype=np.float64)[:, 1]
    iu = round_half_away((u[:, None] * s[None, :]) * fov)
    iv = round_half_away((v[:, None] * s[None, :]) * fov)
    half = npix // 2
    ongrid = (np.abs(iu) < half) & (np.abs(iv) < half)
    return iu, iv, ongrid


def n_valid_times(nint: int, max_delay: int, dt: int, edge: str) -> int:
    """Number of output integrations t' searched for one (DM, dt) trial.

    FULL: the whole dispersed sweep must lie inside the segment (segments
    overlap by the largest sweep, Sec. 3.2), so t' < floor((nint - max delay) / dt).
    PARTIAL: t' < floor(nint / dt); samples past the segment get weight 0.
    """
    if edge == EDGE_FULL:
        span = nint - int(max_delay)
        return max(span // dt, 0) if span > 0 else 0
    return nint // dt


# ----------------------------------------------------------------------------
# Per-image arithmetic
# ----------------------------------------------------------------------------

def stokes_i(vis: np.ndarray) -> np.ndarray:
    """Stokes I = mean over the polarisation axis (Sec. 3.1, Table 1: two pols).

    vis: complex [nint, nbl, nchan, npol] -> complex128 [nint, nbl, nchan].
    """
    v = np.asarray(vis)
    return v.astype(np.complex128).mean(axis=3)


def subtract_mean(S: np.ndarray, nint: Optional[int] = None) -> np.ndarray:
    """Mean-visibility subtraction (Sec. 3.1): the mean over the segment's
    integrations of every (baseline, channel) is removed, so sources that
    are constant over the segment (shorter than the fringe-rate time scale,
    Sec. 3.2) vanish.  S: [nint, nbl, nchan]; returns a new array."""
    n = S.shape[0] if nint is None else nint
    return S - S[:n].mean(axis=0, keepdims=True)


def dedisperse_resample(S: np.ndarray, delays_d: np.ndarray, dt: int, t: int, nint: Optional[int] = None):
    """R[b,c] = sum_{j<dt} S[t*dt + j + delta[c]][b, c] and n[c] = samples present.

    Samples at index >= nint carry weight 0 (only reachable under PARTIAL).
    ``S`` is indexed by absolute integration; pass ``nint`` when S holds a
    longer buffer than the segment.
    """
    nint_s = S.shape[0] if nint is None else nint
    nbl, nchan = S.shape[1], S.shape[2]
    R = np.zeros((nbl, nchan), dtype=np.complex128)
    n = np.zeros(nchan, dtype=np.int64)
    cidx = np.arange(nchan)
    for j in range(dt):
        tt = t * dt + j + np.asarray(delays_d, dtype=np.int64)
        ok = tt < nint_s
        if not np.any(ok):
            continue
        tcl = np.where(ok, tt, 0)
        samp = S[tcl[None, :], np.arange(nbl)[:, None], cidx[None, :]]
        R += np.where(ok[None, :], samp, 0)
        n += ok
    return R, n


def grid_full_plane(R: np.ndarray, iu: np.ndarray, iv: np.ndarray, ongrid: np.ndarray, npix: int) -> np.ndarray:
    """Full-plane Hermitian uv grid G[v mod N][u mod N] (nearest-neighbour).

    Each on-grid visibility adds R at (iu, iv) and conj(R) at (-iu, -iv), so
    the sky image is real.
    """
    N = npix
    m = ongrid
    r = R[m]
    u = iu[m]
    v = iv[m]
    i1 = (v % N) * N + (u % N)
    i2 = ((-v) % N) * N + ((-u) % N)
    re = np.bincount(i1, weights=r.real, minlength=N * N) + np.bincount(i2, weights=r.real, minlength=N * N)
    im = np.bincount(i1, weights=r.imag, minlength=N * N) - np.bincount(i2, weights=r.imag, minlength=N * N)
    return (re + 1j * im).reshape(N, N)


def dirty_image_fft(G: np.ndarray, W: float) -> np.ndarray:
    """I[y][x] = Re(sum_{v,u} G[v][u] e^{+2 pi i (u (x - N/2) + v (y - N/2)) / N}) / (2W).

    numpy's inverse FFT is used as the DFT step (it divides by N^2, which is
    multiplied back); the (x - N/2, y - N/2) shift is an fftshift.
    """
    N = G.shape[0]
    raw = np.fft.ifft2(G) * (N * N)
    return np.fft.fftshift(raw).real / (2.0 * W)


def dirty_image_complex(G: np.ndarray) -> np.ndarray:
    """The shifted complex DFT of the full plane (before taking Re and scaling)."""
    N = G.shape[0]
    return np.fft.fftshift(np.fft.ifft2(G) * (N * N))


def dirty_image_dft(R: np.ndarray, iu: np.ndarray, iv: np.ndarray, ongrid: np.ndarray, npix: int, W: float) -> np.ndarray:
    """Brute-force O(N^2 nvis) evaluation of the image definition (small N only)."""
    N = npix
    m = ongrid
    r = R[m]
    u = iu[m].astype(np.float64)
    v = iv[m].astype(np.float64)
    xs = np.arange(N, dtype=np.float64) - N // 2
    ex = np.exp(2j * np.pi * np.outer(u, xs) / N)       # [nvis, N] over x
    ey = np.exp(2j * np.pi * np.outer(v, xs) / N)       # [nvis, N] over y
    img = np.einsum("k,ky,kx->yx", r, ey, ex)
    return img.real / W


@dataclasses.dataclass
class ImageStats:
    mean: float
    sigma: float
    peak: float
    x: int
    y: int
    snr: float


CLIP_SIGMA = 5.0


def image_stats(I: np.ndarray, clip: bool = False) -> ImageStats:
    """Population mean/std of all pixels, the maximum pixel and peak/sigma (Sec. 3.1).

    Ties for the maximum go to the lowest linear index y N + x.  With
    ``clip`` the noise takes one clipping pass: with mu0, sigma0 over all
    pixels, mean and sigma are recomputed over the pixels with
    |I - mu0| <= 5 sigma0 (the peak is still the maximum of all pixels).
    """
    N = I.shape[1]
    flat = np.asarray(I, dtype=np.float64).ravel()
    mu = flat.mean()
    sigma = float(np.sqrt(np.mean((flat - mu) ** 2)))
    if clip:
        kept = flat[np.abs(flat - mu) <= CLIP_SIGMA * sigma]
        mu = kept.mean()
        sigma = float(np.sqrt(np.mean((kept - mu) ** 2)))
    k = int(np.argmax(flat))
    peak = float(flat[k])
    y, x = divmod(k, N)
    snr = peak / sigma if sigma > 0 else 0.0
    return ImageStats(float(mu), sigma, peak, x, y, snr)


# ----------------------------------------------------------------------------
# Segment search
# ----------------------------------------------------------------------------

@dataclasses.dataclass
class OraclePlan:
    """Everything fixed for a segment shape (the 'state' of Sec. 3.2)."""
    ant_uvw: np.ndarray
    freq_hz: np.ndarray
    inttime_s: float
    npix: int
    cell_rad: float
    dm_list: np.ndarray
    dt_list: List[int]
    threshold: float
    edge: str = EDGE_FULL
    npol: int = 2
    mean_subtract: bool = False
    noise_clipped: bool = False

    def __post_init__(self):
        self.bl_uvw = baseline_uvw(self.ant_uvw)
        self.delays = delay_table(self.dm_list, self.freq_hz, self.inttime_s)
        self.iu, self.iv, self.ongrid = cell_table(self.bl_uvw, self.freq_hz, self.npix, self.cell_rad)
        self.max_delay = self.delays.max(axis=1)

    @property
    def nbl(self):
        return self.bl_uvw.shape[0]

    def n_times(self, nint: int, d: int, s: int) -> int:
        return n_valid_times(nint, int(self.max_delay[d]), int(self.dt_list[s]), self.edge)

    def image_list(self, nint: int):
        """All searched images (d, s, t') in (d, s, t') order."""
        out = []
        for d in range(len(self.dm_list)):
            for s in range(len(self.dt_list)):
                for t in range(self.n_times(nint, d, s)):
                    out.append((d, s, t))
        return out

    def count_images(self, nint: int) -> int:
        return sum(self.n_times(nint, d, s) for d in range(len(self.dm_list)) for s in range(len(self.dt_list)))

    def weight(self, n: np.ndarray) -> float:
        """W = sum over on-grid (b, c) of the samples summed into R[b, c]."""
        return float((self.ongrid.sum(axis=0) * n).sum())

    def stokes(self, vis: np.ndarray, nint: Optional[int] = None) -> np.ndarray:
        """Stokes I of the segment, mean-subtracted if the plan says so."""
        n = vis.shape[0] if nint is None else nint
        S = stokes_i(vis[:n])
        return subtract_mean(S, n) if self.mean_subtract else S

    def image(self, S: np.ndarray, d: int, s: int, t: int, nint: Optional[int] = None, method: str = "fft"):
        """Dirty image of trial (d, s, t') and its weight W (None if W = 0)."""
        R, n = dedisperse_resample(S, self.delays[d], int(self.dt_list[s]), t, nint)
        W = self.weight(n)
        if W <= 0:
            return None, 0.0
        if method == "dft":
            return dirty_image_dft(R, self.iu, self.iv, self.ongrid, self.npix, W), W
        G = grid_full_plane(R, self.iu, self.iv, self.ongrid, self.npix)
        return dirty_image_fft(G, W), W

    def stats(self, I: np.ndarray) -> ImageStats:
        """Image statistics under the plan's noise rule."""
        return image_stats(I, self.noise_clipped)

    def candidate(self, d: int, s: int, t: int, st: ImageStats) -> Dict:
        N = self.npix
        return dict(dm_idx=d, dt_idx=s, t_idx=t, x=st.x, y=st.y, snr=st.snr, peak=st.peak,
                    sigma=st.sigma, dm=float(self.dm_list[d]),
                    l_rad=(st.x - N // 2) * self.cell_rad, m_rad=(st.y - N // 2) * self.cell_rad)


def search_segment(plan: OraclePlan, vis: np.ndarray, nint: Optional[int] = None,
                   images: Optional[Sequence] = None, with_stats: bool = False):
    """Run the search over every image (or the listed (d, s, t') images).

    Returns the candidate list sorted by (dm_idx, dt_idx, t_idx) and, with
    ``with_stats``, a dict (d, s, t) -> ImageStats for every imaged trial.
    """
    n = vis.shape[0] if nint is None else nint
    S = plan.stokes(vis, n)
    todo = plan.image_list(n) if images is None else list(images)
    cands, stats = [], {}
    for (d, s, t) in todo:
        I, W = plan.image(S, d, s, t, n)
        if I is None:
            continue
        st = plan.stats(I)
        if with_stats:
            stats[(d, s, t)] = st
        if st.sigma > 0 and st.snr >= plan.threshold:
            cands.append(plan.candidate(d, s, t, st))
    cands.sort(key=lambda c: (c["dm_idx"], c["dt_idx"], c["t_idx"]))
    return (cands, stats) if with_stats else cands


def stream_overlap(plan: OraclePlan) -> int:
    """Integrations shared by consecutive segments of a stream: the longest
    dispersion sweep of the plan, max over DM trials and channels of delta
    (Sec. 3.2: segments overlap by the maximum sweep so that every pulse lies
    whole inside one segment)."""
    return int(np.max(plan.delays)) if plan.delays.size else 0


def search_stream(plan: OraclePlan, vis: np.ndarray, stride: int, with_stats: bool = False):
    """Search a continuous run of integrations cut into overlapping segments (Sec. 3.2).

    Segment k covers integrations [k stride, k stride + stride + overlap).
    Every DM trial and width dt (stride a multiple of every dt) searches
    t' < stride / dt there, so each sweep lies inside the segment and each
    start time k stride + t' dt is searched by exactly one segment.  Once
    fewer than stride + overlap integrations remain, the rest (from the
    next segment start to the end) is searched as one last segment under
    the plan's own edge rule.  Mean subtraction, if on, takes each segment's
    own mean.  t_idx in the output counts from the start of the run:
    k stride / dt + t'.
    """
    dts = [int(x) for x in plan.dt_list]
    for dt in dts:
        if stride % dt:
            raise ValueError("stride must be a multiple of every dt")
    overlap = stream_overlap(plan)
    nseg = stride + overlap
    total = vis.shape[0]
    windows = []
    k = 0
    while k * stride + nseg <= total:
        keys = [(d, s, t) for d in range(len(plan.dm_list)) for s, dt in enumerate(dts) for t in range(stride // dt)]
        windows.append((k * stride, nseg, keys))
        k += 1
    rest = total - k * stride
    if rest > 0:
        windows.append((k * stride, rest, plan.image_list(rest)))
    cands, stats = [], {}
    for start, n, keys in windows:
        S = plan.stokes(vis[start:start + n], n)
        for (d, s, t) in keys:
            I, W = plan.image(S, d, s, t, n)
            if I is None:
                continue
            st = plan.stats(I)
            key = (d, s, start // dts[s] + t)
            if with_stats:
                stats[key] = st
            if st.sigma > 0 and st.snr >= plan.threshold:
                cands.append(plan.candidate(*key, st))
    cands.sort(key=lambda c: (c["dm_idx"], c["dt_idx"], c["t_idx"]))
    return (cands, stats) if with_stats else cands


# ----------------------------------------------------------------------------
# Candidate products (Sec. 3.3: statistics from each candidate's image and
# spectrum at a low threshold, image and spectrum plots at a higher one)
# ----------------------------------------------------------------------------

def moments(v: np.ndarray):
    """Population mean, standard deviation, skewness and excess kurtosis:
    mu, sqrt(m2), m3 / m2^1.5, m4 / m2^2 - 3 with m_k = mean((v - mu)^k).
    Skewness and kurtosis are 0 when m2 = 0."""
    v = np.asarray(v, dtype=np.float64).ravel()
    if v.size == 0:
        return 0.0, 0.0, 0.0, 0.0
    mu = v.mean()
    d = v - mu
    m2 = float(np.mean(d * d))
    if m2 <= 0:
        return float(mu), 0.0, 0.0, 0.0
    m3 = float(np.mean(d * d * d))
    m4 = float(np.mean(d * d * d * d))
    return float(mu), float(np.sqrt(m2)), m3 / m2 ** 1.5, m4 / (m2 * m2) - 3.0


def candidate_spectrum(plan: OraclePlan, S: np.ndarray, d: int, s: int, t: int, x: int, y: int,
                       nint: Optional[int] = None):
    """Spectrum of a candidate: per channel, the dedispersed, resampled
    visibilities phased to pixel (x, y) with the image's own cell phases,
    averaged over the on-grid baselines and samples:

        spec[c] = sum_{b on-grid} R[b,c] exp(+2 pi i (iu (x - N/2) + iv (y - N/2)) / N) / w_c,
        w_c = (on-grid baselines at c) * n_c.

    Returns (spec complex128 [nchan], w_c [nchan]); spec is 0 where w_c = 0.
    The w-weighted mean of Re(spec) is the image value at (x, y)."""
    N = plan.npix
    R, n = dedisperse_resample(S, plan.delays[d], int(plan.dt_list[s]), t, nint)
    k = plan.iu * (x - N // 2) + plan.iv * (y - N // 2)
    ph = np.exp(2j * np.pi * (k % N) / N)
    w = plan.ongrid.sum(axis=0) * n
    num = np.where(plan.ongrid, R * ph, 0).sum(axis=0)
    spec = np.where(w > 0, num / np.where(w > 0, w, 1), 0)
    return spec, w.astype(np.float64)


def candidate_features(plan: OraclePlan, S: np.ndarray, d: int, s: int, t: int, nint: Optional[int] = None):
    """Image and spectrum statistics of trial (d, s, t') at its peak pixel.

    Image moments are over all N^2 pixels; spectrum moments over the real
    part of the spectrum at the channels with data (w_c > 0)."""
    I, W = plan.image(S, d, s, t, nint)
    st = plan.stats(I)
    spec, w = candidate_spectrum(plan, S, d, s, t, st.x, st.y, nint)
    im = moments(I)
    used = w > 0
    sp = moments(spec.real[used])
    return dict(dm_idx=d, dt_idx=s, t_idx=t, x=st.x, y=st.y, snr=st.snr,
                image_mean=im[0], image_sigma=im[1], image_skew=im[2], image_kurtosis=im[3],
                spec_mean=sp[0], spec_std=sp[1], spec_skew=sp[2], spec_kurtosis=sp[3],
                peak_from_spectrum=float((w * spec.real).sum() / w.sum()), nchan_used=int(used.sum()),
                spectrum=spec, image=I)


# ----------------------------------------------------------------------------
# Periodicity search (Sec. 3.1 footnote: a time segment is Fourier transformed
# and each fluctuation frequency imaged; Fig. 2: a change of the innermost loop)
# ----------------------------------------------------------------------------

def periodic_series_transform(plan: OraclePlan, S: np.ndarray, d: int, L: int, ks: Sequence[int]):
    """Cosine and sine sums of the dedispersed series of DM trial d.

    For each (b, c) the series is x[t] = S[t + delta[d][c]][b, c], t < L (the
    window starts at the segment start, the whole sweep inside it).  For each
    fluctuation frequency k:

        U_k[b,c] = (1/L) sum_t x[t] cos(2 pi k t / L),
        Q_k[b,c] = (1/L) sum_t x[t] sin(2 pi k t / L).

    Returns complex arrays U, Q of shape [len(ks), nbl, nchan]."""
    nbl, nchan = S.shape[1], S.shape[2]
    t = np.arange(L)
    X = np.zeros((L, nbl, nchan), dtype=np.complex128)
    cidx = np.arange(nchan)
    for ti in range(L):
        X[ti] = S[ti + plan.delays[d][cidx], np.arange(nbl)[:, None], cidx[None, :]]
    U = np.zeros((len(ks), nbl, nchan), dtype=np.complex128)
    Q = np.zeros((len(ks), nbl, nchan), dtype=np.complex128)
    for j, k in enumerate(ks):
        c = np.cos(2 * np.pi * k * t / L) / L
        s = np.sin(2 * np.pi * k * t / L) / L
        U[j] = np.tensordot(c, X, axes=(0, 0))
        Q[j] = np.tensordot(s, X, axes=(0, 0))
    return U, Q


def periodic_image(plan: OraclePlan, U: np.ndarray, Q: np.ndarray):
    """Power image of one fluctuation frequency.

    A source whose flux varies as A(t) has visibility A(t) e^{-i theta_b} on
    baseline b and A(t) e^{+i theta_b} on its mirror; imaging the time
    transform at frequency k over both gives 2 (I_U - i I_Q), with I_U and
    I_Q the ordinary dirty images (Sec. 3.1 arithmetic, weight W = on-grid
    pairs) of U and Q.  The power image is P = I_U^2 + I_Q^2; a flux
    A1 cos(2 pi k t / L + psi) at a pixel gives sqrt(P) = A1 / 2 there.
    Returns (I_U, I_Q, P)."""
    W = float(plan.ongrid.sum())
    IU = dirty_image_fft(grid_full_plane(U, plan.iu, plan.iv, plan.ongrid, plan.npix), W)
    IQ = dirty_image_fft(grid_full_plane(Q, plan.iu, plan.iv, plan.ongrid, plan.npix), W)
    return IU, IQ, IU * IU + IQ * IQ


@dataclasses.dataclass
class PeriodicStats:
    amplitude: float   # sqrt(max P)
    sigma: float       # per-quadrature noise: sqrt((var(I_U) + var(I_Q)) / 2)
    x: int
    y: int
    snr: float         # amplitude / sigma


def periodic_stats(IU: np.ndarray, IQ: np.ndarray) -> PeriodicStats:
    """Peak of the power image (lowest index on ties) against the noise of
    the two quadrature images (population variances)."""
    N = IU.shape[1]
    P = (IU * IU + IQ * IQ).ravel()
    k = int(np.argmax(P))
    y, x = divmod(k, N)
    sig = float(np.sqrt((IU.var() + IQ.var()) / 2.0))
    amp = float(np.sqrt(P[k]))
    return PeriodicStats(amp, sig, x, y, amp / sig if sig > 0 else 0.0)


def periodic_dm_trials(plan: OraclePlan, nint: int, L: int) -> List[int]:
    """DM trials whose whole window of L integrations and sweep fit in the segment."""
    return [d for d in range(len(plan.dm_list)) if int(plan.max_delay[d]) + L <= nint]


def search_periodic(plan: OraclePlan, vis: np.ndarray, L: int, kmin: int, kmax: int, threshold: float,
                    nint: Optional[int] = None, with_stats: bool = False):
    """Periodicity search of a segment: every DM trial whose window fits, every
    k in [kmin, kmax] (1 <= kmin <= kmax <= L/2); a candidate (dm_idx, k, x,
    y, snr) for each power image whose snr reaches the threshold."""
    n = vis.shape[0] if nint is None else nint
    S = plan.stokes(vis, n)
    ks = list(range(kmin, kmax + 1))
    cands, stats = [], {}
    for d in periodic_dm_trials(plan, n, L):
        U, Q = periodic_series_transform(plan, S, d, L, ks)
        for j, k in enumerate(ks):
            IU, IQ, _ = periodic_image(plan, U[j], Q[j])
            st = periodic_stats(IU, IQ)
            if with_stats:
                stats[(d, k)] = st
            if st.sigma > 0 and st.snr >= threshold:
                cands.append(dict(dm_idx=d, k=k, x=st.x, y=st.y, snr=st.snr, amplitude=st.amplitude,
                                  sigma=st.sigma))
    cands.sort(key=lambda c: (c["dm_idx"], c["k"]))
    return (cands, stats) if with_stats else cands
