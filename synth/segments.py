"""Synthetic VLA-like visibility segments (inputs only).

The shapes follow the paper's example correlator modes (Table 1: 27 antennas,
351 baselines, two polarisations, 256-1024 channels, 5-50 ms integrations) and
the five workload configurations this engine is measured on:

* ``tiny``      64 ch over 1-2 GHz, 128 x 5 ms, 8 DM trials 0-700, dt {1},
                256^2 image, one pulse (A=0.5, DM 300, 10 ms), threshold 6.
* ``realtime``  256 ch over 1-2 GHz, 1024 x 5 ms, 128 DM trials 0-1500 on the
                smearing grid, dt {1,2,4,8}, 1024^2 image, five pulses,
                threshold 7.
* ``batching``  1024 ch over 1-2 GHz, 2048 x 5 ms, 256 DM trials 0-3000,
                dt {1,2,4,8,16}, 2048^2 image, FP16 storage, threshold 7.
* ``serving``   mixed shapes, see :func:`serving_shapes`.
* ``stress``    2048 ch over 1-3 GHz, 4096 x 10 ms, 512 DM trials 0-3000,
                dt {1..32}, 4096^2 image, a 100-sigma continuum source.

Noise model: every polarisation sample is circular complex Gaussian with
E|n|^2 = 1 (real and imaginary parts N(0, 1/2)).  A source of amplitude A is
added identically to both polarisations, so its Stokes-I amplitude is A.

Signal model (the forward model of a dispersed pulse, not the search): a pulse
of dispersion measure D arriving at the top channel at time t0 reaches channel
c at t0 + K D (f_c^-2 - f_top^-2) with K = 4.1488e-3 s GHz^2 (the cold-plasma
law of Sec. 2.1), lasts ``width`` seconds, and each integration receives the
fraction of the integration it overlaps.  Its visibility on baseline b is
A exp(-2 pi i (u_b l + v_b m)) with u, v in wavelengths at f_c and
(l, m) = ((x - N/2) cell, (y - N/2) cell) for the pixel (x, y) it is put at.

Array: a Y with arms at azimuths 0/120/240 deg plus a seeded common rotation,
nine antennas per arm at log-spaced radii 40..600 m (inner eight jittered by a
seeded factor in [0.95, 1)).  uvw at hour angle 0 and declination +30 deg from
the VLA latitude with the textbook local-to-equatorial rotation (U = 0):
u = E, v = N cos(lat - dec), w = N sin(dec - lat).
"""

from __future__ import annotations

import dataclasses
import math
from typing import Dict, List, Optional, Sequence

import numpy as np

C_LIGHT = 299792458.0            # m/s
K_DISP = 4.1488e-3               # s GHz^2 per (pc cm^-3): forward model only
VLA_LAT_DEG = 34.0784
ARCSEC = math.pi / (180.0 * 3600.0)

CONFIG_NAMES = ("tiny", "realtime", "batching", "serving", "stress")


@dataclasses.dataclass
class SegmentSpec:
    name: str
    nchan: int
    f_lo_hz: float
    bw_hz: float
    nint: int
    inttime_s: float
    npix: int
    dm_list: np.ndarray
    dt_list: List[int]
    threshold: float
    nant: int = 27
    npol: int = 2
    cell_rad: float = 10.0 * ARCSEC
    edge: str = "full"            # "full" or "partial"
    store: str = "fp32"           # "fp32" or "fp16"
    mean_subtract: bool = False   # remove the per-(baseline, channel) segment mean first
    pulses: List[Dict] = dataclasses.field(default_factory=list)
    continuum: List[Dict] = dataclasses.field(default_factory=list)
    seed: int = 0
    dec_deg: float = 30.0

    @property
    def nbl(self) -> int:
        return self.nant * (self.nant - 1) // 2

    def input_bytes(self, nint: Optional[int] = None) -> int:
        n = self.nint if nint is None else nint
        return n * self.nbl * self.nchan * self.npol * 8


def channel_freqs(f_lo_hz: float, bw_hz: float, nchan: int) -> np.ndarray:
    """Channel centres evenly spanning [f_lo, f_lo + bw)."""
    return f_lo_hz + (np.arange(nchan, dtype=np.float64) + 0.5) * (bw_hz / nchan)


def array_uvw(seed: int, nant: int = 27, dec_deg: float = 30.0,
              rmin: float = 40.0, rmax: float = 600.0) -> np.ndarray:
    """Per-antenna (u, v, w) in metres for a seeded Y-shaped array at HA 0."""
    if nant % 3:
        raise ValueError("Y array needs a multiple of 3 antennas")
    per_arm = nant // 3
    rng = np.random.Generator(np.random.PCG64(seed))
    rot = rng.uniform(0.0, 2.0 * math.pi)
    radii = np.geomspace(rmin, rmax, per_arm)
    east, north = [], []
    for arm in range(3):
        az = rot + arm * 2.0 * math.pi / 3.0
        jit = np.ones(per_arm)
        jit[:-1] = rng.uniform(0.95, 1.0, per_arm - 1)
        r = radii * jit
        east.append(r * math.sin(az))
        north.append(r * math.cos(az))
    e = np.concatenate(east)
    n = np.concatenate(north)
    lat = math.radians(VLA_LAT_DEG)
    dec = math.radians(dec_deg)
    u = e
    v = n * math.cos(lat - dec)
    w = n * math.sin(dec - lat)
    return np.stack([u, v, w], axis=1).astype(np.float64)


def baseline_pairs(nant: int):
    """Baseline order of the engine's input: (i, j) with i < j, row major."""
    ii, jj = np.triu_indices(nant, k=1)
    return ii, jj


def dm_grid_linear(dm_max: float, n: int) -> np.ndarray:
    return np.linspace(0.0, dm_max, n)


def dm_grid_smearing(dm_max: float, n: Optional[int], f_lo_hz: float, bw_hz: float,
                     nchan: int, inttime_s: float) -> np.ndarray:
    """DM trials with equal steps of one effective pulse width of added delay.

    The effective width at DM D is sqrt(t_int^2 + (a D)^2), with a the
    intra-channel smearing per unit DM at the lowest channel centre
    (2 K dnu / f^3, the derivative of the dispersion law).  Counting steps of
    that width gives Phi(D) = (K_band / a) asinh(a D / t_int) with
    K_band = K (f_lo^-2 - f_top^-2).  With ``n`` given, the n trials are equal
    steps in Phi from 0 to dm_max; with ``n=None`` the count is ceil(Phi)+1.
    """
    f = channel_freqs(f_lo_hz, bw_hz, nchan) * 1e-9
    flo, ftop = f.min(), f.max()
    dnu_mhz = bw_hz / nchan * 1e-6
    a = 2.0 * K_DISP * 1e-3 * dnu_mhz / flo ** 3          # s per unit DM
    k_band = K_DISP * (flo ** -2 - ftop ** -2)             # s per unit DM
    phi_max = (k_band / a) * math.asinh(a * dm_max / inttime_s)
    if n is None:
        n = int(math.ceil(phi_max)) + 1
    x = np.arange(n, dtype=np.float64) / (n - 1) * math.asinh(a * dm_max / inttime_s)
    return (inttime_s / a) * np.sinh(x)


def _pixel_offsets(rng, npix: int, k: int, frac: float = 0.125):
    span = max(1, int(npix * frac))
    xs = rng.integers(npix // 2 - span, npix // 2 + span, size=k)
    ys = rng.integers(npix // 2 - span, npix // 2 + span, size=k)
    return xs, ys


def config(name: str, seed: Optional[int] = None) -> SegmentSpec:
    """The named workload configuration with its seeded pulse parameters."""
    seeds = {"tiny": 101, "realtime": 102, "batching": 103, "serving": 104, "stress": 105}
    s = seeds[name] if seed is None else seed
    rng = np.random.Generator(np.random.PCG64(s + 7919))
    if name == "tiny":
        spec = SegmentSpec(name=name, nchan=64, f_lo_hz=1.0e9, bw_hz=1.0e9, nint=128,
                           inttime_s=5e-3, npix=256, dm_list=dm_grid_linear(700.0, 8),
                           dt_list=[1], threshold=6.0, edge="partial", seed=s)
        x, y = _pixel_offsets(rng, spec.npix, 1)
        t0 = int(rng.integers(8, 40)) * spec.inttime_s
        spec.pulses = [dict(dm=300.0, t0_s=t0, width_s=10e-3, amp=0.5, x=int(x[0]), y=int(y[0]))]
        return spec
    if name == "realtime":
        spec = SegmentSpec(name=name, nchan=256, f_lo_hz=1.0e9, bw_hz=1.0e9, nint=1024,
                           inttime_s=5e-3, npix=1024,
                           dm_list=dm_grid_smearing(1500.0, 128, 1.0e9, 1.0e9, 256, 5e-3),
                           dt_list=[1, 2, 4, 8], threshold=7.0, seed=s)
        spec.pulses = _random_pulses(rng, spec, 5, (50.0, 1000.0), (5e-3, 40e-3), (0.2, 1.0))
        return spec
    if name == "batching":
        spec = SegmentSpec(name=name, nchan=1024, f_lo_hz=1.0e9, bw_hz=1.0e9, nint=2048,
                           inttime_s=5e-3, npix=2048, dm_list=dm_grid_linear(3000.0, 256),
                           dt_list=[1, 2, 4, 8, 16], threshold=7.0, store="fp16", seed=s)
        spec.pulses = _random_pulses(rng, spec, 5, (50.0, 1000.0), (5e-3, 40e-3), (0.2, 1.0))
        return spec
    if name == "stress":
        spec = SegmentSpec(name=name, nchan=2048, f_lo_hz=1.0e9, bw_hz=2.0e9, nint=4096,
                           inttime_s=10e-3, npix=4096, dm_list=dm_grid_linear(3000.0, 512),
                           dt_list=[1, 2, 4, 8, 16, 32], threshold=7.0, store="fp16", seed=s)
        x, y = _pixel_offsets(rng, spec.npix, 1)
        # 100 x the Stokes-I per-component noise sigma (0.5)
        spec.continuum = [dict(amp=50.0, x=int(x[0]), y=int(y[0]))]
        spec.pulses = _random_pulses(rng, spec, 3, (50.0, 500.0), (10e-3, 40e-3), (0.2, 1.0))
        return spec
    if name == "serving":
        return serving_shapes(s)[0]
    raise KeyError(name)


def _random_pulses(rng, spec: SegmentSpec, k: int, dm_rng, w_rng, a_rng) -> List[Dict]:
    f = channel_freqs(spec.f_lo_hz, spec.bw_hz, spec.nchan) * 1e-9
    seg = spec.nint * spec.inttime_s
    xs, ys = _pixel_offsets(rng, spec.npix, k)
    out = []
    for i in range(k):
        dm = float(rng.uniform(*dm_rng))
        w = float(rng.uniform(*w_rng))
        amp = float(rng.uniform(*a_rng))
        sweep = K_DISP * dm * (f.min() ** -2 - f.max() ** -2)
        latest = seg - sweep - w - 2 * spec.inttime_s
        t0 = float(rng.uniform(0.0, max(latest, 0.0)))
        out.append(dict(dm=dm, t0_s=t0, width_s=w, amp=amp, x=int(xs[i]), y=int(ys[i])))
    return out


def serving_shapes(seed: int, count: int = 12) -> List[SegmentSpec]:
    """Mixed-shape segments: {64,256,1024} ch x {512,1024,2048} int x {512,1024,2048} px."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for k in range(count):
        nchan = int(rng.choice([64, 256, 1024]))
        nint = int(rng.choice([512, 1024, 2048]))
        npix = int(rng.choice([512, 1024, 2048]))
        dms = dm_grid_smearing(1500.0, None, 1.0e9, 1.0e9, nchan, 5e-3)
        spec = SegmentSpec(name=f"serving-{k}", nchan=nchan, f_lo_hz=1.0e9, bw_hz=1.0e9,
                           nint=nint, inttime_s=5e-3, npix=npix, dm_list=dms,
                           dt_list=[1, 2, 4], threshold=7.0, seed=seed * 1000 + k)
        prng = np.random.Generator(np.random.PCG64(spec.seed + 7919))
        spec.pulses = _random_pulses(prng, spec, 2, (50.0, 600.0), (5e-3, 20e-3), (0.3, 1.0))
        out.append(spec)
    return out


def _phases(bl_uvw: np.ndarray, freq_hz: np.ndarray, npix: int, cell: float, x: int, y: int):
    l = (x - npix // 2) * cell
    m = (y - npix // 2) * cell
    lam_inv = freq_hz / C_LIGHT
    ph = -2.0 * math.pi * (np.outer(bl_uvw[:, 0], lam_inv) * l + np.outer(bl_uvw[:, 1], lam_inv) * m)
    return np.exp(1j * ph)                                       # [nbl, nchan]


def make_segment(spec: SegmentSpec, nint: Optional[int] = None, t_start: int = 0) -> Dict:
    """Build the segment's inputs.

    Returns ``ant_uvw`` [nant, 3] (m), ``bl_uvw`` [nbl, 3] (m, for the signal
    model), ``freq_hz`` [nchan] and ``vis`` complex64 [nint, nbl, nchan, npol].
    ``t_start``/``nint`` select a window of the full segment: the noise stream
    is generated per integration block from the seed, so any window equals
    the matching slice of the whole segment.
    """
    n_total = spec.nint
    nint = n_total if nint is None else nint
    ant = array_uvw(spec.seed, spec.nant, spec.dec_deg)
    ii, jj = baseline_pairs(spec.nant)
    bl = ant[jj] - ant[ii]
    freq = channel_freqs(spec.f_lo_hz, spec.bw_hz, spec.nchan)
    nbl = bl.shape[0]
    vis = np.empty((nint, nbl, spec.nchan, spec.npol), dtype=np.complex64)
    _fill_noise(vis, spec, t_start)
    fg = freq * 1e-9
    ftop = fg.max()
    tint = spec.inttime_s
    for src in spec.continuum:
        ph = (src["amp"] * _phases(bl, freq, spec.npix, spec.cell_rad, src["x"], src["y"])).astype(np.complex64)
        vis += ph[None, :, :, None]
    for p in spec.pulses:
        ph = p["amp"] * _phases(bl, freq, spec.npix, spec.cell_rad, p["x"], p["y"])
        start = p["t0_s"] + K_DISP * p["dm"] * (fg ** -2 - ftop ** -2)   # [nchan]
        end = start + p["width_s"]
        k0 = np.floor(start / tint).astype(np.int64)
        k1 = np.floor(end / tint).astype(np.int64)
        for c in range(spec.nchan):
            for k in range(k0[c], k1[c] + 1):
                kk = k - t_start
                if kk < 0 or kk >= nint:
                    continue
                ov = min(end[c], (k + 1) * tint) - max(start[c], k * tint)
                if ov <= 0:
                    continue
                vis[kk, :, c, :] += (ph[:, c] * (ov / tint)).astype(np.complex64)[:, None]
    return dict(ant_uvw=ant, bl_uvw=bl, freq_hz=freq, vis=vis)


_NOISE_BLOCK = 16


def _fill_noise(vis: np.ndarray, spec: SegmentSpec, t_start: int):
    """Circular Gaussian noise, E|n|^2 = 1, generated in fixed 16-integration blocks."""
    nint, nbl, nchan, npol = vis.shape
    flat = vis.view(np.float32).reshape(nint, nbl * nchan * npol * 2)
    per = nbl * nchan * npol * 2
    b0 = t_start // _NOISE_BLOCK
    b1 = (t_start + nint + _NOISE_BLOCK - 1) // _NOISE_BLOCK
    scale = np.float32(math.sqrt(0.5))
    for blk in range(b0, b1):
        rng = np.random.Generator(np.random.PCG64([spec.seed, blk]))
        block = rng.standard_normal((_NOISE_BLOCK, per), dtype=np.float32)
        block *= scale
        lo = blk * _NOISE_BLOCK
        a = max(lo, t_start)
        b = min(lo + _NOISE_BLOCK, t_start + nint)
        flat[a - t_start:b - t_start] = block[a - lo:b - lo]
