#!/usr/bin/env python
"""Throughput benchmark of the realfast search engine on GB300.

One step = one full segment search (every DM x dt x t' dirty image, peak,
noise, threshold, candidates) of the ``batching`` workload: 351 baselines,
1024 channels over 1-2 GHz, 2048 x 5 ms integrations stored in FP16, 256 DM
trials 0-3000, dt {1,2,4,8,16}, 2048^2 images: 553,095 images per segment.
The segment (11.8 GB of complex64 visibilities) is far larger than L2, so
the inputs are not L2-resident between steps.  ``--config realtime`` times
the 1024^2 workload (177,521 images) instead; by default its images/s are
also reported under the key ``realtime``.

``value``: dirty images per second with the segment resident in HBM.
``e2e``: the same metric through the same C-ABI call with the segment in
pinned host memory (host-to-device copies inside the timed region).
``roofline``: the dominant kernel's algorithmic HBM bytes per launch over
its average launch time, from CUDA events recorded around each of its
launches during the timed region, against the measured copy bandwidth; its
FP32 issue rate against the derived ALU peak rides along under ``alu``.
``cpu_baseline``: the FP64 oracle on a bounded sample of the same images on
the host cores (a reported baseline, not the target).

``--impl reference`` times the oracle alone on the host cores, each step a
bounded sample of the same workload.

Multi-GPU (torchrun): every rank searches its own segment (weak scaling, no
data-path collective); timing is the max over ranks.
"""

from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "dirty images/sec (DM×dt×int) and visibility GB/s vs HBM peak; p99 latency/real-time"
UNIT = "images/s"
FP32_LANES_PER_SM = 128


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="engine", choices=["engine", "reference"])
    ap.add_argument("--config", default=None,
                    help="workload (default: batching; realtime for --next-rows)")
    ap.add_argument("--no-realtime-extra", action="store_true",
                    help="do not also time the realtime workload under the key `realtime`")
    ap.add_argument("--form", default="batched", choices=["batched", "plain"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--wave-images", type=int, default=0, help="images per wave (0 = engine default)")
    ap.add_argument("--no-plain", action="store_true", help="skip timing the plain per-trial form")
    ap.add_argument("--no-autotune", action="store_true", help="keep the engine's default tuning")
    ap.add_argument("--fused", type=int, default=-1, choices=[-1, 0, 1],
                    help="force the fused imaging pass off (0) or on (1); -1: the autotuner's or default choice")
    ap.add_argument("--ring", type=int, default=0, help="chunk slots of the fused pass's ring (0: default)")
    ap.add_argument("--overlap", type=int, default=-1, choices=[-1, 0, 1],
                    help="force overlapped waves off (0) or on (1); -1: the autotuner's or default choice")
    ap.add_argument("--tune-cache", default=os.path.expanduser("~/.cache/realfast_gb300/tune.json"))
    ap.add_argument("--serving", action="store_true",
                    help="Poisson stream of mixed-shape segments at 1.0x real time through rf_server_*")
    ap.add_argument("--serving-segments", type=int, default=16)
    ap.add_argument("--serving-slots", type=int, default=3)
    ap.add_argument("--serving-load", type=float, default=1.0, help="offered load in units of real time")
    ap.add_argument("--next-rows", action="store_true",
                    help="time the periodicity search, stream, mean subtraction, clipped noise and candidate products")
    ap.add_argument("--host-input", action="store_true",
                    help="time the search from pinned host input only (small device footprint for profilers)")
    ap.add_argument("--nchan", type=int, default=0,
                    help="search the workload with this many channels over the same band (a smaller device "
                         "footprint for profilers; 0 = the workload's own)")
    ap.add_argument("--write-traffic", metavar="RAW_CSV",
                    help="write profiles/traffic.json from `ncu -i <rep> --page raw --csv` output of the imaging "
                         "kernels (no GPU needed) and exit")
    ap.add_argument("--traffic-images", type=int, default=256, help="images per captured launch (the wave size)")
    ap.add_argument("--traffic-command", default="", help="the ncu command the capture came from")
    return ap.parse_args()


# ----------------------------------------------------------- multi-rank --
def rank_seed(seed, rank):
    """Seed of rank `rank`'s segment: every rank searches its own segment."""
    return seed + 1000 * rank


def max_over_ranks(value, dist, device):
    """The slowest rank's time, returned on every rank (no-op without dist)."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(world, steps, units_per_rank, ms):
    """Whole-job throughput: the units all ranks processed over the slowest rank's time."""
    return world * steps * units_per_rank / (ms / 1e3)


def peaks():
    """HBM copy bandwidth (GB/s) and the maximum SM clock (MHz), measured
    on the GB300s when MEASURED_PEAKS.json is present."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            m = json.load(f)
        return float(m["hbm_gbs"]), float(m.get("sm_max_mhz", 2070.0)), "measured"
    except Exception:
        return 6800.0, 2070.0, "fallback"


# ------------------------------------------------------------------ clocks --
class Clocks:
    """nvidia-smi sampling of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", str(self.index)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out = ""
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# -------------------------------------------------------------- CPU oracle --
def _oracle_worker(args):
    import numpy as np
    from multiprocessing import shared_memory
    import oracle
    (shm_name, shape, plan_kw, items) = args
    shm = shared_memory.SharedMemory(name=shm_name)
    try:
        S = np.ndarray(shape, dtype=np.complex128, buffer=shm.buf)
        op = oracle.OraclePlan(**plan_kw)
        out = []
        for (d, s, t) in items:
            I, W = op.image(S, d, s, t)
            st = oracle.image_stats(I)
            out.append((d, s, t, st.peak, st.sigma, st.x, st.y))
        del S
        return out
    finally:
        shm.close()


class OracleRunner:
    """The FP64 oracle, as it stands, over a spawn pool of all host cores."""

    def __init__(self, spec, seg):
        import numpy as np
        import multiprocessing as mp
        from multiprocessing import shared_memory
        import oracle
        self.np = np
        S = oracle.stokes_i(seg["vis"])
        self.shm = shared_memory.SharedMemory(create=True, size=S.nbytes)
        buf = np.ndarray(S.shape, dtype=np.complex128, buffer=self.shm.buf)
        buf[...] = S
        self.shape = S.shape
        del S, buf
        self.plan_kw = dict(ant_uvw=seg["ant_uvw"], freq_hz=seg["freq_hz"], inttime_s=spec.inttime_s,
                            npix=spec.npix, cell_rad=spec.cell_rad, dm_list=spec.dm_list, dt_list=spec.dt_list,
                            threshold=spec.threshold, edge=spec.edge)
        op = oracle.OraclePlan(**self.plan_kw)
        self.images = op.image_list(spec.nint)
        self.cores = os.cpu_count() or 1
        self.pool = mp.get_context("spawn").Pool(self.cores)
        self.rng = np.random.default_rng(12345)

    def sample(self, n):
        idx = self.rng.choice(len(self.images), size=n, replace=False)
        return [self.images[i] for i in sorted(idx)]

    def run(self, items):
        chunks = [items[i::self.cores] for i in range(self.cores)]
        jobs = [(self.shm.name, self.shape, self.plan_kw, c) for c in chunks if c]
        t0 = time.perf_counter()
        res = self.pool.map(_oracle_worker, jobs)
        return time.perf_counter() - t0, [r for part in res for r in part]

    def close(self):
        self.pool.close()
        self.pool.join()
        self.shm.close()
        self.shm.unlink()


def cpu_baseline(spec, seg, seconds):
    run = OracleRunner(spec, seg)
    try:
        run.run(run.sample(run.cores))                      # warm the workers
        t1, _ = run.run(run.sample(run.cores))              # one image per core: per-image time
        n = max(run.cores, int(run.cores * seconds / max(t1, 1e-3)))
        n = min(n, len(run.images))
        t, _ = run.run(run.sample(n))
        return {"value": n / t, "unit": UNIT, "cores": run.cores, "kind": "oracle",
                "sample": f"{n} images drawn uniformly (seed 12345) from the {len(run.images)} (DM, dt, t') "
                          f"images of the {spec.name} segment, FP64 numpy, {t:.1f} s wall"}
    finally:
        run.close()


# ------------------------------------------------------------ work counts --
def dt1_fraction(plan, spec, nint):
    """Fraction of the segment's images at dt = 1 (counted from the plan's
    delay table and edge rule): those gather the stored samples, the others
    the FP32 resampled series."""
    import numpy as np
    maxd = plan.delays().max(axis=1)
    n = {}
    for dt in spec.dt_list:
        if spec.edge == "partial":
            n[dt] = len(maxd) * (nint // dt)
        else:
            n[dt] = int(np.sum(np.maximum(nint - maxd, 0) // dt))
    tot = sum(n.values())
    return n.get(1, 0) / tot if tot else 1.0


def work_per_image(spec, info, frac_dt1):
    """Algorithmic HBM bytes and FP32 flops per image of each imaging kernel
    (columns beyond the longest baseline are pruned: ncol = iu_max + 1).

    grid_cells: one sample per gridding entry read (dt = 1: the stored
    sample, 4 B FP16 or 8 B FP32; dt > 1: the FP32 resampled sum, 8 B) and
    one 8-byte cell value written per occupied cell.
    grid_colfft (the column FFTs): cells read, column-FFT output T (8 N ncol
    B) written; ncol length-N FFTs.
    rowfft_stats: T read once; N/2 length-N FFTs (two image rows per complex
    transform).  FFTs count 5 N log2 N flops.
    image_fused (the column and row passes in one launch): the same bytes and
    flops as grid_colfft and rowfft_stats together -- T counted written and
    read once, as the byte model of a two-pass FFT does, although the fused
    pass keeps it in an L2-resident ring (its DRAM traffic, from ncu, is far
    lower).
    """
    N = spec.npix
    ncol = info.iu_max + 1
    esz1 = 4 if spec.store == "fp16" else 8
    gather = (frac_dt1 * esz1 + (1.0 - frac_dt1) * 8) * info.n_entries
    fft = 5.0 * N * math.log2(N)
    return {
        "grid_cells": {"bytes": gather + 8 * info.n_cells, "flops": 0.0},
        "grid_colfft": {"bytes": 8 * info.n_cells + 8 * N * ncol, "flops": ncol * fft},
        "rowfft_stats": {"bytes": 8 * N * ncol, "flops": (N / 2) * fft},
        "image_fused": {"bytes": 8 * info.n_cells + 16 * N * ncol, "flops": (ncol + N / 2) * fft},
    }


def fp32_peak_tflops(sms, mhz):
    return sms * FP32_LANES_PER_SM * 2 * mhz * 1e6 / 1e12


def load_traffic(kernel, images_per_launch):
    """DRAM bytes per launch from the committed ncu summary, scaled to this
    launch's images; None if the summary is missing or was taken from other
    kernel sources."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            t = json.load(f)
    except (OSError, ValueError):
        return None
    k = t.get("kernels", {}).get(kernel)
    if not k or t.get("source_hash") != source_hash():
        return None
    return k["dram_bytes_per_image"] * images_per_launch


KERNEL_SOURCES = ("rf_async.cuh", "rf_fft.cuh", "rf_image.cuh", "rf_image_small.cu", "rf_image_large.cu",
                  "rf_image_fused.cu", "rf_kernels.cu")


def source_hash():
    """Hash of the sources of the search kernels whose DRAM traffic the
    committed ncu summary records."""
    import hashlib
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1802_03084_gb300", "csrc")
    for name in KERNEL_SOURCES:
        with open(os.path.join(csrc, name), "rb") as f:
            h.update(name.encode() + f.read())
    return h.hexdigest()[:16]


TRAFFIC_KERNELS = (("k_grid_cells", "grid_cells"), ("k_colfft", "grid_colfft"), ("k_rowfft_stats", "rowfft_stats"),
                   ("k_image_fused", "image_fused"))
_BYTE_UNITS = {"byte": 1.0, "kbyte": 1e3, "mbyte": 1e6, "gbyte": 1e9, "tbyte": 1e12}


def write_traffic(raw_csv, images_per_launch, command, workload, path=None):
    """profiles/traffic.json (or `path`) from an ncu raw-page CSV (header row,
    unit row, one row per captured launch): DRAM read + write bytes per launch
    of each imaging kernel, averaged over its captured launches, and per image."""
    import csv
    with open(raw_csv, newline="") as f:
        rows = [r for r in csv.reader(f) if r]
    hdr = next(i for i, r in enumerate(rows) if "Kernel Name" in r)
    names, units = rows[hdr], rows[hdr + 1]
    data = [r for r in rows[hdr + 2:] if len(r) == len(names)]  # launch rows (not ncu's notes)
    col = {n: i for i, n in enumerate(names)}

    def value(r, metric):
        i = col[metric]
        return float(r[i].replace(",", "")) * _BYTE_UNITS[units[i].strip().lower()]

    out = {}
    for pattern, key in TRAFFIC_KERNELS:
        per = [value(r, "dram__bytes_read.sum") + value(r, "dram__bytes_write.sum")
               for r in data if pattern in r[col["Kernel Name"]]]
        if per:
            b = sum(per) / len(per)
            out[key] = {"dram_bytes_per_launch": b, "images_per_launch": images_per_launch,
                        "dram_bytes_per_image": b / images_per_launch, "launches_captured": len(per)}
    doc = {"source_hash": source_hash(), "workload": workload, "command": command, "kernels": out}
    path = path or os.path.join(ROOT, "profiles", "traffic.json")
    with open(path, "w") as f:
        json.dump(doc, f, indent=1)
        f.write("\n")
    return doc


def roofline(prof, spec, info, n_images, steps, frac_dt1, hbm_peak, peak_kind, sms, sm_mhz, step_ms):
    """The dominant kernel's roofline on HBM: its algorithmic bytes per
    launch (work_per_image x images per launch) over its average launch time
    (CUDA events around every launch in the timed region), against the
    measured copy bandwidth.  Its FP32 rate against the derived ALU peak, and
    the whole step's algorithmic bytes over the step time, ride along."""
    work = work_per_image(spec, info, frac_dt1)
    alu_peak = fp32_peak_tflops(sms, sm_mhz)
    per = {}
    for name, w in work.items():
        launches, ms = prof.get(name, (0, 0.0))
        if launches == 0:
            continue
        imgs = n_images * steps / launches
        avg_s = ms / launches / 1e3
        per[name] = dict(launches=launches, total_ms=ms, avg_us=avg_s * 1e6, images_per_launch=imgs,
                         bytes_per_image=w["bytes"], gbs=w["bytes"] * imgs / avg_s / 1e9,
                         hbm_frac=w["bytes"] * imgs / avg_s / 1e9 / hbm_peak,
                         tflops=w["flops"] * imgs / avg_s / 1e12)
    if not per:
        return None, per
    dom = max(per, key=lambda k: per[k]["total_ms"])
    d = per[dom]
    traffic = load_traffic(dom, d["images_per_launch"])
    # the step's bytes: gridding, then the fused pass or the two passes it replaces
    step_kernels = ["grid_cells"] + (["image_fused"] if "image_fused" in per else ["grid_colfft", "rowfft_stats"])
    step_bytes = sum(work[k]["bytes"] for k in step_kernels) * n_images
    r = {"bound": "hbm", "achieved": round(d["gbs"], 1), "peak": hbm_peak, "unit": "GB/s",
         "frac": round(d["gbs"] / hbm_peak, 4), "traffic": traffic, "kernel": dom,
         "peak_source": f"MEASURED_PEAKS.json hbm_gbs ({peak_kind}, copy bandwidth)",
         "bytes_per_image": round(d["bytes_per_image"]),
         "bytes_model": "pruned algorithmic bytes: see work_per_image",
         "avg_launch_us": round(d["avg_us"], 2), "images_per_launch": round(d["images_per_launch"], 1),
         "alu": {"achieved": round(d["tflops"], 3), "peak": round(alu_peak, 2), "unit": "TFLOP/s",
                 "frac": round(d["tflops"] / alu_peak, 4),
                 "peak_source": f"derived: {sms} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 flop x {sm_mhz:.0f} MHz",
                 "flops_model": "5 N log2 N per length-N complex FFT"},
         "step": {"bytes_per_image": round(step_bytes / max(n_images, 1)),
                  "gbs": round(step_bytes / (step_ms / 1e3) / 1e9, 1),
                  "frac": round(step_bytes / (step_ms / 1e3) / 1e9 / hbm_peak, 4)}}
    return r, per


# ---------------------------------------------------------------- reference --
def run_reference(args, rank, world):
    if rank != 0:
        return 0
    import numpy as np
    import synth
    spec = synth.config(args.config)
    seg = synth.make_segment(spec)
    run = OracleRunner(spec, seg)
    try:
        n = run.cores * 8   # about 0.3 s of oracle work per step
        for _ in range(args.warmup):
            run.run(run.sample(n))
        t_total = 0.0
        for _ in range(args.steps):
            t, _ = run.run(run.sample(n))
            t_total += t
        value = args.steps * n / t_total
        sample = f"{n} images per step drawn uniformly from the {len(run.images)} images of the {spec.name} segment"
        line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_total / args.steps * 1e3,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic", "config": {"workload": workload_name(spec)},
                "cpu_baseline": {"value": value, "unit": UNIT, "cores": run.cores, "kind": "oracle",
                                 "sample": sample},
                "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
    finally:
        run.close()
    return 0


def workload_name(spec):
    return (f"{spec.name}: 351 baselines x {spec.nchan} ch ({spec.f_lo_hz/1e9:.1f}-{(spec.f_lo_hz+spec.bw_hz)/1e9:.1f}"
            f" GHz) x {spec.nint} x {spec.inttime_s*1e3:g} ms, {len(spec.dm_list)} DM trials "
            f"0-{spec.dm_list.max():.0f}, dt {list(spec.dt_list)}, {spec.npix}^2 images, "
            f"{'FP16' if spec.store == 'fp16' else 'FP32'} storage")


# ------------------------------------------------------------------ serving --
def run_serving(args):
    """Segments of the serving shape set arrive as a Poisson process whose
    rate makes the offered data rate `load` times real time; each is
    submitted at its arrival time and its latency (arrival to candidates on
    the host) is compared with its own duration."""
    import numpy as np
    import torch
    import synth
    import paper_1802_03084_gb300 as rf
    from paper_1802_03084_gb300.build import build

    build()
    rf.lib()
    torch.cuda.init()
    shapes = synth.serving_shapes(104, count=args.serving_segments)
    durations = np.array([sp.nint * sp.inttime_s for sp in shapes])
    rng = np.random.default_rng(2024)
    gaps = rng.exponential(durations.mean() / args.serving_load, size=len(shapes))
    arrivals = np.cumsum(gaps) - gaps[0]
    # one visibility buffer per (channels, integrations) class: same-class
    # segments share data (the work is the same); generated before the clock starts
    data = {}
    items = []
    for sp in shapes:
        key = (sp.nchan, sp.nint)
        if key not in data:
            data[key] = synth.make_segment(sp)
        seg = data[key]
        desc = rf.make_desc(seg["ant_uvw"], seg["freq_hz"], sp.inttime_s, sp.npix, sp.cell_rad, sp.dm_list,
                            sp.dt_list, sp.threshold, max_nint=sp.nint)
        items.append((sp, seg, desc))
    free, total = torch.cuda.mem_get_info()
    budget = int(free * 0.8)
    lat, ratio, images, vis_bytes = [], [], 0, 0
    with rf.Server(device=0, slots=args.serving_slots, hbm_budget_bytes=budget) as sv:
        # warm: one pass over the distinct shapes so plans and code are resident
        t_warm = time.perf_counter()
        seen = set()
        for sp, seg, desc in items:
            k = (sp.nchan, sp.nint, sp.npix)
            if k not in seen:
                seen.add(k)
                sv.results(sv.submit(desc, seg["vis"], sp.nint))
        warm_s = time.perf_counter() - t_warm
        t0 = time.perf_counter()
        tickets = []
        for (sp, seg, desc), at in zip(items, arrivals):
            delay = t0 + at - time.perf_counter()
            if delay > 0:
                time.sleep(delay)
            tickets.append(sv.submit(desc, seg["vis"], sp.nint))
        infos = [sv.wait(t) for t in tickets]
        t_end = time.perf_counter()
        for t in tickets:
            sv.results(t)
    for (sp, seg, desc), info in zip(items, infos):
        l = info["done_s"] - info["submit_s"]
        lat.append(l)
        ratio.append(l / (sp.nint * sp.inttime_s))
        images += info["n_images"]
        vis_bytes += seg["vis"].nbytes
    wall = t_end - t0
    line = {"metric": "serving: p99 segment latency / segment duration (Poisson stream at %.2fx real time)"
                      % args.serving_load,
            "value": float(np.percentile(ratio, 99)), "unit": "latency / duration", "higher_is_better": False,
            "n_gpus": 1, "segments": len(items), "slots": args.serving_slots,
            "p50_latency_s": float(np.percentile(lat, 50)), "p99_latency_s": float(np.percentile(lat, 99)),
            "p50_latency_over_duration": float(np.percentile(ratio, 50)),
            "p99_latency_over_duration": float(np.percentile(ratio, 99)),
            "max_latency_over_duration": float(np.max(ratio)),
            "offered_segment_seconds": float(durations.sum()), "wall_s": wall, "warm_s": warm_s,
            "sustained_visibility_gbs": vis_bytes / wall / 1e9, "images_per_s": images / wall,
            "hbm_budget_gb": budget / 1e9, "data": "synthetic",
            "config": {"workload": "serving: {64,256,1024} ch x {512,1024,2048} x 5 ms x {512,1024,2048}^2 px, "
                                   "351 baselines, DM trials by the smearing criterion to 1500, dt {1,2,4}",
                       "shapes": [[sp.nchan, sp.nint, sp.npix, len(sp.dm_list)] for sp in shapes]},
            "per_segment": [{"nchan": sp.nchan, "nint": sp.nint, "npix": sp.npix, "latency_s": round(l, 3),
                             "duration_s": sp.nint * sp.inttime_s, "images": int(i["n_images"]),
                             "plan_reused": int(i["plan_reused"])}
                            for (sp, _, _), l, i in zip(items, lat, infos)]}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------- engine --
def run_next_rows(args):
    """Times the rows around the search on the same segment (one GPU, events on
    the default stream): the periodicity search, the overlapping-segment
    stream, mean subtraction and candidate products.  One JSON line."""
    import numpy as np
    import torch
    import synth
    import paper_1802_03084_gb300 as rf
    from paper_1802_03084_gb300.build import build
    build()
    rf.lib()
    spec = synth.config(args.config)
    seg = synth.make_segment(spec)
    nint = spec.nint
    vis = torch.from_numpy(seg["vis"]).cuda()
    torch.cuda.synchronize()

    def timed(fn, reps):
        fn()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            out = fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps, out

    def kernel_ms(p, name):
        """CUDA-event time of one kind of launch in one profiled search (graph bypassed)."""
        p.set_profiling(True)
        p.search(vis, nint)
        torch.cuda.synchronize()
        launches, total = p.profile().get(name, (0, 0.0))
        p.set_profiling(False)
        return total

    line = {"metric": "rows around the search", "config": {"workload": workload_name(spec)}, "n_gpus": 1}
    plan = rf.Plan.from_spec(spec, seg["ant_uvw"], seg["freq_hz"], max_nint=nint)
    n_images = plan.count_images(nint)
    ms, cands = timed(lambda: plan.search(vis, nint), 3)
    line["search_ms"] = ms
    line["rowfft_stats_kernel_ms"] = kernel_ms(plan, "rowfft_stats")
    # periodicity: L = 64, k = 1 .. 32 over every DM trial whose window fits
    L, kmin, kmax = 64, 1, 32
    pms, (pc, pst) = timed(lambda: plan.periodicity_search(vis, L, kmin, kmax, 7.0, nint, with_stats=True), 3)
    line["periodicity"] = {"L": L, "k": [kmin, kmax], "pairs": int(len(pst)), "power_images": int(2 * len(pst)),
                           "ms": pms, "images_per_s": 2 * len(pst) / (pms / 1e3), "candidates": int(len(pc))}
    # candidate products of up to 64 candidates
    c64 = cands[np.argsort(-cands["snr"])[:64]] if len(cands) else cands
    if len(c64):
        cms, _ = timed(lambda: plan.candidate_products(vis, c64, nint), 2)
        line["candidate_products"] = {"candidates": int(len(c64)), "ms": cms}
    plan.close()
    # mean subtraction on the same search
    spec_m = synth.config(args.config)
    spec_m.mean_subtract = True
    plan_m = rf.Plan.from_spec(spec_m, seg["ant_uvw"], seg["freq_hz"], max_nint=nint)
    mms, _ = timed(lambda: plan_m.search(vis, nint), 3)
    line["mean_subtract"] = {"ms": mms, "overhead_ms": mms - ms,
                             "kernel_ms": kernel_ms(plan_m, "mean_subtract")}
    plan_m.close()
    # clipped noise (one 5-sigma clipping pass) on the same search
    spec_c = synth.config(args.config)
    spec_c.noise_clipped = True
    plan_c = rf.Plan.from_spec(spec_c, seg["ant_uvw"], seg["freq_hz"], max_nint=nint)
    cms_, cc = timed(lambda: plan_c.search(vis, nint), 3)
    line["noise_clipped"] = {"ms": cms_, "overhead_ms": cms_ - ms, "candidates": int(len(cc)),
                             "candidates_plain_noise": int(len(cands)),
                             "clip_window_kernel_ms": kernel_ms(plan_c, "clip_window"),
                             "rowfft_stats_kernel_ms": kernel_ms(plan_c, "rowfft_stats")}
    plan_c.close()
    # stream: segments of nint integrations overlapping by the longest sweep,
    # fed the same segment repeatedly in chunks of 128 integrations
    plan_s = rf.Plan.from_spec(spec, seg["ant_uvw"], seg["freq_hz"], max_nint=nint)
    overlap = int(plan_s.info().max_delay)
    lcm = int(np.lcm.reduce(spec.dt_list))
    stride = (nint - overlap) // lcm * lcm
    reps = 4
    with rf.Stream(plan_s, stride) as st:
        st.push(vis, nint)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(reps):
            for c0 in range(0, nint, 128):
                st.push(vis[c0:c0 + 128], min(128, nint - c0))
        t1 = time.perf_counter()
        info = st.info()
        st.pop()
    plan_s.close()
    ints = reps * nint
    line["stream"] = {"stride": stride, "overlap": overlap, "segment_nint": stride + overlap,
                      "integrations_per_s": ints / (t1 - t0),
                      "realtime_factor": ints * spec.inttime_s / (t1 - t0), "segments": int(info["segments"])}
    print(json.dumps(line))
    return 0


def time_search(plan, vis, nint, steps, dist):
    """CUDA-event time (ms, max over ranks) of `steps` back-to-back searches."""
    import torch
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        out = plan.search(vis, nint)
    e1.record()
    torch.cuda.synchronize()
    return max_over_ranks(e0.elapsed_time(e1), dist, "cuda"), out


def run_workload(args, config, rank, world, dist, local_rank, lite=False):
    """One workload's bench fields.  `lite`: images/s, the roofline and the
    realtime factor only (no e2e, plain form or CPU baseline)."""
    import numpy as np
    import torch
    import synth
    import paper_1802_03084_gb300 as rf

    spec = synth.config(config)
    if args.nchan:
        spec.nchan = args.nchan
    spec.seed = rank_seed(spec.seed, rank)   # each rank searches its own segment
    seg = synth.make_segment(spec)
    nint = spec.nint
    want_e2e = not args.no_e2e and not lite
    vis_pin = torch.from_numpy(seg["vis"]).pin_memory() if (want_e2e or args.host_input) else None
    vis_dev = vis_pin if args.host_input else torch.from_numpy(seg["vis"]).cuda()
    torch.cuda.synchronize()
    plan = rf.Plan.from_spec(spec, seg["ant_uvw"], seg["freq_hz"], max_nint=nint, device=local_rank)
    if args.form == "plain":
        plan.set_form(rf.RF_FORM_PLAIN)
    tuning = None
    if args.wave_images:
        plan.set_wave_images(args.wave_images)
    elif not args.no_autotune and args.form == "batched":
        tuning = plan.autotune(vis_dev, nint, cache_path=args.tune_cache)
    if args.fused >= 0:
        plan.set_fused(bool(args.fused))
    if args.overlap >= 0:
        plan.set_overlap(bool(args.overlap))
    if args.ring:
        plan.set_ring(args.ring)
    info = plan.info()
    n_images = plan.count_images(nint)
    frac_dt1 = dt1_fraction(plan, spec, nint)
    warmup = max(args.warmup, 0)
    steps = args.steps if not lite else max(3, min(args.steps, 5))
    for _ in range(warmup):
        cands = plan.search(vis_dev, nint)
    plan.set_profiling(True)
    clocks = Clocks(local_rank)
    clocks.start()
    time.sleep(0.3)
    ms, cands = time_search(plan, vis_dev, nint, steps, dist)
    clk = clocks.stop()
    prof = plan.profile()
    plan.set_profiling(False)
    n_cand = len(cands)

    e2e = None
    if vis_pin is not None and want_e2e:
        plan.search(vis_pin, nint)
        ems, c2 = time_search(plan, vis_pin, nint, steps, dist)
        e2e = {"value": job_rate(world, steps, n_images, ems), "unit": UNIT,
               "h2d_bytes_per_step": int(seg["vis"].nbytes),
               "d2h_bytes_per_step": int(4 + len(c2) * rf.CANDIDATE_DTYPE.itemsize),
               "ms_per_step": ems / steps, "api": "rf_search_segment from pinned host memory"}

    # the same segment without per-kernel events (graph replay), and the
    # plain one-launch-set-per-trial form on the same GPU
    plan.search(vis_dev, nint)
    gms, _ = time_search(plan, vis_dev, nint, steps, dist)
    graph_value = job_rate(world, steps, n_images, gms)
    plain = None
    if not args.no_plain and args.form == "batched" and not lite:
        plan.set_form(rf.RF_FORM_PLAIN)
        plan.search(vis_dev, max(1, nint // 4))   # allocates the plain form's buffers
        pms, _ = time_search(plan, vis_dev, nint, 1, dist)
        plain = {"value": job_rate(world, 1, n_images, pms), "unit": UNIT, "ms_per_step": pms, "steps": 1,
                 "form": "one unfused launch set per (DM, dt) trial, intermediates in HBM"}
        plan.set_form(rf.RF_FORM_BATCHED)

    hbm_peak, sm_max_mhz, peak_kind = peaks()
    sms = torch.cuda.get_device_properties(local_rank).multi_processor_count
    roof, per_kernel = roofline(prof, spec, info, n_images, steps, frac_dt1, hbm_peak, peak_kind, sms,
                                clk.get("sm_max_mhz") or sm_max_mhz, ms / steps)
    launches = sum(v[0] for k, v in prof.items() if k != "h2d_copy")
    value = job_rate(world, steps, n_images, ms)
    seg_s = nint * spec.inttime_s
    out = {
        "value": value, "steps": steps, "warmup": warmup, "ms_per_step": ms / steps,
        "dtype": "f32" if spec.store != "fp16" else "f16-storage/f32",
        "config": {"workload": workload_name(spec), "images_per_step": n_images, "form": args.form,
                   "wave_images": plan.wave_images(), "input": "pinned host" if args.host_input else "HBM",
                   "autotune": tuning,
                   "l2": f"inputs larger than L2 ({seg['vis'].nbytes / 1e9:.2f} GB segment per step)",
                   "parallelism": f"dp{world} (one segment per GPU)"},
        "visibility_gbs": world * steps * seg["vis"].nbytes / (ms / 1e3) / 1e9,
        "realtime_factor": seg_s / (ms / steps / 1e3),
        "segment_latency_ms": ms / steps,
        "segment_duration_ms": seg_s * 1e3,
        "candidates_per_step": n_cand,
        "roofline": roof,
        "kernels": {k: {kk: (round(vv, 4) if isinstance(vv, float) else vv) for kk, vv in v.items()}
                    for k, v in per_kernel.items()},
        "kernel_source_hash": source_hash(),
        "e2e": e2e,
        "graph_replay_value": graph_value,
        "plain_form": plain,
        "batched_over_plain": (value / plain["value"]) if plain else None,
        "gpu_launches": int(launches),
        "clocks": clk,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline and not lite:
        out["cpu_baseline"] = cpu_baseline(spec, seg, args.cpu_seconds)
    plan.close()
    del vis_dev, vis_pin, seg
    torch.cuda.empty_cache()
    return out


def main():
    args = parse()
    if args.config is None:
        args.config = "realtime" if args.next_rows else "batching"
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.write_traffic:
        doc = write_traffic(args.write_traffic, args.traffic_images, args.traffic_command,
                            f"{args.config}, {args.traffic_images}-image waves, pinned host input")
        print(json.dumps(doc))
        return 0
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.serving:
        return run_serving(args) if rank == 0 else 0
    if args.next_rows:
        return run_next_rows(args) if rank == 0 else 0

    import torch
    import paper_1802_03084_gb300 as rf
    from paper_1802_03084_gb300.build import build

    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    if rank == 0:
        build()
    if dist:
        dist.barrier()
    rf.lib()

    main_fields = run_workload(args, args.config, rank, world, dist, local_rank)
    extra = None
    if args.config == "batching" and not args.no_realtime_extra and not args.nchan and not args.host_input:
        r = run_workload(args, "realtime", rank, world, dist, local_rank, lite=True)
        extra = {k: r[k] for k in ("value", "ms_per_step", "steps", "realtime_factor", "roofline", "kernels",
                                   "graph_replay_value", "clocks", "config", "dtype")}
        extra["unit"] = UNIT
    line = {"metric": METRIC, "value": main_fields["value"], "unit": UNIT, "n_gpus": world,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "data": "synthetic"}
    line.update(main_fields)
    if extra is not None:
        line["realtime"] = extra
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
