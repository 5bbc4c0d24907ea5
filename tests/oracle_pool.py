"""The FP64 oracle's image statistics over a spawn pool of all host cores.

Test infrastructure for the configuration-scale parity tests: the engine
searches whole segments, and the oracle computes the statistics of chosen
images one by one, in worker processes started with ``spawn`` (never forked
from a process that holds a CUDA context).  Stokes I of a window [a, b) of
integrations is put in shared memory once; every worker images its share of
the (d, s, t') list with ``oracle.OraclePlan.image`` and returns the
statistics and, for a tie check, the oracle's value at the engine's pixel.
"""

from __future__ import annotations

import multiprocessing as mp
import os
from multiprocessing import shared_memory

import numpy as np

import oracle


def _worker(args):
    shm_name, shape, plan_kw, a, nwin, items = args
    shm = shared_memory.SharedMemory(name=shm_name)
    try:
        S = np.ndarray(shape, dtype=np.complex128, buffer=shm.buf)
        op = oracle.OraclePlan(**plan_kw)
        out = []
        for (d, s, t, xe, ye) in items:
            dt = int(op.dt_list[s])
            # S starts at integration a (a multiple of every dt): t' counts from a / dt there
            I, W = op.image(S, d, s, t - a // dt, nint=nwin)
            st = op.stats(I)
            v = float(I[ye, xe]) if xe >= 0 else float("nan")
            out.append(((d, s, t), st, v, W))
            del I
        del S
        return out
    finally:
        shm.close()


class OraclePool:
    """A spawn pool of worker processes computing oracle image statistics."""

    def __init__(self, processes: int | None = None):
        self.processes = processes or os.cpu_count() or 1
        self.pool = mp.get_context("spawn").Pool(self.processes)

    def close(self):
        self.pool.close()
        self.pool.join()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def stats(self, vis, plan_kw, items, a=0, b=None, chunk=4096):
        """Oracle statistics of every listed image.

        vis: [nint][nbl][nchan][npol] complex64 of the whole segment; only the
        window [a, b) of integrations is read (a a multiple of every dt of the
        plan, and b past the last sample any listed image reads).  items:
        (d, s, t') or (d, s, t', x_engine, y_engine).  Returns a dict
        (d, s, t') -> (ImageStats, oracle value at the engine pixel, W).
        """
        nint = vis.shape[0]
        b = nint if b is None else min(b, nint)
        for dt in plan_kw["dt_list"]:
            assert a % int(dt) == 0, (a, dt)
        nbl, nchan = vis.shape[1], vis.shape[2]
        shape = (b - a, nbl, nchan)
        shm = shared_memory.SharedMemory(create=True, size=int(np.prod(shape)) * 16)
        try:
            S = np.ndarray(shape, dtype=np.complex128, buffer=shm.buf)
            for i0 in range(0, b - a, 64):
                i1 = min(b - a, i0 + 64)
                S[i0:i1] = oracle.stokes_i(vis[a + i0:a + i1])
            del S
            full = [tuple(it) + (-1, -1) if len(it) == 3 else tuple(it) for it in items]
            k = max(1, min(len(full), 4 * self.processes))
            jobs = [(shm.name, shape, plan_kw, a, b - a, full[i::k]) for i in range(k) if full[i::k]]
            res = self.pool.map(_worker, jobs, chunksize=1)
        finally:
            shm.close()
            shm.unlink()
        return {key: (st, v, W) for part in res for (key, st, v, W) in part}


def plan_kwargs(spec, seg, dm_list=None, dt_list=None, edge=None):
    """Keyword arguments of oracle.OraclePlan for a synthetic segment."""
    return dict(ant_uvw=seg["ant_uvw"], freq_hz=seg["freq_hz"], inttime_s=spec.inttime_s, npix=spec.npix,
                cell_rad=spec.cell_rad, dm_list=np.asarray(spec.dm_list if dm_list is None else dm_list),
                dt_list=list(spec.dt_list if dt_list is None else dt_list),
                threshold=spec.threshold, edge=spec.edge if edge is None else edge, npol=spec.npol,
                mean_subtract=bool(getattr(spec, "mean_subtract", False)),
                noise_clipped=bool(getattr(spec, "noise_clipped", False)))
