"""Streaming of large birth samples with checkpoint and resume, and sharding.

A workload of n births (e.g. 1e8 for Ar, 2000 nm, 20 cycles) does not fit one
call: its births are produced and propagated in chunks of consecutive births
(birth-time order, since the sample is sorted by n0), and the dipole bins are
accumulated across chunks.  After every chunk the bins and the chunk index are
written to a checkpoint directory (`bins.npy` + `state.json`, replaced
atomically), so that an interrupted run resumes at the next chunk.  With
`log_path`, every chunk appends a JSON line with its counters (removed and
escalated trajectories, trajectory-steps and their rate).

The same chunking shards a sample across processes: `shard_range` gives each
rank a contiguous range of births with about equal trajectory-steps, and the
bins of the ranks are summed.

The computing backend is any object with
    sample(first, count) -> births        (births first .. first+count-1)
    dipole(births, d_len, d_vel) -> dict  (accumulates; returns counters)
    n_bins
`GpuBackend` drives the CUDA library through its C ABI.
"""
from __future__ import annotations

import json
import math
import os
import time
from dataclasses import dataclass
from typing import Optional

import numpy as np

from .workloads import Workload


def shard_range(n: int, rank: int, world: int):
    """Contiguous births [lo, hi) of rank `rank`, balanced in trajectory-steps.

    Births are sorted by birth time and spread over the pulse, so birth i lives
    for about (1 - i/n) of the grid: the cumulative work is x - x^2/2 at
    x = i/n, and rank r takes the births between x_r and x_{r+1} with
    x_k - x_k^2/2 = k/(2 world), x_k = 1 - sqrt(1 - k/world)."""
    if not (0 <= rank < world):
        raise ValueError("rank out of range")

    def cut(k):
        return n if k >= world else int(round(n * (1.0 - math.sqrt(1.0 - k / world))))
    return cut(rank), cut(rank + 1)


@dataclass
class StreamState:
    workload: str
    n: int
    chunk: int
    seed: int
    next_chunk: int = 0
    traj_steps: float = 0.0
    escalated: int = 0
    removed: int = 0


class StreamRun:
    """Chunked accumulation of the dipole bins of births [lo, hi) of an n-birth sample."""

    def __init__(self, workload: Workload, backend, chunk: int, checkpoint_dir: Optional[str] = None,
                 lo: int = 0, hi: Optional[int] = None, log_path: Optional[str] = None):
        self.w = workload
        self.backend = backend
        self.chunk = int(chunk)
        self.dir = checkpoint_dir
        self.log_path = log_path
        self.lo = int(lo)
        self.hi = int(workload.n if hi is None else hi)
        if self.chunk <= 0 or not (0 <= self.lo <= self.hi <= workload.n):
            raise ValueError("bad chunk or range")
        self.n_chunks = (self.hi - self.lo + self.chunk - 1) // self.chunk
        nb = backend.n_bins
        self.d_len = np.zeros(nb)
        self.d_vel = np.zeros(nb)
        self.state = StreamState(workload.name, workload.n, self.chunk, workload.seed)
        if self.dir:
            self._load()

    # -- checkpoint --------------------------------------------------------
    def _paths(self):
        return os.path.join(self.dir, "bins.npy"), os.path.join(self.dir, "state.json")

    def _load(self):
        bins_p, state_p = self._paths()
        if not os.path.exists(state_p):
            return
        with open(state_p) as fh:
            st = StreamState(**json.load(fh))
        if (st.workload, st.n, st.chunk, st.seed) != (self.w.name, self.w.n, self.chunk, self.w.seed):
            raise ValueError(f"checkpoint in {self.dir} belongs to another run: {st}")
        bins = np.load(bins_p)
        self.d_len[:], self.d_vel[:] = bins[0], bins[1]
        self.state = st

    def _save(self):
        os.makedirs(self.dir, exist_ok=True)
        bins_p, state_p = self._paths()
        tmp_b, tmp_s = bins_p + ".tmp.npy", state_p + ".tmp"
        np.save(tmp_b, np.stack([self.d_len, self.d_vel]))
        with open(tmp_s, "w") as fh:
            json.dump(self.state.__dict__, fh)
        os.replace(tmp_b, bins_p)       # bins first: a state never points past its bins
        os.replace(tmp_s, state_p)

    # -- run ---------------------------------------------------------------
    def run(self, max_chunks: Optional[int] = None):
        """Processes chunks from the checkpointed position on; returns (d_len, d_vel)."""
        done = 0
        while self.state.next_chunk < self.n_chunks:
            if max_chunks is not None and done >= max_chunks:
                break
            k = self.state.next_chunk
            first = self.lo + k * self.chunk
            count = min(self.chunk, self.hi - first)
            t_start = time.time()
            births = self.backend.sample(first, count)
            cnt = self.backend.dipole(births, self.d_len, self.d_vel)
            if self.log_path:
                # one JSON line per chunk: the chunk's counters and wall time
                wall = time.time() - t_start
                rec = {"workload": self.w.name, "chunk": k, "first": first, "count": count, "wall_s": wall,
                       "traj_steps": float(cnt.get("traj_steps", 0)),
                       "trajectory_steps_per_s": float(cnt.get("traj_steps", 0)) / wall if wall > 0 else None,
                       "removed": int(cnt.get("removed", 0)), "removed_fraction": int(cnt.get("removed", 0)) / count,
                       "escalated": int(cnt.get("escalated", 0)), "nonfinite": int(cnt.get("nonfinite", 0))}
                with open(self.log_path, "a") as fh:
                    fh.write(json.dumps(rec) + "\n")
            self.state.next_chunk = k + 1
            self.state.traj_steps += float(cnt.get("traj_steps", 0))
            self.state.escalated += int(cnt.get("escalated", 0))
            self.state.removed += int(cnt.get("removed", 0))
            if self.dir:
                self._save()
            done += 1
        return self.d_len, self.d_vel

    @property
    def finished(self) -> bool:
        return self.state.next_chunk >= self.n_chunks


class GpuBackend:
    """Backend on the CUDA library (current device); accumulates on the device per chunk.
    `prop` overrides propagation parameters (sfhk.prop_params keywords).  The mixed
    path's escalation floor and its large-contribution tier are relative to the
    largest amplitude of each call, i.e. of each chunk; with esc_floor = esc_big = 0
    the chunked bins equal one call over all births (up to summation order)."""

    def __init__(self, workload: Workload, precision: int, chunk: int, **prop):
        import torch

        from . import pipeline as PL
        from . import sfhk as S
        self.S, self.torch = S, torch
        self.w = workload
        self.field, self.target = PL.make_handles(workload)
        self.n_bins = self.field.info["n_bins"]
        self.births = S.Births.empty(chunk)
        self.pp = S.prop_params(precision, workload.gamma, workload.d_t, **prop)
        self.dl = torch.zeros(self.n_bins, dtype=torch.float64, device="cuda")
        self.dv = torch.zeros_like(self.dl)
        self.stats = S.new_stats()

    def sample(self, first, count):
        w = self.w
        self.S.sfhk_sample_births(self.field, self.target, w.birth_mode, w.n, self.births, w.n_t, w.n_k,
                                  w.sigma or 1.0, w.kmax or 1.0, w.seed, first=first, count=count)
        return (self.births, count)

    def dipole(self, births, d_len, d_vel):
        b, count = births
        self.dl.zero_()
        self.dv.zero_()
        self.stats.zero_()
        self.S.sfhk_dipole(self.field, self.target, b, count, self.pp, self.dl, self.dv, self.stats)
        d_len += self.dl.cpu().numpy()
        d_vel += self.dv.cpu().numpy()
        return self.S.stats_dict(self.stats)
