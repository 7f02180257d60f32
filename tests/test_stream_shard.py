"""Streaming with checkpoint/resume and sharding across processes (host logic,
run on the CPU with the oracle as the computing backend; gloo for the
two-process sum)."""
import json
import os
import tempfile

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle as O
from paper_2601_17164_gb300 import workloads as W
from paper_2601_17164_gb300.stream import StreamRun, shard_range
from tests.helpers import oracle_objects


class OracleBackend:
    """The oracle behind the streaming interface (CPU)."""

    def __init__(self, w):
        self.w = w
        self.P, self.T, self.G = oracle_objects(w)
        self.n_bins = self.G.n_steps // self.G.n_out + 1

    def sample(self, first, count):
        w = self.w
        return O.sample_births_at(self.P, self.T, self.G, w.birth_mode, w.n, np.arange(first, first + count),
                                  w.n_t, w.n_k, w.sigma, w.kmax, w.seed)

    def dipole(self, births, d_len, d_vel):
        _, _, st = O.dipole(self.P, self.T, self.G, births, d_len, d_vel)
        return st


def _small():
    # H, 800 nm, 2 cycles, uniform/gaussian births: 600 births in chunks of 128
    return W.Workload("H 800nm 2cyc 600 births stream test", W.HYDROGEN, W.P1, dt=0.02, n=600,
                      sigma=W.adk_sigma(1e14, 0.5), seed=9)


def test_chunked_stream_equals_one_shot_and_resumes_after_interruption():
    w = _small()
    be = OracleBackend(w)
    full_l, full_v = np.zeros(be.n_bins), np.zeros(be.n_bins)
    be.dipole(be.sample(0, w.n), full_l, full_v)
    with tempfile.TemporaryDirectory() as d:
        log = os.path.join(d, "run.jsonl")
        r = StreamRun(w, be, chunk=128, checkpoint_dir=d, log_path=log)
        r.run(max_chunks=2)                     # "crash" after two chunks
        recs = [json.loads(x) for x in open(log)]
        assert [x["chunk"] for x in recs] == [0, 1] and all(x["count"] == 128 for x in recs)
        assert all(0.0 <= x["removed_fraction"] <= 1.0 and x["traj_steps"] > 0 for x in recs)
        assert not r.finished and r.state.next_chunk == 2
        r2 = StreamRun(w, be, chunk=128, checkpoint_dir=d)   # fresh process view
        assert r2.state.next_chunk == 2
        dl, dv = r2.run()
        assert r2.finished and r2.n_chunks == 5
        scale = np.max(np.abs(full_l))
        assert np.max(np.abs(dl - full_l)) < 1e-13 * scale
        assert np.max(np.abs(dv - full_v)) < 1e-13 * np.max(np.abs(full_v))
        # a checkpoint of another run is refused
        other = W.Workload(w.name + " other", w.target, w.pulse, w.dt, n=w.n, sigma=w.sigma, seed=w.seed)
        with pytest.raises(ValueError):
            StreamRun(other, be, chunk=128, checkpoint_dir=d)


def test_shard_ranges_cover_and_balance():
    n, world = 100000, 4
    rs = [shard_range(n, r, world) for r in range(world)]
    assert rs[0][0] == 0 and rs[-1][1] == n
    assert all(rs[k][1] == rs[k + 1][0] for k in range(world - 1))
    work = [sum(1 - i / n for i in range(lo, hi)) for lo, hi in rs]
    assert max(work) / min(work) < 1.01


def _rank(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w = _small()
    be = OracleBackend(w)
    lo, hi = shard_range(w.n, rank, world)
    r = StreamRun(w, be, chunk=100, lo=lo, hi=hi)
    dl, dv = r.run()
    t = torch.tensor(np.stack([dl, dv]))
    dist.all_reduce(t)                          # the one exchange: a sum of the bins
    if rank == 0:
        np.save(out, t.numpy())
    dist.destroy_process_group()


def test_two_process_shards_sum_to_unsharded_bins():
    w = _small()
    be = OracleBackend(w)
    full_l, full_v = np.zeros(be.n_bins), np.zeros(be.n_bins)
    be.dipole(be.sample(0, w.n), full_l, full_v)
    with tempfile.TemporaryDirectory() as d:
        out = os.path.join(d, "sum.npy")
        port = 29500 + (os.getpid() % 1000)
        mp.start_processes(_rank, args=(2, port, out), nprocs=2, join=True, start_method="spawn")
        got = np.load(out)
    assert np.max(np.abs(got[0] - full_l)) < 1e-13 * np.max(np.abs(full_l))
    assert np.max(np.abs(got[1] - full_v)) < 1e-13 * np.max(np.abs(full_v))
