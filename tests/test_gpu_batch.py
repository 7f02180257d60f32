"""Batched configurations in one persistent launch (sfhk_batch_*) against the
single-configuration path and the oracle; CUDA-graph capture of a run."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2601_17164_gb300 import workloads as W
from tests.helpers import oracle_births, oracle_objects, rel_max

pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    from paper_2601_17164_gb300 import pipeline as PL
    from paper_2601_17164_gb300 import sfhk as S


def _small_sweep():
    ws = W.batched_sweep(n_cfg=6, seed=11, n_lo=300, n_hi=3000, dt=0.02)
    return [w for w in ws]


def _setup(ws):
    hs, bs, dls, dvs = [], [], [], []
    for w in ws:
        f, t = PL.make_handles(w)
        b = PL.sample(w, f, t)
        nb = f.info["n_bins"]
        hs.append((f, t))
        bs.append(b)
        dls.append(torch.zeros(nb, dtype=torch.float64, device="cuda"))
        dvs.append(torch.zeros(nb, dtype=torch.float64, device="cuda"))
    return hs, bs, dls, dvs


@pytest.mark.parametrize("precision", [0, 1])
def test_batch_matches_single_configuration_calls(precision):
    ws = _small_sweep()
    hs, bs, dls, dvs = _setup(ws)
    pp = S.prop_params(precision, 0.5, 1e30)
    st = S.new_stats()
    batch = S.Batch([h[0] for h in hs], [h[1] for h in hs], bs, [len(b) for b in bs], pp, dls, dvs, st)
    batch.run()
    torch.cuda.synchronize()
    st_single = S.new_stats()
    for (f, t), b, dl, dv, w in zip(hs, bs, dls, dvs, ws):
        rl, rv = torch.zeros_like(dl), torch.zeros_like(dv)
        S.sfhk_dipole(f, t, b, len(b), pp, rl, rv, st_single)
        e = max(rel_max(dl.cpu().numpy(), rl.cpu().numpy()), rel_max(dv.cpu().numpy(), rv.cpu().numpy()))
        assert e < 1e-12, (w.name, e)
    a, c = S.stats_dict(st), S.stats_dict(st_single)
    assert a["traj_steps"] == c["traj_steps"] and a["escalated"] == c["escalated"]


def test_one_shot_batched_dipole_equals_the_plan():
    # sfhk_dipole_batch (plan, run, wait, free in one call) against a plan run
    ws = _small_sweep()
    hs, bs, dls, dvs = _setup(ws)
    pp = S.prop_params(S.MIXED, 0.5, 1e30)
    batch = S.Batch([h[0] for h in hs], [h[1] for h in hs], bs, [len(b) for b in bs], pp, dls, dvs)
    batch.run()
    torch.cuda.synchronize()
    ols = [torch.zeros_like(d) for d in dls]
    ovs = [torch.zeros_like(d) for d in dvs]
    st = S.new_stats()
    S.sfhk_dipole_batch([h[0] for h in hs], [h[1] for h in hs], bs, [len(b) for b in bs], pp, ols, ovs, st)
    for a, b, c, d in zip(dls, ols, dvs, ovs):
        assert rel_max(b.cpu().numpy(), a.cpu().numpy()) < 1e-12 and rel_max(d.cpu().numpy(), c.cpu().numpy()) < 1e-12
    assert S.stats_dict(st)["traj_steps"] > 0
    with pytest.raises(S.SfhkError):
        S.sfhk_dipole_batch([], [], [], [], pp, [], [])


def test_batch_fp64_matches_oracle_and_graph_replay():
    ws = _small_sweep()[:3]
    hs, bs, dls, dvs = _setup(ws)
    batch = S.Batch([h[0] for h in hs], [h[1] for h in hs], bs, [len(b) for b in bs], S.prop_params(S.FP64),
                    dls, dvs)
    # warm-up run, then capture one run in a CUDA graph and replay it twice
    batch.run()
    torch.cuda.synchronize()
    first = [d.clone() for d in dls]
    for d in dls + dvs:
        d.zero_()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            batch.run(stream=s)
    g.replay()
    g.replay()
    torch.cuda.synchronize()
    for d, f0 in zip(dls, first):
        assert rel_max(d.cpu().numpy(), 2 * f0.cpu().numpy()) < 1e-12
    # FP64 against the FP64 oracle: soft-core H to 1e-10 of max |D|; the Tong-Lin Ar
    # sample holds chaotic near-core orbits whose rounding-order differences (FMA
    # contraction) grow to ~1e-5 of the bins, so Ar is held to 1e-4
    for w, d in zip(ws, first):
        P, T, G = oracle_objects(w)
        dl, dv, _ = O.dipole(P, T, G, oracle_births(w))
        tol = 1e-4 if T.pot == O.POT_TONGLIN else 1e-10
        assert rel_max(d.cpu().numpy(), dl) < tol, (w.name, rel_max(d.cpu().numpy(), dl))


def test_autotune_picks_a_valid_shape_and_is_used():
    w = W.H_800_8CYC_1M.with_n(4096)
    f, t = PL.make_handles(w)
    b = PL.sample(w, f, t)
    pp = S.prop_params(S.MIXED, esc_ratio=0.0)
    block, chunk, ms = S.sfhk_autotune(f, t, b, 2048, pp)
    assert block in (64, 128) and chunk % f.info["n_out"] == 0 and ms > 0
    nb = f.info["n_bins"]
    d1, v1 = torch.zeros(nb, dtype=torch.float64, device="cuda"), torch.zeros(nb, dtype=torch.float64, device="cuda")
    d2, v2 = torch.zeros_like(d1), torch.zeros_like(v1)
    S.sfhk_dipole(f, t, b, len(b), pp, d1, v1)                       # tuned shape (block = chunk = 0)
    S.sfhk_dipole(f, t, b, len(b), S.prop_params(S.MIXED, esc_ratio=0.0, block=block, chunk_steps=chunk), d2, v2)
    torch.cuda.synchronize()
    assert rel_max(d1.cpu().numpy(), d2.cpu().numpy()) < 1e-12
