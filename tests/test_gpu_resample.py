"""|I0| importance resampling on the GPU (sfhk_resample_births, App. A importance
sampling) against the oracle, bit for bit: the same pool (the oracle's own
births, uploaded) gives the same draws, multiplicities and rescaled amplitudes
on both sides, at small sizes (several scan blocks, ragged tails, n above and
below m) and at the bench size (1e6 births drawn from a 4e6 pool)."""
import numpy as np
import pytest
import torch

import oracle as O
from oracle import resample as RS
from paper_2601_17164_gb300 import workloads as W
from tests.helpers import oracle_births, oracle_objects, rel_max

pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    from paper_2601_17164_gb300 import pipeline as PL
    from paper_2601_17164_gb300 import sfhk as S

KEYS = (("n0", "n0"), ("t0", "t0"), ("px", "p0x"), ("py", "p0y"), ("pz", "p0z"), ("qz", "q0z"),
        ("amp_re", "amp_re"), ("amp_im", "amp_im"))


def _upload(b):
    return S.Births(*(torch.tensor(np.ascontiguousarray(b[k]), device="cuda") for k, _ in KEYS))


def _download(g):
    return {k: getattr(g, a).cpu().numpy() for k, a in KEYS}


def _gpu_resample(pool_np, m, n, seed):
    pool = _upload(pool_np)
    out = S.Births.empty(n)
    nd = torch.full((1,), -7, dtype=torch.int64, device="cuda")
    S.sfhk_resample_births(pool, m, n, seed, out, nd)
    torch.cuda.synchronize()
    return _download(out), int(nd.item())


def _assert_same(g, o):
    for k, _ in KEYS:
        assert g[k].dtype == o[k].dtype, k
        assert np.array_equal(g[k].view(np.uint8), o[k].view(np.uint8)), k    # bit for bit


@pytest.mark.parametrize("m,n,seed", [(4000, 1000, 5), (3001, 3001, 9), (1025, 40, 2), (2500, 7000, 3)])
def test_resample_bit_exact(m, n, seed):
    w = W.H_800_8CYC_1M
    pool = oracle_births(w, n=m, seed=seed + 100)
    g, r_g = _gpu_resample(pool, m, n, seed)
    o, r_o = RS.resample(pool, n, seed)
    assert r_g == r_o and 0 < r_o <= min(n, m)
    _assert_same(g, o)


def test_resample_bench_size_bit_exact():
    # the importance-sampled bench workload: 1e6 births from a pool of 4e6
    w = W.H_800_8CYC_1M
    m, n = 4 * w.n, w.n
    pool = oracle_births(w, n=m, seed=11)
    g, r_g = _gpu_resample(pool, m, n, 12)
    o, r_o = RS.resample(pool, n, 12)
    assert r_g == r_o
    _assert_same(g, o)


def test_resampled_dipole_matches_oracle():
    # FP64 bins of the resampled births (GPU resampling and propagation) against the
    # oracle's bins of its own resampled births, same pool: the 1024 grid births of
    # H 800 nm 2 cycles (regular trajectories, where FP64 bins agree to 1e-10)
    w = W.H_800_2CYC_GRID
    P, T, G = oracle_objects(w)
    m, n = w.n, 300
    pool = oracle_births(w)
    o, r = RS.resample(pool, n, 4)
    field, target = PL.make_handles(w)
    gp = _upload(pool)
    out = S.Births.empty(n)
    S.sfhk_resample_births(gp, m, n, 4, out)
    nb = field.info["n_bins"]
    dl = torch.zeros(nb, dtype=torch.float64, device="cuda")
    dv = torch.zeros_like(dl)
    S.sfhk_dipole(field, target, out, n, S.prop_params(S.FP64, w.gamma, w.d_t, deterministic=1), dl, dv)
    torch.cuda.synchronize()
    ol, ov, _ = O.dipole(P, T, G, o)
    assert rel_max(dl.cpu().numpy(), ol) < 1e-10 and rel_max(dv.cpu().numpy(), ov) < 1e-10


def test_sample_importance_runs():
    w = W.H_800_8CYC_1M.with_n(5000)
    field, target = PL.make_handles(w)
    b, nd = PL.sample_importance(w, field, target, pool_factor=4)
    torch.cuda.synchronize()
    r = int(nd.item())
    assert 0 < r <= 5000
    n0 = b.n0.cpu().numpy()
    assert np.all(np.diff(n0[:r]) >= 0)
    amp = (b.amp_re.cpu().numpy() + 1j * b.amp_im.cpu().numpy())
    assert np.all(amp[:r] != 0) and np.all(amp[r:] == 0)


def test_resample_degenerate_pools_and_errors():
    base = {"n0": np.arange(10, dtype=np.int32), "t0": np.linspace(0, 1, 10), "px": np.linspace(1, 2, 10),
            "py": np.zeros(10), "pz": np.linspace(-1, 1, 10), "qz": np.linspace(3, 4, 10),
            "amp_re": np.zeros(10), "amp_im": np.zeros(10)}
    g, r = _gpu_resample(base, 10, 5, 1)           # nothing to draw
    o, ro = RS.resample(base, 5, 1)
    assert r == ro == 0
    _assert_same(g, o)
    one = {k: v.copy() for k, v in base.items()}
    one["amp_re"][3] = 2.5
    g, r = _gpu_resample(one, 10, 4, 1)            # one weight: drawn n times, weight a
    o, ro = RS.resample(one, 4, 1)
    assert r == ro == 1
    _assert_same(g, o)
    for bad in (np.inf, np.nan):
        b = {k: v.copy() for k, v in one.items()}
        b["amp_im"][5] = bad
        g, r = _gpu_resample(b, 10, 4, 1)
        o, ro = RS.resample(b, 4, 1)
        assert r == ro == 0
        _assert_same(g, o)
    pool = _upload(one)
    out = S.Births.empty(4)
    nd = torch.full((1,), 5, dtype=torch.int64, device="cuda")
    S.sfhk_resample_births(pool, 10, 0, 1, out, nd)     # n = 0: r = 0, nothing else
    assert int(nd.item()) == 0
    with pytest.raises(S.SfhkError):
        S.sfhk_resample_births(pool, 0, 4, 1, out)       # empty pool
    with pytest.raises(S.SfhkError):
        S.sfhk_resample_births(pool, 11, 4, 1, out)      # m above the pool's capacity
    with pytest.raises(S.SfhkError):
        S.sfhk_resample_births(pool, 10, 5, 1, out)      # n above out's capacity
    with pytest.raises(S.SfhkError):
        S.sfhk_resample_births(pool, 10, 4, 1, pool)     # pool and out share arrays
