"""Gabor map and emission times on the GPU (sfhk_gabor, sfhk_emission_time)
against the oracle, on the oracle's own dipole bins and on synthetic bursts."""
import numpy as np
import pytest
import torch

import oracle as O
from oracle import gabor as GB
from paper_2601_17164_gb300 import workloads as W
from tests.helpers import oracle_births, oracle_objects

pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    from paper_2601_17164_gb300 import pipeline as PL
    from paper_2601_17164_gb300 import sfhk as S


def _dev(a):
    return torch.tensor(np.asarray(a, dtype=np.float64), device="cuda")


def _gpu_gabor(x, t0, dt, sigma, times, omega):
    re = torch.empty(len(times), len(omega), dtype=torch.float64, device="cuda")
    im = torch.empty_like(re)
    S.sfhk_gabor(_dev(x), t0, dt, sigma, _dev(times), _dev(omega), re, im)
    return re, im


def _c(re, im):
    return re.cpu().numpy() + 1j * im.cpu().numpy()


def test_gabor_synthetic_ragged_and_clipped_windows():
    # 3001 bins (ragged tail of the 1024-bin tiles), 300 frequencies (ragged over 128-thread
    # blocks), analysis times before, inside and after the bins (clipped windows)
    t0, dt, n = -150.0, 0.1, 3001
    t = t0 + np.arange(n) * dt
    rng = np.random.default_rng(3)
    x = np.exp(-((t - 20.0) ** 2) / 800.0) * np.cos(1.1 * t) + 0.01 * rng.standard_normal(n)
    times = np.linspace(-260.0, 260.0, 37)
    omega = np.linspace(0.05, 3.0, 300)
    sigma = 7.5
    G = _c(*_gpu_gabor(x, t0, dt, sigma, times, omega))
    ref = GB.gabor(x, t0, dt, sigma, times, omega)
    assert np.max(np.abs(G - ref)) < 1e-12 * np.max(np.abs(ref))


def test_gabor_and_emission_time_of_oracle_bins():
    # the oracle's FP64 dipole velocity of H, 800 nm, 2 cycles (32 x 32 grid births)
    w = W.H_800_2CYC_GRID
    P, T, G = oracle_objects(w)
    _, dv, _ = O.dipole(P, T, G, oracle_births(w))
    dt_out = G.dt * G.n_out
    w0 = P.omega
    sigma = 1.0 / (3.0 * w0)
    times = np.arange(-110.0, 110.0, 1.0)
    omega = np.arange(1, 30, 0.25) * w0
    g_re, g_im = _gpu_gabor(dv, G.t_start, dt_out, sigma, times, omega)
    ref = GB.gabor(dv, G.t_start, dt_out, sigma, times, omega)
    assert np.max(np.abs(_c(g_re, g_im) - ref)) < 1e-12 * np.max(np.abs(ref))
    # emission time of the burst in [0, T0/2] (first return after the peak)
    t_a, t_b = 0.0, np.pi / w0
    cen = torch.empty(omega.size, dtype=torch.float64, device="cuda")
    peak = torch.empty_like(cen)
    S.sfhk_emission_time(g_re, g_im, _dev(times), t_a, t_b, cen, peak)
    c_o, p_o = GB.emission_time(ref, times, t_a, t_b)
    c_g, p_g = cen.cpu().numpy(), peak.cpu().numpy()
    assert np.array_equal(np.isnan(c_g), np.isnan(c_o)) and np.array_equal(np.isnan(p_g), np.isnan(p_o))
    ok = ~np.isnan(c_o)
    assert np.max(np.abs(c_g[ok] - c_o[ok])) < 1e-9
    assert np.max(np.abs(p_g[ok] - p_o[ok])) < 1e-6


def test_gabor_full_size_sampled():
    # dipole bins of the H 800 nm 8-cycle grid (8827 bins), 2000 times x 3000 frequencies;
    # sampled (time, frequency) pairs against the oracle one by one
    w = W.H_800_8CYC_1M
    f, _ = PL.make_handles(w)
    info = f.info
    nb = info["n_bins"]
    dt_out = info["dt"] * info["n_out"]
    t = info["t_start"] + np.arange(nb) * dt_out
    rng = np.random.default_rng(5)
    x = np.cos(0.9 * t) * np.exp(-(t / 300.0) ** 2) + 0.1 * rng.standard_normal(nb)
    times = np.linspace(info["t_start"], -info["t_start"], 2000)
    omega = np.linspace(0.01, 3.0, 3000)
    sigma = 1.0 / (3.0 * info["omega"])
    g_re, g_im = PL.gabor_of(_dev(x), f, _dev(times), _dev(omega))
    Gg = _c(g_re, g_im)
    js = rng.integers(0, times.size, 16)
    ms = rng.integers(0, omega.size, 16)
    for j, m in zip(js, ms):
        ref = GB.gabor(x, info["t_start"], dt_out, sigma, times[j:j + 1], omega[m:m + 1])[0, 0]
        scale = np.sum(np.abs(x)) * dt_out
        assert abs(Gg[j, m] - ref) < 1e-12 * scale, (j, m)


def test_gabor_edge_cases():
    x = _dev(np.ones(10))
    om = _dev([1.0])
    tm = _dev([0.0])
    re = torch.empty(1, dtype=torch.float64, device="cuda")
    im = torch.empty_like(re)
    with pytest.raises(S.SfhkError):
        S.sfhk_gabor(x, 0.0, 0.1, 0.0, tm, om, re, im)        # sigma <= 0
    with pytest.raises(S.SfhkError):
        S.sfhk_gabor(x, 0.0, -0.1, 1.0, tm, om, re, im)       # dt_out <= 0
    # empty bins give zeros; empty frequency or time lists are no-ops
    S.sfhk_gabor(x[:0], 0.0, 0.1, 1.0, tm, om, re, im)
    assert float(re.abs().sum()) == 0.0 and float(im.abs().sum()) == 0.0
    e = torch.empty(0, dtype=torch.float64, device="cuda")
    S.sfhk_gabor(x, 0.0, 0.1, 1.0, tm, e, e, e)
    S.sfhk_gabor(x, 0.0, 0.1, 1.0, e, om, e, e)
    torch.cuda.synchronize()
