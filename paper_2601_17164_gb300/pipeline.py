"""One spectrum run through the C ABI: field -> births -> dipole bins -> spectrum.

Orchestration and marshalling only; every step runs in the CUDA library.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import Optional

import torch

from . import sfhk as S
from .workloads import Workload, omega_grid


@dataclass
class Run:
    field: S.Field
    target: S.Target
    births: S.Births
    d_len: torch.Tensor
    d_vel: torch.Tensor
    omega: torch.Tensor
    D_re: torch.Tensor
    D_im: torch.Tensor
    V_re: torch.Tensor
    V_im: torch.Tensor
    stats: torch.Tensor


def make_handles(w: Workload, amp_kind: Optional[int] = None):
    p = w.pulse
    field = S.Field(p.intensity_wcm2, p.lambda_nm, p.cycles, p.cep, w.dt, w.t_out)
    t = w.target
    target = S.Target(t.pot, t.pot_param, t.ip, t.gto_l, t.c, t.alpha, t.amp_kind if amp_kind is None else amp_kind)
    return field, target


def sample(w: Workload, field: S.Field, target: S.Target, births: Optional[S.Births] = None, n: Optional[int] = None,
           seed: Optional[int] = None, stream=None) -> S.Births:
    n = w.n if n is None else n
    births = births if births is not None else S.Births.empty(n)
    S.sfhk_sample_births(field, target, w.birth_mode, n, births, n_t=w.n_t, n_k=w.n_k, sigma_k=w.sigma or 1.0,
                         kmax=w.kmax or 1.0, seed=w.seed if seed is None else seed, stream=stream)
    return births


def sample_importance(w: Workload, field: S.Field, target: S.Target, n: Optional[int] = None, pool_factor: int = 4,
                      seed: Optional[int] = None, stream=None):
    """n births drawn in proportion to |I0| (App. A importance sampling) from a pool of
    pool_factor * n births of the workload's own sampler; returns (births, n_distinct)."""
    if w.birth_mode != S.BIRTH_UNIFORM_GAUSS:
        raise ValueError("importance sampling draws from the Gaussian-momentum sampler (birth mode 1)")
    n = w.n if n is None else n
    m = max(1, pool_factor * n)
    seed = w.seed if seed is None else seed
    pool = sample(w, field, target, n=m, seed=seed, stream=stream)
    out = S.Births.empty(n)
    nd = torch.zeros(1, dtype=torch.int64, device="cuda")
    S.sfhk_resample_births(pool, m, n, seed, out, nd, stream)
    return out, nd


def spectrum_of(bins: torch.Tensor, field: S.Field, omega: torch.Tensor, stream=None):
    info = field.info
    re = torch.empty_like(omega)
    im = torch.empty_like(omega)
    S.sfhk_spectrum(bins, info["t_start"], info["dt"] * info["n_out"], 0.5 * info["Tp"], omega, re, im, stream)
    return re, im


def gabor_of(bins: torch.Tensor, field: S.Field, times: torch.Tensor, omega: torch.Tensor,
             sigma: Optional[float] = None, stream=None):
    """Gabor map (re, im) of shape (len(times), len(omega)); window width 1/(3 w0) by default."""
    info = field.info
    sigma = 1.0 / (3.0 * info["omega"]) if sigma is None else sigma
    re = torch.empty(times.numel(), omega.numel(), dtype=torch.float64, device=bins.device)
    im = torch.empty_like(re)
    S.sfhk_gabor(bins, info["t_start"], info["dt"] * info["n_out"], sigma, times, omega, re, im, stream)
    return re, im


def emission_times(g_re: torch.Tensor, g_im: torch.Tensor, times: torch.Tensor, t_a: float, t_b: float,
                   stream=None):
    """(centroid, peak) emission time per frequency of the burst in [t_a, t_b]."""
    n_w = g_re.shape[1]
    cen = torch.empty(n_w, dtype=torch.float64, device=g_re.device)
    peak = torch.empty_like(cen)
    S.sfhk_emission_time(g_re, g_im, times, t_a, t_b, cen, peak, stream)
    return cen, peak


def run(w: Workload, precision: int = S.MIXED, deterministic: int = 0, block: int = 0, chunk_steps: int = 0,
        stream=None) -> Run:
    field, target = make_handles(w)
    births = sample(w, field, target, stream=stream)
    nb = field.info["n_bins"]
    d_len = torch.zeros(nb, dtype=torch.float64, device="cuda")
    d_vel = torch.zeros(nb, dtype=torch.float64, device="cuda")
    stats = S.new_stats()
    pp = S.prop_params(precision, w.gamma, w.d_t, deterministic, block, chunk_steps)
    S.sfhk_dipole(field, target, births, len(births), pp, d_len, d_vel, stats, stream)
    omega = torch.tensor(omega_grid(w), dtype=torch.float64, device="cuda")
    D_re, D_im = spectrum_of(d_len, field, omega, stream)
    V_re, V_im = spectrum_of(d_vel, field, omega, stream)
    return Run(field, target, births, d_len, d_vel, omega, D_re, D_im, V_re, V_im, stats)

