"""Shared helpers of the test suite: oracle records from a workload, tolerances."""
import os

import numpy as np

import oracle as O
from paper_2601_17164_gb300 import workloads as W


def oracle_objects(w: W.Workload, amp_kind=None):
    p = w.pulse
    P = O.make_pulse(p.intensity_wcm2, p.lambda_nm, p.cycles, p.cep)
    t = w.target
    T = O.make_target(t.pot, t.pot_param, t.ip, t.gto_l, t.c, t.alpha,
                      amp_kind=t.amp_kind if amp_kind is None else amp_kind)
    G = O.pulse_grid(P, w.dt, w.t_out, w.gamma, w.d_t)
    return P, T, G


def oracle_births(w: W.Workload, n=None, seed=None):
    P, T, G = oracle_objects(w)
    n = w.n if n is None else n
    return O.sample_births(P, T, G, w.birth_mode, n, w.n_t, w.n_k, w.sigma, w.kmax,
                           w.seed if seed is None else seed)


_GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def paper_value(key: str):
    """(value, tolerance) of a number printed in the paper (tests/golden/paper_values.txt)."""
    with open(os.path.join(_GOLDEN, "paper_values.txt")) as fh:
        for line in fh:
            f = line.split()
            if f and not f[0].startswith("#") and f[0] == key:
                return float(f[1]), float(f[2])
    raise KeyError(key)


def rel_max(a, b, scale=None):
    a, b = np.asarray(a), np.asarray(b)
    s = np.max(np.abs(b)) if scale is None else scale
    return float(np.max(np.abs(a - b)) / s) if s > 0 else float(np.max(np.abs(a - b)))


def plateau_harmonics(w: W.Workload, lo=None):
    """Odd harmonics from just above Ip to the classical cutoff Ip + 3.17 Up."""
    E0 = np.sqrt(w.pulse.intensity_wcm2 / 3.50944758e16)
    w0 = 45.5633525 / w.pulse.lambda_nm
    hi = (w.target.ip + 3.17 * E0 ** 2 / (4 * w0 ** 2)) / w0
    start = int(np.ceil(w.target.ip / w0)) if lo is None else lo
    return [h for h in range(start, int(hi) + 1) if h % 2 == 1]


def band_yield(omega, X, w0, power, harmonics):
    y = np.abs(X) ** 2 * omega ** power
    return np.array([y[np.abs(omega / w0 - h) <= 0.5].sum() for h in harmonics])


def harmonic_phase(omega, X, w0, harmonics):
    out = []
    for h in harmonics:
        j = np.argmin(np.abs(omega - h * w0))
        out.append(np.angle(X[j]))
    return np.array(out)
