"""Gabor time-frequency analysis of the dipole bins and the emission time of a
burst (Sec. III.A, Fig. HGabor and Fig. HGabortime): plain numpy, FP64.

Test infrastructure only: loaded by tests, the smoke check and the CPU
baseline of the benchmark.

Definitions (the paper shows the maps but prints no formula; the reading is
the usual Gabor transform of the dipole velocity):

  G(t, w) = sum_k x(t_k) exp(-(t_k - t)^2 / (2 sigma^2)) e^{i w t_k} dt_out

with t_k = t0 + k dt_out the output bins, the same e^{+i w t} convention as
the spectrum (App. D), and a Gaussian window of width sigma (default
1/(3 w0), w0 the laser frequency).  The full sum over k is taken.

The emission time of harmonic w in a burst window [t_a, t_b] is read two ways
from |G(t, w)|^2 on the analysis times t_j:
  * centroid: sum_j t_j |G_j|^2 / sum_j |G_j|^2 over t_j in [t_a, t_b];
  * peak: the t_j in [t_a, t_b] with the largest |G_j|^2, refined by the vertex
    of the parabola through ln|G|^2 at t_{j-1}, t_j, t_{j+1} (exact for a
    Gaussian burst); the sample itself where a neighbour is missing or the
    parabola does not open downwards.
Pinned by tests/test_oracle_gabor.py (closed-form Gaussian burst, time shift).
"""
from __future__ import annotations

import numpy as np


def gabor(x, t0: float, dt_out: float, sigma: float, times, omega):
    """G[j, m] = G(times[j], omega[m]) as complex128 of shape (len(times), len(omega))."""
    x = np.asarray(x, dtype=np.float64)
    times = np.asarray(times, dtype=np.float64)
    omega = np.asarray(omega, dtype=np.float64)
    tk = t0 + np.arange(x.size, dtype=np.float64) * dt_out
    out = np.empty((times.size, omega.size), dtype=np.complex128)
    for m0 in range(0, omega.size, 256):
        F = np.exp(1j * np.outer(tk, omega[m0:m0 + 256]))          # e^{i w t_k}
        for j, t in enumerate(times):
            g = x * np.exp(-((tk - t) ** 2) / (2.0 * sigma * sigma)) * dt_out
            out[j, m0:m0 + 256] = g @ F
    return out


def emission_time(G, times, t_a: float, t_b: float):
    """(centroid[m], peak[m]) of |G[:, m]|^2 over times in [t_a, t_b]; NaN where the window is empty
    or |G| vanishes there."""
    times = np.asarray(times, dtype=np.float64)
    P = np.abs(np.asarray(G)) ** 2
    n_t, n_w = P.shape
    sel = np.nonzero((times >= t_a) & (times <= t_b))[0]
    cen = np.full(n_w, np.nan)
    peak = np.full(n_w, np.nan)
    if sel.size == 0:
        return cen, peak
    for m in range(n_w):
        p = P[sel, m]
        tot = p.sum()
        if not tot > 0.0:
            continue
        cen[m] = float((times[sel] * p).sum() / tot)
        j = int(sel[int(np.argmax(p))])
        peak[m] = times[j]
        if sel[0] < j < sel[-1] and P[j - 1, m] > 0 and P[j + 1, m] > 0:
            ym, y0, yp = np.log(P[j - 1, m]), np.log(P[j, m]), np.log(P[j + 1, m])
            h = times[j + 1] - times[j]
            curv = ym - 2.0 * y0 + yp
            if curv < 0.0 and abs(times[j] - times[j - 1] - h) <= 1e-9 * abs(h):
                peak[m] = times[j] + 0.5 * h * (ym - yp) / curv
    return cen, peak
