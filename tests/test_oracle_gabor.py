"""Pins of the Gabor oracle (Sec. III.A time-frequency maps and emission times):
a Gaussian burst with a closed-form transform, the time-shift law, and the
emission time of bursts with known centres."""
import numpy as np

from oracle import gabor as GB


def _burst(tc, s, Om, t0, dt, n):
    t = t0 + np.arange(n) * dt
    return np.exp(-((t - tc) ** 2) / (2 * s * s)) * np.cos(Om * t)


def _closed_form(t, w, tc, s, sigma, Om):
    """int exp(-(u-tc)^2/2s^2) cos(Om u) exp(-(u-t)^2/2sigma^2) e^{i w u} du (both rotating terms)."""
    a = 1 / (2 * s * s) + 1 / (2 * sigma * sigma)
    tot = 0
    for nu in (w + Om, w - Om):
        b = tc / (s * s) + t / (sigma * sigma) + 1j * nu
        c = -tc * tc / (2 * s * s) - t * t / (2 * sigma * sigma)
        tot = tot + 0.5 * np.sqrt(np.pi / a) * np.exp(b * b / (4 * a) + c)
    return tot


def test_gabor_of_gaussian_burst_matches_closed_form():
    t0, dt, n = -300.0, 0.1, 6001
    tc, s, sigma, Om = 17.0, 20.0, 12.0, 1.3
    x = _burst(tc, s, Om, t0, dt, n)
    times = np.linspace(-60, 90, 31)
    omega = np.linspace(0.2, 2.6, 25)
    G = GB.gabor(x, t0, dt, sigma, times, omega)
    ref = np.array([[_closed_form(t, w, tc, s, sigma, Om) for w in omega] for t in times])
    assert np.max(np.abs(G - ref)) < 1e-12 * np.max(np.abs(ref))


def test_time_shift_multiplies_by_a_phase():
    t0, dt, n, m = -100.0, 0.1, 1500, 37
    rng = np.random.default_rng(4)
    x = rng.standard_normal(n)
    xs = np.concatenate([np.zeros(m), x])
    times = np.array([-20.0, 0.0, 13.0])
    omega = np.array([0.3, 1.1, 2.9])
    sigma = 5.0
    G = GB.gabor(x, t0, dt, sigma, times, omega)
    Gs = GB.gabor(xs, t0, dt, sigma, times + m * dt, omega)
    assert np.max(np.abs(Gs - G * np.exp(1j * omega * m * dt))) < 1e-12 * np.max(np.abs(G))


def test_emission_time_of_bursts():
    # two bursts at tc1, tc2 with different frequencies; the window picks one
    t0, dt, n = -300.0, 0.1, 6001
    sigma = 12.0
    x = _burst(-23.4, 15.0, 1.0, t0, dt, n) + 0.5 * _burst(61.7, 15.0, 1.8, t0, dt, n)
    times = np.arange(-200.0, 200.0, 0.5)
    omega = np.array([1.0, 1.8])
    G = GB.gabor(x, t0, dt, sigma, times, omega)
    # windows of +-8 widths of |G|^2 (width sqrt((s^2 + sigma^2)/2) = 13.6) around each centre
    cen, peak = GB.emission_time(G, times, -23.4 - 110, -23.4 + 110)
    assert abs(peak[0] + 23.4) < 1e-6 and abs(cen[0] + 23.4) < 1e-6
    cen2, peak2 = GB.emission_time(G, times, 61.7 - 110, 61.7 + 110)
    assert abs(peak2[1] - 61.7) < 1e-6 and abs(cen2[1] - 61.7) < 1e-6
    # empty window and vanishing signal give NaN
    c3, p3 = GB.emission_time(G, times, 500.0, 600.0)
    assert np.all(np.isnan(c3)) and np.all(np.isnan(p3))
    c4, p4 = GB.emission_time(np.zeros_like(G), times, -10.0, 10.0)
    assert np.all(np.isnan(c4)) and np.all(np.isnan(p4))
