"""Oracle pins: SFA births (App. A Eq. SAPeq, Eq. SFAwf, Eq. Int; App. B.1),
the tunnelling matrix elements and the birth sampler.

Pins: the saddle-point equation itself, brute-force scans for the smallest
root, the quasi-static (tunnelling) limit, Gauss-Legendre quadrature of the
contour integrals, 3D numerical Fourier integrals, numpy's Philox and exact
big-integer arithmetic.
"""
import numpy as np
import pytest

import oracle as O
from paper_2601_17164_gb300 import workloads as W


def _h_target(l=0):
    if l == 0:
        return O.make_target(O.POT_SOFTCORE, [0.3], ip=0.5, gto_l=0, c=W.H_C, alpha=W.H_ALPHA)
    t = W.ARGON
    return O.make_target(t.pot, t.pot_param, t.ip, 1, t.c, t.alpha)


CASES = [(-12.0, 0.0, 0.0), (3.0, 0.1, -0.05), (-52.0, 0.25, 0.1), (45.0, 0.0, 0.3), (0.0, 0.0, 0.0)]


@pytest.mark.parametrize("l", [0, 1])
def test_saddle_point_equation_and_smallest_root(l):
    P = O.make_pulse(1.5e14, 800.0, 8.0, cep=0.2)
    T = _h_target(l)
    ip = T.ip
    t0, kx, ky = (np.array(v) for v in zip(*CASES))
    b = O.births_at(P, T, t0, kx, ky)
    assert np.all(b["valid"] == 1)
    for i in range(len(t0)):
        ts = t0[i] + 1j * b["tt"][i]
        A_ts, A_t0 = O.field(P, "A", [ts, t0[i]])
        vz = b["kz"][i] + A_ts - A_t0.real
        resid = (kx[i] ** 2 + ky[i] ** 2 + vz ** 2) / 2 + ip          # Eq. SAPeq
        assert abs(resid) < 1e-12
        # Im S_down^0 > 0 : the tunnelling factor decays
        assert b["S_im"][i] > 0
        # no root of Im A(t0 + i tau) = s kappa below tt (brute-force scan)
        kappa = np.sqrt(2 * ip + kx[i] ** 2 + ky[i] ** 2)
        s = -np.sign(O.field(P, "E", [t0[i]])[0].real)
        tau = np.linspace(0, b["tt"][i], 4001)[1:-1]
        f = O.field(P, "A", t0[i] + 1j * tau).imag - s * kappa
        assert np.all(np.sign(f) == np.sign(f[0]))


def test_births_without_saddle_only_near_field_zeros():
    # With s = -sign E(t0) a root exists except close to zeros of E(t0), where
    # the tunnelling factor is negligible; such births carry zero weight.
    P = O.make_pulse(1.5e14, 800.0, 8.0, cep=0.2)
    T = _h_target(0)
    t0 = np.linspace(-0.45 * P.Tp, 0.45 * P.Tp, 801)
    b = O.births_at(P, T, t0, 0 * t0, 0 * t0)
    E = np.abs(O.field(P, "E", t0).real)
    env = np.cos(np.pi * t0 / P.Tp) ** 2 * P.E0
    bad = b["valid"] == 0
    assert bad.sum() < 0.2 * len(t0)
    # |E| < E0/4 means a tunnelling factor exp(-2 kappa^3/3|E|) below e^{-40}
    assert np.all(E[bad] < 0.25 * P.E0)
    # where valid, the tunnelling factor e^{-Im S} is tiny wherever |E| is that small
    good_small = (~bad) & (E < 0.05 * env)
    assert np.all(b["S_im"][good_small] > 20)


def test_quasistatic_tunnelling_limit():
    # omega -> 0 at a field crest, k_perp = 0: q0 -> -Ip/E, kz -> 0,
    # |e^{i S}|^2 -> exp(-2 kappa^3 / (3|E|)) (tunnelling exponent).
    E0 = 0.05
    P = O.make_pulse(E0=E0, omega=2e-4, cycles=2.0)
    T = _h_target(0)
    b = O.births_at(P, T, [0.0], [0.0], [0.0])
    kappa = 1.0
    assert abs(b["qz"][0] - (-T.ip / E0)) < 2e-4 * T.ip / E0
    assert abs(b["kz"][0]) < 1e-6
    assert abs(2 * b["S_im"][0] - 2 * kappa ** 3 / (3 * E0)) < 1e-4 * 2 * kappa ** 3 / (3 * E0)


@pytest.mark.parametrize("l", [0, 1])
def test_action_and_exit_against_contour_quadrature(l):
    # S_down^0 = Ip ts - int_{ts}^{t0} (k + A - A(t0))^2/2 ; q0 = Re int_{ts}^{t0} A
    P = O.make_pulse(1e14, 1600.0, 3.0, cep=0.5)
    T = _h_target(l)
    x, wq = np.polynomial.legendre.leggauss(64)
    t0, kx, ky = (np.array(v) for v in zip(*CASES[:4]))
    b = O.births_at(P, T, t0, kx, ky)
    for i in range(len(t0)):
        ts = t0[i] + 1j * b["tt"][i]
        tau = 0.5 * (ts + t0[i]) + 0.5 * (t0[i] - ts) * x
        A = O.field(P, "A", tau)
        A0 = O.field(P, "A", [t0[i]])[0].real
        v2 = kx[i] ** 2 + ky[i] ** 2 + (b["kz"][i] + A - A0) ** 2
        S = T.ip * ts - 0.5 * (t0[i] - ts) * np.sum(wq * v2 / 2)
        q = (0.5 * (t0[i] - ts) * np.sum(wq * A)).real
        assert abs(S - (b["S_re"][i] + 1j * b["S_im"][i])) < 1e-11 * max(1, abs(S))
        assert abs(q - b["qz"][i]) < 1e-11 * max(1, abs(q))


def _fourier_1d(kc, alpha, power, L=90.0, h=0.004):
    """int x^power e^{-alpha x^2 - i k x} dx, trapezoid (spectrally exact here)."""
    x = np.arange(-L, L + h / 2, h)
    return h * np.sum(x ** power * np.exp(-alpha * x * x - 1j * kc * x))


@pytest.mark.parametrize("l", [0, 1])
def test_tunnel_element_against_3d_fourier_integral(l):
    # m(k) = (2 pi)^{-3/2} int e^{-i k.r} z psi0(r) d^3 r, complex k allowed
    T = _h_target(l)
    n = T.n_gto
    c, a = np.array(T.c[:n]), np.array(T.alpha[:n])
    for k in [np.array([0.1, -0.2, 0.3]), np.array([0.05, 0.0, 0.0 + 0.95j]),
              np.array([0.2, 0.1, 0.1 - 1.1j])]:
        ref = 0
        for cj, aj in zip(c, a):
            ref += cj * (_fourier_1d(k[0], aj, 0) * _fourier_1d(k[1], aj, 0) * _fourier_1d(k[2], aj, 1 + l))
        ref *= (2 * np.pi) ** -1.5
        got = O.tunnel_element(T, k)
        assert abs(got - ref) < 1e-10 * abs(ref)


def _cs_1d(x, q, p, gam):
    return np.exp(-gam * (x - q) ** 2 + 1j * p * (x - q))


@pytest.mark.parametrize("l", [0, 1])
def test_recombination_elements_against_3d_quadrature(l):
    # d_len = <psi0| z |p,q,gamma>, d_vel = <psi0| -i d/dz |p,q,gamma>
    # = i <d psi0/dz | p,q,gamma> (integration by parts), normalised coherent
    # state (2 gamma/pi)^{3/4} e^{-gamma (r-q)^2 + i p.(r-q)} (App. A/C).
    T = _h_target(l)
    n = T.n_gto
    c, a = np.array(T.c[:n]), np.array(T.alpha[:n])
    gam = 0.5
    rng = np.random.default_rng(7)
    h = 0.004
    x = np.arange(-40, 40 + h / 2, h)
    for _ in range(3):
        p = rng.uniform(-1.5, 1.5, 3)
        q = rng.uniform(-2.5, 2.5, 3)
        N = (2 * gam / np.pi) ** 0.75
        dl = dv = 0
        for cj, aj in zip(c, a):
            g = np.exp(-aj * x * x)
            I = [h * np.sum(g * _cs_1d(x, q[d], p[d], gam)) for d in range(3)]
            cs_z = _cs_1d(x, q[2], p[2], gam)
            if l == 0:
                Iz = h * np.sum(x * g * cs_z)                       # psi0 = e^{-a r^2}
                dpsi = h * np.sum(-2 * aj * x * g * cs_z)           # d/dz e^{-a r^2}
            else:
                Iz = h * np.sum(x * x * g * cs_z)                   # psi0 = z e^{-a r^2}
                dpsi = h * np.sum((1 - 2 * aj * x * x) * g * cs_z)  # d/dz (z e^{-a r^2})
            dl += cj * I[0] * I[1] * Iz
            dv += cj * I[0] * I[1] * 1j * dpsi
        dl *= N
        dv *= N
        got_l, got_v = O.dipole_elements(T, gam, p, q)
        assert abs(got_l - dl) < 1e-10 * abs(dl)
        assert abs(got_v - dv) < 1e-10 * abs(dv)


def test_philox_matches_numpy_bit_generator():
    # numpy's Philox (4x64-10) bumps the counter before each block: its first
    # block for counter c is our block c+1.
    for key, ctr in [((0, 0), 0), ((5, 7), 10), ((2 ** 64 - 1, 123), 2 ** 40 + 3)]:
        bg = np.random.Philox(key=np.array(key, dtype=np.uint64),
                              counter=np.array([ctr, 0, 0, 0], dtype=np.uint64))
        ref = bg.random_raw(4)
        got = O.philox4x64([ctr + 1, 0, 0, 0], key)
        assert np.array_equal(got, ref)


def test_uniform_births_stratified_integer_rule_and_moments():
    w = W.H_800_8CYC_1M
    P = O.make_pulse(w.pulse.intensity_wcm2, w.pulse.lambda_nm, w.pulse.cycles)
    T = _h_target(0)
    G = O.pulse_grid(P, w.dt, w.t_out)
    n = 20000
    b = O.sample_births(P, T, G, 1, n, sigma=w.sigma, seed=w.seed)
    M = G.n_steps - 1
    n0 = b["n0"].astype(np.int64)
    assert np.all(np.diff(n0) >= 0) and n0.min() >= 1 and n0.max() <= M
    # exact big-integer recomputation of n0 from numpy's Philox words
    for i in [0, 1, 17, 9999, n - 1]:
        x = O.philox4x64([i, 0, 0, 0], [w.seed, 0])
        r = int(x[0]) >> 32
        assert n0[i] == 1 + ((i << 32) + r) * M // (n << 32)
    # stratification: each birth lies in its own stratum
    i = np.arange(n)
    assert np.all(n0 >= 1 + (i * M) // n) and np.all(n0 <= 1 + ((i + 1) * M) // n)
    # k_perp ~ N(0, sigma^2) per component
    k = np.concatenate([b["px"], b["py"]]) / w.sigma
    assert abs(k.mean()) < 0.03 and abs(k.var() - 1) < 0.03 and abs(np.mean(k ** 4) - 3) < 0.15
    # the birth kz, qz are those of the single-birth solver at the same (t0, k)
    bb = O.births_at(P, T, b["t0"][:50], b["px"][:50], b["py"][:50])
    assert np.array_equal(bb["kz"], b["pz"][:50]) and np.array_equal(bb["qz"], b["qz"][:50])


def test_birth_weights_measure():
    # grid mode: sum of weights = pi kmax^2 * (grid duration)  (2 pi k dk dt0)
    w = W.H_800_2CYC_GRID
    P = O.make_pulse(w.pulse.intensity_wcm2, w.pulse.lambda_nm, w.pulse.cycles)
    T = _h_target(0)
    G = O.pulse_grid(P, w.dt, w.t_out)
    b = O.sample_births(P, T, G, 0, w.n, w.n_t, w.n_k, kmax=w.kmax)
    u = O.births_at(P, T, b["t0"], b["px"], b["py"])
    ok = (u["valid"] == 1) & (np.abs(u["amp_re"]) > 1e-250) & (np.abs(u["amp_im"]) > 1e-250)
    wt = b["amp_re"][ok] / u["amp_re"][ok]
    assert np.allclose(b["amp_im"][ok], wt * u["amp_im"][ok], rtol=1e-13, atol=0)
    k = b["px"][ok]
    # weight per birth is 2 pi k dk dt0
    dk = w.kmax / w.n_k
    dt0 = G.n_steps * G.dt / w.n_t
    assert np.allclose(wt, 2 * np.pi * k * dk * dt0, rtol=1e-13)
    assert abs(np.sum(2 * np.pi * ((np.arange(w.n_k) + 0.5) * dk) * dk) - np.pi * w.kmax ** 2) < 1e-12
    # gaussian mode: w = 1/(N pdf):  sum_i w_i g(k_i) estimates int g d^2k * T
    w2 = W.H_800_8CYC_1M
    P2 = O.make_pulse(w2.pulse.intensity_wcm2, w2.pulse.lambda_nm, w2.pulse.cycles)
    G2 = O.pulse_grid(P2, w2.dt, w2.t_out)
    n = 20000
    b2 = O.sample_births(P2, T, G2, 1, n, sigma=w2.sigma, seed=3)
    u2 = O.births_at(P2, T, b2["t0"], b2["px"], b2["py"])
    ok = (u2["valid"] == 1) & (np.abs(u2["amp_re"]) > 1e-250)
    wt2 = b2["amp_re"][ok] / u2["amp_re"][ok]
    k2 = b2["px"][ok] ** 2 + b2["py"][ok] ** 2
    s2 = w2.sigma ** 2
    Tg = (G2.n_steps - 1) * G2.dt
    est = np.sum(wt2 * np.exp(-k2 / s2)) * n / ok.sum()   # int e^{-k^2/s^2} d^2k = pi s^2
    assert abs(est / (np.pi * s2 * Tg) - 1) < 0.03


def test_modified_spa_amplitude_magnitude():
    # App. B.2: the modified SPA weight is e^{i(S + p0.q0)} / (E(ts).v_s).
    P = O.make_pulse(1e14, 1600.0, 3.0)
    T0 = _h_target(0)
    T1 = O.make_target(O.POT_SOFTCORE, [0.3], ip=0.5, gto_l=0, c=W.H_C, alpha=W.H_ALPHA, amp_kind=1)
    b1 = O.births_at(P, T1, [5.0], [0.1], [0.0])
    b0 = O.births_at(P, T0, [5.0], [0.1], [0.0])
    ts = 5.0 + 1j * b1["tt"][0]
    E_ts = O.field(P, "E", [ts])[0]
    vz = b1["kz"][0] + O.field(P, "A", [ts])[0] - O.field(P, "A", [5.0])[0].real
    mag = np.exp(-b1["S_im"][0]) / abs(E_ts * vz)
    assert abs(abs(b1["amp_re"][0] + 1j * b1["amp_im"][0]) - mag) < 1e-12 * mag
    assert b0["tt"][0] == b1["tt"][0] and b0["S_im"][0] == b1["S_im"][0]
