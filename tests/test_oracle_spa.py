"""Oracle pins for the birth amplitude (App. A: Eq. SFAwf, Eq. Int, Eq. SFHKwf;
App. B.2: Eq. SFHKmodSPA).

The oracle assembles the amplitude of a birth (t0, k) from closed forms:
  standard saddle point   M(v_s) / sqrt(E(t_s) v_s) e^{i(S + p0.q0)},
  modified saddle point   e^{i(S + p0.q0)} / (E(t_s) v_s),
with M(v) = E(t_s) <v|z|psi0>, v_s = k + A(t_s) - A(t0) and S the tunnelling
action at the saddle t_s.  Each closed form is the saddle-point value of the SFA
time integral behind Eq. SFAwf,
  J = int dt E(t) m(k + A(t) - A(t0)) e^{i S(t)},
  S(t) = Ip t - int_t^{t0} (k + A(t'') - A(t0))^2 / 2 dt'',
times the factor e^{i p0.q0} of the coherent-state overlap in Eq. Int.  The tests
below evaluate J by quadrature along a line through the saddle (the integrand is
entire for GTO matrix elements) or just below it (the hydrogenic matrix element
has a pole of order 3 at the saddle, the case App. B.2 addresses), S(t_s) by
quadrature along the segment [t_s, t0], and e^{i p0.q0} by brute-force quadrature
of the position-space overlap of the coherent state with its own plane wave.
None of these use the oracle's action, exit point or amplitude code; they use
its field A(t), E(t) and tunnelling element, each pinned elsewhere.

In the saddle-point limit (weak field: the reduced field E/kappa^3 -> 0, kappa =
sqrt(2 Ip + k_perp^2)) J divided by the oracle's amplitude tends to a constant
that does not depend on the birth:
  standard:  -i sqrt(2 pi i) = sqrt(2 pi) e^{-i pi/4}  (the constant dropped in
             Eq. SFAwf: S''(t_s) = -E(t_s).v_s and the Gaussian integral along the
             steepest-descent direction);
  modified:  -pi/16 for m(v) = v_z / (v^2 + 2 Ip)^3, from
             int u^{-3} e^{i S'' u^2/2} du = -(pi/2) S'' on a contour below the pole
             (the real-time contour passes below t_s).
The standard ratio approaches its limit linearly in E, the modified one as
sqrt(E); the tests check the ratios and their Richardson extrapolations.  A
missing square root, the other branch of the root, 1/sqrt(E.v) in place of
1/(E.v), or e^{-i p0.q0} in place of e^{+i p0.q0} (kz qz reaches hundreds of
radians here) each moves a ratio far from its constant.
"""
import numpy as np
import pytest

import oracle as O

_XG, _WG = np.polynomial.legendre.leggauss(16)
_X64, _W64 = np.polynomial.legendre.leggauss(64)


def _action_along(P, ip, k_perp2, kz, A0, path):
    """S(path[j]) - S(path[0]) = int (Ip + v^2/2) dt along the polyline `path`
    (S as a function of its lower limit: dS/dt = Ip + v(t)^2 / 2)."""
    a, b = path[:-1], path[1:]
    s = 0.5 * (a + b)[:, None] + 0.5 * (b - a)[:, None] * _XG[None, :]
    A = O.field(P, "A", s.ravel()).reshape(s.shape)
    v2 = k_perp2 + (kz + A - A0) ** 2
    seg = 0.5 * (b - a) * np.sum(_WG[None, :] * (ip + 0.5 * v2), axis=1)
    return np.concatenate([[0.0], np.cumsum(seg)])


def _action_at_saddle(P, ip, k_perp2, kz, A0, t0, ts):
    """S(t_s) = Ip t_s - int_{t_s}^{t0} v^2/2 along the segment, 64-point Gauss-Legendre."""
    tau = 0.5 * (ts + t0) + 0.5 * (t0 - ts) * _X64
    A = O.field(P, "A", tau)
    v2 = k_perp2 + (kz + A - A0) ** 2
    return ip * ts - 0.5 * (t0 - ts) * np.sum(_W64 * v2 / 2)


def _overlap_phase(p, q, gam=0.05):
    """e^{i arg <p, q, gamma | k = p>} by quadrature of the 1D position-space overlap,
    coherent state (2 gamma/pi)^{1/4} e^{-gamma (x-q)^2 + i p (x-q)} (the convention of
    the recombination elements, App. C) and plane wave <x|k> = (2 pi)^{-1/2} e^{i k x}
    (the conjugate of the tunnelling element's <k|x>)."""
    h = 0.01
    x = q + np.arange(-40.0, 40.0 + h / 2, h) / np.sqrt(gam)
    phi = (2 * gam / np.pi) ** 0.25 * np.exp(-gam * (x - q) ** 2 + 1j * p * (x - q))
    ov = np.sum(np.conj(phi) * np.exp(1j * p * x)) * (x[1] - x[0]) / np.sqrt(2 * np.pi)
    return ov / abs(ov)


def _birth(P, T, t0, kx, ky):
    b = O.births_at(P, T, [t0], [kx], [ky])
    assert b["valid"][0] == 1
    return {k: v[0] for k, v in b.items()}


def _spa_ratio(P, T, t0, kx, ky, n=801, width=10.0):
    """J (line through t_s) / oracle amplitude, with e^{iS(t_s)} and e^{i p0.q0} from
    the quadratures above."""
    b = _birth(P, T, t0, kx, ky)
    kz, qz, ts = b["kz"], b["qz"], t0 + 1j * b["tt"]
    kp2 = kx * kx + ky * ky
    A0 = O.field(P, "A", [t0])[0].real
    Spp = -O.field(P, "E", [ts])[0] * (kz + O.field(P, "A", [ts])[0] - A0)
    u = np.linspace(-width, width, n) / np.sqrt(abs(Spp))
    dS = _action_along(P, T.ip, kp2, kz, A0, ts + u)
    dS -= dS[n // 2]
    A, E = O.field(P, "A", ts + u), O.field(P, "E", ts + u)
    m = np.array([O.tunnel_element(T, [kx, ky, kz + A[j] - A0]) for j in range(n)])
    g = E * m * np.exp(1j * dS)
    assert abs(g[0]) < 1e-12 * np.max(abs(g)) and abs(g[-1]) < 1e-12 * np.max(abs(g))   # truncation
    J = np.trapezoid(g, u)
    S = _action_at_saddle(P, T.ip, kp2, kz, A0, t0, ts)
    amp = b["amp_re"] + 1j * b["amp_im"]
    return J * np.exp(1j * S) * _overlap_phase(kz, qz) / amp


def _pole_ratio(P, ip, t0, kx, ky, n=4001, width=12.0, depth=1.0):
    """J for m(v) = v_z/(v^2 + 2 Ip)^3 on the line Im t = t_t - depth/sqrt|S''| (below the
    pole at t_s), divided by the oracle's modified-SPA amplitude."""
    T = O.make_target(O.POT_ZERO, [], ip=ip, gto_l=0, c=[1.0], alpha=[1.0], amp_kind=1)
    b = _birth(P, T, t0, kx, ky)
    kz, qz, ts = b["kz"], b["qz"], t0 + 1j * b["tt"]
    kp2 = kx * kx + ky * ky
    A0 = O.field(P, "A", [t0])[0].real
    Spp = -O.field(P, "E", [ts])[0] * (kz + O.field(P, "A", [ts])[0] - A0)
    sig = 1.0 / np.sqrt(abs(Spp))
    base = ts - 1j * depth * sig
    x = np.linspace(-width, width, n) * sig
    # S relative to S(t_s): down from t_s to the line, then along it from its centre
    down = _action_along(P, ip, kp2, kz, A0, ts - 1j * np.linspace(0.0, depth * sig, 65))[-1]
    right = _action_along(P, ip, kp2, kz, A0, base + x[n // 2:])
    left = _action_along(P, ip, kp2, kz, A0, base + x[: n // 2 + 1][::-1])[::-1]
    dS = down + np.concatenate([left[:-1], right])
    line = base + x
    A, E = O.field(P, "A", line), O.field(P, "E", line)
    vz = kz + A - A0
    g = E * vz / (kp2 + vz * vz + 2 * ip) ** 3 * np.exp(1j * dS)
    J = np.trapezoid(g, x)
    S = _action_at_saddle(P, ip, kp2, kz, A0, t0, ts)
    amp = b["amp_re"] + 1j * b["amp_im"]
    return J * np.exp(1j * S) * _overlap_phase(kz, qz) / amp


def _births(E0):
    w = 0.25 * E0           # Keldysh parameter ~ 1: kz and hence kz qz are far from zero
    return [(0.0, 0.0, 0.0), (0.8 / w, 0.3, -0.2), ((np.pi + 0.4) / w, 0.1, 0.0)]


def test_overlap_phase_is_plus_p_dot_q():
    # <p, q, gamma | p> = |.| e^{+i p q} for any gamma (Eq. Int's e^{i p0.q0})
    for p, q, g in [(0.3, -150.0, 0.05), (-1.1, 37.5, 0.5), (0.02, 2000.0, 0.01)]:
        z = _overlap_phase(p, q, g)
        assert abs(z - np.exp(1j * p * q)) < 1e-10


def test_second_derivative_of_tunnelling_action():
    # S''(t_s) = -E(t_s).v_s: the quantity under the root of Eq. SFAwf (up to sign)
    P = O.make_pulse(1.5e14, 800.0, 8.0, cep=0.2)
    T = O.make_target(O.POT_ZERO, [], ip=0.5, gto_l=0, c=[1.0], alpha=[1.0])
    for t0, kx, ky in [(-12.0, 0.0, 0.0), (3.0, 0.1, -0.05), (45.0, 0.0, 0.3)]:
        b = _birth(P, T, t0, kx, ky)
        ts = t0 + 1j * b["tt"]
        A0 = O.field(P, "A", [t0])[0].real
        vz = b["kz"] + O.field(P, "A", [ts])[0] - A0
        h = 0.05
        pts = ts + h * np.arange(-2, 3)
        S = _action_along(P, T.ip, kx * kx + ky * ky, b["kz"], A0, pts)
        d2 = (-S[4] + 16 * S[3] - 30 * S[2] + 16 * S[1] - S[0]) / (12 * h * h)
        want = -O.field(P, "E", [ts])[0] * vz
        assert abs(d2 - want) < 1e-6 * abs(want)
        # the first derivative vanishes there: Eq. SAPeq
        d1 = (S[0] - 8 * S[1] + 8 * S[3] - S[4]) / (12 * h)
        assert abs(d1) < 1e-8 * abs(want)


@pytest.mark.parametrize("l", [0, 1])
def test_standard_spa_amplitude_is_the_saddle_value_of_the_sfa_integral(l):
    c0 = np.sqrt(2 * np.pi) * np.exp(-0.25j * np.pi)       # -i sqrt(2 pi i)
    T = O.make_target(O.POT_ZERO, [], ip=2.0, gto_l=l, c=[1.0], alpha=[2.0])
    R = {}
    for E0 in (0.02, 0.01):
        P = O.make_pulse(E0=E0, omega=0.25 * E0, cw=True)
        R[E0] = np.array([_spa_ratio(P, T, *b) for b in _births(E0)]) / c0
    # O(E) approach to the constant, then Richardson in E
    assert np.all(np.abs(R[0.01] - 1) < 6e-3), R[0.01]
    assert np.all(np.abs(R[0.02] - 1) > np.abs(R[0.01] - 1))
    assert np.all(np.abs(2 * R[0.01] - R[0.02] - 1) < 5e-4), 2 * R[0.01] - R[0.02]


def test_modified_spa_amplitude_is_the_pole_value_of_the_sfa_integral():
    c0 = -np.pi / 16
    R = {}
    for E0 in (0.02, 0.005):
        P = O.make_pulse(E0=E0, omega=0.25 * E0, cw=True)
        R[E0] = np.array([_pole_ratio(P, 1.0, *b) for b in _births(E0)]) / c0
    # the contour's depth below the pole does not matter (the integrand is analytic there)
    P = O.make_pulse(E0=0.02, omega=0.005, cw=True)
    t0, kx, ky = _births(0.02)[1]
    assert abs(_pole_ratio(P, 1.0, t0, kx, ky, depth=0.6) / c0 - R[0.02][1]) < 1e-9
    # O(sqrt E) approach to the constant, then Richardson in sqrt E
    assert np.all(np.abs(R[0.005] - 1) < 0.04), R[0.005]
    assert np.all(np.abs(2 * R[0.005] - R[0.02] - 1) < 2e-3), 2 * R[0.005] - R[0.02]
