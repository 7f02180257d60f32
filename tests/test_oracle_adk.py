"""Oracle pins for the ADK births (Sec. III.C): the ADK rate in place of the SFA
amplitude's modulus, the quasi-static tunnel exit, and the renormalisation to
the SFA rate near the pulse's two sub-peaks.

Pins:
  * the hydrogen ground state's static tunnelling rate (4/F) e^{-2/(3F)} (the
    textbook result for H(1s), whose tail constant is C_0 = 2);
  * in the quasi-static limit (w -> 0) the ADK density and the oracle's SFA
    amplitude |a|^2 share the tunnelling exponent exp(-2 kappa^3/(3F)) and the
    transverse width exp(-kappa k^2/F): their ratio carries no exponential in
    1/F nor in k^2/F, only the power F^3 of the prefactors;
  * the sub-peaks of the 1600 nm, 3-cycle pulse sit near +-110 a.u. (Sec.
    III.C, tests/golden/paper_values.txt);
  * after renormalisation, the ADK births' rate summed over the two sub-peaks
    equals the SFA births' rate there, both integrated over k_perp by a
    quadrature other than the renormalisation's own;
  * an ADK birth has kz = 0, q0 = -Ip/E(t0) and the phase Re S_down^0 of the
    SFA saddle of the same (t0, k_perp).
"""
import numpy as np
import pytest

import oracle as O
from paper_2601_17164_gb300 import workloads as W
from tests.helpers import paper_value


def _h(amp_kind=0):
    return O.make_target(O.POT_SOFTCORE, [0.3], ip=0.5, gto_l=0, c=W.H_C, alpha=W.H_ALPHA, amp_kind=amp_kind)


def _ar(amp_kind=0):
    t = W.ARGON
    return O.make_target(t.pot, t.pot_param, t.ip, 1, t.c, t.alpha, amp_kind=amp_kind)


def test_hydrogen_static_rate():
    T = _h()
    for F in (0.02, 0.035, 0.05, 0.08, 0.12):
        # C_0^2 = 4 times the oracle's rate (which leaves the tail constant out)
        assert abs(4 * O.adk_rate(T, F) / ((4 / F) * np.exp(-2 / (3 * F))) - 1) < 1e-13


@pytest.mark.parametrize("target", ["H", "Ar"])
def test_adk_and_sfa_share_the_quasistatic_exponent_and_width(target):
    T = _h() if target == "H" else _ar()
    kappa = np.sqrt(2 * T.ip)
    E0, w = 0.05, 2e-4                       # Keldysh parameter w kappa / E0 ~ 0.005
    P = O.make_pulse(E0=E0, omega=w, cw=True)
    cs = np.linspace(0.5, 1.0, 11)
    t0 = np.arccos(cs) / w
    F = E0 * cs
    for kp in (0.0, 0.15):
        b = O.births_at(P, T, t0, np.full_like(t0, kp), 0 * t0)
        a2 = b["amp_re"] ** 2 + b["amp_im"] ** 2
        rho = np.array([O.adk_density(T, f, kp * kp) for f in F])
        lr = np.log(a2 / rho)
        coef = np.linalg.lstsq(np.stack([np.ones_like(F), np.log(F), 1 / F], 1), lr, rcond=None)[0]
        # no leftover of the exponent 2 kappa^3/3 (0.67 for H) in 1/F
        assert abs(coef[2]) < 1e-3 * (2 * kappa ** 3 / 3), coef
    # the transverse widths agree: exp(-kappa k^2 / F) on both sides; what is left is
    # the SFA prefactor's slow k dependence (|v_s|, of order k^2/kappa^2) and the next
    # order of the exponent (k^4/(4 kappa F)), both a few per cent of the width term
    ks = np.array([0.0, 0.05, 0.1, 0.15, 0.2])
    b = O.births_at(P, T, np.zeros_like(ks), ks, 0 * ks)
    a2 = b["amp_re"] ** 2 + b["amp_im"] ** 2
    rho = np.array([O.adk_density(T, E0, k * k) for k in ks])
    drift = np.abs(np.log(a2 / rho) - np.log(a2[0] / rho[0]))
    assert np.all(drift <= 0.1 * kappa * ks ** 2 / E0), (drift, kappa * ks ** 2 / E0)


def test_subpeaks_of_the_1600nm_pulse():
    v, tol = paper_value("subpeak_time_au")
    P = O.make_pulse(1e14, 1600.0, 3.0)
    t = O.adk_subpeaks(P)
    assert abs(t[0] + v) < tol and abs(t[1] - v) < tol
    # carrier crests next to the central one: the opposite sign of E, and within a few
    # hundredths of a cycle of the local maxima of |E| (which the steep envelope shifts)
    T0 = 2 * np.pi / P.omega
    Ec = O.field(P, "E", [0.0])[0].real
    Es = O.field(P, "E", t).real
    assert np.all(np.sign(Es) == -np.sign(Ec))
    for tj in t:
        tt = tj + np.linspace(-0.2, 0.2, 4001) * T0
        tmax = tt[np.argmax(np.abs(O.field(P, "E", tt).real))]
        assert abs(tmax - tj) < 0.06 * T0


@pytest.mark.parametrize("target", ["H", "Ar"])
def test_renormalised_adk_rate_matches_sfa_at_the_subpeaks(target):
    T0, T2 = (_h(), _h(2)) if target == "H" else (_ar(), _ar(2))
    P = O.make_pulse(1e14, 1600.0, 3.0, cep=0.3)
    x, wq = np.polynomial.legendre.leggauss(200)
    kappa = np.sqrt(2 * T0.ip)
    tot = {0: 0.0, 2: 0.0}
    for tj in O.adk_subpeaks(P):
        F = abs(O.field(P, "E", [tj])[0].real)
        kmax = 10 * np.sqrt(F / kappa)
        k = 0.5 * kmax * (x + 1)
        for kind, T in ((0, T0), (2, T2)):
            b = O.births_at(P, T, np.full_like(k, tj), k, 0 * k)
            a2 = b["amp_re"] ** 2 + b["amp_im"] ** 2
            tot[kind] += np.sum(0.5 * kmax * wq * 2 * np.pi * k * a2)
    assert abs(tot[2] / tot[0] - 1) < 1e-5, tot


def test_adk_birth_exit_phase_and_modulus():
    P = O.make_pulse(1.5e14, 800.0, 8.0, cep=0.2)
    T0, T2 = _h(), _h(2)
    t0 = np.array([-12.0, 3.0, 45.0, -52.0])
    kx = np.array([0.0, 0.1, 0.0, 0.25])
    ky = np.array([0.0, -0.05, 0.3, 0.1])
    s = O.births_at(P, T0, t0, kx, ky)
    a = O.births_at(P, T2, t0, kx, ky)
    E = O.field(P, "E", t0).real
    n2 = O.adk_norm2(P, T2)
    assert n2 > 0
    assert np.all(a["kz"] == 0.0)
    assert np.allclose(a["qz"], -T2.ip / E, rtol=1e-15, atol=0)
    amp = a["amp_re"] + 1j * a["amp_im"]
    rho = np.array([O.adk_density(T2, abs(e), x * x + y * y) for e, x, y in zip(E, kx, ky)])
    assert np.allclose(np.abs(amp), np.sqrt(n2 * rho), rtol=1e-13, atol=0)
    # the phase is the SFA saddle's real action (same saddle: same t_t and S)
    assert np.array_equal(a["tt"], s["tt"]) and np.array_equal(a["S_re"], s["S_re"])
    assert np.all(np.abs(np.angle(amp * np.exp(-1j * s["S_re"]))) < 1e-12)
