"""Oracle pins: units and laser field (Sec. II.2 Eq. EfieldTDSE; Sec. III.C).

Each test checks the oracle against something it does not compute itself:
numbers the paper prints, complex-step derivatives, Gauss-Legendre quadrature.
"""
import numpy as np
import pytest

import oracle as O
from tests.helpers import paper_value

HARTREE_EV = 27.211386


def test_cutoff_near_90_eV_for_h_1600nm():
    # Sec. III.C: the cutoff for H at 1600 nm, 1e14 W/cm^2 lies "near 90 eV".
    # Ip + 3.17 Up with Up = E0^2 / (4 w^2) (textbook ponderomotive energy).
    E0 = O.E0_from_intensity(1e14)
    w = O.omega_from_lambda(1600.0)
    cutoff_ev = (0.5 + 3.17 * E0 ** 2 / (4 * w ** 2)) * HARTREE_EV
    assert abs(cutoff_ev - 89.4) < 0.1
    v, tol = paper_value("h_1600nm_1e14_cutoff_ev")
    assert abs(cutoff_ev - v) < tol
    # photon energy of 800 nm is 1.55 eV
    assert abs(O.omega_from_lambda(800.0) * HARTREE_EV - 1.5498) < 1e-3


def test_field_is_minus_dA_dt_complex_step():
    P = O.make_pulse(1.5e14, 800.0, 8.0, cep=0.7)
    t = np.linspace(-0.49 * P.Tp, 0.49 * P.Tp, 97)
    h = 1e-30
    dA = np.imag(O.field(P, "A", t + 1j * h)) / h          # complex-step derivative
    E = O.field(P, "E", t).real
    assert np.max(np.abs(E + dA)) < 1e-14 * P.E0 * 10


def test_F_and_G_are_antiderivatives_of_A_and_A2():
    P = O.make_pulse(1e14, 1600.0, 3.0, cep=0.3)
    t = np.linspace(-0.5 * P.Tp, 0.5 * P.Tp, 41)
    h = 1e-30
    A = O.field(P, "A", t).real
    dF = np.imag(O.field(P, "F", t + 1j * h)) / h
    dG = np.imag(O.field(P, "G", t + 1j * h)) / h
    assert np.max(np.abs(dF - A)) < 1e-13 * np.max(np.abs(A))
    assert np.max(np.abs(dG - A * A)) < 1e-13 * np.max(A * A)
    assert abs(O.field(P, "F", [0.0])[0]) == 0.0 and abs(O.field(P, "G", [0.0])[0]) == 0.0


@pytest.mark.parametrize("cycles", [1.0, 2.0, 6.0])
def test_complex_continuation_against_gauss_legendre(cycles):
    # int_{ta}^{tb} A and A^2 along a complex segment, 64-point Gauss-Legendre.
    P = O.make_pulse(1e14, 800.0, cycles, cep=0.4)
    x, wq = np.polynomial.legendre.leggauss(64)
    for ta, tb in [(10.0 + 0j, 30.0 + 15.0j), (-40.0 + 25.0j, -35.0 + 0j), (5.0 + 3j, 5.0 + 28j)]:
        tau = 0.5 * (ta + tb) + 0.5 * (tb - ta) * x
        A = O.field(P, "A", tau)
        qA = 0.5 * (tb - ta) * np.sum(wq * A)
        qA2 = 0.5 * (tb - ta) * np.sum(wq * A * A)
        F = O.field(P, "F", [ta, tb])
        G = O.field(P, "G", [ta, tb])
        assert abs((F[1] - F[0]) - qA) < 1e-12 * max(1.0, abs(qA))
        assert abs((G[1] - G[0]) - qA2) < 1e-12 * max(1.0, abs(qA2))


def test_pulse_edges_and_zero_area():
    P = O.make_pulse(1e14, 1600.0, 3.0)
    edges = [-0.5 * P.Tp, 0.5 * P.Tp]
    assert np.max(np.abs(O.field(P, "A", edges))) < 1e-16
    assert np.max(np.abs(O.field(P, "E", edges))) < 1e-16
    # E beyond the pulse is zero on the integrator's real grid
    assert np.all(O.field_E_grid(P, [-0.51 * P.Tp, 0.6 * P.Tp]) == 0.0)
    # the pulse has zero area: int E dt = A(-Tp/2) - A(Tp/2) = 0 (Simpson)
    t = np.linspace(-0.5 * P.Tp, 0.5 * P.Tp, 20001)
    E = O.field_E_grid(P, t)
    h = t[1] - t[0]
    area = h / 3 * (E[0] + E[-1] + 4 * E[1:-1:2].sum() + 2 * E[2:-1:2].sum())
    assert abs(area) < 1e-10


def test_envelope_reading_subpeaks_almost_factor_two_weaker():
    # Sec. III.C: at 1600 nm, 3 cycles, the sub-cycle peaks near +-110 a.u. are
    # "almost a factor of two weaker" in intensity than the central peak.  The
    # zero-to-zero N-cycle sin^2 reading gives cos^4(pi/6) = 0.5625.
    P = O.make_pulse(1e14, 1600.0, 3.0)
    t = np.linspace(-0.5 * P.Tp, 0.5 * P.Tp, 200001)
    E = O.field_E_grid(P, t)
    i0 = np.argmax(np.abs(E))
    assert abs(t[i0]) < 0.5                     # the peak is at t = 0 (CEP 0)
    T0 = 2 * np.pi / P.omega
    a = np.abs(E)
    is_max = (a[1:-1] > a[:-2]) & (a[1:-1] >= a[2:])
    t_max = t[1:-1][is_max]
    for sgn in (-1, 1):
        # at t = +-T0/2 the envelope-derivative term vanishes (sin(w t) = 0), so
        # the intensity ratio is exactly cos^4(pi/6); the 2N-cycle reading gives 0.87
        e_half = O.field_E_grid(P, [sgn * 0.5 * T0])[0]
        assert abs((e_half / E[i0]) ** 2 - np.cos(np.pi / 6) ** 4) < 1e-12
        j = np.argmin(np.abs(t_max - sgn * 0.5 * T0))     # local maximum nearest to +-T0/2
        tj = t_max[j]
        v, tol = paper_value("subpeak_time_au")
        assert abs(abs(tj) - v) < tol                    # sub-peaks near +-110 a.u.
        ratio = (O.field_E_grid(P, [tj])[0] / E[i0]) ** 2
        v, tol = paper_value("subpeak_intensity_ratio")
        assert abs(ratio - v) < tol and ratio > 0.5


def test_hanning_window_vanishes_at_pulse_end():
    # App. D: W_H = 0 when the pulse ends; tau_H = Tp/2.  The oracle's DFT of a
    # constant signal weights the bins with W_H; check W_H via a one-bin signal.
    P = O.make_pulse(1e14, 800.0, 2.0)
    tau = 0.5 * P.Tp
    for t_k, W in [(-tau, 0.0), (0.0, 1.0), (0.5 * tau, 0.5), (tau, 0.0)]:
        X = O.spectrum([1.0], t_k, 1.0, tau, [0.0])
        assert abs(X[0] - W) < 1e-15


def test_thresholds_and_run_parameters_printed_in_the_paper():
    # the SFA parameters Ip of the workloads sit at the thresholds the paper marks
    from paper_2601_17164_gb300 import workloads as W
    v, tol = paper_value("h_threshold_ev")
    assert abs(W.HYDROGEN.ip * HARTREE_EV - v) < tol
    v, tol = paper_value("ar_threshold_ev")
    assert abs(W.ARGON.ip * HARTREE_EV - v) < tol
    # every workload uses the paper's coherent-state width and removal cutoff
    for w in (W.H_800_2CYC_GRID, W.H_800_8CYC_1M, W.AR_1600_6CYC_10M, W.AR_2000_20CYC_100M, W.H_1600_3CYC_2M):
        assert w.gamma == paper_value("coherent_state_gamma")[0]
        assert w.d_t == paper_value("removal_d_t")[0]
