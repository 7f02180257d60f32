"""Oracle pins: classical propagation, stability blocks, action, HK prefactor
(App. A after Eq. HKpropa, Eq. C_HK) and trajectory removal (Sec. III.A).

Pins: Volkov closed forms (V = 0), free-particle prefactor (1 - i gamma t)^{3/2},
harmonic-oscillator closed forms and the exact RK4 amplification matrix,
Duhamel's formula, the whole HK contribution of one trajectory and the HK
phase-space integral against grid quantum mechanics where HK is exact (driven
harmonic oscillator), symplecticity / energy / reversibility scaling as dt^4,
the 3.17 Up classical return energy, rotational invariance and sharding.
"""
import numpy as np
import pytest
from scipy import optimize
from scipy.integrate import solve_ivp

import oracle as O
from paper_2601_17164_gb300 import workloads as W

IQ, IP, IMQQ, IMQP, IMPQ, IMPP, IS = 0, 3, 6, 15, 24, 33, 42


def blocks(y):
    return (y[IMQQ:IMQQ + 9].reshape(3, 3), y[IMQP:IMQP + 9].reshape(3, 3),
            y[IMPQ:IMPQ + 9].reshape(3, 3), y[IMPP:IMPP + 9].reshape(3, 3))


def zero_target(pot=O.POT_ZERO, param=()):
    return O.make_target(pot, param, ip=0.5, gto_l=0, c=W.H_C, alpha=W.H_ALPHA)


def test_volkov_closed_forms():
    # V = 0 with the field on: p(t) = p0 + A(t) - A(t0) z, q and S from the
    # closed-form integrals of A and A^2; Mqq = Mpp = I, Mqp = (t - t0) I, Mpq = 0.
    P = O.make_pulse(1.5e14, 800.0, 4.0, cep=0.3)
    T = zero_target()
    G = O.pulse_grid(P, 0.02, 0.1)
    rng = np.random.default_rng(1)
    n = 6
    n0 = np.sort(rng.integers(100, G.n_steps // 2, n)).astype(np.int32)
    q0 = rng.uniform(-3, 3, (3, n))
    p0 = rng.uniform(-1, 1, (3, n))
    n_end = int(0.8 * G.n_steps)
    st, Cc, fl = O.propagate(P, T, G, n0, q0, p0, n_end)
    assert np.all(fl == 0)
    t = G.t_start + n_end * G.dt
    At = O.field(P, "A", [t])[0].real
    Ft, Gt = O.field(P, "F", [t])[0].real, O.field(P, "G", [t])[0].real
    for i in range(n):
        t0 = G.t_start + n0[i] * G.dt
        A0 = O.field(P, "A", [t0])[0].real
        F0, G0 = O.field(P, "F", [t0])[0].real, O.field(P, "G", [t0])[0].real
        tau = t - t0
        c = p0[2, i] - A0
        p = p0[:, i] + np.array([0, 0, At - A0])
        q = q0[:, i] + np.array([p0[0, i], p0[1, i], c]) * tau + np.array([0, 0, Ft - F0])
        pperp2 = p0[0, i] ** 2 + p0[1, i] ** 2
        S = 0.5 * (pperp2 + c * c) * tau - 0.5 * (Gt - G0) + q[2] * At - q0[2, i] * A0
        y = st[:, i]
        assert np.allclose(y[IP:IP + 3], p, rtol=0, atol=1e-12)
        assert np.allclose(y[IQ:IQ + 3], q, rtol=0, atol=1e-10)
        assert abs(y[IS] - S) < 1e-10 * max(1, abs(S))
        Mqq, Mqp, Mpq, Mpp = blocks(y)
        assert np.allclose(Mqq, np.eye(3), atol=1e-13) and np.allclose(Mpp, np.eye(3), atol=1e-13)
        assert np.allclose(Mqp, tau * np.eye(3), atol=1e-10) and np.allclose(Mpq, 0, atol=1e-13)
        M = np.block([[Mqq, Mqp], [Mpq, Mpp]])
        assert abs(np.linalg.det(M) - 1) < 1e-12


@pytest.mark.parametrize("gam", [0.5, 0.2])
def test_free_particle_prefactor_and_branch(gam):
    # C(tau) = (1 - i gamma tau)^{3/2}; det Z = (1 - i gamma tau)^3 crosses the
    # negative real axis at tau = sqrt(3)/gamma where the principal sqrt flips.
    P = O.make_pulse(E0=0.0, omega=0.057, cycles=2.0)
    T = zero_target()
    G = O.make_grid(0.0, 0.02, 2000, 5, gamma=gam)
    for n_end in [50, 150, int(np.sqrt(3) / gam / 0.02) + 5, 1000, 2000]:
        st, Cc, fl = O.propagate(P, T, G, [0], [0.1, 0.2, -0.3], [0.3, -0.1, 0.5], n_end)
        tau = n_end * 0.02
        ref = np.exp(1.5 * np.log(1 - 1j * gam * tau))   # continuous (Re > 0 branch)
        assert abs(Cc[0] - ref) < 1e-12 * abs(ref)
        assert abs(abs(Cc[0]) ** 2 - (1 + gam ** 2 * tau ** 2) ** 1.5) < 1e-11 * abs(ref) ** 2
        # principal sqrt of det Z disagrees beyond tau = sqrt(3)/gamma
        if tau > np.sqrt(3) / gam:
            assert abs(np.sqrt(O.det_Z(st[:, 0], gam)) + ref) < 1e-10 * abs(ref)


def _rk4_amplification(w, h):
    L = np.array([[0.0, 1.0], [-w * w, 0.0]]) * h
    return np.eye(2) + L + L @ L / 2 + L @ L @ L / 6 + L @ L @ L @ L / 24


def test_harmonic_oscillator_rk4_exact_and_closed_forms():
    # V = w^2 r^2/2, field off, gamma = w/2: M blocks are cos/sin; C = e^{-3 i w tau/2}
    # continuous over many windings; S = (p.q - p0.q0)/2; and the computed M equals
    # the RK4 amplification matrix to the N-th power (exact for a linear ODE).
    w = 1.3
    P = O.make_pulse(E0=0.0, omega=0.057, cycles=2.0)
    T = zero_target(O.POT_HARMONIC, [w])
    h = 0.01
    N = 3000
    G = O.make_grid(0.0, h, N, 10, gamma=w / 2)
    q0 = np.array([0.3, -0.2, 0.5])
    p0 = np.array([0.1, 0.4, -0.3])
    st, Cc, fl = O.propagate(P, T, G, [0], q0, p0, N)
    y = st[:, 0]
    Mqq, Mqp, Mpq, Mpp = blocks(y)
    R = np.linalg.matrix_power(_rk4_amplification(w, h), N)
    for B, ref in [(Mqq, R[0, 0]), (Mqp, R[0, 1]), (Mpq, R[1, 0]), (Mpp, R[1, 1])]:
        assert np.allclose(B, ref * np.eye(3), rtol=0, atol=1e-12 * max(1, abs(ref)))
    tau = N * h
    assert np.allclose([Mqq[0, 0], Mqp[0, 0], Mpq[0, 0]], [np.cos(w * tau), np.sin(w * tau) / w,
                                                           -w * np.sin(w * tau)], atol=1e-7)
    assert abs(Cc[0] - np.exp(-1.5j * w * tau)) < 1e-6    # 1.5 w tau ~ 58 rad: many windings
    q, p = y[IQ:IQ + 3], y[IP:IP + 3]
    assert abs(y[IS] - 0.5 * (p @ q - p0 @ q0)) < 1e-7
    x = w * h
    M6 = np.block([[Mqq, Mqp], [Mpq, Mpp]])
    assert abs(np.linalg.det(M6) / (1 - x ** 6 / 72 + x ** 8 / 576) ** (3 * N) - 1) < 1e-12


def test_harmonic_oscillator_driven_duhamel():
    # field on: q_z(t) = q0 cos w tau + p0 sin(w tau)/w - int sin(w (t - s))/w E(s) ds
    w = 0.9
    P = O.make_pulse(1e14, 800.0, 2.0, cep=0.4)
    T = zero_target(O.POT_HARMONIC, [w])
    G = O.pulse_grid(P, 0.002, 0.1, gamma=w / 2)
    n0, n_end = 20000, 90000
    q0 = np.array([0.0, 0.1, 0.4])
    p0 = np.array([0.2, 0.0, -0.1])
    st, Cc, fl = O.propagate(P, T, G, [n0], q0, p0, n_end)
    t0, t1 = G.t_start + n0 * G.dt, G.t_start + n_end * G.dt
    x, wq = np.polynomial.legendre.leggauss(40)
    edges = np.linspace(t0, t1, 201)
    integ = 0.0
    dinteg = 0.0
    for a, b in zip(edges[:-1], edges[1:]):
        s = 0.5 * (a + b) + 0.5 * (b - a) * x
        E = O.field_E_grid(P, s)
        integ += 0.5 * (b - a) * np.sum(wq * np.sin(w * (t1 - s)) / w * E)
        dinteg += 0.5 * (b - a) * np.sum(wq * np.cos(w * (t1 - s)) * E)
    tau = t1 - t0
    qz = q0[2] * np.cos(w * tau) + p0[2] * np.sin(w * tau) / w - integ
    pz = -w * q0[2] * np.sin(w * tau) + p0[2] * np.cos(w * tau) - dinteg
    assert abs(st[IQ + 2, 0] - qz) < 1e-10
    assert abs(st[IP + 2, 0] - pz) < 1e-10
    assert abs(Cc[0] - np.exp(-1.5j * w * tau)) < 1e-10   # the field does not change M



def _fourier_grid(L, N, w):
    # Fourier-grid Hamiltonian on [-L, L): exact kinetic energy k^2/2 in the plane-wave
    # basis, V = w^2 x^2/2 on the points; eigenpairs by dense diagonalisation
    h = 2 * L / N
    x = (np.arange(N) - N // 2) * h
    k = 2 * np.pi * np.fft.fftfreq(N, d=h)
    T = np.fft.ifft(np.fft.fft(np.eye(N), axis=0) * (0.5 * k * k)[:, None], axis=0).real
    E, U = np.linalg.eigh(0.5 * (T + T.T) + np.diag(0.5 * w * w * x * x))
    return x, h, k, E, U


def _cs(x, q, p, gam):
    return (2 * gam / np.pi) ** 0.25 * np.exp(-gam * (x - q) ** 2 + 1j * p * (x - q))


def _quantum_bins(P, T, G, w, birth, M=40):
    """-2 Re[e^{-i Ip t} amp <psi0| d e^{-iH(t-t0)} |p0,q0,gamma>] on the bins (Eq. D_t,
    Eq. V_t) for H = p^2/2 + w^2 r^2/2 + z E(t), by grid quantum mechanics: every factor
    separates in x, y, z; x and y by the eigenpairs, z by the TDSE in the lowest M
    eigenstates (interaction picture about t0, DOP853)."""
    x, h, k, E, U = _fourier_grid(16.0, 512, w)
    gam = G.gamma
    t0 = G.t_start + birth["n0"] * G.dt
    nb = G.n_steps // G.n_out + 1
    kk = np.arange(nb)
    sel = kk * G.n_out >= birth["n0"]
    tk = G.t_start + kk[sel] * G.n_out * G.dt
    tau = tk - t0

    def free(q, p):
        return (U @ (np.exp(-1j * np.outer(E, tau)) * (U.T @ _cs(x, q, p, gam))[:, None])).T

    fx, fy = free(0.0, birth["px"]), free(0.0, birth["py"])
    Um, Em = U[:, :M], E[:M]
    Zm = Um.T @ (x[:, None] * Um)
    c0 = np.sqrt(h) * (Um.T @ _cs(x, birth["qz"], birth["pz"], gam)).astype(complex)
    assert abs(np.vdot(c0, c0) - 1) < 1e-13          # the truncated basis holds the state

    def rhs(t, b):
        ph = np.exp(1j * Em * (t - t0))
        return -1j * O.field_E_grid(P, np.array([t]))[0] * (ph * (Zm @ (b / ph)))
    if P.E0 != 0.0:
        B = solve_ivp(rhs, (t0, tk[-1]), c0, method="DOP853", rtol=1e-12, atol=1e-14, t_eval=tk).y
    else:
        B = np.repeat(c0[:, None], len(tk), axis=1)
    fz = (Um @ (np.exp(-1j * np.outer(Em, tau)) * B)).T / np.sqrt(h)
    kz_fz = np.fft.ifft(k[None, :] * np.fft.fft(fz, axis=1), axis=1)     # -i d/dz
    dl = np.zeros(len(tk), complex)
    dv = np.zeros(len(tk), complex)
    for cj, aj in zip(T.c[:T.n_gto], T.alpha[:T.n_gto]):
        g = np.exp(-aj * x * x)
        gz = g if T.gto_l == 0 else x * g                 # psi0 = (1 or z) sum_j c_j e^{-a_j r^2}
        ixy = (h * fx @ g) * (h * fy @ g)
        dl += cj * ixy * (h * fz @ (x * gz))
        dv += cj * ixy * (h * kz_fz @ gz)
    ph = np.exp(-1j * T.ip * tk) * (birth["amp_re"] + 1j * birth["amp_im"])
    out_l, out_v = np.zeros(nb), np.zeros(nb)
    out_l[sel], out_v[sel] = -2 * np.real(dl * ph), -2 * np.real(dv * ph)
    return out_l, out_v


@pytest.mark.parametrize("l", [0, 1])
@pytest.mark.parametrize("E0", [0.0, 0.09])
def test_hk_contribution_exact_for_driven_harmonic_oscillator(l, E0):
    # For a Hamiltonian at most quadratic in (q, p) -- here V = w^2 r^2/2 plus the
    # length-gauge z E(t) -- and gamma = w/2 the coherent state stays a coherent state,
    # and one trajectory's C e^{iS} |p_t,q_t,gamma> (Eq. HKpropa, Eq. C_HK) is the exact
    # propagated state. So the oracle's bins of a single birth must equal grid quantum
    # mechanics, over hundreds of windings of C (branch), with the field's share of S,
    # the e^{-i Ip t} phase, the coherent-state convention and both dipole forms.
    # The residual is the RK4 error: 1.7e-7, 1.1e-8, 5.9e-10 at dt = 0.01, 0.005, 0.0025.
    w = 1.3 if E0 == 0.0 else 0.9
    P = O.make_pulse(E0=E0, omega=0.057, cycles=2.0)
    T = O.make_target(O.POT_HARMONIC, [w], ip=0.37, gto_l=l, c=[0.5, 0.3, 0.2], alpha=[0.25, 0.9, 2.5])
    dt = 0.005
    G = O.make_grid(-0.5 * P.Tp, dt, int(round(P.Tp / dt)), 200, gamma=w / 2)
    for b in ({"n0": 1000, "px": 0.3, "py": -0.5, "pz": 0.9, "qz": 1.2, "amp_re": 0.7, "amp_im": -0.4},
              {"n0": 7321, "px": -0.2, "py": 0.1, "pz": -1.1, "qz": -0.8, "amp_re": -0.3, "amp_im": 0.5}):
        ql, qv = _quantum_bins(P, T, G, w, b)
        births = {k: np.array([v], dtype=np.int32 if k == "n0" else np.float64) for k, v in b.items()}
        ol, ov, st = O.dipole(P, T, G, births)
        assert st["removed"] == 0 and st["branch_guard"] == 0
        assert np.max(np.abs(ol - ql)) < 3e-8 * np.max(np.abs(ql))
        assert np.max(np.abs(ov - qv)) < 3e-8 * np.max(np.abs(qv))


def _cs_overlap(a, b):
    """<a|b> of normalised 1D coherent states (2g/pi)^{1/4} e^{-g (x-q)^2 + i p (x-q)},
    a = (g, q, p), by the Gaussian integral (arrays broadcast)."""
    g1, q1, p1 = a
    g2, q2, p2 = b
    A = g1 + g2
    B = 2 * g1 * q1 + 2 * g2 * q2 + 1j * (p2 - p1)
    c = -g1 * q1 ** 2 - g2 * q2 ** 2 + 1j * (p1 * q1 - p2 * q2)
    return (4 * g1 * g2 / np.pi ** 2) ** 0.25 * np.sqrt(np.pi / A) * np.exp(B * B / (4 * A) + c)


@pytest.mark.parametrize("gam,E0", [(0.65, 0.0), (0.3, 0.3), (1.1, 0.3)])
def test_hk_phase_space_integral_exact_for_harmonic_oscillator(gam, E0):
    # <g'| K_HK |g> = (2 pi)^{-1} sum over a 64 x 64 rectangle rule in the (q0, p0) plane of
    # <g'|p_t,q_t,gamma> C e^{iS} <p0,q0,gamma|g> (Eq. HKpropa, 1D slice along z), with C the
    # square root of the z entry of Z from the z-blocks of the 3D integrator (Eq. C_HK). For a
    # Hamiltonian at most quadratic in (q, p) HK is exact for every gamma, also where single
    # trajectories are not (gamma != w/2): against grid quantum mechanics (Fourier grid,
    # TDSE in the oscillator eigenbasis). The integrand is Gaussian, so the rule converges
    # spectrally; what remains is the RK4 error.
    w = 1.3
    P = O.make_pulse(E0=E0, omega=0.057, cycles=2.0)
    T = zero_target(O.POT_HARMONIC, [w])
    dt = 0.005
    G = O.make_grid(-0.5 * P.Tp, dt, int(round(P.Tp / dt)), 200, gamma=gam)
    n0, n1 = 4000, 12000                       # tau = 40: ~8 windings of e^{-i w tau/2}
    t0, t1 = G.t_start + n0 * dt, G.t_start + n1 * dt
    ga, qa, pa = 0.5, 0.8, 0.4                 # |g>
    rq, rp = np.sqrt(40 * (gam + ga) / (gam * ga)), np.sqrt(160 * (gam + ga))
    Q0, P0 = (m.ravel() for m in np.meshgrid(qa + np.linspace(-rq, rq, 64), pa + np.linspace(-rp, rp, 64),
                                              indexing="ij"))
    hq, hp = 2 * rq / 63, 2 * rp / 63
    n = Q0.size
    q0, p0 = np.zeros((3, n)), np.zeros((3, n))
    q0[2], p0[2] = Q0, P0
    st, C3, fl = O.propagate(P, T, G, np.full(n, n0, np.int32), q0, p0, n1)
    assert np.all(fl == 0)
    zz = [st[o + 8] for o in (IMQQ, IMQP, IMPQ, IMPP)]     # z-z entries of the four blocks
    Z = 0.5 * (zz[0] + zz[3] - 2j * gam * zz[1] - zz[2] / (2j * gam))
    C = np.sqrt(Z)
    C = np.where(np.abs(C ** 3 - C3) < np.abs(C ** 3 + C3), C, -C)   # branch of the tracked 3D C
    assert np.max(np.abs(C ** 3 - C3) / np.abs(C3)) < 1e-12           # isotropic: det Z = Z_zz^3
    if gam == w / 2:                                                  # matched: C = e^{-i w tau/2}
        assert np.max(np.abs(C - np.exp(-0.5j * w * (t1 - t0)))) < 1e-7
    wg = _cs_overlap((gam, Q0, P0), (ga, qa, pa))
    x, h, k, E, U = _fourier_grid(16.0, 512, w)
    Um, Em = U[:, :60], E[:60]
    c0 = np.sqrt(h) * (Um.T @ _cs(x, qa, pa, ga)).astype(complex)
    assert abs(np.vdot(c0, c0) - 1) < 1e-12
    if E0 != 0.0:
        Zm = Um.T @ (x[:, None] * Um)

        def rhs(t, b):
            ph = np.exp(1j * Em * (t - t0))
            return -1j * O.field_E_grid(P, np.array([t]))[0] * (ph * (Zm @ (b / ph)))
        c0 = solve_ivp(rhs, (t0, t1), c0, method="DOP853", rtol=1e-12, atol=1e-14).y[:, -1]
    psi = (Um @ (np.exp(-1j * Em * (t1 - t0)) * c0)) / np.sqrt(h)
    for gb, qb, pb in ((0.5, 0.8, 0.4), (0.9, -1.0, 0.7), (0.4, 1.5, -1.2), (0.65, 0.0, 0.0)):
        quad = h * np.vdot(_cs(x, qb, pb, gb), _cs(x, -0.3, 0.2, 0.7))          # the overlap by quadrature
        assert abs(_cs_overlap((gb, qb, pb), (0.7, -0.3, 0.2)) - quad) < 1e-13
        hk = hq * hp / (2 * np.pi) * np.sum(_cs_overlap((gb, qb, pb), (gam, st[IQ + 2], st[IP + 2])) * C
                                             * np.exp(1j * st[IS]) * wg)
        ex = h * np.vdot(_cs(x, qb, pb, gb), psi)
        assert abs(hk - ex) < 1e-8, (gb, qb, pb, hk, ex)

def _J():
    return np.block([[np.zeros((3, 3)), np.eye(3)], [-np.eye(3), np.zeros((3, 3))]])


def _sympl_err(y):
    Mqq, Mqp, Mpq, Mpp = blocks(y)
    M = np.block([[Mqq, Mqp], [Mpq, Mpp]])
    return np.max(np.abs(M.T @ _J() @ M - _J()))


@pytest.mark.parametrize("pot,param,q0,p0", [
    (O.POT_SOFTCORE, [0.3], [0.6, 0.0, 1.2], [0.0, 0.55, 0.1]),
    (O.POT_TONGLIN, W.TONGLIN_AR, [2.0, 0.0, -6.0], [0.0, 0.1, 2.0]),
])
def test_symplecticity_energy_reversibility_scale_as_dt4(pot, param, q0, p0):
    P0 = O.make_pulse(E0=0.0, omega=0.057, cycles=2.0)
    T = zero_target(pot, param)
    tend = 6.0
    res = {}
    for h in (0.01, 0.005):
        N = int(round(tend / h))
        G = O.make_grid(0.0, h, N, 1)
        st, Cc, fl = O.propagate(P0, T, G, [0], q0, p0, N)
        y = st[:, 0]
        V0 = O.potential_radial(T, [np.linalg.norm(q0)])[0, 0]
        V1 = O.potential_radial(T, [np.linalg.norm(y[IQ:IQ + 3])])[0, 0]
        dE = abs(0.5 * y[IP:IP + 3] @ y[IP:IP + 3] + V1 - 0.5 * np.dot(p0, p0) - V0)
        # backwards with -h from the endpoint
        Gb = O.make_grid(tend, -h, N, 1)
        sb, _, _ = O.propagate(P0, T, Gb, [0], y[IQ:IQ + 3], y[IP:IP + 3], N)
        rev = np.max(np.abs(np.concatenate([sb[IQ:IQ + 3, 0] - q0, sb[IP:IP + 3, 0] - p0])))
        res[h] = (_sympl_err(y), dE, rev)
    for k in range(3):
        ratio = res[0.01][k] / res[0.005][k]
        assert 12 < ratio < 40, (k, res)      # fourth order (h^5 local terms can dominate)


def test_potential_derivatives_against_finite_differences():
    for pot, param in [(O.POT_SOFTCORE, [0.3]), (O.POT_TONGLIN, W.TONGLIN_AR), (O.POT_HARMONIC, [0.7])]:
        T = zero_target(pot, param)
        r = np.array([0.2, 0.7, 1.5, 3.0, 8.0])
        h = 1e-3
        f = [O.potential_radial(T, r + k * h) for k in (-2, -1, 0, 1, 2)]

        def d5(col):   # fifth-order-accurate central difference
            return (f[0][:, col] - 8 * f[1][:, col] + 8 * f[3][:, col] - f[4][:, col]) / (12 * h)
        assert np.allclose(f[2][:, 1], d5(0), rtol=1e-7, atol=1e-10)
        assert np.allclose(f[2][:, 2], d5(1), rtol=1e-7, atol=1e-10)
    # Tong-Lin: V -> -(1 + a1 + a5)/r at the origin side, -1/r far out
    T = zero_target(O.POT_TONGLIN, W.TONGLIN_AR)
    assert abs(O.potential_radial(T, [60.0])[0, 0] * 60.0 + 1.0) < 1e-9


def test_classical_return_energy_3p17_Up():
    # V = 0, flat CW field, electron born at rest at the origin at phase w t0:
    # the largest kinetic energy at the first return to z = 0 is 3.17 Up.
    E0, w = 0.05, 0.057
    Up = E0 ** 2 / (4 * w ** 2)
    P = O.make_pulse(E0=E0, omega=w, cw=True)
    T = zero_target()
    h = 0.01
    T0 = 2 * np.pi / w
    best = 0.0
    for ph in np.linspace(0.05, 0.8, 76):       # births after the crest return
        t0 = ph / w
        N = int(1.2 * T0 / h)
        G = O.make_grid(t0, h, N, 1)
        path = O.trajectory(P, T, G, 0, N, [0, 0, 0], [0, 0, 0])
        z = path[:, IQ + 2]
        k = np.nonzero((z[1:-1] * z[2:] <= 0))[0]
        if len(k) == 0:
            continue
        j = k[0] + 1
        f = z[j] / (z[j] - z[j + 1])
        pz = path[j, IP + 2] * (1 - f) + path[j + 1, IP + 2] * f
        best = max(best, 0.5 * pz * pz)

    # independent: the same physics by root finding on the closed-form orbit
    def ke_return(ph):
        t0 = ph / w
        zf = lambda t: (E0 / w ** 2) * (np.cos(w * t) - np.cos(w * t0)) + (E0 / w) * np.sin(w * t0) * (t - t0)
        tr = optimize.brentq(zf, t0 + 1e-3, t0 + 1.2 * T0 if zf(t0 + 1.2 * T0) < 0 else t0 + 0.99 * T0)
        v = -(E0 / w) * (np.sin(w * tr) - np.sin(w * t0))
        return 0.5 * v * v
    r = optimize.minimize_scalar(lambda ph: -ke_return(ph), bounds=(0.1, 0.6), method="bounded",
                                 options={"xatol": 1e-10})
    assert abs(-r.fun / Up - 3.1731) < 1e-3
    assert abs(best / Up - 3.1731) < 3e-3


def _cfg1():
    w = W.H_800_2CYC_GRID
    P = O.make_pulse(w.pulse.intensity_wcm2, w.pulse.lambda_nm, w.pulse.cycles, w.pulse.cep)
    t = w.target
    T = O.make_target(t.pot, t.pot_param, t.ip, t.gto_l, t.c, t.alpha)
    G = O.pulse_grid(P, w.dt, w.t_out, w.gamma, w.d_t)
    return w, P, T, G


def test_rotational_invariance_about_polarisation_axis():
    w, P, T, G = _cfg1()
    t0 = G.t_start + np.array([4000, 4800, 5600]) * G.dt
    k = np.array([0.05, 0.2, 0.12])
    out = []
    for th in (0.0, 0.7, 2.9):
        kx, ky = k * np.cos(th), k * np.sin(th)
        b = O.births_at(P, T, t0, kx, ky)
        births = {"n0": np.array([4000, 4800, 5600], np.int32), "px": kx, "py": ky, "pz": b["kz"],
                  "qz": b["qz"], "amp_re": b["amp_re"], "amp_im": b["amp_im"]}
        dl, dv, _ = O.dipole(P, T, G, births)
        out.append((dl, dv))
    for dl, dv in out[1:]:
        assert np.max(np.abs(dl - out[0][0])) < 1e-12 * np.max(np.abs(out[0][0]))
        assert np.max(np.abs(dv - out[0][1])) < 1e-12 * np.max(np.abs(out[0][1]))


def test_sharded_bins_sum_to_unsharded():
    w, P, T, G = _cfg1()
    b = O.sample_births(P, T, G, w.birth_mode, w.n, w.n_t, w.n_k, w.sigma, w.kmax, w.seed)
    full_l, full_v, st = O.dipole(P, T, G, b)
    acc_l = np.zeros_like(full_l)
    acc_v = np.zeros_like(full_v)
    for sl in (slice(0, 300), slice(300, 701), slice(701, None)):
        O.dipole(P, T, G, {k: v[sl] for k, v in b.items()}, acc_l, acc_v)
    assert np.max(np.abs(acc_l - full_l)) < 1e-13 * np.max(np.abs(full_l))
    assert np.max(np.abs(acc_v - full_v)) < 1e-13 * np.max(np.abs(full_v))
    assert st["traj_steps"] > 0


def test_causal_removal_freezes_at_first_exceeding_bin():
    # free particle, D_t = 10: |C|^2 = (1 + g^2 tau^2)^{3/2} exceeds 10 at
    # tau* = sqrt(10^{2/3} - 1)/g ; removal happens at the first output bin >= tau*
    gam, h, n_out = 0.5, 0.02, 5
    P = O.make_pulse(E0=0.0, omega=0.057, cycles=2.0)
    T = zero_target()
    G = O.make_grid(0.0, h, 1000, n_out, gamma=gam, d_t=10.0)
    q0, p0 = np.array([0.1, 0.0, 0.2]), np.array([0.2, -0.1, 0.4])
    st, Cc, fl = O.propagate(P, T, G, [0], q0, p0, 1000)
    assert fl[0] & O.FLAG_REMOVED
    tstar = np.sqrt(10 ** (2 / 3) - 1) / gam
    nb = int(np.ceil(tstar / (h * n_out))) * n_out        # first bin index past tau*
    assert np.allclose(st[IQ:IQ + 3, 0], q0 + p0 * nb * h, atol=1e-12)
    # the returned C is the last accepted one (one bin earlier)
    tau_prev = (nb - n_out) * h
    assert abs(Cc[0] - (1 - 1j * gam * tau_prev) ** 1.5) < 1e-12
