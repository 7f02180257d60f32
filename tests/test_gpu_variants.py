"""GPU parity of the birth variants and of the FP64 path on the bench's workload
shape, through the C ABI against the oracle; and the mixed path's planar
determinant against exact arithmetic.

  * modified saddle point (App. B.2, Eq. SFHKmodSPA) and ADK births (Sec.
    III.C): births element by element (integers bit-exact), FP64 dipole bins
    of the 32x32 grid workload;
  * FP64 dipole bins on a sample of the H 800 nm, 8-cycle, dt = 0.01 workload
    (uniform birth times, Gaussian transverse momenta), the shape the bench
    times, against the oracle on the same births;
  * det Z of the planar float pass (Eq. C_HK) from float entries, against the
    exact determinant of the same float values (rational arithmetic), on
    random entries with heavy cancellation and on Z formed from float
    trajectory endpoints.
"""
from fractions import Fraction

import numpy as np
import pytest
import torch

import oracle as O
from paper_2601_17164_gb300 import workloads as W
from tests.helpers import oracle_births, oracle_objects, rel_max

pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    from paper_2601_17164_gb300 import pipeline as PL
    from paper_2601_17164_gb300 import sfhk as S


def _np(t):
    return t.detach().cpu().numpy()


def _births_np(b):
    return {"n0": _np(b.n0), "t0": _np(b.t0), "px": _np(b.p0x), "py": _np(b.p0y), "pz": _np(b.p0z),
            "qz": _np(b.q0z), "amp_re": _np(b.amp_re), "amp_im": _np(b.amp_im)}


@pytest.mark.parametrize("wl,n", [(W.H_800_2CYC_GRID, None), (W.H_800_8CYC_1M, 3000), (W.AR_1600_6CYC_10M, 2000)])
def test_modified_spa_births_match_oracle(wl, n):
    w = wl if n is None else wl.with_n(n)
    field, target = PL.make_handles(w, amp_kind=1)
    g = _births_np(PL.sample(w, field, target))
    P, T, G = oracle_objects(w, amp_kind=1)
    o = O.sample_births(P, T, G, w.birth_mode, w.n, w.n_t, w.n_k, w.sigma, w.kmax, w.seed)
    assert np.array_equal(g["n0"], o["n0"])
    for k in ("px", "py", "pz", "qz"):
        assert rel_max(g[k], o[k], max(1.0, np.max(np.abs(o[k])))) < 1e-12, k
    a_g, a_o = g["amp_re"] + 1j * g["amp_im"], o["amp_re"] + 1j * o["amp_im"]
    assert np.array_equal(a_g == 0, a_o == 0)
    assert np.max(np.abs(a_g - a_o)) < 1e-11 * np.max(np.abs(a_o))
    # the two amplitude forms differ: the modified one carries no matrix element, so the
    # log-ratio of the moduli varies from birth to birth (amplitudes far from underflow)
    b0 = oracle_births(w)
    a0 = b0["amp_re"] + 1j * b0["amp_im"]
    big = (np.abs(a0) > 1e-250) & (np.abs(a_o) > 1e-250)
    assert big.sum() > 10
    assert np.std(np.log(np.abs(a_o[big])) - np.log(np.abs(a0[big]))) > 1e-3


def test_modified_spa_fp64_bins_match_oracle():
    w = W.H_800_2CYC_GRID
    field, target = PL.make_handles(w, amp_kind=1)
    b = PL.sample(w, field, target)
    nb = field.info["n_bins"]
    dl = torch.zeros(nb, dtype=torch.float64, device="cuda")
    dv = torch.zeros_like(dl)
    st = S.new_stats()
    S.sfhk_dipole(field, target, b, len(b), S.prop_params(S.FP64, w.gamma, w.d_t), dl, dv, st)
    P, T, G = oracle_objects(w, amp_kind=1)
    ob = O.sample_births(P, T, G, w.birth_mode, w.n, w.n_t, w.n_k, w.sigma, w.kmax, w.seed)
    ol, ov, ost = O.dipole(P, T, G, ob)
    e_l, e_v = rel_max(_np(dl), ol), rel_max(_np(dv), ov)
    print(f"modified SPA, FP64 bins vs oracle: len {e_l:.3e} vel {e_v:.3e}")
    assert e_l < 1e-10 and e_v < 1e-10
    gs = S.stats_dict(st)
    assert gs["traj_steps"] == ost["traj_steps"] and gs["removed"] == ost["removed"]


@pytest.mark.parametrize("wl,n", [(W.H_800_2CYC_GRID, None), (W.H_1600_3CYC_2M, 3000), (W.AR_1600_6CYC_10M, 2000)])
def test_adk_births_match_oracle(wl, n):
    # Sec. III.C: ADK modulus renormalised at the two sub-peaks, quasi-static exit, the
    # saddle's real action as the phase (the renormalisation is evaluated on both sides)
    w = wl if n is None else wl.with_n(n)
    field, target = PL.make_handles(w, amp_kind=2)
    g = _births_np(PL.sample(w, field, target))
    P, T, G = oracle_objects(w, amp_kind=2)
    o = O.sample_births(P, T, G, w.birth_mode, w.n, w.n_t, w.n_k, w.sigma, w.kmax, w.seed)
    assert np.array_equal(g["n0"], o["n0"])
    assert np.all(g["pz"] == 0.0) and np.all(o["pz"] == 0.0)
    for k in ("px", "py", "qz"):
        assert rel_max(g[k], o[k], max(1.0, np.max(np.abs(o[k])))) < 1e-12, k
    a_g, a_o = g["amp_re"] + 1j * g["amp_im"], o["amp_re"] + 1j * o["amp_im"]
    assert np.array_equal(a_g == 0, a_o == 0)
    assert np.max(np.abs(a_g - a_o)) < 1e-11 * np.max(np.abs(a_o))
    assert np.count_nonzero(a_o) > len(a_o) // 2


def test_adk_fp64_bins_match_oracle():
    w = W.H_800_2CYC_GRID
    field, target = PL.make_handles(w, amp_kind=2)
    b = PL.sample(w, field, target)
    nb = field.info["n_bins"]
    dl = torch.zeros(nb, dtype=torch.float64, device="cuda")
    dv = torch.zeros_like(dl)
    st = S.new_stats()
    S.sfhk_dipole(field, target, b, len(b), S.prop_params(S.FP64, w.gamma, w.d_t), dl, dv, st)
    P, T, G = oracle_objects(w, amp_kind=2)
    ob = O.sample_births(P, T, G, w.birth_mode, w.n, w.n_t, w.n_k, w.sigma, w.kmax, w.seed)
    ol, ov, ost = O.dipole(P, T, G, ob)
    e_l, e_v = rel_max(_np(dl), ol), rel_max(_np(dv), ov)
    print(f"ADK births, FP64 bins vs oracle: len {e_l:.3e} vel {e_v:.3e}")
    assert e_l < 1e-10 and e_v < 1e-10
    gs = S.stats_dict(st)
    assert gs["traj_steps"] == ost["traj_steps"] and gs["removed"] == ost["removed"]


def test_fp64_bins_match_oracle_on_the_8_cycle_workload():
    # 2048 births of the bench's workload (H 800 nm, 8 cycles, 1.5e14 W/cm^2, dt 0.01,
    # uniform birth times over the pulse, Gaussian k_perp); both sides FP64 (the GPU
    # contracts products into FMAs, the oracle does not), compared bin by bin relative
    # to max |D|.  Trajectories that scatter chaotically off the core amplify the
    # differing roundings, so the bound is looser than on the 2-cycle grid workload.
    w = W.H_800_8CYC_1M.with_n(2048)
    field, target = PL.make_handles(w)
    b = PL.sample(w, field, target)
    nb = field.info["n_bins"]
    dl = torch.zeros(nb, dtype=torch.float64, device="cuda")
    dv = torch.zeros_like(dl)
    st = S.new_stats()
    S.sfhk_dipole(field, target, b, len(b), S.prop_params(S.FP64, w.gamma, w.d_t), dl, dv, st)
    P, T, G = oracle_objects(w)
    ol, ov, ost = O.dipole(P, T, G, oracle_births(w))
    e_l, e_v = rel_max(_np(dl), ol), rel_max(_np(dv), ov)
    print(f"8-cycle workload, 2048 births, FP64 bins vs oracle: len {e_l:.3e} vel {e_v:.3e}")
    assert e_l < 1e-8 and e_v < 1e-8
    gs = S.stats_dict(st)
    assert gs["traj_steps"] == ost["traj_steps"] and gs["removed"] == ost["removed"]


def _exact_det(z):
    """det Z of one column of z [10] (float32 values) in rational arithmetic, as a complex
    double, and the condition number of the in-plane determinant: the sum of the moduli
    of the eight real products over the modulus of their signed sum."""
    f = [Fraction(float(v)) for v in z]
    r00, r01, r10, r11, i00, i01, i10, i11, yr, yi = f
    pr = [r00 * r11, -(i00 * i11), -(r01 * r10), i01 * i10]
    pi = [r00 * i11, i00 * r11, -(r01 * i10), -(i01 * r10)]
    ar, ai = sum(pr), sum(pi)
    a = complex(float(ar), float(ai))
    cond = float(sum(abs(x) for x in pr + pi)) / abs(a)
    return complex(float(ar * yr - ai * yi), float(ar * yi + ai * yr)), cond


def _check_det(z32):
    """Relative error of the device's det Z and its bound: the float rounding of the
    result (a few 2^-24) plus the in-plane determinant's error as if evaluated in twice
    the float precision (condition number times a few 2^-48)."""
    re, im, e = S.sfhk_det_z_planar_f32(torch.tensor(z32, device="cuda"))
    torch.cuda.synchronize()
    got = (_np(re) + 1j * _np(im)) * np.exp2(2.0 * _np(e))
    ex = [_exact_det(z32[:, i]) for i in range(z32.shape[1])]
    want = np.array([x[0] for x in ex])
    cond = np.array([x[1] for x in ex])
    err = np.abs(got - want) / np.abs(want)
    bound = 4 * 2.0 ** -24 + 16 * 2.0 ** -48 * cond
    return err, cond, bound


def test_planar_det_z_is_as_accurate_as_twice_float():
    rng = np.random.default_rng(11)
    n = 4000
    z = rng.standard_normal((10, n)) * np.exp2(rng.integers(-20, 20, (1, n)))
    # heavy cancellation: the in-plane block close to rank one, entries up to 2^26 times
    # larger than the perturbation that sets the determinant
    m = n // 2
    u = rng.standard_normal((2, m)) + 1j * rng.standard_normal((2, m))
    v = rng.standard_normal((2, m)) + 1j * rng.standard_normal((2, m))
    big = np.exp2(rng.integers(4, 27, m))
    blk = big * np.stack([u[0] * v[0], u[0] * v[1], u[1] * v[0], u[1] * v[1]])
    blk += rng.standard_normal((4, m)) + 1j * rng.standard_normal((4, m))
    z[0:4, :m], z[4:8, :m] = blk.real, blk.imag
    z32 = z.astype(np.float32)
    err, cond, bound = _check_det(z32)
    print(f"planar det Z vs exact: max rel err {err.max():.3e}, max err/bound {np.max(err / bound):.3f}, "
          f"max condition {cond.max():.3e}")
    assert np.all(err <= bound)
    # a plain float evaluation would lose cond * 2^-24: the cancelling cases show the gain
    hard = cond > 2.0 ** 20
    assert hard.sum() > 100 and np.all(err[hard] < 1e-3 * cond[hard] * 2.0 ** -24)


def test_planar_det_z_on_float_trajectory_states():
    # Z formed in float from the monodromy blocks of float (MIXED) trajectories of the
    # 8-cycle workload, births in the x-z plane, as the float pass forms Z's entries
    w = W.H_800_8CYC_1M.with_n(512)
    field, target = PL.make_handles(w)
    b = PL.sample(w, field, target)
    b.p0y.zero_()                                   # motion in the x-z plane
    nst = field.info["n_steps"]
    st, _, fl = S.sfhk_propagate(field, target, b, len(b), S.prop_params(S.MIXED, w.gamma, w.d_t), int(0.8 * nst))
    st = _np(st)
    ok = ((_np(fl) & 3) == 0) & (_np(b.n0) < int(0.8 * nst) - 1000)
    g, q = np.float32(w.gamma), np.float32(0.25 / w.gamma)
    blk = lambda base, i, j: st[base + 3 * i + j].astype(np.float32)   # row i, column j (x=0, z=2)
    Mqq, Mqp, Mpq, Mpp = 6, 15, 24, 33
    z = np.zeros((10, st.shape[1]), np.float32)
    for k, (i, j) in enumerate(((0, 0), (0, 2), (2, 0), (2, 2))):
        z[k] = np.float32(0.5) * (blk(Mpp, i, j) + blk(Mqq, i, j))
        z[4 + k] = (-g * blk(Mqp, i, j).astype(np.float64) + (q * blk(Mpq, i, j)).astype(np.float64)).astype(np.float32)
    z[8] = np.float32(0.5) * (blk(Mpp, 1, 1) + blk(Mqq, 1, 1))
    z[9] = (-g * blk(Mqp, 1, 1).astype(np.float64) + (q * blk(Mpq, 1, 1)).astype(np.float64)).astype(np.float32)
    z = np.ascontiguousarray(z[:, ok])
    err, cond, bound = _check_det(z)
    print(f"planar det Z on {z.shape[1]} float states: max rel err {err.max():.3e}, max condition {cond.max():.3e}")
    assert z.shape[1] > 300 and np.all(err <= bound)
