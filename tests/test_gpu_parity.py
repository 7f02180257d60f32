"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Births are compared element by element (integers bit-exact); FP64 endpoints to
1e-10 relative on regular trajectories; dipole bins relative to max |D|; the
spectrum DFT to 1e-12; the mixed path by plateau harmonic yield (1e-3
relative) and phase (0.01 rad) against the oracle on the same births.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2601_17164_gb300 import workloads as W
from tests.helpers import band_yield, harmonic_phase, oracle_births, oracle_objects, plateau_harmonics, rel_max

pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    from paper_2601_17164_gb300 import pipeline as PL
    from paper_2601_17164_gb300 import sfhk as S


def _np(t):
    return t.detach().cpu().numpy()


def _births_np(b):
    return {"n0": _np(b.n0), "t0": _np(b.t0), "px": _np(b.p0x), "py": _np(b.p0y), "pz": _np(b.p0z),
            "qz": _np(b.q0z), "amp_re": _np(b.amp_re), "amp_im": _np(b.amp_im)}


def _compare_births(g, o, t_scale=None):
    assert np.array_equal(g["n0"], o["n0"])
    # t0 = t_start + n0 dt: rounding of the sum, relative to its operands' size
    t_scale = np.max(np.abs(o["t0"])) if t_scale is None else t_scale
    assert np.max(np.abs(g["t0"] - o["t0"])) <= 1e-15 * t_scale
    for k in ("px", "py", "pz", "qz"):
        assert rel_max(g[k], o[k], max(1.0, np.max(np.abs(o[k])))) < 1e-12, k
    a_g = g["amp_re"] + 1j * g["amp_im"]
    a_o = o["amp_re"] + 1j * o["amp_im"]
    assert np.array_equal(a_g == 0, a_o == 0)
    assert np.max(np.abs(a_g - a_o)) < 1e-11 * np.max(np.abs(a_o))


@pytest.mark.parametrize("wl,n", [(W.H_800_2CYC_GRID, None), (W.H_800_8CYC_1M, 3000),
                                  (W.AR_1600_6CYC_10M, 2000)])
def test_births_match_oracle(wl, n):
    w = wl if n is None else wl.with_n(n)
    field, target = PL.make_handles(w)
    b = PL.sample(w, field, target)
    torch.cuda.synchronize()
    _compare_births(_births_np(b), oracle_births(w))


def test_births_full_size_sampled():
    # 1e6 births at the bench size, checked at sampled indices (incl. first/last)
    w = W.H_800_8CYC_1M
    field, target = PL.make_handles(w)
    b = PL.sample(w, field, target)
    g = _births_np(b)
    rng = np.random.default_rng(0)
    idx = np.unique(np.concatenate([[0, 1, w.n - 1], rng.integers(0, w.n, 400)]))
    P, T, G = oracle_objects(w)
    o = O.sample_births_at(P, T, G, w.birth_mode, w.n, idx, w.n_t, w.n_k, w.sigma, w.kmax, w.seed)
    _compare_births({k: v[idx] for k, v in g.items()}, o)
    assert np.all(np.diff(g["n0"]) >= 0)


def test_births_streamed_chunk_of_the_1e8_sample():
    # the streamed mid-IR workload (Ar 2000 nm, 20 cycles, 1e8 births in chunks of 2^22):
    # one chunk from the middle of the sample, element by element against the oracle's
    # births at the same indices of the 1e8-birth sample
    w = W.AR_2000_20CYC_100M
    field, target = PL.make_handles(w)
    first, count = 50_000_000 - 2048, 4096
    b = S.Births.empty(count)
    S.sfhk_sample_births(field, target, w.birth_mode, w.n, b, w.n_t, w.n_k, w.sigma, w.kmax, w.seed,
                         first=first, count=count)
    torch.cuda.synchronize()
    g = _births_np(b)
    P, T, G = oracle_objects(w)
    o = O.sample_births_at(P, T, G, w.birth_mode, w.n, np.arange(first, first + count), w.n_t, w.n_k, w.sigma,
                           w.kmax, w.seed)
    _compare_births(g, o, t_scale=abs(G.t_start))   # births near t = 0: t0 is a difference of ~2758
    assert np.any(g["amp_re"] != 0)


def test_mixed_streamed_chunk_against_fp64_path():
    # the same workload: the mixed path (default escalation) on 1024 consecutive births of
    # the 1e8 sample against the FP64 path on the same births, plateau yields and phases.
    # (Over 20 cycles, Ar's chaotic returns make two FP64 evaluations that round
    # differently disagree at the 1e-3 level on so few births; the FP64 path's own
    # parity with the oracle is pinned on the other workloads.)
    w = W.AR_2000_20CYC_100M
    field, target = PL.make_handles(w)
    first, count = 50_000_000 - 512, 1024
    b = S.Births.empty(count)
    S.sfhk_sample_births(field, target, w.birth_mode, w.n, b, w.n_t, w.n_k, w.sigma, w.kmax, w.seed,
                         first=first, count=count)
    nb = field.info["n_bins"]
    om = torch.tensor(W.omega_grid(w), dtype=torch.float64, device="cuda")
    X = {}
    for name, pp in (("fp64", S.prop_params(S.FP64, w.gamma, w.d_t)), ("mixed", S.prop_params(S.MIXED, w.gamma, w.d_t))):
        dl = torch.zeros(nb, dtype=torch.float64, device="cuda")
        dv = torch.zeros_like(dl)
        S.sfhk_dipole(field, target, b, count, pp, dl, dv)
        X[name] = [re.cpu().numpy() + 1j * im.cpu().numpy() for re, im in (PL.spectrum_of(d, field, om) for d in (dl, dv))]
    omn = om.cpu().numpy()
    w0 = 45.5633525 / w.pulse.lambda_nm
    hs = plateau_harmonics(w)
    for k, power in ((0, 4), (1, 2)):
        yo, yg = band_yield(omn, X["fp64"][k], w0, power, hs), band_yield(omn, X["mixed"][k], w0, power, hs)
        po, pg = harmonic_phase(omn, X["fp64"][k], w0, hs), harmonic_phase(omn, X["mixed"][k], w0, hs)
        strong = yo > 1e-3 * yo.max()
        ey = np.max(np.abs(yg / yo - 1)[strong])
        ep = np.max(np.abs(np.angle(np.exp(1j * (pg - po))))[strong])
        print(f"Ar 2000 nm chunk, mixed vs FP64 ({'len' if k == 0 else 'vel'}): yield {ey:.3e} phase {ep:.3e}")
        assert ey < 1e-3 and ep < 0.01, (k, ey, ep)


def _regular(state, thresh=1e3):
    return np.max(np.abs(state[6:42]), axis=0) < thresh


@pytest.mark.parametrize("frac", [0.5, 1.0])
def test_fp64_endpoints_match_oracle(frac):
    w = W.H_800_2CYC_GRID
    field, target = PL.make_handles(w)
    b = PL.sample(w, field, target)
    P, T, G = oracle_objects(w)
    n_end = int(frac * G.n_steps)
    bn = _births_np(b)
    keep = bn["n0"] <= n_end
    idx = np.nonzero(keep)[0]
    sub = b.slice(0, len(b))
    pp = S.prop_params(S.FP64, w.gamma, w.d_t)
    st, C, fl = S.sfhk_propagate(field, target, sub, int(idx.max()) + 1, pp, n_end)
    st, C, fl = _np(st)[:, idx], _np(C)[idx], _np(fl)[idx]
    q0 = np.zeros((3, len(idx)))
    q0[2] = bn["qz"][idx]
    p0 = np.stack([bn["px"][idx], bn["py"][idx], bn["pz"][idx]])
    so, Co, fo = O.propagate(P, T, G, bn["n0"][idx], q0, p0, n_end)
    reg = _regular(so) & ((fo & 1) == 0)
    assert reg.sum() > 0.8 * len(idx)
    scale = np.maximum(1.0, np.abs(so[:, reg]))
    err = np.max(np.abs(st[:, reg] - so[:, reg]) / scale)
    assert err < 1e-10, err
    assert np.max(np.abs(C[reg] - Co[reg]) / np.maximum(1, np.abs(Co[reg]))) < 1e-10
    assert np.array_equal(fl[reg] & 1, fo[reg] & 1)


@pytest.mark.parametrize("pot,param", [(O.POT_ZERO, ()), (O.POT_HARMONIC, (0.8,)), (O.POT_SOFTCORE, (0.3,)),
                                       (O.POT_TONGLIN, tuple(W.TONGLIN_AR))])
@pytest.mark.parametrize("precision", [0, 1])
def test_endpoints_closed_form_potentials(pot, param, precision):
    # general 3D initial conditions (q0x, q0y set), ragged count (not a block multiple)
    w = W.H_800_2CYC_GRID
    p = w.pulse
    field = S.Field(p.intensity_wcm2, p.lambda_nm, p.cycles, p.cep, w.dt, w.t_out)
    target = S.Target(pot, param, 0.5, 0, W.H_C, W.H_ALPHA)
    P = O.make_pulse(p.intensity_wcm2, p.lambda_nm, p.cycles, p.cep)
    T = O.make_target(pot, param, 0.5, 0, W.H_C, W.H_ALPHA)
    G = O.pulse_grid(P, w.dt, w.t_out, 0.5, 1e30)
    rng = np.random.default_rng(3)
    n = 301
    n0 = np.sort(rng.integers(1, G.n_steps // 2, n)).astype(np.int32)
    q0 = rng.uniform(4, 8, (3, n)) * rng.choice([-1, 1], (3, n))
    p0 = rng.uniform(-0.5, 0.5, (3, n))
    dev = "cuda"
    tt = lambda a: torch.tensor(a, device=dev)
    b = S.Births(tt(n0), tt(G.t_start + n0 * G.dt), tt(p0[0]), tt(p0[1]), tt(p0[2]), tt(q0[2]),
                 torch.ones(n, dtype=torch.float64, device=dev), torch.zeros(n, dtype=torch.float64, device=dev),
                 tt(q0[0]), tt(q0[1]))
    n_end = int(0.7 * G.n_steps)
    st, C, fl = S.sfhk_propagate(field, target, b, n, S.prop_params(precision, 0.5, 1e30), n_end)
    st, C, fl = _np(st), _np(C), _np(fl)
    so, Co, fo = O.propagate(P, T, G, n0, q0, p0, n_end)
    # Rounding differences are amplified by the monodromy matrix M: the claim is
    # made on well-conditioned trajectories (max|M| <= 10 (1 + t - t0), i.e. at
    # most ten times free-particle drift), and the worst error of the others is
    # reported.
    # growth of M beyond free drift (M_qp = tau for a free particle)
    tau = (n_end - n0) * G.dt
    kappa = np.max(np.abs(so[6:42]), axis=0) / (1.0 + tau)
    ok = ((fo & 1) == 0) & ((fl & 1) == 0)
    well = ok & (kappa <= 10.0)
    assert well.sum() > 0.5 * n
    # Tong-Lin's -18/r core makes close passes locally very sensitive even when
    # the final monodromy matrix is moderate; the mixed path hands such
    # trajectories to its escalation pass, so only the median is held there.
    tol = {0: {O.POT_ZERO: 1e-12, O.POT_HARMONIC: 1e-11, O.POT_SOFTCORE: 1e-10, O.POT_TONGLIN: 1e-8},
           1: {O.POT_ZERO: 1e-5, O.POT_HARMONIC: 3e-4, O.POT_SOFTCORE: 3e-4, O.POT_TONGLIN: None}}[precision][pot]
    scale = np.maximum(1.0, np.abs(so))
    err = np.max(np.abs(st - so) / scale, axis=0)
    cerr = np.abs(C - Co) / np.maximum(1, np.abs(Co))
    rest = ok & ~well
    print(f"pot {pot} prec {precision}: {well.sum()}/{n} with max|M| <= 10 (1 + tau): state err {err[well].max():.2e}, "
          f"C err {cerr[well].max():.2e}; others ({rest.sum()}): {err[rest].max() if rest.any() else 0:.2e}")
    if tol is None:
        assert np.median(err[well]) < 1e-4 and np.median(cerr[well]) < 1e-4
    else:
        assert err[well].max() < tol
        assert cerr[well].max() < tol


def test_fp64_dipole_bins_match_oracle():
    w = W.H_800_2CYC_GRID
    r = PL.run(w, precision=S.FP64)
    P, T, G = oracle_objects(w)
    ob = oracle_births(w)
    dl, dv, st = O.dipole(P, T, G, ob)
    gl, gv = _np(r.d_len), _np(r.d_vel)
    e_l = rel_max(gl, dl)
    e_v = rel_max(gv, dv)
    print(f"fp64 bins rel err: len {e_l:.3e} vel {e_v:.3e}")
    assert e_l < 1e-10 and e_v < 1e-10
    gs = S.stats_dict(r.stats)
    assert gs["traj_steps"] == st["traj_steps"]
    assert gs["removed"] == st["removed"]


@pytest.mark.parametrize("wl,n", [(W.H_800_2CYC_GRID, None), (W.AR_1600_6CYC_10M, 512)])
def test_planar_form_equals_full_3d_state(wl, n):
    # the planar (25-real) form is the same computation as the 43-real one
    w = wl if n is None else wl.with_n(n)
    field, target = PL.make_handles(w)
    b = PL.sample(w, field, target)
    nb = field.info["n_bins"]
    out = []
    for geo in (0, 1):
        dl = torch.zeros(nb, dtype=torch.float64, device="cuda")
        dv = torch.zeros_like(dl)
        S.sfhk_dipole(field, target, b, len(b), S.prop_params(S.FP64, w.gamma, w.d_t, geometry=geo), dl, dv)
        out.append((_np(dl), _np(dv)))
    e = max(rel_max(out[0][0], out[1][0]), rel_max(out[0][1], out[1][1]))
    print(f"planar vs 3D ({w.name}): {e:.2e}")
    # identical arithmetic up to rounding order; the argon sample contains
    # trajectories through the -18/r core, which amplify rounding differences
    assert e < (1e-12 if n is None else 1e-3)


def test_double_float_dipole_matches_oracle():
    # precision 2: the planar state in double-float arithmetic on the FP32 pipe;
    # the recombination terms are evaluated in float (relative 1e-7)
    w = W.H_800_2CYC_GRID
    r = PL.run(w, precision=S.DF)
    P, T, G = oracle_objects(w)
    dl, dv, st = O.dipole(P, T, G, oracle_births(w))
    e_l, e_v = rel_max(_np(r.d_len), dl), rel_max(_np(r.d_vel), dv)
    print(f"double-float bins rel err: len {e_l:.3e} vel {e_v:.3e}")
    assert e_l < 2e-6 and e_v < 2e-6


def test_deterministic_reduction_is_bitwise_reproducible():
    w = W.H_800_2CYC_GRID
    a = PL.run(w, precision=S.FP64, deterministic=1)
    b = PL.run(w, precision=S.FP64, deterministic=1)
    c = PL.run(w, precision=S.FP64, deterministic=0)
    assert torch.equal(a.d_len, b.d_len) and torch.equal(a.d_vel, b.d_vel)
    assert rel_max(_np(a.d_len), _np(c.d_len)) < 1e-13


@pytest.mark.parametrize("wl,n,chunk", [(W.H_800_8CYC_1M, 20000, 0), (W.AR_1600_6CYC_10M, 6000, 700)])
def test_escalation_schedules_agree(wl, n, chunk):
    # the mixed path with escalation overlaps the redo with the float pass by birth
    # chunks (esc_overlap 0) or by time segments with the float state saved in device
    # memory between launches (esc_overlap 1), or runs them in sequence (2); the
    # deterministic mode runs one float launch and one redo with one thread per
    # trajectory, the others the redo that splits each step over four warps (or, with
    # esc_precision 2, the one-thread redo).  Same arithmetic per trajectory: bins
    # agree to summation order, the counters exactly.
    w = wl.with_n(n)
    f, t = PL.make_handles(w)
    b = PL.sample(w, f, t)
    nb = f.info["n_bins"]
    out = []
    for det, ov, ep in ((1, 0, 0), (0, 0, 0), (0, 1, 0), (0, 2, 0), (0, 2, 2)):
        dl = torch.zeros(nb, dtype=torch.float64, device="cuda")
        dv = torch.zeros_like(dl)
        st = S.new_stats()
        S.sfhk_dipole(f, t, b, len(b), S.prop_params(S.MIXED, w.gamma, w.d_t, deterministic=det, chunk_steps=chunk,
                                                     esc_ratio=30.0, esc_overlap=ov, esc_precision=ep), dl, dv, st)
        out.append((_np(dl), _np(dv), S.stats_dict(st)))
    (l1, v1, s1) = out[0]
    assert s1["escalated"] > 0
    for l0, v0, s0 in out[1:]:
        assert s0 == s1, (s0, s1)
        assert rel_max(l0, l1) < 1e-12 and rel_max(v0, v1) < 1e-12


def test_two_tier_escalation_reduces_to_one_ratio():
    # esc_big = 0: the single-ratio rule; esc_big tiny: every contribution takes the second
    # ratio, i.e. the single-ratio rule at that ratio (counters equal, bins to 1e-12)
    w = W.H_800_8CYC_1M.with_n(8192)
    f, t = PL.make_handles(w)
    b = PL.sample(w, f, t)
    nb = f.info["n_bins"]

    def run(**kw):
        dl = torch.zeros(nb, dtype=torch.float64, device="cuda")
        dv = torch.zeros_like(dl)
        st = S.new_stats()
        S.sfhk_dipole(f, t, b, len(b), S.prop_params(S.MIXED, w.gamma, w.d_t, **kw), dl, dv, st)
        return _np(dl), _np(dv), S.stats_dict(st)

    for single, two in (({"esc_ratio": 100.0, "esc_big": 0.0}, {"esc_ratio": 100.0, "esc_ratio_big": 40.0, "esc_big": 0.0}),
                        ({"esc_ratio": 40.0, "esc_big": 0.0}, {"esc_ratio": 100.0, "esc_ratio_big": 40.0, "esc_big": 1e-30})):
        l1, v1, s1 = run(**single)
        l2, v2, s2 = run(**two)
        assert s1 == s2, (single, two, s1, s2)
        assert rel_max(l1, l2) < 1e-12 and rel_max(v1, v2) < 1e-12
    # between the two: at least the escalations of the larger ratio, at most those of the smaller
    n_hi = run(esc_ratio=100.0, esc_big=0.0)[2]["escalated"]
    n_lo = run(esc_ratio=40.0, esc_big=0.0)[2]["escalated"]
    n_mid = run(esc_ratio=100.0, esc_ratio_big=40.0, esc_big=1.0)[2]["escalated"]
    assert n_hi <= n_mid <= n_lo and n_hi < n_lo


def test_pipelined_redo_with_partial_waves_and_removal():
    # the four-warp redo against the one-thread FP64 redo on lists that exercise the
    # partial-wave labels (p and d waves kept) and removal (small d_t), H and Ar; bins
    # every 10 steps (one GTO term per step in the bins warp), every 5 (two terms) and
    # every step (all terms at once)
    from dataclasses import replace
    h_every_step = replace(W.H_800_8CYC_1M, t_out=0.01, name="H 800nm 8cyc, bins every step")
    h_five = replace(W.H_800_8CYC_1M, dt=0.02, name="H 800nm 8cyc dt 0.02, bins every 5 steps")
    for wl, n, d_t, mask in ((W.H_800_8CYC_1M, 8000, 1e4, 2), (W.AR_1600_6CYC_10M, 3000, 1e5, 6),
                             (h_every_step, 3000, 1e4, 0), (h_five, 5000, 1e5, 0)):
        w = wl.with_n(n)
        f, t = PL.make_handles(w)
        b = PL.sample(w, f, t)
        nb = f.info["n_bins"]
        res = []
        for ep in (0, 2):
            dl = torch.zeros(nb, dtype=torch.float64, device="cuda")
            dv = torch.zeros_like(dl)
            st = S.new_stats()
            pp = S.prop_params(S.MIXED, w.gamma, d_t, esc_ratio=10.0, esc_overlap=2, esc_precision=ep,
                               pw_mask=mask, pw_radius=3.0)
            S.sfhk_dipole(f, t, b, len(b), pp, dl, dv, st)
            res.append((_np(dl), _np(dv), S.stats_dict(st)))
        (l0, v0, s0), (l2, v2, s2) = res
        assert s0 == s2, (s0, s2)
        assert s0["escalated"] > 0 and s0["removed"] > 0
        print(f"{wl.name}: escalated {s0['escalated']} removed {s0['removed']}")
        assert rel_max(l0, l2) < 1e-12 and rel_max(v0, v2) < 1e-12


def test_redo_plan_with_more_groups_than_blocks():
    # a list longer than the persistent grid holds at once (4 blocks per SM): the
    # longest-first plan gives every SM's list several groups and the blocks steal
    # from other lists at the end; against the one-thread FP64 redo (esc_precision 2):
    # equal counters, bins to summation order.  Also an empty list and a single group.
    w = W.H_800_8CYC_1M.with_n(120000)
    f, t = PL.make_handles(w)
    b = PL.sample(w, f, t)
    nb = f.info["n_bins"]

    def run(ep, births, ratio):
        dl = torch.zeros(nb, dtype=torch.float64, device="cuda")
        dv = torch.zeros_like(dl)
        st = S.new_stats()
        pp = S.prop_params(S.MIXED, w.gamma, w.d_t, esc_ratio=ratio, esc_floor=0.0, esc_big=0.0, esc_precision=ep)
        S.sfhk_dipole(f, t, births, len(births), pp, dl, dv, st)
        return _np(dl), _np(dv), S.stats_dict(st)

    sm = torch.cuda.get_device_properties(0).multi_processor_count
    # a window of 32 consecutive births of which some escalate: a single, partly filled group
    one = next(b.slice(k, k + 32) for k in range(0, len(b) - 32, 3000)
               if 0 < run(2, b.slice(k, k + 32), 2.0)[2]["escalated"] <= 32)
    for births, ratio in ((b, 2.0), (one, 2.0), (b.slice(0, 4000), 1e12)):
        l0, v0, s0 = run(0, births, ratio)
        l2, v2, s2 = run(2, births, ratio)
        assert s0 == s2, (s0, s2)
        if births is b:
            assert (s0["escalated"] + 31) // 32 > 4 * sm, s0   # more groups than resident blocks
        assert (s0["escalated"] == 0) == (ratio == 1e12), s0
        assert rel_max(l0, l2) < 1e-12 and rel_max(v0, v2) < 1e-12


@pytest.mark.parametrize("block,chunk", [(64, 200), (64, 1000), (128, 4000)])
def test_launch_shapes_agree(block, chunk):
    w = W.H_800_2CYC_GRID
    ref = PL.run(w, precision=S.FP64, deterministic=1)
    r = PL.run(w, precision=S.FP64, block=block, chunk_steps=chunk)
    assert rel_max(_np(r.d_len), _np(ref.d_len)) < 1e-13
    assert rel_max(_np(r.d_vel), _np(ref.d_vel)) < 1e-13


def test_spectrum_matches_oracle_dft():
    w = W.H_800_2CYC_GRID
    P, T, G = oracle_objects(w)
    rng = np.random.default_rng(5)
    nb = G.n_steps // G.n_out + 1
    x = rng.standard_normal(nb)
    om = np.array(W.omega_grid(w))
    ref = O.spectrum(x, G.t_start, G.dt * G.n_out, P.Tp / 2, om)
    field, _ = PL.make_handles(w)
    re, im = PL.spectrum_of(torch.tensor(x, device="cuda"), field, torch.tensor(om, device="cuda"))
    got = _np(re) + 1j * _np(im)
    assert np.max(np.abs(got - ref)) < 1e-12 * np.max(np.abs(ref))


def _mixed_vs_oracle(w, n):
    w = w.with_n(n)
    r = PL.run(w, precision=S.MIXED)
    P, T, G = oracle_objects(w)
    dl, dv, st = O.dipole(P, T, G, oracle_births(w))
    om = _np(r.omega)
    w0 = P.omega
    hs = plateau_harmonics(w)
    out = {}
    for name, bins, power in (("len", dl, 4), ("vel", dv, 2)):
        X_o = O.spectrum(bins, G.t_start, G.dt * G.n_out, P.Tp / 2, om)
        X_g = (_np(r.D_re) + 1j * _np(r.D_im)) if name == "len" else (_np(r.V_re) + 1j * _np(r.V_im))
        yo, yg = band_yield(om, X_o, w0, power, hs), band_yield(om, X_g, w0, power, hs)
        po, pg = harmonic_phase(om, X_o, w0, hs), harmonic_phase(om, X_g, w0, hs)
        strong = yo > 1e-3 * yo.max()
        dphi = np.abs(np.angle(np.exp(1j * (pg - po))))[strong]
        out[name] = (np.max(np.abs(yg / yo - 1)[strong]), np.max(dphi))
    return out


@pytest.mark.parametrize("wl,n", [(W.H_800_8CYC_1M, 4096), (W.AR_1600_6CYC_10M, 2048)])
def test_mixed_path_yield_and_phase(wl, n):
    res = _mixed_vs_oracle(wl, n)
    print("mixed vs oracle (max rel yield err, max phase err):", res)
    for name, (ey, ep) in res.items():
        assert ey < 1e-3, (name, ey)
        assert ep < 0.01, (name, ep)


def test_mixed_full_size_against_fp64_path():
    # the bench workload at full size (1e6 births, H 800 nm 8 cycles): the mixed path with
    # its default escalation against the FP64 GPU path on the same births (the FP64 path is
    # pinned to the oracle above); plateau yields and phases within the stated tolerances
    w = W.H_800_8CYC_1M
    f, t = PL.make_handles(w)
    b = PL.sample(w, f, t)
    nb = f.info["n_bins"]
    om = torch.tensor(W.omega_grid(w), dtype=torch.float64, device="cuda")
    X = {}
    for name, pp in (("fp64", S.prop_params(S.FP64, w.gamma, w.d_t)), ("mixed", S.prop_params(S.MIXED, w.gamma, w.d_t))):
        dl = torch.zeros(nb, dtype=torch.float64, device="cuda")
        dv = torch.zeros_like(dl)
        S.sfhk_dipole(f, t, b, len(b), pp, dl, dv)
        X[name] = [re.cpu().numpy() + 1j * im.cpu().numpy() for re, im in (PL.spectrum_of(d, f, om) for d in (dl, dv))]
    w0 = 45.5633525 / w.pulse.lambda_nm
    omn = om.cpu().numpy()
    hs = plateau_harmonics(w)
    for k, power in ((0, 4), (1, 2)):
        yo, yg = band_yield(omn, X["fp64"][k], w0, power, hs), band_yield(omn, X["mixed"][k], w0, power, hs)
        po, pg = harmonic_phase(omn, X["fp64"][k], w0, hs), harmonic_phase(omn, X["mixed"][k], w0, hs)
        strong = yo > 1e-3 * yo.max()
        ey = np.max(np.abs(yg / yo - 1)[strong])
        ep = np.max(np.abs(np.angle(np.exp(1j * (pg - po))))[strong])
        print(f"full size mixed vs FP64 ({'len' if k == 0 else 'vel'}): yield {ey:.3e} phase {ep:.3e}")
        assert ey < 1e-3 and ep < 0.01, (k, ey, ep)


def test_edge_cases_and_errors():
    w = W.H_800_2CYC_GRID
    field, target = PL.make_handles(w)
    nb = field.info["n_bins"]
    d_len = torch.zeros(nb, dtype=torch.float64, device="cuda")
    d_vel = torch.zeros_like(d_len)
    b = S.Births.empty(0)
    S.sfhk_dipole(field, target, b, 0, S.prop_params(), d_len, d_vel)      # empty: no-op
    assert float(d_len.abs().sum()) == 0.0
    # all-zero amplitudes: nothing integrated, everything counted as skipped
    b = S.Births.empty(5)
    b.n0[:] = 10
    st = S.new_stats()
    S.sfhk_dipole(field, target, b, 5, S.prop_params(), d_len, d_vel, st)
    assert float(d_len.abs().sum()) == 0.0 and S.stats_dict(st)["skipped"] == 5
    with pytest.raises(S.SfhkError, match="EINVAL"):
        S.sfhk_dipole(field, target, b, 6, S.prop_params(), d_len, d_vel)  # n > capacity
    with pytest.raises(S.SfhkError, match="EINVAL"):
        S.sfhk_dipole(field, target, b, 5, S.prop_params(gamma=-1.0), d_len, d_vel)
    with pytest.raises(S.SfhkError, match="EINVAL"):
        S.sfhk_dipole(field, target, b, 5, S.prop_params(block=100), d_len, d_vel)
    with pytest.raises(S.SfhkError, match="EINVAL"):
        S.Field(1e14, 800, 2, 0, 0.03, 0.1)                                 # non-integer n_out
    with pytest.raises(S.SfhkError, match="EINVAL"):
        S.sfhk_propagate(field, target, b, 5, S.prop_params(), field.info["n_steps"] + 1)
    S.sfhk_sync()
