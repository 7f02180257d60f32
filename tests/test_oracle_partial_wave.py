"""Pins of the oracle's partial-wave filter (Sec. III.A-B: trajectories labelled
s, p, d by their angular momentum L = |q x p| when they come within r < 3 of
the core; only the selected waves contribute).

* closed form: isotropic oscillator with the field off, where L is conserved
  and the entry time into the sphere is known analytically;
* brute force: soft-core H births with the field on, the label recomputed in
  numpy from the oracle's full path at every grid point."""
import numpy as np

import oracle as O
from paper_2601_17164_gb300 import workloads as W
from tests.helpers import paper_value, oracle_births, oracle_objects


RADIUS = paper_value("partial_wave_radius")[0]   # r < 3 a.u. (Sec. III.A)


def _one(b, i):
    return {k: np.ascontiguousarray(np.asarray(b[k])[i:i + 1]) for k in ("n0", "px", "py", "pz", "qz",
                                                                         "amp_re", "amp_im")}


def _bins(P, T, G, births):
    dl, dv, _ = O.dipole(P, T, G, births)
    return dl, dv


def test_oscillator_entry_time_and_class_closed_form():
    # V = r^2/2 (w_h = 1), E0 = 0, q0 = (0, 0, 4), p0 = (px, 0, 0):
    # L = 4 px (conserved), r^2(tau) = 16 cos^2 tau + px^2 sin^2 tau, first inside r < 3
    # once cos^2 tau < (9 - px^2) / (16 - px^2)
    P = O.make_pulse(E0=0.0, omega=0.057, cycles=2.0)
    T = O.make_target(O.POT_HARMONIC, [1.0], ip=0.5, gto_l=0, c=W.H_C, alpha=W.H_ALPHA)
    dt, N, n_out = 0.01, 4000, 10
    for px, cls in ((0.075, 0), (0.25, 1), (0.5, 2), (0.8, 3)):
        b = {"n0": np.array([0], np.int32), "px": np.array([px]), "py": np.zeros(1), "pz": np.zeros(1),
             "qz": np.array([4.0]), "amp_re": np.array([1.0]), "amp_im": np.array([0.3])}
        G0 = O.make_grid(0.0, dt, N, n_out, gamma=0.5)
        ref_l, ref_v = _bins(P, T, G0, b)
        tau_e = np.arccos(np.sqrt((9 - px * px) / (16 - px * px)))
        n_e = int(np.floor(tau_e / dt)) + 1                   # first grid point inside
        assert abs(n_e * dt - tau_e) > 1e-6 and abs((n_e - 1) * dt - tau_e) > 1e-6   # no grid point at r = 3
        after = (np.arange(ref_l.size) * n_out) >= n_e
        assert after.any() and (~after).any() and np.any(ref_l[after] != 0)
        for mask in (1, 2, 4, 8, 15, 5):
            G = O.make_grid(0.0, dt, N, n_out, gamma=0.5, pw_mask=mask, pw_radius=RADIUS)
            fl, fv = _bins(P, T, G, b)
            keep = after & bool((mask >> cls) & 1)
            assert np.array_equal(fl, np.where(keep, ref_l, 0.0)), (px, mask)
            assert np.array_equal(fv, np.where(keep, ref_v, 0.0)), (px, mask)


def _classes_from_path(path, radius):
    """Latest entry class at every grid point of a path [n][43] (-1 before the first entry)."""
    q, p = path[:, 0:3], path[:, 3:6]
    inside = np.einsum("ij,ij->i", q, q) < radius * radius
    L = np.linalg.norm(np.cross(q, p), axis=1)
    lab = np.where(L < 0.5, 0, np.where(L < 1.5, 1, np.where(L < 2.5, 2, 3)))
    out = np.full(len(path), -1)
    cur, was = -1, False
    for n in range(len(path)):
        if inside[n] and not was:
            cur = lab[n]
        was = inside[n]
        out[n] = cur
    return out


def test_filter_matches_labels_recomputed_from_the_path():
    w = W.H_800_2CYC_GRID
    P, T, G0 = oracle_objects(w)
    b = oracle_births(w)
    live = np.nonzero(np.hypot(b["amp_re"], b["amp_im"]) > 0)[0]
    pick = live[np.linspace(0, live.size - 1, 12).astype(int)]
    seen = set()
    for i in pick:
        one = _one(b, i)
        ref_l, ref_v = _bins(P, T, G0, one)
        n0 = int(one["n0"][0])
        path = O.trajectory(P, T, G0, n0, G0.n_steps, [0.0, 0.0, one["qz"][0]],
                            [one["px"][0], one["py"][0], one["pz"][0]])
        cls = _classes_from_path(path, RADIUS)
        seen.update(set(cls.tolist()))
        k = np.arange(ref_l.size)
        n = k * G0.n_out
        lab = np.where(n >= n0, cls[np.clip(n - n0, 0, len(cls) - 1)], -1)
        for mask in (2, 5, 15):
            G = O.pulse_grid(P, w.dt, w.t_out, w.gamma, w.d_t, pw_mask=mask, pw_radius=RADIUS)
            fl, fv = _bins(P, T, G, one)
            keep = (lab >= 0) & ((mask >> np.maximum(lab, 0)) & 1).astype(bool)
            assert np.array_equal(fl, np.where(keep, ref_l, 0.0)), (i, mask)
            assert np.array_equal(fv, np.where(keep, ref_v, 0.0)), (i, mask)
    assert len(seen - {-1}) >= 2          # the sample reaches the core with more than one wave
