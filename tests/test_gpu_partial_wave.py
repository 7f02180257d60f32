"""Partial-wave filter on the GPU (Sec. III.A-B: only trajectories whose angular
momentum at their latest entry into r < 3 falls in the selected waves
contribute) against the oracle with the same filter."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2601_17164_gb300 import workloads as W
from tests.helpers import paper_value, band_yield, harmonic_phase, oracle_births, oracle_objects, plateau_harmonics, rel_max

pytestmark = pytest.mark.gpu
RADIUS = paper_value("partial_wave_radius")[0]   # r < 3 a.u. (Sec. III.A)

if torch.cuda.is_available():
    from paper_2601_17164_gb300 import pipeline as PL
    from paper_2601_17164_gb300 import sfhk as S


def _gpu_bins(w, precision, mask, n=None, spectra=False):
    w = w if n is None else w.with_n(n)
    f, t = PL.make_handles(w)
    b = PL.sample(w, f, t)
    nb = f.info["n_bins"]
    dl = torch.zeros(nb, dtype=torch.float64, device="cuda")
    dv = torch.zeros_like(dl)
    pp = S.prop_params(precision, w.gamma, w.d_t, pw_mask=mask, pw_radius=RADIUS)
    S.sfhk_dipole(f, t, b, len(b), pp, dl, dv)
    if spectra:
        om = torch.tensor(W.omega_grid(w), dtype=torch.float64, device="cuda")
        out = []
        for d in (dl, dv):
            re, im = PL.spectrum_of(d, f, om)
            out.append(re.cpu().numpy() + 1j * im.cpu().numpy())
        return out
    torch.cuda.synchronize()
    return dl.cpu().numpy(), dv.cpu().numpy()


def _oracle_bins(w, mask, n=None):
    w = w if n is None else w.with_n(n)
    P, T, _ = oracle_objects(w)
    G = O.pulse_grid(P, w.dt, w.t_out, w.gamma, w.d_t, pw_mask=mask, pw_radius=RADIUS)
    dl, dv, _ = O.dipole(P, T, G, oracle_births(w))
    return dl, dv


def test_fp64_filtered_bins_match_oracle_and_partition():
    w = W.H_800_2CYC_GRID
    parts = []
    for mask in (1, 2, 4, 8, 5, 15):
        gl, gv = _gpu_bins(w, S.FP64, mask)
        ol, ov = _oracle_bins(w, mask)
        if mask in (1, 2, 4, 8):
            parts.append((gl, gv))
        if np.max(np.abs(ol)) == 0:
            assert np.max(np.abs(gl)) == 0 and np.max(np.abs(gv)) == 0, mask
            continue
        e = max(rel_max(gl, ol), rel_max(gv, ov))
        print(f"pw mask {mask}: rel err {e:.3e}")
        assert e < 1e-10, (mask, e)
    # the four classes partition the labelled trajectories
    all_l, all_v = _gpu_bins(w, S.FP64, 15)
    sl = sum(p[0] for p in parts)
    sv = sum(p[1] for p in parts)
    assert rel_max(sl, all_l) < 1e-12 and rel_max(sv, all_v) < 1e-12


def test_mixed_filtered_yield_and_phase():
    # p-wave trajectories only (the selection the paper uses for H 1s)
    w = W.H_800_8CYC_1M.with_n(4096)
    Xg = _gpu_bins(w, S.MIXED, 2, spectra=True)
    ol, ov = _oracle_bins(w, 2)
    P, _, G = oracle_objects(w)
    om = np.array(W.omega_grid(w))
    hs = plateau_harmonics(w)
    for name, X_g, o, power in (("len", Xg[0], ol, 4), ("vel", Xg[1], ov, 2)):
        X_o = O.spectrum(o, G.t_start, G.dt * G.n_out, P.Tp / 2, om)
        yo, yg = band_yield(om, X_o, P.omega, power, hs), band_yield(om, X_g, P.omega, power, hs)
        po, pg = harmonic_phase(om, X_o, P.omega, hs), harmonic_phase(om, X_g, P.omega, hs)
        strong = yo > 1e-3 * yo.max()
        ey = np.max(np.abs(yg / yo - 1)[strong])
        ep = np.max(np.abs(np.angle(np.exp(1j * (pg - po))))[strong])
        print(f"mixed p-wave {name}: yield {ey:.3e} phase {ep:.3e}")
        assert ey < 1e-3 and ep < 0.01, (name, ey, ep)


def test_filter_parameter_errors():
    w = W.H_800_2CYC_GRID
    f, t = PL.make_handles(w)
    b = PL.sample(w, f, t)
    nb = f.info["n_bins"]
    dl = torch.zeros(nb, dtype=torch.float64, device="cuda")
    dv = torch.zeros_like(dl)
    for bad in (dict(pw_mask=16), dict(pw_mask=-1), dict(pw_mask=2, pw_radius=0.0),
                dict(pw_mask=2, pw_radius=float("nan"))):
        with pytest.raises(S.SfhkError):
            S.sfhk_dipole(f, t, b, len(b), S.prop_params(S.FP64, **bad), dl, dv)
