"""Pins of the |I0| importance resampling oracle (App. A): the closed-form
multiplicities against a brute-force count of the systematic thresholds, the
systematic-resampling bounds, exact conservation of the draw count, the
unbiasedness of the weighted sum over draws, and the degenerate cases."""
import numpy as np

import oracle as O
from oracle import resample as RS
from paper_2601_17164_gb300 import workloads as W
from tests.helpers import oracle_objects


def _brute_multiplicities(q, n, U):
    C = np.cumsum(np.array(q, dtype=object))
    t = RS.thresholds(n, int(C[-1]), U)
    m = [0] * len(q)
    for tj in t:                         # first i with C_i > t_j
        lo, hi = 0, len(q) - 1
        while lo < hi:
            mid = (lo + hi) // 2
            if C[mid] > tj:
                hi = mid
            else:
                lo = mid + 1
        m[lo] += 1
    return m


def test_closed_form_multiplicities_match_thresholds():
    rng = np.random.default_rng(2)
    for m_pool, n in ((50, 7), (300, 300), (1000, 64), (200, 1000)):
        w = rng.lognormal(0.0, 3.0, m_pool)
        w[rng.random(m_pool) < 0.2] = 0.0
        q, Q, B, A = RS.quantized_weights(w, np.zeros(m_pool))
        assert Q < 2 ** 62 and max(q) <= 2 ** B
        for U in (0, 1, 2 ** 31, 2 ** 32 - 1, int(rng.integers(0, 2 ** 32))):
            mult = RS.multiplicities(q, n, U)
            assert mult == _brute_multiplicities(q, n, U)
            assert sum(mult) == n
            for qi, mi in zip(q, mult):        # systematic: floor or ceil of the expected count
                e = n * qi / Q
                assert np.floor(e) - 1e-9 <= mi <= np.ceil(e) + 1e-9
                if qi == 0:
                    assert mi == 0


def test_weighted_sum_is_unbiased_over_draws():
    rng = np.random.default_rng(7)
    m_pool, n = 400, 40
    re = rng.standard_normal(m_pool) * rng.lognormal(0, 2, m_pool)
    im = rng.standard_normal(m_pool) * rng.lognormal(0, 2, m_pool)
    q, Q, _, _ = RS.quantized_weights(re, im)
    a = re + 1j * im
    target = a.sum()
    K = 4000
    tot = 0.0
    for _ in range(K):
        U = int(rng.integers(0, 2 ** 32))
        mult = RS.multiplicities(q, n, U)
        tot += sum(a[i] * mi * Q / (n * q[i]) for i, mi in enumerate(mult) if mi)
    mean = tot / K
    scale = np.abs(a).sum() / np.sqrt(K)
    assert abs(mean - target) < 3 * scale


def test_resampled_births_from_the_sampler():
    w = W.H_800_8CYC_1M
    P, T, G = oracle_objects(w)
    m_pool, n = 4000, 1000
    pool = O.sample_births(P, T, G, w.birth_mode, m_pool, w.n_t, w.n_k, w.sigma, w.kmax, w.seed)
    out, r = RS.resample(pool, n, seed=5)
    assert 0 < r <= n
    assert np.all(np.diff(out["n0"]) >= 0)                      # still sorted by birth step
    mag = np.hypot(out["amp_re"][:r], out["amp_im"][:r])
    q, Q, _, _ = RS.quantized_weights(pool["amp_re"], pool["amp_im"])
    A = np.hypot(pool["amp_re"], pool["amp_im"]).max()
    # every drawn birth carries |a| Q m / (n q) ~ A Q m / (n 2^B): magnitudes equal up to m
    unit = A * Q / (n * 2.0 ** RS.scale_bits(m_pool))
    ratio = mag / unit
    assert np.all(ratio > 0.999) and np.all(np.abs(ratio - np.round(ratio)) < 1e-6 * ratio + 1e-9)
    assert np.all(out["amp_re"][r:] == 0) and np.all(out["amp_im"][r:] == 0)
    # the phases are the pool's
    idx = {(int(a), float(b), float(c)): k for k, (a, b, c) in enumerate(zip(pool["n0"], pool["px"], pool["py"]))}
    for k in range(0, r, max(1, r // 50)):
        i = idx[(int(out["n0"][k]), float(out["px"][k]), float(out["py"][k]))]
        ph_in = np.angle(pool["amp_re"][i] + 1j * pool["amp_im"][i])
        ph_out = np.angle(out["amp_re"][k] + 1j * out["amp_im"][k])
        assert abs(np.angle(np.exp(1j * (ph_out - ph_in)))) < 1e-12


def test_degenerate_pools():
    z = {k: np.zeros(10) for k in ("t0", "px", "py", "pz", "qz", "amp_re", "amp_im")}
    z["n0"] = np.arange(10, dtype=np.int32)
    out, r = RS.resample(z, 5, seed=1)
    assert r == 0 and np.all(out["amp_re"] == 0)
    one = {k: v.copy() for k, v in z.items()}
    one["amp_re"][3] = 2.5
    out, r = RS.resample(one, 4, seed=1)
    assert r == 1 and out["n0"][0] == 3 and out["amp_re"][0] == 2.5   # drawn 4 times, weight Q 4/(4 Q)
    # an infinite or NaN amplitude: no weight scale, nothing drawn
    for bad in (np.inf, np.nan):
        b = {k: v.copy() for k, v in one.items()}
        b["amp_im"][5] = bad
        out, r = RS.resample(b, 4, seed=1)
        assert r == 0 and np.all(out["amp_re"] == 0) and out["n0"][0] == 0
