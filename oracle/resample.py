"""Importance sampling of births in proportion to |I0| (App. A, Eq. Int: a
momentum k that satisfies the saddle-point equation carries a weight
proportional to |I0|, which implements importance sampling of the Monte Carlo
integral), as systematic resampling of a proposal pool.

Test infrastructure only: loaded by tests, the smoke check and the CPU
baseline of the benchmark.  Integer steps in Python integers (exact); the
floating-point steps are single IEEE operations in the order the CUDA side
uses, so the two agree bit for bit.

Definition (reading of the paper's one-sentence scheme):
  pool      m proposal births i = 0..m-1 (the sampler's own, sorted by birth
            step), amplitudes a_i that already carry the proposal weight;
  weights   w_i = sqrt(Re a_i * Re a_i + Im a_i * Im a_i) (= |I0| times the
            proposal weight, no fused multiply-add), A = max w_i;
            q_i = floor(w_i * (2^B / A)) with B = 62 - ceil(log2 m) (integers,
            Q = sum q_i < 2^62; a birth with q_i = 0 is never drawn);
  draw      one 32-bit uniform U (Philox4x64-10, key (seed, 1), counter
            (0, 0, 0, 0), word 0's high half); n thresholds
            t_j = floor((j 2^32 + U) Q / (n 2^32)), j = 0..n-1 (systematic);
  selection pool birth i is drawn m_i = #{j : C_{i-1} <= t_j < C_i} times,
            C_i = q_0 + ... + q_i;
            A pool whose A is 0, infinite or NaN draws nothing.
  output    the births with m_i > 0 in pool order (so still sorted by birth
            step), amplitude a_i * ((m_i Q) / (n q_i)), then zero-amplitude
            padding up to n entries (not integrated).
The estimator sum_out amp = sum_i a_i m_i Q / (n q_i) has expectation
sum_i a_i over U (unbiased except for the q_i = 0 births, |a_i| < 2^-B A).
Pinned by tests/test_oracle_resample.py.
"""
from __future__ import annotations

import math

import numpy as np

from . import oracle as O


def scale_bits(m: int) -> int:
    return 62 - max(1, math.ceil(math.log2(max(2, m))))


def quantized_weights(amp_re, amp_im):
    """(q as Python ints, Q, B, A)."""
    re = np.asarray(amp_re, dtype=np.float64)
    im = np.asarray(amp_im, dtype=np.float64)
    w = np.sqrt(re * re + im * im)        # separate multiply and add, correctly rounded sqrt
    m = w.size
    B = scale_bits(m)
    A = float(w.max()) if m else 0.0
    if not (A > 0.0 and math.isfinite(A)):       # no pool weight, or an infinite / NaN one: no draws
        return [0] * m, 0, B, A
    s = math.ldexp(1.0, B) / A
    q = [int(math.floor(float(x) * s)) for x in w]
    return q, sum(q), B, A


def uniform32(seed: int) -> int:
    x = O.philox4x64([0, 0, 0, 0], [seed, 1])
    return int(x[0]) >> 32


def thresholds(n: int, Q: int, U: int):
    """t_j = floor((j 2^32 + U) Q / (n 2^32)), the systematic draw points."""
    return [((j << 32) + U) * Q // (n << 32) for j in range(n)]


def multiplicities(q, n: int, U: int):
    """m_i from the count of thresholds below each cumulative sum (closed form of the
    inverse of t_j: #{j : t_j < c} = clamp(ceil((ceil(c n 2^32 / Q) - U) / 2^32), 0, n))."""
    Q = sum(q)
    if Q == 0:
        return [0] * len(q)

    def J(c):
        L = -((-c * n << 32) // Q)            # ceil(c n 2^32 / Q)
        k = -(-(L - U) // (1 << 32))          # ceil((L - U) / 2^32)
        return min(max(k, 0), n)
    out, c_prev, j_prev = [], 0, 0
    for qi in q:
        c = c_prev + qi
        jc = J(c)
        out.append(jc - j_prev)
        c_prev, j_prev = c, jc
    return out


def resample(births: dict, n: int, seed: int):
    """Resampled births (dict of arrays, n entries) and the number of distinct ones."""
    q, Q, _, _ = quantized_weights(births["amp_re"], births["amp_im"])
    U = uniform32(seed)
    mult = multiplicities(q, n, U)
    keys = ("n0", "t0", "px", "py", "pz", "qz", "amp_re", "amp_im")
    out = {k: np.zeros(n, dtype=np.asarray(births[k]).dtype) for k in keys}
    r = 0
    for i, mi in enumerate(mult):
        if mi == 0:
            continue
        for k in ("n0", "t0", "px", "py", "pz", "qz"):
            out[k][r] = births[k][i]
        f = (float(mi) * float(Q)) / (float(n) * float(q[i]))
        out["amp_re"][r] = births["amp_re"][i] * f
        out["amp_im"][r] = births["amp_im"][i] * f
        r += 1
    if r < n:
        for k in ("n0", "t0", "px", "py", "pz", "qz"):
            out[k][r:] = out[k][r - 1] if r > 0 else births[k][0]
        out["amp_re"][r:] = 0.0
        out["amp_im"][r:] = 0.0
    return out, r
