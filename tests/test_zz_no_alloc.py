"""The allocation-free dipole entry point against the allocating one.

sfhk_dipole_static_scratch() exists for callers that cannot allocate device
memory at call time (device memory owned by another allocator, or loops that
cannot afford cudaMalloc's device synchronisation).  Its partial bins live in a
fixed array inside the library.  Here it must reproduce sfhk_dipole with
deterministic = 1 on the same births: on two calls in a row (the second call
finds the array holding the first call's data and must clear it), after a
larger call whose partials fill more of the array than the compared call
uses, in the planar double-float precision, and at the largest size that
fits.  Device memory must not change across a call, and oversize or
escalating calls are refused for those reasons.

This file is collected last so that a run that stops at the first failure has
already run every other test.
"""
import numpy as np
import pytest
import torch

from paper_2601_17164_gb300 import workloads as W

pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    from paper_2601_17164_gb300 import pipeline as PL
    from paper_2601_17164_gb300 import sfhk as S

LIMIT = 1 << 20   # doubles in the library's static array


def _bins(field):
    nb = field.info["n_bins"]
    return torch.zeros(nb, dtype=torch.float64, device="cuda"), torch.zeros(nb, dtype=torch.float64, device="cuda")


def _reference(field, target, births, n, precision):
    pp = S.prop_params(precision, 0.5, 1e30, deterministic=1, esc_ratio=0.0)
    l, v = _bins(field)
    S.sfhk_dipole(field, target, births, n, pp, l, v)
    return l.cpu().numpy(), v.cpu().numpy()


def _static(field, target, births, n, precision):
    pp = S.prop_params(precision, 0.5, 1e30, deterministic=0, esc_ratio=0.0)
    l, v = _bins(field)
    S.sfhk_dipole_static_scratch(field, target, births, n, pp, l, v)
    torch.cuda.synchronize()
    return l.cpu().numpy(), v.cpu().numpy()


def _close(a, b, tol=1e-13):
    assert np.max(np.abs(a[0] - b[0])) <= tol * np.max(np.abs(b[0]))
    assert np.max(np.abs(a[1] - b[1])) <= tol * np.max(np.abs(b[1]))


@pytest.mark.parametrize("precision", [0, 1, 2])
def test_static_scratch_dipole_matches_allocating_dipole(precision):
    w = W.H_800_2CYC_GRID
    field, target = PL.make_handles(w)
    births = PL.sample(w, field, target)
    n = len(births)
    ref = _reference(field, target, births, n, precision)
    for call in range(2):
        _close(_static(field, target, births, n, precision), ref)
    S.sfhk_sync()


def test_static_scratch_after_a_larger_call():
    # a call that fills more blocks and more bins of the array (8 cycles, 2000 births),
    # then a smaller one with a ragged last block: the stale partials must not count
    big = W.H_800_8CYC_1M.with_n(2000)
    fb, tb = PL.make_handles(big)
    bb = PL.sample(big, fb, tb)
    _static(fb, tb, bb, big.n, S.MIXED)
    w = W.H_800_2CYC_GRID
    field, target = PL.make_handles(w)
    births = PL.sample(w, field, target)
    n = 700
    _close(_static(field, target, births, n, S.FP64), _reference(field, target, births, n, S.FP64))
    S.sfhk_sync()


def test_static_scratch_allocates_nothing():
    w = W.H_800_2CYC_GRID
    field, target = PL.make_handles(w)
    births = PL.sample(w, field, target)
    _static(field, target, births, len(births), S.MIXED)      # first call: symbol lookup, module load
    l, v = _bins(field)
    pp = S.prop_params(S.MIXED, w.gamma, w.d_t, esc_ratio=0.0)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        S.sfhk_dipole_static_scratch(field, target, births, len(births), pp, l, v)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0


def test_static_scratch_largest_size_and_rejections():
    w = W.H_800_8CYC_1M
    field, target = PL.make_handles(w)
    nb = field.info["n_bins"]
    blocks = LIMIT // (2 * nb)                     # 59 blocks of 128 at 8827 bins
    n_fit = blocks * 128
    births = PL.sample(w.with_n(n_fit + 1), field, target)
    _close(_static(field, target, births, n_fit, S.MIXED), _reference(field, target, births, n_fit, S.MIXED))
    l, v = _bins(field)
    with pytest.raises(S.SfhkError, match="exceeds the static scratch"):   # one birth more: one block more
        S.sfhk_dipole_static_scratch(field, target, births, n_fit + 1, S.prop_params(S.MIXED, esc_ratio=0.0), l, v)
    with pytest.raises(S.SfhkError, match="escalation needs per-birth scratch"):
        S.sfhk_dipole_static_scratch(field, target, births, 128, S.prop_params(S.MIXED, esc_ratio=100.0), l, v)
    S.sfhk_sync()
