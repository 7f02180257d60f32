"""The allocation-free dipole entry point against the allocating one.

sfhk_dipole_static_scratch() exists for callers that cannot allocate device
memory at call time (device memory owned by another allocator, or loops that
cannot afford cudaMalloc's device synchronisation).  Its partial bins live in a
fixed array inside the library.  Here it must reproduce sfhk_dipole with
deterministic = 1 on the same births, on two calls in a row (the second call
finds the array holding the first call's data and must clear it).

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


def _bins(field):
    nb = field.info["n_bins"]
    return torch.zeros(nb, dtype=torch.float64, device="cuda"), torch.zeros(nb, dtype=torch.float64, device="cuda")


@pytest.mark.parametrize("precision", [0, 1])
def test_static_scratch_dipole_matches_allocating_dipole(precision):
    w = W.H_800_2CYC_GRID
    field, target = PL.make_handles(w)
    births = PL.sample(w, field, target)
    n = len(births)
    pp_ref = S.prop_params(precision, w.gamma, w.d_t, deterministic=1, esc_ratio=0.0)
    ref_l, ref_v = _bins(field)
    S.sfhk_dipole(field, target, births, n, pp_ref, ref_l, ref_v)
    pp = S.prop_params(precision, w.gamma, w.d_t, deterministic=0, esc_ratio=0.0)
    for call in range(2):
        d_l, d_v = _bins(field)
        S.sfhk_dipole_static_scratch(field, target, births, n, pp, d_l, d_v)
        torch.cuda.synchronize()
        a, b = d_l.cpu().numpy(), ref_l.cpu().numpy()
        c, d = d_v.cpu().numpy(), ref_v.cpu().numpy()
        assert np.max(np.abs(a - b)) <= 1e-13 * np.max(np.abs(b)), call
        assert np.max(np.abs(c - d)) <= 1e-13 * np.max(np.abs(d)), call
    S.sfhk_sync()


def test_static_scratch_rejects_oversize_and_escalation():
    w = W.H_800_8CYC_1M.with_n(200_000)
    field, target = PL.make_handles(w)
    births = S.Births.empty(w.n)
    d_l, d_v = _bins(field)
    with pytest.raises(S.SfhkError, match="EINVAL"):   # 1563 blocks * 2 * 8827 bins > 2^20
        S.sfhk_dipole_static_scratch(field, target, births, w.n, S.prop_params(S.FP64), d_l, d_v)
    with pytest.raises(S.SfhkError, match="EINVAL"):
        S.sfhk_dipole_static_scratch(field, target, births, 128, S.prop_params(S.MIXED, esc_ratio=100.0), d_l, d_v)
