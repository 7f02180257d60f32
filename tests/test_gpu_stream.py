"""The streamed workload through the CUDA library: Ar (Tong-Lin), 2000 nm, 20
cycles, 8e13 W/cm^2, births of the 1e8-birth sample produced and propagated in
chunks of consecutive births, the bins accumulated across chunks with a
checkpoint after each; a run stopped after two chunks resumes from its
checkpoint in a fresh StreamRun and ends with the bins of one call over all
the births (to 1e-13 of max |D|, the summation order aside).
"""
import tempfile

import numpy as np
import pytest
import torch

from paper_2601_17164_gb300 import workloads as W

pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    from paper_2601_17164_gb300 import sfhk as S
    from paper_2601_17164_gb300.stream import GpuBackend, StreamRun


# the mixed path's escalation floor and large-contribution tier are relative to each
# call's largest amplitude, so chunks and one call agree with both off
@pytest.mark.parametrize("precision,prop", [("fp64", {}), ("mixed", {"esc_floor": 0.0, "esc_big": 0.0})])
def test_gpu_stream_resumes_and_equals_one_call(precision, prop):
    w = W.AR_2000_20CYC_100M
    prec = S.FP64 if precision == "fp64" else S.MIXED
    lo = 50_000_000 - 2048 if precision == "fp64" else 50_000_000 - 8192
    n_sub = 4096 if precision == "fp64" else 16384
    chunk = n_sub // 4
    be = GpuBackend(w, prec, n_sub, **prop)
    # one call over all the births of the range
    births = be.sample(lo, n_sub)
    full_l, full_v = np.zeros(be.n_bins), np.zeros(be.n_bins)
    st_full = be.dipole(births, full_l, full_v)
    with tempfile.TemporaryDirectory() as d:
        r = StreamRun(w, be, chunk=chunk, checkpoint_dir=d, lo=lo, hi=lo + n_sub)
        r.run(max_chunks=2)                       # stopped after two chunks
        assert r.state.next_chunk == 2 and not r.finished
        r2 = StreamRun(w, be, chunk=chunk, checkpoint_dir=d, lo=lo, hi=lo + n_sub)
        assert r2.state.next_chunk == 2
        dl, dv = r2.run()
        assert r2.finished and r2.n_chunks == 4
    e_l = np.max(np.abs(dl - full_l)) / np.max(np.abs(full_l))
    e_v = np.max(np.abs(dv - full_v)) / np.max(np.abs(full_v))
    print(f"{precision}: streamed vs one call: len {e_l:.2e} vel {e_v:.2e}, "
          f"escalated {r2.state.escalated} (one call {st_full['escalated']})")
    assert e_l < 1e-13 and e_v < 1e-13
    assert r2.state.traj_steps == st_full["traj_steps"]
    assert r2.state.escalated == st_full["escalated"]
    S.sfhk_sync()
