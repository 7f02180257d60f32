"""Benchmark of the SFHK trajectory hot path on GB300.

One step = one pass of the whole path over one batch of synthetic births:
births (SFA saddle points) -> propagation + prefactor + fused dipole bins ->
windowed spectra (length and velocity forms), for the workload
"H 800 nm, 8 cycles, 1.5e14 W/cm^2, 1e6 births, dt = 0.01 a.u." in the
FP32-mixed precision mode.  Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

--impl reference times the FP64 CPU oracle on the host cores (a bounded
stride sample of the same births per step).  Under torchrun each rank runs its
own births (weak scaling) and the bins are summed across ranks once per step.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2601_17164_gb300 import workloads as W  # noqa: E402

WORKLOAD = W.H_800_8CYC_1M
METRIC = "trajectory-steps/s (FP32-mixed SFHK path, births->dipole->spectrum)"
UNIT = "trajectory-steps/s"
FP32_LANES_PER_SM = 128
FP64_LANES_PER_SM = 2
SM_COUNT = 152
SM_MAX_MHZ = 2070.0
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one launch of the float pass
# at the default configuration, per birth of the launch, from one full-size ncu capture of
# the bench's own command (one pass, --clock-control none; the mean of its three launches:
# 53,931,861 + 171 B for 1e6 births).  None while no capture of the kernel as it stands exists.
FLOAT_PASS_DRAM_BYTES_PER_BIRTH = 53.932032
# The same for the FP64 redo at the default configuration (6,989,739 + 0 B), keyed by
# (births, esc_ratio, esc_floor, esc_ratio_big, esc_big); other configurations, and
# kernels changed since the capture, report null.
REDO_DRAM_BYTES_DEFAULT = {(1_000_000, 200.0, 1e-2, 40.0, 1000.0): 6989739}


# ----------------------------------------------------------------------------
# algorithmic work of the dominant kernel (operation counts of the planar and 3D steps)
# ----------------------------------------------------------------------------
def flops_per_traj_step(pot: int, planar: bool = True, compensated: bool = True) -> float:
    """Floating-point operations of one RK4 trajectory-step as written in traj_block.cuh
    (an FMA counts 2; add, mul, rsqrt, exp 1): potential evaluations, stage derivatives
    and inputs, the RK4 combination, Kahan compensation (float path), the stability
    columns and the determinant that follows the branch (every step; the planar float
    pass every fifth one, with n_out a multiple of 5).  The planar form advances the
    columns with the RK4 step written as one matrix from the stage Hessians; the 3D
    form propagates each column through the four stages."""
    if planar:
        pot_cost = {W.POT_SOFTCORE: 9, W.POT_TONGLIN: 38, W.POT_HARMONIC: 5, W.POT_ZERO: 0}[pot]
        qps = 4 * pot_cost + 4 * (3 + 7) + 3 * 8 + 25       # (q, p, S) stages and combination
        branch = 45 + 8                                       # det of the rescaled 2x2 block x Z_yy, follow
        if compensated:
            branch *= 0.2                                     # the float pass: every fifth step
        # q, p with Kahan's carries (4 each); the float pass's action: its increment
        # joins the low word in the combination's FMA (1) and is folded with TwoSum,
        # the carry and the 2 pi reduction (9) every fifth step
        comp = 16 + 1 + 0.2 * 9 if compensated else 0
        hess = 4 * 7                                          # H_s entries a, b, c per stage
        blocks = 8 + 3 + 24 + 16 + 5 + 28 + 16                # constants, sums, H3H1, H4H2, A, B, C, D
        cols = 4 * 4 * 7 + (16 * 4 if compensated else 16)   # 4 columns x 4 rows of [A B; C D] x, (Kahan) adds
        oop = 21 + 4 * 3 + (4 * 4 if compensated else 4)      # out-of-plane 2x2 step matrix, 2 columns
        return float(qps + comp + hess + blocks + cols + oop + branch)
    pot_cost = {W.POT_SOFTCORE: 11, W.POT_TONGLIN: 40, W.POT_HARMONIC: 6, W.POT_ZERO: 0}[pot]
    qps = 4 * pot_cost + 4 * (4 + 9) + 3 * 12 + 35
    comp = 33 if compensated else 0
    cols = 6 * 156 - (0 if compensated else 6 * 18)
    branch = 109 + 8
    return float(qps + comp + cols + branch)


def launches_per_step(n: int, n_steps: int, chunk: int, prec: int, floor: bool, overlap: int = 0,
                      block: int = 128, side: int = 8, esc_precision: int = 0) -> int:
    """Our kernels per step: births, the trajectory pass(es), spectra (x2).  The mixed
    path with escalation (as sfhk_dipole runs it) adds the amplitude maximum and, per
    birth chunk (overlap 0) or time segment (overlap 1) of the float pass, or once
    (overlap 2, sequential), the float launch, three compaction kernels and the
    high-precision redo (the four-warp redo of esc_precision 0, planar form, with its
    one-warp group plan before it)."""
    if prec != 1:
        return 1 + 1 + 2
    if overlap == 2:
        parts = 1
    elif overlap == 0:
        per = -(-n // side)
        csz = max(-(-per // block) * block, 64 * block)
        parts = -(-n // csz)
    else:
        parts = min(side, (n_steps + chunk) // chunk)
    return 1 + (1 if floor else 0) + parts * (6 if esc_precision == 0 else 5) + 2


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(prefix="clk", suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), float(parts[3]), parts[5:9]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i, v in enumerate(r[3]) if v.lower() == "active"})
        loaded = [r for r in rows if r[2] > 200.0] or rows
        return {"sm_mhz": statistics.median(r[0] for r in loaded), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows), "power_w_max": max(r[2] for r in rows)}


# ----------------------------------------------------------------------------
# reference arm: the FP64 oracle on the host cores
# ----------------------------------------------------------------------------
def oracle_sample(w, stride):
    import numpy as np

    import oracle as O
    p = w.pulse
    P = O.make_pulse(p.intensity_wcm2, p.lambda_nm, p.cycles, p.cep)
    t = w.target
    T = O.make_target(t.pot, t.pot_param, t.ip, t.gto_l, t.c, t.alpha)
    G = O.pulse_grid(P, w.dt, w.t_out, w.gamma, w.d_t)
    idx = np.arange(0, w.n, stride, dtype=np.int64)
    return O, P, T, G, idx


def run_oracle_step(w, stride):
    """One bounded oracle step: births + dipole + spectra for every stride-th birth."""
    import numpy as np
    O, P, T, G, idx = oracle_sample(w, stride)
    t0 = time.perf_counter()
    b = O.sample_births_at(P, T, G, w.birth_mode, w.n, idx, w.n_t, w.n_k, w.sigma, w.kmax, w.seed)
    dl, dv, st = O.dipole(P, T, G, b)
    om = np.array(W.omega_grid(w))
    O.spectrum(dl, G.t_start, G.dt * G.n_out, P.Tp / 2, om)
    O.spectrum(dv, G.t_start, G.dt * G.n_out, P.Tp / 2, om)
    return time.perf_counter() - t0, st["traj_steps"], len(idx)


def cpu_model() -> str:
    """The host CPU's model name as lscpu prints it (else the platform's processor string)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    import platform
    return platform.processor() or platform.machine()


def cpu_baseline(w, stride, target_s=20.0):
    """The oracle on every host thread on a stride sample, and on one thread on a sample
    as many times sparser (so both take about the same wall time)."""
    import oracle as O
    secs, steps, m = run_oracle_step(w, stride)
    cores = O.max_threads()
    O.set_threads(1)
    try:
        s1, st1, m1 = run_oracle_step(w, stride * cores)
    finally:
        O.set_threads(cores)
    return {"value": steps / secs, "unit": UNIT, "cores": cores, "kind": "oracle", "cpu_model": cpu_model(),
            "sample": f"every {stride}th of the {w.n} births ({m} births, {steps:.3g} trajectory-steps, "
                      f"{secs:.1f} s), births + dipole + spectra",
            "one_thread": {"value": st1 / s1, "unit": UNIT,
                           "sample": f"every {stride * cores}th birth ({m1} births, {st1:.3g} trajectory-steps, "
                                     f"{s1:.1f} s)"}}


def reference_arm(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle as O
    O.build()
    w = WORKLOAD
    stride = args.ref_stride
    for _ in range(args.warmup):
        run_oracle_step(w, stride * 4)
    tot_s, tot_steps, m = 0.0, 0.0, 0
    for _ in range(args.steps):
        s, st, m = run_oracle_step(w, stride)
        tot_s += s
        tot_steps += st
    v = tot_steps / tot_s
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_s / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": w.name, "sample_births_per_step": m},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": O.max_threads(), "kind": "oracle",
                             "sample": f"every {stride}th of the {w.n} births ({m} births) per step"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def run_record(w, field, target, births, info, pp, prec, omega, stream, n_det=64, stride=64):
    """Health figures of a run for the JSON-lines record: max |det M - 1| of the 6x6
    monodromy matrix over a sampled subset propagated in FP64 to the pulse's end
    (removed trajectories left out; the sample's largest |M| entry is reported beside
    it, since rounding grows with it), and the plateau yield and phase errors of the
    configured path against the FP64 path on a stride sample of the same births."""
    import numpy as np
    import torch

    from paper_2601_17164_gb300 import pipeline as PL
    from paper_2601_17164_gb300 import sfhk as S
    idx = torch.linspace(0, w.n - 1, n_det, device="cuda").long()
    sub = S.Births(*(getattr(births, k)[idx].contiguous() for k in ("n0", "t0", "p0x", "p0y", "p0z", "q0z",
                                                                    "amp_re", "amp_im")))
    st, _, fl = S.sfhk_propagate(field, target, sub, n_det, S.prop_params(S.FP64, w.gamma, w.d_t), info["n_steps"])
    st, fl = st.cpu().numpy(), fl.cpu().numpy()
    keep = (fl & 3) == 0
    M = np.zeros((keep.sum(), 6, 6))
    for a, (b0, c0) in enumerate(((6, 0), (15, 3), (24, 0), (33, 3))):   # Mqq, Mqp, Mpq, Mpp blocks
        r0 = 0 if a < 2 else 3
        for i in range(3):
            for j in range(3):
                M[:, r0 + i, c0 + j] = st[b0 + 3 * i + j, keep]
    det_err = float(np.max(np.abs(np.linalg.det(M) - 1))) if len(M) else None
    # the configured path and the FP64 path on every stride-th birth
    idx = torch.arange(0, w.n, stride, device="cuda")
    sb = S.Births(*(getattr(births, k)[idx].contiguous() for k in ("n0", "t0", "p0x", "p0y", "p0z", "q0z",
                                                                   "amp_re", "amp_im")))
    X = {}
    for name, q in (("run", pp), ("fp64", S.prop_params(S.FP64, w.gamma, w.d_t))):
        dl = torch.zeros(info["n_bins"], dtype=torch.float64, device="cuda")
        dv = torch.zeros_like(dl)
        S.sfhk_dipole(field, target, sb, len(sb), q, dl, dv, None, stream)
        X[name] = [re.cpu().numpy() + 1j * im.cpu().numpy() for re, im in (PL.spectrum_of(d, field, omega, stream)
                                                                            for d in (dl, dv))]
    om = omega.cpu().numpy()
    w0 = 45.5633525 / w.pulse.lambda_nm
    E0 = (w.pulse.intensity_wcm2 / 3.50944758e16) ** 0.5
    # odd harmonics from just above Ip to the classical cutoff Ip + 3.17 Up
    hs = [h for h in range(int(np.ceil(w.target.ip / w0)), int((w.target.ip + 3.17 * E0 ** 2 / (4 * w0 ** 2)) / w0) + 1)
          if h % 2 == 1]
    band = lambda X, p: np.array([(np.abs(X) ** 2 * om ** p)[np.abs(om / w0 - h) <= 0.5].sum() for h in hs])
    phase = lambda X: np.array([np.angle(X[np.argmin(np.abs(om - h * w0))]) for h in hs])
    errs = {}
    for k, name, power in ((0, "length", 4), (1, "velocity", 2)):
        yo, yg = band(X["fp64"][k], power), band(X["run"][k], power)
        po, pg = phase(X["fp64"][k]), phase(X["run"][k])
        strong = yo > 1e-3 * yo.max()
        errs[name] = {"yield": float(np.max(np.abs(yg / yo - 1)[strong])),
                      "phase_rad": float(np.max(np.abs(np.angle(np.exp(1j * (pg - po))))[strong]))}
    return {"max_abs_detM_minus_1": det_err, "detM_sample": int(keep.sum()),
            "max_abs_M_entry": float(np.max(np.abs(M))) if len(M) else None,
            "errors_vs_fp64_path": errs, "errors_sample": f"every {stride}th birth ({len(sb)} births)"}


# ----------------------------------------------------------------------------
# GPU arm
# ----------------------------------------------------------------------------
def gpu_arm(args):
    import torch
    import torch.distributed as dist

    from paper_2601_17164_gb300 import pipeline as PL
    from paper_2601_17164_gb300 import sfhk as S

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    w = WORKLOAD if not args.births else WORKLOAD.with_n(args.births)
    prec = S.MIXED if args.precision == "mixed" else S.FP64
    seed = w.seed + 1000 * rank
    stream = torch.cuda.current_stream()
    field, target = PL.make_handles(w)
    info = field.info
    nb = info["n_bins"]
    births = S.Births.empty(w.n)
    d_len = torch.zeros(nb, dtype=torch.float64, device="cuda")
    d_vel = torch.zeros_like(d_len)
    omega = torch.tensor(W.omega_grid(w), dtype=torch.float64, device="cuda")
    X = [torch.empty_like(omega) for _ in range(4)]
    stats = S.new_stats()
    pp = S.prop_params(prec, w.gamma, w.d_t, 0, args.block, args.chunk, esc_ratio=args.esc_ratio,
                       esc_floor=args.esc_floor, esc_overlap=args.esc_overlap, esc_precision=args.esc_precision)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    tau = 0.5 * info["Tp"]
    dto = info["dt"] * info["n_out"]
    ev = lambda: torch.cuda.Event(enable_timing=True)

    def step(record=None, handles=None):
        fh, th = handles if handles is not None else (field, target)
        d_len.zero_()
        d_vel.zero_()
        stats.zero_()
        S.sfhk_sample_births(fh, th, w.birth_mode, w.n, births, w.n_t, w.n_k, w.sigma, w.kmax, seed, stream)
        if record:
            record[0].record(stream)
        S.sfhk_dipole(fh, th, births, w.n, pp, d_len, d_vel, stats, stream)
        if record:
            record[1].record(stream)
        if world > 1:
            dist.all_reduce(d_len)
            dist.all_reduce(d_vel)
        S.sfhk_spectrum(d_len, info["t_start"], dto, tau, omega, X[0], X[1], stream)
        S.sfhk_spectrum(d_vel, info["t_start"], dto, tau, omega, X[2], X[3], stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    S.sfhk_sync()
    warm_stats = S.stats_dict(stats)
    steps_per_launch = warm_stats["traj_steps"]

    clocks = Clocks(local)
    starts, ends, kstarts, kends, phases = [], [], [], [], []
    S.sfhk_set_phase_timing(True)   # CUDA events around each launch inside sfhk_dipole
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    t_wall = time.perf_counter()
    for _ in range(args.steps):
        flush.fill_(1.0)                        # L2 flush between steps (256 MiB write)
        s0, s1, k0, k1 = ev(), ev(), ev(), ev()
        s0.record(stream)
        step(record=(k0, k1))
        s1.record(stream)
        starts.append(s0), ends.append(s1), kstarts.append(k0), kends.append(k1)
        phases.append(S.sfhk_get_phase_times())   # waits for this step's dipole call only
    torch.cuda.synchronize()
    S.sfhk_set_phase_timing(False)
    if world > 1:
        dist.barrier()
    wall = time.perf_counter() - t_wall
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in zip(starts, ends)]
    kern_ms = [a.elapsed_time(b) for a, b in zip(kstarts, kends)]
    t_dev = sum(step_ms) / 1e3
    S.sfhk_sync()
    if world > 1:
        tt = torch.tensor([t_dev], dtype=torch.float64, device="cuda")
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t_dev = float(tt)
    total_steps = steps_per_launch * world * args.steps
    value = total_steps / t_dev

    # --- end to end through the public API with host buffers --------------
    # every step makes the configuration's handles (sfhk_make_field computes the
    # half-step E tables on the host and uploads them; sfhk_make_target), copies the
    # frequency grid in from pinned memory, runs births -> dipole -> spectra and reads
    # the spectra and counters back; wall-clock time over the steps (host work included)
    e2e = None
    if rank == 0 and not args.no_e2e:
        om_host = torch.tensor(W.omega_grid(w), dtype=torch.float64).pin_memory()
        out_host = torch.empty((4, om_host.numel()), dtype=torch.float64).pin_memory()
        st_host = torch.empty(8, dtype=torch.int64).pin_memory()
        table_len = (2 * info["n_steps"] + 1 + 64) // 64 * 64
        h2d = om_host.numel() * 8 + table_len * (8 + 4)      # frequencies + the FP64 and float E tables
        d2h = out_host.numel() * 8 + st_host.numel() * 8
        reps = max(1, args.steps // 2)
        keep = []                                            # handles freed after the timed region
        torch.cuda.synchronize()
        t_e = time.perf_counter()
        for _ in range(reps):
            keep.append(PL.make_handles(w))
            omega.copy_(om_host, non_blocking=True)
            step(handles=keep[-1])
            for j in range(4):
                out_host[j].copy_(X[j], non_blocking=True)
            st_host.copy_(stats, non_blocking=True)
        torch.cuda.synchronize()
        e2e_s = time.perf_counter() - t_e
        del keep
        e2e = {"value": steps_per_launch * reps / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "spectra_per_s": 2 * reps / e2e_s,
               "timing": "host wall clock per step: handles (host E tables + upload), frequencies in, "
                         "births -> dipole -> spectra, spectra and counters out"}

    # --- FP64 path on a stride subset of the same births --------------------
    fp64 = None
    if rank == 0 and not args.no_fp64 and prec == S.MIXED:
        sub = births.slice(0, w.n)
        stride = args.fp64_stride
        idx = torch.arange(0, w.n, stride, device="cuda")
        sb = S.Births(*(getattr(sub, k)[idx].contiguous() for k in ("n0", "t0", "p0x", "p0y", "p0z", "q0z",
                                                                  "amp_re", "amp_im")))
        st64 = S.new_stats()
        dl64, dv64 = torch.zeros_like(d_len), torch.zeros_like(d_vel)
        pp64 = S.prop_params(S.FP64, w.gamma, w.d_t)
        S.sfhk_dipole(field, target, sb, len(sb), pp64, dl64, dv64, st64, stream)   # warm-up
        st64.zero_()
        a, b = ev(), ev()
        a.record(stream)
        S.sfhk_dipole(field, target, sb, len(sb), pp64, dl64, dv64, st64, stream)
        b.record(stream)
        torch.cuda.synchronize()
        s64 = S.stats_dict(st64)["traj_steps"]
        v64 = s64 / (a.elapsed_time(b) / 1e3)
        f64_flops = flops_per_traj_step(w.target.pot, planar=True, compensated=False)
        peak64 = 2 * FP64_LANES_PER_SM * SM_COUNT * SM_MAX_MHZ * 1e6 / 1e12
        fp64 = {"value": v64, "unit": UNIT,
                "sample": f"every {stride}th birth ({len(sb)} births), propagation+dipole kernel only",
                "dtype": "f64", "flops_per_traj_step": f64_flops, "achieved_tflops": v64 * f64_flops / 1e12,
                "peak_tflops": peak64, "frac": v64 * f64_flops / 1e12 / peak64,
                "peak_basis": "152 SMs x 2 FP64 lanes x 2 flops x 2070 MHz",
                "mixed_over_fp64": None}

    # --- run record (--record): symplecticity of a sampled subset and errors against the FP64 path
    record = None
    if rank == 0 and args.record:
        record = run_record(w, field, target, births, info, pp, prec, omega, stream)

    # --- measured FMA peaks -------------------------------------------------
    peaks = None
    if rank == 0 and not args.no_peaks:
        f32, _ = S.sfhk_peak_flops(0)
        f64, _ = S.sfhk_peak_flops(1)
        peaks = {"fp32_fma_tflops": f32, "fp64_fma_tflops": f64}

    if rank == 0:
        kms = statistics.mean(kern_ms)
        peak32 = 2 * FP32_LANES_PER_SM * SM_COUNT * SM_MAX_MHZ * 1e6 / 1e12
        peak64 = 2 * FP64_LANES_PER_SM * SM_COUNT * SM_MAX_MHZ * 1e6 / 1e12
        f64_fps = flops_per_traj_step(w.target.pot, planar=True, compensated=False)
        have_ph = all(p["phases"] for p in phases)
        traj_ms = statistics.mean(p["traj_ms"] for p in phases) if have_ph else None
        redo_ms = statistics.mean(p["redo_ms"] for p in phases) if have_ph else None
        roof_float = roof_redo = None
        if prec == S.MIXED and have_ph:
            # the float pass of the live call: every trajectory-step except the redo's
            # steps from the escalation bin on
            esc_steps = warm_stats["esc_steps"]
            esc_pre = warm_stats["esc_steps_pre"]
            float_steps = steps_per_launch - (esc_steps - esc_pre)
            fps = flops_per_traj_step(w.target.pot, planar=True, compensated=True)
            ach = fps * float_steps / (traj_ms * 1e-3) / 1e12
            roof_float = {"bound": "alu", "achieved": ach, "peak": peak32, "unit": "TFLOP/s", "frac": ach / peak32,
                          "traffic": (FLOAT_PASS_DRAM_BYTES_PER_BIRTH * w.n
                                      if FLOAT_PASS_DRAM_BYTES_PER_BIRTH is not None else None),
                          "kernel": "traj_kernel<float,SOFTCORE,planar> (float pass of the timed calls)",
                          "kernel_ms": traj_ms, "timing": "CUDA events around the launch inside sfhk_dipole "
                                                          "(with the amplitude maximum before it)",
                          "flops_per_traj_step": fps, "traj_steps": float_steps,
                          "flops_per_traj_step_3d_form": flops_per_traj_step(w.target.pot, planar=False),
                          "peak_basis": "152 SMs x 128 FP32 lanes x 2 flops x 2070 MHz (of nominal; measured FFMA "
                                        "in measured_peaks)"}
            if esc_steps > 0:
                ach = f64_fps * esc_steps / (redo_ms * 1e-3) / 1e12
                roof_redo = {"bound": "alu", "achieved": ach, "peak": peak64, "unit": "TFLOP/s",
                             "frac": ach / peak64,
                             "traffic": REDO_DRAM_BYTES_DEFAULT.get((w.n, pp.esc_ratio, pp.esc_floor,
                                                                     pp.esc_ratio_big, pp.esc_big)),
                             "kernel": "redo_kernel<SOFTCORE> (four-warp FP64 redo of the escalated births)",
                             "kernel_ms": redo_ms, "timing": "CUDA events around the launch inside sfhk_dipole",
                             "flops_per_traj_step": f64_fps, "traj_steps": esc_steps,
                             "traj_steps_before_escalation_bin": esc_pre,
                             "peak_basis": "152 SMs x 2 FP64 lanes x 2 flops x 2070 MHz (of nominal)"}
            roofline = roof_redo if (roof_redo is not None and redo_ms > traj_ms) else roof_float
        elif prec == S.MIXED:
            # overlapped schedules (esc_overlap 0, 1) run the float pass and the redo as
            # several concurrent launches: no one kernel's time to set against its work
            roofline = {"bound": "alu", "achieved": None, "peak": peak32, "unit": "TFLOP/s", "frac": None,
                        "traffic": None, "kernel": "float pass and redo overlapped (esc_overlap %d): not timed "
                                                   "per kernel" % pp.esc_overlap, "kernel_ms": None}
        else:
            ach = f64_fps * steps_per_launch / (kms * 1e-3) / 1e12
            roofline = {"bound": "alu", "achieved": ach, "peak": peak64, "unit": "TFLOP/s", "frac": ach / peak64,
                        "traffic": None, "kernel": "traj_kernel<double,SOFTCORE,planar>", "kernel_ms": kms,
                        "flops_per_traj_step": f64_fps,
                        "peak_basis": "152 SMs x 2 FP64 lanes x 2 flops x 2070 MHz (of nominal)"}
        roofline = dict(roofline, dipole_call_ms=kms)
        if fp64 is not None:
            fp64["mixed_over_fp64"] = value / fp64["value"]
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t_dev / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32/f64-mixed" if prec == S.MIXED else "f64",
            "data": "synthetic",
            "config": {"workload": w.name, "births_per_gpu": w.n, "precision": args.precision,
                       "trajectory_steps_per_step": steps_per_launch * world, "block": args.block or 128,
                       "escalated_per_step": warm_stats["escalated"], "removed_per_step": warm_stats["removed"],
                       "esc_ratio": pp.esc_ratio, "esc_floor": pp.esc_floor,
                       "esc_steps_per_step": warm_stats.get("esc_steps", 0),
                       "esc_steps_before_escalation_bin": warm_stats.get("esc_steps_pre", 0),
                       "esc_overlap": pp.esc_overlap, "esc_precision": pp.esc_precision,
                       "chunk_steps": args.chunk or 1000, "l2": "flushed between steps (256 MiB write)",
                       "parallelism": f"replicas x{world}, bins summed"},
            "spectra_per_s": 2 * world * args.steps / t_dev,
            "roofline": roofline,
            "roofline_float_pass": roof_float,
            "roofline_fp64_redo": roof_redo,
            "phase_ms": ({k: statistics.mean(p[k] for p in phases) for k in ("traj_ms", "compact_ms", "redo_ms",
                                                                          "total_ms")} if phases else None),
            "measured_peaks": peaks,
            "fp64_path": fp64,
            "e2e": e2e,
            "gpu_launches": launches_per_step(w.n, info["n_steps"], args.chunk or 1000, prec,
                                              pp.esc_floor > 0.0, pp.esc_overlap,
                                              esc_precision=pp.esc_precision) * args.steps,
            "clocks": clk,
            "wall_s": wall,
        }
        if not args.no_cpu:
            line["cpu_baseline"] = cpu_baseline(w, args.ref_stride)
        print(json.dumps(line))
        if record is not None:
            record.update({"time": time.strftime("%Y-%m-%dT%H:%M:%SZ", time.gmtime()), "workload": w.name,
                           "precision": args.precision, "trajectory_steps_per_s": value,
                           "spectra_per_s": line["spectra_per_s"], "ms_per_step": line["ms_per_step"],
                           "removed_fraction": warm_stats["removed"] / w.n,
                           "escalated_fraction": warm_stats["escalated"] / w.n,
                           "roofline_frac": {"redo": (roof_redo or {}).get("frac"),
                                             "float_pass": (roof_float or {}).get("frac")},
                           "clocks": clk})
            with open(args.record, "a") as fh:
                fh.write(json.dumps(record) + "\n")
    if world > 1:
        dist.destroy_process_group()
    return 0


def sweep_arm(args):
    """Batched uneven sweep: 64 laser configurations (H or Ar) with 1e4..1e6 births each in
    one persistent launch (sfhk_batch), births and spectra of every configuration around it;
    the whole step optionally captured once in a CUDA graph and replayed."""
    import torch

    from paper_2601_17164_gb300 import pipeline as PL
    from paper_2601_17164_gb300 import sfhk as S

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    ws = W.batched_sweep(n_cfg=args.sweep_configs, seed=4, n_lo=1e4, n_hi=1e6, dt=0.01)
    prec = S.MIXED if args.precision == "mixed" else S.FP64
    stream = torch.cuda.Stream()
    hs, bs, dls, dvs, oms, outs = [], [], [], [], [], []
    for w in ws:
        f, t = PL.make_handles(w)
        nb = f.info["n_bins"]
        hs.append((f, t))
        bs.append(S.Births.empty(w.n))
        dls.append(torch.zeros(nb, dtype=torch.float64, device="cuda"))
        dvs.append(torch.zeros(nb, dtype=torch.float64, device="cuda"))
        om = torch.tensor(W.omega_grid(w), dtype=torch.float64, device="cuda")
        oms.append(om)
        outs.append([torch.empty_like(om) for _ in range(4)])
    stats = S.new_stats()
    pp = S.prop_params(prec, 0.5, 1e30, esc_ratio=args.esc_ratio, esc_floor=args.esc_floor,
                       esc_precision=args.esc_precision)
    batch = S.Batch([h[0] for h in hs], [h[1] for h in hs], bs, [w.n for w in ws], pp, dls, dvs, stats)

    def step():
        for d in dls + dvs:
            d.zero_()
        stats.zero_()
        for w, (f, t), b in zip(ws, hs, bs):
            S.sfhk_sample_births(f, t, w.birth_mode, w.n, b, w.n_t, w.n_k, w.sigma, w.kmax, w.seed, stream)
        batch.run(stream)
        for (f, _), dl, dv, om, X in zip(hs, dls, dvs, oms, outs):
            info = f.info
            dto, tau = info["dt"] * info["n_out"], 0.5 * info["Tp"]
            S.sfhk_spectrum(dl, info["t_start"], dto, tau, om, X[0], X[1], stream)
            S.sfhk_spectrum(dv, info["t_start"], dto, tau, om, X[2], X[3], stream)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step()
    torch.cuda.synchronize()
    steps_per = S.stats_dict(stats)["traj_steps"]
    esc = S.stats_dict(stats)["escalated"]
    graph = None
    if args.graph:
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.stream(stream):
            with torch.cuda.graph(graph, stream=stream):
                step()
        torch.cuda.synchronize()
    clocks = Clocks(int(os.environ.get("LOCAL_RANK", "0")))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    times = []
    clocks.start()
    for _ in range(args.steps):
        with torch.cuda.stream(stream):
            flush.fill_(1.0)
            e0.record(stream)
            if graph is not None:
                graph.replay()
            else:
                step()
            e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1) / 1e3)
    clk = clocks.stop()
    t_dev = sum(times)
    line = {"metric": METRIC, "value": steps_per * args.steps / t_dev, "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_dev / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32/f64-mixed" if prec == S.MIXED else "f64", "data": "synthetic",
            "config": {"workload": f"batched sweep: {len(ws)} configurations (H/Ar, 800-2000 nm, 2-10 cycles, "
                                   f"0.5-3e14 W/cm^2, 1e4-1e6 births log-uniform), one persistent launch",
                       "births_per_step": sum(w.n for w in ws), "trajectory_steps_per_step": steps_per,
                       "escalated_per_step": esc, "cuda_graph": bool(graph is not None),
                       "l2": "flushed between steps (256 MiB write)", "parallelism": "1 GPU"},
            "spectra_per_s": 2 * len(ws) * args.steps / t_dev, "clocks": clk}
    print(json.dumps(line))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--block", type=int, default=0)
    ap.add_argument("--chunk", type=int, default=0)
    ap.add_argument("--ref-stride", type=int, default=500)
    ap.add_argument("--fp64-stride", type=int, default=16)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-peaks", action="store_true")
    ap.add_argument("--births", type=int, default=0, help="births per GPU (default: the workload's 1e6)")
    ap.add_argument("--esc-ratio", type=float, default=None, help="mixed-path escalation threshold (0: off)")
    ap.add_argument("--esc-floor", type=float, default=None, help="escalation amplitude floor")
    ap.add_argument("--esc-overlap", type=int, default=2, choices=[0, 1, 2],
                    help="escalation schedule: 0 birth chunks, 1 time segments, 2 sequential")
    ap.add_argument("--esc-precision", type=int, default=0, choices=[0, 1, 2],
                    help="escalation redo: 0 FP64 (four-warp kernel), 1 double-float, 2 FP64 one thread per trajectory")
    ap.add_argument("--workload", default="h800", choices=["h800", "sweep"],
                    help="h800: H 800 nm 8 cycles 1e6 births (default); sweep: the batched 64-configuration sweep")
    ap.add_argument("--sweep-configs", type=int, default=64)
    ap.add_argument("--graph", action="store_true", help="sweep: capture one step in a CUDA graph and replay it")
    ap.add_argument("--record", default="", help="append a JSON-lines run record (counters, det M check, errors "
                                                 "against the FP64 path) to this file")
    args = ap.parse_args()
    if args.impl == "reference":
        return reference_arm(args)
    if args.workload == "sweep":
        return sweep_arm(args)
    return gpu_arm(args)


if __name__ == "__main__":
    sys.exit(main())
