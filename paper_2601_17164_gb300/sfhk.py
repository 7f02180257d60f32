"""Python binding of the SFHK C ABI (``include/sfhk.h``).

Argument marshalling only: every step of the trajectory path runs in the CUDA
library ``_build/libsfhk.so``.  Torch tensors supply device memory and
streams.  If the library cannot be built or loaded this module raises; there
is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import threading
from dataclasses import dataclass
from typing import Optional

import torch

from . import build as _build

SFHK_OK = 0
_STATUS = {0: "SFHK_OK", 1: "SFHK_EINVAL", 2: "SFHK_ENOMEM", 3: "SFHK_ECUDA", 4: "SFHK_ETIMEOUT",
           5: "SFHK_ENUMERIC", 6: "SFHK_EUNSUPPORTED"}
FP64, MIXED, DF = 0, 1, 2
BIRTH_GRID, BIRTH_UNIFORM_GAUSS = 0, 1


class SfhkError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


class Pulse(C.Structure):
    _fields_ = [("intensity_wcm2", C.c_double), ("lambda_nm", C.c_double), ("cycles", C.c_double),
                ("cep_rad", C.c_double), ("envelope", C.c_int32), ("reserved", C.c_int32)]


class FieldInfo(C.Structure):
    _fields_ = [("E0", C.c_double), ("omega", C.c_double), ("Tp", C.c_double), ("t_start", C.c_double),
                ("dt", C.c_double), ("t_out", C.c_double), ("n_steps", C.c_int64), ("n_out", C.c_int64),
                ("n_bins", C.c_int64)]


class TargetDesc(C.Structure):
    _fields_ = [("potential", C.c_int32), ("gto_l", C.c_int32), ("n_gto", C.c_int32), ("amp", C.c_int32),
                ("pot_param", C.c_double * 8), ("ip", C.c_double), ("gto_c", C.POINTER(C.c_double)),
                ("gto_alpha", C.POINTER(C.c_double))]


class BirthParams(C.Structure):
    _fields_ = [("n", C.c_int64), ("mode", C.c_int32), ("n_t", C.c_int32), ("n_k", C.c_int32),
                ("reserved", C.c_int32), ("sigma_k", C.c_double), ("kmax", C.c_double), ("seed", C.c_uint64),
                ("first", C.c_int64), ("count", C.c_int64)]


class BirthsC(C.Structure):
    _fields_ = [("n0", C.c_void_p), ("t0", C.c_void_p), ("p0x", C.c_void_p), ("p0y", C.c_void_p),
                ("p0z", C.c_void_p), ("q0z", C.c_void_p), ("amp_re", C.c_void_p), ("amp_im", C.c_void_p),
                ("q0x", C.c_void_p), ("q0y", C.c_void_p), ("capacity", C.c_int64)]


class PropParams(C.Structure):
    _fields_ = [("precision", C.c_int32), ("deterministic", C.c_int32), ("gamma", C.c_double), ("d_t", C.c_double),
                ("block", C.c_int32), ("chunk_steps", C.c_int32), ("esc_ratio", C.c_double),
                ("geometry", C.c_int32), ("esc_precision", C.c_int32), ("esc_floor", C.c_double),
                ("pw_radius", C.c_double), ("pw_mask", C.c_int32), ("esc_overlap", C.c_int32),
                ("esc_ratio_big", C.c_double), ("esc_big", C.c_double)]


class PhaseTimes(C.Structure):
    _fields_ = [("traj_ms", C.c_float), ("compact_ms", C.c_float), ("redo_ms", C.c_float), ("total_ms", C.c_float),
                ("phases", C.c_int32), ("reserved", C.c_int32)]


class EndpointsC(C.Structure):
    _fields_ = [("state", C.c_void_p), ("c_re", C.c_void_p), ("c_im", C.c_void_p), ("flags", C.c_void_p),
                ("n_end", C.c_int64)]


STATS_FIELDS = ("removed", "nonfinite", "branch_guard", "skipped", "traj_steps", "escalated", "esc_steps",
                "esc_steps_pre")
STATS_WORDS = 8

_lock = threading.Lock()
_lib = None


def lib():
    """Loads (building first if needed) the CUDA library; raises if impossible."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build()
            L = C.CDLL(path)
            vp, i64, dbl = C.c_void_p, C.c_int64, C.c_double
            L.sfhk_last_error.restype = C.c_char_p
            L.sfhk_version.restype = C.c_char_p
            L.sfhk_sync.argtypes = [vp]
            L.sfhk_make_field.argtypes = [C.POINTER(Pulse), dbl, dbl, C.POINTER(vp)]
            L.sfhk_field_get_info.argtypes = [vp, C.POINTER(FieldInfo)]
            L.sfhk_field_destroy.argtypes = [vp]
            L.sfhk_field_destroy.restype = None
            L.sfhk_make_target.argtypes = [C.POINTER(TargetDesc), C.POINTER(vp)]
            L.sfhk_target_destroy.argtypes = [vp]
            L.sfhk_target_destroy.restype = None
            L.sfhk_sample_births.argtypes = [vp, vp, C.POINTER(BirthParams), C.POINTER(BirthsC), vp]
            L.sfhk_propagate.argtypes = [vp, vp, C.POINTER(BirthsC), i64, C.POINTER(PropParams),
                                         C.POINTER(EndpointsC), vp, vp]
            L.sfhk_dipole.argtypes = [vp, vp, C.POINTER(BirthsC), i64, C.POINTER(PropParams), vp, vp, vp, vp]
            L.sfhk_spectrum.argtypes = [vp, i64, dbl, dbl, dbl, vp, i64, vp, vp, vp]
            L.sfhk_dipole_static_scratch.argtypes = L.sfhk_dipole.argtypes
            L.sfhk_gabor.argtypes = [vp, i64, dbl, dbl, dbl, vp, i64, vp, i64, vp, vp, vp]
            L.sfhk_emission_time.argtypes = [vp, vp, i64, i64, vp, dbl, dbl, vp, vp, vp]
            L.sfhk_batch_create.argtypes = [C.c_int32, C.POINTER(vp), C.POINTER(vp), C.POINTER(BirthsC),
                                            C.POINTER(C.c_int64), C.POINTER(PropParams), C.POINTER(vp),
                                            C.POINTER(vp), vp, C.POINTER(vp)]
            L.sfhk_batch_run.argtypes = [vp, vp]
            L.sfhk_dipole_batch.argtypes = [C.c_int32, C.POINTER(vp), C.POINTER(vp), C.POINTER(BirthsC),
                                            C.POINTER(C.c_int64), C.POINTER(PropParams), C.POINTER(vp),
                                            C.POINTER(vp), vp, vp]
            L.sfhk_autotune.argtypes = [vp, vp, C.POINTER(BirthsC), i64, C.POINTER(PropParams),
                                        C.POINTER(C.c_int32), C.POINTER(C.c_int32), C.POINTER(C.c_double), vp]
            L.sfhk_batch_destroy.argtypes = [vp]
            L.sfhk_batch_destroy.restype = None
            L.sfhk_peak_flops.argtypes = [C.c_int32, C.POINTER(C.c_double), C.POINTER(C.c_float), vp]
            L.sfhk_resample_births.argtypes = [C.POINTER(BirthsC), i64, i64, C.c_uint64, C.POINTER(BirthsC), vp, vp]
            L.sfhk_det_z_planar_f32.argtypes = [vp, i64, vp, vp, vp, vp]
            L.sfhk_set_phase_timing.argtypes = [C.c_int32]
            L.sfhk_get_phase_times.argtypes = [C.POINTER(PhaseTimes)]
            for name in ("sfhk_peak_flops", "sfhk_sync", "sfhk_make_field", "sfhk_field_get_info", "sfhk_make_target",
                         "sfhk_sample_births", "sfhk_propagate", "sfhk_dipole", "sfhk_spectrum",
                         "sfhk_dipole_static_scratch", "sfhk_batch_create", "sfhk_batch_run", "sfhk_autotune",
                         "sfhk_gabor", "sfhk_emission_time", "sfhk_resample_births", "sfhk_dipole_batch",
                         "sfhk_set_phase_timing", "sfhk_get_phase_times", "sfhk_det_z_planar_f32"):
                getattr(L, name).restype = C.c_int
            _lib = L
    return _lib


def library_path() -> str:
    return _build.LIB


def _check(status: int):
    if status != SFHK_OK:
        raise SfhkError(status, lib().sfhk_last_error().decode())


def _stream_ptr(stream: Optional[torch.cuda.Stream]) -> Optional[int]:
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def _ptr(t: Optional[torch.Tensor]) -> Optional[int]:
    return None if t is None else t.data_ptr()


def sfhk_last_error() -> str:
    return lib().sfhk_last_error().decode()


def sfhk_version() -> str:
    return lib().sfhk_version().decode()


def sfhk_peak_flops(kind: int, stream=None):
    """Measured FMA throughput (TFLOP/s, ms) of the current device: kind 0 FP32, 1 FP64."""
    tf, ms = C.c_double(), C.c_float()
    _check(lib().sfhk_peak_flops(int(kind), C.byref(tf), C.byref(ms), _stream_ptr(stream)))
    return tf.value, ms.value


def sfhk_set_phase_timing(on: bool):
    """Enables (or disables) the per-launch CUDA-event timing inside sfhk_dipole."""
    _check(lib().sfhk_set_phase_timing(1 if on else 0))


def sfhk_get_phase_times() -> dict:
    """Device times (ms) of the phases of the last timed sfhk_dipole call on the current device."""
    t = PhaseTimes()
    _check(lib().sfhk_get_phase_times(C.byref(t)))
    return {k: getattr(t, k) for k, _ in PhaseTimes._fields_ if k != "reserved"}


def sfhk_sync(stream=None):
    _check(lib().sfhk_sync(_stream_ptr(stream)))


class Field:
    """Owns an sfhk_field handle (current CUDA device)."""

    def __init__(self, intensity_wcm2, lambda_nm, cycles, cep=0.0, dt=0.01, t_out=0.1):
        h = C.c_void_p()
        p = Pulse(float(intensity_wcm2), float(lambda_nm), float(cycles), float(cep), 0, 0)
        _check(lib().sfhk_make_field(C.byref(p), float(dt), float(t_out), C.byref(h)))
        self.handle = h
        info = FieldInfo()
        _check(lib().sfhk_field_get_info(h, C.byref(info)))
        self.info = {k: getattr(info, k) for k, _ in FieldInfo._fields_}

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.sfhk_field_destroy(self.handle)
            self.handle = None


def sfhk_make_field(intensity_wcm2, lambda_nm, cycles, cep=0.0, dt=0.01, t_out=0.1) -> Field:
    return Field(intensity_wcm2, lambda_nm, cycles, cep, dt, t_out)


class Target:
    def __init__(self, potential, pot_param, ip, gto_l, c, alpha, amp=0):
        d = TargetDesc()
        d.potential = int(potential)
        d.gto_l = int(gto_l)
        d.n_gto = len(c)
        d.amp = int(amp)
        for i, v in enumerate(pot_param):
            d.pot_param[i] = float(v)
        d.ip = float(ip)
        self._c = (C.c_double * len(c))(*map(float, c))
        self._a = (C.c_double * len(alpha))(*map(float, alpha))
        d.gto_c = C.cast(self._c, C.POINTER(C.c_double))
        d.gto_alpha = C.cast(self._a, C.POINTER(C.c_double))
        h = C.c_void_p()
        _check(lib().sfhk_make_target(C.byref(d), C.byref(h)))
        self.handle = h

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.sfhk_target_destroy(self.handle)
            self.handle = None


def sfhk_make_target(potential, pot_param, ip, gto_l, c, alpha, amp=0) -> Target:
    return Target(potential, pot_param, ip, gto_l, c, alpha, amp)


@dataclass
class Births:
    """Device SoA of births (torch tensors on one CUDA device)."""
    n0: torch.Tensor
    t0: torch.Tensor
    p0x: torch.Tensor
    p0y: torch.Tensor
    p0z: torch.Tensor
    q0z: torch.Tensor
    amp_re: torch.Tensor
    amp_im: torch.Tensor
    q0x: Optional[torch.Tensor] = None
    q0y: Optional[torch.Tensor] = None

    @staticmethod
    def empty(n: int, device="cuda") -> "Births":
        f = lambda: torch.zeros(n, dtype=torch.float64, device=device)
        return Births(torch.zeros(n, dtype=torch.int32, device=device), f(), f(), f(), f(), f(), f(), f())

    def __len__(self):
        return self.n0.numel()

    def c(self) -> BirthsC:
        return BirthsC(_ptr(self.n0), _ptr(self.t0), _ptr(self.p0x), _ptr(self.p0y), _ptr(self.p0z), _ptr(self.q0z),
                       _ptr(self.amp_re), _ptr(self.amp_im), _ptr(self.q0x), _ptr(self.q0y), len(self))

    def slice(self, a: int, b: int) -> "Births":
        g = lambda t: None if t is None else t[a:b]
        return Births(*(g(getattr(self, k)) for k in ("n0", "t0", "p0x", "p0y", "p0z", "q0z", "amp_re", "amp_im",
                                                         "q0x", "q0y")))


def sfhk_sample_births(field: Field, target: Target, mode: int, n: int, births: Births, n_t=0, n_k=0, sigma_k=0.0,
                       kmax=0.0, seed=1, stream=None, first=0, count=0):
    """Births first .. first+count-1 (count 0: to the end) of an n-birth sample into `births`."""
    p = BirthParams(int(n), int(mode), int(n_t), int(n_k), 0, float(sigma_k), float(kmax), int(seed), int(first),
                    int(count))
    bc = births.c()
    _check(lib().sfhk_sample_births(field.handle, target.handle, C.byref(p), C.byref(bc), _stream_ptr(stream)))


def sfhk_resample_births(pool: Births, m: int, n: int, seed: int, out: Births,
                         n_distinct: Optional[torch.Tensor] = None, stream=None):
    """Systematic |I0| resampling of the first m pool births to n births in `out`
    (App. A importance sampling); n_distinct (device int64, optional) receives the
    number of distinct births drawn."""
    pc, oc = pool.c(), out.c()
    _check(lib().sfhk_resample_births(C.byref(pc), int(m), int(n), int(seed), C.byref(oc), _ptr(n_distinct),
                                      _stream_ptr(stream)))


# Escalation defaults of the mixed path: growth ratio 200 above free spreading, amplitude
# floor 1e-2 of the largest birth amplitude, and growth ratio 40 for the few contributions
# with |amp| |C| >= 1000 max|amp| (those that carry a large part of a small sample's signal).
# Floors 1e-3 and 1e-2 give the same plateau errors against FP64 (H 8 cycles and Ar 1600 nm
# at 1e6 births, Ar 2000 nm 20 cycles at 65536) and 1e-2 escalates 7 % fewer H births whose
# redo is 9 % shorter; 3e-2 moves the Ar 1600 nm phases.  Growth ratios 150 and 200 keep
# five 1e6-birth H samples within 1.1e-4 (yields) / 2.4e-4 rad of FP64 and the 4096-birth
# H sample within 2.7e-5 of the oracle; 250 puts the latter at 6.1e-4.
ESC_RATIO = 200.0
ESC_FLOOR = 1e-2
ESC_RATIO_BIG = 40.0
ESC_BIG = 1000.0


def prop_params(precision=FP64, gamma=0.5, d_t=1e30, deterministic=0, block=0, chunk_steps=0,
                esc_ratio=None, geometry=0, esc_precision=0, esc_floor=None, pw_mask=0,
                pw_radius=3.0, esc_overlap=2, esc_ratio_big=None, esc_big=None) -> PropParams:
    """esc_ratio / esc_floor / esc_ratio_big / esc_big default to the ESC_* values for the mixed
    path (escalation on) and 0 for FP64; geometry 0 = planar form where it applies, 1 = full 3D."""
    mixed = precision == MIXED
    if esc_ratio is None:
        esc_ratio = ESC_RATIO if mixed else 0.0
    if esc_floor is None:
        esc_floor = ESC_FLOOR if mixed else 0.0
    if esc_ratio_big is None:
        esc_ratio_big = ESC_RATIO_BIG if mixed else 0.0
    if esc_big is None:
        esc_big = ESC_BIG if mixed else 0.0
    return PropParams(int(precision), int(deterministic), float(gamma), float(d_t), int(block), int(chunk_steps),
                      float(esc_ratio), int(geometry), int(esc_precision), float(esc_floor), float(pw_radius),
                      int(pw_mask), int(esc_overlap), float(esc_ratio_big), float(esc_big))


def new_stats(device="cuda") -> torch.Tensor:
    return torch.zeros(STATS_WORDS, dtype=torch.int64, device=device)


def stats_dict(stats: torch.Tensor) -> dict:
    v = stats.cpu().tolist()
    return {k: v[i] for i, k in enumerate(STATS_FIELDS)}


def sfhk_propagate(field: Field, target: Target, births: Births, n: int, params: PropParams, n_end: int,
                   stats: Optional[torch.Tensor] = None, stream=None):
    dev = births.n0.device
    state = torch.empty((43, n), dtype=torch.float64, device=dev)
    c_re = torch.empty(n, dtype=torch.float64, device=dev)
    c_im = torch.empty(n, dtype=torch.float64, device=dev)
    flags = torch.empty(n, dtype=torch.uint8, device=dev)
    ep = EndpointsC(_ptr(state), _ptr(c_re), _ptr(c_im), _ptr(flags), int(n_end))
    bc = births.c()
    _check(lib().sfhk_propagate(field.handle, target.handle, C.byref(bc), int(n), C.byref(params), C.byref(ep),
                                _ptr(stats), _stream_ptr(stream)))
    return state, torch.complex(c_re, c_im), flags


def sfhk_dipole(field: Field, target: Target, births: Births, n: int, params: PropParams, d_len: torch.Tensor,
                d_vel: torch.Tensor, stats: Optional[torch.Tensor] = None, stream=None):
    bc = births.c()
    _check(lib().sfhk_dipole(field.handle, target.handle, C.byref(bc), int(n), C.byref(params), _ptr(d_len),
                             _ptr(d_vel), _ptr(stats), _stream_ptr(stream)))


def sfhk_dipole_static_scratch(field: Field, target: Target, births: Births, n: int, params: PropParams,
                               d_len: torch.Tensor, d_vel: torch.Tensor, stats: Optional[torch.Tensor] = None,
                               stream=None):
    """Deterministic dipole without any device allocation (library-static 8 MiB scratch)."""
    bc = births.c()
    _check(lib().sfhk_dipole_static_scratch(field.handle, target.handle, C.byref(bc), int(n), C.byref(params),
                                            _ptr(d_len), _ptr(d_vel), _ptr(stats), _stream_ptr(stream)))


def sfhk_autotune(field: Field, target: Target, births: Births, n_sample: int, params: PropParams, stream=None):
    """Times launch shapes on a sample; returns (block, chunk_steps, ms) and caches the choice."""
    bb, bc, ms = C.c_int32(), C.c_int32(), C.c_double()
    bcs = births.c()
    _check(lib().sfhk_autotune(field.handle, target.handle, C.byref(bcs), int(n_sample), C.byref(params),
                               C.byref(bb), C.byref(bc), C.byref(ms), _stream_ptr(stream)))
    return bb.value, bc.value, ms.value


class Batch:
    """Owns an sfhk_batch plan over several configurations (see include/sfhk.h)."""

    def __init__(self, fields, targets, births, ns, params: PropParams, d_lens, d_vels, stats=None):
        k = len(fields)
        vp = C.c_void_p
        self._keep = (fields, targets, births, d_lens, d_vels, stats)
        F = (vp * k)(*[f.handle.value for f in fields])
        T = (vp * k)(*[t.handle.value for t in targets])
        B = (BirthsC * k)(*[b.c() for b in births])
        N = (C.c_int64 * k)(*[int(n) for n in ns])
        L = (vp * k)(*[d.data_ptr() for d in d_lens])
        V = (vp * k)(*[d.data_ptr() for d in d_vels])
        h = C.c_void_p()
        _check(lib().sfhk_batch_create(k, F, T, B, N, C.byref(params), L, V, _ptr(stats), C.byref(h)))
        self.handle = h

    def run(self, stream=None):
        _check(lib().sfhk_batch_run(self.handle, _stream_ptr(stream)))

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.sfhk_batch_destroy(self.handle)
            self.handle = None


def sfhk_batch_create(fields, targets, births, ns, params, d_lens, d_vels, stats=None) -> Batch:
    return Batch(fields, targets, births, ns, params, d_lens, d_vels, stats)


def sfhk_batch_run(batch: Batch, stream=None):
    batch.run(stream)


def sfhk_dipole_batch(fields, targets, births, ns, params: PropParams, d_lens, d_vels, stats=None, stream=None):
    """One-shot batched dipole: plan, run on `stream`, wait, free (synchronous)."""
    k = len(fields)
    vp = C.c_void_p
    F = (vp * k)(*[f.handle.value for f in fields])
    T = (vp * k)(*[t.handle.value for t in targets])
    B = (BirthsC * k)(*[b.c() for b in births])
    N = (C.c_int64 * k)(*[int(n) for n in ns])
    L = (vp * k)(*[d.data_ptr() for d in d_lens])
    V = (vp * k)(*[d.data_ptr() for d in d_vels])
    _check(lib().sfhk_dipole_batch(k, F, T, B, N, C.byref(params), L, V, _ptr(stats), _stream_ptr(stream)))


def sfhk_gabor(bins: torch.Tensor, t0: float, dt_out: float, sigma: float, times: torch.Tensor,
               omega: torch.Tensor, out_re: torch.Tensor, out_im: torch.Tensor, stream=None):
    """out_re/out_im: device double[len(times), len(omega)] (row j = time t_j)."""
    if out_re.numel() != times.numel() * omega.numel() or out_im.numel() != out_re.numel():
        raise ValueError("out_re/out_im must hold len(times) * len(omega) values")
    _check(lib().sfhk_gabor(_ptr(bins), bins.numel(), float(t0), float(dt_out), float(sigma), _ptr(times),
                            times.numel(), _ptr(omega), omega.numel(), _ptr(out_re), _ptr(out_im),
                            _stream_ptr(stream)))


def sfhk_emission_time(g_re: torch.Tensor, g_im: torch.Tensor, times: torch.Tensor, t_a: float, t_b: float,
                       centroid: torch.Tensor, peak: torch.Tensor, stream=None):
    n_t = times.numel()
    n_w = centroid.numel()
    if g_re.numel() != n_t * n_w or g_im.numel() != n_t * n_w or peak.numel() != n_w:
        raise ValueError("inconsistent sizes")
    _check(lib().sfhk_emission_time(_ptr(g_re), _ptr(g_im), n_t, n_w, _ptr(times), float(t_a), float(t_b),
                                    _ptr(centroid), _ptr(peak), _stream_ptr(stream)))


def sfhk_det_z_planar_f32(z: torch.Tensor, stream=None):
    """The float pass's planar det Z from float entries z [10, n] (see include/sfhk.h);
    returns (re, im, e) with det Z = (re + i im) 2^(2e)."""
    if z.dtype != torch.float32 or z.dim() != 2 or z.shape[0] != 10 or not z.is_contiguous():
        raise ValueError("z must be a contiguous float32 tensor of shape [10, n]")
    n = z.shape[1]
    re = torch.empty(n, dtype=torch.float64, device=z.device)
    im = torch.empty_like(re)
    e = torch.empty(n, dtype=torch.int32, device=z.device)
    _check(lib().sfhk_det_z_planar_f32(_ptr(z), n, _ptr(re), _ptr(im), _ptr(e), _stream_ptr(stream)))
    return re, im, e


def sfhk_spectrum(bins: torch.Tensor, t0: float, dt_out: float, tau_h: float, omega: torch.Tensor,
                  out_re: torch.Tensor, out_im: torch.Tensor, stream=None):
    _check(lib().sfhk_spectrum(_ptr(bins), bins.numel(), float(t0), float(dt_out), float(tau_h), _ptr(omega),
                               omega.numel(), _ptr(out_re), _ptr(out_im), _stream_ptr(stream)))
