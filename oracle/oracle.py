"""ctypes binding of the SFHK oracle (``oracle/sfhk_oracle.c``).

Test infrastructure only: loaded by tests, the smoke check and the CPU
baseline of the benchmark.  Every function here marshals arguments; the
arithmetic lives in the C file, which cites the paper section by section.

Parity pinned by tests/test_oracle_*.py except where a function says
otherwise.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sfhk_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libsfhk_oracle.so")
_lock = threading.Lock()
_lib = None

POT_ZERO, POT_SOFTCORE, POT_TONGLIN, POT_HARMONIC = 0, 1, 2, 3
FLAG_REMOVED, FLAG_NONFINITE, FLAG_BRANCH_GUARD = 1, 2, 4


class Pulse(C.Structure):
    _fields_ = [("E0", C.c_double), ("omega", C.c_double), ("Tp", C.c_double), ("cep", C.c_double),
                ("kind", C.c_int32), ("pad", C.c_int32)]


class Target(C.Structure):
    _fields_ = [("pot", C.c_int32), ("gto_l", C.c_int32), ("n_gto", C.c_int32), ("amp_kind", C.c_int32),
                ("pot_param", C.c_double * 8), ("ip", C.c_double), ("c", C.c_double * 32),
                ("alpha", C.c_double * 32)]


class Grid(C.Structure):
    _fields_ = [("t_start", C.c_double), ("dt", C.c_double), ("n_steps", C.c_int64), ("n_out", C.c_int64),
                ("gamma", C.c_double), ("d_t", C.c_double), ("removal_whole", C.c_int32), ("pw_mask", C.c_int32),
                ("pw_radius", C.c_double)]


class BirthOut(C.Structure):
    _fields_ = [("kz", C.c_double), ("qz", C.c_double), ("tt", C.c_double), ("S_re", C.c_double),
                ("S_im", C.c_double), ("amp_re", C.c_double), ("amp_im", C.c_double),
                ("valid", C.c_int32), ("pad", C.c_int32)]


class Stats(C.Structure):
    _fields_ = [("removed", C.c_int64), ("nonfinite", C.c_int64), ("branch_guard", C.c_int64),
                ("traj_steps", C.c_double)]


def build(force: bool = False) -> str:
    """Compile the oracle shared library with gcc (FP64, no FMA contraction)."""
    with _lock:
        if (not force and os.path.exists(_SO)
                and os.path.getmtime(_SO) >= os.path.getmtime(_SRC)):
            return _SO
        os.makedirs(_BUILD, exist_ok=True)
        tmp = _SO + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-shared", "-fPIC",
               "-std=gnu11", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _SO)
        return _SO


def lib():
    global _lib
    if _lib is None:
        path = build()
        L = C.CDLL(path)
        dp = C.POINTER(C.c_double)
        ip32 = C.POINTER(C.c_int32)
        L.or_philox4x64.argtypes = [C.POINTER(C.c_uint64), C.POINTER(C.c_uint64), C.POINTER(C.c_uint64)]
        L.or_E0_from_intensity.restype = C.c_double
        L.or_E0_from_intensity.argtypes = [C.c_double]
        L.or_omega_from_lambda.restype = C.c_double
        L.or_omega_from_lambda.argtypes = [C.c_double]
        L.or_field_eval.argtypes = [C.POINTER(Pulse), C.c_int, C.c_int64, dp, dp, dp, dp]
        L.or_field_E_grid.argtypes = [C.POINTER(Pulse), C.c_int64, dp, dp]
        L.or_tunnel_element.argtypes = [C.POINTER(Target), dp, dp, dp]
        L.or_dipole_elements.argtypes = [C.POINTER(Target), C.c_double, dp, dp, dp]
        L.or_birth.argtypes = [C.POINTER(Pulse), C.POINTER(Target), C.c_int64, dp, dp, dp, C.POINTER(BirthOut)]
        L.or_sample_births.argtypes = [C.POINTER(Pulse), C.POINTER(Target), C.POINTER(Grid), C.c_int32,
                                       C.c_int64, C.c_int32, C.c_int32, C.c_double, C.c_double, C.c_uint64,
                                       ip32, dp, dp, dp, dp, dp, dp, dp]
        L.or_sample_births_at.argtypes = [C.POINTER(Pulse), C.POINTER(Target), C.POINTER(Grid), C.c_int32,
                                          C.c_int64, C.c_int32, C.c_int32, C.c_double, C.c_double, C.c_uint64,
                                          C.POINTER(C.c_int64), C.c_int64, ip32, dp, dp, dp, dp, dp, dp, dp]
        L.or_potential_radial.argtypes = [C.POINTER(Target), C.c_int64, dp, dp]
        L.or_det_Z.argtypes = [dp, C.c_double, dp]
        L.or_propagate.argtypes = [C.POINTER(Pulse), C.POINTER(Target), C.POINTER(Grid), C.c_int64, ip32,
                                   dp, dp, C.c_int64, dp, dp, ip32]
        L.or_trajectory.argtypes = [C.POINTER(Pulse), C.POINTER(Target), C.POINTER(Grid), C.c_int64,
                                    C.c_int64, dp, dp, dp]
        L.or_dipole.argtypes = [C.POINTER(Pulse), C.POINTER(Target), C.POINTER(Grid), C.c_int64, ip32,
                                dp, dp, dp, dp, dp, dp, dp, dp, C.POINTER(Stats)]
        L.or_spectrum.argtypes = [dp, C.c_int64, C.c_double, C.c_double, C.c_double, dp, C.c_int64, dp, dp]
        L.or_adk_rate.restype = C.c_double
        L.or_adk_rate.argtypes = [C.POINTER(Target), C.c_double]
        L.or_adk_density.restype = C.c_double
        L.or_adk_density.argtypes = [C.POINTER(Target), C.c_double, C.c_double]
        L.or_adk_norm2.restype = C.c_double
        L.or_adk_norm2.argtypes = [C.POINTER(Pulse), C.POINTER(Target)]
        L.or_adk_subpeaks.argtypes = [C.POINTER(Pulse), dp]
        L.or_max_threads.restype = C.c_int
        L.or_set_threads.argtypes = [C.c_int]
        _lib = L
    return _lib


def _d(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _i32(a):
    return a.ctypes.data_as(C.POINTER(C.c_int32))


def _f64(x):
    return np.ascontiguousarray(np.asarray(x, dtype=np.float64))


# ----------------------------------------------------------------------------
# records
# ----------------------------------------------------------------------------
def E0_from_intensity(wcm2: float) -> float:
    return lib().or_E0_from_intensity(float(wcm2))


def omega_from_lambda(nm: float) -> float:
    return lib().or_omega_from_lambda(float(nm))


def make_pulse(intensity_wcm2=None, lambda_nm=None, cycles=None, cep=0.0, *, E0=None, omega=None,
               cw=False) -> Pulse:
    """sin^2 pulse of `cycles` optical cycles, zero to zero, centred at t = 0."""
    E0 = E0 if E0 is not None else E0_from_intensity(intensity_wcm2)
    w = omega if omega is not None else omega_from_lambda(lambda_nm)
    Tp = 0.0 if cw else cycles * 2.0 * np.pi / w
    return Pulse(E0, w, Tp, cep, 1 if cw else 0, 0)


def make_target(pot: int, pot_param=(), ip=0.5, gto_l=0, c=(), alpha=(), amp_kind=0) -> Target:
    t = Target()
    t.pot = pot
    t.gto_l = gto_l
    t.n_gto = len(c)
    t.amp_kind = amp_kind
    for i, v in enumerate(pot_param):
        t.pot_param[i] = v
    t.ip = ip
    for i, (cc, aa) in enumerate(zip(c, alpha)):
        t.c[i] = cc
        t.alpha[i] = aa
    return t


def make_grid(t_start, dt, n_steps, n_out, gamma=0.5, d_t=1e30, removal_whole=False, pw_mask=0,
              pw_radius=3.0) -> Grid:
    """pw_mask: partial-wave filter, bit c keeps trajectories whose latest entry into
    r < pw_radius had class c (0 s, 1 p, 2 d, 3 higher); 0 = no filter."""
    return Grid(float(t_start), float(dt), int(n_steps), int(n_out), float(gamma), float(d_t),
                1 if removal_whole else 0, int(pw_mask), float(pw_radius))


def pulse_grid(pulse: Pulse, dt: float, t_out: float, gamma=0.5, d_t=1e30, removal_whole=False, pw_mask=0,
               pw_radius=3.0) -> Grid:
    """Integrator grid t_n = -Tp/2 + n dt, n = 0..ceil(Tp/dt); bins every t_out."""
    n_steps = int(np.ceil(pulse.Tp / dt - 1e-9))
    n_out = int(round(t_out / dt))
    assert abs(n_out * dt - t_out) < 1e-12
    return make_grid(-0.5 * pulse.Tp, dt, n_steps, n_out, gamma, d_t, removal_whole, pw_mask, pw_radius)


# ----------------------------------------------------------------------------
# functions
# ----------------------------------------------------------------------------
def philox4x64(ctr, key):
    c = np.ascontiguousarray(np.asarray(ctr, dtype=np.uint64))
    k = np.ascontiguousarray(np.asarray(key, dtype=np.uint64))
    out = np.zeros(4, dtype=np.uint64)
    u64p = C.POINTER(C.c_uint64)
    lib().or_philox4x64(c.ctypes.data_as(u64p), k.ctypes.data_as(u64p), out.ctypes.data_as(u64p))
    return out


def field(pulse: Pulse, which: str, t):
    """which in {'A','E','F','G'}; t real or complex array (in-pulse expression)."""
    t = np.asarray(t, dtype=np.complex128).ravel()
    tr, ti = _f64(t.real), _f64(t.imag)
    o_r, o_i = np.zeros_like(tr), np.zeros_like(tr)
    lib().or_field_eval(C.byref(pulse), "AEFG".index(which), len(tr), _d(tr), _d(ti), _d(o_r), _d(o_i))
    return o_r + 1j * o_i


def field_E_grid(pulse: Pulse, t):
    t = _f64(t).ravel()
    out = np.zeros_like(t)
    lib().or_field_E_grid(C.byref(pulse), len(t), _d(t), _d(out))
    return out


def tunnel_element(target: Target, k):
    k = np.asarray(k, dtype=np.complex128)
    kr, ki, out = _f64(k.real), _f64(k.imag), np.zeros(2)
    lib().or_tunnel_element(C.byref(target), _d(kr), _d(ki), _d(out))
    return out[0] + 1j * out[1]


def dipole_elements(target: Target, gamma, p, q):
    p, q, out = _f64(p), _f64(q), np.zeros(4)
    lib().or_dipole_elements(C.byref(target), float(gamma), _d(p), _d(q), _d(out))
    return out[0] + 1j * out[1], out[2] + 1j * out[3]


def births_at(pulse: Pulse, target: Target, t0, kx, ky):
    t0, kx, ky = _f64(t0).ravel(), _f64(kx).ravel(), _f64(ky).ravel()
    out = (BirthOut * len(t0))()
    lib().or_birth(C.byref(pulse), C.byref(target), len(t0), _d(t0), _d(kx), _d(ky), out)
    rec = np.ctypeslib.as_array(out)
    return {name: np.array(rec[name]) for name, _ in BirthOut._fields_ if name != "pad"}


def sample_births(pulse: Pulse, target: Target, grid: Grid, mode: int, n: int, n_t=32, n_k=32,
                  sigma=0.0, kmax=0.0, seed=1):
    n = int(n)
    b = {"n0": np.zeros(n, np.int32)}
    for k in ("t0", "px", "py", "pz", "qz", "amp_re", "amp_im"):
        b[k] = np.zeros(n, np.float64)
    lib().or_sample_births(C.byref(pulse), C.byref(target), C.byref(grid), int(mode), n, int(n_t), int(n_k),
                           float(sigma), float(kmax), C.c_uint64(int(seed)), _i32(b["n0"]), _d(b["t0"]),
                           _d(b["px"]), _d(b["py"]), _d(b["pz"]), _d(b["qz"]), _d(b["amp_re"]),
                           _d(b["amp_im"]))
    return b


def sample_births_at(pulse: Pulse, target: Target, grid: Grid, mode: int, n: int, idx, n_t=32, n_k=32,
                     sigma=0.0, kmax=0.0, seed=1):
    """Births number `idx` of an n-birth sample (same values as sample_births)."""
    idx = np.ascontiguousarray(np.asarray(idx, dtype=np.int64).ravel())
    m = len(idx)
    b = {"n0": np.zeros(m, np.int32)}
    for k in ("t0", "px", "py", "pz", "qz", "amp_re", "amp_im"):
        b[k] = np.zeros(m, np.float64)
    lib().or_sample_births_at(C.byref(pulse), C.byref(target), C.byref(grid), int(mode), int(n), int(n_t), int(n_k),
                              float(sigma), float(kmax), C.c_uint64(int(seed)),
                              idx.ctypes.data_as(C.POINTER(C.c_int64)), m, _i32(b["n0"]), _d(b["t0"]),
                              _d(b["px"]), _d(b["py"]), _d(b["pz"]), _d(b["qz"]), _d(b["amp_re"]),
                              _d(b["amp_im"]))
    return b


def potential_radial(target: Target, r):
    r = _f64(r).ravel()
    out = np.zeros(3 * len(r))
    lib().or_potential_radial(C.byref(target), len(r), _d(r), _d(out))
    return out.reshape(-1, 3)


def det_Z(y43, gamma):
    y, out = _f64(y43), np.zeros(2)
    lib().or_det_Z(_d(y), float(gamma), _d(out))
    return out[0] + 1j * out[1]


def propagate(pulse: Pulse, target: Target, grid: Grid, n0, q0, p0, n_end):
    """Endpoints. q0, p0: arrays [3][n]. Returns state [43][n], C [n], flags [n]."""
    n0 = np.ascontiguousarray(np.asarray(n0, dtype=np.int32).ravel())
    n = len(n0)
    q0 = _f64(np.broadcast_to(np.asarray(q0, dtype=np.float64).reshape(3, -1), (3, n)))
    p0 = _f64(np.broadcast_to(np.asarray(p0, dtype=np.float64).reshape(3, -1), (3, n)))
    st = np.zeros((43, n))
    Cc = np.zeros((2, n))
    fl = np.zeros(n, np.int32)
    lib().or_propagate(C.byref(pulse), C.byref(target), C.byref(grid), n, _i32(n0), _d(q0), _d(p0),
                       int(n_end), _d(st), _d(Cc), _i32(fl))
    return st, Cc[0] + 1j * Cc[1], fl


def trajectory(pulse: Pulse, target: Target, grid: Grid, n0, n_end, q0, p0):
    """State [n_end-n0+1][43] at every grid index (no prefactor, no removal)."""
    q0, p0 = _f64(q0), _f64(p0)
    path = np.zeros((int(n_end) - int(n0) + 1, 43))
    lib().or_trajectory(C.byref(pulse), C.byref(target), C.byref(grid), int(n0), int(n_end), _d(q0), _d(p0),
                        _d(path))
    return path


def dipole(pulse: Pulse, target: Target, grid: Grid, births, d_len=None, d_vel=None):
    """Accumulates into d_len, d_vel (allocated zero if None). Returns (d_len, d_vel, stats dict)."""
    nb = grid.n_steps // grid.n_out + 1
    d_len = np.zeros(nb) if d_len is None else d_len
    d_vel = np.zeros(nb) if d_vel is None else d_vel
    b = {k: np.ascontiguousarray(births[k]) for k in ("n0", "px", "py", "pz", "qz", "amp_re", "amp_im")}
    st = Stats()
    lib().or_dipole(C.byref(pulse), C.byref(target), C.byref(grid), len(b["n0"]), _i32(b["n0"]), _d(b["px"]),
                    _d(b["py"]), _d(b["pz"]), _d(b["qz"]), _d(b["amp_re"]), _d(b["amp_im"]), _d(d_len),
                    _d(d_vel), C.byref(st))
    return d_len, d_vel, {"removed": st.removed, "nonfinite": st.nonfinite, "branch_guard": st.branch_guard,
                          "traj_steps": st.traj_steps}


def spectrum(x, t0, dt_out, tau_h, omega):
    x, om = _f64(x), _f64(omega)
    o_r, o_i = np.zeros(len(om)), np.zeros(len(om))
    lib().or_spectrum(_d(x), len(x), float(t0), float(dt_out), float(tau_h), _d(om), len(om), _d(o_r), _d(o_i))
    return o_r + 1j * o_i


def adk_rate(target: Target, F: float) -> float:
    """Static ADK rate w(F) (Sec. III.C reading; without the tail constant C_l^2)."""
    return lib().or_adk_rate(C.byref(target), float(F))


def adk_density(target: Target, F: float, kperp2: float) -> float:
    """ADK rate per unit time and per d^2 k_perp at field strength F."""
    return lib().or_adk_density(C.byref(target), float(F), float(kperp2))


def adk_norm2(pulse: Pulse, target: Target) -> float:
    """Renormalisation N^2 of the ADK births: SFA rate over ADK rate at the two sub-peaks."""
    return lib().or_adk_norm2(C.byref(pulse), C.byref(target))


def adk_subpeaks(pulse: Pulse):
    """The two sub-peak times (carrier crests next to the one nearest the envelope's peak)."""
    out = np.zeros(2)
    lib().or_adk_subpeaks(C.byref(pulse), _d(out))
    return out


def max_threads() -> int:
    return lib().or_max_threads()


def set_threads(n: int) -> None:
    lib().or_set_threads(int(n))
