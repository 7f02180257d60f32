"""Seeded synthetic workloads shaped like the paper's runs.

This module holds input recipes only: laser parameters, target parameters,
GTO coefficients (fitted by ``gto_fit.py``), proposal widths and seeds.  It
contains none of the trajectory arithmetic and is shared by the CUDA path,
the oracle-based tests and the benchmark.

The paper's hydrogen runs (Sec. III.A) use 800-1600 nm, 1e14 W/cm^2, few-cycle
sin^2 pulses, gamma = 0.5, D_t = 1e30 and 2-20 million trajectories; the argon
run (Sec. III.B) uses 1200 nm, 1.2e14 W/cm^2, 6 cycles and ~20 million
trajectories.  The workloads below keep those shapes.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace
from typing import List

HARTREE_EV = 27.211386
AU_INTENSITY_WCM2 = 3.50944758e16

# --- targets -----------------------------------------------------------------
H_ALPHA = [0.05 * 3.0 ** j for j in range(8)]
H_C = [0.006051431287859099, 0.08330118536846186, 0.1519997395775271, 0.12219083127367794,
       0.08500649039358171, 0.04570168041822804, 0.030514392613697486, 0.0211036335333716]
AR_ALPHA = [0.04 * 2.2 ** j for j in range(14)]
AR_C = [5.4268460107496736e-05, 0.0054367599531044974, 0.05487784490675948, 0.20472978115721185,
        0.41816649222591573, 0.19095733939751797, -1.16713989458534, -3.0029149542320557,
        -4.43832953781788, -4.674254675370149, -4.137893608821666, -3.1104565776647983,
        -2.0583002284504284, -2.316239313570728]
TONGLIN_AR = [1.0, 16.039, 2.007, -25.543, 4.525, 0.961, 0.443]

POT_ZERO, POT_SOFTCORE, POT_TONGLIN, POT_HARMONIC = 0, 1, 2, 3
BIRTH_GRID, BIRTH_UNIFORM_GAUSS = 0, 1
AMP_STD_SPA, AMP_MOD_SPA, AMP_ADK = 0, 1, 2


@dataclass(frozen=True)
class Target:
    name: str
    pot: int
    pot_param: tuple
    ip: float
    gto_l: int
    c: tuple
    alpha: tuple
    amp_kind: int = AMP_STD_SPA


HYDROGEN = Target("H(softcore a=0.3)", POT_SOFTCORE, (0.3,), 0.5, 0, tuple(H_C), tuple(H_ALPHA))
ARGON = Target("Ar(Tong-Lin)", POT_TONGLIN, tuple(TONGLIN_AR), 15.76 / HARTREE_EV, 1, tuple(AR_C),
               tuple(AR_ALPHA))


@dataclass(frozen=True)
class Pulse:
    intensity_wcm2: float
    lambda_nm: float
    cycles: float
    cep: float = 0.0


@dataclass(frozen=True)
class Workload:
    name: str
    target: Target
    pulse: Pulse
    dt: float
    t_out: float = 0.1
    gamma: float = 0.5
    d_t: float = 1e30
    birth_mode: int = BIRTH_UNIFORM_GAUSS
    n: int = 1024
    n_t: int = 32
    n_k: int = 32
    sigma: float = 0.0
    kmax: float = 0.0
    seed: int = 1
    h_max: int = 60            # spectrum up to h_max harmonics
    per_harmonic: int = 20     # spectrum points per harmonic
    chunk: int = 0             # births per streamed chunk (0: one chunk)

    def with_n(self, n: int) -> "Workload":
        return replace(self, n=int(n))


def adk_sigma(intensity_wcm2: float, ip: float) -> float:
    """ADK transverse-momentum width sqrt(E0 / (2 sqrt(2 Ip))) used as the proposal sigma."""
    E0 = math.sqrt(intensity_wcm2 / AU_INTENSITY_WCM2)
    return math.sqrt(E0 / (2.0 * math.sqrt(2.0 * ip)))


def _h(name, pulse, **kw):
    return Workload(name, HYDROGEN, pulse, **kw)


# 1: H, 800 nm, 2 cycles, 1e14, 32 x 32 grid births, FP64.
P1 = Pulse(1e14, 800.0, 2.0)
H_800_2CYC_GRID = _h("H 800nm 2cyc 1e14 32x32 grid dt=0.02", P1, dt=0.02, birth_mode=BIRTH_GRID, n=1024,
                     n_t=32, n_k=32, kmax=4.0 * adk_sigma(1e14, 0.5), seed=1, h_max=40)

# 2: H, 800 nm, 8 cycles, 1.5e14, 1e6 births uniform in t0, gaussian k_perp.
P2 = Pulse(1.5e14, 800.0, 8.0)
H_800_8CYC_1M = _h("H 800nm 8cyc 1.5e14 1e6 births dt=0.01", P2, dt=0.01, n=1_000_000,
                   sigma=adk_sigma(1.5e14, 0.5), seed=2, h_max=60)

# 3: Ar Tong-Lin, 1600 nm, 6 cycles, 1e14, 1e7 births.
P3 = Pulse(1e14, 1600.0, 6.0)
AR_1600_6CYC_10M = Workload("Ar 1600nm 6cyc 1e14 1e7 births dt=0.01", ARGON, P3, dt=0.01, n=10_000_000,
                            sigma=adk_sigma(1e14, 15.76 / HARTREE_EV), seed=3, h_max=120)

# 5: Ar, 2000 nm, 20 cycles, 8e13, 1e8 births streamed in chunks of 2^22.
P5 = Pulse(8e13, 2000.0, 20.0)
AR_2000_20CYC_100M = Workload("Ar 2000nm 20cyc 8e13 1e8 births dt=0.01", ARGON, P5, dt=0.01,
                              n=100_000_000, sigma=adk_sigma(8e13, 15.76 / HARTREE_EV), seed=5,
                              h_max=300, chunk=1 << 22)

# Paper-shaped extra run (Fig. 1 shape): H, 1600 nm, 3 cycles, 1e14, 2e6 births.
H_1600_3CYC_2M = _h("H 1600nm 3cyc 1e14 2e6 births dt=0.02", Pulse(1e14, 1600.0, 3.0), dt=0.02,
                    n=2_000_000, sigma=adk_sigma(1e14, 0.5), seed=6, h_max=80)


def batched_sweep(n_cfg: int = 64, seed: int = 4, n_lo: float = 1e4, n_hi: float = 1e6,
                  dt: float = 0.01) -> List[Workload]:
    """4: uneven sweep. I ~ U[0.5,3]e14, lambda ~ U[800,2000] nm, CEP ~ U[0,2pi),
    cycles ~ U{2..10}, counts log-uniform on [n_lo, n_hi], target H or Ar with p = 1/2.
    Drawn with Python's Mersenne Twister from `seed` (input recipe only)."""
    import random
    rng = random.Random(seed)
    out = []
    for i in range(n_cfg):
        I0 = rng.uniform(0.5e14, 3e14)
        lam = rng.uniform(800.0, 2000.0)
        cep = rng.uniform(0.0, 2.0 * math.pi)
        cyc = rng.randint(2, 10)
        n = int(round(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))))
        tgt = HYDROGEN if rng.random() < 0.5 else ARGON
        out.append(Workload(f"sweep[{i}] {tgt.name} {lam:.0f}nm {cyc}cyc {I0:.2e}", tgt,
                            Pulse(I0, lam, float(cyc), cep), dt=dt, n=n,
                            sigma=adk_sigma(I0, tgt.ip), seed=1000 + i, h_max=40))
    return out


def omega_grid(w: Workload) -> List[float]:
    """Spectrum frequencies: per_harmonic points per harmonic up to h_max harmonics."""
    w0 = 45.5633525 / w.pulse.lambda_nm
    n = w.h_max * w.per_harmonic
    return [(m + 1) * w0 / w.per_harmonic for m in range(n)]
