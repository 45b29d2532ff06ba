"""Seeded synthetic workloads shared by the tests, the bench and the oracle.

This module holds only workload definitions and seeded random numbers: no
arithmetic of the method itself (no grids, stencils, solvers or combination).
Both the CUDA path and the CPU oracle receive the values generated here.

Random numbers come from SplitMix64 (Steele, Lea, Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014): state += 0x9E3779B97F4A7C15,
then two xor-shift-multiply rounds.  Uniform doubles take the top 53 bits;
normals use the Box-Muller transform.

The five workloads restate the heat, Ornstein-Uhlenbeck and variable-
coefficient heat problems on which the method is measured: d-dimensional
parabolic problems (Sec. 2, Eq. "parabolic_problem") on the component grids of
the combination technique at level n (Eq. "combination_technique_solution"),
stepped by backward Euler and solved in time by MGRIT (Sec. 3.3).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, count: int) -> np.ndarray:
    """`count` consecutive SplitMix64 outputs (uint64) from `seed`."""
    with np.errstate(over="ignore"):
        k = np.arange(1, count + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + k * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed: int, count: int) -> np.ndarray:
    """Uniform doubles in [0, 1) from the top 53 bits of SplitMix64."""
    return (splitmix64(seed, count) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def normal(seed: int, count: int) -> np.ndarray:
    """Standard normals by Box-Muller on pairs of uniforms."""
    m = (count + 1) // 2
    u = uniform(seed, 2 * m)
    u1 = 1.0 - u[0::2]  # (0, 1]
    u2 = u[1::2]
    r = np.sqrt(-2.0 * np.log(u1))
    z = np.empty(2 * m)
    z[0::2] = r * np.cos(2.0 * math.pi * u2)
    z[1::2] = r * np.sin(2.0 * math.pi * u2)
    return z[:count]


def random_vector(seed: int, n: int, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    return lo + (hi - lo) * uniform(seed, n)


OP_HEAT, OP_VARHEAT, OP_OU = 0, 1, 2
IC_SINES, IC_GAUSS = 0, 1
PREC_FP64, PREC_MIXED = 0, 1
COARSE_IMPLICIT, COARSE_EXACT, COARSE_LEARNED = 0, 1, 2


@dataclass
class Workload:
    name: str
    d: int
    n: int                     # combination level (the paper's L)
    op: int
    lo: list
    hi: list
    t0: float
    t1: float
    nsteps: int
    m: int                     # MGRIT coarsening factor
    levels: int                # MGRIT levels
    ic_kind: int
    ic_params: np.ndarray
    L0: int = 1
    theta: float = 1.0
    sigma: float = 1.0
    vamp: float = 0.5
    prec: int = PREC_FP64
    coarse: int = COARSE_IMPLICIT
    note: str = ""
    extra: dict = field(default_factory=dict)

    @property
    def dt(self) -> float:
        return (self.t1 - self.t0) / self.nsteps


def sine_modes(d: int, modes) -> np.ndarray:
    """Parameter block of a sum of product-sine modes: [K, (A_k, m_k1..m_kd)...]."""
    out = [float(len(modes))]
    for amp, freqs in modes:
        assert len(freqs) == d
        out.append(float(amp))
        out.extend(float(f) for f in freqs)
    return np.array(out)


def gauss_params(mean, std) -> np.ndarray:
    return np.array(list(mean) + list(std), dtype=np.float64)


def random_sine_modes(d: int, K: int = 8, fmax: int = 4, seed: int = 0) -> np.ndarray:
    """K modes with N(0,1) amplitudes and integer frequencies uniform in 1..fmax."""
    amps = normal(seed, K)
    fr = 1 + np.floor(uniform(seed ^ 0x5DEECE66D, K * d) * fmax).astype(np.int64)
    fr = np.minimum(fr, fmax)
    return sine_modes(d, [(amps[k], fr[k * d:(k + 1) * d].tolist()) for k in range(K)])


def workload(k: int) -> Workload:
    """The five measured workloads (1..5)."""
    if k == 1:
        return Workload("heat2d_n5", 2, 5, OP_HEAT, [0.0] * 2, [1.0] * 2, 0.0, 0.1, 64, 4, 2,
                        IC_SINES, sine_modes(2, [(1.0, [1, 1])]), prec=PREC_FP64,
                        note="d=2 heat, level 5, 64 BE steps on [0,0.1], two-level MGRIT m=4")
    if k == 2:
        return Workload("heat3d_n9", 3, 9, OP_HEAT, [0.0] * 3, [1.0] * 3, 0.0, 0.05, 1024, 16, 2,
                        IC_SINES, sine_modes(3, [(1.0, [1, 1, 1]), (0.1, [3, 3, 3])]),
                        prec=PREC_MIXED,
                        note="d=3 heat, level 9, 1024 BE steps on [0,0.05], two-level MGRIT m=16")
    if k == 3:
        return Workload("ou4d_n7", 4, 7, OP_OU, [-6.0] * 4, [6.0] * 4, 0.0, 1.0, 512, 8, 2,
                        IC_GAUSS, gauss_params([1.0] * 4, [0.5] * 4), prec=PREC_MIXED,
                        note="d=4 Ornstein-Uhlenbeck Fokker-Planck, level 7, 512 steps on [0,1], m=8")
    if k == 4:
        return Workload("varheat3d_n8", 3, 8, OP_VARHEAT, [0.0] * 3, [1.0] * 3, 0.0, 0.1, 2048, 32, 2,
                        IC_SINES, random_sine_modes(3, 8, 4, seed=0), prec=PREC_MIXED,
                        coarse=COARSE_LEARNED,
                        note="d=3 variable-coefficient heat, level 8, 2048 steps on [0,0.1], m=32")
    if k == 5:
        return Workload("heat6d_n10", 6, 10, OP_HEAT, [0.0] * 6, [1.0] * 6, 0.0, 0.02, 512, 16, 3,
                        IC_SINES, sine_modes(6, [(1.0, [1] * 6)]), prec=PREC_MIXED,
                        coarse=COARSE_LEARNED,
                        note="d=6 heat, level 10, 512 steps on [0,0.02], three-level MGRIT m=16")
    raise ValueError(k)


def eval_points(d: int, lo, hi, n_uniform: int = 65536, n_diag: int = 257, seed: int = 1) -> np.ndarray:
    """Evaluation set of the combined solution: seeded uniform points in the
    domain, points on the main diagonal, and the centre."""
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    u = uniform(seed, n_uniform * d).reshape(n_uniform, d)
    pts = [lo + u * (hi - lo)]
    if n_diag > 0:
        t = np.linspace(0.0, 1.0, n_diag)[:, None]
        pts.append(lo + t * (hi - lo))
    pts.append(((lo + hi) / 2.0)[None, :])
    return np.ascontiguousarray(np.concatenate(pts, axis=0))
