"""Seeded synthetic inputs shared by the CUDA path, the oracle and the benchmark.

This module holds no arithmetic of the method itself: it only describes workloads
(lattice dimensions, sample counts, temperature sets, seeds).  Both sides receive the
same doubles for the temperatures, so neither recomputes them.

Temperature sets (Sec. 2.3): the geometric set, a constant ratio between neighbouring
temperatures, T_k = T_min (T_max/T_min)^(k/(n-1)); the inverse-linear set, constant
steps in beta; and the phi-family of Eqs. 6-7, T_i = i^phi T_norm + T_min with
T_norm = (T_max - T_min)/(N_T - 1)^phi.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace
from typing import List, Sequence


def geometric_temps(t_min: float, t_max: float, n: int) -> List[float]:
    """Geometric temperature set (Sec. 2.3): constant ratio between neighbours."""
    if n == 1:
        return [float(t_min)]
    return [t_min * math.pow(t_max / t_min, k / (n - 1)) for k in range(n)]


def inverse_linear_temps(t_min: float, t_max: float, n: int) -> List[float]:
    """Constant steps in inverse temperature (Sec. 2.3)."""
    if n == 1:
        return [float(t_min)]
    b0, b1 = 1.0 / t_min, 1.0 / t_max
    return [1.0 / (b0 + (b1 - b0) * k / (n - 1)) for k in range(n)]


def phi_temps(t_min: float, t_max: float, n: int, phi: float) -> List[float]:
    """The phi-family of Eqs. 6-7."""
    if n == 1:
        return [float(t_min)]
    t_norm = (t_max - t_min) / math.pow(n - 1, phi)
    return [math.pow(i, phi) * t_norm + t_min for i in range(n)]


# The fitted optimum of the phi protocol for the 2D Gaussian EA model (Sec. 2.3, Eqs. 8-9):
# phi*(L) = 0.406 + 0.014 L, N_T*(L) = 0.025 + 0.644 L, with T_min = 0.2 and T_max = 1.5.
PHI_FIT = {"a_phi": 0.406, "b_phi": 0.014, "a_NT": 0.025, "b_NT": 0.644, "T_min": 0.2, "T_max": 1.5}


def phi_protocol(L: int, n: int | None = None) -> List[float]:
    """The phi-family set at the fitted optimum for linear size L (Eqs. 6-9): phi*(L),
    and N_T*(L) rounded to the nearest integer (at least 2) unless n is given."""
    phi = PHI_FIT["a_phi"] + PHI_FIT["b_phi"] * L
    if n is None:
        n = max(2, int(round(PHI_FIT["a_NT"] + PHI_FIT["b_NT"] * L)))
    return phi_temps(PHI_FIT["T_min"], PHI_FIT["T_max"], n, phi)


@dataclass
class Workload:
    """One simulation job: the parameters the C-ABI's create call takes."""

    name: str
    ndim: int
    dims: Sequence[int]
    n_samples: int
    n_chains: int
    temps: Sequence[float]
    coupling_seed: int = 1
    sim_seed: int = 1
    p_plus: float = 0.5
    spin_format: str = "packed"  # "packed" (32 replicas per word) or "int8"
    houdayer: bool = False
    n_mcs: int = 1
    sample_offset: int = 0
    notes: str = field(default="")

    @property
    def N(self) -> int:
        n = 1
        for x in self.dims[: self.ndim]:
            n *= int(x)
        return n

    @property
    def T(self) -> int:
        return len(self.temps)

    @property
    def replicas(self) -> int:
        return self.n_samples * self.n_chains * self.T

    @property
    def attempts_per_sweep(self) -> int:
        return self.N * self.replicas

    def with_(self, **kw) -> "Workload":
        return replace(self, **kw)


def workload_3d_l6() -> Workload:
    """3D +-J L=6, 8 samples x 2 chains x 12 geometric temps in [1, 2], int8 spins,
    200 MCS of Metropolis + PT, seeds 1."""
    return Workload("3d_L6_S8_T12_int8", 3, (6, 6, 6), 8, 2, geometric_temps(1.0, 2.0, 12),
                    spin_format="int8", n_mcs=200)


def workload_3d_l16() -> Workload:
    """3D +-J L=16, 1024 samples x 2 chains x 32 geometric temps in [0.9, 2.0],
    bit-packed spins + 3-bit couplings, 10^4 MCS of Metropolis + PT."""
    return Workload("3d_L16_S1024_T32_packed", 3, (16, 16, 16), 1024, 2,
                    geometric_temps(0.9, 2.0, 32), n_mcs=10000)


def workload_3d_l16_t40() -> Workload:
    """The 3D L=16 job with 40 temperatures per chain (two words per chain, the second
    holding 8 replicas): the case the paired last words serve."""
    return Workload("3d_L16_S1024_T40_packed", 3, (16, 16, 16), 1024, 2,
                    geometric_temps(0.9, 2.0, 40), n_mcs=10000)


def workload_2d_l128_houdayer() -> Workload:
    """2D +-J L=128, 256 samples x 2 chains x 24 geometric temps in [0.2, 1.6],
    Metropolis + Houdayer + PT each MCS, 5000 MCS."""
    return Workload("2d_L128_S256_T24_houdayer", 2, (128, 128), 256, 2,
                    geometric_temps(0.2, 1.6, 24), houdayer=True, n_mcs=5000)


def workload_batched_uneven(seed: int = 1, n_mcs: int = 2000) -> List[Workload]:
    """3D +-J batches of uneven size: L = 8, 12, 16, 24, 32 with 2048, 1024, 512, 128 and 32
    samples; each sample draws its number of temperatures uniformly in 16..48 (MT19937,
    `seed`), geometric in [0.9, 2.0].  Samples of equal (L, T) form one job; a job's
    samples are numbered consecutively after those of the same L with fewer temperatures,
    and that number is the sample's job-wide index (its random keys)."""
    import numpy as np

    rng = np.random.Generator(np.random.MT19937(seed))
    jobs = []
    for L, S in ((8, 2048), (12, 1024), (16, 512), (24, 128), (32, 32)):
        Ts = rng.integers(16, 49, size=S)
        base = 0
        for T in sorted(set(int(x) for x in Ts)):
            count = int((Ts == T).sum())
            jobs.append(Workload(f"3d_L{L}_T{T}", 3, (L, L, L), count, 2, geometric_temps(0.9, 2.0, T),
                                 sample_offset=base, n_mcs=n_mcs))
            base += count
    return jobs


JFIX_SCALE = 1 << 20  # fixed-point couplings: J = J_fixed / 2^20


def gaussian_couplings_fixed(n_samples: int, dims: Sequence[int], seed: int = 1, sample_offset: int = 0):
    """Standard-normal couplings J_ij (Sec. 2.1) for every forward bond, as int32 fixed
    point in units of 2^-20, [S][N][d] in canonical site order (i = x + L0 (y + L1 z)).
    Drawn per sample from numpy's PCG64 seeded by (seed, job-wide sample index), so a
    shard of samples gets the same couplings as inside the whole job; |J| is clipped to
    8 (a 1e-15 tail)."""
    import numpy as np

    d = len(dims)
    N = 1
    for x in dims:
        N *= int(x)
    out = np.empty((n_samples, N, d), np.int32)
    for s in range(n_samples):
        rng = np.random.Generator(np.random.PCG64([int(seed), int(sample_offset + s)]))
        J = np.clip(rng.standard_normal((N, d)), -8.0, 8.0)
        out[s] = np.rint(J * JFIX_SCALE).astype(np.int32)
    return out


def workload_2d_gauss_l16() -> Workload:
    """2D Gaussian EA, L=16 (the paper's L=15 sample size made even for the checkerboard),
    512 samples x 2 chains x 32 temperatures of the phi-family (Eqs. 6-7) in [0.2, 1.5]
    with phi = 0.406 + 0.014 L (the fit of Eq. 8), int8 spins; couplings from
    gaussian_couplings_fixed(seed = coupling_seed)."""
    L = 16
    return Workload("2d_L16_S512_T32_gauss", 2, (L, L), 512, 2, phi_protocol(L, 32), spin_format="int8",
                    n_mcs=10000)
