"""Two-replica observables from the overlap plane sums (host post-processing).

The engine measures, per (sample, temperature slot), the integer plane sums of the
overlap field q_i = s_i^(1) s_i^(2) (the summand of Eq. 4): P[mu][x] = sum of q_i over
the sites with coordinate x along axis mu.  They hold the Fourier modes of q along the
axes exactly,

    q(k e_mu) = (1/N) sum_x exp(i k x) P[mu][x],

from which the spin-glass susceptibility chi_SG(k) = N [<|q(k)|^2>] and the second-moment
correlation length follow; the paper measures both with the two-replica kernels of
Sec. 3 without printing their formulas, so the standard definitions are used:

    xi = sqrt(chi(0) / chi(k_min) - 1) / (2 sin(k_min / 2)),   k_min = 2 pi / L.

Thermal and disorder averages are the caller's (means over measurements and samples).
"""
from __future__ import annotations

import math
from typing import Sequence

import numpy as np


def q_modes(P: np.ndarray, dims: Sequence[int]):
    """(q(0), |q(k_min e_mu)|^2 per axis) for plane sums P[..., mu, x].

    Returns arrays shaped P.shape[:-2] and P.shape[:-2] + (d,)."""
    P = np.asarray(P, dtype=np.float64)
    d = len(dims)
    N = float(np.prod(dims))
    q0 = P[..., 0, : dims[0]].sum(axis=-1) / N
    qk2 = np.empty(P.shape[:-2] + (d,), np.float64)
    for mu in range(d):
        L = int(dims[mu])
        x = np.arange(L)
        ph = np.exp(2j * math.pi * x / L)
        qk = (P[..., mu, :L] * ph).sum(axis=-1) / N
        qk2[..., mu] = np.abs(qk) ** 2
    return q0, qk2


def chi_sg(P: np.ndarray, dims: Sequence[int]):
    """(chi_SG(0), chi_SG(k_min)) averaged over every leading axis of P (measurements,
    samples) and, for k_min, over the lattice axes: N <q(0)^2> and N <|q(k_min)|^2>."""
    q0, qk2 = q_modes(P, dims)
    N = float(np.prod(dims))
    return N * float(np.mean(q0**2)), N * float(np.mean(qk2))


def xi_second_moment(chi0: float, chik: float, L: int) -> float:
    """Second-moment correlation length from chi(0) and chi(k_min), k_min = 2 pi / L."""
    kmin = 2.0 * math.pi / L
    r = chi0 / chik - 1.0
    return math.sqrt(max(r, 0.0)) / (2.0 * math.sin(kmin / 2.0))


def tunnelling_time(n_trips: np.ndarray, total: np.ndarray) -> float:
    """Mean round-trip time in temperature (Sec. 2.3: lowest -> highest -> lowest), in
    exchange passes, from the per-chain trip counters; nan if no trip has completed."""
    n = float(np.sum(np.asarray(n_trips, dtype=np.float64)))
    return float(np.sum(np.asarray(total, dtype=np.float64))) / n if n > 0 else float("nan")
