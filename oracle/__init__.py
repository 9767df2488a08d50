"""CPU oracle for the +-J Edwards-Anderson parallel-tempering Monte Carlo.

TEST INFRASTRUCTURE ONLY.  Only the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this package.  The product
library never links or calls it and shares no code with it.

The arithmetic lives in ``sg_oracle.c`` (plain C, fp64, one Philox call per random
word); this module compiles it with gcc and wraps it with ctypes.  Arrays cross the
boundary as numpy arrays in the oracle's own plain layouts:

    spins      uint8  [S][C][T][N]   1 iff the spin is -1, indexed by replica j
    couplings  int8   [S][N][d]      +-1, bond (i, mu) joins i and i + e_mu
    energies   int32  [S][C][T]      by replica j
    perm       int32  [S][C][T]      temperature slot k -> replica j
    E by slot  int32  [S][C][T]      energies ordered by temperature slot
    NQ         int32  [S][T]         N q between chain 0 and chain 1 at each slot

Site index i = x + L0 (y + L1 z).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass
from typing import Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sg_oracle.c")
_SRC_GAUSS = os.path.join(_HERE, "sg_oracle_gauss.c")
_LIB = os.path.join(_HERE, "libsgoracle.so")

# -ffp-contract=off: no fused multiply-add may change an fp64 result.  -O3 without
# -march=native: the same flags give the same code paths on the x86 and the Arm hosts.
CFLAGS = ["-O3", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math"]


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/libsgoracle.so`` (plain gcc, no GPU code)."""
    stale = not os.path.exists(_LIB) or any(os.path.getmtime(_LIB) < os.path.getmtime(f)
                                            for f in (_SRC, _SRC_GAUSS, __file__))
    if force or stale:
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", *CFLAGS, _SRC, _SRC_GAUSS, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Params(ctypes.Structure):
    _fields_ = [
        ("ndim", ctypes.c_int32),
        ("dims", ctypes.c_int32 * 3),
        ("n_samples", ctypes.c_int32),
        ("sample_offset", ctypes.c_int32),
        ("n_chains", ctypes.c_int32),
        ("n_temps", ctypes.c_int32),
        ("temps", ctypes.POINTER(ctypes.c_double)),
        ("coupling_seed", ctypes.c_uint64),
        ("p_plus", ctypes.c_double),
        ("sim_seed", ctypes.c_uint64),
    ]


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        lib.or_create.restype = P
        lib.or_create.argtypes = [ctypes.POINTER(_Params)]
        lib.or_destroy.argtypes = [P]
        lib.or_sweep.argtypes = [P, ctypes.c_int]
        lib.or_exchange.argtypes = [P]
        lib.or_houdayer.argtypes = [P]
        lib.or_houdayer_multi.argtypes = [P]
        lib.or_mcs.argtypes = [P, ctypes.c_int, ctypes.c_int, ctypes.c_int]
        for name in ("or_measure",):
            getattr(lib, name).argtypes = [P, P, P]
        lib.or_qmodes.argtypes = [P, P]
        lib.or_get_trips.argtypes = [P, P, P]
        lib.or_check_energies.restype = ctypes.c_int
        lib.or_check_energies.argtypes = [P]
        for name in ("or_get_spins", "or_set_spins", "or_get_couplings", "or_set_couplings",
                     "or_get_energies", "or_get_thresholds", "or_get_counters", "or_set_perm"):
            getattr(lib, name).argtypes = [P, P]
        lib.or_get_perm.argtypes = [P, P, P]
        lib.or_get_pt_stats.argtypes = [P, P, P]
        lib.or_get_class_stats.argtypes = [P, P, P]
        lib.or_set_counters.argtypes = [P, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32]
        lib.or_set_houdayer_slots.argtypes = [P, ctypes.c_int]
        lib.or_set_typewriter.argtypes = [P, ctypes.c_int]
        lib.or_run_binned.argtypes = [P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                      ctypes.c_int, P, P]
        lib.or_enumerate.restype = ctypes.c_int
        lib.or_enumerate.argtypes = [P, ctypes.c_int, P]
        lib.or_philox4x32_10.argtypes = [P, P, P]
        # general (fixed-point) couplings, sg_oracle_gauss.c
        lib.og_create.restype = P
        lib.og_create.argtypes = [ctypes.c_int, P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, P,
                                  ctypes.c_uint64, P]
        lib.og_destroy.argtypes = [P]
        lib.og_sweep.argtypes = [P, ctypes.c_int]
        lib.og_exchange.argtypes = [P]
        lib.og_mcs.argtypes = [P, ctypes.c_int, ctypes.c_int]
        for name in ("og_get_spins", "og_set_spins", "og_get_energies", "og_get_perm", "og_get_counters"):
            getattr(lib, name).argtypes = [P, P]
        lib.og_measure.argtypes = [P, P, P]
        lib.og_check_energies.restype = ctypes.c_int
        lib.og_check_energies.argtypes = [P]
        lib.og_enumerate.restype = ctypes.c_int
        lib.og_enumerate.argtypes = [P, ctypes.c_int, P]
        lib.og_run_binned.argtypes = [P, ctypes.c_int, ctypes.c_int, P, P]
        lib.og_exp_f.restype = ctypes.c_float
        lib.og_exp_f.argtypes = [ctypes.c_float]
        lib.og_threshold.restype = ctypes.c_uint32
        lib.og_threshold.argtypes = [ctypes.c_float, ctypes.c_int32]
        _lib = lib
    return _lib


def philox4x32_10(ctr: Sequence[int], key: Sequence[int]) -> tuple[int, int, int, int]:
    """One Philox4x32-10 block: four 32-bit counter words, two key words."""
    lib = _load()
    c = np.asarray(ctr, dtype=np.uint32)
    k = np.asarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib.or_philox4x32_10(c.ctypes.data, k.ctypes.data, out.ctypes.data)
    return tuple(int(v) for v in out)


def _ptr(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data


def _houd_mode(h) -> int:
    if h is True:
        return 1
    if h is False or h is None:
        return 0
    return int(h)


@dataclass
class OracleParams:
    ndim: int
    dims: Sequence[int]
    n_samples: int
    n_chains: int
    temps: Sequence[float]
    coupling_seed: int = 1
    p_plus: float = 0.5
    sim_seed: int = 1
    sample_offset: int = 0
    houdayer_slots: int = 0  # the cluster move acts on slots k < houdayer_slots (0: every slot)
    typewriter: bool = False  # sweeps in index order (lattices with an odd extent)


class Oracle:
    """One oracle simulation: ``n_samples`` samples x ``n_chains`` x ``len(temps)``."""

    def __init__(self, p: OracleParams):
        lib = _load()
        self.p = p
        self.d = int(p.ndim)
        self.dims = tuple(int(x) for x in p.dims)[: self.d]
        self.N = int(np.prod(self.dims))
        self.S, self.C, self.T = int(p.n_samples), int(p.n_chains), len(p.temps)
        self._temps = np.ascontiguousarray(np.asarray(p.temps, dtype=np.float64))
        cp = _Params()
        cp.ndim = self.d
        for a in range(3):
            cp.dims[a] = self.dims[a] if a < self.d else 1
        cp.n_samples = self.S
        cp.sample_offset = int(p.sample_offset)
        cp.n_chains = self.C
        cp.n_temps = self.T
        cp.temps = self._temps.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        cp.coupling_seed = int(p.coupling_seed)
        cp.p_plus = float(p.p_plus)
        cp.sim_seed = int(p.sim_seed)
        self._h = lib.or_create(ctypes.byref(cp))
        if not self._h:
            raise ValueError("oracle rejected the parameters")
        self._lib = lib
        if p.houdayer_slots:
            if not 0 <= int(p.houdayer_slots) <= self.T:
                raise ValueError("houdayer_slots must lie in 0..n_temps")
            lib.or_set_houdayer_slots(self._h, int(p.houdayer_slots))
        if p.typewriter:
            lib.or_set_typewriter(self._h, 1)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._lib.or_destroy(h)
            self._h = None

    # dynamics
    def sweep(self, n: int = 1):
        self._lib.or_sweep(self._h, int(n))

    def exchange(self):
        self._lib.or_exchange(self._h)

    def houdayer(self):
        self._lib.or_houdayer(self._h)

    def houdayer_multi(self):
        """Multi-cluster variant: every q = -1 cluster of a pair exchanged by its own coin."""
        self._lib.or_houdayer_multi(self._h)

    def mcs(self, n: int = 1, n_metro: int = 1, houdayer=False):
        """houdayer: False/0 none, True/1 the single-cluster move, 2 the multi-cluster variant."""
        self._lib.or_mcs(self._h, int(n), int(n_metro), _houd_mode(houdayer))

    # observables and state
    def measure(self):
        e = np.zeros((self.S, self.C, self.T), np.int32)
        q = np.zeros((self.S, self.T), np.int32)
        self._lib.or_measure(self._h, _ptr(e), _ptr(q) if self.C >= 2 else None)
        return e, (q if self.C >= 2 else None)

    def trips(self):
        """(round trips completed [S][C] uint32, their total duration [S][C] uint64)."""
        n = np.zeros((self.S, self.C), np.uint32)
        tot = np.zeros((self.S, self.C), np.uint64)
        self._lib.or_get_trips(self._h, _ptr(n), _ptr(tot))
        return n, tot

    def qmodes(self) -> np.ndarray:
        """Overlap plane sums P[s][k][mu][x] (int32, x < max extent)."""
        Lmax = max(self.dims[: self.d])
        out = np.zeros((self.S, self.T, self.d, Lmax), np.int32)
        self._lib.or_qmodes(self._h, _ptr(out))
        return out

    def spins(self) -> np.ndarray:
        out = np.zeros((self.S, self.C, self.T, self.N), np.uint8)
        self._lib.or_get_spins(self._h, _ptr(out))
        return out

    def set_spins(self, bits: np.ndarray):
        b = np.ascontiguousarray(bits, dtype=np.uint8).reshape(self.S, self.C, self.T, self.N)
        self._lib.or_set_spins(self._h, _ptr(b))

    def couplings(self) -> np.ndarray:
        out = np.zeros((self.S, self.N, self.d), np.int8)
        self._lib.or_get_couplings(self._h, _ptr(out))
        return out

    def set_couplings(self, J: np.ndarray):
        j = np.ascontiguousarray(J, dtype=np.int8).reshape(self.S, self.N, self.d)
        self._lib.or_set_couplings(self._h, _ptr(j))

    def energies(self) -> np.ndarray:
        out = np.zeros((self.S, self.C, self.T), np.int32)
        self._lib.or_get_energies(self._h, _ptr(out))
        return out

    def perm(self):
        perm = np.zeros((self.S, self.C, self.T), np.int32)
        slot = np.zeros((self.S, self.C, self.T), np.int32)
        self._lib.or_get_perm(self._h, _ptr(perm), _ptr(slot))
        return perm, slot

    def set_perm(self, perm: np.ndarray):
        p = np.ascontiguousarray(perm, dtype=np.int32).reshape(self.S, self.C, self.T)
        self._lib.or_set_perm(self._h, _ptr(p))

    def thresholds(self) -> np.ndarray:
        out = np.zeros((self.T, self.d), np.uint32)
        self._lib.or_get_thresholds(self._h, _ptr(out))
        return out

    def counters(self) -> dict:
        out = np.zeros(7, np.uint64)
        self._lib.or_get_counters(self._h, _ptr(out))
        keys = ("t_metro", "t_pt", "t_houd", "near_threshold", "houd_moves", "houd_flipped", "error")
        return {k: int(v) for k, v in zip(keys, out)}

    def set_counters(self, t_metro: int, t_pt: int, t_houd: int):
        self._lib.or_set_counters(self._h, t_metro, t_pt, t_houd)

    def pt_stats(self):
        acc = np.zeros(max(self.T - 1, 1), np.uint64)
        tries = np.zeros(max(self.T - 1, 1), np.uint64)
        self._lib.or_get_pt_stats(self._h, _ptr(acc), _ptr(tries))
        return acc[: self.T - 1], tries[: self.T - 1]

    def class_stats(self):
        tries = np.zeros((self.T, self.d), np.uint64)
        acc = np.zeros((self.T, self.d), np.uint64)
        self._lib.or_get_class_stats(self._h, _ptr(tries), _ptr(acc))
        return tries, acc

    def check_energies(self) -> int:
        return int(self._lib.or_check_energies(self._h))

    def run_binned(self, n_mcs: int, n_bins: int, houdayer: bool = False, pt: bool = True,
                   n_metro: int = 1):
        """Bin means of E and E^2 per temperature slot, measured after every MCS."""
        sE = np.zeros((self.T, n_bins), np.float64)
        sE2 = np.zeros((self.T, n_bins), np.float64)
        self._lib.or_run_binned(self._h, int(n_mcs), int(n_metro), _houd_mode(houdayer), int(bool(pt)),
                                int(n_bins), _ptr(sE), _ptr(sE2))
        per = (n_mcs // n_bins) * self.S * self.C
        return sE / per, sE2 / per

    def enumerate(self, s: int = 0) -> np.ndarray:
        """Energy histogram of sample s over all 2^N states; index e + d N."""
        hist = np.zeros(2 * self.d * self.N + 1, np.uint64)
        if self._lib.or_enumerate(self._h, int(s), _ptr(hist)) != 0:
            raise ValueError("lattice too large to enumerate")
        return hist


class OracleGauss:
    """The general-coupling oracle (sg_oracle_gauss.c): couplings J [S][N][d] as int32
    fixed point in units of 2^-20, energies int64 in the same units."""

    def __init__(self, ndim: int, dims: Sequence[int], n_samples: int, n_chains: int, temps: Sequence[float],
                 J_fixed: np.ndarray, sim_seed: int = 1, sample_offset: int = 0):
        self._lib = _load()
        self.d = int(ndim)
        self.dims = tuple(int(x) for x in dims)[: self.d]
        self.N = int(np.prod(self.dims))
        self.S, self.C, self.T = int(n_samples), int(n_chains), len(temps)
        d3 = np.array(list(self.dims) + [1] * (3 - self.d), np.int32)
        t = np.ascontiguousarray(np.asarray(temps, np.float64))
        J = np.ascontiguousarray(np.asarray(J_fixed, np.int32).reshape(self.S, self.N, self.d))
        self._h = self._lib.og_create(self.d, _ptr(d3), self.S, int(sample_offset), self.C, self.T, _ptr(t),
                                      int(sim_seed), _ptr(J))
        if not self._h:
            raise ValueError("og_create failed")

    def __del__(self):
        if getattr(self, "_h", None):
            self._lib.og_destroy(self._h)
            self._h = None

    def sweep(self, n: int = 1):
        self._lib.og_sweep(self._h, int(n))

    def exchange(self):
        self._lib.og_exchange(self._h)

    def mcs(self, n: int = 1, n_metro: int = 1):
        self._lib.og_mcs(self._h, int(n), int(n_metro))

    def spins(self) -> np.ndarray:
        out = np.zeros((self.S, self.C, self.T, self.N), np.uint8)
        self._lib.og_get_spins(self._h, _ptr(out))
        return out

    def set_spins(self, bits: np.ndarray):
        b = np.ascontiguousarray(np.asarray(bits, np.uint8).reshape(self.S, self.C, self.T, self.N))
        self._lib.og_set_spins(self._h, _ptr(b))

    def energies(self) -> np.ndarray:
        out = np.zeros((self.S, self.C, self.T), np.int64)
        self._lib.og_get_energies(self._h, _ptr(out))
        return out

    def perm(self) -> np.ndarray:
        out = np.zeros((self.S, self.C, self.T), np.int32)
        self._lib.og_get_perm(self._h, _ptr(out))
        return out

    def measure(self):
        e = np.zeros((self.S, self.C, self.T), np.int64)
        q = np.zeros((self.S, self.T), np.int32)
        self._lib.og_measure(self._h, _ptr(e), _ptr(q) if self.C >= 2 else None)
        return e, (q if self.C >= 2 else None)

    def counters(self) -> dict:
        c = np.zeros(4, np.uint64)
        self._lib.og_get_counters(self._h, _ptr(c))
        return {"t_metro": int(c[0]), "t_pt": int(c[1]), "near_threshold": int(c[2])}

    def check_energies(self) -> int:
        return int(self._lib.og_check_energies(self._h))

    def enumerate(self, s: int = 0) -> np.ndarray:
        out = np.zeros(1 << self.N, np.int64)
        if self._lib.og_enumerate(self._h, int(s), _ptr(out)) != 0:
            raise ValueError("too many sites to enumerate")
        return out

    def run_binned(self, n_mcs: int, n_bins: int):
        sE = np.zeros((self.T, n_bins), np.float64)
        sE2 = np.zeros((self.T, n_bins), np.float64)
        self._lib.og_run_binned(self._h, int(n_mcs), int(n_bins), _ptr(sE), _ptr(sE2))
        return sE, sE2


def exp_f(x: float) -> float:
    """The general-coupling oracle's fp32 exp (Cody-Waite reduction, Taylor to r^6)."""
    return float(_load().og_exp_f(float(x)))


def gauss_threshold(beta_f: float, dE_fixed: int) -> int:
    return int(_load().og_threshold(float(beta_f), int(dE_fixed)))
