"""Python binding of the engine's C-ABI (``include/sgmc.h``, ``libsgmc.so``).

Argument marshalling only: every step of the simulation runs in the library's CUDA
kernels.  PyTorch supplies the device buffer the handle lives in and the CUDA stream
its work is queued on.  There is no CPU fallback: if the library is not built, or no
CUDA device is present, constructing a Simulation raises.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsgmc.so")

SG_PACKED32 = 0
SG_INT8 = 1

STATUS = {0: "SG_OK", 1: "SG_EINVAL", 2: "SG_ENOMEM", 3: "SG_ECUDA", 4: "SG_ETIMEOUT", 5: "SG_EUNSUPPORTED",
          6: "SG_ELIMIT"}


class SGError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {STATUS.get(status, status)}")


class Params(ctypes.Structure):
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
        ("spin_format", ctypes.c_int32),
        ("houdayer", ctypes.c_int32),
        ("n_metro", ctypes.c_int32),
        ("track_trips", ctypes.c_int32),
        ("coupling_kind", ctypes.c_int32),
        ("houdayer_slots", ctypes.c_int32),
    ]


EXPORTED = (
    "sg_query_bytes", "sg_create", "sg_sweep", "sg_exchange", "sg_houdayer", "sg_houdayer_multi", "sg_run_mcs",
    "sg_measure", "sg_measure_device", "sg_measure_async", "sg_measure_wait", "sg_run_mcs_measure_async", "sg_measure_qmodes", "sg_measure_qmodes_device", "sg_trips",
    "sg_import_couplings_fixed", "sg_measure64", "sg_get_state64", "sg_checkpoint_bytes", "sg_checkpoint",
    "sg_restore", "sg_selftest_wait", "sg_export_spins", "sg_import_spins", "sg_export_couplings", "sg_import_couplings",
    "sg_get_state", "sg_counters", "sg_exact_path_counters", "sg_thresholds", "sg_set_launch", "sg_set_pairing", "sg_get_launch", "sg_batch_create",
    "sg_batch_run", "sg_batch_destroy", "sg_sweep_streaming_static", "sg_probe_philox", "sg_destroy",
    "sg_strerror",
)

_lib = None


def lib():
    """Load ``libsgmc.so``; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is not built; run paper_2003_04621_gb300.build.build() (needs nvcc)")
    L = ctypes.CDLL(LIB_PATH)
    # uintptr_t stream handles are 64-bit on every supported platform
    P, U, I32, SZ = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int32, ctypes.c_size_t
    PP = ctypes.POINTER(Params)
    sig = {
        "sg_query_bytes": [PP, ctypes.POINTER(SZ)],
        "sg_create": [PP, P, SZ, U, ctypes.POINTER(P)],
        "sg_sweep": [P, I32, U],
        "sg_exchange": [P, U],
        "sg_houdayer": [P, U],
        "sg_houdayer_multi": [P, U],
        "sg_run_mcs": [P, I32, U],
        "sg_measure": [P, P, P, U],
        "sg_measure_device": [P, P, P, U],
        "sg_measure_async": [P, P, P, U],
        "sg_measure_wait": [P],
        "sg_run_mcs_measure_async": [P, I32, P, P, U],
        "sg_measure_qmodes": [P, P, U],
        "sg_trips": [P, P, P, U],
        "sg_measure_qmodes_device": [P, P, U],
        "sg_export_spins": [P, P, U],
        "sg_import_spins": [P, P, U],
        "sg_export_couplings": [P, P, U],
        "sg_import_couplings": [P, P, U],
        "sg_get_state": [P, P, P, P, U],
        "sg_import_couplings_fixed": [P, P, U],
        "sg_measure64": [P, P, P, U],
        "sg_get_state64": [P, P, P, P, U],
        "sg_checkpoint_bytes": [P, ctypes.POINTER(SZ)],
        "sg_checkpoint": [P, P, SZ, U],
        "sg_restore": [P, P, SZ, U],
        "sg_selftest_wait": [P, I32, U],
        "sg_counters": [P, P, P, P, U],
        "sg_exact_path_counters": [P, P, P, U],
        "sg_thresholds": [P, P],
        "sg_set_launch": [P, I32, I32],
        "sg_set_pairing": [P, I32],
        "sg_get_launch": [P, P, P, P],
        "sg_batch_create": [P, I32, I32, U, ctypes.POINTER(P)],
        "sg_batch_run": [P, I32, U],
        "sg_sweep_streaming_static": [P, I32, U],
        "sg_probe_philox": [I32, I32, I32, U, P, U],
    }
    for name, args in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = ctypes.c_int
    L.sg_destroy.argtypes = [P]
    L.sg_destroy.restype = None
    L.sg_batch_destroy.argtypes = [P]
    L.sg_batch_destroy.restype = None
    L.sg_strerror.argtypes = [ctypes.c_int]
    L.sg_strerror.restype = ctypes.c_char_p
    _lib = L
    return L


def _check(status: int, where: str):
    if status != 0:
        raise SGError(status, where)


def make_params(ndim: int, dims: Sequence[int], n_samples: int, n_chains: int, temps: Sequence[float],
                coupling_seed: int = 1, sim_seed: int = 1, p_plus: float = 0.5, spin_format: str = "packed",
                houdayer=False, n_metro: int = 1, sample_offset: int = 0, track_trips: bool = False,
                couplings: str = "pm", houdayer_slots: int = 0):
    """Fill an sg_params; returns (params, temps_array) -- keep the array alive.
    houdayer_slots: 0, or K to keep the cluster move to the K lowest temperature slots."""
    t = np.ascontiguousarray(np.asarray(temps, dtype=np.float64))
    p = Params()
    p.ndim = int(ndim)
    for a in range(3):
        p.dims[a] = int(dims[a]) if a < ndim else 1
    p.n_samples = int(n_samples)
    p.sample_offset = int(sample_offset)
    p.n_chains = int(n_chains)
    p.n_temps = len(t)
    p.temps = t.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    p.coupling_seed = int(coupling_seed)
    p.p_plus = float(p_plus)
    p.sim_seed = int(sim_seed)
    p.spin_format = SG_INT8 if spin_format == "int8" else SG_PACKED32
    p.houdayer = 2 if (houdayer is not True and houdayer == 2) else int(bool(houdayer))
    p.n_metro = int(n_metro)
    p.track_trips = int(bool(track_trips))
    if couplings not in ("pm", "fixed"):
        raise ValueError("couplings must be 'pm' (+-J from coupling_seed) or 'fixed' (set_couplings_fixed)")
    p.coupling_kind = 0 if couplings == "pm" else 1
    p.houdayer_slots = int(houdayer_slots)
    return p, t


def query_bytes(params: Params) -> int:
    n = ctypes.c_size_t(0)
    _check(lib().sg_query_bytes(ctypes.byref(params), ctypes.byref(n)), "sg_query_bytes")
    return int(n.value)


def _stream_handle(stream) -> int:
    import torch

    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream)


class Simulation:
    """One simulation job on the current CUDA device (see ``include/sgmc.h``)."""

    def __init__(self, ndim, dims, n_samples, n_chains, temps, coupling_seed=1, sim_seed=1, p_plus=0.5,
                 spin_format="packed", houdayer=False, n_metro=1, sample_offset=0, stream=None, device=None,
                 device_buffer=None, track_trips=False, couplings="pm", houdayer_slots=0):
        """device_buffer: optional (device pointer, bytes) the job lives in (256-byte
        aligned, at least query_bytes); by default a torch buffer is allocated."""
        import torch

        L = lib()
        if not torch.cuda.is_available():
            raise RuntimeError("no CUDA device: the engine has no CPU path")
        self.device = torch.device(device if device is not None else "cuda")
        self.ndim, self.dims = int(ndim), tuple(int(x) for x in dims)[: int(ndim)]
        self.N = int(np.prod(self.dims))
        self.S, self.C, self.T = int(n_samples), int(n_chains), len(temps)
        self.params, self._temps = make_params(ndim, dims, n_samples, n_chains, temps, coupling_seed, sim_seed,
                                               p_plus, spin_format, houdayer, n_metro, sample_offset,
                                               track_trips, couplings, houdayer_slots)
        self.gauss = couplings == "fixed"
        self.bytes = query_bytes(self.params)
        if device_buffer is not None:
            self._buf = None
            self._ptr, nbytes = int(device_buffer[0]), int(device_buffer[1])
            if self._ptr & 255 or nbytes < self.bytes:
                raise ValueError("device_buffer must be 256-byte aligned and hold query_bytes() bytes")
        else:
            # 256-byte alignment: over-allocate and offset
            self._buf = torch.empty(self.bytes + 256, dtype=torch.uint8, device=self.device)
            base = self._buf.data_ptr()
            self._ptr = (base + 255) & ~255
        self._stream = stream
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            _check(L.sg_create(ctypes.byref(self.params), ctypes.c_void_p(self._ptr), self.bytes,
                               _stream_handle(stream), ctypes.byref(h)), "sg_create")
        self._h = h

    # -- lifetime -------------------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None):
            lib().sg_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _s(self, stream=None):
        return _stream_handle(stream if stream is not None else self._stream)

    # -- dynamics -------------------------------------------------------------------
    def sweep(self, n: int = 1, stream=None):
        _check(lib().sg_sweep(self._h, int(n), self._s(stream)), "sg_sweep")

    def exchange(self, stream=None):
        _check(lib().sg_exchange(self._h, self._s(stream)), "sg_exchange")

    def houdayer(self, stream=None):
        _check(lib().sg_houdayer(self._h, self._s(stream)), "sg_houdayer")

    def houdayer_multi(self, stream=None):
        """Multi-cluster variant: every q = -1 cluster of a pair exchanged by its own coin."""
        _check(lib().sg_houdayer_multi(self._h, self._s(stream)), "sg_houdayer_multi")

    def run_mcs(self, n: int = 1, stream=None):
        _check(lib().sg_run_mcs(self._h, int(n), self._s(stream)), "sg_run_mcs")

    def sweep_streaming_static(self, n: int = 1, stream=None):
        """Sweeps that allocate nothing (library-held scratch; see sgmc.h)."""
        _check(lib().sg_sweep_streaming_static(self._h, int(n), self._s(stream)), "sg_sweep_streaming_static")

    # -- observables and state --------------------------------------------------------
    def _measure64(self, stream=None):
        E = np.zeros((self.S, self.C, self.T), np.int64)
        Q = np.zeros((self.S, self.T), np.int32) if self.C >= 2 else None
        _check(lib().sg_measure64(self._h, E.ctypes.data, Q.ctypes.data if Q is not None else None,
                                  self._s(stream)), "sg_measure64")
        return E, Q

    def measure(self, stream=None, out=None):
        """(E by slot [S][C][T], N q [S][T] or None) as numpy arrays; synchronises.
        `out` = (E, Q) writes into given C-contiguous int32 arrays instead (e.g. numpy
        views of pinned host tensors, so that the device-to-host copies are direct)."""
        if self.gauss:
            return self._measure64(stream)
        if out is None:
            E = np.zeros((self.S, self.C, self.T), np.int32)
            Q = np.zeros((self.S, self.T), np.int32) if self.C >= 2 else None
        else:
            E, Q = out
            if E.dtype != np.int32 or E.shape != (self.S, self.C, self.T) or not E.flags.c_contiguous:
                raise ValueError("E must be a C-contiguous int32 array of shape [S][C][T]")
            if self.C >= 2 and (Q is None or Q.dtype != np.int32 or Q.shape != (self.S, self.T)
                                or not Q.flags.c_contiguous):
                raise ValueError("Q must be a C-contiguous int32 array of shape [S][T]")
            if self.C < 2:
                Q = None
        _check(lib().sg_measure(self._h, E.ctypes.data, Q.ctypes.data if Q is not None else None, self._s(stream)),
               "sg_measure")
        return E, Q

    def measure_async(self, E, Q=None, stream=None):
        """As measure(out=(E, Q)) but only enqueued: the arrays (C-contiguous int32 of the
        measure shapes, ideally views of pinned tensors) hold the values once measure_wait()
        has returned or the device has been synchronised.  Keep them alive until then."""
        if self.gauss:
            raise SGError(5, "sg_measure_async")
        if E.dtype != np.int32 or E.shape != (self.S, self.C, self.T) or not E.flags.c_contiguous:
            raise ValueError("E must be a C-contiguous int32 array of shape [S][C][T]")
        if Q is not None and (Q.dtype != np.int32 or Q.shape != (self.S, self.T) or not Q.flags.c_contiguous):
            raise ValueError("Q must be a C-contiguous int32 array of shape [S][T]")
        _check(lib().sg_measure_async(self._h, E.ctypes.data, Q.ctypes.data if Q is not None else None,
                                      self._s(stream)), "sg_measure_async")

    def run_mcs_measure_async(self, n, E, Q=None, stream=None):
        """run_mcs(n) then measure_async(E, Q); the measurement runs inside the last MCS's
        launch when the kernel holds both chains of a sample (see sgmc.h)."""
        if E.dtype != np.int32 or E.shape != (self.S, self.C, self.T) or not E.flags.c_contiguous:
            raise ValueError("E must be a C-contiguous int32 array of shape [S][C][T]")
        if Q is not None and (Q.dtype != np.int32 or Q.shape != (self.S, self.T) or not Q.flags.c_contiguous):
            raise ValueError("Q must be a C-contiguous int32 array of shape [S][T]")
        _check(lib().sg_run_mcs_measure_async(self._h, int(n), E.ctypes.data, Q.ctypes.data if Q is not None else None,
                                              self._s(stream)), "sg_run_mcs_measure_async")

    def measure_wait(self):
        """Wait for the copies of every measure_async call on this simulation."""
        _check(lib().sg_measure_wait(self._h), "sg_measure_wait")

    def measure_device(self, E_out, Q_out=None, stream=None):
        """As measure, into torch int32 device tensors; does not synchronise."""
        _check(lib().sg_measure_device(self._h, E_out.data_ptr(), Q_out.data_ptr() if Q_out is not None else None,
                                       self._s(stream)), "sg_measure_device")

    def trips(self, stream=None):
        """(round trips completed [S][C] uint32, their total duration [S][C] uint64), in
        exchange passes (needs track_trips=True at creation).  Synchronises."""
        n = np.zeros((self.S, self.C), np.uint32)
        tot = np.zeros((self.S, self.C), np.uint64)
        _check(lib().sg_trips(self._h, n.ctypes.data, tot.ctypes.data, self._s(stream)), "sg_trips")
        return n, tot

    def qmodes(self, stream=None):
        """Overlap plane sums P[s][k][mu][x] (numpy int32, x < the largest extent); the
        integer part of the Fourier modes of q (see observables.q_modes).  Synchronises."""
        out = np.zeros((self.S, self.T, self.ndim, max(self.dims)), np.int32)
        _check(lib().sg_measure_qmodes(self._h, out.ctypes.data, self._s(stream)), "sg_measure_qmodes")
        return out

    def qmodes_device(self, P_out, stream=None):
        """As qmodes, into an int32 device tensor [S][T][d][Lmax]; does not synchronise."""
        _check(lib().sg_measure_qmodes_device(self._h, P_out.data_ptr(), self._s(stream)), "sg_measure_qmodes_device")

    def spins(self, stream=None):
        """uint8 device tensor [S][C][T][N], 1 iff the spin is -1 (replica order)."""
        import torch

        out = torch.empty((self.S, self.C, self.T, self.N), dtype=torch.uint8, device=self.device)
        _check(lib().sg_export_spins(self._h, out.data_ptr(), self._s(stream)), "sg_export_spins")
        return out

    def set_spins(self, bits, stream=None):
        import torch

        t = torch.as_tensor(np.asarray(bits, dtype=np.uint8) if not torch.is_tensor(bits) else bits)
        t = t.to(device=self.device, dtype=torch.uint8).contiguous().reshape(self.S, self.C, self.T, self.N)
        _check(lib().sg_import_spins(self._h, t.data_ptr(), self._s(stream)), "sg_import_spins")
        torch.cuda.current_stream().synchronize() if stream is None else stream.synchronize()

    def couplings(self, stream=None):
        """int8 device tensor [S][N][d] of +-1 couplings."""
        import torch

        out = torch.empty((self.S, self.N, self.ndim), dtype=torch.int8, device=self.device)
        _check(lib().sg_export_couplings(self._h, out.data_ptr(), self._s(stream)), "sg_export_couplings")
        return out

    def set_couplings(self, J, stream=None):
        import torch

        t = torch.as_tensor(np.asarray(J, dtype=np.int8) if not torch.is_tensor(J) else J)
        t = t.to(device=self.device, dtype=torch.int8).contiguous().reshape(self.S, self.N, self.ndim)
        _check(lib().sg_import_couplings(self._h, t.data_ptr(), self._s(stream)), "sg_import_couplings")
        torch.cuda.current_stream().synchronize() if stream is None else stream.synchronize()

    def state(self, stream=None):
        """(E by replica [S][C][T], perm [S][C][T], steps (t_metro, t_pt, t_houd)).  E is
        int32 for +-J jobs, int64 in units of 2^-20 for general couplings."""
        perm = np.zeros((self.S, self.C, self.T), np.int32)
        steps = np.zeros(3, np.uint64)
        if self.gauss:
            E = np.zeros((self.S, self.C, self.T), np.int64)
            _check(lib().sg_get_state64(self._h, E.ctypes.data, perm.ctypes.data, steps.ctypes.data,
                                        self._s(stream)), "sg_get_state64")
        else:
            E = np.zeros((self.S, self.C, self.T), np.int32)
            _check(lib().sg_get_state(self._h, E.ctypes.data, perm.ctypes.data, steps.ctypes.data,
                                      self._s(stream)), "sg_get_state")
        return E, perm, tuple(int(x) for x in steps)

    def checkpoint(self, stream=None) -> np.ndarray:
        """The job's whole state as a host byte array (see sg_checkpoint)."""
        n = ctypes.c_size_t()
        _check(lib().sg_checkpoint_bytes(self._h, ctypes.byref(n)), "sg_checkpoint_bytes")
        blob = np.empty(n.value, np.uint8)
        _check(lib().sg_checkpoint(self._h, blob.ctypes.data, n.value, self._s(stream)), "sg_checkpoint")
        return blob

    def restore(self, blob: np.ndarray, stream=None):
        """Resume from a checkpoint of a job with the same parameters."""
        b = np.ascontiguousarray(blob, dtype=np.uint8)
        _check(lib().sg_restore(self._h, b.ctypes.data, b.size, self._s(stream)), "sg_restore")

    def set_couplings_fixed(self, J_fixed, stream=None):
        """General couplings: int32 [S][N][d] in units of 2^-20 (canonical site order);
        recomputes the energies."""
        J = np.ascontiguousarray(np.asarray(J_fixed, np.int32).reshape(self.S, self.N, self.ndim))
        _check(lib().sg_import_couplings_fixed(self._h, J.ctypes.data, self._s(stream)), "sg_import_couplings_fixed")

    def counters(self, stream=None) -> dict:
        near = np.zeros(1, np.uint64)
        acc = np.zeros(max(self.T - 1, 1), np.uint64)
        hs = np.zeros(1, np.uint64)
        _check(lib().sg_counters(self._h, near.ctypes.data, acc.ctypes.data, hs.ctypes.data, self._s(stream)),
               "sg_counters")
        xe = np.zeros(1, np.uint64)
        mb = np.zeros(1, np.uint64)
        _check(lib().sg_exact_path_counters(self._h, xe.ctypes.data, mb.ctypes.data, self._s(stream)),
               "sg_exact_path_counters")
        return {"near_threshold": int(near[0]), "pt_accepts": acc[: self.T - 1].copy(),
                "houdayer_sites": int(hs[0]), "exchange_exact": int(xe[0]), "metropolis_band": int(mb[0])}

    def set_launch(self, threads: int = 0, words: int = 0):
        """Resident-kernel launch shape (threads per CTA, words per CTA); results are
        identical for every accepted shape."""
        _check(lib().sg_set_launch(self._h, int(threads), int(words)), "sg_set_launch")

    def set_pairing(self, on: bool = True):
        """Allow (default) or forbid pairing the two chains' partial last words in one
        word in the fused MCS; the results are identical either way."""
        _check(lib().sg_set_pairing(self._h, 1 if on else 0), "sg_set_pairing")

    def launch(self):
        v = np.zeros(3, np.int32)
        _check(lib().sg_get_launch(self._h, v[0:].ctypes.data, v[1:].ctypes.data, v[2:].ctypes.data),
               "sg_get_launch")
        return {"threads": int(v[0]), "words": int(v[1]), "smem": int(v[2])}

    def thresholds(self) -> np.ndarray:
        out = np.zeros((self.T, self.ndim), np.uint32)
        _check(lib().sg_thresholds(self._h, out.ctypes.data), "sg_thresholds")
        return out


class Batch:
    """Several simulations advanced together by one CUDA graph per launch (each job a
    branch; see sg_batch_create).  Results equal those of running each job alone."""

    def __init__(self, sims, mcs_per_launch: int = 1, stream=None):
        self.sims = list(sims)
        self.mcs_per_launch = int(mcs_per_launch)
        self._stream = stream
        arr = (ctypes.c_void_p * len(self.sims))(*[s_._h for s_ in self.sims])
        b = ctypes.c_void_p()
        _check(lib().sg_batch_create(arr, len(self.sims), self.mcs_per_launch, _stream_handle(stream),
                                     ctypes.byref(b)), "sg_batch_create")
        self._b = b

    def run(self, n_launches: int = 1, stream=None):
        _check(lib().sg_batch_run(self._b, int(n_launches), _stream_handle(stream if stream is not None
                                                                             else self._stream)), "sg_batch_run")

    def close(self):
        if getattr(self, "_b", None):
            lib().sg_batch_destroy(self._b)
            self._b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def from_workload(w, stream=None, **overrides) -> Simulation:
    """Create a Simulation from a ``paper_2003_04621_gb300.inputs.Workload``."""
    kw = dict(ndim=w.ndim, dims=w.dims, n_samples=w.n_samples, n_chains=w.n_chains, temps=list(w.temps),
              coupling_seed=w.coupling_seed, sim_seed=w.sim_seed, p_plus=w.p_plus, spin_format=w.spin_format,
              houdayer=w.houdayer, sample_offset=w.sample_offset)
    kw.update(overrides)
    return Simulation(stream=stream, **kw)


def probe_philox(n_sites: int, n_sweeps: int, n_blocks: int, out, stream=None, sim_seed: int = 1):
    """Enqueue the Philox-ceiling probe (see sg_probe_philox) on `stream`; `out` is an
    int32 device tensor of at least n_blocks x 256 elements.  Returns the words it draws."""
    if out.numel() < n_blocks * 256:
        raise ValueError("out needs n_blocks x 256 elements")
    _check(lib().sg_probe_philox(int(n_sites), int(n_sweeps), int(n_blocks), int(sim_seed), out.data_ptr(),
                                 _stream_handle(stream)), "sg_probe_philox")
    return 64 * int(n_sites) * int(n_sweeps)
