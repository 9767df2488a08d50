"""Serving: continuous batching of simulation jobs on one GPU.

Jobs (lattice, samples, temperatures, sweeps) arrive over time.  The server keeps a
device-memory arena; a waiting job is admitted (first come, first served) as soon as the
arena can hold its state, and then stays resident until it has made all its MCS.  Every
scheduling quantum advances all resident jobs by `quantum` MCS with ONE CUDA-graph
launch in which each job is a branch of its own (sg_batch), so jobs of different sizes
overlap on the device; the graph is re-captured only when the set of resident jobs
changes.  A finished job is measured (E by slot and N q, read back to the host), its
memory is returned, and the next waiting job is admitted.

A job's results are those of running it alone: the dynamics depend only on the job's
own parameters, never on which other jobs share the device.

Latency is measured from a job's arrival to the moment its results are on the host.
"""
from __future__ import annotations

import bisect
import math
import time
from collections import deque
from dataclasses import dataclass, field
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np

from .inputs import geometric_temps


@dataclass
class JobSpec:
    job_id: int
    ndim: int
    dims: Tuple[int, ...]
    n_samples: int
    temps: Sequence[float]
    n_mcs: int
    arrival: float = 0.0  # seconds after the start of the trace
    coupling_seed: int = 1
    sim_seed: int = 1

    @property
    def attempts(self) -> int:
        return int(np.prod(self.dims)) * self.n_samples * 2 * len(self.temps) * self.n_mcs


def poisson_trace(n_jobs: int, rate: float = 50.0, seed: int = 7, quantum: int = 100,
                  max_sweeps: int = 5000, min_sweeps: int = 500) -> List[JobSpec]:
    """The serving workload: Poisson arrivals at `rate` per second; each job is 3D (L even
    in 8..32, temperatures geometric in [0.9, 2.0]) or 2D (L even in 32..256, [0.2, 1.6])
    with probability 1/2, 16..256 samples, 16..40 temperatures, and a number of sweeps in
    [min_sweeps, max_sweeps] rounded to a multiple of the scheduling quantum."""
    rng = np.random.Generator(np.random.MT19937(seed))
    t = 0.0
    jobs = []
    for j in range(n_jobs):
        t += rng.exponential(1.0 / rate)
        if rng.random() < 0.5:
            L = int(rng.choice(np.arange(8, 33, 2)))
            ndim, dims, tmin, tmax = 3, (L, L, L), 0.9, 2.0
        else:
            L = int(rng.choice(np.arange(32, 257, 2)))
            ndim, dims, tmin, tmax = 2, (L, L), 0.2, 1.6
        S = int(rng.integers(16, 257))
        T = int(rng.integers(16, 41))
        sweeps = int(rng.integers(min_sweeps, max_sweeps + 1))
        sweeps = max(quantum, int(round(sweeps / quantum)) * quantum)
        jobs.append(JobSpec(j, ndim, dims, S, geometric_temps(tmin, tmax, T), sweeps, arrival=t,
                            coupling_seed=int(rng.integers(1, 2**31)), sim_seed=int(rng.integers(1, 2**31))))
    return jobs


class Arena:
    """First-fit allocator over one device buffer (256-byte granules)."""

    ALIGN = 256

    def __init__(self, nbytes: int, device="cuda"):
        import torch

        self.capacity = (int(nbytes) // self.ALIGN) * self.ALIGN
        self._buf = torch.empty(self.capacity + self.ALIGN, dtype=torch.uint8, device=device)
        self.base = (self._buf.data_ptr() + self.ALIGN - 1) & ~(self.ALIGN - 1)
        self._free: List[Tuple[int, int]] = [(0, self.capacity)]  # (offset, size), sorted

    def alloc(self, nbytes: int) -> Optional[int]:
        need = ((int(nbytes) + self.ALIGN - 1) // self.ALIGN) * self.ALIGN
        for k, (off, size) in enumerate(self._free):
            if size >= need:
                if size == need:
                    self._free.pop(k)
                else:
                    self._free[k] = (off + need, size - need)
                return off
        return None

    def free(self, off: int, nbytes: int):
        need = ((int(nbytes) + self.ALIGN - 1) // self.ALIGN) * self.ALIGN
        k = bisect.bisect_left(self._free, (off, 0))
        self._free.insert(k, (off, need))
        merged: List[Tuple[int, int]] = []
        for o, s in self._free:
            if merged and merged[-1][0] + merged[-1][1] == o:
                merged[-1] = (merged[-1][0], merged[-1][1] + s)
            else:
                merged.append((o, s))
        self._free = merged

    @property
    def free_bytes(self) -> int:
        return sum(s for _, s in self._free)


@dataclass
class JobResult:
    job_id: int
    arrival: float
    admitted: float
    finished: float
    attempts: int
    E: np.ndarray = field(repr=False)
    Q: np.ndarray = field(repr=False)

    @property
    def latency(self) -> float:
        return self.finished - self.arrival


class Server:
    """Continuous-batching server over one GPU (see the module docstring)."""

    def __init__(self, arena_bytes: int, quantum: int = 100, stream=None, tune: bool = False):
        import torch

        self.arena = Arena(arena_bytes)
        self.quantum = int(quantum)
        self.stream = stream if stream is not None else torch.cuda.Stream()
        self.tune = tune
        self.graph_builds = 0
        self.graph_launches = 0

    def _make(self, spec: JobSpec, off: int):
        from .sgmc import Simulation

        return Simulation(spec.ndim, spec.dims, spec.n_samples, 2, list(spec.temps),
                          coupling_seed=spec.coupling_seed, sim_seed=spec.sim_seed, stream=self.stream,
                          device_buffer=(self.arena.base + off, self.arena.capacity - off))

    def run(self, trace: Sequence[JobSpec], time_scale: float = 1.0) -> List[JobResult]:
        """Serve `trace` (arrival times scaled by `time_scale`); returns one result per job."""
        import torch

        from .sgmc import Batch, make_params, query_bytes

        pending = deque(sorted(trace, key=lambda j: j.arrival))
        waiting: deque = deque()
        active: Dict[int, dict] = {}
        results: List[JobResult] = []
        batch = None
        dirty = True
        t0 = time.perf_counter()
        while pending or waiting or active:
            now = time.perf_counter() - t0
            while pending and pending[0].arrival * time_scale <= now:
                waiting.append(pending.popleft())
            while waiting:
                spec = waiting[0]
                p, _t = make_params(spec.ndim, spec.dims, spec.n_samples, 2, list(spec.temps))
                need = query_bytes(p)
                if need > self.arena.capacity:
                    raise ValueError(f"job {spec.job_id} needs {need} bytes, more than the arena")
                off = self.arena.alloc(need)
                if off is None:
                    break
                waiting.popleft()
                sim = self._make(spec, off)
                active[spec.job_id] = dict(spec=spec, sim=sim, off=off, bytes=need, left=spec.n_mcs,
                                           admitted=time.perf_counter() - t0)
                dirty = True
            if not active:
                if pending:
                    time.sleep(max(0.0, pending[0].arrival * time_scale - (time.perf_counter() - t0)))
                continue
            if dirty:
                if batch is not None:
                    batch.close()
                jobs = list(active.values())
                batch = Batch([j["sim"] for j in jobs], mcs_per_launch=self.quantum, stream=self.stream)
                self.graph_builds += 1
                dirty = False
            batch.run(1, stream=self.stream)
            self.graph_launches += 1
            self.stream.synchronize()
            done = []
            for jid, j in active.items():
                j["left"] -= self.quantum
                if j["left"] <= 0:
                    done.append(jid)
            for jid in done:
                j = active.pop(jid)
                E, Q = j["sim"].measure(stream=self.stream)
                fin = time.perf_counter() - t0
                results.append(JobResult(jid, j["spec"].arrival * time_scale, j["admitted"], fin,
                                         j["spec"].attempts, E, Q))
                j["sim"].close()
                self.arena.free(j["off"], j["bytes"])
                dirty = True
        if batch is not None:
            batch.close()
        return results


def summarize(results: List[JobResult]) -> dict:
    lat = np.array([r.latency for r in results])
    span = max(r.finished for r in results) - min(r.arrival for r in results)
    att = sum(r.attempts for r in results)
    return {"jobs": len(results), "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "mean_s": float(lat.mean()), "makespan_s": float(span), "jobs_per_s": len(results) / span,
            "attempts_per_ns": att / (span * 1e9)}
