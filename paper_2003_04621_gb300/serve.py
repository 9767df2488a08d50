"""Serving: continuous batching of simulation jobs on one GPU.

Jobs (lattice, samples, temperatures, sweeps) arrive over time.  The server keeps a
device-memory arena; a waiting job is admitted (first come, first served) as soon as the
arena can hold its state and the resident jobs do not already fill the GPU, and then
stays resident until it has made all its MCS.  Every replay advances all resident jobs
by the same number q of MCS with ONE CUDA-graph launch in which each job is a branch of
its own (sg_batch), so jobs of different sizes overlap on the device; q is the scheduling
quantum, cut to the smallest number of MCS any resident job has left, so that every job
makes exactly its own number of MCS.  The graph is re-captured only when the resident
set or q changes.

The host never waits for a whole replay: it keeps up to two replays queued on the GPU,
and between them it polls their completion events, admits arrivals, and retires the
jobs whose last replay has finished (their E by slot and N q are read back on a side
stream, their memory returned to the arena).

A job's results are those of running it alone: the dynamics depend only on the job's
own parameters, never on which other jobs share the device.

Latency is measured from a job's arrival to the moment its results are on the host.
"""
from __future__ import annotations

import bisect
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


def poisson_trace(n_jobs: int, rate: float = 50.0, seed: int = 7, max_sweeps: int = 5000,
                  min_sweeps: int = 500) -> List[JobSpec]:
    """The serving workload: Poisson arrivals at `rate` per second; each job is 3D (L even
    in 8..32, temperatures geometric in [0.9, 2.0]) or 2D (L even in 32..256, [0.2, 1.6])
    with probability 1/2, 16..256 samples, 16..40 temperatures, and a number of sweeps
    uniform in [min_sweeps, max_sweeps]."""
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


class _CudaBackend:
    """What the server needs from the device: streams, events, the SM count, and the
    engine's binding (simulations, batches, sizes).  Tests substitute a host fake."""

    def __init__(self):
        import torch

        from . import sgmc

        self.torch = torch
        self.sgmc = sgmc

    def stream(self):
        return self.torch.cuda.Stream()

    def event(self, stream):
        ev = self.torch.cuda.Event()
        ev.record(stream)
        return ev

    def n_sm(self) -> int:
        return self.torch.cuda.get_device_properties(self.torch.cuda.current_device()).multi_processor_count

    def arena(self, nbytes: int) -> "Arena":
        return Arena(nbytes)

    def query_bytes(self, spec: JobSpec) -> int:
        p, _t = self.sgmc.make_params(spec.ndim, spec.dims, spec.n_samples, 2, list(spec.temps))
        return self.sgmc.query_bytes(p)

    def simulation(self, spec: JobSpec, ptr: int, nbytes: int, stream):
        return self.sgmc.Simulation(spec.ndim, spec.dims, spec.n_samples, 2, list(spec.temps),
                                    coupling_seed=spec.coupling_seed, sim_seed=spec.sim_seed, stream=stream,
                                    device_buffer=(ptr, nbytes))

    def batch(self, sims, mcs_per_launch: int, stream):
        return self.sgmc.Batch(sims, mcs_per_launch=mcs_per_launch, stream=stream)

    def synchronize(self):
        self.torch.cuda.synchronize()


class Server:
    """Continuous-batching server over one GPU (see the module docstring).

    quantum      MCS per replay (cut to the smallest number any resident job has left)
    max_ctas     admission stops while the resident jobs' sweep CTAs reach this many (a
                 few waves of the GPU: more resident jobs would only share it more
                 thinly and delay every one of them); 0 derives it from the device
    max_inflight replays queued on the GPU ahead of the host (2: one runs while the
                 next waits, so the GPU never idles on the host)
    """

    def __init__(self, arena_bytes: int, quantum: int = 100, stream=None, tune: bool = False, max_ctas: int = 0,
                 max_inflight: int = 2, backend=None):
        self.dev = backend if backend is not None else _CudaBackend()
        self.arena = self.dev.arena(arena_bytes)
        self.quantum = int(quantum)
        self.stream = stream if stream is not None else self.dev.stream()
        self.side = self.dev.stream()  # job creation and final measurements
        self.tune = tune
        if max_ctas <= 0:
            # 24 sweep CTAs per SM: about eight waves of the resident kernels, enough that
            # the device stays full as jobs of different lengths come and go
            max_ctas = 24 * self.dev.n_sm()
        self.max_ctas = int(max_ctas)
        self.max_inflight = max(1, int(max_inflight))
        self.graph_builds = 0
        self.graph_launches = 0

    def _make(self, spec: JobSpec, off: int):
        return self.dev.simulation(spec, self.arena.base + off, self.arena.capacity - off, self.side)

    @staticmethod
    def _ctas(sim) -> int:
        """Sweep CTAs of one MCS of the job: (sample, word group) items of the resident
        kernel, or for a lattice streamed from global memory its sites x words / 512
        (one thread per site of a colour and word, 256-thread CTAs)."""
        shape = sim.launch()
        words = sim.C * ((sim.T + 31) // 32)
        if shape["words"] < 0:
            return max(1, sim.S * words * sim.N // 512)
        return sim.S * max(1, words // max(1, shape["words"]))

    def run(self, trace: Sequence[JobSpec], time_scale: float = 1.0) -> List[JobResult]:
        """Serve `trace` (arrival times scaled by `time_scale`); returns one result per job."""
        pending = deque(sorted(trace, key=lambda j: j.arrival))
        waiting: deque = deque()
        active: Dict[int, dict] = {}
        results: List[JobResult] = []
        inflight: deque = deque()  # (event, batch, job ids whose last MCS are in that replay)
        batch, batch_key = None, None
        t0 = time.perf_counter()

        def now():
            return time.perf_counter() - t0

        def in_use(b):
            return any(x is b for _, x, _ in inflight)

        while pending or waiting or active:
            progressed = False
            t = now()
            while pending and pending[0].arrival * time_scale <= t:
                waiting.append(pending.popleft())
            # retire the replays that have finished, oldest first
            while inflight and inflight[0][0].query():
                _ev, b, fin = inflight.popleft()
                for jid in fin:
                    j = active.pop(jid)
                    E, Q = j["sim"].measure(stream=self.side)
                    results.append(JobResult(jid, j["spec"].arrival * time_scale, j["admitted"], now(),
                                             j["spec"].attempts, E, Q))
                    j["sim"].close()
                    self.arena.free(j["off"], j["bytes"])
                if b is not None and b is not batch and not in_use(b):
                    b.close()
                progressed = True
            # admit waiting jobs while memory and the GPU's width allow
            load = sum(j["ctas"] for j in active.values() if j["left"] > 0)
            while waiting and (load < self.max_ctas or not active):
                spec = waiting[0]
                need = self.dev.query_bytes(spec)
                if need > self.arena.capacity:
                    raise ValueError(f"job {spec.job_id} needs {need} bytes, more than the arena")
                off = self.arena.alloc(need)
                if off is None:
                    break
                waiting.popleft()
                sim = self._make(spec, off)
                ctas = self._ctas(sim)
                active[spec.job_id] = dict(spec=spec, sim=sim, off=off, bytes=need, left=max(0, spec.n_mcs),
                                           admitted=now(), ctas=ctas)
                if spec.n_mcs <= 0:  # nothing to run: its results are those of the fresh state
                    inflight.append((self.dev.event(self.side), None, [spec.job_id]))
                else:
                    load += ctas
                progressed = True
            # keep up to max_inflight replays queued
            while len(inflight) < self.max_inflight:
                run = [j for j in active.values() if j["left"] > 0]
                if not run:
                    break
                q = min(self.quantum, min(j["left"] for j in run))
                key = (tuple(j["spec"].job_id for j in run), q)
                if key != batch_key:
                    if batch is not None and not in_use(batch):
                        batch.close()
                    batch = self.dev.batch([j["sim"] for j in run], q, self.stream)
                    batch_key = key
                    self.graph_builds += 1
                batch.run(1, stream=self.stream)
                ev = self.dev.event(self.stream)
                self.graph_launches += 1
                fin = []
                for j in run:
                    j["left"] -= q
                    if j["left"] == 0:
                        fin.append(j["spec"].job_id)
                inflight.append((ev, batch, fin))
                progressed = True
            if not progressed:
                if inflight:
                    time.sleep(2e-4)
                elif pending and not waiting:
                    time.sleep(max(0.0, pending[0].arrival * time_scale - now()))
        if batch is not None:
            batch.close()
        self.dev.synchronize()
        return results


def summarize(results: List[JobResult]) -> dict:
    lat = np.array([r.latency for r in results])
    span = max(r.finished for r in results) - min(r.arrival for r in results)
    att = sum(r.attempts for r in results)
    return {"jobs": len(results), "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "mean_s": float(lat.mean()), "makespan_s": float(span), "jobs_per_s": len(results) / span,
            "attempts_per_ns": att / (span * 1e9)}
