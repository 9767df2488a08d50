"""Benchmark: spin-flip attempts per ns of the parallel-tempering Monte Carlo step.

Workload: 3D +-J Edwards-Anderson spin glass, L = 16 periodic, 1024 disorder samples x
2 chains x 32 geometric temperatures in [0.9, 2.0], bit-packed spins and couplings.
One step is one MCS over the whole batch: a checkerboard Metropolis sweep of every
replica (with the energies) and one replica-exchange pass (Eq. 5), i.e. one launch of
the resident kernel.  Inputs are synthetic (seeded couplings and hot start).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  Under torchrun each rank simulates its own 1024
samples (job-wide sample offsets rank * 1024), so per-GPU work is fixed: weak scaling.
`--impl reference` times the CPU oracle (the plain C implementation the tests check the
engine against) on the host cores, on bounded samples of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "spin-flip attempts/ns"
UNIT = "attempts/ns"
BYTES_PER_ATTEMPT = 0.25  # 1 bit read + 1 bit written per spin per sweep (packed)


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.file = None

    def start(self):
        try:
            self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=self.file, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.file.flush()
        rows = []
        with open(self.file.name) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.file.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        smax = [num(r[2]) for r in rows if num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        loaded = [v for v in sm if smax and v > 0.5 * max(smax)] or sm
        return {"sm_mhz": statistics.median(loaded) if loaded else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": reasons, "samples": len(rows)}


def cpu_model() -> str:
    """The host CPU's model name (x86 'model name', or the Arm implementer/part)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.split(":")[0].strip() in ("Model name", "Model"):
                name = line.split(":", 1)[1].strip()
                if name and not name.isdigit():
                    return name
    except (OSError, subprocess.SubprocessError):
        pass
    import platform

    return platform.processor() or platform.machine()


def cpu_baseline(workload, n_threads: int, n_mcs: int, n_samples: int, metropolis_only: bool = False):
    """Time the CPU oracle, as it is, on `n_samples` samples of the workload for `n_mcs`
    MCS each (with the workload's Houdayer moves), or `n_mcs` Metropolis sweeps alone,
    one oracle per thread (ctypes releases the GIL).  The oracles are created untimed."""
    import oracle
    from concurrent.futures import ThreadPoolExecutor

    oracle.build()
    per = max(1, n_samples // n_threads)
    orcs = [oracle.Oracle(oracle.OracleParams(workload.ndim, workload.dims, per, workload.n_chains,
                                              list(workload.temps), coupling_seed=workload.coupling_seed,
                                              sim_seed=workload.sim_seed, sample_offset=t * per))
            for t in range(n_threads)]

    def run(o):
        if metropolis_only:
            o.sweep(n_mcs)
        else:
            o.mcs(n_mcs, houdayer=bool(workload.houdayer))
        return o.S

    t0 = time.perf_counter()
    with ThreadPoolExecutor(max_workers=n_threads) as ex:
        done = sum(ex.map(run, orcs))
    dt = time.perf_counter() - t0
    attempts = workload.N * workload.n_chains * workload.T * done * n_mcs
    return attempts / (dt * 1e9), dt, done


def cpu_baselines(w, houd: bool) -> dict:
    """The oracle on the host: all cores (one thread per sample) and one thread, full MCS
    and Metropolis sweeps alone; the all-core full-MCS figure is the headline value."""
    import oracle

    cores = os.cpu_count() or 1
    mcs = 8 if houd else 120  # a few seconds of oracle work per figure
    v, dt, done = cpu_baseline(w, cores, mcs, cores)
    out = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "cpu": cpu_model(),
           "build": "gcc " + " ".join(oracle.CFLAGS),
           "sample": f"{done} of the {w.n_samples} samples x {mcs} MCS, one oracle thread per sample "
                     f"({dt:.1f} s wall, {dt * cores:.0f} core-s)"}
    v1, dt1, _ = cpu_baseline(w, 1, max(1, mcs // 4), 1)
    out["one_thread"] = {"value": v1, "unit": UNIT, "cores": 1, "sample": f"1 sample x {max(1, mcs // 4)} MCS "
                                                                            f"({dt1:.1f} s)"}
    vm, dtm, donem = cpu_baseline(w, cores, mcs, cores, metropolis_only=True)
    out["metropolis_only"] = {"value": vm, "unit": UNIT, "cores": cores,
                              "sample": f"{donem} samples x {mcs} Metropolis sweeps ({dtm:.1f} s)"}
    vm1, dtm1, _ = cpu_baseline(w, 1, max(1, mcs // 4), 1, metropolis_only=True)
    out["metropolis_only_one_thread"] = {"value": vm1, "unit": UNIT, "cores": 1,
                                         "sample": f"1 sample x {max(1, mcs // 4)} Metropolis sweeps ({dtm1:.1f} s)"}
    return out


def philox_ceiling(stream, attempts_per_step: int, reps: int = 5) -> dict:
    """Time the Philox-only probe (sg_probe_philox: the sweep's Philox work and nothing
    else, same launch shape) over as many words as one MCS of the workload draws; the
    median rate is the ceiling the sweep's attempts/ns is reported against."""
    import torch

    from paper_2003_04621_gb300.sgmc import probe_philox

    n_sm = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    blocks = 3 * n_sm
    out = torch.zeros(blocks * 256, dtype=torch.int32, device="cuda")
    n_sites = max(1, attempts_per_step // 64)
    probe_philox(n_sites, 1, blocks, out, stream=stream)
    ms = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        words = probe_philox(n_sites, 1, blocks, out, stream=stream)
        b.record(stream)
        b.synchronize()
        ms.append(a.elapsed_time(b))
    med = statistics.median(ms)
    return {"words_per_ns": words / (med * 1e6), "ms": med, "words": words, "blocks": blocks, "threads": 256}


def run_reference(args, ws, rank):
    """Reference arm: the CPU oracle on the host cores, same metric and workload."""
    if rank != 0:
        return
    w = WORKLOADS[args.workload]()
    import oracle
    from concurrent.futures import ThreadPoolExecutor

    oracle.build()
    cores = os.cpu_count() or 1
    samples_per_step = cores
    # one oracle per host thread, each holding one sample of the job (created untimed)
    orcs = [oracle.Oracle(oracle.OracleParams(w.ndim, w.dims, 1, w.n_chains, list(w.temps),
                                              coupling_seed=w.coupling_seed, sim_seed=w.sim_seed, sample_offset=s))
            for s in range(samples_per_step)]
    houd = bool(w.houdayer)
    with ThreadPoolExecutor(max_workers=cores) as ex:
        def step():
            list(ex.map(lambda o: o.mcs(1, houdayer=houd), orcs))

        for _ in range(args.warmup):
            step()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            step()
        dt = time.perf_counter() - t0
    total_attempts = w.N * w.n_chains * w.T * samples_per_step * args.steps
    value = total_attempts / (dt * 1e9)
    sample = f"{samples_per_step} of the {w.n_samples} samples x 1 MCS per step, one oracle thread per sample"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / max(args.steps, 1),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
        "data": "synthetic (seeded couplings and hot start)",
        "config": {"workload": w.name, "lattice": f"{w.ndim}D L={w.dims[0]} periodic", "samples": w.n_samples,
                   "chains": w.n_chains, "temps": w.T, "houdayer": bool(w.houdayer),
                   "parallelism": "cpu threads over samples"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def bench_batched(stream, steps: int, mcs_per_launch: int = 10, warmup: int = 1):
    """The uneven 3D batch (153 jobs of L = 8..32 and 16..48 temperatures) advanced
    `mcs_per_launch` MCS per CUDA-graph launch: the jobs of one lattice size and words per
    chain are swept by one resident launch (a job table in the kernel's parameters), the
    groups run as parallel branches.  Compared with (a) the same jobs advanced one after
    another through the plain per-job path (identical results), and (b) the uniform
    L=16 x 32-temperature job, all advanced the same number of MCS per launch."""
    import torch

    from paper_2003_04621_gb300 import autotune
    from paper_2003_04621_gb300.inputs import geometric_temps, workload_3d_l16, workload_batched_uneven
    from paper_2003_04621_gb300.sgmc import Batch, Simulation

    def mk(w):
        return Simulation(w.ndim, w.dims, w.n_samples, w.n_chains, list(w.temps), coupling_seed=w.coupling_seed,
                          sim_seed=w.sim_seed, sample_offset=w.sample_offset, stream=stream)

    def timed(run, n):
        a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(stream)
        run(n)
        e.record(stream)
        e.synchronize()
        return a.elapsed_time(e)

    jobs = workload_batched_uneven()
    # one launch shape per (lattice size, words per chain) group, tuned on a stand-in with
    # the group's samples and 32 or 48 temperatures; the group's largest job leads it
    groups = {}
    for w in jobs:
        groups.setdefault((w.dims[0], (w.T + 31) // 32), []).append(w)
    ordered, shapes = [], {}
    for key, ws in groups.items():
        ws.sort(key=lambda w: -w.n_samples * w.T)
        ordered.extend(ws)
    sims = [mk(w) for w in ordered]
    k = 0
    for (L, wc), ws in groups.items():
        rep = Simulation(3, (L, L, L), sum(w.n_samples for w in ws), 2, geometric_temps(0.9, 2.0, 32 * wc - 16 * (wc - 1)),
                         stream=stream)
        autotune.tune(rep, stream=stream)
        shapes[(L, wc)] = rep.launch()
        rep.close()
        for s_ in sims[k:k + len(ws)]:
            s_.set_launch(shapes[(L, wc)]["threads"], shapes[(L, wc)]["words"])
        k += len(ws)
    attempts_per_mcs = sum(w.attempts_per_sweep for w in jobs)
    # (a) the plain path: every job alone, one after another
    for s_ in sims:
        s_.run_mcs(mcs_per_launch, stream=stream)
    pms = timed(lambda n: [s_.run_mcs(mcs_per_launch, stream=stream) for _ in range(n) for s_ in sims], 1)
    plain = attempts_per_mcs * mcs_per_launch / (pms * 1e6)
    b = Batch(sims, mcs_per_launch=mcs_per_launch, stream=stream)
    b.run(warmup, stream=stream)
    ms = timed(lambda n: b.run(n, stream=stream), steps)
    b.close()
    for s_ in sims:
        s_.close()
    # (b) the uniform single-size job
    u = workload_3d_l16()
    us = mk(u)
    autotune.tune(us, stream=stream)
    us.run_mcs(mcs_per_launch, stream=stream)
    ums = timed(lambda n: [us.run_mcs(mcs_per_launch, stream=stream) for _ in range(n)], steps)
    uni = u.attempts_per_sweep * steps * mcs_per_launch / (ums * 1e6)
    us.close()
    value = attempts_per_mcs * steps * mcs_per_launch / (ms * 1e6)
    # fraction of the 32-replica words' lanes that hold a replica (the rest are masked)
    lanes = sum(w.N * w.n_samples * w.n_chains * 32 * ((w.T + 31) // 32) for w in jobs)
    return {"workload": "3D L in {8,12,16,24,32} x {2048,1024,512,128,32} samples, 16..48 temps per sample",
            "jobs": len(jobs), "value": value, "unit": UNIT, "launches": steps, "mcs_per_launch": mcs_per_launch,
            "ms_per_mcs": ms / (steps * mcs_per_launch),
            "plain_same_jobs_value": plain, "vs_plain_same_jobs": value / plain,
            "uniform_l16_value": uni, "vs_uniform_l16": value / uni,
            "lane_occupancy": attempts_per_mcs / lanes,
            "shapes": {f"L{L}_wc{wc}": v for (L, wc), v in shapes.items()},
            "launch": "per graph launch: one resident launch per (L, words per chain) group (job table), "
                      "groups in parallel"}


EXTENSIONS = ("houdayer", "gauss", "trips", "houdayer3d", "smalljob", "pairing")


def _inputs():
    from paper_2003_04621_gb300 import inputs

    return inputs


# the workloads --workload can time (the default is the headline job)
WORKLOADS = {
    "3d_l16": lambda: _inputs().workload_3d_l16(),
    "3d_l16_t40": lambda: _inputs().workload_3d_l16_t40(),
    "2d_l128_houdayer": lambda: _inputs().workload_2d_l128_houdayer(),
}


def bench_extensions(stream, steps: int = 5, only=None):
    """The rows beyond the core path, each timed with CUDA events on its own stream:
    the 2D L=128 Houdayer MCS with the single-cluster move and with the multi-cluster
    variant; the 2D L=16 Gaussian-coupling MCS; one overlap plane-sum measurement of the
    3D L=16 job; the 3D L=16 MCS with round-trip counting on and off, and with the
    cluster move on its 8 lowest temperature slots; Metropolis sweeps alone; the 3D L=16
    job with 40 temperatures with and without paired last words."""
    import torch

    from paper_2003_04621_gb300.inputs import workload_2d_l128_houdayer, workload_3d_l16
    from paper_2003_04621_gb300.sgmc import Simulation

    def timed(fn, n):
        fn(1)
        a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(stream)
        fn(n)
        e.record(stream)
        e.synchronize()
        return a.elapsed_time(e) / n

    out = {}
    want = set(only or EXTENSIONS)
    h = workload_2d_l128_houdayer()
    for mode, name in ((True, "houdayer_single"), (2, "houdayer_multicluster")) if "houdayer" in want else ():
        sim = Simulation(2, h.dims, h.n_samples, 2, list(h.temps), houdayer=mode, stream=stream)
        sim.set_launch(512, 2)
        ms = timed(lambda n: sim.run_mcs(n, stream=stream), steps)
        out[name] = {"ms_per_mcs": ms, "attempts_per_ns": h.attempts_per_sweep / (ms * 1e6),
                     "workload": h.name}
        sim.close()
    # the 2D Gaussian job (general couplings, int8 spins, fixed-point energies)
    from paper_2003_04621_gb300.inputs import gaussian_couplings_fixed, workload_2d_gauss_l16

    gw = workload_2d_gauss_l16()
    if "gauss" in want:
        sim = Simulation(2, gw.dims, gw.n_samples, 2, list(gw.temps), spin_format="int8", couplings="fixed",
                         stream=stream)
        sim.set_couplings_fixed(gaussian_couplings_fixed(gw.n_samples, gw.dims, seed=gw.coupling_seed),
                                stream=stream)
        ms = timed(lambda n: sim.run_mcs(n, stream=stream), steps)
        out["gauss_2d_l16"] = {"ms_per_mcs": ms, "attempts_per_ns": gw.attempts_per_sweep / (ms * 1e6),
                               "workload": gw.name}
        sim.close()
    u = workload_3d_l16()
    for track in (False, True) if "trips" in want else ():
        sim = Simulation(3, u.dims, u.n_samples, 2, list(u.temps), track_trips=track, stream=stream)
        sim.set_launch(256, 2)
        ms = timed(lambda n: sim.run_mcs(n, stream=stream), steps)
        out["mcs_trips_on" if track else "mcs_trips_off"] = {"ms_per_mcs": ms,
                                                             "attempts_per_ns": u.attempts_per_sweep / (ms * 1e6)}
        if not track:
            # Metropolis alone (the paper's per-update time), same resident kernel without
            # the exchange passes
            ms_sw = timed(lambda n: sim.sweep(n, stream=stream), steps)
            out["metropolis_only_l16"] = {"ms_per_sweep": ms_sw, "attempts_per_ns": u.attempts_per_sweep / (ms_sw * 1e6)}
            P = torch.empty((u.n_samples, u.T, 3, 16), dtype=torch.int32, device="cuda")
            qms = timed(lambda n: [sim.qmodes_device(P, stream=stream) for _ in range(n)], steps)
            out["qmodes_l16"] = {"ms_per_measurement": qms, "pairs": u.n_samples * u.T}
        sim.close()
    # the small int8 job (3D L=6, 8 samples x 2 chains x 12 temperatures): its 200 MCS in
    # one launch, as the whole run would be made
    if "smalljob" in want:
        from paper_2003_04621_gb300.inputs import workload_3d_l6

        w6 = workload_3d_l6()
        sim = Simulation(3, w6.dims, w6.n_samples, 2, list(w6.temps), spin_format="int8", stream=stream)
        ms = timed(lambda n: [sim.run_mcs(200, stream=stream) for _ in range(n)], steps)
        out["int8_3d_l6_200mcs"] = {"ms_per_200_mcs": ms, "us_per_mcs": ms * 5.0,
                                    "attempts_per_ns": w6.attempts_per_sweep * 200 / (ms * 1e6),
                                    "workload": w6.name + " (int8, 200 MCS per launch)"}
        sim.close()
    # the 3D L=16 job with the cluster move kept to its 8 lowest temperatures (0.9-1.1)
    if "houdayer3d" in want:
        for K in (8, 32):
            sim = Simulation(3, u.dims, u.n_samples, 2, list(u.temps), houdayer=True,
                             houdayer_slots=K if K < u.T else 0, stream=stream)
            sim.set_launch(256, 2)
            ms = timed(lambda n: sim.run_mcs(n, stream=stream), steps)
            out[f"houdayer_3d_l16_low{K}" if K < u.T else "houdayer_3d_l16_all"] = {
                "ms_per_mcs": ms, "attempts_per_ns": u.attempts_per_sweep / (ms * 1e6),
                "workload": u.name + (f"_houdayer_slots{K}" if K < u.T else "_houdayer_all_slots")}
            sim.close()
    # paired last words: the 3D L=16 job with 40 temperatures per chain, paired and not
    if "pairing" in want:
        from paper_2003_04621_gb300.inputs import workload_3d_l16_t40

        w40 = workload_3d_l16_t40()
        for on in (True, False):
            sim = Simulation(3, w40.dims, w40.n_samples, 2, list(w40.temps), stream=stream)
            sim.set_launch(256, 2)
            sim.set_pairing(on)
            ms = timed(lambda n: sim.run_mcs(n, stream=stream), steps)
            out["t40_paired" if on else "t40_unpaired"] = {"ms_per_mcs": ms,
                                                          "attempts_per_ns": w40.attempts_per_sweep / (ms * 1e6),
                                                          "workload": w40.name}
            sim.close()
    return out


SERVING_RATES = ((50.0, 200), (10.0, 30), (5.0, 30), (2.0, 20), (1.0, 15))


def bench_serving(rates=SERVING_RATES, quantum: int = 50):
    """The Poisson(seed 7) stream of jobs served by continuous batching, at each (rate per
    second, arrivals) of `rates`: the first of them is the serving workload (the first 200
    arrivals at 50/s, above the GPU's capacity, where latency is mostly time in the queue),
    the others a sweep of slower rates down to below saturation, where latency is the
    jobs' own run time.  p50/p99 latency from arrival to results on the host, jobs/s and
    served attempts/ns over the makespan."""
    import torch

    from paper_2003_04621_gb300.serve import Server, poisson_trace, summarize

    free, _total = torch.cuda.mem_get_info()
    arena = int(min(32 << 30, free // 3))

    def serve(n, r):
        server = Server(arena_bytes=arena, quantum=quantum)
        res = summarize(server.run(poisson_trace(n, rate=r, seed=7)))
        res.update({"rate_per_s": r, "graph_builds": server.graph_builds, "graph_launches": server.graph_launches,
                    "trace": f"first {n} arrivals of the Poisson({r}/s, seed 7) stream"})
        del server
        torch.cuda.synchronize()
        return res

    (r0, n0), rest = rates[0], rates[1:]
    out = serve(n0, r0)
    out.update({"arena_gb": arena / 2**30, "quantum_mcs": quantum, "rate_sweep": [serve(n, r) for r, n in rest]})
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the batched and serving measurements")
    ap.add_argument("--shape", default=None, help="fixed resident launch shape THREADSxWORDS (no autotuning)")
    ap.add_argument("--workload", default="3d_l16", choices=sorted(WORKLOADS),
                    help="3d_l16: the headline job; 3d_l16_t40: the same with 40 temperatures (paired last "
                         "words); 2d_l128_houdayer: Metropolis + Houdayer + exchange")
    ap.add_argument("--extension", action="append", choices=EXTENSIONS,
                    help="time only these extension rows (repeatable) and print them as one JSON line")
    args = ap.parse_args()
    from paper_2003_04621_gb300.shard import dist_env, max_over_ranks, weak_shard

    ws, rank, local = dist_env()

    if args.impl == "reference":
        run_reference(args, ws, rank)
        return

    import numpy as np
    import torch

    from paper_2003_04621_gb300 import build as _build
    from paper_2003_04621_gb300.inputs import workload_3d_l16
    from paper_2003_04621_gb300.sgmc import Simulation

    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    _build.build()
    if args.extension:
        print(json.dumps({"extensions": bench_extensions(torch.cuda.Stream(), steps=max(1, args.steps),
                                                         only=args.extension)}))
        return
    base = WORKLOADS[args.workload]()
    w = weak_shard(base, rank)
    stream = torch.cuda.Stream()
    kw = dict(ndim=w.ndim, dims=w.dims, n_samples=w.n_samples, n_chains=w.n_chains, temps=list(w.temps),
              coupling_seed=w.coupling_seed, sim_seed=w.sim_seed, sample_offset=w.sample_offset,
              houdayer=w.houdayer)
    sim = Simulation(stream=stream, **kw)
    attempts_per_step = w.attempts_per_sweep

    def barrier():
        if ws > 1:
            torch.distributed.barrier()

    # pick the resident kernel's launch shape on a scratch copy (results do not depend on it)
    from paper_2003_04621_gb300 import autotune

    if args.shape:
        nt, words = (int(x) for x in args.shape.lower().split("x"))
        sim.set_launch(nt, words)
    else:
        autotune.tune(sim, stream=stream)
    launch = sim.launch()
    for _ in range(max(args.warmup, 3)):
        sim.run_mcs(1)
    # the packed state (36 MB) fits in L2 (129 MB): flush L2 between timed steps
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    torch.cuda.synchronize()
    barrier()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    torch.cuda.synchronize()
    t_wall0 = time.perf_counter()
    for k in range(args.steps):
        with torch.cuda.stream(stream):
            flush.fill_(k & 0xFF)
            starts[k].record(stream)
            sim.run_mcs(1)
            ends[k].record(stream)
    torch.cuda.synchronize()
    barrier()
    wall = time.perf_counter() - t_wall0
    clk = clocks.stop()
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    total_ms = float(sum(step_ms))
    total_ms = max_over_ranks(total_ms, device="cuda")
    value = attempts_per_step * ws * args.steps / (total_ms * 1e6)
    mean_launch_ms = total_ms / args.steps

    # end to end through the public API: create from host parameters, then per step one
    # MCS and a device->host read of that step's observables (E by slot and N q) into its
    # own slot of a pinned ring; the copies run on the simulation's copy stream while the
    # next MCS runs, and the timed region ends when the last has landed
    # every rank runs its shard end to end; the whole job's time is the slowest rank's
    E = torch.empty((args.steps, w.n_samples, w.n_chains, w.T), dtype=torch.int32, pin_memory=True).numpy()
    Q = torch.empty((args.steps, w.n_samples, w.T), dtype=torch.int32, pin_memory=True).numpy()
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    sim2 = Simulation(stream=stream, **kw)
    sim2.set_launch(launch["threads"], launch["words"])
    for k in range(args.steps):
        sim2.run_mcs_measure_async(1, E[k], Q[k], stream=stream)
    sim2.measure_wait()
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(time.perf_counter() - t0, device="cuda")
    E_last, Q_last = sim2.measure(stream=stream)  # a synchronous read: the ring's last slot
    if not (np.array_equal(E_last, E[-1]) and np.array_equal(Q_last, Q[-1])):
        raise RuntimeError("asynchronous and synchronous measurements differ")
    d2h = (E[0].nbytes + Q[0].nbytes) * ws
    h2d = (w.T * 8 + w.T * 16) * ws / args.steps
    e2e = {"value": attempts_per_step * ws * args.steps / (e2e_s * 1e9), "unit": UNIT,
           "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
           "includes": "create (H2D tables, device init) + per step one MCS and a D2H read of E and q "
                       "into a pinned per-step ring (the measurement inside the MCS launch where the kernel "
                       "holds both chains, copies on the simulation's copy stream overlapping the next MCS); "
                       "timed until all have landed; whole job over all ranks (slowest rank's time)"}
    sim2.close()

    pk, pk_kind = peaks()
    sm_mhz = clk.get("sm_mhz") or pk.get("sm_max_mhz", 2070.0)
    n_sm = torch.cuda.get_device_properties(local).multi_processor_count
    # the binding bound: the Philox words the sweep must draw, one per attempt, measured
    # live by the Philox-only probe on the same launch shape
    ceiling = philox_ceiling(stream, attempts_per_step)
    kernel_rate = attempts_per_step / (mean_launch_ms * 1e6)  # attempts/ns of the timed launch
    # issue rate: lane-instructions per second at the sampled SM clock (4 schedulers x 32
    # lanes x 1 instruction per clock per SM), against the algorithmic instructions of an
    # attempt: Philox4x32-10 costs 10 rounds x (2 wide multiplies + 2 three-input xors) per
    # 4 words = 10 per attempt, plus the compare and the accept-bit insert = 12.
    instr_per_attempt = 12.0
    peak_tips = n_sm * 4 * 32 * sm_mhz * 1e6 / 1e12
    achieved_tips = attempts_per_step * instr_per_attempt / (mean_launch_ms * 1e-3) / 1e12
    hbm_eff = attempts_per_step * BYTES_PER_ATTEMPT / (mean_launch_ms * 1e-3) / 1e9
    traffic = None
    prof = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(prof):
        try:
            traffic = json.load(open(prof)).get("resident_packed_3d_l16_bytes_per_launch")
        except (OSError, ValueError):
            traffic = None
    houd = args.workload == "2d_l128_houdayer"
    # Houdayer MCS: the sweep (q bitmaps out), the seed-cluster fill, the flips with the
    # energies and the exchange
    launches_per_step = 3 if houd else 1
    line_pairs = bool(not houd and (w.T <= 16 or 32 < w.T <= 48))
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "u32", "data": "synthetic (seeded +-J couplings and hot start)",
        "config": {"workload": w.name,
                   "lattice": "2D L=128 periodic" if houd else "3D L=16 periodic",
                   "paired_last_words": line_pairs, "samples_per_gpu": w.n_samples,
                   "chains": w.n_chains, "temps": w.T,
                   "temp_range": [round(w.temps[0], 6), round(w.temps[-1], 6)], "spin_format": "packed32",
                   "step": ("one MCS = Metropolis sweep, one Houdayer move per (sample, temperature) pair, "
                            "exchange: 3 launches") if houd else
                           "one MCS = checkerboard Metropolis sweep + replica exchange, one fused launch",
                   "l2": "flushed between timed steps (256 MB write)", "parallelism": f"samples x{ws}",
                   "launch": launch},
        "gpu_launches": args.steps * launches_per_step,
        "wall_s": wall,
        "clocks": clk,
        "roofline": {"bound": "alu", "achieved": kernel_rate, "peak": ceiling["words_per_ns"], "unit": "attempts/ns",
                     "frac": kernel_rate / ceiling["words_per_ns"], "traffic": traffic if args.workload == "3d_l16" else None,
                     "kernel": (f"k_resident_packed<{w.ndim},{launch['threads']},"
                                f"{'paired last words' if line_pairs else str(launch['words'])},fused exchange>")
                     if not houd else "whole MCS (3 kernels; see profiles/)",
                     "peak_kind": "measured live: Philox-only probe (sg_probe_philox), the sweep's Philox words "
                                  f"of one MCS ({ceiling['words']}) on {ceiling['blocks']} CTAs x 256 threads, "
                                  f"median of 5: {ceiling['ms']:.4f} ms",
                     "traffic_note": "DRAM bytes of one launch (ncu, profiles/); its updated words (4 N W S bytes) "
                                     "stay dirty in L2 and are written back during the next step's L2 flush, "
                                     "outside the timed launch",
                     "issue": {"achieved": achieved_tips, "peak": peak_tips, "unit": "Tinstr/s",
                               "frac": achieved_tips / peak_tips, "instr_per_attempt": instr_per_attempt,
                               "peak_kind": f"derived: {n_sm} SMs x 128 lanes x {sm_mhz:.0f} MHz (sampled)"}},
        "hbm_effective": {"achieved_gbs": hbm_eff, "peak_gbs": pk["hbm_gbs"], "frac": hbm_eff / pk["hbm_gbs"],
                          "peak_kind": pk_kind, "bytes_per_attempt": BYTES_PER_ATTEMPT},
        "e2e": e2e,
    }
    if ws == 1 and not args.no_extras:
        line["batched"] = bench_batched(stream, steps=max(4, args.steps // 8))
        line["serving"] = bench_serving()
        line["serving"]["vs_uniform_l16"] = line["serving"]["attempts_per_ns"] / line["batched"]["uniform_l16_value"]
        line["extensions"] = bench_extensions(stream)
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baselines(w, houd)
    if rank == 0:
        print(json.dumps(line))
    if ws > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
