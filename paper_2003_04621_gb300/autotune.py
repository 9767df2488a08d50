"""Autotuner for the resident sweep kernel's launch shape.

For a workload it times every accepted (threads per CTA, words per CTA) shape with CUDA
events on a scratch simulation of the same lattice, temperatures and sample count, and
returns the fastest.  Results do not depend on the shape (the kernels are bit-exact for
every shape), so the choice is a pure performance decision; it is cached per
(ndim, dims, temperatures, chains, samples) for the process.
"""
from __future__ import annotations

from typing import Dict, Tuple

SHAPES = [(nt, w) for w in (2, 1) for nt in (64, 128, 256, 512, 1024)]
_cache: Dict[Tuple, Tuple[int, int]] = {}


def key_of(sim) -> Tuple:
    return (sim.ndim, sim.dims, sim.T, sim.C, sim.S)


def tune(sim, mcs_per_trial: int = 3, trials: int = 3, stream=None) -> Dict:
    """Time each launch shape on a scratch copy of `sim`'s workload and apply the best
    one to `sim`.  Returns {(threads, words): ms per MCS}."""
    import torch

    from .sgmc import SGError, Simulation

    k = key_of(sim)
    timings = {}
    p = sim.params
    temps = list(sim._temps)
    scratch = Simulation(sim.ndim, sim.dims, sim.S, sim.C, temps, coupling_seed=p.coupling_seed,
                         sim_seed=p.sim_seed ^ 0x5A5A, spin_format="packed", stream=stream)
    st = stream if stream is not None else torch.cuda.current_stream()
    for nt, w in SHAPES:
        try:
            scratch.set_launch(nt, w)
        except SGError:
            continue
        scratch.run_mcs(1, stream=stream)  # warm up this shape
        best = None
        for _ in range(trials):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(st)
            scratch.run_mcs(mcs_per_trial, stream=stream)
            b.record(st)
            b.synchronize()
            ms = a.elapsed_time(b) / mcs_per_trial
            best = ms if best is None else min(best, ms)
        timings[(nt, w)] = best
    scratch.close()
    if timings:
        choice = min(timings, key=timings.get)
        _cache[k] = choice
        sim.set_launch(*choice)
    return timings


def apply_cached(sim) -> bool:
    choice = _cache.get(key_of(sim))
    if choice is None:
        return False
    sim.set_launch(*choice)
    return True
