"""Serving: continuous batching keeps every job's results identical to running it alone.

Small jobs arrive over a few hundredths of a second into an arena that holds only some
of them, so jobs wait, are admitted as others finish, and share graph launches with
different partners; their sweep counts are not all multiples of the scheduling quantum.
Each job's final E by slot and N q must equal those of the same job simulated on its
own for exactly its number of MCS.
"""
import numpy as np
import pytest

from paper_2003_04621_gb300.inputs import geometric_temps

pytestmark = pytest.mark.gpu


def small_trace():
    from paper_2003_04621_gb300.serve import JobSpec

    # sweep counts that are and are not multiples of the quantum (100), one job with none,
    # and one lattice streamed from global memory (240 KB per word lattice)
    specs = [
        (3, (8, 8, 8), 40, 20, 250), (2, (48, 48), 30, 16, 200), (3, (12, 12, 12), 20, 36, 137),
        (2, (64, 32), 24, 24, 300), (3, (6, 6, 6), 64, 12, 401), (2, (32, 32), 50, 40, 37),
        (3, (10, 10, 10), 16, 28, 200), (2, (16, 16), 8, 8, 0), (2, (256, 240), 2, 8, 30),
    ]
    jobs = []
    for k, (d, dims, S, T, mcs) in enumerate(specs):
        tmin, tmax = (0.9, 2.0) if d == 3 else (0.2, 1.6)
        jobs.append(JobSpec(k, d, dims, S, geometric_temps(tmin, tmax, T), mcs, arrival=0.005 * k,
                            coupling_seed=100 + k, sim_seed=200 + k))
    return jobs


def test_served_results_equal_jobs_run_alone():
    import torch

    from paper_2003_04621_gb300 import build
    from paper_2003_04621_gb300.serve import Server, summarize
    from paper_2003_04621_gb300.sgmc import Simulation, make_params, query_bytes

    build.build()
    trace = small_trace()
    sizes = []
    for j in trace:
        p, _t = make_params(j.ndim, j.dims, j.n_samples, 2, list(j.temps))
        sizes.append(query_bytes(p))
    server = Server(arena_bytes=int(2.2 * max(sizes)), quantum=100)
    results = server.run(trace)
    assert sorted(r.job_id for r in results) == list(range(len(trace)))
    assert server.graph_builds > 2  # the resident set changed as jobs came and went
    for r in results:
        j = trace[r.job_id]
        alone = Simulation(j.ndim, j.dims, j.n_samples, 2, list(j.temps), coupling_seed=j.coupling_seed,
                           sim_seed=j.sim_seed)
        alone.run_mcs(j.n_mcs)
        assert alone.state()[2][1] == j.n_mcs
        E, Q = alone.measure()
        np.testing.assert_array_equal(E, r.E)
        np.testing.assert_array_equal(Q, r.Q)
        assert r.finished >= r.admitted >= r.arrival - 1e-9
    s = summarize(results)
    assert s["p99_s"] >= s["p50_s"] > 0
    torch.cuda.synchronize()
