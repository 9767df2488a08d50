"""Host logic of the continuous-batching server (no GPU): the first-fit arena allocator
over one buffer, the Poisson job trace, and the latency summary."""
import numpy as np

from paper_2003_04621_gb300.serve import Arena, JobResult, poisson_trace, summarize


def test_arena_first_fit_alignment_and_coalescing():
    a = Arena(10 * 256 + 100, device="cpu")
    assert a.capacity == 10 * 256 and a.base % 256 == 0 and a.free_bytes == a.capacity
    x = a.alloc(1)        # rounds up to one 256-byte granule
    y = a.alloc(513)      # three granules
    z = a.alloc(256)
    assert (x, y, z) == (0, 256, 4 * 256)
    assert a.free_bytes == 5 * 256
    assert a.alloc(6 * 256) is None  # more than what is left
    a.free(y, 513)
    assert a.alloc(2 * 256) == 256  # first fit reuses the hole
    a.free(256, 2 * 256)
    a.free(x, 1)
    a.free(z, 256)
    # every hole merged back into one block
    assert a.free_bytes == a.capacity and a.alloc(a.capacity) == 0


def test_arena_random_alloc_free_never_overlaps():
    rng = np.random.default_rng(3)
    a = Arena(64 * 256, device="cpu")
    live = {}
    for _ in range(500):
        if live and rng.random() < 0.45:
            off = list(live)[rng.integers(len(live))]
            a.free(off, live.pop(off))
        else:
            n = int(rng.integers(1, 6 * 256))
            off = a.alloc(n)
            if off is not None:
                live[off] = n
        spans = sorted((o, o + ((n + 255) // 256) * 256) for o, n in live.items())
        assert all(e0 <= s1 for (_, e0), (s1, _) in zip(spans, spans[1:]))
        assert all(0 <= s and e <= a.capacity for s, e in spans)
        assert a.free_bytes + sum(e - s for s, e in spans) == a.capacity


def test_poisson_trace_is_seeded_and_shaped():
    t1, t2 = poisson_trace(200, rate=50.0, seed=7), poisson_trace(200, rate=50.0, seed=7)
    assert [(j.arrival, j.dims, j.n_samples, j.n_mcs) for j in t1] == [(j.arrival, j.dims, j.n_samples, j.n_mcs)
                                                                       for j in t2]
    arr = np.array([j.arrival for j in t1])
    assert np.all(np.diff(arr) > 0)
    # mean inter-arrival 1/rate within a few standard errors (exponential, 200 draws)
    gaps = np.diff(np.concatenate([[0.0], arr]))
    assert abs(gaps.mean() - 1 / 50.0) < 4 * (1 / 50.0) / np.sqrt(len(gaps))
    for j in t1:
        assert len(j.dims) in (2, 3) and all(L % 2 == 0 for L in j.dims)
        assert 16 <= j.n_samples <= 256 and 16 <= len(j.temps) <= 40
        assert j.n_mcs % 100 == 0 and 500 <= j.n_mcs <= 5000


def test_summary_percentiles():
    res = [JobResult(i, arrival=float(i), admitted=float(i), finished=float(i) + 1.0 + i, attempts=10**9,
                     E=np.zeros(1), Q=np.zeros(1)) for i in range(5)]
    s = summarize(res)
    lat = np.array([1.0 + i for i in range(5)])
    assert s["jobs"] == 5 and s["p50_s"] == np.percentile(lat, 50) and s["p99_s"] == np.percentile(lat, 99)
    assert abs(s["makespan_s"] - (4 + 5.0)) < 1e-12 and abs(s["attempts_per_ns"] - 5 * 10**9 / (9.0 * 1e9)) < 1e-12
