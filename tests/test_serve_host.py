"""Host logic of the continuous-batching server (no GPU): the first-fit arena allocator
over one buffer, the Poisson job trace, the latency summary, and the scheduler run
against a host fake of the device."""
import numpy as np

from paper_2003_04621_gb300.inputs import geometric_temps
from paper_2003_04621_gb300.serve import Arena, JobResult, JobSpec, Server, poisson_trace, summarize


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
        assert 500 <= j.n_mcs <= 5000
    assert any(j.n_mcs % 100 for j in t1)  # sweep counts are not rounded to a quantum


def test_summary_percentiles():
    res = [JobResult(i, arrival=float(i), admitted=float(i), finished=float(i) + 1.0 + i, attempts=10**9,
                     E=np.zeros(1), Q=np.zeros(1)) for i in range(5)]
    s = summarize(res)
    lat = np.array([1.0 + i for i in range(5)])
    assert s["jobs"] == 5 and s["p50_s"] == np.percentile(lat, 50) and s["p99_s"] == np.percentile(lat, 99)
    assert abs(s["makespan_s"] - (4 + 5.0)) < 1e-12 and abs(s["attempts_per_ns"] - 5 * 10**9 / (9.0 * 1e9)) < 1e-12


class FakeSim:
    """A job as the scheduler sees it: its MCS so far, a launch shape, a measurement."""

    def __init__(self, spec, log):
        self.spec, self.log = spec, log
        self.S, self.C, self.T, self.N = spec.n_samples, 2, len(spec.temps), int(np.prod(spec.dims))
        self.mcs = 0
        self.closed = False

    def launch(self):
        return {"threads": 256, "words": 2, "smem": 0}

    def measure(self, stream=None):
        return np.array([self.mcs]), np.array([self.spec.job_id])

    def close(self):
        self.closed = True


class FakeEvent:
    """Completes after a fixed number of polls (the device finishing in its own time)."""

    def __init__(self, log, polls=3):
        self.left, self.log = polls, log

    def query(self):
        self.left -= 1
        return self.left <= 0


class FakeBatch:
    def __init__(self, sims, q, log):
        self.sims, self.q, self.log, self.closed = list(sims), q, log, False
        log["builds"].append((tuple(s.spec.job_id for s in sims), q))

    def run(self, n, stream=None):
        assert not self.closed and n == 1
        for s in self.sims:
            assert not s.closed
            s.mcs += self.q
        self.log["resident"].append(sum(s.S for s in self.sims))

    def close(self):
        self.closed = True


class FakeBackend:
    def __init__(self):
        self.log = {"builds": [], "resident": [], "events": []}

    def stream(self):
        return object()

    def event(self, stream):
        ev = FakeEvent(self.log)
        self.log["events"].append(ev)
        return ev

    def n_sm(self):
        return 4

    def arena(self, nbytes):
        return Arena(nbytes, device="cpu")

    def query_bytes(self, spec):
        return spec.n_samples * 1000

    def simulation(self, spec, ptr, nbytes, stream):
        return FakeSim(spec, self.log)

    def batch(self, sims, q, stream):
        return FakeBatch(sims, q, self.log)

    def synchronize(self):
        pass


def test_scheduler_gives_every_job_exactly_its_mcs():
    rng = np.random.default_rng(11)
    trace = [JobSpec(k, 3, (8, 8, 8), int(rng.integers(16, 64)), geometric_temps(0.9, 2.0, 20),
                     int(rng.integers(0, 400)), arrival=0.0005 * k) for k in range(40)]
    dev = FakeBackend()
    server = Server(arena_bytes=200 * 1000, quantum=100, max_ctas=150, backend=dev)
    results = server.run(trace)
    assert sorted(r.job_id for r in results) == list(range(40))
    for r in results:
        assert int(r.E[0]) == trace[r.job_id].n_mcs  # exactly n_mcs, whatever the quantum
        assert r.finished >= r.admitted >= r.arrival - 1e-9
    # every replay ran at most one quantum; a short replay only where some job had fewer left
    assert all(q <= 100 for _, q in dev.log["builds"])
    assert any(q < 100 for _, q in dev.log["builds"])
    # the arena held the resident jobs, and admission stopped at the GPU's width (150
    # sweep CTAs, i.e. 150 samples of two one-word chains) unless a single job exceeds it
    assert max(dev.log["resident"]) <= 150 + 64
    assert server.arena.free_bytes == server.arena.capacity
