"""GPU parity of the streaming (global-memory) sweep path and of batches.

The streaming path stages nothing in shared memory; it takes over when a word lattice
does not fit a CTA (2D L=256 here) and can be forced on any job.  A batch captures the
MCS cycles of several uneven jobs into one CUDA graph.  Both must give exactly the
oracle's states, and a batched job exactly the state of the same job run alone.
"""
import numpy as np
import pytest

from helpers import assert_same_state, gpu_of, oracle_of
from paper_2003_04621_gb300.inputs import geometric_temps

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2003_04621_gb300 import build

    build.build()


def _okw(kw):
    return {k: v for k, v in kw.items() if k not in ("spin_format", "houdayer", "n_metro")}


@pytest.mark.parametrize("ndim,dims,T,houd", [(3, (8, 6, 4), 12, False), (2, (40, 24), 40, False),
                                              (2, (32, 16), 24, True), (3, (6, 6, 6), 33, False)])
def test_streaming_path_forced(oracle_mod, ndim, dims, T, houd):
    kw = dict(ndim=ndim, dims=dims, n_samples=3, n_chains=2, temps=geometric_temps(0.3, 2.0, T), sim_seed=23,
              houdayer=houd)
    sim, orc = gpu_of(**kw), oracle_of(oracle_mod, **_okw(kw))
    sim.set_launch(0, -1)
    assert sim.launch()["words"] == -1
    for t in range(5):
        sim.run_mcs(1)
        orc.mcs(1, houdayer=houd)
        assert_same_state(sim, orc, f"mcs {t}")
    for op in "sxsx":
        (sim.sweep if op == "s" else sim.exchange)()
        (orc.sweep if op == "s" else orc.exchange)()
        assert_same_state(sim, orc, op)


def test_streaming_path_taken_for_large_2d(oracle_mod):
    """2D L=256: a 32-replica word lattice is 256 KB, beyond a CTA's shared memory."""
    kw = dict(ndim=2, dims=(256, 256), n_samples=1, n_chains=2, temps=geometric_temps(0.5, 1.6, 16), sim_seed=4)
    sim, orc = gpu_of(**kw), oracle_of(oracle_mod, **_okw(kw))
    assert sim.launch()["words"] == -1
    for t in range(3):
        sim.run_mcs(1)
        orc.mcs(1)
        assert_same_state(sim, orc, f"mcs {t}")


def test_batch_equals_jobs_run_alone(oracle_mod):
    from paper_2003_04621_gb300.sgmc import Batch

    specs = [
        dict(ndim=3, dims=(8, 8, 8), n_samples=6, n_chains=2, temps=geometric_temps(0.9, 2.0, 20), sim_seed=1),
        dict(ndim=3, dims=(12, 12, 12), n_samples=3, n_chains=2, temps=geometric_temps(0.9, 2.0, 40), sim_seed=1,
             sample_offset=5),
        dict(ndim=2, dims=(32, 32), n_samples=2, n_chains=2, temps=geometric_temps(0.2, 1.6, 16), sim_seed=9,
             houdayer=True),
        dict(ndim=3, dims=(6, 6, 6), n_samples=4, n_chains=2, temps=geometric_temps(1.0, 2.0, 12), sim_seed=3,
             spin_format="int8"),
    ]
    batched = [gpu_of(**kw) for kw in specs]
    alone = [gpu_of(**kw) for kw in specs]
    b = Batch(batched, mcs_per_launch=2)
    b.run(3)
    for sim in alone:
        sim.run_mcs(6)
    for kw, a, s in zip(specs, alone, batched):
        assert (a.spins() == s.spins()).all()
        np.testing.assert_array_equal(a.state()[0], s.state()[0])
        np.testing.assert_array_equal(a.state()[1], s.state()[1])
        assert a.state()[2] == s.state()[2]
    # and the small ones against the oracle
    for kw, s in zip(specs, batched):
        if kw["ndim"] == 3 and kw["dims"][0] <= 8:
            orc = oracle_of(oracle_mod, **_okw(kw))
            orc.mcs(6, houdayer=bool(kw.get("houdayer")))
            assert_same_state(s, orc, f"batched {kw['dims']}")
    # a batch can be replayed after its jobs ran alone in between
    for s in batched:
        s.run_mcs(1)
    b.run(1)
    for a in alone:
        a.run_mcs(3)
    for a, s in zip(alone, batched):
        assert (a.spins() == s.spins()).all()
    b.close()


def test_batch_of_one_lattice_many_temperature_counts(oracle_mod):
    """Jobs sharing one lattice shape are swept by ONE resident launch per MCS chunk (a
    job table in the kernel's parameters), including chains of 33..48 replicas exchanged
    inside the kernel; a one-chain job forces one word per CTA for its group."""
    from paper_2003_04621_gb300.sgmc import Batch

    dims = (8, 6, 8)
    specs = [dict(ndim=3, dims=dims, n_samples=S, n_chains=2, temps=geometric_temps(0.9, 2.0, T), sim_seed=7,
                  sample_offset=off)
             for S, T, off in ((5, 12, 0), (3, 20, 5), (2, 33, 8), (4, 40, 10), (1, 48, 14))]
    specs2 = [dict(ndim=2, dims=(24, 16), n_samples=3, n_chains=2, temps=geometric_temps(0.3, 1.5, 16), sim_seed=8),
              dict(ndim=2, dims=(24, 16), n_samples=2, n_chains=1, temps=geometric_temps(0.3, 1.5, 9), sim_seed=8,
                   sample_offset=3)]
    batched = [gpu_of(**kw) for kw in specs + specs2]
    b = Batch(batched, mcs_per_launch=3)
    b.run(2)
    for kw, sim in zip(specs + specs2, batched):
        orc = oracle_of(oracle_mod, **_okw(kw))
        orc.mcs(6)
        assert_same_state(sim, orc, f"batched T={len(kw['temps'])} C={kw['n_chains']}")
    b.close()


def test_batch_of_more_jobs_than_one_table_equals_jobs_run_alone(oracle_mod):
    """More jobs of one lattice shape than one launch's job table holds (96), next to
    jobs of two other sizes: that group's resident launches run in two chunks; every job
    must equal the same job run alone."""
    from paper_2003_04621_gb300.sgmc import Batch

    rng = np.random.default_rng(5)
    specs = []
    for k in range(110):
        # 100 jobs of one group (L = 6, one word per chain): two chunks of its job table
        L = 6 if k < 100 else int(rng.choice([4, 8]))
        T = int(rng.integers(8, 33)) if k < 100 else int(rng.integers(8, 49))
        specs.append(dict(ndim=3, dims=(L, L, L), n_samples=int(rng.integers(1, 3)), n_chains=2,
                          temps=geometric_temps(0.9, 2.0, T), sim_seed=11, coupling_seed=k + 1, sample_offset=k))
    batched = [gpu_of(**kw) for kw in specs]
    alone = [gpu_of(**kw) for kw in specs]
    b = Batch(batched, mcs_per_launch=3)
    b.run(2)
    for a in alone:
        a.run_mcs(6)
    for kw, a, s in zip(specs, alone, batched):
        assert (a.spins() == s.spins()).all(), kw
        np.testing.assert_array_equal(a.state()[0], s.state()[0])
        np.testing.assert_array_equal(a.state()[1], s.state()[1])
        assert a.state()[2] == s.state()[2]
    for kw, s in list(zip(specs, batched))[::37]:
        orc = oracle_of(oracle_mod, **_okw(kw))
        orc.mcs(6)
        assert_same_state(s, orc, f"large batch L={kw['dims'][0]} T={len(kw['temps'])}")
    b.close()
