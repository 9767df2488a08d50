"""GPU parity of the Houdayer cluster move (Sec. 2.4, Eq. 10) against the oracle.

Every (sample, temperature slot) pair chooses its seed from its own Philox word and the
floor(u M / 2^32)-th q = -1 site in site order; the cluster is the seed's connected q = -1
component, grown on the GPU row by row (periodic runs, queue of rows) and by breadth-
first search in the oracle.  After every step the spins, energies, replica maps, N q and
the number of flipped sites must be identical.  The multi-cluster variant ("H", or
houdayer=2 in the MCS) exchanges every q = -1 cluster by its own coin, keyed by the
cluster's smallest site: the GPU labels all clusters by union-find over row runs, the
oracle by breadth-first search from each unlabelled site in increasing order.
"""
import numpy as np
import pytest

from helpers import assert_same_state, gpu_of, oracle_of
from paper_2003_04621_gb300.inputs import geometric_temps, workload_2d_l128_houdayer

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2003_04621_gb300 import build

    build.build()


def _okw(kw):
    return {k: v for k, v in kw.items() if k not in ("spin_format", "houdayer", "n_metro")}


def run_pair(oracle_mod, kw, ops, check_every=1):
    sim, orc = gpu_of(**kw), oracle_of(oracle_mod, **_okw(kw))
    for t, op in enumerate(ops):
        if op == "s":
            sim.sweep(1)
            orc.sweep(1)
        elif op == "h":
            sim.houdayer()
            orc.houdayer()
        elif op == "H":
            sim.houdayer_multi()
            orc.houdayer_multi()
        elif op == "x":
            sim.exchange()
            orc.exchange()
        elif op == "m":
            sim.run_mcs(1)
            orc.mcs(1, houdayer=kw.get("houdayer", False))
        if t % check_every == 0 or t == len(ops) - 1:
            assert_same_state(sim, orc, f"step {t} ({op})")
    c = orc.counters()
    assert c["error"] == 0
    assert sim.counters()["houdayer_sites"] == c["houd_flipped"]
    return sim, orc


# split=False: a handle made without the per-MCS move has no bitmap scratch and runs the
# single-CTA kernel; split=True: the handle holds the scratch and runs the split form
# (q maps per sample, one warp per pair, flips per sample).
@pytest.mark.parametrize("split", [False, True])
@pytest.mark.parametrize("dims", [(16, 16), (40, 24), (66, 4), (2, 8), (8, 2), (96, 6)])
def test_houdayer_calls_2d(oracle_mod, dims, split):
    kw = dict(ndim=2, dims=dims, n_samples=3, n_chains=2, temps=geometric_temps(0.2, 1.6, 8), sim_seed=7,
              coupling_seed=5, houdayer=split)
    run_pair(oracle_mod, kw, list("sshxshhxsxh"))


@pytest.mark.parametrize("split", [False, True])
@pytest.mark.parametrize("dims,T", [((8, 8, 8), 12), ((4, 6, 2), 32), ((16, 4, 8), 5)])
def test_houdayer_calls_3d(oracle_mod, dims, T, split):
    kw = dict(ndim=3, dims=dims, n_samples=2, n_chains=2, temps=geometric_temps(0.5, 2.5, T), sim_seed=19,
              houdayer=split)
    run_pair(oracle_mod, kw, list("shxshhx"))


def test_houdayer_mcs_2d_l128(oracle_mod):
    """2D L=128 x 24 temperatures in [0.2, 1.6], Metropolis + Houdayer + exchange per
    MCS: two samples of the 256-sample job, compared after every MCS."""
    w = workload_2d_l128_houdayer()
    kw = dict(ndim=2, dims=w.dims, n_samples=2, n_chains=2, temps=list(w.temps), sim_seed=w.sim_seed,
              coupling_seed=w.coupling_seed, sample_offset=200, houdayer=True)
    sim, orc = run_pair(oracle_mod, kw, ["m"] * 6)
    assert orc.counters()["houd_moves"] > 0


@pytest.mark.parametrize("multi", [False, True])
@pytest.mark.parametrize("ndim,dims,T", [(2, (64, 32), 24), (3, (8, 8, 8), 12), (3, (8, 6, 4), 32)])
def test_houdayer_mcs_fused_and_split_phases(oracle_mod, multi, ndim, dims, T):
    """The MCS with the move, once with its q bitmaps and flips taken by the resident
    launches around the cluster phase (two one-word chains per CTA), once with the three
    separate move kernels (one word per CTA): both equal the oracle after every call, for
    calls of one and of several MCS."""
    kw = dict(ndim=ndim, dims=dims, n_samples=3, n_chains=2, temps=geometric_temps(0.3, 1.8, T), sim_seed=11,
              coupling_seed=2, houdayer=2 if multi else True)
    states = []
    for words in (2, 1):
        sim, orc = gpu_of(**kw), oracle_of(oracle_mod, **_okw(kw))
        sim.set_launch(256, words)
        assert sim.launch()["words"] == words
        # one MCS per call, then several (the fused form then runs the move's flips, the
        # energies and the exchange inside the next MCS's sweep launch)
        for t, n in enumerate((1, 1, 3, 2, 4)):
            sim.run_mcs(n)
            orc.mcs(n, houdayer=kw["houdayer"])
            assert_same_state(sim, orc, f"words {words} call {t} ({n} MCS)")
        assert sim.counters()["houdayer_sites"] == orc.counters()["houd_flipped"]
        states.append(sim.spins().cpu().numpy())
    np.testing.assert_array_equal(states[0], states[1])


def test_houdayer_cold_percolating_clusters(oracle_mod):
    """Low temperatures and a q field of many large clusters (chains started apart)."""
    kw = dict(ndim=2, dims=(64, 32), n_samples=2, n_chains=2, temps=geometric_temps(0.05, 0.3, 6), sim_seed=3,
              houdayer=True)
    run_pair(oracle_mod, kw, ["m"] * 8)


def test_houdayer_bitmaps_in_global_scratch(oracle_mod):
    """3D L=32 x 32 temperatures: a sample's bitmaps exceed the single-CTA kernel's
    shared-memory budget, so even a handle made without the per-MCS move holds the
    scratch and runs the split form."""
    kw = dict(ndim=3, dims=(32, 32, 32), n_samples=1, n_chains=2, temps=geometric_temps(0.9, 2.0, 32),
              sim_seed=2)
    run_pair(oracle_mod, kw, ["s", "h", "x", "s", "h"])


def test_houdayer_fill_in_global_memory(oracle_mod):
    """2D 256 x 3200: one pair's q and cluster bitmaps (2 x 100 KB) exceed the fill
    kernel's shared-memory budget, so the clusters are grown in the global scratch."""
    kw = dict(ndim=2, dims=(256, 3200), n_samples=1, n_chains=2, temps=geometric_temps(0.3, 1.5, 4),
              sim_seed=4, houdayer=True)
    run_pair(oracle_mod, kw, ["m", "m", "m"], check_every=3)


def test_houdayer_full_size_sampled(oracle_mod):
    """The whole 256-sample 2D L=128 job on the GPU; two samples recomputed by the oracle."""
    w = workload_2d_l128_houdayer()
    kw = dict(ndim=2, dims=w.dims, n_samples=w.n_samples, n_chains=2, temps=list(w.temps), sim_seed=w.sim_seed,
              coupling_seed=w.coupling_seed, houdayer=True)
    sim = gpu_of(**kw)
    picks = [3, 255]
    orcs = [oracle_of(oracle_mod, **_okw(dict(kw, n_samples=1, sample_offset=s))) for s in picks]
    for t in range(3):
        sim.run_mcs(1)
        E, perm, _ = sim.state()
        Em, Q = sim.measure()
        sp = sim.spins()
        for s, o in zip(picks, orcs):
            o.mcs(1, houdayer=True)
            np.testing.assert_array_equal(E[s:s + 1], o.energies())
            np.testing.assert_array_equal(perm[s:s + 1], o.perm()[0])
            np.testing.assert_array_equal(Em[s:s + 1], o.measure()[0])
            np.testing.assert_array_equal(Q[s:s + 1], o.measure()[1])
            np.testing.assert_array_equal(sp[s:s + 1].cpu().numpy(), o.spins(), err_msg=f"spins {s} mcs {t}")
        del sp
    assert sim.counters()["near_threshold"] == 0


def test_houdayer_refused_where_unsupported():
    from paper_2003_04621_gb300.sgmc import SGError

    sim = gpu_of(ndim=2, dims=(8, 8), n_samples=1, n_chains=2, temps=geometric_temps(0.5, 2.0, 40))
    with pytest.raises(SGError) as e:
        sim.houdayer()
    assert e.value.status == 5
    one = gpu_of(ndim=2, dims=(8, 8), n_samples=1, n_chains=1, temps=[1.0, 2.0])
    with pytest.raises(SGError) as e:
        one.houdayer()
    assert e.value.status == 1


@pytest.mark.parametrize("ndim,dims,T", [(2, (16, 16), 8), (2, (40, 24), 12), (2, (66, 4), 5), (2, (2, 8), 3),
                                         (3, (8, 8, 8), 12), (3, (4, 6, 2), 32), (3, (16, 4, 8), 5)])
def test_multicluster_calls(oracle_mod, ndim, dims, T):
    kw = dict(ndim=ndim, dims=dims, n_samples=3, n_chains=2, temps=geometric_temps(0.2, 2.0, T), sim_seed=23,
              coupling_seed=6, houdayer=2)
    run_pair(oracle_mod, kw, list("sHxsHhxHs"))


def test_multicluster_mcs_2d_l128(oracle_mod):
    """The 2D L=128 x 24-temperature job with the multi-cluster variant in every MCS."""
    w = workload_2d_l128_houdayer()
    kw = dict(ndim=2, dims=w.dims, n_samples=2, n_chains=2, temps=list(w.temps), sim_seed=w.sim_seed,
              coupling_seed=w.coupling_seed, sample_offset=100, houdayer=2)
    sim, orc = run_pair(oracle_mod, kw, ["m"] * 5)
    assert orc.counters()["houd_moves"] > 0


def test_multicluster_refused_without_scratch():
    from paper_2003_04621_gb300.sgmc import SGError

    sim = gpu_of(ndim=2, dims=(8, 8), n_samples=1, n_chains=2, temps=[1.0, 2.0])  # houdayer=0: no scratch
    with pytest.raises(SGError) as e:
        sim.houdayer_multi()
    assert e.value.status == 5
    big = gpu_of(ndim=2, dims=(256, 3200), n_samples=1, n_chains=2, temps=[1.0, 2.0], houdayer=True)
    with pytest.raises(SGError) as e:  # labels beyond one CTA's shared memory
        big.houdayer_multi()
    assert e.value.status == 5


@pytest.mark.parametrize("multi", [False, True])
def test_houdayer_striped_q_field(oracle_mod, multi):
    """Chains planted to differ on every odd column: N/2 q = -1 sites in L0/2 rings, with
    more run-graph edges than the labelling keeps in shared memory, so the labels are
    built from edges recomputed every round."""
    kw = dict(ndim=2, dims=(32, 16), n_samples=2, n_chains=2, temps=geometric_temps(0.4, 1.5, 4), sim_seed=9,
              houdayer=2 if multi else True)
    sim, orc = gpu_of(**kw), oracle_of(oracle_mod, **_okw(kw))
    bits = orc.spins()
    x = np.arange(32 * 16) % 32
    stripe = (x & 1).astype(np.uint8)
    perm = orc.perm()[0]
    for s in range(2):
        for k in range(4):
            a, b = perm[s, 0, k], perm[s, 1, k]
            bits[s, 1, b] = bits[s, 0, a] ^ stripe
    orc.set_spins(bits)
    sim.set_spins(bits)
    assert_same_state(sim, orc, "planted")
    op = "H" if multi else "h"
    run_pair_from(sim, orc, [op, op, "x", op])


def run_pair_from(sim, orc, ops):
    for t, op in enumerate(ops):
        if op == "h":
            sim.houdayer()
            orc.houdayer()
        elif op == "H":
            sim.houdayer_multi()
            orc.houdayer_multi()
        elif op == "x":
            sim.exchange()
            orc.exchange()
        assert_same_state(sim, orc, f"step {t} ({op})")


# the move kept to the K lowest temperature slots (houdayer_slots = K): both kernels
# (single-CTA and split), both variants, K below, at and (for 0) equal to T
@pytest.mark.parametrize("split", [False, True])
@pytest.mark.parametrize("K", [1, 3, 8])
def test_houdayer_low_slots_2d(oracle_mod, K, split):
    kw = dict(ndim=2, dims=(24, 16), n_samples=3, n_chains=2, temps=geometric_temps(0.2, 1.6, 8), sim_seed=23,
              coupling_seed=3, houdayer=split, houdayer_slots=K)
    run_pair(oracle_mod, kw, list("sxsxhsxhhx"))


@pytest.mark.parametrize("multi", [False, True])
def test_houdayer_low_slots_mcs_3d(oracle_mod, multi):
    kw = dict(ndim=3, dims=(8, 8, 8), n_samples=2, n_chains=2, temps=geometric_temps(0.5, 2.5, 12), sim_seed=29,
              houdayer=2 if multi else True, houdayer_slots=4)
    run_pair(oracle_mod, kw, ["m"] * 8)


@pytest.mark.parametrize("multi", [False, True])
def test_houdayer_low_slots_multi_mcs_calls(oracle_mod, multi):
    """The move kept to 4 of 12 slots, in calls of several MCS: between two moves the
    sweep launch also takes the previous move's flips, the energies and the exchange."""
    kw = dict(ndim=3, dims=(8, 8, 8), n_samples=2, n_chains=2, temps=geometric_temps(0.5, 2.5, 12), sim_seed=31,
              houdayer=2 if multi else True, houdayer_slots=4)
    sim, orc = gpu_of(**kw), oracle_of(oracle_mod, **_okw(kw))
    for t, n in enumerate((3, 1, 4)):
        sim.run_mcs(n)
        orc.mcs(n, houdayer=kw["houdayer"])
        assert_same_state(sim, orc, f"call {t} ({n} MCS)")
    assert sim.counters()["houdayer_sites"] == orc.counters()["houd_flipped"]
