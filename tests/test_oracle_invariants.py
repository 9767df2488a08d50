"""Exact invariants of the oracle's dynamics (bitwise, any run length).

* Gauge covariance of Eq. 1: with tau_i = +-1, couplings J'_ij = tau_i J_ij tau_j and
  start s'(0) = tau s(0) under the same random stream, s'(t) = tau s(t) and the
  energies, replica maps and Houdayer clusters are identical at every t (dE, E and q
  are gauge invariant).  Catches any bond looked up at the wrong site or direction.
* Global-flip covariance: s(0) -> -s(0) gives s(t) -> -s(t).
* Energies kept incrementally equal energies recomputed from Eq. 1.
* Houdayer move (Sec. 2.4): E1 + E2 conserved, the overlap field q unchanged, and the
  flipped set of every pair is exactly one connected component of the q = -1 sites
  (checked with networkx on the periodic lattice graph).  Over repeated moves on a
  fixed q-field the chosen component is hit with frequency size / M (uniform seed).
* Multi-cluster variant: E1 + E2 conserved, q unchanged, the flipped set of every pair
  is a union of whole q = -1 components, and each component is flipped with
  probability 1/2 (binomial over many components).
* Replica maps stay mutually inverse permutations.
* Samples are independent and keyed by their job-wide index: a shard of samples
  evolves exactly as the same samples inside the whole job.
"""
import math

import numpy as np
import pytest

from paper_2003_04621_gb300.inputs import geometric_temps


def make(oracle_mod, ndim, dims, S, C, temps, **kw):
    return oracle_mod.Oracle(oracle_mod.OracleParams(ndim, dims, S, C, list(temps), **kw))


def coords_of(dims):
    d = len(dims)
    N = int(np.prod(dims))
    i = np.arange(N)
    out = []
    stride = 1
    for a in range(d):
        out.append((i // stride) % dims[a])
        stride *= dims[a]
    return out


def forward_neighbour(dims, mu):
    c = coords_of(dims)
    c[mu] = (c[mu] + 1) % dims[mu]
    stride = 1
    idx = 0
    for a in range(len(dims)):
        idx = idx + c[a] * stride
        stride *= dims[a]
    return idx


@pytest.mark.parametrize("ndim,dims,houd", [(2, (8, 6), True), (3, (4, 4, 6), True), (3, (2, 4, 2), False),
                                            (2, (8, 6), 2)])
def test_gauge_covariance(oracle_mod, ndim, dims, houd):
    temps = geometric_temps(0.5, 2.0, 6)
    a = make(oracle_mod, ndim, dims, 3, 2, temps, coupling_seed=5, sim_seed=8)
    b = make(oracle_mod, ndim, dims, 3, 2, temps, coupling_seed=5, sim_seed=8)
    N = a.N
    rng = np.random.default_rng(0)
    tau = rng.choice([-1, 1], size=(3, N)).astype(np.int64)
    J = a.couplings().astype(np.int64)
    Jg = np.empty_like(J)
    for mu in range(ndim):
        nb = forward_neighbour(dims, mu)
        Jg[:, :, mu] = tau * J[:, :, mu] * tau[:, nb]
    b.set_couplings(Jg.astype(np.int8))
    s0 = 1 - 2 * a.spins().astype(np.int64)
    sg = s0 * tau[:, None, None, :]
    b.set_spins(((1 - sg) // 2).astype(np.uint8))
    np.testing.assert_array_equal(a.energies(), b.energies())
    for _ in range(25):
        a.mcs(1, houdayer=houd)
        b.mcs(1, houdayer=houd)
        sa = 1 - 2 * a.spins().astype(np.int64)
        sb = 1 - 2 * b.spins().astype(np.int64)
        np.testing.assert_array_equal(sb, sa * tau[:, None, None, :])
        np.testing.assert_array_equal(a.energies(), b.energies())
        np.testing.assert_array_equal(a.perm()[0], b.perm()[0])
    assert a.counters()["houd_flipped"] == b.counters()["houd_flipped"]


def test_global_flip_covariance(oracle_mod):
    temps = geometric_temps(0.4, 1.6, 8)
    a = make(oracle_mod, 2, (10, 8), 2, 2, temps, sim_seed=21)
    b = make(oracle_mod, 2, (10, 8), 2, 2, temps, sim_seed=21)
    b.set_spins(1 - a.spins())
    for _ in range(20):
        a.mcs(1, houdayer=True)
        b.mcs(1, houdayer=True)
        np.testing.assert_array_equal(b.spins(), 1 - a.spins())
        np.testing.assert_array_equal(a.energies(), b.energies())


def test_incremental_energy_and_maps(oracle_mod):
    temps = geometric_temps(0.3, 1.6, 10)
    o = make(oracle_mod, 2, (12, 10), 3, 2, temps, sim_seed=2)
    for _ in range(40):
        o.sweep(1)
        o.houdayer()
        o.exchange()
        assert o.check_energies() == 0
        perm, slot = o.perm()
        for s in range(3):
            for c in range(2):
                assert sorted(perm[s, c].tolist()) == list(range(10))
                np.testing.assert_array_equal(slot[s, c][perm[s, c]], np.arange(10))
    assert o.counters()["error"] == 0


def _q_components(dims, qneg):
    nx = pytest.importorskip("networkx")
    G = nx.grid_graph(dim=list(dims), periodic=True)  # nodes are (.., y, x) tuples
    strides = [int(np.prod(dims[:a])) for a in range(len(dims))]

    def idx(node):
        c = tuple(reversed(node))
        return sum(c[a] * strides[a] for a in range(len(dims)))

    keep = [n for n in G.nodes() if qneg[idx(n)]]
    H = G.subgraph(keep)
    return [frozenset(idx(n) for n in comp) for comp in nx.connected_components(H)]


@pytest.mark.parametrize("ndim,dims", [(2, (8, 8)), (3, (4, 4, 4)), (2, (12, 6))])
def test_houdayer_flips_one_whole_component(oracle_mod, ndim, dims):
    temps = geometric_temps(0.4, 2.0, 5)
    o = make(oracle_mod, ndim, dims, 2, 2, temps, sim_seed=13)
    o.mcs(3)
    for _ in range(6):
        before = o.spins()
        E0 = o.energies()
        perm, _ = o.perm()
        o.houdayer()
        after = o.spins()
        E1 = o.energies()
        for s in range(2):
            for k in range(len(temps)):
                a, b = perm[s, 0, k], perm[s, 1, k]
                qneg0 = before[s, 0, a] != before[s, 1, b]
                qneg1 = after[s, 0, a] != after[s, 1, b]
                np.testing.assert_array_equal(qneg0, qneg1)  # q-field unchanged
                flipped = np.nonzero(before[s, 0, a] != after[s, 0, a])[0]
                np.testing.assert_array_equal(flipped, np.nonzero(before[s, 1, b] != after[s, 1, b])[0])
                assert E0[s, 0, a] + E0[s, 1, b] == E1[s, 0, a] + E1[s, 1, b]
                if qneg0.sum() == 0:
                    assert flipped.size == 0
                    continue
                comps = _q_components(dims if ndim == 3 else dims, qneg0)
                assert frozenset(flipped.tolist()) in comps
        o.sweep(1)


def test_houdayer_seed_is_uniform_over_q_minus_sites(oracle_mod):
    """Without Metropolis the q-field is fixed, so repeated moves pick component c with
    probability |c| / M."""
    temps = [0.8]
    o = make(oracle_mod, 2, (6, 6), 1, 2, temps, sim_seed=31)
    bits = o.spins()
    # chain 1 differs from chain 0 on three separated clusters of 1, 3 and 6 sites
    diff = np.zeros(36, bool)
    diff[[0]] = True  # (x, y) = (0, 0)
    diff[[3, 4, 9]] = True  # (3, 0), (4, 0), (3, 1)
    diff[[20, 21, 22, 26, 27, 28]] = True  # x = 2..4 on rows y = 3 and 4
    bits[0, 1, 0] = bits[0, 0, 0] ^ diff
    o.set_spins(bits)
    qneg = bits[0, 0, 0] != bits[0, 1, 0]
    comps = _q_components((6, 6), qneg)
    M = int(qneg.sum())
    assert sorted(len(c) for c in comps) == [1, 3, 6]
    hits = {c: 0 for c in comps}
    n = 6000
    for _ in range(n):
        before = o.spins()[0, 0, 0].copy()
        o.houdayer()
        flipped = frozenset(np.nonzero(before != o.spins()[0, 0, 0])[0].tolist())
        hits[flipped] += 1
    for c, h in hits.items():
        p = len(c) / M
        assert abs(h / n - p) < 4.5 * math.sqrt(p * (1 - p) / n) + 1e-12, (len(c), h / n, p)


def test_sample_shards_evolve_like_the_whole_job(oracle_mod):
    temps = geometric_temps(0.5, 1.5, 6)
    whole = make(oracle_mod, 2, (8, 8), 4, 2, temps, sim_seed=77, coupling_seed=3)
    lo = make(oracle_mod, 2, (8, 8), 2, 2, temps, sim_seed=77, coupling_seed=3, sample_offset=0)
    hi = make(oracle_mod, 2, (8, 8), 2, 2, temps, sim_seed=77, coupling_seed=3, sample_offset=2)
    for o in (whole, lo, hi):
        o.mcs(15, houdayer=True)
    np.testing.assert_array_equal(whole.spins(), np.concatenate([lo.spins(), hi.spins()]))
    np.testing.assert_array_equal(whole.measure()[0], np.concatenate([lo.measure()[0], hi.measure()[0]]))
    np.testing.assert_array_equal(whole.measure()[1], np.concatenate([lo.measure()[1], hi.measure()[1]]))


def test_measure_overlap_definition(oracle_mod):
    """N q of Eq. 4 between the chain-0 and chain-1 replicas at the same slot."""
    temps = geometric_temps(0.5, 1.5, 4)
    o = make(oracle_mod, 3, (4, 4, 4), 2, 2, temps)
    o.mcs(5)
    E, NQ = o.measure()
    s = 1 - 2 * o.spins().astype(np.int64)
    perm, _ = o.perm()
    En = o.energies()
    for smp in range(2):
        for k in range(4):
            a, b = perm[smp, 0, k], perm[smp, 1, k]
            assert NQ[smp, k] == int((s[smp, 0, a] * s[smp, 1, b]).sum())
            assert E[smp, 0, k] == En[smp, 0, a] and E[smp, 1, k] == En[smp, 1, b]


@pytest.mark.parametrize("ndim,dims", [(2, (8, 8)), (3, (4, 4, 4)), (2, (12, 6))])
def test_multicluster_move_flips_whole_components_by_coins(oracle_mod, ndim, dims):
    temps = geometric_temps(0.4, 2.0, 5)
    o = make(oracle_mod, ndim, dims, 3, 2, temps, sim_seed=17)
    o.mcs(3)
    n_comp = n_flip = 0
    for _ in range(12):
        before = o.spins()
        E0 = o.energies()
        perm, _ = o.perm()
        o.houdayer_multi()
        after = o.spins()
        E1 = o.energies()
        for s in range(3):
            for k in range(len(temps)):
                a, b = perm[s, 0, k], perm[s, 1, k]
                qneg0 = before[s, 0, a] != before[s, 1, b]
                np.testing.assert_array_equal(qneg0, after[s, 0, a] != after[s, 1, b])
                flipped = before[s, 0, a] != after[s, 0, a]
                np.testing.assert_array_equal(flipped, before[s, 1, b] != after[s, 1, b])
                assert E0[s, 0, a] + E0[s, 1, b] == E1[s, 0, a] + E1[s, 1, b]
                assert not (flipped & ~qneg0).any()  # only q = -1 sites change
                for comp in _q_components(dims, qneg0):
                    idx = np.array(sorted(comp))
                    got = flipped[idx]
                    assert got.all() or not got.any()  # a whole component or none of it
                    n_comp += 1
                    n_flip += int(got.all())
        o.sweep(1)
    assert o.counters()["error"] == 0
    assert n_comp > 200
    p = n_flip / n_comp
    assert abs(p - 0.5) < 4.5 * math.sqrt(0.25 / n_comp), (n_flip, n_comp)


@pytest.mark.parametrize("multi", [False, True])
def test_houdayer_slot_restriction(oracle_mod, multi):
    """The move restricted to the K lowest temperature slots equals the full move on the
    pairs at slots k < K and leaves the pairs at k >= K alone; slots, not replica
    indices, decide (the replica maps are scrambled by exchanges first)."""
    temps = geometric_temps(0.3, 1.6, 8)
    K = 3
    full = make(oracle_mod, 2, (8, 6), 3, 2, temps, sim_seed=11)
    low = make(oracle_mod, 2, (8, 6), 3, 2, temps, sim_seed=11, houdayer_slots=K)
    full.mcs(40)
    low.mcs(40)
    before = full.spins()
    assert np.array_equal(before, low.spins())
    perm, _ = full.perm()
    assert any(not np.array_equal(perm[s, c], np.arange(8)) for s in range(3) for c in range(2))
    for o in (full, low):
        o.houdayer_multi() if multi else o.houdayer()
    sf, sl = full.spins(), low.spins()
    moved_high = 0
    expect_moves = 0
    for s in range(3):
        for k in range(8):
            ja, jb = perm[s, 0, k], perm[s, 1, k]
            if k < K:
                assert np.array_equal(sl[s, 0, ja], sf[s, 0, ja]) and np.array_equal(sl[s, 1, jb], sf[s, 1, jb])
                expect_moves += int(np.any(before[s, 0, ja] != before[s, 1, jb]))
            else:
                assert np.array_equal(sl[s, 0, ja], before[s, 0, ja]) and np.array_equal(sl[s, 1, jb], before[s, 1, jb])
                moved_high += int(not np.array_equal(sf[s, 0, ja], before[s, 0, ja]))
    assert moved_high > 0  # the full move did act on the excluded slots
    c = low.counters()
    assert c["houd_moves"] == expect_moves and c["error"] == 0
    assert low.check_energies() == 0
