"""Statistical pins for the oracle's dynamics against exact enumeration.

The Markov chain of Sec. 2.2/2.4 (Metropolis sweeps, replica exchange by Eq. 5,
Houdayer moves by Eq. 10) must sample the Boltzmann distribution.  On lattices small
enough to enumerate all 2^N states (2D 4x4, 3D 2x2x4, 2x2x2 and 2x2x3, the last in the
sequential typewriter order since an odd extent has no checkerboard), the oracle's
time averages of E and of the specific heat C = beta^2 (<E^2> - <E>^2) / N must agree
with the exact values within their statistical errors (bins of consecutive MCS,
jackknife for C).  The replica-exchange acceptance per pair must equal its exact
expectation, and the Metropolis acceptance of each dE class must equal the
threshold over 2^32 (an exactly binomial test, since every attempt draws a fresh
counter-based word).  A wrong sign in dE or in delta, a wrong threshold, a transposed
replica map or a biased cluster move fails one of these.
"""
import math

import numpy as np
import pytest

TOL_SIGMA = 4.5


def exact_moments(hist, d, N, beta):
    e = (np.arange(hist.size) - d * N).astype(np.float64)
    nz = hist > 0
    x = -beta * e[nz] + np.log(hist[nz].astype(np.float64))
    w = np.exp(x - x.max())
    w /= w.sum()
    m1 = (w * e[nz]).sum()
    m2 = (w * e[nz] ** 2).sum()
    return m1, m2


def exact_energy_pmf(hist, d, N, beta):
    e = (np.arange(hist.size) - d * N).astype(np.float64)
    nz = np.nonzero(hist)[0]
    x = -beta * e[nz] + np.log(hist[nz].astype(np.float64))
    w = np.exp(x - x.max())
    return e[nz], w / w.sum()


def check_against_enumeration(o, hist, temps, sE, sE2, label):
    d, N = o.d, o.N
    nb = sE.shape[1]
    for k, T in enumerate(temps):
        beta = 1.0 / T
        m1, m2 = exact_moments(hist, d, N, beta)
        means = sE[k]
        mean = means.mean()
        err = means.std(ddof=1) / math.sqrt(nb)
        assert abs(mean - m1) < TOL_SIGMA * err + 1e-9, (label, T, mean, m1, err)
        # specific heat, jackknife over bins
        c_exact = beta**2 * (m2 - m1**2) / N
        tot1, tot2 = sE[k].sum(), sE2[k].sum()
        jk = []
        for b in range(nb):
            a1 = (tot1 - sE[k, b]) / (nb - 1)
            a2 = (tot2 - sE2[k, b]) / (nb - 1)
            jk.append(beta**2 * (a2 - a1**2) / N)
        jk = np.array(jk)
        c_all = beta**2 * (tot2 / nb - (tot1 / nb) ** 2) / N
        c_err = math.sqrt((nb - 1) / nb * ((jk - jk.mean()) ** 2).sum())
        assert abs(c_all - c_exact) < TOL_SIGMA * c_err + 1e-9, (label, T, c_all, c_exact, c_err)


CASES = [
    # label, ndim, dims, temps, n_mcs, houdayer, pt
    ("2d4x4_metropolis", 2, (4, 4), [0.7, 1.1, 1.6, 2.5], 120_000, False, False),
    ("2d4x4_pt", 2, (4, 4), [0.5, 0.8, 1.2, 1.8], 120_000, False, True),
    ("2d4x4_pt_houdayer", 2, (4, 4), [0.5, 0.8, 1.2, 1.8], 120_000, True, True),
    ("3d2x2x4_pt", 3, (2, 2, 4), [0.8, 1.2, 1.8, 2.6], 120_000, False, True),
    ("3d2x2x4_pt_houdayer", 3, (2, 2, 4), [0.8, 1.2, 1.8, 2.6], 120_000, True, True),
    ("3d2x2x2_metropolis", 3, (2, 2, 2), [0.6, 1.0, 2.0], 150_000, False, False),
    # the multi-cluster variant of the move (houdayer = 2)
    ("2d4x4_pt_multicluster", 2, (4, 4), [0.5, 0.8, 1.2, 1.8], 120_000, 2, True),
    ("3d2x2x4_pt_multicluster", 3, (2, 2, 4), [0.8, 1.2, 1.8, 2.6], 120_000, 2, True),
    # an odd extent: sequential (typewriter) sweeps
    ("3d2x2x3_metropolis_typewriter", 3, (2, 2, 3), [0.6, 1.0, 1.6, 2.4], 120_000, False, False),
    ("3d2x2x3_pt_typewriter", 3, (2, 2, 3), [0.6, 1.0, 1.6, 2.4], 120_000, False, True),
    ("3d2x2x3_pt_houdayer_typewriter", 3, (2, 2, 3), [0.6, 1.0, 1.6, 2.4], 120_000, True, True),
]


@pytest.mark.parametrize("label,ndim,dims,temps,n_mcs,houd,pt", CASES, ids=[c[0] for c in CASES])
def test_mc_averages_match_enumeration(oracle_mod, label, ndim, dims, temps, n_mcs, houd, pt):
    o = oracle_mod.Oracle(oracle_mod.OracleParams(ndim, dims, 1, 2, temps, coupling_seed=1, sim_seed=5,
                                                  typewriter=any(L % 2 for L in dims)))
    hist = o.enumerate(0)
    o.mcs(2000, houdayer=houd)  # equilibrate (not measured)
    sE, sE2 = o.run_binned(n_mcs, 60, houdayer=houd, pt=pt)
    check_against_enumeration(o, hist, temps, sE * 1.0, sE2 * 1.0, label)
    assert o.check_energies() == 0
    c = o.counters()
    assert c["error"] == 0 and c["near_threshold"] == 0


def test_pt_acceptance_matches_enumeration(oracle_mod):
    temps = [0.6, 0.9, 1.3, 2.0]
    o = oracle_mod.Oracle(oracle_mod.OracleParams(2, (4, 4), 1, 2, temps, coupling_seed=3, sim_seed=9))
    hist = o.enumerate(0)
    o.mcs(2000)
    a0, t0 = o.pt_stats()
    o.mcs(100_000)
    a1, t1 = o.pt_stats()
    acc = (a1 - a0).astype(np.float64)
    tries = (t1 - t0).astype(np.float64)
    for k in range(len(temps) - 1):
        b1, b2 = 1 / temps[k], 1 / temps[k + 1]
        e1, p1 = exact_energy_pmf(hist, 2, 16, b1)
        e2, p2 = exact_energy_pmf(hist, 2, 16, b2)
        delta = (b1 - b2) * (e1[:, None] - e2[None, :])
        expect = (p1[:, None] * p2[None, :] * np.minimum(1.0, np.exp(np.minimum(delta, 0.0)))).sum()
        got = acc[k] / tries[k]
        sigma = math.sqrt(expect * (1 - expect) / tries[k])
        # decisions are correlated in time: allow a generous multiple of the naive error
        assert abs(got - expect) < max(10 * sigma, 0.01), (k, got, expect)


def test_metropolis_class_acceptance_is_threshold_over_2_32(oracle_mod):
    temps = [0.5, 1.0, 2.0, 4.0]
    o = oracle_mod.Oracle(oracle_mod.OracleParams(3, (6, 6, 6), 2, 2, temps, coupling_seed=2, sim_seed=4))
    o.mcs(300)
    tries, acc = o.class_stats()
    thr = o.thresholds().astype(np.float64)
    checked = 0
    for k in range(len(temps)):
        for m in range(3):
            n = float(tries[k, m])
            if n < 500:
                continue
            p = thr[k, m] / 2**32
            assert math.isclose(p, math.exp(-4 * (m + 1) / temps[k]), rel_tol=1e-6, abs_tol=1e-9)
            sigma = math.sqrt(max(p * (1 - p), 1e-12) / n)
            assert abs(acc[k, m] / n - p) < TOL_SIGMA * sigma + 1.0 / n, (k, m, acc[k, m] / n, p)
            checked += 1
    assert checked >= 8


def test_infinite_temperature_flips_every_spin(oracle_mod):
    """beta -> 0: every threshold is 2^32 - 1, so (barring a word equal to 2^32 - 1) every
    spin flips in its half-sweep and one sweep maps s to -s with E unchanged."""
    temps = [1e12, 2e12]
    o = oracle_mod.Oracle(oracle_mod.OracleParams(3, (4, 4, 6), 2, 2, temps))
    assert (o.thresholds() == 0xFFFFFFFF).all()
    s0, e0 = o.spins(), o.energies()
    o.sweep(1)
    np.testing.assert_array_equal(o.spins(), 1 - s0)
    np.testing.assert_array_equal(o.energies(), e0)


def test_low_temperature_houdayer_matches_enumeration(oracle_mod):
    """Metropolis + PT + the move on the two lowest slots only still samples the
    Boltzmann weights of Eq. 1's energy at every temperature."""
    temps = [0.5, 0.8, 1.2, 1.8]
    o = oracle_mod.Oracle(oracle_mod.OracleParams(2, (4, 4), 1, 2, temps, coupling_seed=1, sim_seed=9,
                                                  houdayer_slots=2))
    hist = o.enumerate(0)
    o.mcs(2000, houdayer=True)
    sE, sE2 = o.run_binned(120_000, 60, houdayer=True, pt=True)
    check_against_enumeration(o, hist, temps, sE * 1.0, sE2 * 1.0, "2d4x4_pt_houdayer_low2")
    assert o.check_energies() == 0
    c = o.counters()
    assert c["error"] == 0 and c["near_threshold"] == 0


def test_typewriter_order_is_sequential(oracle_mod):
    """The typewriter order is another update order, not another random stream: from the
    same hot start on an even lattice it reaches a different state than the checkerboard
    (a site sees its same-sweep predecessors' flips), each order is a deterministic
    function of the counters (two runs agree), and both keep the energies exact."""
    kw = dict(ndim=3, dims=(2, 2, 4), n_samples=1, n_chains=1, temps=[0.7, 1.3], coupling_seed=2, sim_seed=3)
    a = oracle_mod.Oracle(oracle_mod.OracleParams(**kw, typewriter=True))
    b = oracle_mod.Oracle(oracle_mod.OracleParams(**kw, typewriter=True))
    c = oracle_mod.Oracle(oracle_mod.OracleParams(**kw))
    for o in (a, b, c):
        o.sweep(3)
    np.testing.assert_array_equal(a.spins(), b.spins())
    assert not np.array_equal(a.spins(), c.spins())
    assert a.check_energies() == 0 and c.check_energies() == 0
