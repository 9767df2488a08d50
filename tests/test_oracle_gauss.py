"""Pins of the general-coupling oracle (Gaussian couplings, Sec. 2.1).

* Its fp32 exp (Cody-Waite reduction by ln 2, Taylor series to r^6) agrees with the
  library exp within 2e-6 relative on [-23, 0], and the Metropolis threshold it feeds is
  monotone in dE, saturates at 2^32 - 1 for tiny dE and vanishes below x = -23.
* Energies of Eq. 1 equal a networkx sum over the periodic lattice's edges, and the
  ferromagnet J = 1 has E = -dN for aligned spins.
* <E> and the specific heat from Metropolis + exchange agree with exact enumeration of
  the 2^16 states of a 4x4 Gaussian sample within their statistical errors.
* Kept energies equal recomputed ones; gauge covariance (J' = tau J tau, s' = tau s).
"""
import math

import numpy as np
import pytest

from paper_2003_04621_gb300.inputs import JFIX_SCALE, gaussian_couplings_fixed, geometric_temps


def test_exp_against_library(oracle_mod):
    xs = np.linspace(-23.0, 0.0, 20001)
    for x in xs:
        x32 = float(np.float32(x))
        got = oracle_mod.exp_f(x32)
        assert abs(got - math.exp(x32)) <= 2e-6 * math.exp(x32), (x32, got)


def test_threshold_shape(oracle_mod):
    beta = float(np.float32(1.3))
    prev = 2**32
    for dE in [1, 10, 100, 1000, 10**4, 10**5, 10**6, 4 * 10**6, 16 * 10**6, 10**8]:
        t = oracle_mod.gauss_threshold(beta, dE)
        assert t <= prev
        prev = t
    assert oracle_mod.gauss_threshold(float(np.float32(1e-3)), 1) == 2**32 - 1  # e rounds to 1
    assert oracle_mod.gauss_threshold(beta, 30 * JFIX_SCALE) == 0
    x = -(np.float32(beta) * np.float32(3 * JFIX_SCALE) * np.float32(2.0**-20))
    assert abs(oracle_mod.gauss_threshold(beta, 3 * JFIX_SCALE) / 2**32 - math.exp(float(x))) < 1e-6


@pytest.mark.parametrize("ndim,dims", [(2, (4, 6)), (3, (4, 4, 2)), (2, (2, 6))])
def test_energy_matches_networkx(oracle_mod, ndim, dims):
    nx = pytest.importorskip("networkx")
    J = gaussian_couplings_fixed(2, dims, seed=3)
    o = oracle_mod.OracleGauss(ndim, dims, 2, 2, [1.0, 2.0], J, sim_seed=4)
    sp = 1 - 2 * o.spins().astype(np.int64)
    N = o.N
    E = o.energies()
    for s in range(2):
        G = nx.MultiGraph()
        for i in range(N):
            c = [i % dims[0], (i // dims[0]) % dims[1], i // (dims[0] * dims[1]) if ndim == 3 else 0]
            for mu in range(ndim):
                cc = list(c)
                cc[mu] = (cc[mu] + 1) % dims[mu]
                j = cc[0] + dims[0] * (cc[1] + dims[1] * cc[2])
                G.add_edge(i, j, J=int(J[s, i, mu]))
        for c in range(2):
            for r in range(2):
                e = -sum(int(a["J"]) * sp[s, c, r, u] * sp[s, c, r, v] for u, v, a in G.edges(data=True))
                assert e == E[s, c, r]


def test_ferromagnet_ground_state(oracle_mod):
    dims = (4, 6)
    J = np.full((1, 24, 2), JFIX_SCALE, np.int32)
    o = oracle_mod.OracleGauss(2, dims, 1, 1, [0.5], J)
    o.set_spins(np.zeros((1, 1, 1, 24), np.uint8))
    assert o.energies()[0, 0, 0] == -2 * 24 * JFIX_SCALE


def test_averages_match_enumeration(oracle_mod):
    dims = (4, 4)
    temps = [0.4, 0.7, 1.1, 1.8]
    J = gaussian_couplings_fixed(1, dims, seed=11)
    o = oracle_mod.OracleGauss(2, dims, 1, 2, temps, J, sim_seed=7)
    levels = o.enumerate(0).astype(np.float64) / JFIX_SCALE
    o.mcs(2000)
    nb = 60
    sE, sE2 = o.run_binned(120_000, nb)
    for k, T in enumerate(temps):
        beta = 1.0 / T
        w = np.exp(-beta * (levels - levels.min()))
        w /= w.sum()
        m1, m2 = (w * levels).sum(), (w * levels**2).sum()
        means = sE[k] / (2 * (120_000 // nb))  # both chains pooled in the bin sums
        err = means.std(ddof=1) / math.sqrt(nb)
        assert abs(means.mean() - m1) < 4.5 * err + 1e-12, (T, means.mean(), m1, err)
        per = 2 * (120_000 // nb)
        c_exact = beta**2 * (m2 - m1**2) / o.N
        tot1, tot2 = sE[k].sum() / per, sE2[k].sum() / per
        jk = []
        for b in range(nb):
            a1 = (sE[k].sum() - sE[k, b]) / (per * (nb - 1))
            a2 = (sE2[k].sum() - sE2[k, b]) / (per * (nb - 1))
            jk.append(beta**2 * (a2 - a1**2) / o.N)
        jk = np.array(jk)
        c_all = beta**2 * (tot2 / nb - (tot1 / nb) ** 2) / o.N
        c_err = math.sqrt((nb - 1) / nb * ((jk - jk.mean()) ** 2).sum())
        assert abs(c_all - c_exact) < 4.5 * c_err + 1e-12, (T, c_all, c_exact, c_err)
    assert o.check_energies() == 0
    assert o.counters()["near_threshold"] == 0


def test_gauge_covariance(oracle_mod):
    dims = (6, 4)
    temps = geometric_temps(0.3, 1.5, 5)
    J = gaussian_couplings_fixed(2, dims, seed=5)
    N = 24
    rng = np.random.default_rng(1)
    tau = rng.choice([-1, 1], size=(2, N)).astype(np.int64)
    Jg = J.astype(np.int64).copy()
    for mu in range(2):
        c = np.arange(N)
        x, y = c % 6, c // 6
        nb = ((x + 1) % 6 + 6 * y) if mu == 0 else (x + 6 * ((y + 1) % 4))
        Jg[:, :, mu] = tau * J[:, :, mu] * tau[:, nb]
    a = oracle_mod.OracleGauss(2, dims, 2, 2, temps, J, sim_seed=8)
    b = oracle_mod.OracleGauss(2, dims, 2, 2, temps, Jg.astype(np.int32), sim_seed=8)
    s0 = 1 - 2 * a.spins().astype(np.int64)
    b.set_spins(((1 - s0 * tau[:, None, None, :]) // 2).astype(np.uint8))
    for _ in range(30):
        a.mcs(1)
        b.mcs(1)
        sa = 1 - 2 * a.spins().astype(np.int64)
        sb = 1 - 2 * b.spins().astype(np.int64)
        np.testing.assert_array_equal(sb, sa * tau[:, None, None, :])
        np.testing.assert_array_equal(a.energies(), b.energies())
        np.testing.assert_array_equal(a.perm(), b.perm())
