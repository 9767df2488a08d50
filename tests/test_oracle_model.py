"""Pins for the oracle's model: the lattice, the couplings (Eq. 2) and the energy
(Eq. 1 with H = 0), checked against things other than the oracle itself.

* Kaufman's exact finite-lattice partition function of the 2D Ising ferromagnet on an
  m x n torus (Kaufman, Phys. Rev. 76, 1232 (1949)), against the oracle's exact
  enumeration with every J = +1.  A wrong neighbour, a missing periodic wrap or a
  wrong sign in the energy changes Z.
* A brute-force energy over a periodic lattice graph built by networkx (an
  independent construction of the neighbour structure), for random +-J couplings and
  random spins, against the oracle's energies.
* Closed forms: J = +1 aligned state E = -dN, checkerboard state E = +dN.
* Eq. 2: the fraction of J = +1 bonds is binomial(p).
"""
import math

import numpy as np
import pytest

from paper_2003_04621_gb300.inputs import geometric_temps


def make(oracle_mod, ndim, dims, S=1, C=1, temps=(1.0,), **kw):
    return oracle_mod.Oracle(oracle_mod.OracleParams(ndim, dims, S, C, list(temps), **kw))


def kaufman_logZ(K: float, m: int, n: int) -> float:
    """ln Z of the 2D Ising ferromagnet on an m x n torus at coupling K = beta J."""
    def gamma(l):
        if l == 0:
            return 2 * K + math.log(math.tanh(K))
        c = math.cosh(2 * K) / math.tanh(2 * K) - math.cos(math.pi * l / n)
        return math.log(c + math.sqrt(c * c - 1))

    g_odd = [gamma(2 * r + 1) for r in range(n)]
    g_even = [gamma(2 * r) for r in range(n)]
    z1 = np.prod([2 * math.cosh(m * g / 2) for g in g_odd])
    z2 = np.prod([2 * math.sinh(m * g / 2) for g in g_odd])
    z3 = np.prod([2 * math.cosh(m * g / 2) for g in g_even])
    z4 = np.prod([2 * math.sinh(m * g / 2) for g in g_even])
    return math.log(0.5) + (m * n / 2) * math.log(2 * math.sinh(2 * K)) + math.log(z1 + z2 + z3 + z4)


def logZ_from_hist(hist: np.ndarray, d: int, N: int, beta: float) -> float:
    e = np.arange(hist.size) - d * N
    nz = hist > 0
    x = -beta * e[nz] + np.log(hist[nz].astype(np.float64))
    mx = x.max()
    return mx + math.log(np.exp(x - mx).sum())


@pytest.mark.parametrize("dims", [(4, 4), (6, 4)])
def test_enumeration_matches_kaufman_ferromagnet(oracle_mod, dims):
    o = make(oracle_mod, 2, dims)
    N = dims[0] * dims[1]
    o.set_couplings(np.ones((1, N, 2), np.int8))
    hist = o.enumerate(0)
    assert hist.sum() == 2**N
    for beta in (0.1, 0.3, 0.4406868, 0.6, 1.0):
        # dims = (L0, L1): L1 rows of L0 columns
        ref = kaufman_logZ(beta, dims[1], dims[0])
        got = logZ_from_hist(hist, 2, N, beta)
        assert abs(got - ref) < 1e-9 * max(1.0, abs(ref)), (beta, got, ref)


def _nx_energy(dims, J, spins):
    nx = pytest.importorskip("networkx")
    d = len(dims)
    # networkx labels the nodes of grid_graph(dim=[L0, L1, L2]) by (z, y, x) tuples
    G = nx.grid_graph(dim=list(dims), periodic=True)
    strides = [int(np.prod(dims[:a])) for a in range(d)]
    E = 0
    for u, v in G.edges():
        cu = tuple(reversed(u))  # (x, y, z)
        cv = tuple(reversed(v))
        diff = [a for a in range(d) if cu[a] != cv[a]]
        assert len(diff) == 1
        mu = diff[0]
        # the bond is stored at the endpoint from which the other is one step forward
        base = cu if (cu[mu] + 1) % dims[mu] == cv[mu] else cv
        i = sum(base[a] * strides[a] for a in range(d))
        iu = sum(cu[a] * strides[a] for a in range(d))
        iv = sum(cv[a] * strides[a] for a in range(d))
        E -= int(J[i, mu]) * int(spins[iu]) * int(spins[iv])
    return E


@pytest.mark.parametrize("ndim,dims", [(2, (5, 3)), (2, (4, 6)), (3, (3, 4, 5)), (3, (4, 4, 4))])
def test_energy_matches_networkx_lattice(oracle_mod, ndim, dims):
    o = make(oracle_mod, ndim, dims, S=2, C=1, temps=(1.0, 2.0), coupling_seed=7, sim_seed=3)
    J = o.couplings()
    bits = o.spins()
    E = o.energies()
    for s in range(2):
        for j in range(2):
            spins = 1 - 2 * bits[s, 0, j].astype(np.int64)
            assert E[s, 0, j] == _nx_energy(dims, J[s], spins)


@pytest.mark.parametrize("ndim,dims", [(2, (4, 4)), (2, (2, 6)), (3, (2, 2, 4)), (3, (6, 6, 6))])
def test_ferromagnet_closed_forms(oracle_mod, ndim, dims):
    o = make(oracle_mod, ndim, dims, S=1, C=1, temps=(1.0, 1.5))
    N = int(np.prod(dims))
    o.set_couplings(np.ones((1, N, ndim), np.int8))
    coords = np.indices(tuple(reversed(dims))).reshape(ndim, -1)[::-1]  # x fastest
    checker = (coords.sum(axis=0) % 2).astype(np.uint8)
    bits = np.zeros((1, 1, 2, N), np.uint8)
    bits[0, 0, 1] = checker
    o.set_spins(bits)
    E = o.energies()
    assert E[0, 0, 0] == -ndim * N
    assert E[0, 0, 1] == ndim * N


@pytest.mark.parametrize("p", [0.5, 0.25, 0.0, 1.0])
def test_coupling_fraction_is_binomial(oracle_mod, p):
    o = make(oracle_mod, 3, (8, 8, 8), S=4, C=1, temps=(1.0,), p_plus=p, coupling_seed=11)
    J = o.couplings()
    frac = (J == 1).mean()
    n = J.size
    if p in (0.0, 1.0):
        assert frac == p
    else:
        assert abs(frac - p) < 4.5 * math.sqrt(p * (1 - p) / n)
    assert set(np.unique(J).tolist()) <= {-1, 1}


def test_hot_start_is_balanced_and_keyed_by_sample(oracle_mod):
    temps = geometric_temps(1.0, 2.0, 12)
    a = make(oracle_mod, 3, (6, 6, 6), S=4, C=2, temps=temps)
    b = make(oracle_mod, 3, (6, 6, 6), S=2, C=2, temps=temps, sample_offset=2)
    bits = a.spins()
    assert abs(bits.mean() - 0.5) < 4.5 * math.sqrt(0.25 / bits.size)
    # samples are keyed by their job-wide index: a shard reproduces the same samples
    np.testing.assert_array_equal(bits[2:], b.spins())
    np.testing.assert_array_equal(a.couplings()[2:], b.couplings())
    np.testing.assert_array_equal(a.energies()[2:], b.energies())


def _golden(name):
    import os

    out = {}
    with open(os.path.join(os.path.dirname(__file__), "golden", name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                k, v = line.split()
                out[k] = float(v)
    return out


def test_phi_protocol_matches_the_printed_fit():
    """Sec. 2.3: the phi family (Eqs. 6-7) at the fitted optimum of Eqs. 8-9, constants as
    printed (tests/golden/phi_protocol_fit.txt)."""
    from paper_2003_04621_gb300 import inputs

    g = _golden("phi_protocol_fit.txt")
    assert inputs.PHI_FIT == g
    for L in (8, 15, 16, 40, 64):
        T = inputs.phi_protocol(L)
        phi = g["a_phi"] + g["b_phi"] * L
        n = max(2, round(g["a_NT"] + g["b_NT"] * L))
        assert len(T) == n
        assert T[0] == g["T_min"] and abs(T[-1] - g["T_max"]) < 1e-12
        steps = np.diff(T)
        assert np.all(steps > 0)
        # phi < 1 spaces the set more densely towards high temperatures, phi > 1 towards low
        if phi < 1:
            assert steps[-1] < steps[0]
        elif phi > 1:
            assert steps[-1] > steps[0]
    # phi = 1 is the linear schedule
    lin = inputs.phi_temps(0.2, 1.5, 11, 1.0)
    assert np.allclose(lin, np.linspace(0.2, 1.5, 11), rtol=0, atol=1e-12)
    # the 2D Gaussian job uses phi*(16) with 32 points
    w = inputs.workload_2d_gauss_l16()
    assert np.allclose(w.temps, inputs.phi_temps(0.2, 1.5, 32, 0.406 + 0.014 * 16), rtol=0, atol=0)
