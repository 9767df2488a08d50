"""Pins of the overlap plane sums (two-replica measurements, Sec. 3) and of the host
formulas built on them.

* Identical replicas: q = +1 everywhere, so every plane sum is N / L_mu and every mode
  at k != 0 vanishes.
* A planted domain wall pair along axis mu (chain 1 flipped on x_mu < L_mu / 2): the
  plane sums are -N/L_mu then +N/L_mu along mu and 0 along the other axes, and
  |q(2 pi / L)|^2 = 4 / (L^2 sin^2(pi / L)) in closed form.
* Every plane-sum family adds up to N q of Eq. 4 (the oracle's own overlap).
* The correlation-length formula inverts the Ornstein-Zernike form exactly.
"""
import math

import numpy as np
import pytest

from paper_2003_04621_gb300.inputs import geometric_temps
from paper_2003_04621_gb300.observables import chi_sg, q_modes, xi_second_moment


def make(oracle_mod, ndim, dims, S=2, T=3, **kw):
    return oracle_mod.Oracle(oracle_mod.OracleParams(ndim, dims, S, 2, geometric_temps(0.5, 2.0, T), **kw))


@pytest.mark.parametrize("ndim,dims", [(2, (8, 6)), (3, (4, 6, 2)), (3, (6, 6, 6))])
def test_identical_replicas(oracle_mod, ndim, dims):
    o = make(oracle_mod, ndim, dims)
    sp = o.spins()
    sp[:, 1] = sp[:, 0]
    o.set_spins(sp)
    P = o.qmodes()
    N = int(np.prod(dims))
    for mu in range(ndim):
        np.testing.assert_array_equal(P[:, :, mu, : dims[mu]], N // dims[mu])
        assert (P[:, :, mu, dims[mu]:] == 0).all()
    q0, qk2 = q_modes(P, dims)
    np.testing.assert_allclose(q0, 1.0)
    np.testing.assert_allclose(qk2, 0.0, atol=1e-24)


@pytest.mark.parametrize("ndim,dims,mu", [(2, (8, 6), 0), (2, (8, 6), 1), (3, (4, 6, 10), 2), (3, (6, 4, 4), 0)])
def test_planted_domain_walls(oracle_mod, ndim, dims, mu):
    o = make(oracle_mod, ndim, dims, S=1, T=1)
    sp = o.spins()
    N = int(np.prod(dims))
    i = np.arange(N)
    stride = int(np.prod(dims[:mu]))
    x = (i // stride) % dims[mu]
    L = dims[mu]
    sp[0, 1, 0] = sp[0, 0, 0] ^ (x < L // 2).astype(np.uint8)
    o.set_spins(sp)
    P = o.qmodes()[0, 0]
    expect = np.where(np.arange(L) < L // 2, -(N // L), N // L)
    np.testing.assert_array_equal(P[mu, :L], expect)
    for nu in range(ndim):
        if nu != mu:
            np.testing.assert_array_equal(P[nu], 0)
    _, qk2 = q_modes(P, dims)
    assert qk2[mu] == pytest.approx(4.0 / (L * L * math.sin(math.pi / L) ** 2), rel=1e-12)


def test_plane_sums_add_up_to_the_overlap(oracle_mod):
    o = make(oracle_mod, 3, (6, 4, 8), S=3, T=5, sim_seed=9)
    o.mcs(7, houdayer=True)
    P = o.qmodes()
    _, NQ = o.measure()
    for mu, L in enumerate((6, 4, 8)):
        np.testing.assert_array_equal(P[:, :, mu, :L].sum(axis=-1), NQ)


def test_xi_inverts_ornstein_zernike():
    for L, xi in ((8, 1.7), (16, 4.25), (32, 0.6)):
        k = 2 * math.pi / L
        chi0 = 37.0
        chik = chi0 / (1.0 + xi * xi * 4 * math.sin(k / 2) ** 2)
        assert xi_second_moment(chi0, chik, L) == pytest.approx(xi, rel=1e-12)


def test_chi_averages_modes():
    dims = (4, 4)
    P = np.zeros((2, 2, 4), np.int32)  # two measurements
    P[0, 0, :] = 4  # q = 1 everywhere
    P[0, 1, :] = 4
    P[1, 0, :] = [-4, -4, 4, 4]
    P[1, 1, :] = 0
    c0, ck = chi_sg(P, dims)
    assert c0 == pytest.approx(16 * (1.0 + 0.0) / 2)
    assert ck == pytest.approx(16 * np.mean([0, 0, 4.0 / (16 * math.sin(math.pi / 4) ** 2), 0]))
