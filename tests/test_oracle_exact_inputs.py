"""The inputs that force the exchange's exact branch, checked on the oracle alone: the
configurations are frozen (every Metropolis threshold is 0 and no site can lower its
energy), the energies follow the closed form -2N + 4 j L1 (times the coupling scale),
and the first exchange pass of the tuned chain makes exactly the planned decisions,
none of them within the near-threshold window."""
import numpy as np
import pytest

from helpers import L1, oracle_of, tuned_job


@pytest.mark.parametrize("T", [2, 12, 40, 64])
def test_tuned_pm_job_on_the_oracle(oracle_mod, T):
    job = tuned_job(oracle_mod, T)
    N = job["L0"] * L1
    orc = oracle_of(oracle_mod, ndim=2, dims=(job["L0"], L1), n_samples=job["S"], n_chains=2, temps=job["temps"],
                    p_plus=1.0, sim_seed=job["sim_seed"], coupling_seed=3)
    assert (orc.couplings() == 1).all()
    assert not orc.thresholds().any()
    orc.set_spins(job["spins"])
    want_E = np.broadcast_to(np.array([-2 * N + 4 * j * L1 for j in range(T)], np.int32), (job["S"], 2, T))
    np.testing.assert_array_equal(orc.energies(), want_E)
    orc.mcs(1)
    np.testing.assert_array_equal(orc.perm()[0][job["tuned_sample"], 0], job["perm"])
    orc.mcs(3)
    np.testing.assert_array_equal(orc.spins(), job["spins"])
    np.testing.assert_array_equal(orc.energies(), want_E)
    assert orc.counters()["near_threshold"] == 0
    assert job["tuned"] >= min(1, T - 1)


def test_tuned_fixed_point_job_on_the_oracle(oracle_mod):
    T = 24
    job = tuned_job(oracle_mod, T, scale=1 << 20)
    S, N = job["S"], job["L0"] * L1
    J = np.full((S, N, 2), 1 << 20, np.int32)
    orc = oracle_mod.OracleGauss(2, (job["L0"], L1), S, 2, job["temps"], J, sim_seed=job["sim_seed"])
    orc.set_spins(job["spins"])
    want_E = np.array([(-2 * N + 4 * j * L1) << 20 for j in range(T)], np.int64)
    np.testing.assert_array_equal(orc.energies()[0, 0], want_E)
    orc.mcs(1)
    np.testing.assert_array_equal(orc.perm()[job["tuned_sample"], 0], job["perm"])
    orc.mcs(3)
    np.testing.assert_array_equal(orc.spins(), job["spins"])
    assert orc.counters()["near_threshold"] == 0
