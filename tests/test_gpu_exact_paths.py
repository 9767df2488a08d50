"""The exact branches behind the fast screens of the fused kernels, forced and checked.

The one-warp replica exchange inside the sweep kernels (Eq. 5) first compares the
integer energy difference with fp32 bounds around theta = ln(u 2^-32) / dbeta and
evaluates exp(delta) in fp64 only when dE lies inside the screening margin.  Random
inputs almost never land there, so these tests build inputs that do:

- a ferromagnet (p_plus = 1) whose replicas hold 0, 2, 4, ... flat domain walls, so that
  replica j has energy -2N + 4 j L1 and, at inverse temperatures above 5.55, every
  Metropolis threshold floor(exp(-4 m beta) 2^32) is 0 and no site can lower its energy:
  the configurations and energies stay fixed, and only the exchange acts;
- inverse temperatures solved, pair by pair, from the exchange word u of each pair of
  one chain in the first pass, so that dbeta dE = ln(u 2^-32)(1 +- 2e-7): theta then lies
  within 4e-6 of the integer dE, well inside the margin, while |u 2^-32 - exp(delta)|
  stays far above the 1e-12 near-threshold window.

The GPU must match the oracle after every MCS, make the planned decisions, report at
least one exact-path decision per tuned pair, and report no near-threshold decision.
The general-coupling kernel's two screens (its exchange, and its Metropolis band around
the hardware exp) are checked the same way.
"""
import numpy as np
import pytest

from helpers import L1, assert_same_state, gpu_of, oracle_of, tuned_job

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch

    from paper_2003_04621_gb300 import build

    build.build()
    assert torch.cuda.is_available()


@pytest.mark.parametrize("fmt,T", [("packed", 12), ("packed", 40), ("packed", 64), ("int8", 12), ("int8", 40),
                                   ("int8", 64)])
def test_exchange_exact_branch_forced(oracle_mod, fmt, T):
    job = tuned_job(oracle_mod, T)
    assert job["tuned"] >= T // 2
    kw = dict(ndim=2, dims=(job["L0"], L1), n_samples=job["S"], n_chains=2, temps=job["temps"], p_plus=1.0,
              sim_seed=job["sim_seed"], coupling_seed=3)
    sim = gpu_of(spin_format=fmt, **kw)
    orc = oracle_of(oracle_mod, **kw)
    np.testing.assert_array_equal(sim.thresholds(), np.zeros((T, 2), np.uint32))
    sim.set_spins(job["spins"])
    orc.set_spins(job["spins"])
    assert_same_state(sim, orc, "after import")
    for t in range(4):
        sim.run_mcs(1)
        orc.mcs(1)
        assert_same_state(sim, orc, f"{fmt} T={T} mcs {t}")
        if t == 0:
            _, perm, _ = sim.state()
            np.testing.assert_array_equal(perm[job["tuned_sample"], 0], job["perm"], err_msg="planned decisions")
    # the configurations never moved: only the exchange acted
    np.testing.assert_array_equal(sim.spins().cpu().numpy(), job["spins"])
    c = sim.counters()
    assert c["exchange_exact"] >= job["tuned"], c
    assert c["near_threshold"] == 0 and orc.counters()["near_threshold"] == 0
    np.testing.assert_array_equal(c["pt_accepts"], orc.pt_stats()[0])


def test_exchange_exact_branch_general_couplings(oracle_mod):
    """The same construction with fixed-point couplings J = 1.0 (2^20) on every bond: the
    general-coupling kernel's warp exchange, on int64 energies."""
    T = 24
    job = tuned_job(oracle_mod, T, scale=1 << 20)
    S, N = job["S"], job["L0"] * L1
    J = np.full((S, N, 2), 1 << 20, np.int32)
    sim = gpu_of(ndim=2, dims=(job["L0"], L1), n_samples=S, n_chains=2, temps=job["temps"],
                 sim_seed=job["sim_seed"], spin_format="int8", couplings="fixed")
    sim.set_couplings_fixed(J)
    sim.set_spins(job["spins"])
    orc = oracle_mod.OracleGauss(2, (job["L0"], L1), S, 2, job["temps"], J, sim_seed=job["sim_seed"])
    orc.set_spins(job["spins"])
    for t in range(4):
        sim.run_mcs(1)
        orc.mcs(1)
        E_g, perm_g, _ = sim.state()
        np.testing.assert_array_equal(E_g, orc.energies(), err_msg=f"energies mcs {t}")
        np.testing.assert_array_equal(perm_g, orc.perm(), err_msg=f"perm mcs {t}")
        if t == 0:
            np.testing.assert_array_equal(perm_g[job["tuned_sample"], 0], job["perm"])
    np.testing.assert_array_equal(sim.spins().cpu().numpy(), job["spins"])
    c = sim.counters()
    assert c["exchange_exact"] >= job["tuned"], c
    assert c["near_threshold"] == 0 and orc.counters()["near_threshold"] == 0


def test_metropolis_band_general_couplings(oracle_mod):
    """Gaussian couplings at moderate temperatures: some Metropolis draws fall inside the
    2^-14 band around the hardware-exp estimate and take the fixed fp32 threshold; the
    state still equals the oracle's after every MCS."""
    from paper_2003_04621_gb300.inputs import gaussian_couplings_fixed, geometric_temps

    dims, S, T = (16, 16), 24, 16
    temps = geometric_temps(0.3, 1.6, T)
    J = gaussian_couplings_fixed(S, dims, seed=9)
    sim = gpu_of(ndim=2, dims=dims, n_samples=S, n_chains=2, temps=temps, sim_seed=5, spin_format="int8",
                 couplings="fixed")
    sim.set_couplings_fixed(J)
    orc = oracle_mod.OracleGauss(2, dims, S, 2, temps, J, sim_seed=5)
    for t in range(6):
        sim.run_mcs(2)
        orc.mcs(2)
        E_g, perm_g, _ = sim.state()
        np.testing.assert_array_equal(E_g, orc.energies(), err_msg=f"energies {t}")
        np.testing.assert_array_equal(perm_g, orc.perm(), err_msg=f"perm {t}")
    np.testing.assert_array_equal(sim.spins().cpu().numpy(), orc.spins())
    c = sim.counters()
    # 256 sites x 24 samples x 32 replicas x 12 sweeps = 2.4 M attempts; about 1e-4 of
    # those with dE > 0 land in the band
    assert c["metropolis_band"] > 0, c
    assert c["near_threshold"] == 0
