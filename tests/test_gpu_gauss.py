"""GPU parity of the general-coupling engine (Gaussian couplings, Sec. 2.1) with its
oracle, bit-exact: spins, int64 fixed-point energies, replica maps and the measured E by
slot and N q after every step, on 2D and 3D lattices, ragged temperature counts, one
and two chains, separate sweep / exchange calls, and the 2D L=16 Gaussian job."""
import numpy as np
import pytest

from paper_2003_04621_gb300.inputs import gaussian_couplings_fixed, geometric_temps, workload_2d_gauss_l16

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2003_04621_gb300 import build

    build.build()


def pair(oracle_mod, ndim, dims, S, C, temps, seed=3, sim_seed=5, sample_offset=0):
    from paper_2003_04621_gb300.sgmc import Simulation

    J = gaussian_couplings_fixed(S, dims, seed=seed, sample_offset=sample_offset)
    sim = Simulation(ndim, dims, S, C, temps, sim_seed=sim_seed, spin_format="int8", couplings="fixed",
                     sample_offset=sample_offset)
    sim.set_couplings_fixed(J)
    orc = oracle_mod.OracleGauss(ndim, dims, S, C, temps, J, sim_seed=sim_seed, sample_offset=sample_offset)
    return sim, orc


def same(sim, orc, where):
    E, perm, _ = sim.state()
    np.testing.assert_array_equal(E, orc.energies(), err_msg=f"E {where}")
    np.testing.assert_array_equal(perm, orc.perm(), err_msg=f"perm {where}")
    np.testing.assert_array_equal(sim.spins().cpu().numpy(), orc.spins(), err_msg=f"spins {where}")
    Eg, Qg = sim.measure()
    Eo, Qo = orc.measure()
    np.testing.assert_array_equal(Eg, Eo, err_msg=f"E by slot {where}")
    if Qo is not None:
        np.testing.assert_array_equal(Qg, Qo, err_msg=f"N q {where}")


@pytest.mark.parametrize("ndim,dims,C,T", [(2, (16, 16), 2, 8), (3, (6, 6, 6), 2, 12), (2, (8, 10), 2, 5),
                                           (3, (4, 6, 2), 1, 33), (2, (2, 4), 2, 3)])
def test_mcs_equal_oracle(oracle_mod, ndim, dims, C, T):
    sim, orc = pair(oracle_mod, ndim, dims, 3, C, geometric_temps(0.3, 2.0, T))
    same(sim, orc, "create")
    for t in range(6):
        sim.run_mcs(1)
        orc.mcs(1)
        same(sim, orc, f"mcs {t}")
    sim.run_mcs(7)
    orc.mcs(7)
    same(sim, orc, "7 more")
    assert sim.counters()["near_threshold"] == orc.counters()["near_threshold"] == 0


def test_separate_calls(oracle_mod):
    sim, orc = pair(oracle_mod, 2, (12, 8), 2, 2, geometric_temps(0.2, 1.5, 10))
    for op in "ssxsxxssx":
        if op == "s":
            sim.sweep(1)
            orc.sweep(1)
        else:
            sim.exchange()
            orc.exchange()
        same(sim, orc, op)


def test_gauss_job_sampled(oracle_mod):
    """The 512-sample 2D L=16 job on the GPU; two samples recomputed by the oracle."""
    from paper_2003_04621_gb300.sgmc import Simulation

    w = workload_2d_gauss_l16()
    J = gaussian_couplings_fixed(w.n_samples, w.dims, seed=w.coupling_seed)
    sim = Simulation(2, w.dims, w.n_samples, 2, list(w.temps), sim_seed=w.sim_seed, spin_format="int8",
                     couplings="fixed")
    sim.set_couplings_fixed(J)
    sim.run_mcs(5)
    E, perm, _ = sim.state()
    for s in (0, 401):
        o = oracle_mod.OracleGauss(2, w.dims, 1, 2, list(w.temps), J[s:s + 1], sim_seed=w.sim_seed, sample_offset=s)
        o.mcs(5)
        np.testing.assert_array_equal(E[s:s + 1], o.energies())
        np.testing.assert_array_equal(perm[s:s + 1], o.perm())


def test_refusals():
    from paper_2003_04621_gb300.sgmc import SGError, Simulation

    with pytest.raises(SGError) as e:
        Simulation(2, (8, 8), 1, 2, [1.0, 2.0], spin_format="packed", couplings="fixed")
    assert e.value.status == 5
    with pytest.raises(SGError) as e:
        Simulation(2, (8, 8), 1, 2, [1.0, 2.0], spin_format="int8", couplings="fixed", houdayer=True)
    assert e.value.status == 5
    sim = Simulation(2, (8, 8), 1, 2, [1.0, 2.0], spin_format="int8", couplings="fixed")
    bad = np.zeros((1, 64, 2), np.int32)
    bad[0, 0, 0] = (1 << 23) + 1
    with pytest.raises(SGError) as e:
        sim.set_couplings_fixed(bad)
    assert e.value.status == 1
    # int32 host reads are the +-J jobs' (their energies are int64 here)
    E = np.zeros((1, 2, 2), np.int32)
    Q = np.zeros((1, 2), np.int32)
    for call in (lambda: sim.measure_async(E, Q), lambda: sim.run_mcs_measure_async(1, E, Q)):
        with pytest.raises(SGError) as e:
            call()
        assert e.value.status == 5
