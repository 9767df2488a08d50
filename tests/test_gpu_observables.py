"""GPU parity of the overlap plane sums (two-replica measurements of Sec. 3) against
the oracle, bit-exact, for both spin layouts, chains of one and several words, and
lattices whose accumulators outgrow shared memory (kept in global memory)."""
import numpy as np
import pytest

from helpers import gpu_of, oracle_of
from paper_2003_04621_gb300.inputs import geometric_temps, workload_3d_l16

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2003_04621_gb300 import build

    build.build()


def _okw(kw):
    return {k: v for k, v in kw.items() if k not in ("spin_format", "houdayer", "n_metro")}


@pytest.mark.parametrize("ndim,dims,T,fmt", [
    (2, (16, 16), 8, "packed"), (2, (40, 24), 33, "packed"), (3, (8, 8, 8), 12, "packed"),
    (3, (4, 6, 10), 70, "packed"), (3, (6, 6, 6), 12, "int8"), (2, (10, 4), 5, "int8"),
    (2, (8, 800), 4, "packed"),  # 32 lanes x 2 x 800 accumulators exceed shared memory
    (2, (32, 12), 10, "packed"), (3, (24, 4, 4), 40, "packed"),  # half-rows of 16 and 12 sites
    # one-word chains, transposed pass: rows of 6 (5 rows per step, 2 idle lanes), 2 and
    # 40 sites; rows of 96, 128 and 256 sites in 3, 4 and 8 chunks
    (2, (6, 10), 7, "packed"), (3, (2, 6, 4), 9, "packed"), (3, (40, 4, 6), 16, "packed"),
    (2, (96, 16), 8, "packed"), (2, (128, 128), 24, "packed"), (2, (256, 8), 5, "packed"),
])
def test_plane_sums_equal_oracle(oracle_mod, ndim, dims, T, fmt):
    kw = dict(ndim=ndim, dims=dims, n_samples=3, n_chains=2, temps=geometric_temps(0.4, 2.0, T), sim_seed=12,
              coupling_seed=4, spin_format=fmt)
    sim, orc = gpu_of(**kw), oracle_of(oracle_mod, **_okw(kw))
    for t in range(3):
        sim.run_mcs(2)
        orc.mcs(2)
        np.testing.assert_array_equal(sim.qmodes(), orc.qmodes(), err_msg=f"mcs {2 * t + 2}")


def test_plane_sums_full_size_sampled(oracle_mod):
    """The 1024-sample 3D L=16 job; three samples recomputed by the oracle."""
    w = workload_3d_l16()
    kw = dict(ndim=3, dims=w.dims, n_samples=w.n_samples, n_chains=2, temps=list(w.temps), sim_seed=w.sim_seed,
              coupling_seed=w.coupling_seed)
    sim = gpu_of(**kw)
    sim.run_mcs(3)
    P = sim.qmodes()
    for s in (0, 511, 1023):
        o = oracle_of(oracle_mod, **dict(kw, n_samples=1, sample_offset=s))
        o.mcs(3)
        np.testing.assert_array_equal(P[s:s + 1], o.qmodes())
    _, Q = sim.measure()
    np.testing.assert_array_equal(P[:, :, 0, :16].sum(-1), Q)


def test_plane_sums_need_two_chains():
    from paper_2003_04621_gb300.sgmc import SGError

    sim = gpu_of(ndim=2, dims=(8, 8), n_samples=1, n_chains=1, temps=[1.0, 2.0])
    with pytest.raises(SGError) as e:
        sim.qmodes()
    assert e.value.status == 1


@pytest.mark.parametrize("ndim,dims,T", [(2, (256, 256), 5), (3, (48, 48, 48), 32), (2, (2, 2), 3)])
def test_single_pass_measurement_large_lattices(oracle_mod, ndim, dims, T):
    """E by slot and N q of chains of one word come from one pass per sample whose
    bit-sliced counters are summed every 63 iterations: lattices of 65,536 and 110,592
    sites run several such flushes (and the 4-site lattice a partial warp)."""
    kw = dict(ndim=ndim, dims=dims, n_samples=2, n_chains=2, temps=geometric_temps(0.4, 2.0, T), sim_seed=31,
              coupling_seed=8)
    sim, orc = gpu_of(**kw), oracle_of(oracle_mod, **_okw(kw))
    for t in range(2):
        sim.run_mcs(1)
        orc.mcs(1)
        E_g, Q_g = sim.measure()
        E_o, Q_o = orc.measure()
        np.testing.assert_array_equal(E_g, E_o, err_msg=f"E, mcs {t + 1}")
        np.testing.assert_array_equal(Q_g, Q_o, err_msg=f"N q, mcs {t + 1}")


def test_asynchronous_measurement_ring(oracle_mod):
    """sg_measure_async: one read per MCS into its own slot of a pinned ring, queued
    behind the MCS without synchronising (the copies on the simulation's copy stream,
    from alternating staging slots); after sg_measure_wait every slot equals the oracle's
    measurement after the same number of MCS, and a synchronous read afterwards agrees."""
    import torch

    kw = dict(ndim=3, dims=(8, 8, 8), n_samples=3, n_chains=2, temps=geometric_temps(0.5, 2.0, 12), sim_seed=41)
    sim, orc = gpu_of(**kw), oracle_of(oracle_mod, **_okw(kw))
    n = 4
    E = torch.empty((n, 3, 2, 12), dtype=torch.int32, pin_memory=True).numpy()
    Q = torch.empty((n, 3, 12), dtype=torch.int32, pin_memory=True).numpy()
    for k in range(n):
        sim.run_mcs(1)
        sim.measure_async(E[k], Q[k])
    sim.measure_wait()  # the copies, on the simulation's copy stream, are done
    for k in range(n):
        orc.mcs(1)
        E_o, Q_o = orc.measure()
        np.testing.assert_array_equal(E[k], E_o, err_msg=f"E slot {k}")
        np.testing.assert_array_equal(Q[k], Q_o, err_msg=f"N q slot {k}")
    E_s, Q_s = sim.measure()
    np.testing.assert_array_equal(E_s, E[-1])
    np.testing.assert_array_equal(Q_s, Q[-1])



@pytest.mark.parametrize("dims,T", [((32, 64, 64), 4), ((64, 64, 64), 3)])
def test_plane_sums_counter_flushes(oracle_mod, dims, T):
    """Chains of one word on lattices where a warp takes more than 255 steps, so its
    bit-sliced x-plane counters are emptied during the pass (rows of 32 sites, one step
    each; rows of 64 sites in two chunks)."""
    kw = dict(ndim=3, dims=dims, n_samples=1, n_chains=2, temps=geometric_temps(0.6, 1.8, T), sim_seed=5,
              coupling_seed=6)
    sim, orc = gpu_of(**kw), oracle_of(oracle_mod, **_okw(kw))
    sim.run_mcs(2)
    orc.mcs(2)
    np.testing.assert_array_equal(sim.qmodes(), orc.qmodes())



@pytest.mark.parametrize("case", ["fused", "fused_3_mcs", "houdayer", "two_words"])
def test_run_and_measure(oracle_mod, case):
    """sg_run_mcs_measure_async: MCS then the observables in one call, read into a pinned
    ring.  Two one-word chains per CTA measure inside the sweep kernel's last MCS (fused,
    also after 3 MCS in one launch); a Houdayer job and chains of two words fall back to
    the separate kernels.  Every slot equals the oracle's measurement at that point."""
    import torch

    T = 40 if case == "two_words" else 12
    kw = dict(ndim=3, dims=(8, 8, 8), n_samples=3, n_chains=2, temps=geometric_temps(0.5, 2.0, T), sim_seed=43,
              houdayer=(case == "houdayer"))
    sim, orc = gpu_of(**kw), oracle_of(oracle_mod, **_okw(kw))
    if case.startswith("fused"):
        sim.set_launch(256, 2)
    per = 3 if case == "fused_3_mcs" else 1
    n = 4
    E = torch.empty((n, 3, 2, T), dtype=torch.int32, pin_memory=True).numpy()
    Q = torch.empty((n, 3, T), dtype=torch.int32, pin_memory=True).numpy()
    for k in range(n):
        sim.run_mcs_measure_async(per, E[k], Q[k])
    sim.measure_wait()
    for k in range(n):
        orc.mcs(per, houdayer=kw["houdayer"])
        E_o, Q_o = orc.measure()
        np.testing.assert_array_equal(E[k], E_o, err_msg=f"E slot {k}")
        np.testing.assert_array_equal(Q[k], Q_o, err_msg=f"N q slot {k}")
    E_s, Q_s = sim.measure()
    np.testing.assert_array_equal(E_s, E[-1])
    np.testing.assert_array_equal(Q_s, Q[-1])


def test_run_and_measure_one_chain(oracle_mod):
    """With one chain there is no overlap: the call returns E by slot only."""
    import torch

    kw = dict(ndim=2, dims=(16, 16), n_samples=2, n_chains=1, temps=geometric_temps(0.5, 2.0, 20), sim_seed=47)
    sim, orc = gpu_of(**kw), oracle_of(oracle_mod, **_okw(kw))
    E = torch.empty((3, 2, 1, 20), dtype=torch.int32, pin_memory=True).numpy()
    for k in range(3):
        sim.run_mcs_measure_async(2, E[k])
    sim.measure_wait()
    for k in range(3):
        orc.mcs(2)
        np.testing.assert_array_equal(E[k], orc.measure()[0], err_msg=f"E slot {k}")
