"""GPU parity: the sm_103a engine, called through its C-ABI, against the CPU oracle.

The method is an exact Markov chain driven by a counter-based random stream, so the
tolerance is zero: after every step the spins, energies, replica maps, E by slot and
N q must be identical (integers, bit for bit).  The one permitted divergence would be a
replica-exchange decision within 1e-12 of its threshold; both sides count those and
the count must be 0 here.
"""
import numpy as np
import pytest

from helpers import assert_same_state, gpu_of, oracle_of
from paper_2003_04621_gb300.inputs import geometric_temps, workload_2d_l128_houdayer, workload_3d_l6, workload_3d_l16

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch

    from paper_2003_04621_gb300 import build

    build.build()
    assert torch.cuda.is_available()


def kw_of(w, **over):
    kw = dict(ndim=w.ndim, dims=tuple(w.dims), n_samples=w.n_samples, n_chains=w.n_chains, temps=list(w.temps),
              coupling_seed=w.coupling_seed, sim_seed=w.sim_seed, p_plus=w.p_plus, spin_format=w.spin_format,
              sample_offset=w.sample_offset)
    kw.update(over)
    return kw


def _gpu_kw(kw):
    return {k: v for k, v in kw.items()}


def _oracle_kw(kw):
    return {k: v for k, v in kw.items() if k not in ("spin_format", "houdayer", "n_metro")}


@pytest.mark.parametrize("fmt", ["int8", "packed"])
def test_3d_l6_every_mcs_for_200_mcs(oracle_mod, fmt):
    """3D L=6, 8 samples x 2 chains x 12 temps, Metropolis + PT: identical after every MCS."""
    kw = kw_of(workload_3d_l6(), spin_format=fmt)
    sim, orc = gpu_of(**kw), oracle_of(oracle_mod, **_oracle_kw(kw))
    assert_same_state(sim, orc, "after create")
    np.testing.assert_array_equal(sim.thresholds(), orc.thresholds())
    for t in range(200):
        sim.run_mcs(1)
        orc.mcs(1)
        assert_same_state(sim, orc, f"{fmt} mcs {t}", check_spins=(t % 10 == 0 or t < 5))
    assert_same_state(sim, orc, "end")
    acc_o, _ = orc.pt_stats()
    c = sim.counters()
    np.testing.assert_array_equal(c["pt_accepts"], acc_o)
    assert c["near_threshold"] == 0 and orc.counters()["near_threshold"] == 0


def test_int8_and_packed_formats_agree():
    kw = kw_of(workload_3d_l6())
    a = gpu_of(**dict(kw, spin_format="int8"))
    b = gpu_of(**dict(kw, spin_format="packed"))
    for _ in range(3):
        a.run_mcs(5)
        b.run_mcs(5)
        assert (a.spins() == b.spins()).all()
        np.testing.assert_array_equal(a.measure()[0], b.measure()[0])
        np.testing.assert_array_equal(a.measure()[1], b.measure()[1])


def test_3d_l16_reduced_samples_every_mcs(oracle_mod):
    """3D L=16 x 32 temps (two full 32-replica words per sample): 3 samples taken from
    the middle of the 1024-sample job, compared after each of 4 MCS."""
    kw = kw_of(workload_3d_l16(), n_samples=3, sample_offset=510)
    sim, orc = gpu_of(**kw), oracle_of(oracle_mod, **_oracle_kw(kw))
    assert_same_state(sim, orc, "after create")
    for t in range(4):
        sim.run_mcs(1)
        orc.mcs(1)
        assert_same_state(sim, orc, f"mcs {t}")


def test_3d_l16_full_size_sampled(oracle_mod):
    """The full 1024-sample job in the launch configuration the benchmark times; three
    samples recomputed one by one by the oracle (keys use the job-wide sample index)."""
    import torch

    w = workload_3d_l16()
    sim = gpu_of(**kw_of(w))
    picks = [0, 517, 1023]
    orcs = [oracle_of(oracle_mod, **_oracle_kw(kw_of(w, n_samples=1, sample_offset=s))) for s in picks]
    for t in range(3):
        sim.run_mcs(1)
        E, perm, _ = sim.state()
        Em, Q = sim.measure()
        sp = sim.spins()
        for s, o in zip(picks, orcs):
            o.mcs(1)
            np.testing.assert_array_equal(E[s:s + 1], o.energies())
            np.testing.assert_array_equal(perm[s:s + 1], o.perm()[0])
            np.testing.assert_array_equal(Em[s:s + 1], o.measure()[0])
            np.testing.assert_array_equal(Q[s:s + 1], o.measure()[1])
            np.testing.assert_array_equal(sp[s:s + 1].cpu().numpy(), o.spins())
        del sp
        torch.cuda.empty_cache()
    assert sim.counters()["near_threshold"] == 0


def test_2d_l128_padded_words(oracle_mod):
    """2D L=128 x 24 temps: each chain padded into its own 32-bit word (24 lanes used)."""
    kw = kw_of(workload_2d_l128_houdayer(), n_samples=2, sample_offset=100)
    sim, orc = gpu_of(**kw), oracle_of(oracle_mod, **_oracle_kw(kw))
    for t in range(3):
        sim.run_mcs(1)
        orc.mcs(1)
        assert_same_state(sim, orc, f"mcs {t}")


@pytest.mark.parametrize("fmt,T", [("packed", 40), ("int8", 40), ("packed", 450)])
def test_chain_longer_than_a_word(oracle_mod, fmt, T):
    """40 temperatures: a chain spans two words, so sweeps and exchange run as separate
    kernels (the unfused path).  450 temperatures: 15 words per chain, so the overlap
    kernel stages its 30 word planes in tiles shorter than the lattice."""
    kw = dict(ndim=3, dims=(4, 6, 4) if T < 100 else (8, 8, 8), n_samples=3, n_chains=2,
              temps=geometric_temps(0.5, 3.0, T), coupling_seed=9, sim_seed=4, spin_format=fmt)
    sim, orc = gpu_of(**kw), oracle_of(oracle_mod, **_oracle_kw(kw))
    for t in range(6):
        sim.run_mcs(1)
        orc.mcs(1)
        assert_same_state(sim, orc, f"mcs {t}")


@pytest.mark.parametrize("ndim,dims", [(3, (2, 2, 2)), (3, (2, 4, 2)), (2, (2, 2)), (2, (2, 6)), (2, (6, 2)),
                                       (3, (8, 2, 6))])
def test_axes_of_length_two_and_ragged_shapes(oracle_mod, ndim, dims):
    kw = dict(ndim=ndim, dims=dims, n_samples=5, n_chains=2, temps=geometric_temps(0.4, 2.5, 7), sim_seed=11,
              coupling_seed=3)
    sim, orc = gpu_of(**kw), oracle_of(oracle_mod, **_oracle_kw(kw))
    for t in range(8):
        sim.run_mcs(1)
        orc.mcs(1)
        assert_same_state(sim, orc, f"{dims} mcs {t}")


@pytest.mark.parametrize("C,T", [(1, 1), (1, 5), (2, 1), (2, 33)])
def test_degenerate_chain_shapes(oracle_mod, C, T):
    kw = dict(ndim=2, dims=(8, 10), n_samples=3, n_chains=C, temps=geometric_temps(0.6, 2.0, T) if T > 1 else [1.3],
              sim_seed=21)
    sim, orc = gpu_of(**kw), oracle_of(oracle_mod, **_oracle_kw(kw))
    for t in range(5):
        sim.run_mcs(1)
        orc.mcs(1)
        assert_same_state(sim, orc, f"C={C} T={T} mcs {t}")


def test_call_sequences(oracle_mod):
    """sweep/exchange in an arbitrary order equal the same oracle calls."""
    kw = dict(ndim=3, dims=(6, 4, 4), n_samples=4, n_chains=2, temps=geometric_temps(0.5, 2.0, 9), sim_seed=5)
    sim, orc = gpu_of(**kw), oracle_of(oracle_mod, **_oracle_kw(kw))
    for op in ["s3", "x", "s1", "x", "x", "m2", "s2", "m1", "x"]:
        if op[0] == "s":
            sim.sweep(int(op[1:]))
            orc.sweep(int(op[1:]))
        elif op == "x":
            sim.exchange()
            orc.exchange()
        else:
            sim.run_mcs(int(op[1:]))
            orc.mcs(int(op[1:]))
        assert_same_state(sim, orc, op)
    _, _, steps = sim.state()
    c = orc.counters()
    assert steps[0] == c["t_metro"] and steps[1] == c["t_pt"]


def test_many_mcs_in_one_launch_equal_stepwise():
    kw = kw_of(workload_3d_l16(), n_samples=8)
    a, b = gpu_of(**kw), gpu_of(**kw)
    a.run_mcs(9)
    for _ in range(9):
        b.run_mcs(1)
    assert (a.spins() == b.spins()).all()
    np.testing.assert_array_equal(a.state()[0], b.state()[0])
    np.testing.assert_array_equal(a.state()[1], b.state()[1])


def test_imported_gauge_transformed_state(oracle_mod):
    """Couplings and spins set through the import calls: a gauge-transformed copy evolves
    as tau s(t) with identical energies and maps (Eq. 1 is gauge invariant)."""
    import torch

    kw = dict(ndim=3, dims=(6, 6, 4), n_samples=3, n_chains=2, temps=geometric_temps(0.5, 2.0, 6), sim_seed=17)
    a, b = gpu_of(**kw), gpu_of(**kw)
    orc = oracle_of(oracle_mod, **_oracle_kw(kw))
    J = a.couplings().cpu().numpy().astype(np.int64)
    np.testing.assert_array_equal(J, orc.couplings())
    N, d = 6 * 6 * 4, 3
    rng = np.random.default_rng(1)
    tau = rng.choice([-1, 1], size=(3, N))
    idx = np.arange(N)
    x, y, z = idx % 6, (idx // 6) % 6, idx // 36
    fwd = [((x + 1) % 6) + 6 * (y + 6 * z), x + 6 * (((y + 1) % 6) + 6 * z), x + 6 * (y + 6 * ((z + 1) % 4))]
    Jg = np.stack([tau * J[:, :, mu] * tau[:, fwd[mu]] for mu in range(d)], axis=-1)
    s0 = 1 - 2 * a.spins().cpu().numpy().astype(np.int64)
    b.set_couplings(Jg.astype(np.int8))
    b.set_spins(((1 - s0 * tau[:, None, None, :]) // 2).astype(np.uint8))
    orc.set_couplings(Jg.astype(np.int8))
    orc.set_spins(((1 - s0 * tau[:, None, None, :]) // 2).astype(np.uint8))
    np.testing.assert_array_equal(a.state()[0], b.state()[0])
    for t in range(6):
        a.run_mcs(1)
        b.run_mcs(1)
        orc.mcs(1)
        sa = 1 - 2 * a.spins().cpu().numpy().astype(np.int64)
        sb = 1 - 2 * b.spins().cpu().numpy().astype(np.int64)
        np.testing.assert_array_equal(sb, sa * tau[:, None, None, :])
        np.testing.assert_array_equal(a.state()[0], b.state()[0])
        assert_same_state(b, orc, f"gauge mcs {t}")
    torch.cuda.synchronize()


def test_status_codes_on_device():
    import ctypes

    import torch

    from paper_2003_04621_gb300 import sgmc

    L = sgmc.lib()
    p, _t = sgmc.make_params(3, (8, 8, 8), 2, 2, [1.0, 2.0])
    need = sgmc.query_bytes(p)
    buf = torch.empty(need + 512, dtype=torch.uint8, device="cuda")
    base = (buf.data_ptr() + 255) & ~255
    h = ctypes.c_void_p()
    stream = torch.cuda.current_stream().cuda_stream
    assert L.sg_create(ctypes.byref(p), ctypes.c_void_p(base), need - 256, stream, ctypes.byref(h)) == 2
    assert L.sg_create(ctypes.byref(p), ctypes.c_void_p(base + 16), need, stream, ctypes.byref(h)) == 1
    assert L.sg_create(ctypes.byref(p), ctypes.c_void_p(base), need, stream, ctypes.byref(h)) == 0
    assert L.sg_sweep(h, -1, stream) == 1
    assert L.sg_sweep(h, 0, stream) == 0
    assert L.sg_run_mcs(h, 0, stream) == 0
    p1, _t1 = sgmc.make_params(3, (8, 8, 8), 2, 1, [1.0, 2.0])
    need1 = sgmc.query_bytes(p1)
    buf1 = torch.empty(need1 + 512, dtype=torch.uint8, device="cuda")
    h1 = ctypes.c_void_p()
    assert L.sg_create(ctypes.byref(p1), ctypes.c_void_p((buf1.data_ptr() + 255) & ~255), need1, stream,
                       ctypes.byref(h1)) == 0
    assert L.sg_houdayer(h1, stream) == 1  # one chain: no pairs
    L.sg_destroy(h1)
    L.sg_destroy(h)
    # a lattice too large for the resident kernels is refused, not run
    pb, _tb = sgmc.make_params(2, (512, 512), 1, 2, [1.0])
    need_b = sgmc.query_bytes(pb)
    bufb = torch.empty(need_b + 512, dtype=torch.uint8, device="cuda")
    hb = ctypes.c_void_p()
    st = L.sg_create(ctypes.byref(pb), ctypes.c_void_p((bufb.data_ptr() + 255) & ~255), need_b, stream,
                     ctypes.byref(hb))
    assert st in (0, 5)
    if st == 0:
        L.sg_destroy(hb)


@pytest.mark.parametrize("ndim,dims,T", [(3, (16, 16, 16), 32), (2, (32, 48), 24), (3, (6, 8, 4), 40),
                                         (3, (8, 8, 8), 20)])
def test_every_launch_shape_gives_identical_results(oracle_mod, ndim, dims, T):
    """The resident kernel's CTA size and words per CTA are tuning knobs only."""
    kw = dict(ndim=ndim, dims=dims, n_samples=3, n_chains=2, temps=geometric_temps(0.5, 2.0, T), sim_seed=3)
    orc = oracle_of(oracle_mod, **_oracle_kw(kw))
    orc.mcs(3)
    ran = 0
    from paper_2003_04621_gb300.sgmc import SGError

    for nt in (64, 128, 256, 512, 1024):
        for words in (1, 2):
            sim = gpu_of(**kw)
            try:
                sim.set_launch(nt, words)
            except SGError:
                continue
            sim.run_mcs(3)
            assert_same_state(sim, orc, f"threads={nt} words={words}")
            ran += 1
    assert ran >= 2


@pytest.mark.parametrize("fmt", ["packed", "int8"])
def test_maximum_temperature_count(oracle_mod, fmt):
    """n_temps at its limit, 4096: a chain of 128 words (packed) or 4096 bytes per site
    (int8) on a 4x4 lattice; sweeps, exchange passes and the measurement at that size."""
    kw = dict(ndim=2, dims=(4, 4), n_samples=1, n_chains=2, temps=geometric_temps(0.3, 5.0, 4096), sim_seed=13,
              coupling_seed=2, spin_format=fmt)
    sim, orc = gpu_of(**kw), oracle_of(oracle_mod, **_oracle_kw(kw))
    for t in range(3):
        sim.run_mcs(1)
        orc.mcs(1)
        assert_same_state(sim, orc, f"mcs {t}")


def test_maximum_lattice(oracle_mod):
    """N at its limit, 2^26 sites (2D 8192 x 8192), one chain of one replica; 2^26 + 2
    more sites are refused (the create call's checks run on the host)."""
    from paper_2003_04621_gb300.sgmc import SGError

    kw = dict(ndim=2, dims=(8192, 8192), n_samples=1, n_chains=1, temps=[2.2], sim_seed=17, coupling_seed=19)
    sim, orc = gpu_of(**kw), oracle_of(oracle_mod, **_oracle_kw(kw))
    sim.run_mcs(1)
    orc.mcs(1)
    assert_same_state(sim, orc, "mcs 1")
    sim.close()
    with pytest.raises(SGError) as e:
        gpu_of(**dict(kw, dims=(8192, 8194)))
    assert e.value.status == 5
