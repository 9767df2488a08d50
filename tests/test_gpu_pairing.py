"""Paired last words: two chains whose last 32-replica word holds at most 16 replicas
(T <= 16, or 33..48) are swept with a whole sample per CTA, their last words held as ONE
word (lanes 0..15 chain 0, 16..31 chain 1).  Each replica keeps its own Philox counter
(Sec. 2.2) and the fused exchange (Eq. 5) is unchanged, so the state must equal the
oracle's after every MCS and equal the unpaired kernel's bit for bit."""
import numpy as np
import pytest

from helpers import assert_same_state, gpu_of, oracle_of
from paper_2003_04621_gb300.inputs import geometric_temps

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2003_04621_gb300 import build

    build.build()


CASES = [(3, (8, 8, 8), 4), (3, (8, 6, 4), 9), (3, (8, 8, 8), 16), (2, (16, 12), 13), (3, (8, 8, 8), 33),
         (3, (6, 8, 4), 38), (3, (8, 8, 8), 44), (2, (16, 16), 48), (2, (12, 8), 36),
         # lattices smaller than a CTA's threads
         (2, (2, 8), 8), (2, (8, 2), 14), (3, (4, 6, 2), 36), (3, (2, 2, 2), 40)]


@pytest.mark.parametrize("ndim,dims,T", CASES)
def test_paired_mcs_equals_oracle(oracle_mod, ndim, dims, T):
    kw = dict(ndim=ndim, dims=dims, n_samples=3, n_chains=2, temps=geometric_temps(0.4, 2.0, T), sim_seed=21,
              coupling_seed=4, sample_offset=2)
    sim, orc = gpu_of(**kw), oracle_of(oracle_mod, **kw)
    for t in range(4):
        sim.run_mcs(1 if t < 2 else 3)
        orc.mcs(1 if t < 2 else 3)
        assert_same_state(sim, orc, f"T={T} step {t}")
    np.testing.assert_array_equal(sim.counters()["pt_accepts"], orc.pt_stats()[0])


@pytest.mark.parametrize("T", [12, 16, 40, 48])
@pytest.mark.parametrize("shape", [(64, 2), (128, 2), (256, 1), (512, 2)])
def test_paired_equals_unpaired(T, shape):
    """The same job with pairing allowed and forbidden, on several launch shapes: spins,
    energies, maps, round trips and exchange counts identical after 7 MCS."""
    kw = dict(ndim=3, dims=(8, 8, 8), n_samples=5, n_chains=2, temps=geometric_temps(0.9, 2.0, T), sim_seed=5,
              track_trips=True)
    out = []
    for on in (True, False):
        sim = gpu_of(**kw)
        sim.set_launch(*shape)
        sim.set_pairing(on)
        sim.run_mcs(3)
        sim.run_mcs(4)
        E, perm, steps = sim.state()
        out.append((sim.spins().cpu().numpy(), E, perm, steps, sim.trips(), sim.counters()["pt_accepts"]))
    a, b = out
    np.testing.assert_array_equal(a[0], b[0])
    np.testing.assert_array_equal(a[1], b[1])
    np.testing.assert_array_equal(a[2], b[2])
    assert a[3] == b[3]
    for x, y in zip(a[4], b[4]):
        np.testing.assert_array_equal(x, y)
    np.testing.assert_array_equal(a[5], b[5])


def test_paired_then_unpaired_calls(oracle_mod):
    """Paired MCS alternating with the separate sweep / exchange / measure calls (which
    use the unpaired kernels on the re-split words) stay equal to the oracle."""
    kw = dict(ndim=3, dims=(8, 8, 8), n_samples=2, n_chains=2, temps=geometric_temps(0.7, 2.0, 40), sim_seed=3)
    sim, orc = gpu_of(**kw), oracle_of(oracle_mod, **kw)
    for op in "mmsxmsmx":
        if op == "m":
            sim.run_mcs(1)
            orc.mcs(1)
        elif op == "s":
            sim.sweep(1)
            orc.sweep(1)
        else:
            sim.exchange()
            orc.exchange()
        assert_same_state(sim, orc, op)


def test_pairing_switch_refuses_other_values():
    from paper_2003_04621_gb300.sgmc import lib

    sim = gpu_of(ndim=2, dims=(8, 8), n_samples=1, n_chains=2, temps=[1.0, 2.0])
    assert lib().sg_set_pairing(sim._h, 2) == 1
    assert lib().sg_set_pairing(sim._h, 0) == 0


@pytest.mark.parametrize("T", [10, 42])
def test_paired_with_several_sweeps_per_mcs(oracle_mod, T):
    """n_metro = 3 Metropolis sweeps per exchange inside the paired launch."""
    kw = dict(ndim=3, dims=(8, 4, 6), n_samples=2, n_chains=2, temps=geometric_temps(0.5, 1.8, T), sim_seed=9,
              n_metro=3)
    sim = gpu_of(**kw)
    orc = oracle_of(oracle_mod, **{k: v for k, v in kw.items() if k != "n_metro"})
    for t in range(3):
        sim.run_mcs(2)
        orc.mcs(2, n_metro=3)
        assert_same_state(sim, orc, f"T={T} step {t}")


def test_paired_checkpoint_resume():
    """A paired job checkpointed and restored into a fresh handle continues exactly."""
    kw = dict(ndim=3, dims=(8, 8, 8), n_samples=3, n_chains=2, temps=geometric_temps(0.9, 2.0, 44), sim_seed=4,
              track_trips=True)
    a = gpu_of(**kw)
    a.run_mcs(3)
    blob = a.checkpoint()
    a.run_mcs(4)
    b = gpu_of(**kw)
    b.restore(blob)
    b.run_mcs(4)
    np.testing.assert_array_equal(a.spins().cpu().numpy(), b.spins().cpu().numpy())
    for x, y in zip(a.state()[:2], b.state()[:2]):
        np.testing.assert_array_equal(x, y)
    for x, y in zip(a.trips(), b.trips()):
        np.testing.assert_array_equal(x, y)
