"""Checkpoint and resume: a job restored from a checkpoint into a fresh handle with the
same parameters continues exactly as the original (spins, energies, maps, counters,
round trips), for +-J jobs with the cluster move and for general couplings."""
import numpy as np
import pytest

from helpers import gpu_of
from paper_2003_04621_gb300.inputs import gaussian_couplings_fixed, geometric_temps

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2003_04621_gb300 import build

    build.build()


def snapshot(sim):
    E, perm, steps = sim.state()
    out = [E, perm, np.array(steps), sim.spins().cpu().numpy()]
    c = sim.counters()
    out.append(np.array([c["near_threshold"], c["houdayer_sites"]]))
    return out


@pytest.mark.parametrize("fmt", ["packed", "int8"])
def test_resume_equals_uninterrupted(fmt):
    kw = dict(ndim=3, dims=(8, 8, 8), n_samples=3, n_chains=2, temps=geometric_temps(0.5, 2.0, 12), sim_seed=3,
              spin_format=fmt, houdayer=(fmt == "packed"), track_trips=True)
    a = gpu_of(**kw)
    a.run_mcs(4)
    blob = a.checkpoint()
    a.run_mcs(5)
    b = gpu_of(**kw)
    b.restore(blob)
    b.run_mcs(5)
    for x, y in zip(snapshot(a), snapshot(b)):
        np.testing.assert_array_equal(x, y)
    for x, y in zip(a.trips(), b.trips()):
        np.testing.assert_array_equal(x, y)


def test_resume_general_couplings():
    from paper_2003_04621_gb300.sgmc import Simulation

    J = gaussian_couplings_fixed(2, (12, 8), seed=4)
    mk = lambda: Simulation(2, (12, 8), 2, 2, geometric_temps(0.3, 1.5, 6), sim_seed=2, spin_format="int8",
                            couplings="fixed")
    a = mk()
    a.set_couplings_fixed(J)
    a.run_mcs(3)
    blob = a.checkpoint()
    a.run_mcs(4)
    b = mk()
    b.restore(blob)
    b.run_mcs(4)
    for x, y in zip(a.state()[:2], b.state()[:2]):
        np.testing.assert_array_equal(x, y)
    np.testing.assert_array_equal(a.spins().cpu().numpy(), b.spins().cpu().numpy())


def test_restore_refuses_other_parameters():
    from paper_2003_04621_gb300.sgmc import SGError

    a = gpu_of(ndim=2, dims=(8, 8), n_samples=2, n_chains=2, temps=[1.0, 2.0], sim_seed=1)
    blob = a.checkpoint()
    for kw in (dict(sim_seed=2), dict(temps=[1.0, 2.5]), dict(n_samples=3)):
        base = dict(ndim=2, dims=(8, 8), n_samples=2, n_chains=2, temps=[1.0, 2.0], sim_seed=1)
        base.update(kw)
        b = gpu_of(**base)
        with pytest.raises(SGError) as e:
            b.restore(blob)
        assert e.value.status == 1
