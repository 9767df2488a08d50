"""GPU parity of the round-trip counters (tunnelling time, Sec. 2.3) with the oracle on
every exchange path: fused in the resident kernel (packed and int8), the separate
exchange kernel (chains longer than a CTA's words, the streaming sweep), the energy +
exchange launch after a Houdayer move, and a batch."""
import numpy as np
import pytest

from helpers import gpu_of, oracle_of
from paper_2003_04621_gb300.inputs import geometric_temps

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2003_04621_gb300 import build

    build.build()


def _okw(kw):
    return {k: v for k, v in kw.items() if k not in ("spin_format", "houdayer", "n_metro", "track_trips")}


CASES = [
    ("fused_packed", dict(ndim=3, dims=(6, 6, 6), T=12), None),
    ("fused_packed_32", dict(ndim=2, dims=(16, 12), T=32), None),
    ("unfused_40", dict(ndim=3, dims=(4, 6, 4), T=40), None),
    ("int8", dict(ndim=3, dims=(6, 6, 6), T=12, spin_format="int8"), None),
    ("streaming", dict(ndim=2, dims=(16, 16), T=8), "stream"),
    ("houdayer", dict(ndim=2, dims=(16, 16), T=8, houdayer=True), None),
]


@pytest.mark.parametrize("name,cfg,mode", CASES, ids=[c[0] for c in CASES])
def test_trips_equal_oracle(oracle_mod, name, cfg, mode):
    cfg = dict(cfg)
    T = cfg.pop("T")
    kw = dict(n_samples=4, n_chains=2, temps=geometric_temps(0.8, 2.5, T), sim_seed=5, coupling_seed=2,
              track_trips=True, **cfg)
    sim, orc = gpu_of(**kw), oracle_of(oracle_mod, **_okw(kw))
    if mode == "stream":
        sim.set_launch(256, -1)
    houd = bool(kw.get("houdayer", False))
    for step in (1, 7, 25, 40):
        sim.run_mcs(step)
        orc.mcs(step, houdayer=houd)
        n, tot = sim.trips()
        no, toto = orc.trips()
        np.testing.assert_array_equal(n, no)
        np.testing.assert_array_equal(tot, toto)
    if T <= 12:
        assert orc.trips()[0].sum() > 0  # short chains complete trips within the run


def test_rotating_chain_on_the_gpu(oracle_mod):
    """Every swap accepted: each completed trip lasts exactly T passes."""
    T = 12
    kw = dict(ndim=2, dims=(8, 8), n_samples=3, n_chains=2, temps=[1.0 + k * 1e-14 for k in range(T)],
              sim_seed=3, track_trips=True)
    sim = gpu_of(**kw)
    sim.run_mcs(50)
    n, tot = sim.trips()
    first = [T if j == 0 else j for j in range(T)]
    expect = sum(max(0, (50 - t0) // T) for t0 in first)
    np.testing.assert_array_equal(n, expect)
    np.testing.assert_array_equal(tot, T * expect)


def test_trips_in_a_batch_equal_alone():
    from paper_2003_04621_gb300.sgmc import Batch

    mk = lambda: [gpu_of(ndim=3, dims=(8, 8, 8), n_samples=5, n_chains=2, temps=geometric_temps(0.9, 2.0, T),
                         sim_seed=9, track_trips=True) for T in (16, 40)]
    alone = mk()
    for s in alone:
        s.run_mcs(30)
    together = mk()
    b = Batch(together, mcs_per_launch=10)
    b.run(3)
    b.close()
    for a, t in zip(alone, together):
        for x, y in zip(a.trips(), t.trips()):
            np.testing.assert_array_equal(x, y)


def test_trips_need_the_flag():
    from paper_2003_04621_gb300.sgmc import SGError

    sim = gpu_of(ndim=2, dims=(8, 8), n_samples=1, n_chains=2, temps=[1.0, 2.0])
    with pytest.raises(SGError) as e:
        sim.trips()
    assert e.value.status == 1
