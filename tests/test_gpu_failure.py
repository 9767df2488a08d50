"""Failure detection without a fault: a bounded device wait that runs out (an mbarrier
that nothing completes) is reported as SG_ETIMEOUT, poisons only its own handle, and
leaves the CUDA context usable for every other handle."""
import ctypes

import numpy as np
import pytest

from helpers import gpu_of

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2003_04621_gb300 import build

    build.build()


def test_expired_wait_is_reported_and_contained():
    from paper_2003_04621_gb300 import sgmc

    L = sgmc.lib()
    bad = gpu_of(ndim=2, dims=(8, 8), n_samples=1, n_chains=2, temps=[1.0, 2.0])
    good = gpu_of(ndim=2, dims=(8, 8), n_samples=1, n_chains=2, temps=[1.0, 2.0])
    assert L.sg_selftest_wait(bad._h, 1024, 0) == 4  # SG_ETIMEOUT
    assert L.sg_run_mcs(bad._h, 1, 0) == 4  # the handle stays poisoned
    with pytest.raises(sgmc.SGError) as e:
        bad.measure()
    assert e.value.status == 4
    good.run_mcs(3)  # the context is intact
    E, Q = good.measure()
    assert np.isfinite(E).all()
    assert L.sg_selftest_wait(good._h, 0, 0) == 1  # bound out of range
