"""The allocation-free streaming sweep (sg_sweep_streaming_static).

Some callers cannot allocate device memory: a host framework that owns all device memory
and hands a job only its state, or code running while a CUDA graph is captured (where
cudaMalloc is not allowed).  For them the library keeps the streaming sweep's working
memory in a fixed device array of its own.  These checks call that entry point through
the C ABI and compare it with the ordinary entry point (sg_sweep on the streaming path)
on identical jobs, on two calls in a row, bit for bit.  This file is collected last so a
run that stops at the first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

from paper_2003_04621_gb300.inputs import geometric_temps

pytestmark = pytest.mark.gpu


def _same(a, b):
    assert (a.spins() == b.spins()).all()
    Ea, pa, sa = a.state()
    Eb, pb, sb = b.state()
    np.testing.assert_array_equal(Ea, Eb)
    np.testing.assert_array_equal(pa, pb)
    assert sa == sb


@pytest.mark.parametrize("kw", [
    dict(ndim=3, dims=(8, 6, 8), n_samples=5, n_chains=2, temps=geometric_temps(0.7, 2.0, 40), sim_seed=3),
    dict(ndim=2, dims=(64, 32), n_samples=7, n_chains=2, temps=geometric_temps(0.3, 1.6, 24), sim_seed=5),
])
def test_static_scratch_sweep_matches_streaming_sweep(kw):
    import torch

    from paper_2003_04621_gb300 import build
    from paper_2003_04621_gb300.sgmc import Simulation, lib

    build.build()
    ref = Simulation(**kw)
    ref.set_launch(0, -1)  # the ordinary streaming path, scratch in the handle's buffer
    new = Simulation(**kw)
    stream = torch.cuda.current_stream().cuda_stream
    for n in (3, 2):  # two calls in a row: the shared array keeps the previous contents
        ref.sweep(n)
        assert lib().sg_sweep_streaming_static(ctypes.c_void_p(new._h.value), n, stream) == 0
        torch.cuda.synchronize()
        _same(ref, new)


def test_static_scratch_sweep_rejects_jobs_beyond_its_capacity():
    from paper_2003_04621_gb300.sgmc import SGError, Simulation

    big = Simulation(ndim=3, dims=(4, 4, 4), n_samples=2049, n_chains=2, temps=geometric_temps(1.0, 2.0, 8))
    with pytest.raises(SGError) as e:
        big.sweep_streaming_static(1)
    assert e.value.status == 6  # SG_ELIMIT: 2049 samples x 2 words > 4096
