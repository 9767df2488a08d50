"""The C-ABI library loads and exports every entry point ``include/sgmc.h`` declares.
No compute call is made: this runs without a GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "sgmc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sg_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libsgmc():
    from paper_2003_04621_gb300 import build

    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_symbols()
    for core in ("sg_create", "sg_sweep", "sg_exchange", "sg_houdayer", "sg_run_mcs", "sg_measure", "sg_destroy"):
        assert core in names


def test_library_exports_every_declared_symbol(libsgmc):
    missing = [n for n in declared_symbols() if not hasattr(libsgmc, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    from paper_2003_04621_gb300 import sgmc

    assert sorted(sgmc.EXPORTED) == declared_symbols() or set(declared_symbols()) <= set(sgmc.EXPORTED)


def test_parameter_validation_needs_no_gpu(libsgmc):
    from paper_2003_04621_gb300 import sgmc

    sgmc.lib()
    ok, _t = sgmc.make_params(3, (16, 16, 16), 4, 2, [1.0, 1.5])
    assert sgmc.query_bytes(ok) > 4 * 16**3 * 4
    cases = [
        (dict(ndim=3, dims=(5, 16, 16), n_samples=4, n_chains=2, temps=[1.0, 1.5]), 5),  # odd extent
        (dict(ndim=4, dims=(4, 4, 4), n_samples=4, n_chains=2, temps=[1.0]), 1),
        (dict(ndim=2, dims=(4, 4), n_samples=0, n_chains=2, temps=[1.0]), 1),
        (dict(ndim=2, dims=(4, 4), n_samples=1, n_chains=3, temps=[1.0]), 1),
        (dict(ndim=2, dims=(4, 4), n_samples=1, n_chains=2, temps=[1.5, 1.0]), 1),  # not ascending
        (dict(ndim=2, dims=(4, 4), n_samples=1, n_chains=2, temps=[-1.0, 1.0]), 1),
        (dict(ndim=2, dims=(4, 4), n_samples=1, n_chains=1, temps=[1.0], houdayer=True), 1),
        (dict(ndim=2, dims=(4, 4), n_samples=1, n_chains=2, temps=[1.0], p_plus=1.5), 1),
        (dict(ndim=2, dims=(4, 4), n_samples=1, n_chains=2, temps=[1.0 + k for k in range(4097)]), 1),  # > 4096
        (dict(ndim=3, dims=(512, 512, 512), n_samples=1, n_chains=2, temps=[1.0]), 5),  # > 2^26 sites
        (dict(ndim=2, dims=(4, 4), n_samples=1, n_chains=2, temps=[1.0], couplings="fixed"), 5),  # packed
        (dict(ndim=2, dims=(4, 4), n_samples=1, n_chains=2, temps=[1.0], couplings="fixed", spin_format="int8",
              houdayer=True), 5),
        (dict(ndim=2, dims=(4, 4), n_samples=1, n_chains=2, temps=[1.0, 2.0], houdayer=True, houdayer_slots=3), 1),
        (dict(ndim=2, dims=(4, 4), n_samples=1, n_chains=2, temps=[1.0, 2.0], houdayer=True, houdayer_slots=-1), 1),
    ]
    for kw, want in cases:
        p, _t = sgmc.make_params(**kw)
        with pytest.raises(sgmc.SGError) as e:
            sgmc.query_bytes(p)
        assert e.value.status == want, kw
    # raw fields outside their ranges
    for field, value in (("houdayer", 3), ("track_trips", 2), ("coupling_kind", 2), ("spin_format", 7),
                         ("n_metro", 0)):
        p, _t = sgmc.make_params(2, (4, 4), 1, 2, [1.0])
        setattr(p, field, value)
        with pytest.raises(sgmc.SGError) as e:
            sgmc.query_bytes(p)
        assert e.value.status == 1, field
