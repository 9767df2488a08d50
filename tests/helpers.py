"""Shared test helpers: build the same job on the GPU engine and on the oracle, and
compare their complete states."""
from __future__ import annotations

import numpy as np

PARAM_KEYS = ("ndim", "dims", "n_samples", "n_chains", "temps", "coupling_seed", "sim_seed", "p_plus",
              "sample_offset")


def oracle_of(oracle_mod, **kw):
    p = {k: kw[k] for k in PARAM_KEYS if k in kw}
    return oracle_mod.Oracle(oracle_mod.OracleParams(
        p["ndim"], p["dims"], p["n_samples"], p["n_chains"], list(p["temps"]),
        coupling_seed=p.get("coupling_seed", 1), p_plus=p.get("p_plus", 0.5), sim_seed=p.get("sim_seed", 1),
        sample_offset=p.get("sample_offset", 0), houdayer_slots=kw.get("houdayer_slots", 0)))


def gpu_of(**kw):
    from paper_2003_04621_gb300.sgmc import Simulation

    return Simulation(**kw)


def assert_same_state(sim, orc, where="", check_spins=True, samples=None):
    """Spins, energies, replica maps, E by slot and N q must be identical."""
    E_g, perm_g, _ = sim.state()
    E_o = orc.energies()
    perm_o = orc.perm()[0]
    sel = slice(None) if samples is None else samples
    np.testing.assert_array_equal(E_g[sel], E_o, err_msg=f"energies {where}")
    np.testing.assert_array_equal(perm_g[sel], perm_o, err_msg=f"perm {where}")
    Em_g, Q_g = sim.measure()
    Em_o, Q_o = orc.measure()
    np.testing.assert_array_equal(Em_g[sel], Em_o, err_msg=f"E by slot {where}")
    if Q_o is not None:
        np.testing.assert_array_equal(Q_g[sel], Q_o, err_msg=f"N q {where}")
    if check_spins:
        sp = sim.spins()
        sp = (sp[sel] if samples is not None else sp).cpu().numpy()
        np.testing.assert_array_equal(sp, orc.spins(), err_msg=f"spins {where}")
