"""Shared test helpers: build the same job on the GPU engine and on the oracle, and
compare their complete states."""
from __future__ import annotations

import math

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


# Inputs that force the exchange's exact branch (see test_gpu_exact_paths.py).
L1 = 4          # rows of the 2D lattice: every wall has L1 bonds
BETA_TOP = 6.0  # the smallest inverse temperature: thresholds exp(-4 beta) 2^32 < 1 above 5.55
EPS = 2e-7      # relative offset of dbeta from the exact threshold value


def wall_spins(L0, n_bands):
    """One 2D L0 x L1 configuration (bits, 1 = spin -1, canonical order): n_bands bands of
    width 2 at x = 4i, 4i+1 flipped, i.e. 2 n_bands flat walls, every site with at most one
    unsatisfied bond."""
    assert 4 * n_bands <= L0
    row = np.zeros(L0, np.uint8)
    for i in range(n_bands):
        row[4 * i:4 * i + 2] = 1
    return np.tile(row, L1)


def pt_word(oracle_mod, k, t, s, c, sim_seed):
    key = (sim_seed & 0xFFFFFFFF, sim_seed >> 32)
    return oracle_mod.philox4x32_10((k, t, s, (c << 20) | 1), key)[0]


def tuned_job(oracle_mod, T, S=3, tuned_sample=1, sim_seed=11, scale=1):
    """Temperatures whose first exchange pass of chain 0 of `tuned_sample` decides every
    pair with |ln u| in a workable range inside the screening margin; returns (temps,
    spins [S][2][T][N], planned perm of that chain after the pass, tuned pair count).
    `scale` multiplies the energies (2^20 for fixed-point couplings of 1.0)."""
    L0 = 4 * T if T > 1 else 4
    N = L0 * L1
    E = [(-2 * N + 4 * j * L1) * scale for j in range(T)]
    perm = list(range(T))
    dbetas, tuned, plan = [], 0, []
    for k in range(T - 1):
        a, b = perm[k], perm[k + 1]
        dE = E[a] - E[b]
        assert dE < 0
        u = pt_word(oracle_mod, k, 0, tuned_sample, 0, sim_seed)
        lnx = math.log(u * 2.0**-32) if u else 0.0
        if 0.05 < abs(lnx) < 20.0:
            sign = -1.0 if (tuned % 2 == 0) else 1.0  # eps < 0: accept, eps > 0: reject
            db = lnx / (dE / scale) * (1.0 + sign * EPS)
            accept = sign < 0
            tuned += 1
        else:
            db = 0.05
            delta = db * (dE / scale)
            x = u * 2.0**-32
            assert abs(x - math.exp(delta)) > 1e-9
            accept = x < math.exp(delta)
        dbetas.append(db)
        plan.append(accept)
        if accept:
            perm[k], perm[k + 1] = b, a
    betas = [BETA_TOP + sum(dbetas[k:]) for k in range(T)]
    temps = [1.0 / bb for bb in betas]
    assert all(temps[k] < temps[k + 1] for k in range(T - 1))
    spins = np.zeros((S, 2, T, N), np.uint8)
    for j in range(T):
        spins[:, :, j, :] = wall_spins(L0, j)
    return dict(L0=L0, temps=temps, spins=spins, perm=np.array(perm, np.int32), tuned=tuned, plan=plan,
                sim_seed=sim_seed, S=S, tuned_sample=tuned_sample)
