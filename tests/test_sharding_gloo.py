"""The multi-rank path on the CPU: two gloo ranks, each running its shard of a job's
samples (job-wide sample offsets), must together reproduce the whole job run by one
process, and the timing reduction must return the maximum over ranks.

The ranks run the oracle (the GPU engine keys its random words the same way; the GPU
tests check that engine against the oracle with the same offsets)."""
import os
import socket

import numpy as np
import pytest

from paper_2003_04621_gb300.inputs import Workload, geometric_temps


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _job(n_samples):
    return Workload("2d_L8_houdayer", 2, (8, 6), n_samples, 2, geometric_temps(0.4, 2.0, 5), coupling_seed=3,
                    sim_seed=11, houdayer=True, n_mcs=12)


def _run(w):
    import oracle

    o = oracle.Oracle(oracle.OracleParams(w.ndim, w.dims, w.n_samples, w.n_chains, list(w.temps),
                                          coupling_seed=w.coupling_seed, sim_seed=w.sim_seed,
                                          sample_offset=w.sample_offset))
    o.mcs(w.n_mcs, houdayer=w.houdayer)
    E, Q = o.measure()
    return {"spins": o.spins(), "E": o.energies(), "perm": o.perm()[0], "Em": E, "Q": Q}


def _rank_main(rank, world, port, mode, out_dir):
    import torch.distributed as dist

    from paper_2003_04621_gb300 import shard

    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    ws, r, local = shard.dist_env()
    assert (ws, r, local) == (world, rank, rank)
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        if mode == "weak":
            w = shard.weak_shard(_job(3), rank)
        else:
            w = shard.strong_shard(_job(5), world, rank)
        res = _run(w)
        got = [None] * world
        dist.all_gather_object(got, (w.sample_offset, w.n_samples, res))
        # the reduction bench.py applies to its timed region
        t = shard.max_over_ranks(1.5 + rank)
        assert t == 1.5 + (world - 1)
        if rank == 0:
            np.savez(os.path.join(out_dir, "shards.npz"),
                     **{f"{k}_{i}": v for i, (_, _, rr) in enumerate(got) for k, v in rr.items() if v is not None},
                     offsets=np.array([g[0] for g in got]), sizes=np.array([g[1] for g in got]))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("mode", ["weak", "strong"])
def test_two_gloo_ranks_reproduce_the_whole_job(oracle_mod, tmp_path, mode):
    import torch.multiprocessing as mp

    world = 2
    mp.spawn(_rank_main, args=(world, _free_port(), mode, str(tmp_path)), nprocs=world, join=True)
    d = np.load(tmp_path / "shards.npz")
    S = 3 * world if mode == "weak" else 5
    whole = _run(_job(S))
    offs, sizes = d["offsets"], d["sizes"]
    assert list(offs) == [int(x) for x in np.cumsum([0] + list(sizes[:-1]))]
    assert int(sizes.sum()) == S
    for key in ("spins", "E", "perm", "Em", "Q"):
        if whole[key] is None:
            continue
        joined = np.concatenate([d[f"{key}_{i}"] for i in range(world)], axis=0)
        np.testing.assert_array_equal(joined, whole[key], err_msg=key)
