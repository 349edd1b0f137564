"""Sharding boxes across ranks: two gloo ranks on CPU each evolve their box range with the
oracle; the disjoint union of their outputs equals the single-process run bit for bit,
and the benchmark's timing reduction (max over ranks) behaves as stated."""
import importlib.util
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _shard_module():
    spec = importlib.util.spec_from_file_location(
        "_scola_shard", os.path.join(ROOT, "paper_2003_04925_gb300", "shard.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


CFG = dict(L=64.0, Np=16, Ntiles=2, Nbuf=[2, 3, 2, 1, 3, 2, 2, 1], mesh_ratio=1, nsteps=2, a_i=0.05)


def _worker(rank, world, port, out_dir):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import synth_inputs
    from oracle import scola
    shard = _shard_module()
    cfg = scola.ScolaConfig(**CFG)
    costs = [shard.box_cost(scola.box_geometry(cfg, b).Nsc, scola.box_geometry(cfg, b).Ng)
             for b in range(cfg.nboxes)]
    first, count = shard.box_ranges(costs, world)[rank]
    out = scola.run_scola(synth_inputs.white_noise(16, 5), cfg, boxes=range(first, first + count))
    x = torch.from_numpy(out["x"])
    gathered = [torch.empty_like(x) for _ in range(world)]
    dist.all_gather(gathered, x)
    t = torch.tensor([1.0 + rank])
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    if rank == 0:
        np.save(os.path.join(out_dir, "merged.npy"),
                shard.merge_disjoint([g.numpy() for g in gathered], float("nan")))
        np.save(os.path.join(out_dir, "tmax.npy"), t.numpy())
    dist.destroy_process_group()


def test_box_ranges_cover_every_box_once():
    shard = _shard_module()
    costs = [5, 1, 1, 1, 9, 2, 2, 3, 1, 1]
    for world in (1, 2, 3, 4, 10):
        rr = shard.box_ranges(costs, world)
        assert len(rr) == world and all(c >= 1 for _, c in rr)
        assert [b for f, c in rr for b in range(f, f + c)] == list(range(len(costs)))
    with pytest.raises(ValueError):
        shard.box_ranges([1, 2], 3)


@pytest.mark.slow
def test_two_gloo_ranks_reproduce_the_single_run(tmp_path):
    import synth_inputs
    from oracle import scola
    mp.spawn(_worker, args=(2, _free_port(), str(tmp_path)), nprocs=2, join=True)
    merged = np.load(tmp_path / "merged.npy")
    single = scola.run_scola(synth_inputs.white_noise(16, 5), scola.ScolaConfig(**CFG))["x"]
    assert not np.isnan(merged).any()
    assert np.array_equal(merged, single)
    assert float(np.load(tmp_path / "tmax.npy")[0]) == 2.0
