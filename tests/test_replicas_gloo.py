"""Two ranks on CPU (gloo): replica sharding reproduces one process's draws exactly, and
the end-of-run reduction takes the max of the times and the sum of the counts."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist

    from oracle import tnmc
    from paper_2104_13264_gb300 import instances, replicas
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=world)
    inst = instances.random_small(3, 4, 0.8, 2, seed=3)
    env = tnmc.build_env(inst.Jh, inst.Jv, inst.h, inst.beta, inst.chi)
    B = 5
    sp, lq, E, _ = tnmc.sample(env, B, seed=7, sample_offset=replicas.sample_offset(rank, world, 1, B))
    ms, n = replicas.reduce_timing(1.0 + rank, 10 + rank, dist)
    np.savez(os.path.join(out_dir, "rank%d.npz" % rank), sp=sp, lq=lq, ms=ms, n=n)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_shards_and_reduction(tmp_path):
    import torch.multiprocessing as mp
    port = _free_port()
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, start_method="spawn", join=True)
    r0 = np.load(tmp_path / "rank0.npz")
    r1 = np.load(tmp_path / "rank1.npz")
    from oracle import tnmc
    from paper_2104_13264_gb300 import instances, replicas
    inst = instances.random_small(3, 4, 0.8, 2, seed=3)
    env = tnmc.build_env(inst.Jh, inst.Jv, inst.h, inst.beta, inst.chi)
    sp, lq, _, _ = tnmc.sample(env, 10, seed=7, sample_offset=replicas.sample_offset(0, 1, 1, 10))
    assert np.array_equal(np.concatenate([r0["sp"], r1["sp"]]), sp)
    assert np.array_equal(np.concatenate([r0["lq"], r1["lq"]]), lq)
    for r in (r0, r1):
        assert float(r["ms"]) == 2.0 and int(r["n"]) == 21


def test_offsets_are_disjoint():
    from paper_2104_13264_gb300 import replicas
    seen = set()
    for step in range(3):
        for rank in range(4):
            o = replicas.sample_offset(rank, 4, step, 8)
            rng = set(range(o, o + 8))
            assert not (rng & seen)
            seen |= rng
    assert seen == set(range(3 * 4 * 8))
    assert replicas.reduce_timing(3.5, 7) == (3.5, 7)
