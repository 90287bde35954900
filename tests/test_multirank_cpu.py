"""The multi-process (one rank per GPU) form on CPU: two gloo ranks each step
their own env shard with the oracle; the shards gathered on rank 0 equal the
unsharded run, and the benchmark's max-over-ranks reduction and whole-job
throughput behave as the single-GPU form expects."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as tmp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, n_per_rank, steps, out_dir):
    import sys

    sys.path.insert(0, ROOT)
    import oracle
    from paper_2604_27162_gb300 import shard as S
    from paper_2604_27162_gb300 import workloads as W

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        c = W.ten1k()
        base = S.env_base(rank, n_per_rank)
        w = oracle.World(n_per_rank, c["seed"], c["descs"], env_id_base=base)
        obs, rew, done = [], [], []
        for _ in range(steps):
            s = w.step()
            o, r, d = s["obs"], s["reward"], s["done"]
            obs.append(np.array(o, copy=True))
            rew.append(np.array(r, copy=True))
            done.append(np.array(d, copy=True))
        mine = (np.stack(obs), np.stack(rew), np.stack(done))
        gathered = [None] * world
        dist.all_gather_object(gathered, mine)
        # the benchmark's reduction: max of the per-rank times
        t_max = S.max_over_ranks(1.0 + rank)
        if rank == 0:
            np.save(os.path.join(out_dir, "t_max.npy"), np.array([t_max]))
            for i, g in enumerate(gathered):
                for j, a in enumerate(g):
                    np.save(os.path.join(out_dir, "r%d_%d.npy" % (i, j)), a)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_rank_shards_equal_unsharded_run(tmp_path):
    import sys

    sys.path.insert(0, ROOT)
    import oracle
    from paper_2604_27162_gb300 import shard as S
    from paper_2604_27162_gb300 import workloads as W

    world, n_per_rank, steps = 2, 6, 40
    tmp.start_processes(_rank_main, args=(world, _free_port(), n_per_rank, steps, str(tmp_path)),
                        nprocs=world, join=True, start_method="spawn")
    assert float(np.load(tmp_path / "t_max.npy")[0]) == 2.0
    c = W.ten1k()
    whole = oracle.World(world * n_per_rank, c["seed"], c["descs"])
    ref = [[], [], []]
    for _ in range(steps):
        s = whole.step()
        o, r, d = s["obs"], s["reward"], s["done"]
        ref[0].append(np.array(o, copy=True))
        ref[1].append(np.array(r, copy=True))
        ref[2].append(np.array(d, copy=True))
    ref = [np.stack(x) for x in ref]
    parts = [[np.load(tmp_path / ("r%d_%d.npy" % (i, j))) for j in range(3)] for i in range(world)]
    # obs words, rewards and done bytes: per-rank slices concatenate along the env axis
    for j in range(3):
        cat = np.concatenate([parts[i][j] for i in range(world)], axis=1)
        assert cat.shape == ref[j].shape
        assert np.array_equal(cat, ref[j]), "output %d differs between sharded and whole run" % j
    assert S.weak_throughput(100.0, world, 2.0) == 100.0


def test_shard_ranges():
    import sys

    sys.path.insert(0, ROOT)
    from paper_2604_27162_gb300 import shard as S

    assert S.env_base(3, 1024) == 3072
    spans = [S.split_range(1000, 3, r) for r in range(3)]
    assert spans[0][0] == 0 and spans[-1][1] == 1000
    assert all(spans[i][1] == spans[i + 1][0] for i in range(2))
    with pytest.raises(ValueError):
        S.split_range(10, 2, 2)
    assert S.max_over_ranks(4.5) == 4.5  # no process group: identity
