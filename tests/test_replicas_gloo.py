"""The multi-rank host path on CPU: two gloo ranks run the replica helpers that the
benchmark uses under torchrun (barrier, maximum over ranks of the measured times,
per-rank seeds, batch sharding).  The tiled QR itself runs one problem per GPU, so
no data path crosses ranks; these are the only collective operations."""
import json
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    from paper_1303_3182_gb300 import replicas
    import synthetic
    r, local, w = replicas.env_ranks()
    replicas.init("gloo")
    replicas.barrier()
    # each rank measured its own times; the job's time is the slowest rank's
    mx = replicas.max_over_ranks([1.0 + r, 10.0 - r, 3.5])
    seed = replicas.replica_seed(synthetic.SEED_BASE + 3, r)
    part = replicas.shard(2048, r, w)
    shapes = synthetic.ragged_batch_shapes(2048, seed=synthetic.SEED_BASE + 4)
    mine = [shapes[b] for b in part]
    replicas.barrier()
    replicas.finalize()
    with open(os.path.join(out_dir, f"rank{r}.json"), "w") as f:
        json.dump({"rank": r, "local": local, "world": w, "max": mx, "seed": seed, "part": part,
                   "work": sum(m * n * n for m, n in mine)}, f)


def test_two_gloo_ranks(tmp_path):
    world = 2
    mp.start_processes(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, start_method="spawn")
    res = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(world)]
    for r, x in enumerate(res):
        assert x["rank"] == r and x["world"] == world and x["local"] == r
        assert x["max"] == [2.0, 10.0, 3.5]
    # independent replicas: distinct seeds, rank 0 keeps the single-GPU seed
    assert res[0]["seed"] != res[1]["seed"]
    import synthetic
    assert res[0]["seed"] == synthetic.SEED_BASE + 3
    # the batch split covers every matrix once and balances the work within 10 %
    parts = [set(x["part"]) for x in res]
    assert parts[0].isdisjoint(parts[1]) and parts[0] | parts[1] == set(range(2048))
    w0, w1 = res[0]["work"], res[1]["work"]
    assert abs(w0 - w1) / max(w0, w1) < 0.1


def test_single_process_helpers_are_identities(monkeypatch):
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    from paper_1303_3182_gb300 import replicas
    assert replicas.env_ranks() == (0, 0, 1)
    replicas.init("gloo")  # no process group for one rank
    assert not dist.is_initialized()
    assert replicas.max_over_ranks([1.5, 2.5]) == [1.5, 2.5]
    assert replicas.shard(5, 0, 1) == [0, 1, 2, 3, 4]
