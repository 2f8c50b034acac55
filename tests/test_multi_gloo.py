"""The N > 1 path on CPU: two gloo ranks shard a batch by pixel count,
each extracts its own images (here with the CPU oracle, standing in for the
per-rank GPU run), and the merged per-image histograms equal a single-process
run over the whole batch; the job time is the max over ranks."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _batch():
    import synth

    sizes = [synth.sizes(4000 + i, 3, 90) for i in range(23)]
    imgs = [synth.image(4000 + i, h, w, 3.0) for i, (h, w) in enumerate(sizes)]
    return imgs


def _worker(rank, world, port, out_dir):
    import sys

    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    from paper_1810_11518_gb300 import multi

    imgs = _batch()
    shards = multi.shard_images([a.size for a in imgs], world)
    mine = shards[rank]
    hists = np.stack([oracle.extract(imgs[i], k=3, R=3, C=2, want_codes=False)[0].reshape(-1) for i in mine])
    # gather (index, hist) from every rank on the host
    obj = [None] * world
    dist.all_gather_object(obj, (mine.tolist(), hists))
    t = multi.max_over_ranks(float(rank + 1), dist)
    if rank == 0:
        np.savez(os.path.join(out_dir, "merged.npz"),
                 idx=np.concatenate([np.array(o[0]) for o in obj]),
                 hist=np.concatenate([o[1] for o in obj]), tmax=t)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_shards_merge_to_whole(tmp_path):
    import oracle
    from paper_1810_11518_gb300 import multi

    world = 2
    mp.start_processes(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, start_method="spawn")
    z = np.load(tmp_path / "merged.npz")
    imgs = _batch()
    order = np.argsort(z["idx"])
    assert sorted(z["idx"].tolist()) == list(range(len(imgs)))
    whole = np.stack([oracle.extract(a, k=3, R=3, C=2, want_codes=False)[0].reshape(-1) for a in imgs])
    assert np.array_equal(z["hist"][order], whole)
    assert float(z["tmax"]) == 2.0
    # balance: no rank carries more than the average plus one image
    shards = multi.shard_images([a.size for a in imgs], world)
    loads = [sum(imgs[i].size for i in s) for s in shards]
    assert max(loads) - sum(loads) / world <= max(a.size for a in imgs)


def test_shard_images_properties():
    from paper_1810_11518_gb300 import multi

    rng = np.random.default_rng(0)
    px = rng.integers(1, 1000, size=101)
    for world in (1, 2, 3, 8):
        shards = multi.shard_images(px, world)
        allidx = np.concatenate(shards)
        assert sorted(allidx.tolist()) == list(range(101))
        loads = [int(px[s].sum()) for s in shards]
        assert max(loads) - px.sum() / world <= px.max()
    assert (multi.rank_seeds(1, 4) == np.array([4, 5, 6, 7], dtype=np.uint64)).all()
