"""Multi-rank host logic on CPU (gloo, world size 2): pair sharding and the
max-over-ranks timing of bench.py. Each rank aligns its own shard of tiny pairs
with the oracle; nothing crosses ranks but the timing and a final gather."""
import os
import socket

import numpy as np
import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from oracle import kf_oracle as O
    from synth import scenes as S
    cases = bench.shard(rank, world, 2)
    poses = []
    for c in cases:
        pr = S.config1_tiny(c)
        cam = O.Cam(*pr.K.as_tuple())
        r = O.align_from_depth(pr.depth, cam, pr.model_vertex, pr.model_normal, cam,
                               pr.model_pose, pr.prior_R, pr.init_pose, pr.lam,
                               O.Params(levels=1, max_iters=(5,)))
        poses.append(r.pose)
    t = bench.max_over_ranks(10.0 + rank, dist)
    gathered = [None] * world
    dist.all_gather_object(gathered, (rank, cases, [p.tolist() for p in poses]))
    if rank == 0:
        np.save(os.path.join(out_dir, "result.npy"), np.array([t], dtype=np.float64))
        import json
        with open(os.path.join(out_dir, "gathered.json"), "w") as f:
            json.dump(gathered, f)
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_pairs_and_take_the_slowest_time(tmp_path):
    mp = pytest.importorskip("torch.multiprocessing")
    port = _free_port()
    mp.spawn(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    import json
    t = float(np.load(tmp_path / "result.npy")[0])
    assert t == 11.0
    gathered = json.load(open(tmp_path / "gathered.json"))
    cases = sorted(c for _, cs, _ in gathered for c in cs)
    assert cases == [0, 1, 2, 3]
    from oracle import kf_oracle as O
    from synth import scenes as S
    # each rank's result equals a single-process alignment of the same case
    for rank, cs, poses in gathered:
        for c, P in zip(cs, poses):
            pr = S.config1_tiny(c)
            cam = O.Cam(*pr.K.as_tuple())
            r = O.align_from_depth(pr.depth, cam, pr.model_vertex, pr.model_normal, cam,
                                   pr.model_pose, pr.prior_R, pr.init_pose, pr.lam,
                                   O.Params(levels=1, max_iters=(5,)))
            assert np.array_equal(np.array(P), r.pose)


def test_shard_is_disjoint_and_covering():
    import bench
    for world in (1, 2, 4, 8):
        got = sorted(c for r in range(world) for c in bench.shard(r, world, 64))
        assert got == list(range(64 * world))


def test_mixed_batch_shards_balance_pixels_within_one_pair():
    """The 64-pair mixed-resolution batch split over N ranks: the cases sorted
    by size and dealt round-robin, so per-rank pixel loads differ by at most
    one pair's pixels (a contiguous split would give one rank the 16 largest)."""
    import bench
    pix = [bench.case_pixels("batch64", c) for c in range(64)]
    for world in (1, 2, 3, 4, 8):
        shards = [bench.shard(r, world, 64, "batch64") for r in range(world)]
        got = sorted(c for s in shards for c in s)
        assert got == list(range(64))
        loads = [sum(pix[c] for c in s) for s in shards]
        assert max(loads) - min(loads) <= max(pix), (world, loads)
        # each rank gets a share of every resolution when the ranks divide 16
        if 16 % world == 0:
            for s in shards:
                assert sorted({pix[c] for c in s}) == sorted(set(pix))


def _rank_balance(rank, world, port, out_dir):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    cases = bench.shard(rank, world, 64, "batch64")
    load = sum(bench.case_pixels("batch64", c) for c in cases)
    gathered = [None] * world
    dist.all_gather_object(gathered, (rank, cases, load))
    if rank == 0:
        import json
        with open(os.path.join(out_dir, "balance.json"), "w") as f:
            json.dump(gathered, f)
    dist.destroy_process_group()


def test_two_gloo_ranks_split_the_mixed_batch_by_pixels(tmp_path):
    mp = pytest.importorskip("torch.multiprocessing")
    port = _free_port()
    mp.spawn(_rank_balance, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    import json
    got = json.load(open(tmp_path / "balance.json"))
    assert sorted(c for _, cs, _ in got for c in cs) == list(range(64))
    loads = [ld for _, _, ld in got]
    assert abs(loads[0] - loads[1]) <= 1280 * 960
