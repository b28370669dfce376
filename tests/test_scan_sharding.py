"""Sharding of a temperature scan across ranks (host side, no GPU): the betas
are split into contiguous blocks, each rank runs its block, rank 0 gathers
the results in beta order.  The multi-rank tests run world size 2 on the
gloo backend in spawned CPU processes, with a stand-in for the per-block GPU
run."""
import json
import math
import multiprocessing as mp
import os
import socket
import tempfile

import pytest

from paper_2004_08669_gb300.scan import gather_results, run_sharded, shard_range


def test_shard_range_partitions_contiguously():
    for n in range(0, 41):
        for world in range(1, 9):
            ranges = [shard_range(n, r, world) for r in range(world)]
            assert ranges[0][0] == 0 and ranges[-1][1] == n
            for (lo, hi), (lo2, _) in zip(ranges, ranges[1:]):
                assert hi == lo2
            sizes = [hi - lo for lo, hi in ranges]
            assert max(sizes) - min(sizes) <= 1
            assert sizes == sorted(sizes, reverse=True)


def test_shard_range_rejects_bad_ranks():
    with pytest.raises(ValueError):
        shard_range(4, 2, 2)
    with pytest.raises(ValueError):
        shard_range(4, 0, 0)


def test_single_rank_runs_everything():
    betas = [1.0 / t for t in (0.40, 0.44, 0.48)]
    out = run_sharded(betas, lambda blk: [{"beta": b} for b in blk])
    assert [o["beta"] for o in out] == betas
    assert gather_results([1, 2], 0, 1) == [1, 2]


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, betas, out_path, fail_rank):
    import datetime

    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world,
                            timeout=datetime.timedelta(seconds=20))

    def block(blk):
        if rank == fail_rank:
            raise RuntimeError("injected failure of this rank's block")
        return [{"beta": b, "rank": rank, "f": -0.5 / b * math.log(400.0)} for b in blk]

    try:
        res = run_sharded(betas, block, rank, world)
        status = "ok"
    except Exception as e:  # the failing rank itself, or a peer whose gather lost it
        res, status = None, f"{type(e).__name__}"
    if rank == 0:
        with open(out_path, "w") as f:
            json.dump({"status": status, "res": res}, f)
    try:
        dist.destroy_process_group()
    except Exception:
        pass


def _spawn(world, betas, fail_rank=-1, timeout=120):
    ctx = mp.get_context("spawn")
    port = _free_port()
    fd, path = tempfile.mkstemp(suffix=".json")
    os.close(fd)
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, betas, path, fail_rank)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout)
    alive = [p for p in procs if p.is_alive()]
    for p in alive:
        p.kill()
    assert not alive, "a rank did not finish"
    with open(path) as f:
        data = json.load(f)
    os.unlink(path)
    return data


def test_gloo_world2_gathers_in_beta_order():
    temps = [0.40 + 0.08 * i / 6 for i in range(7)]
    betas = [1.0 / t for t in temps]
    data = _spawn(2, betas)
    assert data["status"] == "ok"
    res = data["res"]
    assert [r["beta"] for r in res] == betas
    # rank 0 took the first, larger block (4 of 7), rank 1 the rest
    assert [r["rank"] for r in res] == [0] * 4 + [1] * 3


def test_gloo_world2_failed_rank_is_reported_not_hung():
    """A rank whose block raises never joins the gather: rank 0 gets an
    error from the collective (the peer closed its connection or the
    process-group timeout ran out) instead of waiting forever."""
    betas = [1.0 / t for t in (0.40, 0.42, 0.44, 0.46)]
    data = _spawn(2, betas, fail_rank=1)
    assert data["status"] != "ok"
    assert data["res"] is None
