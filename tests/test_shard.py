"""Sharding of independent games over ranks (paper_1705_02313_gb300/shard.py),
the host logic of the multi-GPU batch: on the CPU, with world_size 2 over
gloo. Each rank packs only its share of a batch (the generator's subset
packing, as the benchmark's batch leg does), solves it with the oracle, and
the gathered results must be those of one process solving every game; the
timing reductions must give the slowest rank's time."""
import os
import socket

import numpy as np
import pytest

from paper_1705_02313_gb300 import gen, shard

COUNT, LO, HI, DMIN, DMAX = 14, 40, 600, 1, 4


def test_lpt_assign_covers_every_game_once_and_balances():
    rng = np.random.default_rng(3)
    for world in (1, 2, 3, 8):
        w = rng.integers(1, 10_000, size=97)
        parts = shard.lpt_assign(w, world)
        allidx = np.sort(np.concatenate(parts))
        assert np.array_equal(allidx, np.arange(w.size))
        loads = [int(w[p].sum()) for p in parts]
        # greedy LPT: no rank exceeds the average by more than the largest game
        assert max(loads) <= w.sum() / world + w.max()
        assert all(np.all(np.diff(p) > 0) for p in parts)
        again = shard.lpt_assign(w, world)  # every rank computes the same split
        assert all(np.array_equal(a, b) for a, b in zip(parts, again))
    assert [p.size for p in shard.lpt_assign([5, 5, 5, 5], 2)] == [2, 2]
    with pytest.raises(ValueError):
        shard.lpt_assign([1], 0)


def test_reductions_without_a_process_group():
    assert shard.max_over_ranks(2.5) == 2.5 and shard.sum_over_ranks(3) == 3.0
    assert shard.gather_to_all({"a": 1}) == [{"a": 1}]
    shard.barrier()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _solve_packed(vb, eb, off, tgt, own, pri, i):
    from oracle import o2
    a, b = int(vb[i]), int(vb[i + 1])
    e0, e1 = int(eb[i]), int(eb[i + 1])
    _, _, out = o2.solve_game(b - a, off[a + i:b + i + 1] - off[a + i], tgt[e0:e1], own[a:b], pri[a:b])
    return out["win"].tobytes(), out["sigma"].tobytes(), int(out["inner"])


def _worker(rank, world, port, outdir):
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=world)
    try:
        sizes = gen.log_uniform_sizes(COUNT, LO, HI).astype(np.int64)
        mine = shard.shard_of(sizes, world, rank)
        vb, eb, off, tgt, own, pri = gen.native_batch(COUNT, LO, HI, DMIN, DMAX, indices=mine, nthreads=1)
        results = {int(g): _solve_packed(vb, eb, off, tgt, own, pri, k) for k, g in enumerate(mine)}
        shard.barrier()
        gathered = shard.gather_to_all(results)
        t_max = shard.max_over_ranks(1.0 + rank)
        total = shard.sum_over_ranks(len(mine))
        counts = shard.gather_to_all(int(mine.size))
        if rank == 0:
            merged = {}
            for part in gathered:
                assert not set(part) & set(merged), "a game solved on two ranks"
                merged.update(part)
            # one process, every game
            vb1, eb1, off1, tgt1, own1, pri1 = gen.native_batch(COUNT, LO, HI, DMIN, DMAX, nthreads=1)
            want = {i: _solve_packed(vb1, eb1, off1, tgt1, own1, pri1, i) for i in range(COUNT)}
            ok = (sorted(merged) == list(range(COUNT)) and all(merged[i] == want[i] for i in range(COUNT))
                  and t_max == float(world) and total == COUNT and sum(counts) == COUNT and min(counts) > 0)
            with open(os.path.join(outdir, "result"), "w") as f:
                f.write("ok" if ok else "mismatch %s %s %s" % (t_max, total, counts))
    finally:
        dist.destroy_process_group()


def test_two_ranks_shard_a_batch_over_gloo(tmp_path):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    if not torch.distributed.is_available():
        pytest.skip("torch.distributed is not available")
    from oracle import o2
    o2.lib()  # the oracle library is built before the ranks start
    mp.spawn(_worker, args=(2, _free_port(), str(tmp_path)), nprocs=2, join=True)
    assert (tmp_path / "result").read_text() == "ok"


STREAM, POOL = 40, 12


def test_stream_assign_is_online_deterministic_and_balanced():
    rng = np.random.default_rng(8)
    for world in (1, 2, 3, 8):
        w = rng.integers(1, 10_000, size=120)
        owner = shard.stream_assign(w, world)
        assert owner.shape == w.shape and owner.min() >= 0 and owner.max() < world
        assert np.array_equal(owner, shard.stream_assign(w, world))
        # online: the owners of the first arrivals do not depend on later ones
        assert np.array_equal(shard.stream_assign(w[:50], world), owner[:50])
        loads = np.bincount(owner, weights=w, minlength=world)
        assert loads.max() - loads.min() <= w.max()  # greedy list scheduling bound
    assert shard.stream_assign([3, 3, 3, 3], 2).tolist() == [0, 1, 0, 1]
    with pytest.raises(ValueError):
        shard.stream_assign([1], 0)


def _stream_worker(rank, world, port, outdir):
    """One rank of a sharded request stream: it takes the arrivals
    stream_assign gives it (arrival j is game j mod POOL of a seeded pool),
    solves each as its server would (the oracle stands in for the GPU solver
    here), and the results meet on rank 0."""
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=world)
    try:
        vb, eb, off, tgt, own, pri = gen.native_batch(POOL, LO, HI, DMIN, DMAX, nthreads=1)
        sizes = np.diff(vb)
        arrival_game = np.arange(STREAM) % POOL
        owner = shard.stream_assign(sizes[arrival_game], world)
        mine = np.nonzero(owner == rank)[0]
        results = {int(j): _solve_packed(vb, eb, off, tgt, own, pri, int(arrival_game[j])) for j in mine}
        gathered = shard.gather_to_all(results)
        served = shard.sum_over_ranks(len(results))
        if rank == 0:
            merged = {}
            for part in gathered:
                assert not set(part) & set(merged), "an arrival served on two ranks"
                merged.update(part)
            want = {j: _solve_packed(vb, eb, off, tgt, own, pri, int(arrival_game[j])) for j in range(STREAM)}
            ok = sorted(merged) == list(range(STREAM)) and all(merged[j] == want[j] for j in range(STREAM)) \
                and served == STREAM and all(len(p) > 0 for p in gathered)
            with open(os.path.join(outdir, "result"), "w") as f:
                f.write("ok" if ok else "mismatch")
    finally:
        dist.destroy_process_group()


def test_two_ranks_shard_a_request_stream_over_gloo(tmp_path):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    if not torch.distributed.is_available():
        pytest.skip("torch.distributed is not available")
    from oracle import o2
    o2.lib()
    mp.spawn(_stream_worker, args=(2, _free_port(), str(tmp_path)), nprocs=2, join=True)
    assert (tmp_path / "result").read_text() == "ok"
