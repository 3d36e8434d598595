"""Multi-rank path on CPU: gloo ranks shard the omega points exactly as the
benchmark does under torchrun (no data-path collective), each evaluates its
shard (with the oracle, since these ranks have no GPU), and the gathered
results equal a single-process evaluation; the max-over-ranks timing
reduction works."""
import os
import socket

import numpy as np
import torch.multiprocessing as mp

from paper_2305_04318_b300 import shard, synth


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, B, steps, out):
    import torch
    import torch.distributed as dist

    import oracle
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w = synth.aniso1000(K=24)
    ds = synth.aniso_dataset(9, 60, 2.5, 3)
    P = w.params[0]
    idx_all, res = [], []
    for s in range(steps):
        idx = shard.step_indices(s, rank, world, B, P.shape[0])
        res.append(oracle.profile_batch(ds.coords, ds.y, ds.X, P[idx], w.lambdas, nthreads=1))
        idx_all.append(idx)
    mine = {k: np.concatenate([r[k] for r in res]) for k in shard.RESULT_KEYS}
    # the product's gather (the one bench.py uses under torchrun), here over
    # gloo with the oracle as the evaluator
    merged, covered = shard.gather_results(np.concatenate(idx_all), mine, P.shape[0], len(w.lambdas), ds.p)
    t = torch.tensor([float(rank + 1)])
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    if rank == 0:
        out.put((merged, covered, float(t.item())))
    dist.destroy_process_group()


def test_two_gloo_ranks_match_single_process():
    world, B, steps = 2, 4, 3
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, B, steps, q)) for r in range(world)]
    for p in procs:
        p.start()
    merged, covered, tmax = q.get(timeout=300)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert tmax == float(world)
    assert covered == world * B * steps == 24
    import oracle
    w = synth.aniso1000(K=24)
    ds = synth.aniso_dataset(9, 60, 2.5, 3)
    ref = oracle.profile_batch(ds.coords, ds.y, ds.X, w.params[0], w.lambdas, nthreads=1)
    for k in shard.RESULT_KEYS:
        np.testing.assert_array_equal(merged[k], ref[k], err_msg=k)


def _uneven_rank_main(rank, world, port, out):
    """Uneven shards (rank 1 evaluates nothing at all) and a point evaluated
    by both ranks."""
    import torch.distributed as dist

    import oracle
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w = synth.aniso1000(K=6)
    ds = synth.aniso_dataset(10, 40, 2.0, 2)
    P, lam = w.params[0], w.lambdas[:3]
    idx = {0: np.array([0, 2, 5]), 1: np.array([], dtype=np.int64), 2: np.array([5, 1])}[rank]
    r = oracle.profile_batch(ds.coords, ds.y, ds.X, P[idx], lam, nthreads=1) if len(idx) else None
    merged, covered = shard.gather_results(idx, r, P.shape[0], len(lam), ds.p)
    if rank == 0:
        out.put((merged, covered))
    dist.destroy_process_group()


def test_gather_uneven_and_empty_shards():
    world = 3
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_uneven_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    merged, covered = q.get(timeout=300)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert covered == 4
    import oracle
    w = synth.aniso1000(K=6)
    ds = synth.aniso_dataset(10, 40, 2.0, 2)
    ref = oracle.profile_batch(ds.coords, ds.y, ds.X, w.params[0], w.lambdas[:3], nthreads=1)
    for k in (0, 1, 2, 5):
        for key in shard.RESULT_KEYS:
            np.testing.assert_array_equal(merged[key][k], ref[key][k])
    assert merged["status"][3] == -1 and np.isnan(merged["logL"][3]).all()


def test_pack_unpack_round_trip():
    rng = np.random.default_rng(1)
    B, M, p = 5, 4, 3
    r = dict(logL=rng.normal(size=(B, M)), sigma2=rng.normal(size=(B, M)), beta=rng.normal(size=(B, M, p)),
             logdet=rng.normal(size=(B, 2)), status=np.array([0, 1, 2, 3, 16 | 1], dtype=np.int32))
    u = shard.unpack_results(shard.pack_results(r), M, p)
    for k in shard.RESULT_KEYS:
        np.testing.assert_array_equal(u[k], r[k])


def test_shards_disjoint_within_a_step_and_cover_the_grid():
    K, B = 1024, 128
    for world in (1, 2, 4, 8):
        seen = set()
        for s in range(-(-K // (world * B))):
            blocks = [set(shard.step_indices(s, r, world, B, K).tolist()) for r in range(world)]
            for a in range(world):
                for b in range(a + 1, world):
                    assert not (blocks[a] & blocks[b])
            for b in blocks:
                seen |= b
        assert seen == set(range(K))


def test_balance_by_cost():
    rng = np.random.default_rng(4)
    n = np.round(np.exp(rng.uniform(np.log(200), np.log(3000), 256)))
    cost = 512 * n ** 3
    for world in (1, 2, 4, 8):
        owner = shard.balance_by_cost(cost, world)
        assert owner.min() >= 0 and owner.max() < world
        loads = np.bincount(owner, weights=cost, minlength=world)
        # greedy largest-first: no rank exceeds the ideal share by more than the largest item
        assert loads.max() <= cost.sum() / world + cost.max() + 1e-6
    # a single dominant item gets a rank of its own
    owner = shard.balance_by_cost([100.0, 1.0, 1.0, 1.0], 2)
    assert (owner == owner[0]).sum() == 1
