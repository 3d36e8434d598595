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
    mine = {}
    for s in range(steps):
        idx = shard.step_indices(s, rank, world, B, P.shape[0])
        r = oracle.profile_batch(ds.coords, ds.y, ds.X, P[idx], w.lambdas, nthreads=1)
        for j, k in enumerate(idx):
            mine[int(k)] = r["logL"][j]
    gathered = [None] * world
    dist.all_gather_object(gathered, mine)
    t = torch.tensor([float(rank + 1)])
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    if rank == 0:
        merged = {}
        for g in gathered:
            for k, v in g.items():
                assert k not in merged or np.array_equal(merged[k], v)
                merged[k] = v
        out.put((merged, float(t.item())))
    dist.destroy_process_group()


def test_two_gloo_ranks_match_single_process():
    world, B, steps = 2, 4, 3
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, B, steps, q)) for r in range(world)]
    for p in procs:
        p.start()
    merged, tmax = q.get(timeout=300)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert tmax == float(world)
    assert len(merged) == world * B * steps == 24
    import oracle
    w = synth.aniso1000(K=24)
    ds = synth.aniso_dataset(9, 60, 2.5, 3)
    ref = oracle.profile_batch(ds.coords, ds.y, ds.X, w.params[0], w.lambdas, nthreads=1)
    for k, v in merged.items():
        np.testing.assert_array_equal(v, ref["logL"][k])


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
