"""Partition of work across ranks (one process per GPU).

Every omega point is independent, so ranks need no exchange:
- one dataset: at step s rank r evaluates the B consecutive points starting
  at ((s * world + r) * B) mod K of the K-point grid (cycling through it);
  within a step the ranks' blocks are disjoint, and over ceil(K / (world B))
  steps every point is covered;
- datasets of uneven size: whole datasets go to ranks, balanced by their cost
  (points x n^3, the factorisation's share): largest first, each to the rank
  with the least cost so far.
"""
import numpy as np


def step_indices(step, rank, world, B, K):
    start = ((step * world + rank) * B) % K
    return (np.arange(B) + start) % K


def balance_by_cost(costs, world):
    """Rank of every item: greedy largest-first assignment of the items to the
    rank with the smallest total cost so far (ties to the lower rank)."""
    costs = np.asarray(costs, dtype=float)
    load = np.zeros(world)
    owner = np.empty(len(costs), dtype=np.int64)
    for i in np.argsort(-costs, kind="stable"):
        r = int(np.argmin(load))
        owner[i] = r
        load[r] += costs[i]
    return owner


RESULT_KEYS = ("logL", "sigma2", "beta", "logdet", "status")


def pack_results(r):
    """Per-point results (logL [B,M], sigma2 [B,M], beta [B,M,p], logdet
    [B,2], status [B]) as one float64 array [B, F], F = 2M + Mp + 3 (the
    int32 status is exact in float64)."""
    B = r["status"].shape[0]
    cols = [np.asarray(r[k], dtype=np.float64).reshape(B, -1) for k in RESULT_KEYS]
    return np.ascontiguousarray(np.concatenate(cols, axis=1))


def unpack_results(a, M, p):
    B = a.shape[0]
    o, out = 0, {}
    for k, width, shape in (("logL", M, (B, M)), ("sigma2", M, (B, M)), ("beta", M * p, (B, M, p)),
                            ("logdet", 2, (B, 2)), ("status", 1, (B,))):
        out[k] = a[:, o:o + width].reshape(shape)
        o += width
    out["status"] = out["status"].astype(np.int32)
    return out


def gather_results(idx, results, K, M, p, device="cpu", strict=True):
    """Merge every rank's per-point results into arrays over all K points.

    idx: the global point indices this rank evaluated ([B_r], any B_r >= 0);
    results: their per-point results (RESULT_KEYS, numpy).  Two collectives
    on the default process group: an all_gather of the counts, then one
    all_gather of the packed results padded to the largest count (tensors on
    `device`: "cuda" under NCCL, "cpu" under gloo).  Every rank returns the
    merged dict (K rows; points no rank evaluated hold NaN and status -1) and
    the number of points evaluated by any rank.  A point evaluated twice must
    have identical results both times (every point's arithmetic depends only
    on its own data): strict raises otherwise; without strict the first
    result is kept and the count of such points is returned as a third value."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size()
    idx = np.asarray(idx, dtype=np.int64)
    packed = pack_results(results) if len(idx) else np.zeros((0, 2 * M + M * p + 3))
    F = 2 * M + M * p + 3
    cnt = torch.tensor([len(idx)], dtype=torch.int64, device=device)
    counts = [torch.zeros_like(cnt) for _ in range(world)]
    dist.all_gather(counts, cnt)
    counts = [int(c.item()) for c in counts]
    Bmax = max(counts)
    buf = np.full((Bmax, F + 1), np.nan)
    buf[:len(idx), 0] = idx
    buf[:len(idx), 1:] = packed
    t = torch.as_tensor(buf, device=device)
    parts = [torch.empty_like(t) for _ in range(world)]
    dist.all_gather(parts, t)
    merged = np.full((K, F), np.nan)
    merged[:, -1] = -1
    seen = np.zeros(K, dtype=bool)
    mismatches = 0
    for c, part in zip(counts, parts):
        a = part.cpu().numpy()[:c]
        ks = a[:, 0].astype(np.int64)
        for j, k in enumerate(ks):
            if seen[k]:
                if not np.array_equal(merged[k], a[j, 1:], equal_nan=True):
                    if strict:
                        raise RuntimeError(f"point {k}: different results in two evaluations")
                    mismatches += 1
                continue
            merged[k] = a[j, 1:]
            seen[k] = True
    out = unpack_results(merged, M, p)
    return (out, int(seen.sum())) if strict else (out, int(seen.sum()), mismatches)
