"""Rank programs for the partitioned-algorithm tests: each runs on one gloo
rank (CPU), computes its shard with the FP64 oracle and exchanges what the
partition needs (an all-gather of y for row shards, an all-reduce of y for
column shards, a gather of C tiles, an all-reduce of A_t for Alg. 3's
sample shards).  Rank 0 returns the assembled results.
"""
import numpy as np
import torch
import torch.distributed as dist

import datagen
import oracle


def _split(n, world, rank):
    """Contiguous block [b, e) of rank out of n items (ragged last block)."""
    per = (n + world - 1) // world
    b = min(n, rank * per)
    return b, min(n, b + per)


def _all_gather_rows(y_local, n, world):
    """All-gather of row blocks of different lengths (padded to the largest)."""
    per = (n + world - 1) // world
    buf = torch.zeros(per, dtype=torch.float64)
    buf[: y_local.size] = torch.from_numpy(y_local)
    parts = [torch.zeros(per, dtype=torch.float64) for _ in range(world)]
    dist.all_gather(parts, buf)
    y = np.concatenate([p.numpy() for p in parts])
    return y[:n]


def row_sharded_mapi(rank, world, op, n, iters, seed):
    """Alg. 1 with A row-partitioned: each rank forms its rows of A (+) w,
    an all-gather assembles y, every rank normalises by the same norm."""
    A = datagen.symmetric_gaussian(n, seed=seed)
    w = datagen.start_vector(n, seed=seed + 1).astype(np.float64)
    w = w / np.sqrt(np.sum(w * w))  # Alg. 1 step 1
    b, e = _split(n, world, rank)
    for _ in range(iters):
        y = _all_gather_rows(oracle.matvec(op, A[b:e], w), n, world)
        L = np.sqrt(np.sum(y * y)) if op == "dot" else np.sum(np.abs(y))
        w = y / L
    return w


def column_sharded_pair_step(rank, world, op, D, N, seed):
    """One pair step with X column-partitioned: each rank applies the step
    to its samples; an all-reduce sums the partial y."""
    X = datagen.spiked_pca_data(D, N, seed=seed).astype(np.float64)
    w = datagen.start_vector(D, seed=seed + 2).astype(np.float64)
    b, e = _split(N, world, rank)
    # the oracle's step divides by denom; use 1 and divide after the sum
    part = oracle.pair_step(op, X[:, b:e], w, 1.0) if e > b else np.zeros(D)
    t = torch.from_numpy(part.copy())
    dist.all_reduce(t)
    return t.numpy() / N


def tiled_mincov(rank, world, op, D, N, seed):
    """Eq. (5) by 2-D tiles of C: tile (I, J) goes to rank (I + J) % world;
    C_IJ[:, j] = X_I (+) x_j / N.  Rank 0 gathers the tiles."""
    X = datagen.spiked_pca_data(D, N, seed=seed).astype(np.float64)
    tiles = 3
    C = np.zeros((D, D))
    for I in range(tiles):
        for J in range(tiles):
            if (I + J) % world != rank:
                continue
            ib, ie = _split(D, tiles, I)
            jb, je = _split(D, tiles, J)
            for j in range(jb, je):
                C[ib:ie, j] = oracle.matvec(op, X[ib:ie], X[j]) / N
    t = torch.from_numpy(C)
    dist.all_reduce(t)  # tiles are disjoint: the sum assembles C
    return t.numpy()


def instance_sharded_batch(rank, world, op, count, iters, seed):
    """Independent instances (batched / served units) dealt round-robin to
    ranks; each solves its own; rank 0 collects every result."""
    sizes = datagen.wishart_sizes(count, seed=seed, nmin=4, nmax=40)
    mine = {}
    for i in range(rank, count, world):
        A = datagen.wishart_instance(int(sizes[i]), seed=seed + i).astype(np.float64)
        w0 = datagen.start_vector(int(sizes[i]), seed=seed + 100 + i).astype(np.float64)
        mine[i] = oracle.mapi(op, A, w0, iters)[1]
    out = [None] * world
    dist.all_gather_object(out, mine)
    merged = {}
    for d in out:
        merged.update(d)
    return [merged[i] for i in range(count)]


def sample_sharded_minibatch(rank, world, op, N, D, T, s, beta, seed):
    """Alg. 3 with each step's draws split over the ranks: every rank adds
    the outer products x (+) x^T of its share, an all-reduce sums A_t, and
    the rest of the step (v = A_t (+) w_t - beta w_{t-1}, both scaled by the
    norm of v) runs alike on every rank."""
    X = datagen.stochastic_pca_data(N, D, seed=seed).astype(np.float64)
    batch = datagen.minibatches(N, T, s, seed=seed + 1)
    w = datagen.start_vector(D, seed=seed + 2).astype(np.float64)
    w = w / np.sqrt(np.sum(w * w))  # step 1
    wp = np.zeros(D)
    b, e = _split(s, world, rank)
    for t in range(T):
        idx = batch[t, b:e]
        part = oracle.mincov(op, X[idx].T, 1.0) if e > b else np.zeros((D, D))
        At = torch.from_numpy(np.ascontiguousarray(part))
        dist.all_reduce(At)
        A = At.numpy() / s
        v = oracle.matvec(op, A, w) - beta * wp
        L = np.sqrt(np.sum(v * v)) if op == "dot" else np.sum(np.abs(v))
        wp, w = w / L, v / L
    return w / np.sqrt(np.sum(w * w))


def max_over_ranks_case(rank, world):
    """The benchmark's timing reduction on gloo: every rank reports its own
    time, all get the maximum."""
    import bench
    t = bench.max_over_ranks(10.0 + rank, dist, "cpu")
    return t


def run_all(rank, world):
    return {
        "row_min1": row_sharded_mapi(rank, world, "min1", 37, 12, 3),
        "row_dot": row_sharded_mapi(rank, world, "dot", 37, 12, 4),
        "pair_min1": column_sharded_pair_step(rank, world, "min1", 12, 101, 5),
        "pair_min2": column_sharded_pair_step(rank, world, "min2", 12, 101, 6),
        "mincov_min1": tiled_mincov(rank, world, "min1", 14, 90, 7),
        "mincov_min2": tiled_mincov(rank, world, "min2", 14, 90, 8),
        "batch_min1": instance_sharded_batch(rank, world, "min1", 7, 15, 9),
        "mb_min1": sample_sharded_minibatch(rank, world, "min1", 500, 6, 8, 13, 0.2, 11),
        "mb_dot": sample_sharded_minibatch(rank, world, "dot", 500, 6, 8, 13, 0.2, 12),
        "tmax": max_over_ranks_case(rank, world),
    }
