"""The partitioned forms of the path on two gloo ranks (CPU): row-sharded
Alg. 1, column-sharded pair step, tiled min-covariance, instance-sharded
batches and sample-sharded Alg. 3 must reproduce the unsharded FP64 oracle;
the benchmark's max-over-ranks timing reduction runs on the same ranks."""
import multiprocessing as mp
import os
import socket

import numpy as np
import pytest

import datagen
import oracle

WORLD = 2


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    import torch.distributed as dist

    from tests import multirank
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        out = multirank.run_all(rank, world)
        q.put((rank, out))
    finally:
        dist.destroy_process_group()


@pytest.fixture(scope="module")
def ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, WORLD, port, q)) for r in range(WORLD)]
    for p in procs:
        p.start()
    res = {}
    for _ in range(WORLD):
        r, out = q.get(timeout=180)
        res[r] = out
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    return res


@pytest.mark.parametrize("op", ["min1", "dot"])
def test_row_sharded_iteration_equals_unsharded(ranks, op):
    A = datagen.symmetric_gaussian(37, seed=3 if op == "min1" else 4)
    w0 = datagen.start_vector(37, seed=(3 if op == "min1" else 4) + 1).astype(np.float64)
    st, want, it, _ = oracle.mapi(op, A, w0, 12)
    for r in range(WORLD):
        got = ranks[r][f"row_{op}"]
        np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-15)


@pytest.mark.parametrize("op,seed", [("min1", 5), ("min2", 6)])
def test_column_sharded_pair_step_sums_to_unsharded(ranks, op, seed):
    X = datagen.spiked_pca_data(12, 101, seed=seed).astype(np.float64)
    w = datagen.start_vector(12, seed=seed + 2).astype(np.float64)
    want = oracle.pair_step(op, X, w, 101.0)
    for r in range(WORLD):
        np.testing.assert_allclose(ranks[r][f"pair_{op}"], want, rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("op,seed", [("min1", 7), ("min2", 8)])
def test_tiled_mincov_equals_unsharded(ranks, op, seed):
    X = datagen.spiked_pca_data(14, 90, seed=seed).astype(np.float64)
    want = oracle.mincov(op, X, 90.0)
    np.testing.assert_allclose(ranks[0][f"mincov_{op}"], want, rtol=1e-13, atol=1e-15)


def test_instance_sharded_batch_equals_unsharded(ranks):
    sizes = datagen.wishart_sizes(7, seed=9, nmin=4, nmax=40)
    for i, got in enumerate(ranks[0]["batch_min1"]):
        A = datagen.wishart_instance(int(sizes[i]), seed=9 + i).astype(np.float64)
        w0 = datagen.start_vector(int(sizes[i]), seed=9 + 100 + i).astype(np.float64)
        np.testing.assert_array_equal(got, oracle.mapi("min1", A, w0, 15)[1])


@pytest.mark.parametrize("op,seed", [("min1", 11), ("dot", 12)])
def test_sample_sharded_minibatch_equals_unsharded(ranks, op, seed):
    """Alg. 3 with every step's 13 draws split 7 / 6 over the ranks."""
    X = datagen.stochastic_pca_data(500, 6, seed=seed).astype(np.float64)
    batch = datagen.minibatches(500, 8, 13, seed=seed + 1)
    w0 = datagen.start_vector(6, seed=seed + 2).astype(np.float64)
    st, want = oracle.minibatch_momentum(op, X, batch, 0.2, w0)
    assert st == oracle.OK
    for r in range(WORLD):
        np.testing.assert_allclose(ranks[r][f"mb_{op}"], want, rtol=1e-11, atol=1e-13)


def test_max_over_ranks(ranks):
    assert ranks[0]["tmax"] == ranks[1]["tmax"] == 10.0 + WORLD - 1
