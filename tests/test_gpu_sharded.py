"""The partitioned forms of the path run by the library on two gloo ranks.

Each rank is a process with its own library context on cuda:0.  It holds
one shard of the data and computes its piece through the C ABI: a block of
rows of A (+) w (mapi_rows_product) for row-partitioned Alg. 1, or the pair
product of its columns of X (mapi_pair_partial) for column-partitioned PCA.
The ranks combine the pieces over gloo (an all-gather of row blocks, an
all-reduce of the partial y) and normalise the whole vector (Eq. (6)).  The
result must equal the unsharded GPU solve and the FP64 oracle within the
FP32 bar.  The ranks take turns on the GPU (one launches while the other
waits at a barrier), so no kernel of one rank waits on another's."""
import multiprocessing as mp
import os
import socket

import numpy as np
import pytest

import datagen
import oracle
from tests.helpers import rel_l1

pytestmark = pytest.mark.gpu

WORLD = 2
TOL32 = 1e-5


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _split(n, world, rank):
    per = (n + world - 1) // world
    b = min(n, rank * per)
    return b, min(n, b + per)


def _rank_main(rank, world, port, q):
    import torch
    import torch.distributed as dist

    import paper_2110_12065_gb300 as M
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    torch.cuda.set_device(0)
    ctx = M.mapi_create(0)
    out = {}

    def turn(fn):
        """Run fn on the GPU in rank order; returns this rank's result."""
        res = None
        for r in range(world):
            if r == rank:
                res = fn()
                torch.cuda.synchronize()
            dist.barrier()
        return res

    try:
        # row-partitioned Alg. 1 (min1), n = 1001, 12 steps
        n, T = 1001, 12
        A = datagen.symmetric_gaussian(n, seed=5).astype(np.float32)
        b, e = _split(n, world, rank)
        mat = turn(lambda: M.mapi_matrix_upload(ctx, torch.from_numpy(A[b:e]).cuda(), "f32"))
        w = datagen.start_vector(n, seed=6).astype(np.float64)
        w = (w / np.linalg.norm(w)).astype(np.float32)
        per = (n + world - 1) // world
        for _ in range(T):
            wd = torch.from_numpy(w).cuda()
            yl = turn(lambda: M.mapi_rows_product(ctx, mat, 0, e - b, "min1", wd).cpu())
            buf = torch.zeros(per, dtype=torch.float32)
            buf[: e - b] = yl
            parts = [torch.zeros(per, dtype=torch.float32) for _ in range(world)]
            dist.all_gather(parts, buf)
            y = torch.cat(parts)[:n].numpy().astype(np.float64)
            w = (y / np.abs(y).sum()).astype(np.float32)
        out["rows"] = w
        turn(lambda: M.mapi_matrix_free(ctx, mat))

        # column-partitioned pair mode (min1 and dot), D = 300, N = 4099
        D, N = 300, 4099
        X = datagen.spiked_pca_data(D, N, seed=7)
        b, e = _split(N, world, rank)
        Xs = turn(lambda: M.mapi_matrix_upload(ctx, torch.from_numpy(
            np.ascontiguousarray(X[:, b:e])).cuda(), "f32"))
        for op, steps in (("min1", 6), ("dot", 4)):
            w = datagen.start_vector(D, seed=8).astype(np.float64)
            w = (w / np.linalg.norm(w)).astype(np.float32)
            first = None
            for s in range(steps):
                wd = torch.from_numpy(w).cuda()
                yp = turn(lambda: M.mapi_pair_partial(ctx, Xs, op, wd).cpu())
                dist.all_reduce(yp)
                y = yp.numpy().astype(np.float64) / N
                if s == 0:
                    first = y.copy()
                L = np.linalg.norm(y) if op == "dot" else np.abs(y).sum()
                w = (y / L).astype(np.float32)
            out[f"pair_{op}_step1"] = first
            out[f"pair_{op}"] = w
        turn(lambda: M.mapi_matrix_free(ctx, Xs))
        if rank == 0:
            q.put(out)
    finally:
        M.mapi_destroy(ctx)
        dist.destroy_process_group()


@pytest.fixture(scope="module")
def sharded():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, WORLD, port, q)) for r in range(WORLD)]
    for p in procs:
        p.start()
    out = q.get(timeout=600)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    return out


def test_row_sharded_mapi_matches_unsharded_gpu_and_oracle(mapi_ctx, sharded):
    import torch

    import paper_2110_12065_gb300 as M
    n, T = 1001, 12
    A = datagen.symmetric_gaussian(n, seed=5).astype(np.float32)
    w0 = datagen.start_vector(n, seed=6)
    st, want, _, _ = oracle.mapi("min1", A, w0.astype(np.float64), T)
    assert st == oracle.OK
    mat = M.mapi_matrix_upload(mapi_ctx, torch.from_numpy(A).cuda(), "f32")
    try:
        w, _, _ = M.mapi_iterate(mapi_ctx, mat, "min1", torch.from_numpy(w0).cuda(), T)
    finally:
        M.mapi_matrix_free(mapi_ctx, mat)
    assert rel_l1(sharded["rows"], want) <= TOL32
    assert rel_l1(sharded["rows"], w.cpu().numpy()) <= TOL32


@pytest.mark.parametrize("op,steps", [("min1", 6), ("dot", 4)])
def test_column_sharded_pair_mode_matches_unsharded_gpu_and_oracle(mapi_ctx, sharded, op,
                                                                    steps):
    import torch

    import paper_2110_12065_gb300 as M
    D, N = 300, 4099
    X = datagen.spiked_pca_data(D, N, seed=7)
    w0 = datagen.start_vector(D, seed=8).astype(np.float64)
    w0 = w0 / np.linalg.norm(w0)
    # one step: the all-reduced partials are the pair product over all of X
    y1 = oracle.pair_step(op, X, w0, float(N))
    assert rel_l1(sharded[f"pair_{op}_step1"], y1) <= TOL32
    mat = M.mapi_matrix_upload(mapi_ctx, torch.from_numpy(X).cuda(), "f32")
    try:
        yg = M.mapi_pair_partial(mapi_ctx, mat, op,
                                 torch.from_numpy(w0.astype(np.float32)).cuda())
        assert rel_l1(sharded[f"pair_{op}_step1"], yg.cpu().numpy() / N) <= TOL32
        # the whole component (no deflation: the first one) against pca_topk
        P, its = M.mapi_pca_topk(mapi_ctx, mat, 1, "pair", op, steps, float(N),
                                 torch.from_numpy(w0[None, :].astype(np.float32)).cuda())
    finally:
        M.mapi_matrix_free(mapi_ctx, mat)
    st, Po, _ = oracle.pca_topk("pair", op, X.astype(np.float64), 1, steps, float(N),
                                w0[:, None])
    got = sharded[f"pair_{op}"].astype(np.float64)
    got = got / np.linalg.norm(got)
    assert rel_l1(got, Po[:, 0]) <= TOL32
    assert rel_l1(got, P.cpu().numpy()[0]) <= TOL32
