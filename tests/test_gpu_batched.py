"""GPU parity of the persistent batched solve (many instances, several start
vectors each, one launch) against the FP64 oracle and the single-instance
entry point."""
import numpy as np
import pytest
import torch

import datagen
import oracle
import paper_2110_12065_gb300 as M
from tests.helpers import rel_l1, to_dev, to_host

pytestmark = pytest.mark.gpu

TOL32 = 1e-5
SIZES = [1, 3, 64, 100, 257, 513, 600, 1000, 2048]


def make_batch(ctx, st, nvec, seed0=0):
    mats, items, hostA, W0s = [], [], [], []
    for k, n in enumerate(SIZES):
        A = datagen.wishart_instance(n, seed=seed0 + k)
        W0 = np.stack([datagen.start_vector(n, seed=1000 * (seed0 + k) + v) for v in range(nvec)])
        mat = M.mapi_matrix_upload(ctx, to_dev(A), st)
        w0 = to_dev(W0)
        items.append((mat, w0, torch.empty_like(w0)))
        mats.append(mat)
        hostA.append(A)
        W0s.append(W0)
    return mats, items, hostA, W0s


@pytest.mark.parametrize("st", ["f32", "bf16"])
@pytest.mark.parametrize("op", ["min1", "min2", "dot"])
@pytest.mark.parametrize("nvec", [1, 4])
def test_batched_parity(mapi_ctx, st, op, nvec):
    mats, items, hostA, W0s = make_batch(mapi_ctx, st, nvec)
    try:
        try:
            it, dl, sts = M.mapi_iterate_batched(mapi_ctx, items, op, nvec, 10)
        except M.MapiError as e:  # some vector stopped on a zero norm (min2)
            it, dl, sts = e.partial
        for k, ((mat, w0, w_out), A, W0) in enumerate(zip(items, hostA, W0s)):
            Ad = A.astype(np.float64) if st == "f32" else oracle.quant_bf16(A)
            got = to_host(w_out)
            for v in range(nvec):
                ost, want, oit, _ = oracle.mapi(op, Ad, W0[v].astype(np.float64), 10)
                assert sts[k, v] == ost and it[k, v] == oit
                assert rel_l1(got[v], want) <= TOL32
    finally:
        for m in mats:
            M.mapi_matrix_free(mapi_ctx, m)


def test_batched_equals_single_instance_solves(mapi_ctx):
    mats, items, hostA, W0s = make_batch(mapi_ctx, "f32", 4, seed0=50)
    try:
        it, dl, sts = M.mapi_iterate_batched(mapi_ctx, items, "min1", 4, 30,
                                             flags=M.FLAG_FINAL_L2)
        for k, (mat, w0, w_out) in enumerate(items):
            w1, it1, dl1 = M.mapi_iterate(mapi_ctx, mat, "min1", w0, 30, flags=M.FLAG_FINAL_L2)
            assert list(it[k]) == it1 == [30] * 4
            assert rel_l1(to_host(w_out), to_host(w1)) <= TOL32
        # stop rule: the two paths sum in different orders, so the step at
        # which delta crosses the tolerance may differ by one
        it, dl, sts = M.mapi_iterate_batched(mapi_ctx, items, "min1", 4, 300, tol_l1=1e-6)
        for k, (mat, w0, w_out) in enumerate(items):
            _, it1, _ = M.mapi_iterate(mapi_ctx, mat, "min1", w0, 300, tol_l1=1e-6)
            assert np.abs(np.asarray(it[k]) - np.asarray(it1)).max() <= 1
            assert ((dl[k] < 1e-6) | (it[k] == 300)).all()
    finally:
        for m in mats:
            M.mapi_matrix_free(mapi_ctx, m)


def test_batched_autotune_keeps_results(mapi_ctx):
    mats, items, hostA, W0s = make_batch(mapi_ctx, "f32", 4, seed0=70)
    try:
        M.mapi_iterate_batched(mapi_ctx, items, "min1", 4, 5)
        ref = [to_host(w_out).copy() for _, _, w_out in items]
        r = M.mapi_autotune_batched(mapi_ctx, items, "min1", 4, iters=2)
        assert r in (1, 2, 4, 8)
        M.mapi_iterate_batched(mapi_ctx, items, "min1", 4, 5)
        for (_, _, w_out), want in zip(items, ref):
            assert rel_l1(to_host(w_out), want) <= TOL32
    finally:
        for m in mats:
            M.mapi_matrix_free(mapi_ctx, m)


def test_batched_rejects_bad_batches(mapi_ctx):
    a = M.mapi_matrix_upload(mapi_ctx, to_dev(np.eye(8, dtype=np.float32)), "f32")
    b = M.mapi_matrix_upload(mapi_ctx, to_dev(np.eye(8, dtype=np.float32)), "bf16")
    big = M.mapi_matrix_upload(mapi_ctx, torch.zeros(2100, 2100, device="cuda"), "f32")
    w = to_dev(np.ones((4, 8), np.float32))
    wb = torch.ones(4, 2100, device="cuda")
    try:
        for items, nvec in (([(a, w, torch.empty_like(w)), (b, w, torch.empty_like(w))], 4),
                            ([(big, wb, torch.empty_like(wb))], 4),
                            ([(a, w[:3], torch.empty_like(w[:3]))], 3)):
            with pytest.raises(M.MapiError) as e:
                M.mapi_iterate_batched(mapi_ctx, items, "min1", nvec, 2)
            assert e.value.name == "EINVAL"
    finally:
        for m in (a, b, big):
            M.mapi_matrix_free(mapi_ctx, m)


def test_batched_full_size_sampled(mapi_ctx):
    """4096 Wishart instances (n log-uniform in [64, 2048]), 4 start vectors,
    one launch; a sample of instances (smallest and largest included) is
    checked against the oracle."""
    sizes = datagen.wishart_sizes(4096, seed=0)
    mats, items = [], []
    try:
        for k, n in enumerate(sizes):
            A = datagen.wishart_instance_device(int(n), seed=k)
            mats.append(M.mapi_matrix_upload(mapi_ctx, A, "f32"))
            w0 = torch.from_numpy(np.stack(
                [datagen.start_vector(int(n), seed=10 * k + v) for v in range(4)])).cuda()
            items.append((mats[-1], w0, torch.empty_like(w0)))
        it, dl, sts = M.mapi_iterate_batched(mapi_ctx, items, "min1", 4, 3)
        assert (it == 3).all() and (sts == 0).all()
        order = np.argsort(sizes)
        sample = list(order[:2]) + list(order[-2:]) + list(datagen.rng(1).integers(0, 4096, 4))
        for k in sample:
            n = int(sizes[k])
            A = datagen.wishart_instance_device(n, seed=int(k)).cpu().numpy().astype(np.float64)
            got = to_host(items[k][2])
            W0 = to_host(items[k][1])
            for v in range(4):
                _, want, _, _ = oracle.mapi("min1", A, W0[v], 3)
                assert rel_l1(got[v], want) <= TOL32
    finally:
        for m in mats:
            M.mapi_matrix_free(mapi_ctx, m)


@pytest.mark.parametrize("st", ["f32", "bf16"])
@pytest.mark.parametrize("nvec", [1, 4])
@pytest.mark.parametrize("rows", [1, 2, 4, 8])
def test_batched_every_rows_per_warp_variant(mapi_ctx, st, nvec, rows):
    # each kernel variant the autotuner may pick (eight BF16 rows per warp
    # read half chunks), forced through mapi_set_batched_rows, against the
    # FP64 oracle on large (cluster) and small (one CTA) instances
    mats, items, hostA, W0s = make_batch(mapi_ctx, st, nvec, seed0=40)
    try:
        M.mapi_set_batched_rows(mapi_ctx, st, nvec, rows)
        it, dl, sts = M.mapi_iterate_batched(mapi_ctx, items, "min1", nvec, 10)
        for k, ((mat, w0, w_out), A, W0) in enumerate(zip(items, hostA, W0s)):
            Ad = A.astype(np.float64) if st == "f32" else oracle.quant_bf16(A)
            got = to_host(w_out)
            for v in range(nvec):
                ost, want, oit, _ = oracle.mapi("min1", Ad, W0[v].astype(np.float64), 10)
                assert sts[k, v] == ost and it[k, v] == oit
                assert rel_l1(got[v], want) <= TOL32, (st, nvec, rows, SIZES[k], v)
    finally:
        M.mapi_set_batched_rows(mapi_ctx, st, nvec, 2)
        for m in mats:
            M.mapi_matrix_free(mapi_ctx, m)


def test_set_batched_rows_rejects_other_values(mapi_ctx):
    for bad in (0, 3, 16):
        with pytest.raises(M.MapiError):
            M.mapi_set_batched_rows(mapi_ctx, "f32", 4, bad)
    with pytest.raises(M.MapiError):
        M.mapi_set_batched_rows(mapi_ctx, "fp8", 4, 2)
