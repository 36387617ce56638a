"""GPU parity of the PCA path through the C ABI: the min-covariance build
(Eq. (5)), deflation (Alg. 2 step 6, sum form), the matrix-free pair step and
the top-k drivers, against the FP64 oracle."""
import numpy as np
import pytest
import torch

import datagen
import oracle
import paper_2110_12065_gb300 as M
from tests.helpers import rel_l1, to_dev, to_host

pytestmark = pytest.mark.gpu

TOL32 = 1e-5


def spiked(D, N, seed):
    return datagen.spiked_pca_data(D, N, seed=seed)


@pytest.mark.parametrize("op", ["min1", "min2", "dot"])
@pytest.mark.parametrize("D,N", [(1, 7), (130, 1000), (300, 777)])
@pytest.mark.parametrize("st", ["f32", "bf16"])
def test_mincov_parity(mapi_ctx, op, D, N, st):
    X = spiked(D, N, seed=D + N)
    mat = M.mapi_matrix_upload(mapi_ctx, to_dev(X), st)
    try:
        Cg = to_host(M.mapi_mincov(mapi_ctx, mat, op, float(N)))
        torch.cuda.synchronize()
        Xs = X.astype(np.float64) if st == "f32" else oracle.quant_bf16(X)
        Co = oracle.mincov(op, Xs, float(N))
        assert rel_l1(Cg, Co) <= TOL32
        np.testing.assert_array_equal(Cg, Cg.T)
    finally:
        M.mapi_matrix_free(mapi_ctx, mat)


@pytest.mark.parametrize("mode", ["mincov", "pair"])
@pytest.mark.parametrize("op", ["min1", "min2", "dot"])
def test_pca_topk_parity(mapi_ctx, mode, op):
    D, N, k, T = 96, 1500, 3, 40
    X = spiked(D, N, seed=21)
    W0 = np.stack([datagen.start_vector(D, seed=200 + c) for c in range(k)])
    mat = M.mapi_matrix_upload(mapi_ctx, to_dev(X), "f32")
    try:
        st, Po, oits = oracle.pca_topk(mode, op, X.astype(np.float64), k, T, float(N), W0.T)
        try:
            P, its = M.mapi_pca_topk(mapi_ctx, mat, k, mode, op, T, float(N), to_dev(W0))
            gst = 0
        except M.MapiError as e:
            (P, its), gst = e.partial, e.status
        # the method itself may stop on a zero norm (min2 after deflation):
        # both sides must stop at the same component and step
        assert gst == st and its == list(oits)
        P = to_host(P)
        # components finished before a stop are compared
        first_stop = next((c for c in range(k) if oits[c] < T), k) if st else k
        for c in range(first_stop):
            err = rel_l1(P[c], Po[:, c])
            assert err <= TOL32, (c, err)
            assert abs(np.linalg.norm(P[c]) - 1) < 1e-5
    finally:
        M.mapi_matrix_free(mapi_ctx, mat)


@pytest.mark.parametrize("D", [200, 256, 1000])
def test_pair_mode_ragged_shapes(mapi_ctx, D):
    N = 2051  # several column tiles plus a ragged tail
    X = spiked(D, N, seed=D)
    W0 = np.stack([datagen.start_vector(D, seed=300 + c) for c in range(2)])
    mat = M.mapi_matrix_upload(mapi_ctx, to_dev(X), "f32")
    try:
        P, _ = M.mapi_pca_topk(mapi_ctx, mat, 2, "pair", "min1", 5, float(N), to_dev(W0))
        _, Po, _ = oracle.pca_topk("pair", "min1", X.astype(np.float64), 2, 5, float(N), W0.T)
        for c in range(2):
            assert rel_l1(to_host(P)[c], Po[:, c]) <= TOL32
    finally:
        M.mapi_matrix_free(mapi_ctx, mat)


@pytest.mark.parametrize("st", ["f32", "bf16"])
def test_pair_mode_many_tiles_per_cluster(mapi_ctx, st):
    """N = 32768: every cluster streams a dozen or more column tiles, so the
    tile pipeline and the cluster exchange slots wrap around many times."""
    D, N, k, T = 256, 32768, 2, 6
    X = spiked(D, N, seed=41)
    W0 = np.stack([datagen.start_vector(D, seed=410 + c) for c in range(k)])
    mat = M.mapi_matrix_upload(mapi_ctx, to_dev(X), st)
    try:
        P, _ = M.mapi_pca_topk(mapi_ctx, mat, k, "pair", "min1", T, float(N), to_dev(W0))
        Xs = X.astype(np.float64) if st == "f32" else oracle.quant_bf16(X)
        _, Po, _ = oracle.pca_topk("pair", "min1", Xs, k, T, float(N), W0.T)
        for c in range(k):
            assert rel_l1(to_host(P)[c], Po[:, c]) <= TOL32
    finally:
        M.mapi_matrix_free(mapi_ctx, mat)


def test_pair_mode_bf16(mapi_ctx):
    D, N = 256, 4096
    X = spiked(D, N, seed=31)
    W0 = np.stack([datagen.start_vector(D, seed=310 + c) for c in range(2)])
    mat = M.mapi_matrix_upload(mapi_ctx, to_dev(X), "bf16")
    try:
        P, _ = M.mapi_pca_topk(mapi_ctx, mat, 2, "pair", "min1", 10, float(N), to_dev(W0))
        P = to_host(P)
        _, Pd, _ = oracle.pca_topk("pair", "min1", oracle.quant_bf16(X), 2, 10, float(N), W0.T)
        _, Po, _ = oracle.pca_topk("pair", "min1", X.astype(np.float64), 2, 10, float(N), W0.T)
        for c in range(2):
            assert rel_l1(P[c], Pd[:, c]) <= TOL32
            assert rel_l1(P[c], Po[:, c]) <= 2e-2
    finally:
        M.mapi_matrix_free(mapi_ctx, mat)


def test_pair_step_full_size(mapi_ctx):
    """D = 1024, N = 65536 (the PCA workload): one pair step of component 1
    from the GPU's own start against the oracle's full pair step."""
    D, N = 1024, 65536
    X = spiked(D, N, seed=0)
    w0 = datagen.start_vector(D, seed=1)
    mat = M.mapi_matrix_upload(mapi_ctx, to_dev(X), "f32")
    try:
        P, _ = M.mapi_pca_topk(mapi_ctx, mat, 1, "pair", "min1", 1, float(N),
                               to_dev(w0[None, :]))
        y = oracle.pair_step("min1", X, w0 / np.linalg.norm(w0.astype(np.float64)), float(N))
        assert rel_l1(to_host(P)[0], y / np.linalg.norm(y)) <= TOL32
    finally:
        M.mapi_matrix_free(mapi_ctx, mat)


def _pair_topk_parity(ctx, X, Xs, k, op, T, W0, st="f32"):
    """Pair-mode top-k on the GPU against the oracle on the stored values Xs:
    the same status, the same steps per component, and every component
    finished before a stop within TOL32."""
    D, N = X.shape
    mat = M.mapi_matrix_upload(ctx, to_dev(X), st)
    try:
        ost, Po, oits = oracle.pca_topk("pair", op, Xs, k, T, float(N), W0.T)
        try:
            P, its = M.mapi_pca_topk(ctx, mat, k, "pair", op, T, float(N), to_dev(W0))
            gst = 0
        except M.MapiError as e:
            (P, its), gst = e.partial, e.status
        assert gst == ost and its == list(oits), (gst, ost, its, list(oits))
        P = to_host(P)
        first_stop = next((c for c in range(k) if oits[c] < T), k) if ost else k
        errs = [rel_l1(P[c], Po[:, c]) for c in range(first_stop)]
        for c, err in enumerate(errs):
            assert err <= TOL32, (c, err, errs)
        return first_stop, errs
    finally:
        M.mapi_matrix_free(ctx, mat)


@pytest.mark.parametrize("op", ["min1", "min2"])
@pytest.mark.parametrize("st", ["f32", "bf16"])
def test_pair_mode_top8_every_deflation_slot(mapi_ctx, op, st):
    """D = 1024, the largest pair-mode order, and k = 8 as in the PCA
    workload: components 2..8 deflate their iterate by 1..7 earlier outer
    products (Alg. 2 step 6 with the sum form of §1).  The epilogue gives
    earlier component m to CTA rank m mod 4 of the last cluster and, within
    it, to warp group m div 4, so this covers all four ranks of both groups."""
    D, N, k, T = 1024, 8192, 8, 12
    X = spiked(D, N, seed=51)
    W0 = np.stack([datagen.start_vector(D, seed=510 + c) for c in range(k)])
    Xs = X.astype(np.float64) if st == "f32" else oracle.quant_bf16(X)
    done, _ = _pair_topk_parity(mapi_ctx, X, Xs, k, op, T, W0, st)
    if op == "min1":
        assert done == k  # min1 never stops on a zero norm here


@pytest.mark.parametrize("op", ["min1", "min2", "dot"])
@pytest.mark.parametrize("k", [12, 20])
def test_pair_mode_more_components_than_epilogue_slots(mapi_ctx, op, k):
    """k = 12 and 20: earlier components beyond the eight the epilogue holds
    at once (m >= 8) are loaded again by the warp group that owns them, up to
    three components per group."""
    D, N, T = 64, 2000, 10
    X = spiked(D, N, seed=61 + k)
    W0 = np.stack([datagen.start_vector(D, seed=610 + c) for c in range(k)])
    done, _ = _pair_topk_parity(mapi_ctx, X, X.astype(np.float64), k, op, T, W0)
    if op != "min2":
        assert done == k


def test_pair_step_full_size_all_deflation_slots(mapi_ctx):
    """D = 1024, N = 65536 (the PCA workload), k = 8 with one step per
    component: component c (c = 1..8) makes one pair step from its start and
    deflates it by the GPU's own components 1..c-1, so the oracle is fed the
    same earlier components and compared one step at a time.  The starts are
    the planted directions, so the components are well separated."""
    D, N, k = 1024, 65536, 8
    X = spiked(D, N, seed=0)
    U = datagen.spiked_pca_basis(D, seed=0)
    W0 = np.ascontiguousarray(U[:, :k].T.astype(np.float32))
    mat = M.mapi_matrix_upload(mapi_ctx, to_dev(X), "f32")
    try:
        P, its = M.mapi_pca_topk(mapi_ctx, mat, k, "pair", "min1", 1, float(N), to_dev(W0))
        assert its == [1] * k
        P = to_host(P)
        for c in range(k):
            w = W0[c].astype(np.float64)
            y = oracle.pair_step("min1", X, w / np.linalg.norm(w), float(N))
            if c:
                y = oracle.deflate_vec("min1", y, P[:c].T)
            want = y / np.abs(y).sum()
            want /= np.linalg.norm(want)
            assert rel_l1(P[c], want) <= TOL32, c
    finally:
        M.mapi_matrix_free(mapi_ctx, mat)


def test_pca_bad_arguments(mapi_ctx):
    X = spiked(16, 64, seed=1)
    mat = M.mapi_matrix_upload(mapi_ctx, to_dev(X), "f32")
    try:
        w0 = to_dev(np.ones((17, 16), np.float32))
        with pytest.raises(M.MapiError):
            M.mapi_pca_topk(mapi_ctx, mat, 17, "pair", "min1", 3, 64.0, w0)
        with pytest.raises(M.MapiError):
            M.mapi_pca_topk(mapi_ctx, mat, 1, "pair", "diamond", 3, 64.0, w0[:1])
        with pytest.raises(M.MapiError):
            M.mapi_pca_topk(mapi_ctx, mat, 1, "pair", "min1", 3, 0.0, w0[:1])
    finally:
        M.mapi_matrix_free(mapi_ctx, mat)
