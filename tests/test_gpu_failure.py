"""Failure detection on the device, tested without faulting the GPU.

Every wait inside the library's kernels (tile copies, cluster exchanges) is
bounded by %globaltimer and reports MAPI_ETIMEOUT when it runs out, so a
missing arrival stops the solve with a status instead of hanging the GPU.
These tests make such a wait run out on purpose: mapi_debug_stall makes the
pair step also wait, through the same bounded wait, on a barrier that
nothing ever arrives at (no copy or store is pending on it), with a 1 ms
limit.  The call must return MAPI_ETIMEOUT, and the same context must then
solve again and give the result it gave before."""
import numpy as np
import pytest
import torch

import datagen
import paper_2110_12065_gb300 as M
from tests.helpers import to_dev

pytestmark = pytest.mark.gpu


def test_a_wait_that_runs_out_stops_the_solve_and_the_context_recovers(mapi_ctx):
    D, N, k, T = 256, 4096, 2, 5
    X = datagen.spiked_pca_data(D, N, seed=71)
    W0 = to_dev(np.stack([datagen.start_vector(D, seed=710 + c) for c in range(k)]))
    mat = M.mapi_matrix_upload(mapi_ctx, to_dev(X), "f32")
    try:
        P_ok, its_ok = M.mapi_pca_topk(mapi_ctx, mat, k, "pair", "min1", T, float(N), W0)
        P_ok = P_ok.clone()
        assert its_ok == [T] * k
        M.mapi_debug_stall(mapi_ctx, 1_000_000)
        try:
            with pytest.raises(M.MapiError) as e:
                M.mapi_pca_topk(mapi_ctx, mat, k, "pair", "min1", T, float(N), W0)
            assert e.value.name == "ETIMEOUT"
            _, its = e.value.partial
            # the step whose wait ran out completes and stops the solve; the
            # later component is skipped
            assert its == [1, 0]
        finally:
            M.mapi_debug_stall(mapi_ctx, 0)
        P, its = M.mapi_pca_topk(mapi_ctx, mat, k, "pair", "min1", T, float(N), W0)
        assert its == its_ok
        assert torch.equal(P, P_ok)
    finally:
        M.mapi_matrix_free(mapi_ctx, mat)


def test_stall_hook_rejects_bad_limits(mapi_ctx):
    for bad in (-1, 3_000_000_000):
        with pytest.raises(M.MapiError) as e:
            M.mapi_debug_stall(mapi_ctx, bad)
        assert e.value.name == "EINVAL"
