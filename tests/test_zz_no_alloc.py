"""The allocation-free entry point (mapi_iterate_noalloc) against the
ordinary one.

Callers whose device memory belongs to another allocator, or that cannot pay
for cudaMalloc's device synchronisation, use mapi_iterate_noalloc: its
scratch is a fixed static device array, so it allocates nothing.  It must
give what mapi_iterate gives on the same input, within the FP32 tolerance,
on consecutive calls that share that array.  This file is collected last so
that a failure here leaves every other test already run.
"""
import numpy as np
import pytest
import torch

import datagen
import paper_2110_12065_gb300 as M
from tests.helpers import rel_l1, to_dev, to_host

pytestmark = pytest.mark.gpu

TOL32 = 1e-5


def reference(ctx, A, op, w0, T, flags=0):
    mat = M.mapi_matrix_upload(ctx, to_dev(A), "f32")
    try:
        w, it, dl = M.mapi_iterate(ctx, mat, op, to_dev(w0), T, flags=flags)
    finally:
        M.mapi_matrix_free(ctx, mat)
    return to_host(w), it[0]


def test_no_alloc_matches_mapi_iterate_on_consecutive_calls(mapi_ctx):
    cases = [(1000, "min1", 20, 0), (301, "min2", 7, M.FLAG_FINAL_L2)]
    for n, op, T, flags in cases:  # two calls in a row share the static scratch
        A = datagen.symmetric_gaussian(n, seed=n).astype(np.float32)
        w0 = datagen.start_vector(n, seed=n + 7)
        # rows padded to a multiple of 4 floats, padding filled with junk
        lda = (n + 3) // 4 * 4 + 4
        Ad = torch.full((n, lda), float("nan"), device="cuda")
        Ad[:, :n] = to_dev(A)
        w_out = torch.empty(n, device="cuda")
        w, it, _ = M.mapi_iterate_noalloc(Ad, op, to_dev(w0), T, flags=flags, w_out=w_out)
        torch.cuda.synchronize()
        want, it_ref = reference(mapi_ctx, A, op, w0, T, flags)
        assert it == it_ref == T
        assert rel_l1(to_host(w), want) <= TOL32


def test_no_alloc_rejects_sizes_beyond_its_maximum():
    A = torch.zeros((8200, 8200), device="cuda")
    w0 = torch.ones(8200, device="cuda")
    with pytest.raises(M.MapiError) as e:
        M.mapi_iterate_noalloc(A, "min1", w0, 1, w_out=torch.empty_like(w0))
    assert e.value.name == "EINVAL"
