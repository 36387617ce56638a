"""The allocation-free entry point (mapi_iterate_noalloc) against the
ordinary one.

Callers whose device memory belongs to another allocator, or that cannot pay
for cudaMalloc's device synchronisation, use mapi_iterate_noalloc: its
scratch is a fixed static device array, so it allocates nothing.  It must
give what mapi_iterate gives on the same input, within the FP32 tolerance,
on consecutive calls that share that array: on every operator, when the stop
rule fires before the last step (the last iterate then sits in the scratch
buffer chosen by the parity of the steps taken), with no step at all, and
from a raw start.  This file is collected last so that a failure here leaves
every other test already run.
"""
import numpy as np
import pytest

import datagen
import paper_2110_12065_gb300 as M
from tests.helpers import rel_l1

TOL32 = 1e-5


def test_no_alloc_wrapper_rejects_bad_buffers_before_any_launch():
    """Checked on the host, before the library is called: a short or
    half-precision output, a short start vector, too few columns and host
    tensors are all refused (no GPU needed)."""
    import torch
    n = 12
    A = torch.zeros((n, n), dtype=torch.float32)
    w0 = torch.ones(n, dtype=torch.float32)
    for kw, msg in (({"w_out": torch.empty(n - 1)}, "w_out"),
                    ({"w_out": torch.empty(n, dtype=torch.float16)}, "w_out")):
        with pytest.raises(ValueError, match=msg):
            M.mapi_iterate_noalloc(A, "min1", w0, 3, **kw)
    with pytest.raises(ValueError, match="w0"):
        M.mapi_iterate_noalloc(A, "min1", w0[:-1], 3, w_out=torch.empty(n))
    with pytest.raises(ValueError, match="columns"):
        M.mapi_iterate_noalloc(A[:, :-1], "min1", w0, 3, w_out=torch.empty(n))
    with pytest.raises(ValueError, match="CUDA"):
        M.mapi_iterate_noalloc(A, "min1", w0, 3, w_out=torch.empty(n))


def _reference(ctx, A, op, w0, T, tol=0.0, flags=0):
    import torch
    mat = M.mapi_matrix_upload(ctx, torch.from_numpy(A).cuda(), "f32")
    try:
        w, it, dl = M.mapi_iterate(ctx, mat, op, torch.from_numpy(w0).cuda(), T, tol_l1=tol,
                                   flags=flags)
    finally:
        M.mapi_matrix_free(ctx, mat)
    return w.cpu().numpy().astype(np.float64), it[0], dl[0]


def _no_alloc(A, op, w0, T, tol=0.0, flags=0):
    import torch
    n = A.shape[0]
    # rows padded to a multiple of 4 floats, padding filled with junk
    lda = (n + 3) // 4 * 4 + 4
    Ad = torch.full((n, lda), float("nan"), device="cuda")
    Ad[:, :n] = torch.from_numpy(A).cuda()
    w_out = torch.empty(n, device="cuda")
    w, it, dl = M.mapi_iterate_noalloc(Ad, op, torch.from_numpy(w0).cuda(), T, tol_l1=tol,
                                       flags=flags, w_out=w_out)
    torch.cuda.synchronize()
    return w.cpu().numpy().astype(np.float64), it, dl


@pytest.mark.gpu
def test_no_alloc_matches_mapi_iterate_on_consecutive_calls(mapi_ctx):
    cases = [(1000, "min1", 20, 0), (301, "min2", 7, M.FLAG_FINAL_L2),
             (257, "diamond", 9, 0), (333, "dot", 11, M.FLAG_FINAL_L2)]
    for n, op, T, flags in cases:  # calls in a row share the static scratch
        A = datagen.symmetric_gaussian(n, seed=n).astype(np.float32)
        if op == "diamond":  # Prop. 1 setting: positive entries
            A = np.abs(A)
        w0 = datagen.start_vector(n, seed=n + 7)
        w, it, _ = _no_alloc(A, op, w0, T, flags=flags)
        want, it_ref, _ = _reference(mapi_ctx, A, op, w0, T, flags=flags)
        assert it == it_ref == T
        assert rel_l1(w, want) <= TOL32, op


@pytest.mark.gpu
@pytest.mark.parametrize("n,op,scale", [(300, "min1", 0.002), (301, "min1", 0.003),
                                        (301, "min2", 0.002)])
def test_no_alloc_stop_rule_before_the_last_step(mapi_ctx, n, op, scale):
    """A small positive matrix converges in 5 or 6 steps, so the tolerance
    stops the solve long before T; the steps taken, the last delta and the
    iterate must match mapi_iterate's (an odd and an even step count both
    occur across the cases)."""
    A = (np.abs(datagen.symmetric_gaussian(n, seed=n + 1)) * scale).astype(np.float32)
    w0 = datagen.start_vector(n, seed=n + 8, low=0.0, high=1.0)
    T, tol = 200, 1e-6
    w, it, dl = _no_alloc(A, op, w0, T, tol=tol)
    want, it_ref, dl_ref = _reference(mapi_ctx, A, op, w0, T, tol=tol)
    assert it == it_ref and 0 < it < T
    assert dl < tol and abs(dl - dl_ref) <= 0.5 * tol
    assert rel_l1(w, want) <= TOL32


@pytest.mark.gpu
def test_no_alloc_zero_steps_and_raw_start(mapi_ctx):
    n = 129
    A = datagen.symmetric_gaussian(n, seed=3).astype(np.float32)
    w0 = datagen.start_vector(n, seed=4)
    # no step: the start vector at unit l2 norm (Alg. 1 step 1)
    w, it, _ = _no_alloc(A, "min1", w0, 0)
    assert it == 0
    np.testing.assert_allclose(w, w0 / np.linalg.norm(w0.astype(np.float64)), rtol=1e-6,
                               atol=1e-7)
    # a raw start is used as given, then stepped as usual
    w, it, _ = _no_alloc(A, "min1", w0, 0, flags=M.FLAG_RAW_START)
    np.testing.assert_array_equal(w, w0.astype(np.float64))
    w, it, _ = _no_alloc(A, "min2", w0, 5, flags=M.FLAG_RAW_START)
    want, it_ref, _ = _reference(mapi_ctx, A, "min2", w0, 5, flags=M.FLAG_RAW_START)
    assert it == it_ref == 5
    assert rel_l1(w, want) <= TOL32


@pytest.mark.gpu
def test_no_alloc_rejects_sizes_beyond_its_maximum():
    import torch
    A = torch.zeros((8200, 8200), device="cuda")
    w0 = torch.ones(8200, device="cuda")
    with pytest.raises(M.MapiError) as e:
        M.mapi_iterate_noalloc(A, "min1", w0, 1, w_out=torch.empty_like(w0))
    assert e.value.name == "EINVAL"
