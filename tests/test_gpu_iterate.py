"""GPU parity of Alg. 1 (MAPI) and RPI through the C ABI against the FP64
oracle: K1 MAVP-GEMV, the fused l1/l2 normalisation and stop test, the
start-vector step and the optional final l2 step.

Tolerances (float storage), relative l1 error of the returned vector:
  FP32 storage                     <= 1e-5 against the FP64 oracle
  BF16 / FP8 storage               <= 1e-5 against the oracle run on the
                                      dequantised stored values (the kernel's
                                      accumulation error only), and BF16
                                      <= 2e-2 against the original matrix
Integer storage: bit-exact.
"""
import numpy as np
import pytest
import torch

import datagen
import oracle
import paper_2110_12065_gb300 as M
from tests.helpers import rel_l1, to_dev, to_host

pytestmark = pytest.mark.gpu

TOL32 = 1e-5


def upload(ctx, A, storage="f32"):
    return M.mapi_matrix_upload(ctx, to_dev(A.astype(np.float32)), storage)


def gpu_iter(ctx, mat, op, w0, T, **kw):
    w, it, dl = M.mapi_iterate(ctx, mat, op, to_dev(w0.astype(np.float32)), T, **kw)
    return to_host(w), it, dl


@pytest.mark.parametrize("op", ["min1", "min2", "dot"])
@pytest.mark.parametrize("n", [1, 3, 37, 130, 512, 1000])
def test_one_step_parity_f32(mapi_ctx, op, n):
    A = datagen.symmetric_gaussian(n, seed=n).astype(np.float32)
    w0 = datagen.start_vector(n, seed=n + 1)
    mat = upload(mapi_ctx, A)
    try:
        st, want, oit, _ = oracle.mapi(op, A, w0.astype(np.float64), 1)
        if st != oracle.OK:  # e.g. n = 1, min2, opposite signs: zero norm
            with pytest.raises(M.MapiError) as e:
                gpu_iter(mapi_ctx, mat, op, w0, 1)
            assert e.value.status == st and e.value.partial[1] == [oit]
            return
        w, it, _ = gpu_iter(mapi_ctx, mat, op, w0, 1)
        assert it == [1] and oit == 1
        assert rel_l1(w, want) <= TOL32
        # step from a GPU iterate (one-step parity, always well conditioned)
        w5, _, _ = gpu_iter(mapi_ctx, mat, op, w0, 5)
        w6, _, _ = gpu_iter(mapi_ctx, mat, op, w5, 1, flags=M.FLAG_RAW_START)
        _, want6, _, _ = oracle.mapi(op, A, w5, 1, raw_start=True)
        assert rel_l1(w6, want6) <= TOL32
    finally:
        M.mapi_matrix_free(mapi_ctx, mat)


@pytest.mark.parametrize("op", ["min1", "min2", "dot"])
def test_trajectory_parity_config1(mapi_ctx, op):
    """n = 512 symmetric Gaussian, 1, 10 and 200 steps (the small workload)."""
    n = 512
    A = datagen.symmetric_gaussian(n, seed=0).astype(np.float32)
    w0 = datagen.start_vector(n, seed=0)
    mat = upload(mapi_ctx, A)
    try:
        for T in (1, 10, 200):
            w, it, _ = gpu_iter(mapi_ctx, mat, op, w0, T)
            st, want, oit, _ = oracle.mapi(op, A, w0.astype(np.float64), T)
            assert it == [T] and oit == T
            err = rel_l1(w, want)
            assert err <= TOL32, (T, err)
    finally:
        M.mapi_matrix_free(mapi_ctx, mat)


def test_l1_norm_and_final_l2(mapi_ctx):
    n = 300
    A = datagen.symmetric_gaussian(n, seed=3).astype(np.float32)
    w0 = datagen.start_vector(n, seed=3)
    mat = upload(mapi_ctx, A)
    try:
        w, _, _ = gpu_iter(mapi_ctx, mat, "min1", w0, 7)
        assert abs(np.abs(w).sum() - 1) < 1e-5
        w2, _, _ = gpu_iter(mapi_ctx, mat, "min1", w0, 7, flags=M.FLAG_FINAL_L2)
        _, want, _, _ = oracle.mapi("min1", A, w0.astype(np.float64), 7, final_l2=True)
        assert abs(np.linalg.norm(w2) - 1) < 1e-5
        assert rel_l1(w2, want) <= TOL32
    finally:
        M.mapi_matrix_free(mapi_ctx, mat)


def test_tolerance_stop(mapi_ctx):
    n = 200
    A = (np.abs(datagen.symmetric_gaussian(n, seed=4)) + 0.5).astype(np.float32)
    w0 = np.abs(datagen.start_vector(n, seed=4)) + 0.1
    mat = upload(mapi_ctx, A)
    try:
        w, it, dl = gpu_iter(mapi_ctx, mat, "min1", w0, 500, tol_l1=1e-6)
        assert it[0] < 500 and dl[0] < 1e-6
        st, want, oit, odl = oracle.mapi("min1", A, w0.astype(np.float64), it[0])
        assert rel_l1(w, want) <= TOL32
        # the oracle with the same tolerance stops within one step of the GPU
        _, _, oit2, _ = oracle.mapi("min1", A, w0.astype(np.float64), 500, tol=1e-6)
        assert abs(oit2 - it[0]) <= 1
    finally:
        M.mapi_matrix_free(mapi_ctx, mat)


@pytest.mark.parametrize("nvec", [2, 3, 4, 8])
def test_multi_vector_matches_single(mapi_ctx, nvec):
    n = 257
    A = datagen.symmetric_gaussian(n, seed=5).astype(np.float32)
    W0 = np.stack([datagen.start_vector(n, seed=50 + v) for v in range(nvec)])
    mat = upload(mapi_ctx, A)
    try:
        w, it, _ = M.mapi_iterate(mapi_ctx, mat, "min1", to_dev(W0), 12)
        w = to_host(w)
        assert it == [12] * nvec
        for v in range(nvec):
            _, want, _, _ = oracle.mapi("min1", A, W0[v].astype(np.float64), 12)
            assert rel_l1(w[v], want) <= TOL32
    finally:
        M.mapi_matrix_free(mapi_ctx, mat)


def test_diamond_proposition1(mapi_ctx):
    """Proposition 1: positive A, positive w0 -> fixed point after two steps."""
    r = datagen.rng(6)
    n = 200
    A = r.uniform(0.01, 2.0, size=(n, n)).astype(np.float32)
    w0 = r.uniform(0.1, 1.0, size=n).astype(np.float32)
    mat = upload(mapi_ctx, A)
    try:
        w, _, _ = gpu_iter(mapi_ctx, mat, "diamond", w0, 2)
        lim = 1.0 + A.astype(np.float64).sum(1)
        assert rel_l1(w, lim / lim.sum()) <= TOL32
        _, want, _, _ = oracle.mapi("diamond", A, w0.astype(np.float64), 2)
        assert rel_l1(w, want) <= TOL32
    finally:
        M.mapi_matrix_free(mapi_ctx, mat)


def test_zero_norm_status(mapi_ctx):
    n = 40
    mat = upload(mapi_ctx, np.zeros((n, n), np.float32))
    try:
        w0 = datagen.start_vector(n, seed=7)
        with pytest.raises(M.MapiError) as e:
            gpu_iter(mapi_ctx, mat, "min1", w0, 3)
        assert e.value.name == "EZERONORM"
        w, it, _ = e.value.partial
        assert it == [0]
        np.testing.assert_allclose(to_host(w), w0 / np.linalg.norm(w0), rtol=1e-6)
    finally:
        M.mapi_matrix_free(mapi_ctx, mat)


def test_min2_all_signs_opposed(mapi_ctx):
    mat = upload(mapi_ctx, -np.ones((8, 8), np.float32))
    try:
        with pytest.raises(M.MapiError) as e:
            gpu_iter(mapi_ctx, mat, "min2", np.ones(8, np.float32), 1)
        assert e.value.name == "EZERONORM"
    finally:
        M.mapi_matrix_free(mapi_ctx, mat)


def test_nonfinite_inputs_rejected(mapi_ctx):
    A = np.ones((5, 5), np.float32)
    A[2, 3] = np.nan
    with pytest.raises(M.MapiError) as e:
        upload(mapi_ctx, A)
    assert e.value.name == "ENONFINITE"
    mat = upload(mapi_ctx, np.ones((5, 5), np.float32))
    try:
        with pytest.raises(M.MapiError) as e:
            gpu_iter(mapi_ctx, mat, "min1", np.array([1, np.inf, 0, 0, 1], np.float32), 1)
        assert e.value.name == "ENONFINITE"
    finally:
        M.mapi_matrix_free(mapi_ctx, mat)


def test_bad_arguments(mapi_ctx):
    mat = upload(mapi_ctx, np.ones((6, 4), np.float32))
    try:
        with pytest.raises(M.MapiError) as e:  # not square
            gpu_iter(mapi_ctx, mat, "min1", np.ones(6, np.float32), 1)
        assert e.value.name == "EINVAL"
    finally:
        M.mapi_matrix_free(mapi_ctx, mat)
    q = upload(mapi_ctx, np.eye(4, dtype=np.float32), "i16")
    try:
        with pytest.raises(M.MapiError):  # dot is not exact in integers
            gpu_iter(mapi_ctx, q, "dot", np.ones(4, np.float32), 1)
    finally:
        M.mapi_matrix_free(mapi_ctx, q)


# ---------------------------------------------------------------- storages

@pytest.mark.parametrize("n", [5, 37, 300])
def test_storage_pack_matches_oracle_quantisers(mapi_ctx, n):
    """a1: the packed copy holds exactly the values the format definitions give."""
    r = datagen.rng(8)
    A = (r.standard_normal((n, n + 3)) * 10.0 ** r.integers(-3, 2, (n, 1))).astype(np.float32)
    for st in ("f32", "bf16", "fp8", "i16", "i8"):
        mat = M.mapi_matrix_upload(mapi_ctx, to_dev(A), st)
        try:
            got, ex = M.mapi_matrix_download(mapi_ctx, mat)
            info = M.mapi_matrix_info(mat)
            if st == "f32":
                want = A.astype(np.float64)
            elif st == "bf16":
                want = oracle.quant_bf16(A)
            elif st == "fp8":
                want, oex = oracle.quant_fp8_rows(A)
                np.testing.assert_array_equal(ex, oex)
            else:
                q = oracle.int_scale(A, 16 if st == "i16" else 8)
                assert info["int_scale_log2"] == q
                want = oracle.quant_int(A, q) / 2.0 ** q
            np.testing.assert_array_equal(got, want)
        finally:
            M.mapi_matrix_free(mapi_ctx, mat)


@pytest.mark.parametrize("st", ["bf16", "fp8"])
@pytest.mark.parametrize("op", ["min1", "min2"])
def test_reduced_precision_parity(mapi_ctx, st, op):
    n = 384
    A = datagen.symmetric_gaussian(n, seed=9).astype(np.float32)
    w0 = datagen.start_vector(n, seed=9)
    deq = oracle.quant_bf16(A) if st == "bf16" else oracle.quant_fp8_rows(A)[0]
    mat = M.mapi_matrix_upload(mapi_ctx, to_dev(A), st)
    try:
        for T in (1, 10):
            w, _, _ = gpu_iter(mapi_ctx, mat, op, w0, T)
            _, want_deq, _, _ = oracle.mapi(op, deq, w0.astype(np.float64), T)
            assert rel_l1(w, want_deq) <= TOL32
            if st == "bf16":
                _, want, _, _ = oracle.mapi(op, A, w0.astype(np.float64), T)
                assert rel_l1(w, want) <= 2e-2
    finally:
        M.mapi_matrix_free(mapi_ctx, mat)


@pytest.mark.parametrize("st,bits", [("i16", 16), ("i8", 8)])
@pytest.mark.parametrize("op", ["min1", "min2"])
@pytest.mark.parametrize("n", [1, 37, 300])
def test_integer_storage_bit_exact(mapi_ctx, st, bits, op, n):
    r = datagen.rng(10 + n)
    A = r.uniform(-0.9, 0.9, size=(n, n)).astype(np.float32)
    w0 = r.uniform(-1, 1, size=n).astype(np.float32)
    q = oracle.int_scale(A, bits)
    Aq = oracle.quant_int(A, q)
    mat = M.mapi_matrix_upload(mapi_ctx, to_dev(A), st)
    try:
        for T in (1, 4, 25):
            try:
                w, it, dl = gpu_iter(mapi_ctx, mat, op, w0, T)
                gst = 0
            except M.MapiError as e:
                w, it, dl = to_host(e.partial[0]), e.partial[1], e.partial[2]
                gst = e.status
            ost, want, oit, odl = oracle.mapi_int(op, Aq, q, w0, T)
            assert gst == ost
            assert it[0] == oit
            np.testing.assert_array_equal(np.rint(w * 2.0 ** q).astype(np.int64), want)
            if oit > 0:
                assert dl[0] * 2.0 ** q == odl
    finally:
        M.mapi_matrix_free(mapi_ctx, mat)


@pytest.mark.parametrize("st", ["i16", "i8", "bf16", "fp8"])
@pytest.mark.parametrize("op", ["min1", "min2"])
def test_large_matrices_take_the_cluster_epilogue(mapi_ctx, st, op):
    """n = 5000 (>= 4096): BF16, FP8 and integer storage run K1 in clusters whose
    last one normalises; the grid is padded to whole clusters.  Integer
    storage stays bit-exact, BF16 and FP8 within 1e-5 of the oracle on the
    stored values."""
    n = 5000
    r = datagen.rng(77)
    # entries near 2^-10: int8 then takes the scale 2^17, fine enough for a
    # unit-l1 vector of 5000 entries (at 2^7 it would round to zero)
    A = (r.uniform(-0.9, 0.9, size=(n, n)) * 2.0 ** -10).astype(np.float32)
    if op == "min2":
        A = np.abs(A)
    w0 = r.uniform(0.0, 1.0, size=n).astype(np.float32)
    mat = M.mapi_matrix_upload(mapi_ctx, to_dev(A), st)
    try:
        w, it, dl = gpu_iter(mapi_ctx, mat, op, w0, 3)
        assert it[0] == 3
        if st in ("bf16", "fp8"):
            deq = oracle.quant_bf16(A) if st == "bf16" else oracle.quant_fp8_rows(A)[0]
            _, want, _, _ = oracle.mapi(op, deq, w0.astype(np.float64), 3)
            assert rel_l1(w, want) <= TOL32
        else:
            q = oracle.int_scale(A, 16 if st == "i16" else 8)
            ost, want, oit, odl = oracle.mapi_int(op, oracle.quant_int(A, q), q, w0, 3)
            assert ost == oracle.OK and oit == 3
            np.testing.assert_array_equal(np.rint(w * 2.0 ** q).astype(np.int64), want)
            assert dl[0] * 2.0 ** q == odl
    finally:
        M.mapi_matrix_free(mapi_ctx, mat)


def test_full_size_one_step_f32(mapi_ctx):
    """n = 16384 (the dense PageRank size), one step from a fixed iterate,
    against the oracle's full product."""
    n = 16384
    A = datagen.symmetric_gaussian(n, seed=11).astype(np.float32)
    w0 = datagen.start_vector(n, seed=11)
    w0 = (w0 / np.abs(w0).sum()).astype(np.float32)
    mat = upload(mapi_ctx, A)
    try:
        w, _, _ = gpu_iter(mapi_ctx, mat, "min1", w0, 1, flags=M.FLAG_RAW_START)
        y = oracle.matvec("min1", A, w0.astype(np.float64))
        assert rel_l1(w, y / np.abs(y).sum()) <= TOL32
    finally:
        M.mapi_matrix_free(mapi_ctx, mat)


@pytest.mark.parametrize("op", ["min1", "min2", "diamond"])
def test_switch_to_rpi_equals_the_two_phases(mapi_ctx, op):
    """MAPI then regular power iteration from its iterate (§3.2)."""
    n = 300
    A = datagen.symmetric_gaussian(n, seed=60).astype(np.float32)
    if op == "min2":
        A = np.abs(A)
    w0 = datagen.start_vector(n, seed=61)
    mat = M.mapi_matrix_upload(mapi_ctx, to_dev(A), "f32")
    try:
        w, it, dl = M.mapi_iterate_switch(mapi_ctx, mat, op, to_dev(w0), 20, 40)
    finally:
        M.mapi_matrix_free(mapi_ctx, mat)
    Ad = A.astype(np.float64)
    st, mid, it1, _ = oracle.mapi(op, Ad, w0.astype(np.float64), 20)
    st2, want, it2, _ = oracle.mapi("dot", Ad, mid, 40)
    assert it == [it1, it2] == [20, 40]
    assert rel_l1(to_host(w), want) <= 1e-5


@pytest.mark.parametrize("t1,t2", [(0, 30), (25, 0), (0, 0)])
def test_switch_with_an_empty_phase(mapi_ctx, t1, t2):
    """No MAPI steps: RPI from w0 at unit l2 norm; no RPI steps: MAPI's
    iterate at unit l2 norm (Alg. 1 step 1 of the second phase)."""
    n = 150
    A = datagen.symmetric_gaussian(n, seed=65).astype(np.float32)
    w0 = datagen.start_vector(n, seed=66)
    mat = M.mapi_matrix_upload(mapi_ctx, to_dev(A), "f32")
    try:
        w, it, _ = M.mapi_iterate_switch(mapi_ctx, mat, "min1", to_dev(w0), t1, t2)
    finally:
        M.mapi_matrix_free(mapi_ctx, mat)
    Ad = A.astype(np.float64)
    _, mid, it1, _ = oracle.mapi("min1", Ad, w0.astype(np.float64), t1)
    _, want, it2, _ = oracle.mapi("dot", Ad, mid, t2)
    assert it == [it1, it2] == [t1, t2]
    assert rel_l1(to_host(w), want) <= 1e-5
    assert abs(np.linalg.norm(to_host(w)) - 1.0) < 1e-5


def test_switch_reaches_the_eigenvector(mapi_ctx):
    """The RPI phase converges to the dominant eigenvector; MAPI alone stops at
    a nearby pseudo-eigenvector."""
    n = 200
    r = datagen.rng(62)
    Q, _ = np.linalg.qr(r.standard_normal((n, n)))
    lam = np.concatenate([[10.0, 5.0], r.uniform(0.0, 2.0, size=n - 2)])
    A = ((Q * lam) @ Q.T).astype(np.float32)
    w0 = datagen.start_vector(n, seed=63)
    mat = M.mapi_matrix_upload(mapi_ctx, to_dev(A), "f32")
    try:
        w, it, dl = M.mapi_iterate_switch(mapi_ctx, mat, "min1", to_dev(w0), 50, 200,
                                          rpi_tol=1e-7)
        wm, _, _ = M.mapi_iterate(mapi_ctx, mat, "min1", to_dev(w0), 50, flags=M.FLAG_FINAL_L2)
    finally:
        M.mapi_matrix_free(mapi_ctx, mat)
    u = np.linalg.eigh(A.astype(np.float64))[1][:, -1]
    got = to_host(w).astype(np.float64)
    err = 1.0 - (got @ u) ** 2
    err_mapi = 1.0 - (to_host(wm).astype(np.float64) @ u) ** 2
    assert it[0] == 50 and it[1] < 200 and dl[1] < 1e-7
    assert err < 1e-6 and err < err_mapi


def test_switch_reports_a_failed_first_phase(mapi_ctx):
    A = np.zeros((40, 40), np.float32)
    mat = M.mapi_matrix_upload(mapi_ctx, to_dev(A), "f32")
    try:
        with pytest.raises(M.MapiError) as e:
            M.mapi_iterate_switch(mapi_ctx, mat, "min1", to_dev(datagen.start_vector(40, 64)),
                                  10, 10)
        assert e.value.name == "EZERONORM"
        assert e.value.partial[1][1] == 0
    finally:
        M.mapi_matrix_free(mapi_ctx, mat)


def test_reused_storage_and_staging_hold_no_stale_data(mapi_ctx):
    # The context keeps the storage of freed matrices for the next matrix of
    # the same size, and one staging buffer for host uploads (grown to the
    # largest): a solve on a matrix that lands in reused storage, or that
    # came through a staging buffer last filled by a larger upload, must
    # equal the solve on a fresh upload in a fresh context.
    n, T = 300, 8
    w0 = to_dev(datagen.start_vector(n, seed=91))
    mats = [datagen.symmetric_gaussian(n, seed=90 + k).astype(np.float32) for k in range(2)]
    big = datagen.symmetric_gaussian(2 * n, seed=95).astype(np.float32)

    w0_big = to_dev(datagen.start_vector(2 * n, seed=96))

    def solve(ctx, A, host):
        mat = M.mapi_matrix_upload(ctx, A if host else to_dev(A), "f32")
        try:
            w, _, _ = M.mapi_iterate(ctx, mat, "min1", w0 if A.shape[0] == n else w0_big, T)
            return to_host(w)
        finally:
            M.mapi_matrix_free(ctx, mat)

    fresh = M.mapi_create(0)
    try:
        want = [solve(fresh, A, host=False) for A in mats]
    finally:
        M.mapi_destroy(fresh)
    got = []
    for k in (0, 1, 0, 1):
        got.append(solve(mapi_ctx, mats[k], host=(k == 1)))
        # a larger host upload in between grows the staging buffer
        solve(mapi_ctx, big, host=True)
    for g, k in zip(got, (0, 1, 0, 1)):
        np.testing.assert_array_equal(g, want[k])
