"""GPU parity of MAPI-PageRank (§3.3): the dense Google matrix of Eq. (11)
built on the device, and the iteration on every storage."""
import numpy as np
import pytest

import datagen
import oracle
import paper_2110_12065_gb300 as M
from tests.helpers import rel_l1, to_dev, to_host

pytestmark = pytest.mark.gpu


def graph(n, m, seed):
    ip, ix = datagen.barabasi_albert_digraph(n, m=m, seed=seed)
    return ip, ix, to_dev(ip), to_dev(ix)


@pytest.mark.parametrize("n", [9, 300, 1001])
def test_google_matrix_is_the_fp64_definition_rounded(mapi_ctx, n):
    ip, ix, dip, dix = graph(n, 4, n)
    G = M.mapi_google_matrix(mapi_ctx, dip, dix, n, 0.85, "f32")
    try:
        got, _ = M.mapi_matrix_download(mapi_ctx, G)
        want = oracle.google_matrix(n, ip, ix, 0.85).astype(np.float32).astype(np.float64)
        np.testing.assert_array_equal(got, want)
    finally:
        M.mapi_matrix_free(mapi_ctx, G)


@pytest.mark.parametrize("op", ["min1", "dot"])
def test_pagerank_f32(mapi_ctx, op):
    n = 700
    ip, ix, dip, dix = graph(n, 8, 1)
    w0 = datagen.start_vector(n, seed=2, low=0.0, high=1.0)
    r, it, dl = M.mapi_pagerank(mapi_ctx, dip, dix, n, to_dev(w0), 30, op=op)
    G = oracle.google_matrix(n, ip, ix, 0.85).astype(np.float32).astype(np.float64)
    st, want, oit, _ = oracle.mapi(op, G, w0.astype(np.float64), 30, final_l2=True)
    assert it == oit == 30
    assert rel_l1(to_host(r), want) <= 1e-5


@pytest.mark.parametrize("st", ["bf16", "fp8"])
def test_pagerank_reduced_precision(mapi_ctx, st):
    n = 513
    ip, ix, dip, dix = graph(n, 8, 3)
    w0 = datagen.start_vector(n, seed=4, low=0.0, high=1.0)
    r, it, _ = M.mapi_pagerank(mapi_ctx, dip, dix, n, to_dev(w0), 20, storage=st)
    G32 = oracle.google_matrix(n, ip, ix, 0.85).astype(np.float32)
    deq = oracle.quant_bf16(G32) if st == "bf16" else oracle.quant_fp8_rows(G32)[0]
    _, want, _, _ = oracle.mapi("min1", deq, w0.astype(np.float64), 20, final_l2=True)
    assert rel_l1(to_host(r), want) <= 1e-5


def test_pagerank_int16_bit_exact(mapi_ctx):
    n = 400
    ip, ix, dip, dix = graph(n, 8, 5)
    w0 = datagen.start_vector(n, seed=6, low=0.0, high=1.0)
    G32 = oracle.google_matrix(n, ip, ix, 0.85).astype(np.float32)
    q = oracle.int_scale(G32, 16)
    Gq = oracle.quant_int(G32, q)
    G = M.mapi_google_matrix(mapi_ctx, dip, dix, n, 0.85, "i16")
    try:
        assert M.mapi_matrix_info(G)["int_scale_log2"] == q
        w, it, _ = M.mapi_iterate(mapi_ctx, G, "min1", to_dev(w0), 15)
        st, want, oit, _ = oracle.mapi_int("min1", Gq, q, w0, 15)
        assert it[0] == oit == 15
        np.testing.assert_array_equal(np.rint(to_host(w) * 2.0 ** q).astype(np.int64), want)
    finally:
        M.mapi_matrix_free(mapi_ctx, G)


def test_pagerank_int16_bit_exact_full_size(mapi_ctx):
    """The dense PageRank workload, n = 16384 (Barabasi-Albert m = 8, seed 0):
    the int16 copy iterated in exact integers (INT32 products, INT64 norm,
    the n integer divisions) equals the oracle's integer MAPI bit for bit."""
    n, T = 16384, 4
    ip, ix, dip, dix = graph(n, 8, 0)
    w0 = datagen.start_vector(n, seed=0, low=0.0, high=1.0)
    G32 = oracle.google_matrix(n, ip, ix, 0.85).astype(np.float32)
    q = oracle.int_scale(G32, 16)
    Gq = oracle.quant_int(G32, q)
    del G32
    G = M.mapi_google_matrix(mapi_ctx, dip, dix, n, 0.85, "i16")
    try:
        assert M.mapi_matrix_info(G)["int_scale_log2"] == q
        w, it, _ = M.mapi_iterate(mapi_ctx, G, "min1", to_dev(w0), T)
        st, want, oit, _ = oracle.mapi_int("min1", Gq, q, w0, T)
        assert st == oracle.OK and it[0] == oit == T
        np.testing.assert_array_equal(np.rint(to_host(w) * 2.0 ** q).astype(np.int64), want)
    finally:
        M.mapi_matrix_free(mapi_ctx, G)
