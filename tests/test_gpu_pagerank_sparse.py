"""GPU parity of MAPI-PageRank without forming G (§3.3, Eq. (11)): the
O(E + n) kernels against the FP64 oracle on the same FP32 entry values, the
dense GPU path, and the edge cases of the in-link construction."""
import numpy as np
import pytest
import torch

import datagen
import oracle
import paper_2110_12065_gb300 as M
from tests.helpers import rel_l1, to_dev, to_host
from tests.test_oracle_pins import _graph_with_duplicates

pytestmark = pytest.mark.gpu

TOL32 = 1e-5


def run(ctx, ip, ix, w0, iters, op="min1", tol=0.0):
    n = ip.shape[0] - 1
    return M.mapi_pagerank_sparse(ctx, to_dev(ip), to_dev(ix), n, to_dev(w0), iters, op=op,
                                  tol_l1=tol)


@pytest.mark.parametrize("op", ["min1", "min2", "dot"])
@pytest.mark.parametrize("n,seed", [(1, 40), (7, 41), (60, 42), (400, 43), (3000, 44)])
def test_sparse_pagerank_matches_oracle(mapi_ctx, op, n, seed):
    ip, ix = _graph_with_duplicates(n, seed)
    w0 = datagen.start_vector(n, seed=seed, low=0.0, high=1.0)
    r, it, dl = run(mapi_ctx, ip, ix, w0, 25, op)
    st, want, oit, odl = oracle.pagerank_sparse(op, n, ip, ix, w0.astype(np.float64), 25)
    assert st == oracle.OK and it == oit == 25
    assert rel_l1(to_host(r), want) <= TOL32


def test_sparse_equals_dense_gpu_path(mapi_ctx):
    n = 2500  # in-links above 32 and 64 per node occur
    ip, ix = datagen.barabasi_albert_digraph(n, m=8, seed=45)
    assert np.bincount(ix, minlength=n).max() > 64
    w0 = datagen.start_vector(n, seed=45, low=0.0, high=1.0)
    r, it, _ = run(mapi_ctx, ip, ix, w0, 40)
    d, it2, _ = M.mapi_pagerank(mapi_ctx, to_dev(ip), to_dev(ix), n, to_dev(w0), 40)
    assert it == it2 == 40
    assert rel_l1(to_host(r), to_host(d)) <= TOL32


def test_sparse_stop_rule(mapi_ctx):
    ip, ix = datagen.barabasi_albert_digraph(800, m=8, seed=46)
    w0 = datagen.start_vector(800, seed=46, low=0.0, high=1.0)
    r, it, dl = run(mapi_ctx, ip, ix, w0, 1000, tol=1e-7)
    st, want, oit, odl = oracle.pagerank_sparse("min1", 800, ip, ix, w0.astype(np.float64), 1000,
                                                tol=1e-7)
    assert dl < 1e-7 and it < 1000 and abs(it - oit) <= 1
    assert abs(float(np.linalg.norm(to_host(r).astype(np.float64))) - 1.0) < 1e-5
    assert rel_l1(to_host(r), want) <= TOL32


def test_sparse_zero_iterations_and_zero_start(mapi_ctx):
    ip, ix = datagen.barabasi_albert_digraph(50, m=4, seed=47)
    w0 = datagen.start_vector(50, seed=47, low=0.0, high=1.0)
    r, it, _ = run(mapi_ctx, ip, ix, w0, 0)
    assert it == 0
    np.testing.assert_allclose(to_host(r), w0 / np.linalg.norm(w0.astype(np.float64)),
                               rtol=1e-6)
    with pytest.raises(M.MapiError) as e:
        run(mapi_ctx, ip, ix, np.zeros(50, np.float32), 5)
    assert e.value.name == "EZERONORM"


def test_sparse_rejects_bad_graphs(mapi_ctx):
    ip, ix = datagen.barabasi_albert_digraph(50, m=4, seed=48)
    w0 = datagen.start_vector(50, seed=48, low=0.0, high=1.0)
    bad = ix.copy()
    bad[7] = 50  # a target out of range, caught on the device
    with pytest.raises(M.MapiError) as e:
        run(mapi_ctx, ip, bad, w0, 5)
    assert e.value.name == "EINVAL"
    # more in-links to one node than one shared-memory sort holds
    n = 20000
    sip = np.arange(n + 1, dtype=np.int32)
    sip[0] = 0
    six = np.zeros(n, dtype=np.int32)
    six[0] = 1
    sw = datagen.start_vector(n, seed=49, low=0.0, high=1.0)
    with pytest.raises(M.MapiError) as e:
        run(mapi_ctx, sip, six, sw, 5)
    assert e.value.name == "ENOTSUP"
    # the context stays usable
    r, it, _ = run(mapi_ctx, ip, ix, w0, 3)
    assert it == 3


def test_sparse_full_size_million_nodes(mapi_ctx):
    n = 1 << 20
    ip, ix = datagen.barabasi_albert_digraph_fast(n, m=8, seed=0)
    w0 = datagen.start_vector(n, seed=0, low=0.0, high=1.0)
    r, it, _ = run(mapi_ctx, ip, ix, w0, 20)
    st, want, oit, _ = oracle.pagerank_sparse("min1", n, ip, ix, w0.astype(np.float64), 20)
    assert st == oracle.OK and it == oit == 20
    assert rel_l1(to_host(r), want) <= TOL32
