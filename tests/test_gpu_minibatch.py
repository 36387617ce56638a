"""GPU parity of mini-batch MAPI with momentum (Alg. 3) against the FP64
oracle on the same sample draws: MIN1, MIN2 and the momentum power method
(DOT), dimensions on both sides of the kernel's split of A_t over thread
groups, batches that fill several staging chunks, the full-size synthetic set
of the §3.2 comparison, and the error cases.

Tolerance: the FP32 bar, relative l1 1e-5.  Each entry of A_t is a sum of
s FP32 terms split over thread groups (bound about s u, u = 2^-24, in the
worst case; random-walk growth in practice), and the normalised steps do not
grow it: the largest distance measured over these cases is 2.1e-6."""
import numpy as np
import pytest
import torch

import datagen
import oracle
import paper_2110_12065_gb300 as M
from tests.helpers import rel_l1, to_dev, to_host

pytestmark = pytest.mark.gpu

TOL = 1e-5


def run(ctx, X, batch, beta, op, w0, final_l2=True):
    return M.mapi_minibatch_momentum(ctx, to_dev(X), torch.from_numpy(batch).cuda(), beta, op,
                                     to_dev(w0), M.FLAG_FINAL_L2 if final_l2 else 0)


def case(N, D, T, s, seed):
    X = datagen.stochastic_pca_data(N, D, seed=seed) * np.float32(np.sqrt(N))
    batch = datagen.minibatches(N, T, s, seed=seed + 1)
    w0 = datagen.start_vector(D, seed=seed + 2)
    return X.astype(np.float32), batch, w0


@pytest.mark.parametrize("op", ["min1", "min2", "dot"])
@pytest.mark.parametrize("beta", [0.0, 0.2025])
@pytest.mark.parametrize("N,D,T,s", [(50, 1, 5, 3), (400, 3, 20, 7), (3000, 10, 30, 1000),
                                     (3000, 10, 12, 1500), (500, 31, 10, 50),
                                     (500, 33, 10, 50), (800, 128, 4, 200)])
def test_minibatch_matches_oracle(mapi_ctx, op, beta, N, D, T, s):
    X, batch, w0 = case(N, D, T, s, seed=N + D)
    st, want = oracle.minibatch_momentum(op, X, batch, beta, w0)
    if st != oracle.OK:
        # D = 1 under MIN2 with w0 < 0: x (+) w is 0 when the signs differ
        assert (op, D, st) == ("min2", 1, oracle.EZERONORM)
        with pytest.raises(M.MapiError) as e:
            run(mapi_ctx, X, batch, beta, op, w0)
        assert e.value.name == "EZERONORM"
        return
    w = to_host(run(mapi_ctx, X, batch, beta, op, w0))
    assert rel_l1(w, want) <= TOL


def test_minibatch_full_size_set(mapi_ctx):
    """N = 10^6 samples of dimension 10, 100 steps of 1000 draws."""
    X, batch, w0 = case(10 ** 6, 10, 100, 1000, seed=7)
    for op in ("min1", "dot"):
        w = to_host(run(mapi_ctx, X, batch, 0.2025, op, w0))
        st, want = oracle.minibatch_momentum(op, X, batch, 0.2025, w0)
        assert st == oracle.OK
        assert rel_l1(w, want) <= TOL


def test_minibatch_without_final_l2(mapi_ctx):
    X, batch, w0 = case(600, 6, 15, 40, seed=3)
    w = to_host(run(mapi_ctx, X, batch, 0.1, "min2", w0, final_l2=False))
    st, want = oracle.minibatch_momentum("min2", X, batch, 0.1, w0, final_l2=False)
    assert st == oracle.OK
    assert rel_l1(w, want) <= TOL
    # the last step divided by the l1 norm of its product
    assert abs(np.abs(w).sum() - 1.0) < 1e-5


def test_minibatch_zero_steps_returns_the_start(mapi_ctx):
    X, _, w0 = case(100, 5, 1, 4, seed=4)
    batch = np.zeros((0, 4), np.int32)
    w = to_host(run(mapi_ctx, X, batch, 0.3, "min1", w0))
    np.testing.assert_allclose(w, w0 / np.linalg.norm(w0), rtol=1e-6, atol=1e-7)


def test_minibatch_errors(mapi_ctx):
    X, batch, w0 = case(100, 5, 3, 4, seed=5)
    with pytest.raises(M.MapiError) as e:
        run(mapi_ctx, X, batch, 0.0, "min1", np.zeros(5, np.float32))
    assert e.value.name == "EZERONORM"
    with pytest.raises(M.MapiError) as e:
        run(mapi_ctx, np.zeros_like(X), batch, 0.0, "min1", w0)
    assert e.value.name == "EZERONORM"
    bad = batch.copy()
    bad[1, 2] = 100
    with pytest.raises(M.MapiError) as e:
        run(mapi_ctx, X, bad, 0.0, "min1", w0)
    assert e.value.name == "EINVAL"
    with pytest.raises(M.MapiError) as e:
        run(mapi_ctx, X, batch, 0.0, "diamond", w0)
    assert e.value.name == "EINVAL"
    Xw = np.zeros((10, 129), np.float32)
    with pytest.raises(M.MapiError) as e:
        run(mapi_ctx, Xw, np.zeros((1, 1), np.int32), 0.0, "min1", np.ones(129, np.float32))
    assert e.value.name == "EINVAL"
    # the context stays usable
    w = to_host(run(mapi_ctx, X, batch, 0.0, "min1", w0))
    assert np.isfinite(w).all()
