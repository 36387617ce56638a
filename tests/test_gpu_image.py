"""GPU parity of the outer-product kernels of Alg. 2 and of the image
reconstruction end to end, against the FP64 oracle.

mapi_mavp_project (step 8) is compared with oracle.reconstruct on the same
components and rows, from one row up to D = 16384 (the order of the 128 x 128
images of §3.1), across the kernel's per-thread widths (D = 1024, 1025, ...):
the output itself (the product plus the offset m, as step 8 writes it) and,
without an offset, the product alone, both within the FP32 bar of relative
l1 1e-5.  (The product alone is not compared after subtracting m from an
output that holds it: the FP32 rounding of product + m is u |m|, which is
several 1e-6 of a product of size 1/sqrt(D).)

mapi_image_reconstruct runs steps 1-8 (mean, centring, Eq. (5) with
1/(N - 1), MAPI with the deflation of step 6, reconstruction) and is compared
with oracle.image_reconstruct on synthetic occluded images (3 of 16 tiles
replaced by U[0, 1] noise), at sizes the oracle finishes in seconds; at the
full 128 x 128 size the dot path (regular power iteration) is checked against
the eigenvectors of C obtained from the N x N Gram matrix, and the MIN1 first
component against the oracle's Alg. 1 on the full C."""
import numpy as np
import pytest
import torch

import datagen
import oracle
import paper_2110_12065_gb300 as M
from tests.helpers import rel_l1, to_dev, to_host

pytestmark = pytest.mark.gpu

TOL = 1e-5


def components(D, k, seed):
    return np.stack([datagen.start_vector(D, seed=seed + c) for c in range(k)])  # (k, D)


@pytest.mark.parametrize("op", ["min1", "min2", "dot"])
@pytest.mark.parametrize("D,k,rows", [(1, 1, 1), (5, 2, 3), (1000, 3, 4), (1024, 1, 2),
                                      (1025, 2, 2), (3000, 3, 5), (16384, 2, 3)])
def test_project_matches_oracle(mapi_ctx, op, D, k, rows):
    W = components(D, k, seed=D + k)
    r = datagen.rng(D)
    Z = r.standard_normal((rows, D)).astype(np.float32)
    m = r.uniform(0, 1, D).astype(np.float32)
    out = to_host(M.mapi_mavp_project(mapi_ctx, op, to_dev(W), to_dev(Z), to_dev(m)))
    prod = oracle.reconstruct(op, W.T, Z.T.astype(np.float64), np.zeros(D)).T
    want = prod + m.astype(np.float64)
    for i in range(rows):
        assert rel_l1(out[i], want[i]) <= TOL, i
    out0 = to_host(M.mapi_mavp_project(mapi_ctx, op, to_dev(W), to_dev(Z)))
    for i in range(rows):
        assert rel_l1(out0[i], prod[i]) <= TOL, i


@pytest.mark.parametrize("op", ["min1", "min2", "dot"])
@pytest.mark.parametrize("D,k", [(2048, 1), (2049, 2), (8193, 1), (128, 64)])
def test_project_width_boundaries_and_most_components(mapi_ctx, op, D, k):
    W = components(D, k, seed=3 * D + k)
    Z = datagen.rng(D + 1).standard_normal((2, D)).astype(np.float32)
    out = to_host(M.mapi_mavp_project(mapi_ctx, op, to_dev(W), to_dev(Z)))
    want = oracle.reconstruct(op, W.T, Z.T.astype(np.float64), np.zeros(D)).T
    assert rel_l1(out, want) <= TOL


def test_project_no_rows(mapi_ctx):
    W = to_dev(components(64, 2, seed=1))
    out = M.mapi_mavp_project(mapi_ctx, "min1", W, torch.empty((0, 64), device="cuda"))
    assert out.shape == (0, 64)


def test_project_without_offset_and_ties(mapi_ctx):
    """Components with many equal magnitudes (ties in the ranking) and zeros."""
    D = 2048
    r = datagen.rng(5)
    W = (r.integers(-3, 4, size=(2, D)) / 4.0).astype(np.float32)
    Z = r.standard_normal((3, D)).astype(np.float32)
    for op in ("min1", "min2"):
        out = to_host(M.mapi_mavp_project(mapi_ctx, op, to_dev(W), to_dev(Z)))
        want = oracle.reconstruct(op, W.T, Z.T.astype(np.float64), np.zeros(D)).T
        assert rel_l1(out, want) <= TOL


def test_project_equal_magnitudes_is_the_projection(mapi_ctx):
    """Unit-l1 MIN1 outer products of equal-magnitude components are u u^T."""
    from scipy.linalg import hadamard
    D = 1024
    H = hadamard(D).astype(np.float32)[[3, 100, 517]]
    U = H / np.sqrt(D)
    Z = datagen.rng(6).standard_normal((2, D)).astype(np.float32)
    out = to_host(M.mapi_mavp_project(mapi_ctx, "min1", to_dev(H * 0.37), to_dev(Z)))
    want = (Z.astype(np.float64) @ U.T.astype(np.float64)) @ U.astype(np.float64)
    np.testing.assert_allclose(out, want, atol=2e-6 * np.abs(Z).sum(axis=1).max() / np.sqrt(D))


def test_project_rejects_bad_shapes(mapi_ctx):
    W = torch.ones((1, 16385), device="cuda")
    Z = torch.ones((1, 16385), device="cuda")
    with pytest.raises(M.MapiError) as e:
        M.mapi_mavp_project(mapi_ctx, "min1", W, Z)
    assert e.value.name == "EINVAL"
    with pytest.raises(M.MapiError) as e:
        M.mapi_mavp_project(mapi_ctx, "diamond", W[:, :8], Z[:, :8])
    assert e.value.name == "EINVAL"


def occluded(side, N, seed):
    clean, imgs = datagen.occluded_images(side, N, grid=4, n_occ=3, seed=seed)
    return clean, imgs.reshape(N, -1)


@pytest.mark.parametrize("op", ["min1", "min2", "dot"])
@pytest.mark.parametrize("side", [16, 24, 32, 40])
def test_image_reconstruct_matches_oracle(mapi_ctx, op, side):
    N, k, T = 10, 2, 20
    _, imgs = occluded(side, N, seed=side)
    P = side * side
    W0 = components(P, k, seed=300 + side)
    st, Wo, Ro, oits = oracle.image_reconstruct(op, imgs.astype(np.float64), k, T, W0.T)
    try:
        W, R, its = M.mapi_image_reconstruct(mapi_ctx, to_dev(imgs), k, op, T, to_dev(W0))
        gst = 0
    except M.MapiError as e:
        (W, R, its), gst = e.partial, e.status
    assert gst == st and its == list(oits)
    if st != oracle.OK:
        return
    W, R = to_host(W), to_host(R)
    for c in range(k):
        assert rel_l1(W[c], Wo[:, c]) <= TOL, c
    assert rel_l1(R, Ro) <= TOL


def test_image_reconstruct_repeated_calls_reuse_the_plan(mapi_ctx):
    _, imgs = occluded(32, 10, seed=9)
    W0 = components(1024, 2, seed=9)
    a = M.mapi_image_reconstruct(mapi_ctx, to_dev(imgs), 2, "min2", 15, to_dev(W0))
    b = M.mapi_image_reconstruct(mapi_ctx, to_dev(imgs), 2, "min2", 15, to_dev(W0))
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])
    # another shape, then the first again
    _, imgs2 = occluded(16, 6, seed=10)
    M.mapi_image_reconstruct(mapi_ctx, to_dev(imgs2), 1, "min1", 5, to_dev(components(256, 1, 3)))
    c = M.mapi_image_reconstruct(mapi_ctx, to_dev(imgs), 2, "min2", 15, to_dev(W0))
    assert torch.equal(a[1], c[1])


def test_image_reconstruct_errors(mapi_ctx):
    _, imgs = occluded(16, 4, seed=11)
    W0 = components(256, 2, seed=11)
    with pytest.raises(M.MapiError) as e:  # N = 1: no denominator N - 1
        M.mapi_image_reconstruct(mapi_ctx, to_dev(imgs[:1]), 1, "min1", 5, to_dev(W0[:1]))
    assert e.value.name == "EINVAL"
    same = np.tile(np.arange(256, dtype=np.float32) / 256, (4, 1))
    with pytest.raises(M.MapiError) as e:  # identical images: V - m = 0
        M.mapi_image_reconstruct(mapi_ctx, to_dev(same), 1, "min1", 5, to_dev(W0[:1]))
    assert e.value.name == "EZERONORM"


def test_image_reconstruct_full_size_dot_is_the_eigen_projection(mapi_ctx):
    """128 x 128 images: RPI components are the top eigenvectors of
    C = Z Z^T / (N - 1), found here from the N x N Gram matrix Z^T Z, and the
    reconstruction is m + U U^T (v_i - m)."""
    N, k, T = 10, 2, 400
    _, imgs = occluded(128, N, seed=13)  # Gram eigenvalue ratios 1.16 and 1.07
    P = imgs.shape[1]
    W, R, its = M.mapi_image_reconstruct(mapi_ctx, to_dev(imgs), k, "dot", T,
                                         to_dev(components(P, k, seed=12)))
    V = imgs.astype(np.float64).T
    m = V.mean(axis=1)
    Z = V - m[:, None]
    ev, Ug = np.linalg.eigh(Z.T @ Z)
    order = np.argsort(ev)[::-1]
    assert ev[order[0]] / ev[order[1]] > 1.05 and ev[order[1]] / ev[order[2]] > 1.05
    U = Z @ Ug[:, order[:k]]
    U /= np.linalg.norm(U, axis=0)
    W = to_host(W)
    for c in range(k):
        assert abs(W[c] @ U[:, c]) > 1 - 1e-6, c
    want = (m[:, None] + U @ (U.T @ Z)).T
    assert rel_l1(to_host(R), want) <= TOL


def test_image_reconstruct_full_size_min1_first_component(mapi_ctx):
    """128 x 128 images, MIN1: the first component against Alg. 1 run by the
    oracle on the full 16384 x 16384 min-covariance."""
    N, T = 10, 8
    _, imgs = occluded(128, N, seed=14)
    P = imgs.shape[1]
    W0 = components(P, 1, seed=13)
    W, R, its = M.mapi_image_reconstruct(mapi_ctx, to_dev(imgs), 1, "min1", T, to_dev(W0))
    V = imgs.astype(np.float64).T
    m = V.mean(axis=1)
    Cm = oracle.mincov("min1", V - m[:, None], float(N - 1))
    st, w, it, _ = oracle.mapi("min1", Cm, W0[0], T, final_l2=True)
    del Cm
    assert st == oracle.OK and its == [it]
    assert rel_l1(to_host(W)[0], w) <= TOL
    Ro = oracle.reconstruct("min1", w[:, None], V, m).T
    assert rel_l1(to_host(R), Ro) <= TOL
