"""Seeded synthetic inputs for MAPI workloads.

This module is the one piece of code that both the CPU oracle (``oracle/``)
and the CUDA path use.  It holds none of the method's arithmetic: it draws
matrices, data sets, graphs and start vectors with numpy's PCG64 generator and
returns them.  Every MAVP product, normalisation, covariance, deflation and
Google-matrix step lives on each side separately.

Workload shapes follow the paper's experiments:

* a dense symmetric Gaussian matrix for plain MAPI / RPI (Alg. 1);
* zero-mean D x N data with a few strong principal directions and impulsive
  outliers, the setting of the min-covariance PCA experiments (§3.1: image
  patches with occluding noise; §2.1 Eq. (5));
* a directed scale-free graph for PageRank (§3.3, Eq. (11)); the paper's
  Gnutella graphs are not available, so a Barabasi-Albert digraph of the same
  kind (power-law in-degree) stands in for them;
* symmetric positive semi-definite Wishart instances of mixed sizes for
  batched runs;
* start vectors drawn uniformly (Alg. 1 step 1 asks for a random w0);
* occluded versions of a synthetic gray-scale image for the reconstruction of
  Alg. 2 (§3.1: 16 tiles, 3 of them replaced by uniform noise); the paper's
  photographs are not available.
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "rng",
    "start_vector",
    "start_vectors",
    "symmetric_gaussian",
    "spiked_pca_data",
    "spiked_pca_basis",
    "barabasi_albert_digraph",
    "wishart_sizes",
    "wishart_instance",
    "small_grid_matrix",
    "wishart_instance_device",
    "barabasi_albert_digraph_fast",
    "stochastic_pca_data",
    "minibatches",
    "clean_image",
    "occluded_images",
]

DEFAULT_SPIKES = (50.0, 30.0, 20.0, 10.0, 5.0, 4.0, 3.0, 2.0)


def rng(seed: int) -> np.random.Generator:
    """numpy Generator over PCG64 with the given seed."""
    return np.random.Generator(np.random.PCG64(seed))


def start_vector(n: int, seed: int, low: float = -1.0, high: float = 1.0,
                 dtype=np.float32) -> np.ndarray:
    """Uniform(low, high)^n draw, cast to ``dtype`` (raw, not normalised)."""
    return rng(seed).uniform(low, high, size=n).astype(dtype)


def start_vectors(n: int, k: int, seed: int, low: float = -1.0,
                  high: float = 1.0, dtype=np.float32) -> np.ndarray:
    """k uniform start vectors as an n x k column-major (Fortran) array."""
    v = rng(seed).uniform(low, high, size=(k, n)).astype(dtype)
    return np.asfortranarray(v.T)


def symmetric_gaussian(n: int, seed: int = 0, dtype=np.float64) -> np.ndarray:
    """A = (G + G^T)/2 with G_ij ~ N(0, 1): a dense symmetric test matrix."""
    g = rng(seed).standard_normal((n, n))
    return ((g + g.T) * 0.5).astype(dtype)


def spiked_pca_data(D: int, N: int, seed: int = 0,
                    spikes=DEFAULT_SPIKES, outlier_frac: float = 0.01,
                    laplace_scale: float = 20.0,
                    dtype=np.float32, chunk: int = 8192) -> np.ndarray:
    """Zero-mean D x N data (row-major) with a spiked covariance and outliers.

    Column x = U diag(sqrt(lambda - 1)) z_k + z_D, where U (D x k) is a random
    orthonormal basis (QR of a Gaussian matrix) and z ~ N(0, I), so the
    population covariance has eigenvalues ``spikes`` and 1 elsewhere.  Then a
    fraction ``outlier_frac`` of the entries (a seeded mask) is replaced by
    Laplace(0, laplace_scale) draws, the impulsive noise the min-covariance is
    meant to resist, and finally every row's mean is removed so that the data
    set is zero-mean as the PCA setting of §1 requires.
    """
    r = rng(seed)
    k = min(len(spikes), D)
    lam = np.asarray(spikes[:k], dtype=np.float64)
    q, _ = np.linalg.qr(r.standard_normal((D, k)))
    scale = np.sqrt(np.maximum(lam - 1.0, 0.0))
    X = np.empty((D, N), dtype=np.float64)
    for c0 in range(0, N, chunk):
        c1 = min(N, c0 + chunk)
        z_k = r.standard_normal((k, c1 - c0))
        z_d = r.standard_normal((D, c1 - c0))
        X[:, c0:c1] = q @ (scale[:, None] * z_k) + z_d
    mask = r.random((D, N)) < outlier_frac
    cnt = int(mask.sum())
    X[mask] = r.laplace(0.0, laplace_scale, size=cnt)
    X -= X.mean(axis=1, keepdims=True)
    return np.ascontiguousarray(X.astype(dtype))


def spiked_pca_basis(D: int, seed: int = 0, spikes=DEFAULT_SPIKES) -> np.ndarray:
    """The orthonormal D x k basis U that ``spiked_pca_data`` plants with the
    same seed (its first draw), for tests that start an iteration near the
    planted directions."""
    k = min(len(spikes), D)
    q, _ = np.linalg.qr(rng(seed).standard_normal((D, k)))
    return q


def barabasi_albert_digraph(n: int, m: int = 8, seed: int = 0):
    """Directed preferential-attachment graph as out-link CSR (indptr, indices).

    The first ``m`` nodes start isolated (they have no out-links, i.e. they are
    dangling).  Every later node v links to ``m`` distinct earlier nodes, each
    picked with probability proportional to (in-degree + out-degree + 1).
    Returns int32 arrays: the out-neighbours of node j are
    ``indices[indptr[j]:indptr[j+1]]`` (sorted ascending).
    """
    r = rng(seed)
    # urn holds every node once (the "+1") plus once per incident edge end
    urn = list(range(min(m, n)))
    out = [[] for _ in range(n)]
    for v in range(m, n):
        chosen = set()
        while len(chosen) < m:
            # draw in small batches to keep the Python loop short
            picks = r.integers(0, len(urn), size=2 * m)
            for p in picks:
                t = urn[int(p)]
                if t not in chosen:
                    chosen.add(t)
                    if len(chosen) == m:
                        break
        tgt = sorted(chosen)
        out[v] = tgt
        urn.extend(tgt)          # targets gain in-degree
        urn.extend([v] * m)      # v gains out-degree
        urn.append(v)            # v joins with weight 1
    indptr = np.zeros(n + 1, dtype=np.int64)
    for j in range(n):
        indptr[j + 1] = indptr[j] + len(out[j])
    indices = np.fromiter((t for j in range(n) for t in out[j]),
                          dtype=np.int32, count=int(indptr[-1]))
    return indptr.astype(np.int32), indices


def wishart_sizes(count: int, seed: int = 0, nmin: int = 64,
                  nmax: int = 2048) -> np.ndarray:
    """Instance sizes n = floor(exp(U(ln nmin, ln nmax))), int32."""
    u = rng(seed).uniform(math.log(nmin), math.log(nmax), size=count)
    return np.clip(np.floor(np.exp(u)), nmin, nmax).astype(np.int32)


def wishart_instance(n: int, seed: int, dtype=np.float32) -> np.ndarray:
    """A = W W^T / k with W ~ N(0,1)^{n x k}, k = max(1, n // 2)."""
    k = max(1, n // 2)
    w = rng(seed).standard_normal((n, k))
    return ((w @ w.T) / k).astype(dtype)


def small_grid_matrix(n: int, seed: int, grid=(-2, -1, 0, 1, 2, 3)) -> np.ndarray:
    """n x n integer matrix with entries drawn from a small signed grid.

    Small integers make exact rational brute force cheap and create ties and
    zeros on purpose.
    """
    g = np.asarray(grid, dtype=np.int64)
    return g[rng(seed).integers(0, len(g), size=(n, n))]


def wishart_instance_device(n: int, seed: int, device="cuda"):
    """A = W W^T / k, W ~ N(0,1)^{n x k}, k = max(1, n // 2), drawn on the GPU
    with a seeded torch generator (FP32), for batches too large to draw on the
    host.  Deterministic for a given seed, device type and torch build."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    k = max(1, n // 2)
    w = torch.randn(n, k, generator=g, device=device, dtype=torch.float32)
    return (w @ w.T) / k


def barabasi_albert_digraph_fast(n: int, m: int = 8, seed: int = 0):
    """The preferential-attachment digraph of ``barabasi_albert_digraph``,
    drawn in blocks for large n: the nodes of a block pick their m distinct
    targets among the nodes before the block, weighted as in the urn at the
    block's start (the block grows with the graph, 1/16 of the nodes so far).
    Same out-link CSR (int32, targets ascending); a different (faster) draw."""
    r = rng(seed)
    m = min(m, max(n - 1, 1))
    urn = np.arange(min(m, n), dtype=np.int64)
    targets = np.zeros((max(n - m, 0), m), dtype=np.int64)
    v0 = m
    while v0 < n:
        v1 = min(n, v0 + max(64, v0 // 16))
        cnt = v1 - v0
        pick = urn[r.integers(0, urn.size, size=(cnt, m))]
        while True:
            srt = np.sort(pick, axis=1)
            dup_rows = np.nonzero((srt[:, 1:] == srt[:, :-1]).any(axis=1))[0]
            if dup_rows.size == 0:
                break
            for k in dup_rows:
                row = pick[k]
                _, first = np.unique(row, return_index=True)
                mask = np.ones(m, dtype=bool)
                mask[first] = False
                row[mask] = urn[r.integers(0, urn.size, size=int(mask.sum()))]
        pick.sort(axis=1)
        targets[v0 - m:v1 - m] = pick
        own = np.repeat(np.arange(v0, v1, dtype=np.int64), m + 1)
        urn = np.concatenate([urn, pick.ravel(), own])
        v0 = v1
    indptr = np.zeros(n + 1, dtype=np.int64)
    indptr[m + 1:] = np.arange(1, n - m + 1, dtype=np.int64) * m
    return indptr.astype(np.int32), targets.ravel().astype(np.int32)


def stochastic_pca_data(N: int = 10 ** 6, D: int = 10, seed: int = 0,
                        dtype=np.float32) -> np.ndarray:
    """X = U diag(1, sqrt(0.9), ..., sqrt(0.9)) V^T (N x D, rows are samples),
    U an N x D random orthonormal basis and V a random D x D orthogonal matrix
    (QR of Gaussians), so X^T X has eigenvalues 1, 0.9, ...: the synthetic
    set of the §3.2 comparison with the stochastic power method."""
    r = rng(seed)
    U, _ = np.linalg.qr(r.standard_normal((N, D)))
    V, _ = np.linalg.qr(r.standard_normal((D, D)))
    sig = np.sqrt(np.array([1.0] + [0.9] * (D - 1)))[:D]
    return np.ascontiguousarray(((U * sig) @ V.T).astype(dtype))


def minibatches(N: int, T: int, s: int, seed: int = 0) -> np.ndarray:
    """T x s sample indices drawn uniformly with replacement (Alg. 3 step 3)."""
    return rng(seed).integers(0, N, size=(T, s)).astype(np.int32)


def clean_image(side: int = 128, seed: int = 0) -> np.ndarray:
    """A smooth side x side gray-scale image in [0, 1] (float32): a soft
    gradient plus a few Gaussian blobs of random place, width and sign."""
    r = rng(seed)
    yy, xx = np.mgrid[0:side, 0:side].astype(np.float64) / max(side - 1, 1)
    img = 0.35 + 0.25 * (xx * r.uniform(-1, 1) + yy * r.uniform(-1, 1))
    for _ in range(6):
        cx, cy = r.uniform(0.1, 0.9, 2)
        sw = r.uniform(0.05, 0.2)
        img += r.uniform(-0.35, 0.35) * np.exp(-((xx - cx) ** 2 + (yy - cy) ** 2) / (2 * sw * sw))
    return np.clip(img, 0.0, 1.0).astype(np.float32)


def occluded_images(side: int = 128, N: int = 10, grid: int = 4, n_occ: int = 3,
                    seed: int = 0):
    """(clean (side x side), corrupted (N x side x side)): each of the N
    versions has n_occ of its grid x grid tiles (chosen without repetition)
    replaced by i.i.d. U[0, 1] pixels (§3.1: 32 x 32 tiles of a 128 x 128
    image, 3 of 16 replaced).  side must be a multiple of grid."""
    if side % grid:
        raise ValueError("side must be a multiple of grid")
    clean = clean_image(side, seed)
    r = rng(seed + 1)
    t = side // grid
    out = np.repeat(clean[None], N, axis=0)
    for i in range(N):
        for tile in r.choice(grid * grid, size=n_occ, replace=False):
            ty, tx = divmod(int(tile), grid)
            out[i, ty * t:(ty + 1) * t, tx * t:(tx + 1) * t] = r.uniform(0, 1, (t, t))
    return clean, out.astype(np.float32)
