"""Pins of the FP64 oracle against what the paper and mathematics fix.

Each test ties one oracle function to something other than itself: a value
the paper states (Proposition 1, the l1-inducing property), a hand-worked
example (tests/golden/), exact rational brute force (tests/exact_ref.py), a
closed form, an invariant, or a library routine that a special case reduces
to (numpy eigh / matrix_power / solve, torch's bf16 and fp8 casts).
"""
import os
from fractions import Fraction as Fr

import numpy as np
import pytest

import datagen
import oracle
from tests import exact_ref as ex

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
MAVPS = ("min1", "min2")


def dyadic(r, shape, scale=8, lo=-16, hi=17):
    """Values k/scale: sums of a few of them are exact in binary64."""
    return r.integers(lo, hi, size=shape).astype(np.float64) / scale


def read_golden(name):
    rows = {}
    blocks = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, val = line.split(":", 1)
            if key == "A" and rows:
                blocks.append(rows)
                rows = {}
            rows[key] = val.strip()
    if rows:
        blocks.append(rows)
    return blocks


# ---------------------------------------------------------------- scalar ops

@pytest.mark.parametrize("op", MAVPS)
def test_l1_inducing_property(op):
    """x (+) x = ||x||_1 for both MAVPs (§2.1, after Eq. (4))."""
    r = datagen.rng(1)
    for n in (1, 5, 64, 1000):
        x = dyadic(r, n)
        assert oracle.vecprod(op, x, x) == np.abs(x).sum()


def test_term_definitions_on_signed_grid():
    """Every sign/zero/tie combination against the exact definitions."""
    grid = [Fr(v, 4) for v in range(-8, 9)]
    for op in ("min1", "min2", "diamond", "dot"):
        for a in grid:
            for b in grid:
                assert oracle.term(op, float(a), float(b)) == float(ex.term(op, a, b))


def test_sign_rules_and_symmetry():
    r = datagen.rng(2)
    for _ in range(20):
        w, x = dyadic(r, 33), dyadic(r, 33)
        m1 = oracle.vecprod("min1", w, x)
        m2 = oracle.vecprod("min2", w, x)
        # symmetry of both products
        assert m1 == oracle.vecprod("min1", x, w)
        assert m2 == oracle.vecprod("min2", x, w)
        # odd in each argument (min1) / even under joint negation (min2)
        assert oracle.vecprod("min1", -w, x) == -m1
        assert oracle.vecprod("min2", -w, -x) == m2
        # min1 = min2(w, x) - min2(-w, x)
        assert m1 == m2 - oracle.vecprod("min2", -w, x)
        # bounds: |w (+) x| <= min(||w||_1, ||x||_1); min2 >= 0 (§3.2)
        assert abs(m1) <= min(np.abs(w).sum(), np.abs(x).sum())
        assert m2 >= 0.0
        # on non-negative vectors the two products agree
        assert oracle.vecprod("min1", abs(w), abs(x)) == oracle.vecprod("min2", abs(w), abs(x))
        # positive homogeneity (c w) (+) (c x) = c (w (+) x) for c = 2^k
        assert oracle.vecprod("min1", 4 * w, 4 * x) == 4 * m1


def test_permutation_equivariance():
    """(P A P^T) (+) (P w) = P (A (+) w)."""
    r = datagen.rng(3)
    A, w = dyadic(r, (40, 40)), dyadic(r, 40)
    p = r.permutation(40)
    for op in MAVPS:
        y = oracle.matvec(op, A, w)
        yp = oracle.matvec(op, A[np.ix_(p, p)], w[p])
        assert np.array_equal(yp, y[p])


# ----------------------------------------------------- MAPI iteration (Alg. 1)

def test_hand_worked_golden_example():
    blk = read_golden("hand_min1_min2_3x3.txt")[0]
    A = ex.parse_matrix(blk["A"])
    w0 = ex.parse_fraction_row(blk["w0"])
    Af = np.array([[float(v) for v in row] for row in A])
    w0f = np.array([float(v) for v in w0])
    # the exact reference reproduces the hand derivation ...
    assert ex.mapi_raw("min1", A, w0, 2) == [ex.parse_fraction_row(blk["min1 w1"]),
                                           ex.parse_fraction_row(blk["min1 w2"])]
    assert ex.mapi_raw("min2", A, w0, 1)[0] == ex.parse_fraction_row(blk["min2 w1"])
    # ... and so does the oracle
    for op, T, key in (("min1", 1, "min1 w1"), ("min1", 2, "min1 w2"), ("min2", 1, "min2 w1")):
        st, w, it, _ = oracle.mapi(op, Af, w0f, T, raw_start=True)
        assert st == oracle.OK and it == T
        want = np.array([float(v) for v in ex.parse_fraction_row(blk[key])])
        np.testing.assert_allclose(w, want, rtol=1e-15, atol=1e-16)


@pytest.mark.parametrize("n", [3, 4])
@pytest.mark.parametrize("op", ["min1", "min2", "diamond"])
def test_brute_force_rational(n, op):
    """Oracle MAPI vs exact rational arithmetic on small grid matrices, T=1..5."""
    count = 40
    for s in range(count):
        Ai = datagen.small_grid_matrix(n, seed=100 * n + s)
        w0i = datagen.small_grid_matrix(n, seed=9000 + 100 * n + s)[0]
        if not np.any(w0i):
            continue
        A = [[Fr(int(v)) for v in row] for row in Ai]
        w0 = [Fr(int(v), 4) for v in w0i]
        try:
            hist = ex.mapi_raw(op, A, w0, 5)
        except ZeroDivisionError:
            st, *_ = oracle.mapi(op, Ai.astype(float), w0i / 4.0, 5, raw_start=True)
            assert st == oracle.EZERONORM
            continue
        for T in range(1, 6):
            st, w, it, _ = oracle.mapi(op, Ai.astype(float), w0i / 4.0, T, raw_start=True)
            assert st == oracle.OK and it == T
            want = np.array([float(v) for v in hist[T - 1]])
            np.testing.assert_allclose(w, want, rtol=1e-13, atol=1e-15)


def test_iterates_have_unit_l1_norm():
    """||w_t||_1 = 1 after every step (§2.2, below Alg. 1)."""
    A = datagen.symmetric_gaussian(64, seed=5)
    w0 = datagen.start_vector(64, seed=5).astype(np.float64)
    for op in MAVPS:
        for T in (1, 2, 7, 30):
            st, w, it, _ = oracle.mapi(op, A, w0, T)
            assert st == oracle.OK and it == T
            assert abs(np.abs(w).sum() - 1.0) < 1e-14


def test_start_vector_is_l2_normalised():
    """Alg. 1 step 1: ||w0|| = 1 (Euclidean); scaling w0 changes nothing."""
    A = datagen.symmetric_gaussian(16, seed=6)
    w0 = datagen.start_vector(16, seed=6).astype(np.float64)
    _, a, _, _ = oracle.mapi("min1", A, w0, 3)
    _, b, _, _ = oracle.mapi("min1", A, 8.0 * w0, 3)
    _, c, _, _ = oracle.mapi("min1", A, w0 / np.linalg.norm(w0), 3, raw_start=True)
    np.testing.assert_array_equal(a, b)
    np.testing.assert_allclose(a, c, rtol=1e-14, atol=1e-16)


@pytest.mark.parametrize("blk", read_golden("prop1_diamond.txt"))
def test_proposition1_diamond_two_step_fixed_point(blk):
    """Proposition 1 (§2.2) with the limits stated in the golden file."""
    A = np.array([[float(v) for v in row] for row in ex.parse_matrix(blk["A"])])
    limit = np.array([float(v) for v in ex.parse_fraction_row(blk["limit"])])
    n = A.shape[0]
    w0 = np.linspace(0.3, 1.7, n)
    for raw in (True, False):
        st, w2, it, _ = oracle.mapi("diamond", A, w0, 2, raw_start=raw)
        assert st == oracle.OK and it == 2
        np.testing.assert_allclose(w2, limit, rtol=1e-14)
    # the first iterate follows the proof: (||a_i|| + ||w0||) / sum_j (...)
    st, w1, _, _ = oracle.mapi("diamond", A, w0, 1, raw_start=True)
    rows = np.abs(A).sum(1) + np.abs(w0).sum()
    np.testing.assert_allclose(w1, rows / rows.sum(), rtol=1e-14)


def test_proposition1_random_positive():
    r = datagen.rng(7)
    for n in (5, 50, 300):
        A = r.uniform(0.01, 3.0, size=(n, n))
        w0 = r.uniform(0.01, 1.0, size=n)
        st, w, _, _ = oracle.mapi("diamond", A, w0, 2)
        lim = 1.0 + A.sum(1)
        np.testing.assert_allclose(w, lim / lim.sum(), rtol=1e-12)


def test_regime_reduction_to_sign_matrix_power_iteration():
    """If every |a_ij| >= 1, then |w_j| <= 1 keeps min(|a|,|w|) = |w|, so
    A (.) w = sign(A) w and MAPI is l1-normalised power iteration on sign(A):
    w_T = sign(A)^T w_0 / ||.||_1, converging to eigh(sign(A))'s top vector."""
    r = datagen.rng(8)
    n = 48
    u = r.choice([-1.0, 1.0], size=n)
    S = np.outer(u, u) * np.where(r.random((n, n)) < 0.08, -1.0, 1.0)
    S = np.triu(S) + np.triu(S, 1).T
    A = S * r.uniform(1.0, 3.0, size=(n, n))
    A = np.triu(A) + np.triu(A, 1).T
    w0 = r.uniform(-1, 1, size=n)
    w0n = w0 / np.linalg.norm(w0)
    for T in (1, 3, 10):
        st, w, _, _ = oracle.mapi("min1", A, w0, T)
        v = np.linalg.matrix_power(np.sign(A), T) @ w0n
        np.testing.assert_allclose(w, v / np.abs(v).sum(), rtol=1e-10, atol=1e-13)
    st, w, _, _ = oracle.mapi("min1", A, w0, 300)
    evals, evecs = np.linalg.eigh(np.sign(A))
    assert evals[-1] > abs(evals[0])
    top = evecs[:, -1] / np.abs(evecs[:, -1]).sum()
    top *= np.sign(top @ w)
    np.testing.assert_allclose(w, top, atol=1e-10)


def test_rpi_closed_form_and_dominant_eigenvector():
    """op = dot is Eq. (1): w_T = A^T w_0 / ||.||_2; converges to the dominant
    eigenvector (numpy eigh) when there is a gap."""
    A = datagen.symmetric_gaussian(32, seed=9)
    w0 = datagen.start_vector(32, seed=9).astype(np.float64)
    for T in (1, 4, 9):
        st, w, _, _ = oracle.mapi("dot", A, w0, T)
        v = np.linalg.matrix_power(A, T) @ (w0 / np.linalg.norm(w0))
        np.testing.assert_allclose(w, v / np.linalg.norm(v), rtol=1e-9, atol=1e-12)
    r = datagen.rng(10)
    q, _ = np.linalg.qr(r.standard_normal((40, 40)))
    lam = np.concatenate([[3.0], np.linspace(1.0, -1.5, 39)])
    B = (q * lam) @ q.T
    st, w, _, _ = oracle.mapi("dot", B, r.uniform(-1, 1, 40), 200)
    top = q[:, 0] * np.sign(q[:, 0] @ w)
    np.testing.assert_allclose(w, top, atol=1e-9)


def test_zero_norm_status():
    """A = 0 gives a zero l1 norm (the paper is silent; the oracle reports it)."""
    st, w, it, _ = oracle.mapi("min1", np.zeros((4, 4)), np.ones(4), 3)
    assert st == oracle.EZERONORM and it == 0
    # min2 with every sign mismatched: all terms vanish
    A = -np.ones((3, 3))
    st, *_ = oracle.mapi("min2", A, np.ones(3), 1)
    assert st == oracle.EZERONORM


def test_tolerance_stops_early():
    A = np.abs(datagen.symmetric_gaussian(20, seed=11)) + 0.5
    st, w, it, dl = oracle.mapi("min1", A, np.ones(20), 500, tol=1e-12)
    assert st == oracle.OK and it < 500 and dl < 1e-12


# ------------------------------------------------------ min-covariance, Eq. (5)

def test_mincov_definition_and_invariants():
    r = datagen.rng(12)
    X = dyadic(r, (7, 11))
    for op in MAVPS + ("dot",):
        Cm = oracle.mincov(op, X, 11.0)
        np.testing.assert_array_equal(Cm, Cm.T)
        Xf = [[Fr(float(v)) for v in row] for row in X]
        want = ex.mincov(op, Xf, 11)
        np.testing.assert_allclose(Cm, np.array([[float(v) for v in row] for row in want]),
                                   rtol=1e-15, atol=1e-15)
    # diagonal = ||x^(p)||_1 / N (l1-inducing property)
    Cm = oracle.mincov("min1", X, 11.0)
    np.testing.assert_allclose(np.diag(Cm), np.abs(X).sum(1) / 11.0, rtol=1e-15)
    # op = dot reduces to the sample covariance of Eq. (2)
    Xg = r.standard_normal((9, 30))
    np.testing.assert_allclose(oracle.mincov("dot", Xg, 30.0), Xg @ Xg.T / 30.0, rtol=1e-12)


def test_mincov_matches_matrix_extension():
    """(W^T (+) X)_ij = w_i^T (+) x_j (§2.1): C equals it for W = X^T."""
    r = datagen.rng(13)
    X = r.standard_normal((6, 25))
    Cm = oracle.mincov("min1", X, 1.0)
    for i in range(6):
        for j in range(6):
            assert Cm[i, j] == oracle.vecprod("min1", X[i], X[j])


# ------------------------------------------------------------ deflation

def prefix_form(op, w, y):
    """(P y)_i for P = w (+) w^T via sorting by |w|:
    min1: s_i [sum_{c_j<=c_i} c_j z_j + c_i sum_{c_j>c_i} z_j], z = s*y;
    min2 = (min1 + the same with all signs +1) / 2."""
    c, s = np.abs(w), np.sign(w)

    def form(sv):
        z = sv * y
        order = np.argsort(c, kind="stable")
        out = np.empty_like(y)
        for i in range(len(w)):
            le = c <= c[i]
            out[i] = sv[i] * ((c[le] * z[le]).sum() + c[i] * z[~le].sum())
        return out
    if op == "min1":
        return form(s)
    return 0.5 * (form(s) + form(np.abs(s)))


@pytest.mark.parametrize("op", MAVPS)
def test_deflation_matches_prefix_form(op):
    r = datagen.rng(14)
    D = 24
    X = r.standard_normal((D, 60))
    Cm = oracle.mincov(op, X, 60.0)
    W = r.standard_normal((D, 3))
    W /= np.linalg.norm(W, axis=0)
    Ck = oracle.deflate(op, Cm, W)
    # the outer products take each component at unit l1 norm
    Wt = W / np.abs(W).sum(axis=0)
    want = Cm.copy()
    for m in range(3):
        for col in range(D):
            want[:, col] -= prefix_form(op, Wt[:, m], Cm[:, col])
    np.testing.assert_allclose(Ck, want, rtol=1e-12, atol=1e-12)
    y = r.standard_normal(D)
    yk = oracle.deflate_vec(op, y, W)
    want_y = y - sum(prefix_form(op, Wt[:, m], y) for m in range(3))
    np.testing.assert_allclose(yk, want_y, rtol=1e-12, atol=1e-12)
    # no earlier components: nothing to deflate
    np.testing.assert_array_equal(oracle.deflate(op, Cm, np.zeros((D, 0))), Cm)


@pytest.mark.parametrize("op", ["min1", "min2"])
def test_min_deflation_of_equal_magnitudes_is_the_projection(op):
    """A component of equal magnitudes (min2: equal signs too) gives, at unit
    l1 norm, the outer product u u^T exactly, so the deflation of Alg. 2
    step 6 is the projection deflation of §1 for it."""
    r = datagen.rng(23)
    D = 16
    s = np.where(r.random(D) < 0.5, -1.0, 1.0) if op == "min1" else np.ones(D)
    u = s / np.sqrt(D)
    Cm = oracle.mincov(op, r.standard_normal((D, 40)), 40.0)
    np.testing.assert_allclose(oracle.deflate(op, Cm, u[:, None]),
                               Cm - np.outer(u, u) @ Cm, rtol=1e-13, atol=1e-13)
    y = r.standard_normal(D)
    np.testing.assert_allclose(oracle.deflate_vec(op, y, u[:, None]), y - u * (u @ y),
                               rtol=1e-13, atol=1e-13)


def test_min1_pca_components_follow_the_spikes():
    """Under the unit-l1 outer products, min1 PCA with deflation finds the
    spiked directions one after another (at unit l2 norm every component
    after the first falls back onto the first spike)."""
    D, N = 96, 6000
    X = datagen.spiked_pca_data(D, N, seed=24, spikes=(60.0, 40.0, 25.0),
                                outlier_frac=0.0).astype(np.float64)
    r = datagen.rng(24)
    U, _ = np.linalg.qr(r.standard_normal((D, 3)))
    W0 = datagen.rng(25).uniform(-1, 1, size=(D, 3))
    st, P, _ = oracle.pca_topk("mincov", "min1", X, 3, 60, float(N), W0)
    assert st == oracle.OK
    ov = np.abs(U.T @ P)
    assert list(ov.argmax(axis=0)) == [0, 1, 2]
    assert ov.max(axis=0).min() > 0.8


def test_dot_deflation_is_projection_and_exposes_second_eigenvector():
    """§1: power iteration on (I - p_1 p_1^T) C yields the second eigenvector."""
    r = datagen.rng(15)
    q, _ = np.linalg.qr(r.standard_normal((30, 30)))
    lam = np.concatenate([[5.0, 3.0], np.linspace(1.0, 0.1, 28)])
    Cm = (q * lam) @ q.T
    Ck = oracle.deflate("dot", Cm, q[:, :1])
    np.testing.assert_allclose(Ck, Cm - np.outer(q[:, 0], q[:, 0]) @ Cm, atol=1e-12)
    st, w, _, _ = oracle.mapi("dot", Ck, r.uniform(-1, 1, 30), 300)
    np.testing.assert_allclose(abs(w @ q[:, 1]), 1.0, atol=1e-10)


def test_pca_dot_mincov_recovers_eigenvectors():
    r = datagen.rng(16)
    D, N = 12, 4000
    X = datagen.spiked_pca_data(D, N, seed=16, spikes=(40.0, 15.0, 5.0),
                                outlier_frac=0.0).astype(np.float64)
    W0 = r.uniform(-1, 1, size=(D, 3))
    st, P, its = oracle.pca_topk("mincov", "dot", X, 3, 400, float(N), W0)
    assert st == oracle.OK and list(its) == [400] * 3
    evals, evecs = np.linalg.eigh(X @ X.T / N)
    for c in range(3):
        assert abs(P[:, c] @ evecs[:, -1 - c]) > 1 - 1e-8
    # the pair mode with dot is the same power iteration without forming C
    st, P2, _ = oracle.pca_topk("pair", "dot", X, 3, 400, float(N), W0)
    for c in range(3):
        assert abs(P2[:, c] @ P[:, c]) > 1 - 1e-8


# ------------------------------------------------- reconstruction (Alg. 2)

def test_reconstruct_dot_is_the_orthogonal_projection():
    r = datagen.rng(26)
    D, N, k = 40, 6, 3
    W, _ = np.linalg.qr(r.standard_normal((D, k)))
    V = r.standard_normal((D, N))
    m = r.standard_normal(D)
    want = m[:, None] + W @ (W.T @ (V - m[:, None]))
    np.testing.assert_allclose(oracle.reconstruct("dot", W, V, m), want, rtol=1e-12,
                               atol=1e-12)
    # a vector in the span comes back unchanged
    V2 = m[:, None] + W @ r.standard_normal((k, N))
    np.testing.assert_allclose(oracle.reconstruct("dot", W, V2, m), V2, rtol=1e-12,
                               atol=1e-12)


def test_reconstruct_min1_of_equal_magnitude_components_is_a_projection():
    """Hadamard columns (equal magnitudes, orthogonal): each outer product at
    unit l1 norm is u u^T, so step 8 projects onto their span."""
    from scipy.linalg import hadamard
    r = datagen.rng(27)
    D = 16
    H = hadamard(D).astype(np.float64)[:, [1, 4, 7]] * r.uniform(0.5, 2.0, 3)
    U = H / np.linalg.norm(H, axis=0)
    V = r.standard_normal((D, 5))
    m = r.standard_normal(D)
    want = m[:, None] + U @ (U.T @ (V - m[:, None]))
    np.testing.assert_allclose(oracle.reconstruct("min1", H, V, m), want, rtol=1e-12,
                               atol=1e-12)


@pytest.mark.parametrize("op", MAVPS)
def test_reconstruct_matches_prefix_form(op):
    r = datagen.rng(28)
    D, N = 30, 4
    W = r.standard_normal((D, 2))
    V = r.uniform(0, 1, (D, N))
    m = V.mean(axis=1)
    Wt = W / np.abs(W).sum(axis=0)
    want = np.stack([m + sum(prefix_form(op, Wt[:, c], V[:, i] - m) for c in range(2))
                     for i in range(N)], axis=1)
    np.testing.assert_allclose(oracle.reconstruct(op, W, V, m), want, rtol=1e-12,
                               atol=1e-12)


def test_image_reconstruct_dot_full_rank_returns_the_images():
    """With k = N - 1 converged RPI components the centred images lie in
    their span, so step 8 returns every image (and m is the plain mean)."""
    r = datagen.rng(29)
    N, P = 4, 48
    base = r.uniform(0.2, 0.8, P)
    imgs = base + 0.3 * r.standard_normal((N, P)) * np.array([[3.0], [2.0], [1.2], [0.5]])
    W0 = r.uniform(-1, 1, (P, N - 1))
    st, W, R, its = oracle.image_reconstruct("dot", imgs, N - 1, 3000, W0, tol=1e-15)
    assert st == oracle.OK
    np.testing.assert_allclose(R, imgs, rtol=0, atol=1e-8)
    np.testing.assert_allclose(W.T @ W, np.eye(N - 1), atol=1e-8)


def test_image_reconstruct_of_identical_images_has_nothing_to_find():
    # dyadic pixels and N = 4: the mean is exact, so V - m is exactly zero
    imgs = np.tile(datagen.rng(30).integers(0, 9, 20) / 8.0, (4, 1))
    st, _, R, _ = oracle.image_reconstruct("min2", imgs, 1, 10, np.ones((20, 1)))
    assert st == oracle.EZERONORM and R is None


# ------------------------------------------------------------ pair step

@pytest.mark.parametrize("op", MAVPS)
def test_pair_step_brute_force(op):
    r = datagen.rng(17)
    X = dyadic(r, (3, 4))
    w = dyadic(r, 3)
    want = ex.pair_step(op, [[Fr(float(v)) for v in row] for row in X],
                        [Fr(float(v)) for v in w], 4)
    np.testing.assert_allclose(oracle.pair_step(op, X, w, 4.0),
                               [float(v) for v in want], rtol=1e-15, atol=1e-15)
    # N = 1 by hand: y_d = term(x_d, x (+) w)
    x = X[:, :1]
    t = sum(ex.term(op, Fr(float(a)), Fr(float(b))) for a, b in zip(x[:, 0], w))
    hand = [float(ex.term(op, Fr(float(a)), t)) for a in x[:, 0]]
    np.testing.assert_allclose(oracle.pair_step(op, x, w, 1.0), hand, rtol=1e-15)


# ------------------------------------------------------------ PageRank

def test_google_matrix_definition():
    # 3 nodes: 0 -> {1, 2}, 1 -> {2}, 2 dangling
    indptr, indices = [0, 2, 3, 3], [1, 2, 2]
    a = 0.85
    G = oracle.google_matrix(3, indptr, indices, a)
    H = np.array([[0, 0, 1 / 3], [0.5, 0, 1 / 3], [0.5, 1, 1 / 3]])
    np.testing.assert_allclose(G, a * H + (1 - a) / 3, rtol=1e-15)
    np.testing.assert_allclose(G.sum(0), 1.0, rtol=1e-15)


def test_rpi_pagerank_matches_linear_solve():
    """RPI on G reaches pi = (1 - a)/n (I - a H)^{-1} 1 (textbook identity)."""
    n = 200
    indptr, indices = datagen.barabasi_albert_digraph(n, m=3, seed=1)
    a = 0.85
    G = oracle.google_matrix(n, indptr, indices, a)
    H = (G - (1 - a) / n) / a
    pi = np.linalg.solve(np.eye(n) - a * H, np.full(n, (1 - a) / n))
    st, w, _, _ = oracle.pagerank("dot", n, indptr, indices,
                                  datagen.start_vector(n, 1, 0.0, 1.0), 300, G=G)
    np.testing.assert_allclose(w, pi / np.linalg.norm(pi), atol=1e-12)


def test_mapi_pagerank_sparse_reformulation():
    """For w >= 0, (G (+) w)_i = sum_j min(G_ij, w_j); G takes only the values
    tau, tau + a/d_j (links) and 1/n (dangling), so the row sum splits into a
    dense part and a correction over in-links:
    sum_j min(tau, w_j) + sum_{j->i} [min(tau + a/d_j, w_j) - min(tau, w_j)]
    + sum_{dangling j} [min(1/n, w_j) - min(tau, w_j)]."""
    n = 150
    indptr, indices = datagen.barabasi_albert_digraph(n, m=4, seed=2)
    a = 0.85
    tau = (1 - a) / n
    G = oracle.google_matrix(n, indptr, indices, a)
    w = datagen.start_vector(n, 2, 0.0, 1.0).astype(np.float64)
    w /= w.sum() * 30
    y = oracle.matvec("min1", G, w)
    assert np.array_equal(y, oracle.matvec("min2", G, w))
    base = np.minimum(tau, w).sum()
    want = np.full(n, base)
    for j in range(n):
        tg = indices[indptr[j]:indptr[j + 1]]
        if len(tg) == 0:
            want += np.minimum(1.0 / n, w[j]) - np.minimum(tau, w[j])
        else:
            want[tg] += np.minimum(tau + a / len(tg), w[j]) - np.minimum(tau, w[j])
    np.testing.assert_allclose(y, want, rtol=1e-12)
    st, v, _, _ = oracle.pagerank("min1", n, indptr, indices, w, 30, G=G)
    assert st == oracle.OK and np.all(v >= 0) and abs(np.linalg.norm(v) - 1) < 1e-14


# ------------------------------------------------------------ storage formats

def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    r = datagen.rng(18)
    x = np.concatenate([r.standard_normal(5000) * 10.0 ** r.integers(-30, 30, 5000),
                        # exact ties between two bf16 neighbours
                        (np.arange(1, 200, dtype=np.float64) * 2 + 1) * 2.0 ** -8,
                        [0.0, -0.0, 1e-40, -3e-39]]).astype(np.float32)
    want = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(oracle.round_bf16(x.astype(np.float64)), want)


def test_e4m3_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    if not hasattr(torch, "float8_e4m3fn"):
        pytest.skip("torch without float8")
    r = datagen.rng(19)
    x = np.concatenate([r.uniform(-448, 448, 4000), r.standard_normal(4000) * 0.01,
                        np.arange(-64, 65) * 2.0 ** -10, [448.0, -448.0, 0.0]])
    x = x.astype(np.float32)
    want = torch.from_numpy(x).to(torch.float8_e4m3fn).to(torch.float64).numpy()
    np.testing.assert_array_equal(oracle.round_e4m3(x.astype(np.float64)), want)
    # saturation beyond the largest finite value
    assert oracle.round_e4m3(np.array([1000.0, -470.0])).tolist() == [448.0, -448.0]


def test_fp8_row_scale_is_smallest_power_of_two():
    r = datagen.rng(20)
    A = (r.standard_normal((30, 50)) * 10.0 ** r.integers(-6, 4, (30, 1))).astype(np.float32)
    A[3] = 0.0
    deq, k = oracle.quant_fp8_rows(A)
    for i in range(30):
        mx = np.abs(A[i].astype(np.float64)).max()
        if mx == 0:
            assert k[i] == 0 and not deq[i].any()
            continue
        assert mx <= 448.0 * 2.0 ** k[i] and mx > 448.0 * 2.0 ** (k[i] - 1)
        np.testing.assert_array_equal(deq[i], oracle.round_e4m3(A[i] / 2.0 ** k[i]) * 2.0 ** k[i])


def test_integer_scale_and_quantisation():
    r = datagen.rng(21)
    A = r.uniform(-0.9, 0.9, size=(20, 20)).astype(np.float32)
    for bits, qmax in ((16, 32767), (8, 127)):
        q = oracle.int_scale(A, bits)
        mx = np.abs(A.astype(np.float64)).max()
        assert mx * 2.0 ** q <= qmax < mx * 2.0 ** (q + 1)
        Aq = oracle.quant_int(A, q)
        np.testing.assert_array_equal(Aq, np.rint(A.astype(np.float64) * 2.0 ** q).astype(np.int64))
        assert np.abs(Aq).max() <= qmax
    with pytest.raises(ValueError):
        oracle.int_scale(np.full((2, 2), 1e6, np.float32), 16)


@pytest.mark.parametrize("op", MAVPS)
def test_integer_mapi_matches_exact_integers(op):
    r = datagen.rng(22)
    for n, q in ((5, 9), (17, 12), (33, 15)):
        A = r.uniform(-1, 1, size=(n, n)).astype(np.float32) * 0.9
        w0 = r.uniform(-1, 1, size=n).astype(np.float32)
        Aq = oracle.quant_int(A, q)
        x0 = [int(v) for v in np.rint(w0.astype(np.float64) * 2.0 ** q)]
        hist = ex.mapi_int(op, [[int(v) for v in row] for row in Aq], q, x0, 6)
        for T in (1, 3, 6):
            st, w, it, _ = oracle.mapi_int(op, Aq, q, w0, T)
            assert st == oracle.OK and it == T
            assert w.tolist() == hist[T - 1]


def test_integer_mapi_approximates_float_mapi():
    """With a fine fixed-point grid the integer iteration tracks the float one."""
    A = (np.abs(datagen.symmetric_gaussian(24, seed=23)) * 0.1).astype(np.float32)
    w0 = np.abs(datagen.start_vector(24, 23))
    q = 20
    Aq = oracle.quant_int(A, q)
    st, wq, _, _ = oracle.mapi_int("min1", Aq, q, w0, 5)
    x0 = np.rint(w0.astype(np.float64) * 2.0 ** q)
    st2, wf, _, _ = oracle.mapi("min1", Aq / 2.0 ** q, x0 / np.abs(x0).sum(), 5, raw_start=True)
    np.testing.assert_allclose(wq / 2.0 ** q, wf, atol=24 * 2.0 ** -q)


def _graph_with_duplicates(n, seed):
    """Out-link CSR with repeated links, dangling nodes and self-links."""
    r = datagen.rng(seed)
    ip, ix = [0], []
    for j in range(n):
        d = 0 if j % 5 == 0 else int(r.integers(1, 7))
        ix.extend(int(v) for v in r.integers(0, n, size=d))
        if d and j % 3 == 0:
            ix.append(ix[-1])            # a repeated link j -> i
        ip.append(len(ix))
    return np.asarray(ip, np.int32), np.asarray(ix, np.int32)


@pytest.mark.parametrize("op", ["min1", "min2", "dot"])
@pytest.mark.parametrize("round32", [False, True])
def test_sparse_pagerank_equals_dense_definition(op, round32):
    """The O(E + n) form of G (+) w is the Eq. (11) matrix product: same
    iterates as Alg. 1 on the dense G (FP64, or G's FP32 values), up to the
    order of FP64 additions."""
    for n, seed in ((1, 30), (7, 31), (60, 32), (400, 33)):
        ip, ix = _graph_with_duplicates(n, seed)
        G = oracle.google_matrix(n, ip, ix, 0.85)
        if round32:
            G = G.astype(np.float32).astype(np.float64)
        w0 = datagen.start_vector(n, seed=seed, low=0.0, high=1.0).astype(np.float64)
        st, want, it, dl = oracle.mapi(op, G, w0, 15, final_l2=True)
        st2, got, it2, dl2 = oracle.pagerank_sparse(op, n, ip, ix, w0, 15, round32=round32)
        assert (st, it) == (st2, it2)
        np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-15)
        assert abs(dl - dl2) <= 1e-12


def test_sparse_pagerank_stop_rule():
    ip, ix = datagen.barabasi_albert_digraph(200, m=4, seed=34)
    w0 = datagen.start_vector(200, seed=34, low=0.0, high=1.0)
    G = oracle.google_matrix(200, ip, ix, 0.85).astype(np.float32).astype(np.float64)
    st, want, it, dl = oracle.mapi("min1", G, w0, 500, tol=1e-9, final_l2=True)
    st2, got, it2, dl2 = oracle.pagerank_sparse("min1", 200, ip, ix, w0, 500, tol=1e-9)
    assert st == st2 == oracle.OK and it == it2 < 500 and dl2 < 1e-9
    np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-15)


@pytest.mark.parametrize("op", ["min1", "min2", "dot"])
def test_minibatch_momentum_full_batch_without_momentum_is_alg1(op):
    """Alg. 3 with beta = 0 and every sample in every batch is Alg. 1 on the
    min-covariance (1/N) sum_k x_k (+) x_k^T of Eq. (5)."""
    N, D, T = 50, 6, 12
    X = datagen.stochastic_pca_data(N, D, seed=70).astype(np.float64)
    batch = np.tile(np.arange(N, dtype=np.int32), (T, 1))
    w0 = datagen.start_vector(D, seed=71).astype(np.float64)
    st, got = oracle.minibatch_momentum(op, X, batch, 0.0, w0)
    C = oracle.mincov(op, X.T.copy(), float(N))
    st2, want, _, _ = oracle.mapi(op, C, w0, T, final_l2=True)
    assert st == st2 == oracle.OK
    np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-15)


def test_minibatch_momentum_dot_is_the_momentum_polynomial():
    """With op = dot and full batches, w_t is p_t(C) w_0 up to scale, where
    p_{t+1}(x) = x p_t(x) - beta p_{t-1}(x), p_0 = 1, p_{-1} = 0 (the
    recurrence of the momentum power method), evaluated on eigh(C)."""
    N, D, T, beta = 80, 7, 25, 0.2
    X = datagen.stochastic_pca_data(N, D, seed=72).astype(np.float64)
    batch = np.tile(np.arange(N, dtype=np.int32), (T, 1))
    w0 = datagen.start_vector(D, seed=73).astype(np.float64)
    st, got = oracle.minibatch_momentum("dot", X, batch, beta, w0)
    lam, Q = np.linalg.eigh(X.T @ X / N)
    p_prev, p = np.zeros(D), np.ones(D)
    for _ in range(T):
        p_prev, p = p, lam * p - beta * p_prev
    want = Q @ (p * (Q.T @ w0))
    want /= np.linalg.norm(want)
    assert st == oracle.OK
    np.testing.assert_allclose(got, want, rtol=1e-9, atol=1e-12)


def test_minibatch_sample_data_spectrum():
    X = datagen.stochastic_pca_data(2000, 10, seed=74).astype(np.float64)
    lam = np.sort(np.linalg.eigvalsh(X.T @ X))[::-1]
    np.testing.assert_allclose(lam, [1.0] + [0.9] * 9, rtol=1e-6)  # FP32 samples
