"""GPU tests of the serving loop (mapi_submit / mapi_poll / mapi_cancel):
every served result equals the same request solved alone through the
synchronous entry points, small cases equal the FP64 oracle, and admission,
cancellation and bad requests behave as documented."""
import time

import numpy as np
import pytest
import torch

import datagen
import oracle
import paper_2110_12065_gb300 as M
from tests.helpers import rel_l1, to_dev, to_host

pytestmark = pytest.mark.gpu

# the served and the synchronous path both compute in FP32 but sum in
# different orders (batched kernel vs the split GEMV), as in the batched tests
TOL32 = 1e-5


def wait(ctx, tickets, timeout=120.0):
    out, t0 = {}, time.time()
    while len(out) < len(tickets):
        for t in tickets:
            if t not in out:
                r = M.mapi_poll(ctx, t)
                if r is not None:
                    out[t] = r
        assert time.time() - t0 < timeout, "served requests did not finish"
        time.sleep(0.002)
    return out


def pca_case(D, N, k, seed):
    X = datagen.spiked_pca_data(D, N, seed=seed)
    W0 = np.stack([datagen.start_vector(D, seed=seed * 10 + c) for c in range(k)])
    return X, W0


def pr_case(n, seed):
    ip, ix = datagen.barabasi_albert_digraph(n, m=8, seed=seed)
    w0 = datagen.start_vector(n, seed=seed, low=0.0, high=1.0)
    return ip, ix, w0


def test_served_results_equal_the_same_requests_alone(mapi_ctx):
    reqs = []
    for (D, N, k, st, seed) in [(64, 1000, 3, "f32", 1), (200, 3000, 2, "bf16", 2),
                                (37, 515, 1, "f32", 3), (256, 2048, 4, "f32", 4)]:
        X, W0 = pca_case(D, N, k, seed)
        reqs.append(("pca", st, (X, W0, k)))
    for (n, st, seed) in [(300, "f32", 5), (1500, "bf16", 6), (1024, "f32", 7), (2500, "f32", 8)]:
        reqs.append(("pagerank", st, pr_case(n, seed)))
    tickets = []
    for kind, st, a in reqs:
        if kind == "pca":
            X, W0, k = a
            tickets.append(M.mapi_submit(mapi_ctx, "pca", W0, op="min1", storage=st,
                                         max_iters=60, X=X, k=k, cov_denom=X.shape[1]))
        else:
            ip, ix, w0 = a
            tickets.append(M.mapi_submit(mapi_ctx, "pagerank", w0, op="min1", storage=st,
                                         max_iters=40, indptr=ip, indices=ix, alpha=0.85))
    res = wait(mapi_ctx, tickets)
    for t, (kind, st, a) in zip(tickets, reqs):
        r = res[t]
        assert r["status"] == 0, r
        assert r["latency_ms"] >= r["run_ms"] >= 0.0 and r["queue_ms"] >= 0.0
        assert abs(r["latency_ms"] - r["queue_ms"] - r["run_ms"]) < 1.0
        if kind == "pca":
            X, W0, k = a
            Xm = M.mapi_matrix_upload(mapi_ctx, to_dev(X), st)
            try:
                P, its = M.mapi_pca_topk(mapi_ctx, Xm, k, "mincov", "min1", 60,
                                         X.shape[1], to_dev(W0))
            finally:
                M.mapi_matrix_free(mapi_ctx, Xm)
            assert r["iters"][:k] == its == [60] * k
            P = to_host(P)
            for c in range(k):
                assert rel_l1(r["out"][c], P[c]) <= TOL32, (c, rel_l1(r["out"][c], P[c]))
        else:
            ip, ix, w0 = a
            n = ip.shape[0] - 1
            want, it, _ = M.mapi_pagerank(mapi_ctx, to_dev(ip), to_dev(ix), n, to_dev(w0), 40,
                                          storage=st)
            assert r["iters"][0] == it == 40
            assert rel_l1(r["out"], to_host(want)) <= TOL32


def test_served_small_cases_equal_the_oracle(mapi_ctx):
    X, W0 = pca_case(48, 700, 2, 11)
    ip, ix, w0 = pr_case(400, 12)
    t1 = M.mapi_submit(mapi_ctx, "pca", W0, op="min1", storage="f32", max_iters=30, X=X, k=2,
                       cov_denom=700)
    t2 = M.mapi_submit(mapi_ctx, "pagerank", w0, op="min1", storage="f32", max_iters=30,
                       indptr=ip, indices=ix)
    res = wait(mapi_ctx, [t1, t2])
    st, P, its = oracle.pca_topk("mincov", "min1", X.astype(np.float64), 2, 30, 700.0,
                                 W0.T.astype(np.float64))
    assert st == 0 and list(its) == res[t1]["iters"][:2]
    for c in range(2):
        assert rel_l1(res[t1]["out"][c], P[:, c]) <= TOL32
    G = oracle.google_matrix(400, ip, ix, 0.85).astype(np.float32).astype(np.float64)
    st, want, oit, _ = oracle.mapi("min1", G, w0.astype(np.float64), 30, final_l2=True)
    assert res[t2]["iters"][0] == oit
    assert rel_l1(res[t2]["out"], want) <= TOL32


@pytest.mark.parametrize("n", [600, 2100])  # batched launch, whole-GPU solve
def test_stop_rule_and_convergence(mapi_ctx, n):
    ip, ix, w0 = pr_case(n, 13)
    t = M.mapi_submit(mapi_ctx, "pagerank", w0, op="min1", storage="f32", max_iters=1000,
                      tol_l1=1e-7, indptr=ip, indices=ix)
    r = wait(mapi_ctx, [t])[t]
    want, it, dl = M.mapi_pagerank(mapi_ctx, to_dev(ip), to_dev(ix), n, to_dev(w0), 1000,
                                   tol_l1=1e-7)
    assert r["status"] == 0 and r["last_delta"] < 1e-7
    assert r["iters"][0] < 1000 and abs(r["iters"][0] - it) <= 1
    # the result is l2-normalised even when the stop rule ends a round early
    assert abs(float(np.linalg.norm(r["out"].astype(np.float64))) - 1.0) < 1e-5
    assert rel_l1(r["out"], to_host(want)) <= 1e-5


def test_budget_rejects_what_can_never_fit():
    ctx = M.mapi_create(0, hbm_budget_bytes=1 << 20)
    try:
        ip, ix, w0 = pr_case(2000, 14)
        with pytest.raises(M.MapiError) as e:
            M.mapi_submit(ctx, "pagerank", w0, indptr=ip, indices=ix)
        assert e.value.name == "EBUDGET"
    finally:
        M.mapi_destroy(ctx)


def test_budget_serialises_and_cancel_drops_queued_and_running():
    # room for one n = 2048 FP32 request at a time
    ctx = M.mapi_create(0, hbm_budget_bytes=60 << 20)
    try:
        ip, ix, w0 = pr_case(2048, 15)
        long1 = M.mapi_submit(ctx, "pagerank", w0, storage="f32", max_iters=10 ** 7,
                              indptr=ip, indices=ix)
        long2 = M.mapi_submit(ctx, "pagerank", w0, storage="f32", max_iters=10 ** 7,
                              indptr=ip, indices=ix)
        time.sleep(0.3)
        assert M.mapi_poll(ctx, long1) is None and M.mapi_poll(ctx, long2) is None
        M.mapi_cancel(ctx, long2)  # still queued: budget holds only one
        r2 = wait(ctx, [long2])[long2]
        assert r2["status_name"] == "ECANCELLED" and r2["run_ms"] == 0.0
        M.mapi_cancel(ctx, long1)  # running: dropped at the end of a round
        r1 = wait(ctx, [long1])[long1]
        assert r1["status_name"] == "ECANCELLED" and r1["run_ms"] > 0.0
        # the loop goes on serving after the cancellations
        small = pr_case(300, 16)
        t = M.mapi_submit(ctx, "pagerank", small[2], storage="f32", max_iters=20,
                          indptr=small[0], indices=small[1])
        assert wait(ctx, [t])[t]["status"] == 0
    finally:
        M.mapi_destroy(ctx)


def test_one_slot_serves_requests_in_turn():
    ctx = M.mapi_create(0, max_slots=1)
    try:
        cases = [pr_case(n, 20 + n) for n in (100, 700, 64)]
        ts = [M.mapi_submit(ctx, "pagerank", w0, storage="f32", max_iters=30, indptr=ip,
                            indices=ix) for ip, ix, w0 in cases]
        res = wait(ctx, ts)
        for t, (ip, ix, w0) in zip(ts, cases):
            n = ip.shape[0] - 1
            want, _, _ = M.mapi_pagerank(ctx, to_dev(ip), to_dev(ix), n, to_dev(w0), 30)
            assert res[t]["status"] == 0
            assert rel_l1(res[t]["out"], to_host(want)) <= TOL32
        # in turn: the last request waited in the queue while the first ran
        assert res[ts[2]]["queue_ms"] >= 0.9 * res[ts[0]]["run_ms"]
    finally:
        M.mapi_destroy(ctx)


def test_bad_requests_and_tickets(mapi_ctx):
    ip, ix, w0 = pr_case(50, 17)
    X, W0 = pca_case(16, 64, 1, 18)
    bad = [dict(kind="pagerank", w0=w0, indptr=ip, indices=ix, storage="fp8"),
           dict(kind="pagerank", w0=w0, indptr=ip, indices=ix, max_iters=0),
           dict(kind="pagerank", w0=w0, indptr=ip, indices=np.where(ix == 3, 50, ix)),
           dict(kind="pca", w0=np.zeros((9, 16)), X=X, k=9),
           dict(kind="pca", w0=W0, X=X, k=1, cov_denom=0.0),
           dict(kind="pca", w0=W0, X=X, k=1, op="diamond")]
    for b in bad:
        with pytest.raises(M.MapiError) as e:
            M.mapi_submit(mapi_ctx, **b)
        assert e.value.name == "EINVAL"
    with pytest.raises(M.MapiError):
        M.mapi_poll(mapi_ctx, 10 ** 12)
    with pytest.raises(M.MapiError):
        M.mapi_cancel(mapi_ctx, 10 ** 12)
    # a reported ticket is forgotten
    t = M.mapi_submit(mapi_ctx, "pagerank", w0, storage="f32", max_iters=5, indptr=ip,
                      indices=ix)
    wait(mapi_ctx, [t])
    with pytest.raises(M.MapiError):
        M.mapi_poll(mapi_ctx, t)


def test_zero_norm_is_reported(mapi_ctx):
    # Alg. 1 step 1 cannot scale a zero start vector to unit norm
    ip, ix, w0 = pr_case(50, 21)
    t = M.mapi_submit(mapi_ctx, "pagerank", np.zeros(50, np.float32), storage="f32",
                      max_iters=5, indptr=ip, indices=ix)
    r = wait(mapi_ctx, [t])[t]
    assert r["status_name"] == "EZERONORM"
