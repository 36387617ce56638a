"""The diagnostic entry points: the ALU roofline probe returns rates that
the hardware allows, the pair step's phase stamps count the steps that ran
and give non-negative phase times and per-cluster loop times, and the
stamping kernel gives the same bits as the plain one."""
import math

import numpy as np
import pytest

import datagen
import paper_2110_12065_gb300 as M
from tests.helpers import to_dev

pytestmark = pytest.mark.gpu


def test_alu_probe_rates_are_consistent(mapi_ctx):
    r = {m: M.mapi_alu_probe(mapi_ctx, m) for m in M.ALU_MIXES}
    assert all(v > 0 and math.isfinite(v) for v in r.values()), r
    # min/max issue at most 64 lanes per clock per SM; a term needs two
    assert r["fmnmx"] <= 64.5
    for m in ("min1_term_f32", "min1_term_bf16", "min1_term_bf16_x4"):
        assert r[m] <= r["fmnmx"] / 2 + 0.5, (m, r)
    # widening each BF16 operand costs issue slots; sharing it over four
    # vectors costs fewer
    assert r["min1_term_bf16"] <= r["min1_term_bf16_x4"] + 0.5
    assert r["min1_term_bf16_x4"] <= r["min1_term_f32"] + 0.5
    with pytest.raises(M.MapiError):
        M.mapi_alu_probe(mapi_ctx, 5)


def test_pair_phase_stamps_count_the_steps(mapi_ctx):
    D, N, k, T = 128, 4096, 2, 5
    X = datagen.spiked_pca_data(D, N, seed=81)
    W0 = to_dev(np.stack([datagen.start_vector(D, seed=810 + c) for c in range(k)]))
    mat = M.mapi_matrix_upload(mapi_ctx, to_dev(X), "f32")
    try:
        M.mapi_pair_phases(mapi_ctx, True)
        M.mapi_pca_topk(mapi_ctx, mat, k, "pair", "min1", T, float(N), W0)
        ph = M.mapi_pair_phases(mapi_ctx, False)
    finally:
        M.mapi_matrix_free(mapi_ctx, mat)
    assert ph["steps"] == k * T
    for name, v in ph.items():
        assert math.isfinite(v) and v >= 0.0, (name, v)
    assert ph["start_to_last_arrival"] >= ph["start_to_first_arrival"]
    # one loop time per streaming cluster, each positive and below the time
    # a whole step took (its CTAs' own clocks, not the step's first start)
    cl = M.mapi_pair_cluster_times(mapi_ctx)
    assert len(cl) >= 1
    step_us = sum(v for name, v in ph.items() if name != "steps")
    assert all(0.0 < v < step_us for v in cl), (cl, ph)
    # stamping off: nothing more is counted
    assert M.mapi_pair_phases(mapi_ctx, False)["steps"] == k * T


@pytest.mark.parametrize("st", ["f32", "bf16"])
def test_stamped_solve_gives_the_same_bits(mapi_ctx, st):
    # the stamping kernel is a separate instantiation of the same arithmetic
    D, N, k, T = 300, 20000, 3, 12
    X = datagen.spiked_pca_data(D, N, seed=82)
    W0 = to_dev(np.stack([datagen.start_vector(D, seed=820 + c) for c in range(k)]))
    mat = M.mapi_matrix_upload(mapi_ctx, to_dev(X), st)
    try:
        P0, it0 = M.mapi_pca_topk(mapi_ctx, mat, k, "pair", "min1", T, float(N), W0)
        M.mapi_pair_phases(mapi_ctx, True)
        P1, it1 = M.mapi_pca_topk(mapi_ctx, mat, k, "pair", "min1", T, float(N), W0)
        assert M.mapi_pair_phases(mapi_ctx, False)["steps"] == k * T
    finally:
        M.mapi_matrix_free(mapi_ctx, mat)
    assert list(it0) == list(it1)
    np.testing.assert_array_equal(P0.cpu().numpy(), P1.cpu().numpy())
