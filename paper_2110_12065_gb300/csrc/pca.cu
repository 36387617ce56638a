// PCA by MAPI: min-covariance build (Eq. (5)), deflation (Alg. 2 step 6 with
// the sum form after Eq. (2)), the matrix-free pair step, and the top-k
// drivers for both modes.
#include <cuda.h>

#include <algorithm>
#include <cmath>
#include <cstring>

#include "device_common.cuh"

namespace mapi {

// ======================================================================
// K2: C = (1/denom) X (+) X^T.  128 x 128 output tiles (upper triangle of
// tiles only), split over the samples (blockIdx.y) so that every SM has
// work; 256 threads, 8 x 8 register micro-tiles; the sample range is swept in
// chunks of 16 through two shared-memory buffers (k-major, padded rows), the
// next chunk prefetched into registers while the current one is consumed.
// Each split writes its partial tile; k_mincov_reduce sums the splits in a
// fixed order, divides by denom and mirrors the tile.
// ======================================================================
constexpr int kMcT = 128, kMcK = 16, kMcPad = 4;

template <int ST>
struct McStage;
template <>
struct McStage<kF32> {  // 128 rows x 16 floats = 512 float4, 2 per thread
  float4 v[2];
  __device__ __forceinline__ void load(const uint8_t* X, int64_t row_bytes, int rows_pad,
                                       int64_t k_end, int r0, int64_t k0) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int idx = threadIdx.x + h * 256;
      const int r = idx >> 2, cc = (idx & 3) * 4;
      v[h] = make_float4(0.f, 0.f, 0.f, 0.f);
      if (r0 + r < rows_pad && k0 + cc < k_end)
        v[h] = __ldg(reinterpret_cast<const float4*>(X + (int64_t)(r0 + r) * row_bytes +
                                                     (k0 + cc) * 4));
    }
  }
  __device__ __forceinline__ void store(float (*S)[kMcT + kMcPad]) const {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int idx = threadIdx.x + h * 256;
      const int r = idx >> 2, cc = (idx & 3) * 4;
      S[cc + 0][r] = v[h].x;
      S[cc + 1][r] = v[h].y;
      S[cc + 2][r] = v[h].z;
      S[cc + 3][r] = v[h].w;
    }
  }
};
template <>
struct McStage<kBF16> {  // 128 rows x 16 bf16 = 256 chunks of 8, 1 per thread
  Chunk<kBF16> c;
  __device__ __forceinline__ void load(const uint8_t* X, int64_t row_bytes, int rows_pad,
                                       int64_t k_end, int r0, int64_t k0) {
    const int r = threadIdx.x >> 1, cc = (threadIdx.x & 1) * 8;
    c.raw = make_uint4(0, 0, 0, 0);
    if (r0 + r < rows_pad && k0 + cc < k_end)
      c.raw = __ldg(reinterpret_cast<const uint4*>(X + (int64_t)(r0 + r) * row_bytes +
                                                   (k0 + cc) * 2));
  }
  __device__ __forceinline__ void store(float (*S)[kMcT + kMcPad]) const {
    const int r = threadIdx.x >> 1, cc = (threadIdx.x & 1) * 8;
#pragma unroll
    for (int e = 0; e < 8; ++e) S[cc + e][r] = c.get(e);
  }
};

__device__ __forceinline__ void mc_tile_of(int b, int T, int& tp, int& tq) {
  tp = 0;
  while (b >= T - tp) {
    b -= T - tp;
    ++tp;
  }
  tq = tp + b;
}

template <int OP, int ST>
__global__ void __launch_bounds__(256, 2)
    k_mincov(const uint8_t* __restrict__ X, int64_t row_bytes, int rows_pad, int64_t ld,
             int D, int64_t kseg, float* __restrict__ part) {
  __shared__ __align__(16) float As[2][kMcK][kMcT + kMcPad];
  __shared__ __align__(16) float Bs[2][kMcK][kMcT + kMcPad];
  const int T = (D + kMcT - 1) / kMcT;
  int tp, tq;
  mc_tile_of(blockIdx.x, T, tp, tq);
  const int p0 = tp * kMcT, q0 = tq * kMcT;
  const int64_t k_beg = (int64_t)blockIdx.y * kseg;
  const int64_t k_end = min(ld, k_beg + kseg);
  const int ty = threadIdx.x >> 4, tx = threadIdx.x & 15;
  float acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;

  McStage<ST> na, nb;
  int buf = 0;
  if (k_beg < k_end) {
    na.load(X, row_bytes, rows_pad, k_end, p0, k_beg);
    nb.load(X, row_bytes, rows_pad, k_end, q0, k_beg);
    na.store(As[0]);
    nb.store(Bs[0]);
  }
  __syncthreads();
  for (int64_t k0 = k_beg; k0 < k_end; k0 += kMcK) {
    const bool more = k0 + kMcK < k_end;
    if (more) {  // prefetch the next chunk into registers
      na.load(X, row_bytes, rows_pad, k_end, p0, k0 + kMcK);
      nb.load(X, row_bytes, rows_pad, k_end, q0, k0 + kMcK);
    }
#pragma unroll 4
    for (int k = 0; k < kMcK; ++k) {
      const float4 a0 = *reinterpret_cast<const float4*>(&As[buf][k][ty * 8]);
      const float4 a1 = *reinterpret_cast<const float4*>(&As[buf][k][ty * 8 + 4]);
      const float4 b0 = *reinterpret_cast<const float4*>(&Bs[buf][k][tx * 8]);
      const float4 b1 = *reinterpret_cast<const float4*>(&Bs[buf][k][tx * 8 + 4]);
      const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const auto p = Op<OP>::prep(bv[j]);
#pragma unroll
        for (int i = 0; i < 8; ++i) acc[i][j] = Op<OP>::term(a[i], p, acc[i][j]);
      }
    }
    if (more) {
      na.store(As[buf ^ 1]);
      nb.store(Bs[buf ^ 1]);
    }
    __syncthreads();
    buf ^= 1;
  }
  // partial tile: part[split][tile][128][128]
  float* out = part + ((int64_t)blockIdx.y * gridDim.x + blockIdx.x) * kMcT * kMcT;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    float4* o = reinterpret_cast<float4*>(out + (ty * 8 + i) * kMcT + tx * 8);
    o[0] = make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]);
    o[1] = make_float4(acc[i][4], acc[i][5], acc[i][6], acc[i][7]);
  }
}

// Sum the splits of each tile in order, divide by denom, write C and its
// mirror.  The tile goes through shared memory in 32 x 32 pieces so that the
// mirror's rows are written whole.
__global__ void __launch_bounds__(256)
    k_mincov_reduce(const float* __restrict__ part, int ntiles, int nsplit, int D, float denom,
                    float* __restrict__ C, int64_t ldc) {
  __shared__ float piece[32][33];
  const int T = (D + kMcT - 1) / kMcT;
  int tp, tq;
  mc_tile_of(blockIdx.x, T, tp, tq);
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (int pi = 0; pi < kMcT; pi += 32)
    for (int pj = 0; pj < kMcT; pj += 32) {
      // rows pi.., columns pj.. of the tile: direct copy, kept for the mirror
      for (int rr = ty; rr < 32; rr += 8) {
        const int e = (pi + rr) * kMcT + pj + tx;
        float sum = 0.f;
        for (int k = 0; k < nsplit; ++k)
          sum += part[((int64_t)k * ntiles + blockIdx.x) * kMcT * kMcT + e];
        const float v = sum / denom;
        piece[rr][tx] = v;
        const int p = tp * kMcT + pi + rr, q = tq * kMcT + pj + tx;
        if (p < D && q < D) C[(int64_t)p * ldc + q] = v;
      }
      __syncthreads();
      if (tp != tq) {
        // mirror: row q of C gets column q - tq*kMcT of the piece
        for (int rr = ty; rr < 32; rr += 8) {
          const int q = tq * kMcT + pj + rr, p = tp * kMcT + pi + tx;
          if (p < D && q < D) C[(int64_t)q * ldc + p] = piece[tx][rr];
        }
      }
      __syncthreads();
    }
}

// Copy a finished component's step count and status out of the control
// block; a failure sets the sticky abort flag that skips later components
// (their step count is recorded as 0 and their status as OK).
__global__ void k_record(const IterCtl* ctl, int* iters, int* status, int* abort, int c) {
  const int st = ctl->v[0].status;
  if (st == MAPI_ECANCELLED) {
    iters[c] = 0;
    status[c] = MAPI_OK;
    return;
  }
  iters[c] = ctl->v[0].iters;
  status[c] = st;
  if (st != MAPI_OK) *abort = 1;
}

// ---------------------------------------------------------------- host side

mapi_status launch_mincov_raw(mapi_ctx* ctx, const mapi_mat* X, mapi_op op, float denom,
                              float* C, int64_t ldc, cudaStream_t s) {
  const int T = (X->rows + kMcT - 1) / kMcT;
  const int nt = T * (T + 1) / 2;
  const int64_t rb = X->ld * elem_bytes(X->storage);
  const uint8_t* x = (const uint8_t*)X->data;
  // split the samples until there are about 4 CTAs per SM (2 resident)
  int nsplit = 1;
  while (nt * nsplit < 4 * ctx->sm_count && X->ld / (nsplit * 2) >= 4 * kMcK) nsplit *= 2;
  const int64_t kseg = ((X->ld + nsplit - 1) / nsplit + kMcK - 1) / kMcK * kMcK;
  mapi_status st = ensure(ctx, ctx->mcpart, sizeof(float) * (size_t)nsplit * nt * kMcT * kMcT);
  if (st != MAPI_OK) return st;
  float* part = (float*)ctx->mcpart.p;
  const dim3 grid(nt, nsplit);
  cudaEvent_t ev = prof_begin(ctx, s);
#define MC(OPV, STV) \
  k_mincov<OPV, STV><<<grid, 256, 0, s>>>(x, rb, X->rows_pad, X->ld, X->rows, kseg, part)
  if (X->storage == MAPI_ST_F32) {
    if (op == MAPI_OP_MIN1) MC(MAPI_OP_MIN1, kF32);
    else if (op == MAPI_OP_MIN2) MC(MAPI_OP_MIN2, kF32);
    else MC(MAPI_OP_DOT, kF32);
  } else if (X->storage == MAPI_ST_BF16) {
    if (op == MAPI_OP_MIN1) MC(MAPI_OP_MIN1, kBF16);
    else if (op == MAPI_OP_MIN2) MC(MAPI_OP_MIN2, kBF16);
    else MC(MAPI_OP_DOT, kBF16);
  } else {
    return fail(ctx, MAPI_EINVAL, "min-covariance supports F32 and BF16 storage");
  }
#undef MC
  MAPI_CUDA_TRY(ctx, cudaGetLastError());
  prof_end(ctx, s, ev, MAPI_KC_MINCOV, (double)X->rows * X->cols * elem_bytes(X->storage),
           (double)X->rows * (X->rows + 1) / 2 * X->cols);
  count_launch(ctx);
  k_mincov_reduce<<<nt, 256, 0, s>>>(part, nt, nsplit, X->rows, denom, C, ldc);
  MAPI_CUDA_TRY(ctx, cudaGetLastError());
  count_launch(ctx);
  return MAPI_OK;
}

// Scratch of the min-covariance splits for X (the launcher grows it; callers
// that capture graphs size it first).
size_t mincov_scratch_bytes(const mapi_ctx* ctx, const mapi_mat* X) {
  const int T = (X->rows + kMcT - 1) / kMcT;
  const int nt = T * (T + 1) / 2;
  int nsplit = 1;
  while (nt * nsplit < 4 * ctx->sm_count && X->ld / (nsplit * 2) >= 4 * kMcK) nsplit *= 2;
  return sizeof(float) * (size_t)nsplit * nt * kMcT * kMcT;
}

namespace {

// Everything one PCA solve touches on the device, sized before capture.
struct PcaPlan {
  int D = 0, k = 0, mode = 0, iters = 0;
  mapi_op op = MAPI_OP_MIN1;
  double tol = 0, denom = 1;
  int64_t ldq = 0;
  int* rec = nullptr;    // [iters 64][status 64][abort]
  int* abort = nullptr;
  // min-covariance mode
  mapi_mat Cm, Ck;
  float* Q = nullptr;
  // pair mode
  PairPlan pl;
  int D_pad = 0;
  int64_t wst = 0;
  void* defl = nullptr;
};

mapi_status pca_enqueue(mapi_ctx* ctx, cudaStream_t s, const mapi_mat* X, const PcaPlan& p,
                        const float* w0, float* P_out) {
  mapi_status st = MAPI_OK;
  const int D = p.D, k = p.k;
  MAPI_CUDA_TRY(ctx, cudaMemsetAsync(p.rec, 0, sizeof(int) * 129, s));
  if (p.mode == MAPI_PCA_MINCOV) {
    const size_t bytes = sizeof(float) * p.Cm.rows_pad * p.Cm.ld;
    MAPI_CUDA_TRY(ctx, cudaMemsetAsync(p.Cm.data, 0, bytes, s));
    MAPI_CUDA_TRY(ctx, cudaMemsetAsync(p.Ck.data, 0, bytes, s));
    if ((st = launch_mincov_raw(ctx, X, p.op, (float)p.denom, (float*)p.Cm.data, p.Cm.ld, s)) !=
        MAPI_OK)
      return st;
    for (int c = 0; c < k; ++c) {
      const mapi_mat* A = &p.Cm;
      if (c > 0) {
        // Alg. 2 step 6: C_c = C - sum_{m<c} P_m C (p.Q holds the transposed product)
        if ((st = launch_deflate_mincov(ctx, p.op, P_out, D, c, D, (const float*)p.Cm.data,
                                        p.ldq, p.Q, p.defl, k, outer_stride(D),
                                        (float*)p.Ck.data, s)) != MAPI_OK)
          return st;
        A = &p.Ck;
      }
      if ((st = enqueue_solve(ctx, s, A, p.op, 1, w0 + (int64_t)c * D, D, p.iters, p.tol,
                              MAPI_FLAG_FINAL_L2, P_out + (int64_t)c * D, D, p.abort)) != MAPI_OK)
        return st;
      k_record<<<1, 1, 0, s>>>((const IterCtl*)ctx->ctl.p, p.rec, p.rec + 64, p.abort, c);
      MAPI_CUDA_TRY(ctx, cudaGetLastError());
      count_launch(ctx);
    }
    return MAPI_OK;
  }
  // pair mode
  float* wb0 = (float*)ctx->wbuf0.p;
  float* wb1 = (float*)ctx->wbuf1.p;
  IterCtl* ctl = (IterCtl*)ctx->ctl.p;
  const int norm_l2 = (p.op == MAPI_OP_DOT) ? 1 : 0;
  const OuterSlot slot0 = outer_slot(p.defl, k, p.D_pad, 0);
  DeflArgs defl{};
  defl.op = p.op;
  // dot deflates with the kept unit-l2 components, min1 / min2 with their
  // unit-l1 copies (launch_outer_prep)
  defl.P = p.op == MAPI_OP_DOT ? P_out : slot0.wt;
  defl.ldp = p.op == MAPI_OP_DOT ? D : p.D_pad;
  defl.stride = p.D_pad;
  defl.perm = slot0.perm;
  defl.wsort = slot0.wsort;
  defl.ubi = slot0.ubi;
  // max |X| (the scale of the exact fixed-point row sums), once per solve
  if ((st = launch_pair_prepare(ctx, s, p.pl, X, ctx->ypart.p)) != MAPI_OK) return st;
  for (int c = 0; c < k; ++c) {
    if (c > 0 && p.op != MAPI_OP_DOT) {
      if ((st = launch_outer_prep(ctx, p.op, P_out + (int64_t)(c - 1) * D, D,
                                  outer_slot(p.defl, k, p.D_pad, c - 1), s)) != MAPI_OK)
        return st;
    }
    defl.nprev = c;
    if ((st = launch_start_float(ctx, s, w0 + (int64_t)c * D, D, D, 1, wb0, wb1, p.wst, 0, ctl,
                                 (float)p.tol, p.abort)) != MAPI_OK)
      return st;
    // all steps of the component in one launch; the tile order alternates
    // over all steps of all components
    if ((st = launch_pair_solve(ctx, s, p.pl, X, ctx->ypart.p, wb0, wb1, defl, ctl, p.iters,
                                norm_l2, (float)p.denom, (c * p.iters) & 1)) != MAPI_OK)
      return st;
    if ((st = launch_finish(ctx, s, wb0, wb1, p.wst, D, 1, ctl, 1, 0, 0, P_out + (int64_t)c * D,
                            D)) != MAPI_OK)
      return st;
    k_record<<<1, 1, 0, s>>>(ctl, p.rec, p.rec + 64, p.abort, c);
    MAPI_CUDA_TRY(ctx, cudaGetLastError());
    count_launch(ctx);
  }
  return MAPI_OK;
}

}  // namespace

mapi_status run_pair_partial(mapi_ctx* ctx, const mapi_mat* X, mapi_op op, const float* w,
                             float* y) {
  PairPlan pl;
  mapi_status st;
  if ((st = plan_pair(ctx, X, op, &pl)) != MAPI_OK) return st;
  const int64_t wst = (pl.D_pad + 15) / 16 * 16;
  if ((st = ensure(ctx, ctx->wbuf0, sizeof(float) * wst)) != MAPI_OK ||
      (st = ensure(ctx, ctx->wbuf1, sizeof(float) * wst)) != MAPI_OK ||
      (st = ensure(ctx, ctx->ypart, pair_scratch_bytes(pl))) != MAPI_OK ||
      (st = ensure(ctx, ctx->ctl, sizeof(IterCtl))) != MAPI_OK)
    return st;
  cudaStream_t s = ctx->stream;
  float* wb0 = (float*)ctx->wbuf0.p;
  float* wb1 = (float*)ctx->wbuf1.p;
  IterCtl* ctl = (IterCtl*)ctx->ctl.p;
  if ((st = launch_pair_prepare(ctx, s, pl, X, ctx->ypart.p)) != MAPI_OK) return st;
  // w is used as given (no start normalisation)
  if ((st = launch_start_float(ctx, s, w, X->rows, X->rows, 1, wb0, wb1, wst, 1, ctl, 0.f)) !=
      MAPI_OK)
    return st;
  DeflArgs defl{};
  defl.op = op;
  if ((st = launch_pair_solve(ctx, s, pl, X, ctx->ypart.p, wb0, wb1, defl, ctl, 1,
                              op == MAPI_OP_DOT ? 1 : 0, 1.f, 0, y)) != MAPI_OK)
    return st;
  IterCtl h;
  MAPI_CUDA_TRY(ctx, cudaMemcpyAsync(&h, ctl, sizeof(IterCtl), cudaMemcpyDeviceToHost, s));
  MAPI_CUDA_TRY(ctx, cudaStreamSynchronize(s));
  if (h.v[0].status != MAPI_OK)
    return fail(ctx, (mapi_status)h.v[0].status, "pair partial did not complete");
  return MAPI_OK;
}

mapi_status run_pca(mapi_ctx* ctx, const mapi_mat* X, int k, int mode, mapi_op op, int iters,
                    double tol, double denom, const float* w0, float* P_out, int* iters_done) {
  if (mode != MAPI_PCA_MINCOV && mode != MAPI_PCA_PAIR)
    return fail(ctx, MAPI_EINVAL, "mode must be MINCOV or PAIR");
  PcaPlan p;
  p.D = X->rows;
  p.k = k;
  p.mode = mode;
  p.op = op;
  p.iters = iters;
  p.tol = tol;
  p.denom = denom;
  p.ldq = (p.D + 3) / 4 * 4;
  mapi_status st;
  // ---- every allocation happens here, before any capture
  if ((st = ensure(ctx, ctx->aux, 64 + sizeof(int) * 129)) != MAPI_OK) return st;
  if (mode == MAPI_PCA_MINCOV) {
    p.Cm.rows = p.Cm.cols = p.D;
    p.Cm.rows_pad = (p.D + 63) / 64 * 64;
    p.Cm.ld = p.ldq;
    p.Cm.storage = MAPI_ST_F32;
    p.Cm.owner = ctx;
    p.Ck = p.Cm;
    const size_t bytes = sizeof(float) * p.Cm.rows_pad * p.Cm.ld;
    if ((st = ensure(ctx, ctx->pca_c0, bytes)) != MAPI_OK ||
        (st = ensure(ctx, ctx->pca_c1, bytes)) != MAPI_OK ||
        (st = ensure(ctx, ctx->mcpart, mincov_scratch_bytes(ctx, X))) != MAPI_OK)
      return st;
    if (k > 1) {
      if (p.D > kOuterMaxD)
        return fail(ctx, MAPI_ENOTSUP, "min-covariance deflation supports D <= 16384");
      if ((st = ensure(ctx, ctx->pca_q, sizeof(float) * p.D * p.ldq)) != MAPI_OK ||
          (st = ensure(ctx, ctx->pca_defl, outer_scratch_bytes(k, p.D))) != MAPI_OK)
        return st;
    }
    if ((st = prepare_solve(ctx, &p.Cm, 1)) != MAPI_OK) return st;
  } else {
    if ((st = plan_pair(ctx, X, op, &p.pl)) != MAPI_OK) return st;
    p.D_pad = p.pl.D_pad;
    p.wst = (p.D_pad + 15) / 16 * 16;
    if ((st = ensure(ctx, ctx->wbuf0, sizeof(float) * p.wst)) != MAPI_OK ||
        (st = ensure(ctx, ctx->wbuf1, sizeof(float) * p.wst)) != MAPI_OK ||
        (st = ensure(ctx, ctx->ypart, pair_scratch_bytes(p.pl))) != MAPI_OK ||
        (st = ensure(ctx, ctx->ctl, sizeof(IterCtl))) != MAPI_OK ||
        (st = ensure(ctx, ctx->pca_defl, sizeof(float) * 4 * (size_t)k * p.D_pad)) != MAPI_OK)
      return st;
  }
  if ((st = outer_prepare(ctx)) != MAPI_OK) return st;
  // addresses are final now (ensure may have moved buffers and dropped graphs)
  p.rec = (int*)((char*)ctx->aux.p + 64);
  p.abort = p.rec + 128;
  p.Cm.data = ctx->pca_c0.p;
  p.Ck.data = ctx->pca_c1.p;
  p.Q = (float*)ctx->pca_q.p;
  p.defl = ctx->pca_defl.p;

  uint64_t tb, db;
  std::memcpy(&tb, &tol, 8);
  std::memcpy(&db, &denom, 8);
  std::vector<int64_t> key = {2,
                              (int64_t)X->id,
                              k,
                              mode,
                              (int64_t)op,
                              iters,
                              (int64_t)tb,
                              (int64_t)db,
                              (int64_t)(uintptr_t)w0,
                              (int64_t)(uintptr_t)P_out,
                              (int64_t)ctx->prof_on,
                              (int64_t)(uintptr_t)ctx->aux.p,
                              (int64_t)(uintptr_t)ctx->wbuf0.p,
                              (int64_t)(uintptr_t)ctx->ypart.p,
                              (int64_t)(uintptr_t)ctx->pca_c0.p,
                              (int64_t)(uintptr_t)ctx->pca_defl.p,
                              (int64_t)ctx->stall_ns,
                              (int64_t)(ctx->phases_on ? (uintptr_t)ctx->pair_phases.p : 0)};
  GraphEntry* ge = nullptr;
  st = launch_cached_graph(
      ctx, key, [&](cudaStream_t cs) { return pca_enqueue(ctx, cs, X, p, w0, P_out); }, &ge);
  if (st != MAPI_OK) return st;
  MAPI_CUDA_TRY(ctx, cudaMemcpyAsync(ctx->rec_host, p.rec, sizeof(int) * 128,
                                     cudaMemcpyDeviceToHost, ctx->stream));
  MAPI_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  finish_graph(ctx, ge);
  mapi_status result = MAPI_OK;
  for (int c = 0; c < k; ++c) {
    if (iters_done) iters_done[c] = ctx->rec_host[c];
    if (result == MAPI_OK && ctx->rec_host[64 + c] != MAPI_OK)
      result = (mapi_status)ctx->rec_host[64 + c];
  }
  if (result != MAPI_OK) fail(ctx, result, "a component stopped early with this status");
  return result;
}

}  // namespace mapi
