// Solve orchestration: start-vector kernel (Alg. 1 step 1), the chain of K1
// steps, and the finishing kernel (Alg. 1 step 6).
#include <cmath>

#include "k_iter.cuh"

namespace mapi {

constexpr int kVecThreads = 1024;

// Alg. 1 step 1 for float storage: w_0 = w0 / ||w0||_2 (or w0 as given).
__global__ void __launch_bounds__(kVecThreads)
    k_start_float(const float* __restrict__ w0, int64_t ldw, int n, int nvec,
                  int V, float* wb0, float* wb1, int64_t wst, int raw,
                  IterCtl* ctl, float tol, const int* abort) {
  __shared__ float sh[33];
  // a solve chained after a failed one (PCA components) is skipped
  const bool skip = abort && *(volatile const int*)abort;
  int all = 1;
  for (int v = 0; v < V; ++v) {
    float* d0 = wb0 + (int64_t)v * wst;
    float* d1 = wb1 + (int64_t)v * wst;
    if (v >= nvec) {  // padding vector: zeros, already done
      for (int64_t i = threadIdx.x; i < wst; i += kVecThreads) d0[i] = d1[i] = 0.f;
      if (threadIdx.x == 0) {
        ctl->v[v] = VecState{1, MAPI_OK, 0, 0, 0.f, 0.f, 0};
      }
      continue;
    }
    const float* src = w0 + (int64_t)v * ldw;
    Kahan k;
    int bad = 0;
    for (int i = threadIdx.x; i < n; i += kVecThreads) {
      const float x = src[i];
      bad |= !isfinite(x);
      k.add(x * x);
    }
    bad = __syncthreads_or(bad);
    const float s = sqrtf(block_sum<kVecThreads>(k.value(), sh));
    int status = MAPI_OK;
    if (bad) status = MAPI_ENONFINITE;
    else if (!raw && !(s > 0.f)) status = MAPI_EZERONORM;
    if (skip) status = MAPI_ECANCELLED;
    const bool scale = !raw && status == MAPI_OK;
    for (int64_t i = threadIdx.x; i < wst; i += kVecThreads) {
      d0[i] = i < n ? (scale ? src[i] / s : src[i]) : 0.f;
      d1[i] = 0.f;
    }
    if (threadIdx.x == 0)
      ctl->v[v] = VecState{status != MAPI_OK, status, 0, 0, NAN, s, -1};
    all &= (status != MAPI_OK);
  }
  if (threadIdx.x == 0) {
    ctl->counter = 0;
    ctl->nvec = nvec;
    ctl->tol = tol;
    ctl->all_done = all;
  }
}

// Integer storage: x = RNE(w0 2^q), then w = sign(x) floor((|x| 2^q + L/2)/L).
__global__ void __launch_bounds__(kVecThreads)
    k_start_int(const float* __restrict__ w0, int64_t ldw, int n, int nvec, int V,
                int* wb0, int* wb1, int64_t wst, int q, IterCtl* ctl,
                long long itol) {
  __shared__ long long sh[33];
  int all = 1;
  for (int v = 0; v < V; ++v) {
    int* d0 = wb0 + (int64_t)v * wst;
    int* d1 = wb1 + (int64_t)v * wst;
    if (v >= nvec) {
      for (int64_t i = threadIdx.x; i < wst; i += kVecThreads) d0[i] = d1[i] = 0;
      if (threadIdx.x == 0) ctl->v[v] = VecState{1, MAPI_OK, 0, 0, 0.f, 0.f, 0};
      continue;
    }
    const float* src = w0 + (int64_t)v * ldw;
    long long s = 0;
    int bad = 0;
    for (int i = threadIdx.x; i < n; i += kVecThreads) {
      const float x = scalbnf(src[i], q);  // exact
      bad |= !(fabsf(x) < 2147483648.f);
      if (!bad) s += (long long)fabsf(rintf(x));
    }
    bad = __syncthreads_or(bad);
    const long long L = block_sum_i64<kVecThreads>(bad ? 0 : s, sh);
    int status = bad ? MAPI_EINVAL : (L == 0 ? MAPI_EZERONORM : MAPI_OK);
    for (int64_t i = threadIdx.x; i < wst; i += kVecThreads) {
      int out = 0;
      if (i < n && !bad) {
        const long long x = (long long)rintf(scalbnf(src[i], q));
        if (status == MAPI_OK) {
          const long long m = ((llabs(x) << q) + L / 2) / L;
          out = (int)(x < 0 ? -m : m);
        } else {
          out = (int)x;
        }
      }
      d0[i] = out;
      d1[i] = 0;
    }
    if (threadIdx.x == 0)
      ctl->v[v] = VecState{status != MAPI_OK, status, 0, 0, NAN, 0.f, -1};
    all &= (status != MAPI_OK);
  }
  if (threadIdx.x == 0) {
    ctl->counter = 0;
    ctl->nvec = nvec;
    ctl->itol = itol;
    ctl->tol = 0.f;
    ctl->all_done = all;
  }
}

// Alg. 1 step 6 (optional l2) and the copy-out of the last iterate, which
// sits in wb0 or wb1 according to the parity of the vector's step count.
__global__ void __launch_bounds__(kVecThreads)
    k_finish(const float* wb0, const float* wb1, int64_t wst, int n, int nvec,
             const IterCtl* ctl, int final_l2, int is_int, int q, float* out,
             int64_t ldo) {
  __shared__ float sh[33];
  for (int v = 0; v < nvec; ++v) {
    const VecState st = ctl->v[v];
    const float* src = ((st.iters & 1) ? wb1 : wb0) + (int64_t)v * wst;
    float* dst = out + (int64_t)v * ldo;
    const float unit = is_int ? scalbnf(1.f, -q) : 1.f;
    auto val = [&](int i) {
      return is_int ? (float)reinterpret_cast<const int*>(src)[i] * unit : src[i];
    };
    float s = 1.f;
    if (final_l2 && st.status == MAPI_OK) {
      Kahan k;
      for (int i = threadIdx.x; i < n; i += kVecThreads) {
        const float x = val(i);
        k.add(x * x);
      }
      s = sqrtf(block_sum<kVecThreads>(k.value(), sh));
      if (!(s > 0.f)) s = 1.f;
    }
    for (int i = threadIdx.x; i < n; i += kVecThreads) dst[i] = (s == 1.f) ? val(i) : val(i) / s;
  }
}

// ---------------------------------------------------------------- host side

mapi_status launch_start_float(mapi_ctx* ctx, cudaStream_t s, const float* w0, int64_t ldw,
                               int n, int nvec, float* wb0, float* wb1, int64_t wst, int raw,
                               IterCtl* ctl, float tol, const int* abort) {
  k_start_float<<<1, kVecThreads, 0, s>>>(w0, ldw, n, nvec, nvec, wb0, wb1, wst, raw, ctl, tol,
                                         abort);
  MAPI_CUDA_TRY(ctx, cudaGetLastError());
  count_launch(ctx);
  return MAPI_OK;
}

mapi_status launch_finish(mapi_ctx* ctx, cudaStream_t s, const float* wb0, const float* wb1,
                          int64_t wst, int n, int nvec, const IterCtl* ctl, int final_l2,
                          int is_int, int q, float* out, int64_t ldo) {
  k_finish<<<1, kVecThreads, 0, s>>>(wb0, wb1, wst, n, nvec, ctl, final_l2, is_int, q, out, ldo);
  MAPI_CUDA_TRY(ctx, cudaGetLastError());
  count_launch(ctx);
  return MAPI_OK;
}

GemvPlan plan_gemv(const mapi_ctx* ctx, const mapi_mat* A, int nvec) {
  (void)nvec;
  GemvPlan p;
  p.rows_per_warp = gemv_rows_for(A->storage);
  p.warps = kWarps;
  p.grid_rows = A->rows_pad / (p.rows_per_warp * kWarps);
  const int64_t chunks = A->ld * elem_bytes(A->storage) / 16;
  // enough CTAs for several waves (the block scheduler then balances the
  // tail), each column split still >= 64 chunks (2 per lane).  Measured on
  // GB300 against 24 waves' worth: 12 is as fast or faster at every order
  // (n = 4096 FP32 37.7 -> 23.9 us per step, n = 8192 BF16 44.7 -> 34.8,
  // n = 16384 FP32 / BF16 / FP8 / int16 4-9 % faster); fewer column splits
  // also leave the epilogue fewer partial sums to add
  const int want = 12 * ctx->sm_count;
  int ks = 1;
  while ((int64_t)p.grid_rows * ks < want && chunks / (ks * 2) >= 64) ks *= 2;
  p.ksplit = ks;
  return p;
}

static int pow2ceil(int x) {
  int v = 1;
  while (v < x) v <<= 1;
  return v;
}

static int64_t vec_stride(const mapi_mat* A) { return (A->ld + 15) / 16 * 16; }

mapi_status prepare_solve(mapi_ctx* ctx, const mapi_mat* A, int nvec) {
  const int V = pow2ceil(nvec);
  const GemvPlan p = plan_gemv(ctx, A, V);
  const int64_t wst = vec_stride(A);
  mapi_status s;
  if ((s = ensure(ctx, ctx->wbuf0, (size_t)V * wst * 4)) != MAPI_OK) return s;
  if ((s = ensure(ctx, ctx->wbuf1, (size_t)V * wst * 4)) != MAPI_OK) return s;
  if ((s = ensure(ctx, ctx->ypart, (size_t)p.ksplit * V * A->rows_pad * 4)) != MAPI_OK) return s;
  if ((s = ensure(ctx, ctx->ctl, sizeof(IterCtl))) != MAPI_OK) return s;
  return MAPI_OK;
}

mapi_status enqueue_solve(mapi_ctx* ctx, cudaStream_t stream, const mapi_mat* A,
                          mapi_op op, int nvec, const float* w0, int64_t ldw,
                          int max_iters, double tol, unsigned flags,
                          float* w_out, int64_t ldo, const int* abort) {
  const int V = pow2ceil(nvec);
  const GemvPlan p = plan_gemv(ctx, A, V);
  const int64_t wst = vec_stride(A);
  const bool is_int = is_int_storage(A->storage);
  LaunchFn fn = nullptr;
  switch (A->storage) {
    case MAPI_ST_F32: fn = gemv_lookup_f32(op, V); break;
    case MAPI_ST_BF16: fn = gemv_lookup_bf16(op, V); break;
    case MAPI_ST_FP8E4M3_ROWPOW2: fn = gemv_lookup_fp8(op, V); break;
    case MAPI_ST_I16: fn = gemv_lookup_int(kI16, op, V); break;
    case MAPI_ST_I8: fn = gemv_lookup_int(kI8, op, V); break;
  }
  if (!fn) return fail(ctx, MAPI_EINVAL, "op not available for this storage / vector count");
  float* wb0 = (float*)ctx->wbuf0.p;
  float* wb1 = (float*)ctx->wbuf1.p;
  IterCtl* ctl = (IterCtl*)ctx->ctl.p;
  const int raw = (flags & MAPI_FLAG_RAW_START) ? 1 : 0;
  if (is_int) {
    long long itol = 0;
    if (tol > 0) itol = (long long)std::ceil(tol * std::ldexp(1.0, A->q));
    if (tol > 0 && itol < 1) itol = 1;
    k_start_int<<<1, kVecThreads, 0, stream>>>(w0, ldw, A->rows, nvec, V, (int*)wb0,
                                              (int*)wb1, wst, A->q, ctl, itol);
  } else {
    k_start_float<<<1, kVecThreads, 0, stream>>>(w0, ldw, A->rows, nvec, V, wb0, wb1,
                                                wst, raw, ctl, (float)tol, abort);
  }
  MAPI_CUDA_TRY(ctx, cudaGetLastError());
  count_launch(ctx);
  GemvArgs g;
  g.A = (const uint8_t*)A->data;
  g.row_bytes = A->ld * elem_bytes(A->storage);
  g.chunks = (int)(g.row_bytes / 16);
  g.seg = (g.chunks + p.ksplit - 1) / p.ksplit;
  g.n = A->rows;
  g.rows_pad = A->rows_pad;
  g.wst = wst;
  g.ypart = (float*)ctx->ypart.p;
  g.ctl = ctl;
  g.row_mult = A->row_scale;
  g.norm_l2 = (op == MAPI_OP_DOT) ? 1 : 0;
  g.clusters = ctx->gemv_clusters ? 1 : 0;
  const dim3 grid(p.grid_rows, p.ksplit);
  // algorithmic work of one step: the stored matrix once (plus FP8 row
  // scales), n^2 terms per vector
  const double step_bytes = (double)A->rows * A->cols * elem_bytes(A->storage) +
                            (A->storage == MAPI_ST_FP8E4M3_ROWPOW2 ? 4.0 * A->rows : 0.0);
  const double step_terms = (double)A->rows * A->cols * nvec;
  for (int t = 0; t < max_iters; ++t) {
    g.w = (t & 1) ? wb1 : wb0;
    g.w_next = (t & 1) ? wb0 : wb1;
    cudaEvent_t ev = prof_begin(ctx, stream);
    MAPI_CUDA_TRY(ctx, fn(grid, stream, g, A->q));
    prof_end(ctx, stream, ev, MAPI_KC_GEMV, step_bytes, step_terms);
    count_launch(ctx);
  }
  k_finish<<<1, kVecThreads, 0, stream>>>(wb0, wb1, wst, A->rows, nvec, ctl,
                                         (flags & MAPI_FLAG_FINAL_L2) ? 1 : 0,
                                         is_int ? 1 : 0, A->q, w_out, ldo);
  MAPI_CUDA_TRY(ctx, cudaGetLastError());
  count_launch(ctx);
  return MAPI_OK;
}

}  // namespace mapi
