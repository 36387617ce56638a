// Outer products w (+) w^T of Alg. 2 applied without forming them: the
// deflation of step 6 (C_c = C - sum_{m<c} P_m C) and the reconstruction of
// step 8 (v^ = (W (+) W^T)(v - m) + m), and Alg. 2 end to end on images.
//
// Each outer product takes its component at the unit norm of the component's
// own iteration: w / ||w||_1 for MIN1 / MIN2 (the normalisation of Eq. (8)),
// w as kept (unit l2) for DOT, whose w w^T is the projector of §1.  For a
// component of equal magnitudes the unit-l1 MIN1 outer product is exactly
// the projector u u^T.
//
// With c = |wt|, s = sign(wt) and z = s * y, MIN1's product is
//   (P y)_i = s_i [ sum_{c_j <= c_i} c_j z_j + c_i sum_{c_j > c_i} z_j ],
// two prefix sums over the order of c; MIN2's outer product is half of MIN1's
// plus the same with every sign +1; DOT's is wt (wt . y).  k_outer_prep ranks
// a component once (perm, wsort, ubi), k_outer_apply runs the prefix sums
// for one input row per CTA with the row, and the two prefix arrays, in
// shared memory.
#include <algorithm>

#include "device_common.cuh"

namespace mapi {

namespace {

constexpr int kPrepThreads = 1024;
constexpr int kApplyThreads = 1024;

// Ranks component w (length D) into one slot, one CTA: wt = the scaled
// component, perm[p] = index at sorted position p (order of |wt|, ties by
// index), wsort[p] = wt[perm[p]], ubi[i] = the last sorted position whose
// |wt| is <= |wt_i|.  The keys (|wt| bits, index) are sorted by a bitonic
// network in shared memory (Dp = D rounded up to a power of two, padded with
// the largest key).  DOT only needs wt.
__global__ void __launch_bounds__(kPrepThreads)
    k_outer_prep(const float* __restrict__ w, int D, int Dp, int op, OuterSlot r) {
  extern __shared__ unsigned long long keys[];
  __shared__ float red[33];
  const int t = threadIdx.x;
  if (op == MAPI_OP_DOT) {
    for (int i = t; i < D; i += kPrepThreads) r.wt[i] = w[i];
    return;
  }
  Kahan k;
  for (int i = t; i < D; i += kPrepThreads) k.add(fabsf(w[i]));
  float L = block_sum<kPrepThreads>(k.value(), red);
  if (!(L > 0.f)) L = 1.f;
  for (int j = t; j < Dp; j += kPrepThreads) {
    unsigned long long key = ~0ull;
    if (j < D) {
      const float wj = w[j] / L;
      r.wt[j] = wj;
      key = ((unsigned long long)__float_as_uint(fabsf(wj)) << 32) | (unsigned)j;
    }
    keys[j] = key;
  }
  __syncthreads();
  for (int size = 2; size <= Dp; size <<= 1)
    for (int lh = __ffs(size) - 2; lh >= 0; --lh) {
      const int half = 1 << lh;
      for (int x = t; x < Dp / 2; x += kPrepThreads) {
        const int i = ((x >> lh) << (lh + 1)) | (x & (half - 1));
        const int l = i + half;
        const bool up = (i & size) == 0;
        const unsigned long long ki = keys[i], kl = keys[l];
        if ((ki > kl) == up) {
          keys[i] = kl;
          keys[l] = ki;
        }
      }
      __syncthreads();
    }
  for (int p = t; p < D; p += kPrepThreads) {
    const unsigned long long key = keys[p];
    const int i = (int)(key & 0xffffffffu);
    const unsigned cb = (unsigned)(key >> 32);
    // last position whose magnitude bits are <= cb
    int lo = p, hi = Dp - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if ((unsigned)(keys[mid] >> 32) <= cb) lo = mid;
      else hi = mid - 1;
    }
    r.perm[p] = i;
    r.wsort[p] = w[i] / L;
    r.ubi[i] = lo;
  }
}

// Inclusive scan of two value sets over positions p = e * 1024 + t (thread
// t holds a[e], b[e] for e < E): a warp scan per e, the warp totals scanned
// by warp e, then the totals of the E blocks of 1024 added in order.
// tot: 2 x E x 32 floats of shared memory.
template <int E>
__device__ __forceinline__ void block_scan_strided(float (&a)[E], float (&b)[E], float* tot) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float* ta = tot;
  float* tb = tot + E * 32;
#pragma unroll
  for (int e = 0; e < E; ++e) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const float na = __shfl_up_sync(0xffffffffu, a[e], o);
      const float nb = __shfl_up_sync(0xffffffffu, b[e], o);
      if (lane >= o) {
        a[e] += na;
        b[e] += nb;
      }
    }
    if (lane == 31) {
      ta[e * 32 + warp] = a[e];
      tb[e * 32 + warp] = b[e];
    }
  }
  __syncthreads();
  if (warp < E) {
    float va = ta[warp * 32 + lane], vb = tb[warp * 32 + lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const float na = __shfl_up_sync(0xffffffffu, va, o);
      const float nb = __shfl_up_sync(0xffffffffu, vb, o);
      if (lane >= o) {
        va += na;
        vb += nb;
      }
    }
    ta[warp * 32 + lane] = va;
    tb[warp * 32 + lane] = vb;
  }
  __syncthreads();
  float oa = 0.f, ob = 0.f;  // totals of the blocks before block e
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const float pa = warp > 0 ? ta[e * 32 + warp - 1] : 0.f;
    const float pb = warp > 0 ? tb[e * 32 + warp - 1] : 0.f;
    a[e] += oa + pa;
    b[e] += ob + pb;
    oa += ta[e * 32 + 31];
    ob += tb[e * 32 + 31];
  }
}

// out_r = sum_{m<nprev} P_m in_r (+ add) for input row r = blockIdx.x;
// D <= E * 1024.  Thread t holds sorted positions and outputs t + e * 1024,
// so every global access is coalesced; the row and the two prefix arrays sit
// in 3 E 1024 floats of shared memory.
template <int OP, int E>
__global__ void __launch_bounds__(kApplyThreads)
    k_outer_apply(const float* __restrict__ in, int64_t ld_in, int D, int nprev, OuterSlot r0,
                  int64_t stride, const float* __restrict__ add, float* __restrict__ out,
                  int64_t ld_out) {
  extern __shared__ float sm[];
  float* row = sm;
  float* A = row + E * kApplyThreads;
  float* B = A + E * kApplyThreads;
  __shared__ float tot[2 * E * 32];
  __shared__ float red[33];
  const int t = threadIdx.x;
  const float* src = in + (int64_t)blockIdx.x * ld_in;
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int i = t + e * kApplyThreads;
    row[i] = i < D ? src[i] : 0.f;
  }
  float acc[E];
#pragma unroll
  for (int e = 0; e < E; ++e) acc[e] = 0.f;
  __syncthreads();
  for (int m = 0; m < nprev; ++m) {
    const float* wt = r0.wt + m * stride;
    if constexpr (OP == MAPI_OP_DOT) {
      float part = 0.f;
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const int i = t + e * kApplyThreads;
        if (i < D) part = fmaf(wt[i], row[i], part);
      }
      const float d = block_sum<kApplyThreads>(part, red);
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const int i = t + e * kApplyThreads;
        if (i < D) acc[e] = fmaf(wt[i], d, acc[e]);
      }
      continue;
    } else {
      const int* perm = r0.perm + m * stride;
      const float* wsort = r0.wsort + m * stride;
      const int* ubi = r0.ubi + m * stride;
      constexpr int NP = (OP == MAPI_OP_MIN2) ? 2 : 1;
      float x0[E];
#pragma unroll
      for (int pass = 0; pass < NP; ++pass) {
        // every load of the pass is issued before the first use; positions
        // past D read a zero of the row with a zero weight
        float a[E], b[E];
        int pv[E];
#pragma unroll
        for (int e = 0; e < E; ++e) {
          const int p = t + e * kApplyThreads;
          pv[e] = p < D ? __ldg(perm + p) : p;
          a[e] = p < D ? __ldg(wsort + p) : 0.f;
        }
#pragma unroll
        for (int e = 0; e < E; ++e) {
          const float y = row[pv[e]];
          const float z = pass == 0 ? sgnf(a[e]) * y : y;
          a[e] = fabsf(a[e]) * z;
          b[e] = z;
        }
        block_scan_strided<E>(a, b, tot);
#pragma unroll
        for (int e = 0; e < E; ++e) {
          A[t + e * kApplyThreads] = a[e];
          B[t + e * kApplyThreads] = b[e];
        }
        __syncthreads();
        const float totB = B[D - 1];
        // outputs i = t + e * 1024 (past D: position 0, discarded)
#pragma unroll
        for (int e = 0; e < E; ++e) {
          const int i = t + e * kApplyThreads;
          pv[e] = i < D ? __ldg(ubi + i) : 0;
          a[e] = i < D ? __ldg(wt + i) : 0.f;
        }
#pragma unroll
        for (int e = 0; e < E; ++e) {
          const int q = pv[e];
          const float v = A[q] + fabsf(a[e]) * (totB - B[q]);
          if (pass == 0) x0[e] = sgnf(a[e]) * v;
          if constexpr (OP == MAPI_OP_MIN1) acc[e] += x0[e];
          else if (pass == 1) acc[e] += 0.5f * (x0[e] + v);
        }
        __syncthreads();  // A, B and the block totals are reused
      }
    }
  }
  float* dst = out + (int64_t)blockIdx.x * ld_out;
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int i = t + e * kApplyThreads;
    if (i < D) dst[i] = acc[e] + (add ? add[i] : 0.f);
  }
}

// Cc[i][j] = C[i][j] - T[j][i] for i, j < D (32 x 32 tiles through shared
// memory); T's row j holds column j of sum_m P_m C (C is symmetric).  The
// tile of C is loaded with the tile of T, before the exchange.
__global__ void __launch_bounds__(256)
    k_sub_transpose(const float* __restrict__ C, const float* __restrict__ T, int D, int64_t ld,
                    float* __restrict__ Cc) {
  __shared__ float tile[32][33];
  const int bi = blockIdx.y * 32, bj = blockIdx.x * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  float cv[4];
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int rr = ty + 8 * u;
    const int j = bj + rr, i = bi + tx;
    tile[rr][tx] = (j < D && i < D) ? __ldcs(T + (int64_t)j * ld + i) : 0.f;
    const int i2 = bi + rr, j2 = bj + tx;
    cv[u] = (i2 < D && j2 < D) ? __ldcs(C + (int64_t)i2 * ld + j2) : 0.f;
  }
  __syncthreads();
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int rr = ty + 8 * u;
    const int i = bi + rr, j = bj + tx;
    if (i < D && j < D) Cc[(int64_t)i * ld + j] = cv[u] - tile[tx][rr];
  }
}

// Alg. 2 steps 1-3 for N images of P pixels (row i = image i): m_p = mean
// over the images (in image order), X[p][i] = v_i[p] - m_p packed (P rows,
// N columns, zero padding up to ld), Z[i][p] the same values row-wise.
// The mean is formed by a compensated (two-sum) addition and kept as the
// unevaluated pair m_hi + m_lo, and each centred value is (v - m_hi) - m_lo,
// so a pixel that every image shares centres to exactly 0 (a plain FP32
// mean would leave +-1 ulp there, where the exact centring has zeros) and
// every other value is rounded about once.
__global__ void k_image_center(const float* __restrict__ img, int N, int P, int64_t ld,
                               float* __restrict__ X, float* __restrict__ Z,
                               float* __restrict__ mean) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P) return;
  TwoSum s;
  for (int i = 0; i < N; ++i) s.add(img[(int64_t)i * P + p]);
  const float fN = (float)N;
  const float mh = s.value() / fN;
  const float ml = (fmaf(-mh, fN, s.hi) + s.lo) / fN;
  mean[p] = mh + ml;
  float* xr = X + (int64_t)p * ld;
  for (int i = 0; i < N; ++i) {
    const float v = (img[(int64_t)i * P + p] - mh) - ml;
    xr[i] = v;
    Z[(int64_t)i * P + p] = v;
  }
  for (int64_t i = N; i < ld; ++i) xr[i] = 0.f;
}

template <int OP>
const void* apply_fn(int E) {
  switch (E) {
    case 1: return (const void*)k_outer_apply<OP, 1>;
    case 2: return (const void*)k_outer_apply<OP, 2>;
    case 4: return (const void*)k_outer_apply<OP, 4>;
    case 8: return (const void*)k_outer_apply<OP, 8>;
    case 16: return (const void*)k_outer_apply<OP, 16>;
  }
  return nullptr;
}

struct DeviceGuardO {
  int prev = -1;
  explicit DeviceGuardO(int d) {
    if (cudaGetDevice(&prev) == cudaSuccess && prev != d) cudaSetDevice(d);
  }
  ~DeviceGuardO() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

}  // namespace

OuterSlot outer_slot(void* base, int k, int64_t stride, int m) {
  OuterSlot s;
  float* f = (float*)base;
  s.wt = f + (int64_t)m * stride;
  s.perm = (int*)(f + (int64_t)k * stride) + (int64_t)m * stride;
  s.wsort = f + 2 * (int64_t)k * stride + (int64_t)m * stride;
  s.ubi = (int*)(f + 3 * (int64_t)k * stride) + (int64_t)m * stride;
  return s;
}

mapi_status outer_prepare(mapi_ctx* ctx) {
  MAPI_CUDA_TRY(ctx, cudaFuncSetAttribute((const void*)k_outer_prep,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)(sizeof(unsigned long long) * kOuterMaxD)));
  for (int E = 1; E <= 16; E *= 2) {
    const int smem = (int)(sizeof(float) * 3 * E * kApplyThreads);
    for (const void* fn : {apply_fn<MAPI_OP_MIN1>(E), apply_fn<MAPI_OP_MIN2>(E),
                           apply_fn<MAPI_OP_DOT>(E)})
      MAPI_CUDA_TRY(ctx, cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              smem));
  }
  return MAPI_OK;
}

mapi_status launch_outer_prep(mapi_ctx* ctx, mapi_op op, const float* w, int D, OuterSlot slot,
                              cudaStream_t s) {
  if (D < 1 || D > kOuterMaxD) return fail(ctx, MAPI_EINVAL, "outer product order outside 1..16384");
  int Dp = 1;
  while (Dp < D) Dp <<= 1;
  if (Dp < 2) Dp = 2;
  const size_t smem = sizeof(unsigned long long) * (size_t)Dp;
  k_outer_prep<<<1, kPrepThreads, smem, s>>>(w, D, Dp, (int)op, slot);
  MAPI_CUDA_TRY(ctx, cudaGetLastError());
  count_launch(ctx);
  return MAPI_OK;
}

mapi_status launch_outer_apply(mapi_ctx* ctx, mapi_op op, int D, int nprev, OuterSlot first,
                               int64_t stride, const float* in, int64_t ld_in, int rows,
                               const float* add, float* out, int64_t ld_out, cudaStream_t s) {
  if (D < 1 || D > kOuterMaxD) return fail(ctx, MAPI_EINVAL, "outer product order outside 1..16384");
  if (rows == 0) return MAPI_OK;
  int E = 1;
  while (E * kApplyThreads < D) E *= 2;
  const void* fn = op == MAPI_OP_MIN1   ? apply_fn<MAPI_OP_MIN1>(E)
                   : op == MAPI_OP_MIN2 ? apply_fn<MAPI_OP_MIN2>(E)
                                        : apply_fn<MAPI_OP_DOT>(E);
  if (!fn) return fail(ctx, MAPI_EINVAL, "outer product operator");
  const size_t smem = sizeof(float) * 3 * (size_t)E * kApplyThreads;
  void* args[] = {(void*)&in, (void*)&ld_in, (void*)&D, (void*)&nprev, (void*)&first,
                  (void*)&stride, (void*)&add, (void*)&out, (void*)&ld_out};
  MAPI_CUDA_TRY(ctx, cudaLaunchKernel(fn, dim3(rows), dim3(kApplyThreads), args, smem, s));
  count_launch(ctx);
  return MAPI_OK;
}

mapi_status launch_deflate_mincov(mapi_ctx* ctx, mapi_op op, const float* P, int64_t ldp, int c,
                                  int D, const float* C, int64_t ld, float* T, void* rank,
                                  int kslots, int64_t stride, float* Cc, cudaStream_t s) {
  if (c < 1 || c > kslots) return fail(ctx, MAPI_EINVAL, "deflation component");
  mapi_status st =
      launch_outer_prep(ctx, op, P + (int64_t)(c - 1) * ldp, D,
                        outer_slot(rank, kslots, stride, c - 1), s);
  if (st != MAPI_OK) return st;
  if ((st = launch_outer_apply(ctx, op, D, c, outer_slot(rank, kslots, stride, 0), stride, C, ld,
                               D, nullptr, T, ld, s)) != MAPI_OK)
    return st;
  const dim3 g((D + 31) / 32, (D + 31) / 32);
  k_sub_transpose<<<g, 256, 0, s>>>(C, T, D, ld, Cc);
  MAPI_CUDA_TRY(ctx, cudaGetLastError());
  count_launch(ctx);
  return MAPI_OK;
}

size_t outer_scratch_bytes(int k, int D) {
  return sizeof(float) * 4 * (size_t)k * outer_stride(D);
}

}  // namespace mapi

using namespace mapi;

extern "C" mapi_status mapi_mavp_project(mapi_ctx* ctx, mapi_op op, const float* W, int64_t ldw,
                                         int D, int k, const float* in, int64_t ld_in, int rows,
                                         const float* add, float* out, int64_t ld_out) {
  if (!ctx) return MAPI_EINVAL;
  if (op != MAPI_OP_MIN1 && op != MAPI_OP_MIN2 && op != MAPI_OP_DOT)
    return fail(ctx, MAPI_EINVAL, "op must be MIN1, MIN2 or DOT");
  if (D < 1 || D > kOuterMaxD || k < 1 || k > kOuterMaxK || rows < 0 || ldw < D || ld_in < D ||
      ld_out < D)
    return fail(ctx, MAPI_EINVAL, "bad shape");
  if (rows == 0) return MAPI_OK;
  if (!W || !in || !out) return fail(ctx, MAPI_EINVAL, "null pointer");
  DeviceGuardO guard(ctx->device);
  const int64_t stride = outer_stride(D);
  mapi_status st = ensure(ctx, ctx->outer, outer_scratch_bytes(k, D));
  if (st != MAPI_OK || (st = outer_prepare(ctx)) != MAPI_OK) return st;
  for (int m = 0; m < k; ++m)
    if ((st = launch_outer_prep(ctx, op, W + (int64_t)m * ldw, D,
                                outer_slot(ctx->outer.p, k, stride, m), ctx->stream)) != MAPI_OK)
      return st;
  return launch_outer_apply(ctx, op, D, k, outer_slot(ctx->outer.p, k, stride, 0), stride, in,
                            ld_in, rows, add, out, ld_out, ctx->stream);
}

extern "C" mapi_status mapi_image_reconstruct(mapi_ctx* ctx, const float* images, int N, int P,
                                              int k, mapi_op op, int iters, double tol_l1,
                                              const float* w0, float* W_out, float* recon_out,
                                              int* iters_done) {
  if (!ctx) return MAPI_EINVAL;
  if (!images || !w0 || !W_out || !recon_out) return fail(ctx, MAPI_EINVAL, "null pointer");
  if (op != MAPI_OP_MIN1 && op != MAPI_OP_MIN2 && op != MAPI_OP_DOT)
    return fail(ctx, MAPI_EINVAL, "op must be MIN1, MIN2 or DOT");
  if (N < 2 || P < 1 || P > kOuterMaxD || k < 1 || k > P || k > kOuterMaxK || iters < 0)
    return fail(ctx, MAPI_EINVAL, "bad shape");
  DeviceGuardO guard(ctx->device);
  mapi_status st;
  // the packed centred images keep their identity (and cached graphs) while
  // the shape stays the same
  if (ctx->img_X && (ctx->img_X->rows != P || ctx->img_X->cols != N)) {
    free_matrix(ctx, ctx->img_X);
    ctx->img_X = nullptr;
  }
  if (!ctx->img_X) {
    if ((st = alloc_matrix(ctx, P, N, MAPI_ST_F32, &ctx->img_X)) != MAPI_OK) return st;
    MAPI_CUDA_TRY(ctx, cudaMemsetAsync(ctx->img_X->data, 0, ctx->img_X->bytes, ctx->stream));
  }
  mapi_mat* X = ctx->img_X;
  if ((st = ensure(ctx, ctx->img, sizeof(float) * ((size_t)P * N + P))) != MAPI_OK) return st;
  float* Z = (float*)ctx->img.p;
  float* mean = Z + (size_t)P * N;
  k_image_center<<<(P + 255) / 256, 256, 0, ctx->stream>>>(images, N, P, X->ld, (float*)X->data,
                                                           Z, mean);
  MAPI_CUDA_TRY(ctx, cudaGetLastError());
  count_launch(ctx);
  // steps 4-7: C = X (+) X^T / (N - 1), k components by MAPI with deflation
  if ((st = mapi_pca_topk(ctx, X, k, MAPI_PCA_MINCOV, op, iters, tol_l1, (double)(N - 1), w0,
                          W_out, iters_done)) != MAPI_OK)
    return st;
  // step 8 for every image
  if ((st = mapi_mavp_project(ctx, op, W_out, P, P, k, Z, P, N, mean, recon_out, P)) != MAPI_OK)
    return st;
  MAPI_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  return MAPI_OK;
}
