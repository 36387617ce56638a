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
// a component once (perm, csort, ubi), k_outer_apply runs the prefix sums
// for one input row per CTA with the row, and the two prefix arrays, in
// shared memory.
#include <algorithm>

#include "device_common.cuh"

namespace mapi {

namespace {

constexpr int kPrepThreads = 256;
constexpr int kApplyThreads = 1024;

// Ranks component w (length D) into one slot: wt = the scaled component,
// perm[p] = index at sorted position p (ties by index), csort[p] = its |wt|,
// ubi[i] = the last sorted position whose |wt| is <= |wt_i|.  Every CTA
// forms the same scale and magnitudes (fixed order); CTA b ranks indices
// [256 b, 256 b + 256).  DOT only needs wt.
__global__ void __launch_bounds__(kPrepThreads)
    k_outer_prep(const float* __restrict__ w, int D, int op, OuterSlot r) {
  extern __shared__ float cs[];  // D magnitudes
  __shared__ float red[33];
  float L = 1.f;
  if (op != MAPI_OP_DOT) {
    Kahan k;
    for (int i = threadIdx.x; i < D; i += kPrepThreads) k.add(fabsf(w[i]));
    L = block_sum<kPrepThreads>(k.value(), red);
    if (!(L > 0.f)) L = 1.f;
  }
  const int i = blockIdx.x * kPrepThreads + threadIdx.x;
  if (op == MAPI_OP_DOT) {
    if (i < D) r.wt[i] = w[i];
    return;
  }
  for (int j = threadIdx.x; j < D; j += kPrepThreads) cs[j] = fabsf(w[j] / L);
  __syncthreads();
  if (i >= D) return;
  const float wi = w[i] / L;
  const float ci = cs[i];
  int below = 0, le = 0, tie_before = 0;
  int j = 0;
  for (; j + 4 <= D; j += 4) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const float cj = cs[j + u];
      below += cj < ci;
      le += cj <= ci;
      tie_before += (cj == ci) & (j + u < i);
    }
  }
  for (; j < D; ++j) {
    const float cj = cs[j];
    below += cj < ci;
    le += cj <= ci;
    tie_before += (cj == ci) & (j < i);
  }
  const int rank = below + tie_before;
  r.perm[rank] = i;
  r.csort[rank] = ci;
  r.ubi[i] = le - 1;
  r.wt[i] = wi;
}

// Inclusive block scan of a[E], b[E] held by each thread over consecutive
// positions (thread t owns [t E, t E + E)); fixed order.
template <int E>
__device__ __forceinline__ void block_scan2(float (&a)[E], float (&b)[E], float* wa, float* wb) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int e = 1; e < E; ++e) {
    a[e] += a[e - 1];
    b[e] += b[e - 1];
  }
  float ta = a[E - 1], tb = b[E - 1];
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const float na = __shfl_up_sync(0xffffffffu, ta, o);
    const float nb = __shfl_up_sync(0xffffffffu, tb, o);
    if (lane >= o) {
      ta += na;
      tb += nb;
    }
  }
  if (lane == 31) {
    wa[warp] = ta;
    wb[warp] = tb;
  }
  __syncthreads();
  if (warp == 0) {
    float va = wa[lane], vb = wb[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const float na = __shfl_up_sync(0xffffffffu, va, o);
      const float nb = __shfl_up_sync(0xffffffffu, vb, o);
      if (lane >= o) {
        va += na;
        vb += nb;
      }
    }
    wa[lane] = va;
    wb[lane] = vb;
  }
  __syncthreads();
  const float oa = (ta - a[E - 1]) + (warp > 0 ? wa[warp - 1] : 0.f);
  const float ob = (tb - b[E - 1]) + (warp > 0 ? wb[warp - 1] : 0.f);
#pragma unroll
  for (int e = 0; e < E; ++e) {
    a[e] += oa;
    b[e] += ob;
  }
}

// out_r = sum_{m<nprev} P_m in_r (+ add) for input row r = blockIdx.x;
// D <= E * 1024.  Rows, prefix arrays: 3 E 1024 floats of shared memory.
template <int OP, int E>
__global__ void __launch_bounds__(kApplyThreads)
    k_outer_apply(const float* __restrict__ in, int64_t ld_in, int D, int nprev, OuterSlot r0,
                  int64_t stride, const float* __restrict__ add, float* __restrict__ out,
                  int64_t ld_out) {
  extern __shared__ float sm[];
  float* row = sm;
  float* A = row + E * kApplyThreads;
  float* B = A + E * kApplyThreads;
  __shared__ float wa[32], wb[32], red[33];
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
      const float* csort = r0.csort + m * stride;
      const int* ubi = r0.ubi + m * stride;
      constexpr int NP = (OP == MAPI_OP_MIN2) ? 2 : 1;
      float x0[E];
#pragma unroll
      for (int pass = 0; pass < NP; ++pass) {
        float a[E], b[E];
#pragma unroll
        for (int e = 0; e < E; ++e) {
          const int p = t * E + e;
          a[e] = b[e] = 0.f;
          if (p < D) {
            const int i = perm[p];
            const float y = row[i];
            const float z = pass == 0 ? sgnf(wt[i]) * y : y;
            a[e] = csort[p] * z;
            b[e] = z;
          }
        }
        block_scan2<E>(a, b, wa, wb);
#pragma unroll
        for (int e = 0; e < E; ++e) {
          A[t * E + e] = a[e];
          B[t * E + e] = b[e];
        }
        __syncthreads();
        const float totB = B[D - 1];
#pragma unroll
        for (int e = 0; e < E; ++e) {
          const int i = t + e * kApplyThreads;
          if (i < D) {
            const float wi = wt[i];
            const int q = ubi[i];
            const float v = A[q] + fabsf(wi) * (totB - B[q]);
            if (pass == 0) x0[e] = sgnf(wi) * v;
            if constexpr (OP == MAPI_OP_MIN1) acc[e] += x0[e];
            else if (pass == 1) acc[e] += 0.5f * (x0[e] + v);
          }
        }
        __syncthreads();  // A, B and the warp totals are reused
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
// memory); T's row j holds column j of sum_m P_m C (C is symmetric).
__global__ void __launch_bounds__(256)
    k_sub_transpose(const float* __restrict__ C, const float* __restrict__ T, int D, int64_t ld,
                    float* __restrict__ Cc) {
  __shared__ float tile[32][33];
  const int bi = blockIdx.y * 32, bj = blockIdx.x * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (int rr = ty; rr < 32; rr += 8) {
    const int j = bj + rr, i = bi + tx;
    tile[rr][tx] = (j < D && i < D) ? T[(int64_t)j * ld + i] : 0.f;
  }
  __syncthreads();
  for (int rr = ty; rr < 32; rr += 8) {
    const int i = bi + rr, j = bj + tx;
    if (i < D && j < D) Cc[(int64_t)i * ld + j] = C[(int64_t)i * ld + j] - tile[tx][rr];
  }
}

// Alg. 2 steps 1-3 for N images of P pixels (row i = image i): m_p = mean
// over the images (in image order), X[p][i] = v_i[p] - m_p packed (P rows,
// N columns, zero padding up to ld), Z[i][p] the same values row-wise.
__global__ void k_image_center(const float* __restrict__ img, int N, int P, int64_t ld,
                               float* __restrict__ X, float* __restrict__ Z,
                               float* __restrict__ mean) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P) return;
  float s = 0.f;
  for (int i = 0; i < N; ++i) s += img[(int64_t)i * P + p];
  const float m = s / (float)N;
  mean[p] = m;
  float* xr = X + (int64_t)p * ld;
  for (int i = 0; i < N; ++i) {
    const float v = img[(int64_t)i * P + p] - m;
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
  s.csort = f + 2 * (int64_t)k * stride + (int64_t)m * stride;
  s.ubi = (int*)(f + 3 * (int64_t)k * stride) + (int64_t)m * stride;
  return s;
}

mapi_status outer_prepare(mapi_ctx* ctx) {
  MAPI_CUDA_TRY(ctx, cudaFuncSetAttribute((const void*)k_outer_prep,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)(sizeof(float) * kOuterMaxD)));
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
  const size_t smem = sizeof(float) * (size_t)D;
  k_outer_prep<<<(D + kPrepThreads - 1) / kPrepThreads, kPrepThreads, smem, s>>>(w, D, (int)op,
                                                                                slot);
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
