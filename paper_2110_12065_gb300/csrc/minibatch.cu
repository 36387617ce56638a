// Mini-batch MAPI with momentum (Alg. 3): one CTA runs all T steps.
//
// Step t averages the MAVP outer products x (+) x^T of the s samples drawn for
// it (the caller passes the draws), forms v = A_t (+) w_t - beta w_{t-1} and
// scales both w_t and v by ||v||_1 (||v||_2 for DOT, the momentum power
// method it is compared with).  D is small (the paper's set has D = 10), so
// the whole step lives in one CTA's shared memory: the batch's samples
// arrive in chunks, groups of threads split the chunk's samples, each thread
// owns entries (p, q) of A_t, and the groups' partials are added in a fixed
// order.
#include <algorithm>

#include "device_common.cuh"

namespace mapi {
namespace {

constexpr int kMbThreads = 1024;
constexpr int kMbMaxD = 128;
constexpr int kMbPairs = kMbMaxD * kMbMaxD / kMbThreads;  // entries of A_t per thread
constexpr int kMbStageFloats = 12288;                      // samples staged at once

template <int OP>
__global__ void __launch_bounds__(kMbThreads)
    k_minibatch(const float* __restrict__ X, int N, int D, const int* __restrict__ batch, int T,
                int s, float beta, const float* __restrict__ w0, int final_l2,
                float* __restrict__ w_out, int* __restrict__ status) {
  extern __shared__ float mb[];
  float* stage = mb;                    // chunk rows x D
  float* A = stage + kMbStageFloats;    // D x D
  __shared__ float w[kMbMaxD], wp[kMbMaxD], v[kMbMaxD];
  __shared__ float red[33];
  __shared__ int bad;
  const int t0 = threadIdx.x;
  const int chunk = kMbStageFloats / D;
  // step 1: w_0 = w0 / ||w0||_2, w_{-1} = 0
  {
    Kahan k;
    for (int p = t0; p < D; p += kMbThreads) k.add(w0[p] * w0[p]);
    const float n2 = sqrtf(block_sum<kMbThreads>(k.value(), red));
    for (int p = t0; p < D; p += kMbThreads) {
      w[p] = n2 > 0.f ? w0[p] / n2 : w0[p];
      wp[p] = 0.f;
    }
    if (t0 == 0) bad = n2 > 0.f ? MAPI_OK : MAPI_EZERONORM;
  }
  __syncthreads();
  // G groups of threads split a chunk's samples (sample i to group i mod G);
  // each thread of a group owns entries j, j + width, ... of A_t
  const int npairs = D * D;
  const int G = npairs >= kMbThreads ? 1 : kMbThreads / npairs;
  const int width = G == 1 ? kMbThreads : npairs;
  const int g = t0 / width, j = t0 - g * width;
  for (int t = 0; t < T && bad == MAPI_OK; ++t) {
    float acc[kMbPairs];
#pragma unroll
    for (int k = 0; k < kMbPairs; ++k) acc[k] = 0.f;
    for (int i0 = 0; i0 < s; i0 += chunk) {
      const int rows = min(chunk, s - i0);
      for (int e = t0; e < rows * D; e += kMbThreads) {
        const int i = e / D, p = e - i * D;
        const int k = batch[(int64_t)t * s + i0 + i];
        const bool in = k >= 0 && k < N;
        stage[e] = in ? X[(int64_t)k * D + p] : 0.f;
        if (!in) bad = MAPI_EINVAL;
      }
      __syncthreads();
      if (g < G) {
#pragma unroll
        for (int k = 0; k < kMbPairs; ++k) {
          const int pq = j + k * width;
          if (pq < npairs) {
            const int p = pq / D, q = pq - p * D;
            float a = acc[k];
            for (int i = g; i < rows; i += G) {
              const float* x = stage + i * D;
              a = Op<OP>::term(x[p], Op<OP>::prep(x[q]), a);
            }
            acc[k] = a;
          }
        }
      }
      __syncthreads();
    }
    if (G == 1) {
#pragma unroll
      for (int k = 0; k < kMbPairs; ++k) {
        const int pq = j + k * width;
        if (pq < npairs) A[pq] = acc[k] / (float)s;
      }
    } else {
      // the groups' partials, added in group order (stage is free here)
      if (g < G) stage[g * npairs + j] = acc[0];
      __syncthreads();
      for (int pq = t0; pq < npairs; pq += kMbThreads) {
        float a = 0.f;
        for (int h = 0; h < G; ++h) a += stage[h * npairs + pq];
        A[pq] = a / (float)s;
      }
    }
    __syncthreads();
    // v = A_t (+) w_t - beta w_{t-1}, rows of A_t against w_t in column order
    for (int p = t0; p < D; p += kMbThreads) {
      float a = 0.f;
      for (int q = 0; q < D; ++q) a = Op<OP>::term(A[p * D + q], Op<OP>::prep(w[q]), a);
      v[p] = a - beta * wp[p];
    }
    __syncthreads();
    Kahan kn;
    for (int p = t0; p < D; p += kMbThreads) kn.add(OP == MAPI_OP_DOT ? v[p] * v[p] : fabsf(v[p]));
    float L = block_sum<kMbThreads>(kn.value(), red);
    if (OP == MAPI_OP_DOT) L = sqrtf(L);
    if (!(L > 0.f) || !isfinite(L)) {
      if (t0 == 0 && bad == MAPI_OK) bad = (L == 0.f) ? MAPI_EZERONORM : MAPI_ENONFINITE;
      __syncthreads();
      break;
    }
    for (int p = t0; p < D; p += kMbThreads) {
      wp[p] = w[p] / L;  // the n divisions of §2.2, for both iterates
      w[p] = v[p] / L;
    }
    __syncthreads();
  }
  // step 7 (optional): w_T / ||w_T||_2
  Kahan k2;
  for (int p = t0; p < D; p += kMbThreads) k2.add(w[p] * w[p]);
  const float n2 = sqrtf(block_sum<kMbThreads>(k2.value(), red));
  const bool scale = final_l2 && bad == MAPI_OK && n2 > 0.f;
  for (int p = t0; p < D; p += kMbThreads) w_out[p] = scale ? w[p] / n2 : w[p];
  if (t0 == 0) *status = bad;
}

struct DeviceGuardM {
  int prev = -1;
  explicit DeviceGuardM(int d) {
    if (cudaGetDevice(&prev) == cudaSuccess && prev != d) cudaSetDevice(d);
  }
  ~DeviceGuardM() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

}  // namespace
}  // namespace mapi

using namespace mapi;

extern "C" mapi_status mapi_minibatch_momentum(mapi_ctx* ctx, const float* X, int N, int D,
                                               const int* batch, int T, int s, double beta,
                                               mapi_op op, const float* w0, unsigned flags,
                                               float* w_out) {
  if (!ctx) return MAPI_EINVAL;
  if (!X || (!batch && T > 0) || !w0 || !w_out || N < 1 || D < 1 || D > kMbMaxD || T < 0 || s < 1)
    return fail(ctx, MAPI_EINVAL, "bad argument");
  if (op != MAPI_OP_MIN1 && op != MAPI_OP_MIN2 && op != MAPI_OP_DOT)
    return fail(ctx, MAPI_EINVAL, "Alg. 3 takes MIN1, MIN2 or DOT");
  DeviceGuardM guard(ctx->device);
  mapi_status st = ensure(ctx, ctx->aux, 64 + sizeof(int) * 129);
  if (st != MAPI_OK) return st;
  int* dstat = (int*)((char*)ctx->aux.p + 64 + sizeof(int) * 128);
  const size_t smem = sizeof(float) * ((size_t)kMbStageFloats + (size_t)D * D);
  void (*fn)(const float*, int, int, const int*, int, int, float, const float*, int, float*,
             int*) = op == MAPI_OP_MIN1   ? k_minibatch<MAPI_OP_MIN1>
                     : op == MAPI_OP_MIN2 ? k_minibatch<MAPI_OP_MIN2>
                                          : k_minibatch<MAPI_OP_DOT>;
  MAPI_CUDA_TRY(ctx, cudaFuncSetAttribute((const void*)fn,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  fn<<<1, kMbThreads, smem, ctx->stream>>>(X, N, D, batch, T, s, (float)beta, w0,
                                           (flags & MAPI_FLAG_FINAL_L2) ? 1 : 0, w_out, dstat);
  MAPI_CUDA_TRY(ctx, cudaGetLastError());
  count_launch(ctx);
  int hs = 0;
  MAPI_CUDA_TRY(ctx, cudaMemcpyAsync(&hs, dstat, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  MAPI_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  if (hs != MAPI_OK) return fail(ctx, (mapi_status)hs, "Alg. 3 stopped early");
  return MAPI_OK;
}
