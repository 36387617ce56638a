// Issue-rate probe of the MAVP term's instruction mixes (diagnostic): a
// register-resident loop of independent chains, timed in SM cycles inside
// the kernel, gives the terms (or instructions) one SM completes per clock.
// It is the ALU roofline that the batched and min-covariance kernels are
// measured against.
#include <vector>

#include "device_common.cuh"

namespace mapi {
namespace {

constexpr int kProbeThreads = 512;
constexpr int kProbeChains = 8;
constexpr int kProbeIters = 4096;

// mix 0: the FP32 min1 term, sign(w) clamp(a, -|w|, |w|) added by a fused
//        multiply-add by +-1 (two min/max and one FMA per term);
// mix 1: FMA alone;  mix 2: min/max alone (two per update);
// mix 3: the min1 term on a BF16 operand widened to FP32 first;
// mix 4: the same, each widened element used against four vectors' bounds.
// Each update of chain j reads chain j + 1, so nothing can be hoisted.
template <int MIX>
__global__ void __launch_bounds__(kProbeThreads)
    k_alu_probe(float seed, long long* cycles, float* sink) {
  float acc[kProbeChains];
#pragma unroll
  for (int j = 0; j < kProbeChains; ++j) acc[j] = seed * (float)(threadIdx.x + j);
  const float lo = -1.f, hi = 1.f, sg = seed > 0.f ? 1.f : -1.f;
  __syncthreads();
  const long long t0 = clock64();
#pragma unroll 4
  for (int it = 0; it < kProbeIters; ++it) {
#pragma unroll
    for (int j = 0; j < kProbeChains; ++j) {
      const float a = acc[(j + 1) % kProbeChains];
      if (MIX == 0) acc[j] = fmaf(fminf(fmaxf(a, lo), hi), sg, acc[j]);
      if (MIX == 1) acc[j] = fmaf(a, 0.999f, acc[j]);
      if (MIX == 2) acc[j] = fminf(fmaxf(a, acc[j]), hi);
      if (MIX == 3) {
        const float x = __uint_as_float(__float_as_uint(a) << 16);
        acc[j] = fmaf(fminf(fmaxf(x, lo), hi), sg, acc[j]);
      }
      if (MIX == 4 && (j & 3) == 0) {
        // one BF16 element widened once and used against four vectors'
        // bounds (the batched kernel's four start vectors)
        const float x = __uint_as_float(__float_as_uint(a) << 16);
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          const float b = 0.25f * (float)(v + 1);
          acc[j + v] = fmaf(fminf(fmaxf(x, -b), b), sg, acc[j + v]);
        }
      }
    }
  }
  __syncthreads();
  const long long t1 = clock64();
  float s = 0.f;
#pragma unroll
  for (int j = 0; j < kProbeChains; ++j) s += acc[j];
  if (s == 1234.5f) sink[threadIdx.x] = s;  // keeps the loop
  if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
}

template <int MIX>
mapi_status run_probe(mapi_ctx* ctx, long long* dcyc, float* dsink, int blocks) {
  k_alu_probe<MIX><<<blocks, kProbeThreads, 0, ctx->stream>>>(1.0001f, dcyc, dsink);
  MAPI_CUDA_TRY(ctx, cudaGetLastError());
  count_launch(ctx);
  return MAPI_OK;
}

}  // namespace
}  // namespace mapi

using namespace mapi;

extern "C" mapi_status mapi_alu_probe(mapi_ctx* ctx, int mix, double* per_clock_per_sm) {
  if (!ctx || !per_clock_per_sm || mix < 0 || mix > 4) return MAPI_EINVAL;
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != ctx->device) cudaSetDevice(ctx->device);
  int per_sm = 0;
  const void* fns[5] = {(const void*)k_alu_probe<0>, (const void*)k_alu_probe<1>,
                        (const void*)k_alu_probe<2>, (const void*)k_alu_probe<3>,
                        (const void*)k_alu_probe<4>};
  mapi_status st = MAPI_OK;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fns[mix], kProbeThreads, 0) !=
          cudaSuccess ||
      per_sm < 1) {
    cudaGetLastError();
    st = fail(ctx, MAPI_ECUDA, "probe occupancy");
  }
  const int blocks = per_sm * ctx->sm_count;  // one full wave, every block resident
  if (st == MAPI_OK)
    st = ensure(ctx, ctx->aux, 64 + sizeof(int) * 129 + sizeof(long long) * blocks +
                                   sizeof(float) * kProbeThreads);
  if (st == MAPI_OK) {
    char* base = (char*)ctx->aux.p + 64 + sizeof(int) * 129;
    long long* dcyc = (long long*)(((uintptr_t)base + 7) & ~(uintptr_t)7);
    float* dsink = (float*)(dcyc + blocks);
    for (int rep = 0; rep < 2 && st == MAPI_OK; ++rep)  // the first run warms up
      st = mix == 0   ? run_probe<0>(ctx, dcyc, dsink, blocks)
           : mix == 1 ? run_probe<1>(ctx, dcyc, dsink, blocks)
           : mix == 2 ? run_probe<2>(ctx, dcyc, dsink, blocks)
           : mix == 3 ? run_probe<3>(ctx, dcyc, dsink, blocks)
                      : run_probe<4>(ctx, dcyc, dsink, blocks);
    std::vector<long long> h(blocks);
    if (st == MAPI_OK) {
      if (cudaMemcpyAsync(h.data(), dcyc, sizeof(long long) * blocks, cudaMemcpyDeviceToHost,
                          ctx->stream) != cudaSuccess ||
          cudaStreamSynchronize(ctx->stream) != cudaSuccess) {
        cudaGetLastError();
        st = fail(ctx, MAPI_ECUDA, "probe copy");
      }
    }
    if (st == MAPI_OK) {
      long long mx = 1;
      for (long long c : h) mx = c > mx ? c : mx;
      // work of the blocks resident on one SM, over the slowest block's cycles
      // (mix 2 counts its min/max instructions, two per update)
      const double work = (double)per_sm * kProbeThreads * kProbeIters * kProbeChains *
                          (mix == 2 ? 2.0 : 1.0);
      *per_clock_per_sm = work / (double)mx;
    }
  }
  if (prev >= 0 && prev != ctx->device) cudaSetDevice(prev);
  return st;
}
