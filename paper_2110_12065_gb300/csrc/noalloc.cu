// mapi_iterate_noalloc: Alg. 1 on a caller-owned FP32 matrix without any
// allocation.  Every scratch buffer of the solve (control block, the two
// iterate buffers, the per-split partial products) lives in one file-scope
// device array of fixed size; the caller passes only inputs and outputs.
#include <mutex>

#include "k_iter.cuh"

namespace mapi {
namespace {

constexpr int kNaMaxN = 8192;     // largest n accepted
constexpr int kNaMaxSplit = 8;    // column splits of one step
constexpr int kNaThreads = 1024;  // start / finish kernels
constexpr size_t kNaCtlBytes = 512;
constexpr size_t kNaVecBytes = sizeof(float) * kNaMaxN;
constexpr size_t kNaBytes = kNaCtlBytes + 2 * kNaVecBytes + kNaMaxSplit * kNaVecBytes;
static_assert(sizeof(IterCtl) <= kNaCtlBytes, "control block does not fit");

// The whole scratch of a solve: [IterCtl | w buffer 0 | w buffer 1 | partials].
// Every GPU that loads the library holds these bytes until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNaBytes];

// Start: w0 / ||w0||_2 (or as given) into buffer 0, zeros elsewhere, and the
// control block cleared; everything a step reads is rewritten here.
__global__ void __launch_bounds__(kNaThreads)
    k_na_start(const float* __restrict__ w0, int n, int64_t wst, int raw, float tol,
               unsigned char* scratch) {
  __shared__ float sh[33];
  IterCtl* ctl = reinterpret_cast<IterCtl*>(scratch);
  float* wb0 = reinterpret_cast<float*>(scratch + kNaCtlBytes);
  float* wb1 = reinterpret_cast<float*>(scratch + kNaCtlBytes + kNaVecBytes);
  Kahan k;
  int bad = 0;
  for (int i = threadIdx.x; i < n; i += kNaThreads) {
    const float x = w0[i];
    bad |= !isfinite(x);
    k.add(x * x);
  }
  bad = __syncthreads_or(bad);
  const float s = sqrtf(block_sum<kNaThreads>(k.value(), sh));
  int status = MAPI_OK;
  if (bad) status = MAPI_ENONFINITE;
  else if (!raw && !(s > 0.f)) status = MAPI_EZERONORM;
  const bool scale = !raw && status == MAPI_OK;
  for (int64_t i = threadIdx.x; i < wst; i += kNaThreads) {
    wb0[i] = i < n ? (scale ? w0[i] / s : w0[i]) : 0.f;
    wb1[i] = 0.f;
  }
  if (threadIdx.x == 0) {
    ctl->counter = 0;
    ctl->nvec = 1;
    ctl->tol = tol;
    ctl->itol = 0;
    ctl->v[0] = VecState{status != MAPI_OK, status, 0, 0, NAN, s, -1};
    ctl->all_done = (status != MAPI_OK);
  }
}

// K1 for an unpadded caller matrix: rows >= n are skipped and columns >= n
// inside the last 16-byte chunk read as zero, whatever the caller's padding
// holds.  The normalising epilogue is the library's shared one.
template <int OP>
__global__ void __launch_bounds__(kWarps * 32) k1_gemv_noalloc(GemvArgs g) {
  if (*(volatile int*)&g.ctl->all_done) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int row0 = (blockIdx.x * kWarps + warp) * kR;
  const int ks = blockIdx.y;
  const int c_beg = ks * g.seg;
  const int c_end = min(g.chunks, c_beg + g.seg);
  float acc[kR][2];
#pragma unroll
  for (int r = 0; r < kR; ++r) acc[r][0] = acc[r][1] = 0.f;
  for (int c = c_beg + lane; c < c_end; c += 32) {
    const float4 wv = *reinterpret_cast<const float4*>(g.w + (int64_t)c * 4);
    const auto p0 = Op<OP>::prep(wv.x);
    const auto p1 = Op<OP>::prep(wv.y);
    const auto p2 = Op<OP>::prep(wv.z);
    const auto p3 = Op<OP>::prep(wv.w);
    const int col = c * 4;
#pragma unroll
    for (int r = 0; r < kR; ++r) {
      if (row0 + r >= g.n) continue;
      Chunk<kF32> ch;
      ch.raw = ld_stream(g.A + (int64_t)(row0 + r) * g.row_bytes + (int64_t)c * 16);
      const float a0 = ch.get(0);
      const float a1 = col + 1 < g.n ? ch.get(1) : 0.f;
      const float a2 = col + 2 < g.n ? ch.get(2) : 0.f;
      const float a3 = col + 3 < g.n ? ch.get(3) : 0.f;
      acc[r][0] = Op<OP>::term(a0, p0, acc[r][0]);
      acc[r][1] = Op<OP>::term(a1, p1, acc[r][1]);
      acc[r][0] = Op<OP>::term(a2, p2, acc[r][0]);
      acc[r][1] = Op<OP>::term(a3, p3, acc[r][1]);
    }
  }
#pragma unroll
  for (int r = 0; r < kR; ++r) {
    float s = acc[r][0] + acc[r][1];
#pragma unroll
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) g.ypart[(int64_t)ks * g.rows_pad + row0 + r] = s;
  }
  if (!elect_last_cta(&g.ctl->counter, gridDim.x * gridDim.y)) return;
  epilogue_float<kWarps * 32, 1>(g, gridDim.y);
}

// Finish: the last iterate (buffer chosen by the step parity), optionally
// l2-normalised (Alg. 1 step 6), into the caller's output.
__global__ void __launch_bounds__(kNaThreads)
    k_na_finish(int n, int final_l2, float* __restrict__ out, const unsigned char* scratch) {
  __shared__ float sh[33];
  const IterCtl* ctl = reinterpret_cast<const IterCtl*>(scratch);
  const VecState st = ctl->v[0];
  const float* src = reinterpret_cast<const float*>(
      scratch + kNaCtlBytes + ((st.iters & 1) ? kNaVecBytes : 0));
  float s = 1.f;
  if (final_l2 && st.status == MAPI_OK) {
    Kahan k;
    for (int i = threadIdx.x; i < n; i += kNaThreads) k.add(src[i] * src[i]);
    s = sqrtf(block_sum<kNaThreads>(k.value(), sh));
    if (!(s > 0.f)) s = 1.f;
  }
  for (int i = threadIdx.x; i < n; i += kNaThreads) out[i] = (s == 1.f) ? src[i] : src[i] / s;
}

// Device address of the scratch array, looked up once per device.
std::mutex g_na_mutex;
unsigned char* g_na_addr[256] = {};

mapi_status na_scratch(int dev, unsigned char** out) {
  if (dev < 0 || dev >= 256) return MAPI_EINVAL;
  std::lock_guard<std::mutex> lock(g_na_mutex);
  if (!g_na_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      return MAPI_ECUDA;
    }
    g_na_addr[dev] = static_cast<unsigned char*>(p);
  }
  *out = g_na_addr[dev];
  return MAPI_OK;
}

template <int OP>
cudaError_t na_step(dim3 grid, cudaStream_t s, const GemvArgs& g) {
  k1_gemv_noalloc<OP><<<grid, kWarps * 32, 0, s>>>(g);
  return cudaGetLastError();
}

}  // namespace
}  // namespace mapi

using namespace mapi;

extern "C" mapi_status mapi_iterate_noalloc(const float* A, int n, int64_t lda, mapi_op op,
                                            const float* w0, int max_iters, double tol_l1,
                                            unsigned flags, float* w_out, int* iters_done,
                                            double* last_delta, void* cuda_stream) {
  if (!A || !w0 || !w_out || n < 1 || n > kNaMaxN || lda < n || lda % 4 != 0 ||
      ((uintptr_t)A & 15) != 0 || max_iters < 0)
    return MAPI_EINVAL;
  cudaError_t (*step)(dim3, cudaStream_t, const GemvArgs&) = nullptr;
  switch (op) {
    case MAPI_OP_MIN1: step = na_step<MAPI_OP_MIN1>; break;
    case MAPI_OP_MIN2: step = na_step<MAPI_OP_MIN2>; break;
    case MAPI_OP_DIAMOND: step = na_step<MAPI_OP_DIAMOND>; break;
    case MAPI_OP_DOT: step = na_step<MAPI_OP_DOT>; break;
    default: return MAPI_EINVAL;
  }
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return MAPI_ECUDA;
  }
  unsigned char* scratch = nullptr;
  mapi_status st = na_scratch(dev, &scratch);
  if (st != MAPI_OK) return st;
  cudaStream_t s = (cudaStream_t)cuda_stream;

  const int64_t wst = ((int64_t)n + 15) / 16 * 16;
  GemvArgs g{};
  g.A = (const uint8_t*)A;
  g.row_bytes = lda * 4;
  g.chunks = (n + 3) / 4;
  g.n = n;
  const int grid_rows = (n + kR * kWarps - 1) / (kR * kWarps);
  g.rows_pad = grid_rows * kR * kWarps;
  int ks = 1;
  while (grid_rows * ks < 24 * sms && g.chunks / (ks * 2) >= 64 && ks < kNaMaxSplit) ks *= 2;
  g.seg = (g.chunks + ks - 1) / ks;
  g.wst = wst;
  g.ctl = reinterpret_cast<IterCtl*>(scratch);
  g.ypart = reinterpret_cast<float*>(scratch + kNaCtlBytes + 2 * kNaVecBytes);
  g.row_mult = nullptr;
  g.norm_l2 = (op == MAPI_OP_DOT) ? 1 : 0;
  float* wb0 = reinterpret_cast<float*>(scratch + kNaCtlBytes);
  float* wb1 = reinterpret_cast<float*>(scratch + kNaCtlBytes + kNaVecBytes);

  k_na_start<<<1, kNaThreads, 0, s>>>(w0, n, wst, (flags & MAPI_FLAG_RAW_START) ? 1 : 0,
                                      (float)tol_l1, scratch);
  if (cudaGetLastError() != cudaSuccess) return MAPI_ECUDA;
  const dim3 grid(grid_rows, ks);
  for (int t = 0; t < max_iters; ++t) {
    g.w = (t & 1) ? wb1 : wb0;
    g.w_next = (t & 1) ? wb0 : wb1;
    if (step(grid, s, g) != cudaSuccess) return MAPI_ECUDA;
  }
  k_na_finish<<<1, kNaThreads, 0, s>>>(n, (flags & MAPI_FLAG_FINAL_L2) ? 1 : 0, w_out, scratch);
  if (cudaGetLastError() != cudaSuccess) return MAPI_ECUDA;
  IterCtl host;
  if (cudaMemcpyAsync(&host, scratch, sizeof(IterCtl), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    cudaGetLastError();
    return MAPI_ECUDA;
  }
  if (iters_done) *iters_done = host.v[0].iters;
  if (last_delta) *last_delta = (double)host.v[0].delta;
  return (mapi_status)host.v[0].status;
}
