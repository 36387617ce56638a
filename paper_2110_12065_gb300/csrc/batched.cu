// Batched MAPI: many independent instances, several start vectors each, in
// one persistent launch.  Every CTA claims whole instances (largest first)
// from an atomic counter and runs all their steps on its own; the iterates
// and products of all vectors of an instance stay in shared memory, and each
// element of A read from memory serves every vector.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>

#include "device_common.cuh"

namespace mapi {

constexpr int kBatchThreads = 256;
constexpr int kBatchWarps = kBatchThreads / 32;
constexpr int kBatchMaxN = 2048;

// One instance as the kernel sees it.
struct BatchDev {
  const uint8_t* A;   // packed rows (rows_pad x ld)
  int64_t row_bytes;
  int n;
  int chunks;         // 16-byte chunks per row
  const float* w0;    // n x nvec, column-major (ld = n)
  float* w_out;       // n x nvec, column-major (ld = n)
  int* res;           // per vector: iters, status (2 ints)
  float* delta;       // per vector: last delta
};

struct BatchArgs {
  const BatchDev* items;
  const int* order;   // claim order (largest first)
  int count;
  int* next;          // claim counter (zeroed before the launch)
  int max_iters;
  float tol;
  int raw_start;
  int final_l2;
  int norm_l2;
};

// y = A (+) w for V vectors in shared memory; a warp owns R rows at a time,
// its lanes stride over the row's 16-byte chunks.  w_s is [j][V], y_s [i][V].
template <int OP, int ST, int V, int R>
__device__ __forceinline__ void cta_product(const BatchDev& it, const float* __restrict__ w_s,
                                            float* __restrict__ y_s) {
  using Ch = Chunk<ST>;
  constexpr int E = Ch::E;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int row0 = warp * R; row0 < it.n; row0 += kBatchWarps * R) {
    float acc[R][V];
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
      for (int v = 0; v < V; ++v) acc[r][v] = 0.f;
    for (int c = lane; c < it.chunks; c += 32) {
      Ch ch[R];
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int row = min(row0 + r, it.n - 1);  // rows past n repeat the last one
        ch[r].raw = ld_stream(it.A + (int64_t)row * it.row_bytes + (int64_t)c * 16);
      }
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const int j = c * E + e;
        const bool live = j < it.n;  // the packed row's zero padding
#pragma unroll
        for (int v = 0; v < V; ++v) {
          const auto p = Op<OP>::prep(live ? w_s[j * V + v] : 0.f);
#pragma unroll
          for (int r = 0; r < R; ++r) acc[r][v] = Op<OP>::term(ch[r].get(e), p, acc[r][v]);
        }
      }
    }
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
      for (int v = 0; v < V; ++v) {
        float s = acc[r][v];
#pragma unroll
        for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0 && row0 + r < it.n) y_s[(row0 + r) * V + v] = s;
      }
  }
}

template <int OP, int ST, int V, int R>
__global__ void __launch_bounds__(kBatchThreads) k_batched(BatchArgs a) {
  extern __shared__ float bsh[];
  float* w_s = bsh;                       // kBatchMaxN x V
  float* y_s = bsh + kBatchMaxN * V;      // kBatchMaxN x V
  __shared__ float red[33];
  __shared__ float s_norm[V], s_dl[V];
  __shared__ int s_idx, s_done[V], s_it[V], s_st[V];
  for (;;) {
    if (threadIdx.x == 0) {
      const int k = atomicAdd(a.next, 1);
      s_idx = k < a.count ? a.order[k] : -1;
    }
    __syncthreads();
    const int idx = s_idx;
    if (idx < 0) return;
    const BatchDev it = a.items[idx];
    const int n = it.n;
    // Alg. 1 step 1 per vector
    for (int v = 0; v < V; ++v) {
      Kahan k;
      int bad = 0;
      for (int i = threadIdx.x; i < n; i += kBatchThreads) {
        const float x = it.w0[(int64_t)v * n + i];
        bad |= !isfinite(x);
        k.add(x * x);
      }
      bad = __syncthreads_or(bad);
      const float s = sqrtf(block_sum<kBatchThreads>(k.value(), red));
      const bool scale = !a.raw_start && s > 0.f && !bad;
      for (int i = threadIdx.x; i < n; i += kBatchThreads) {
        const float x = it.w0[(int64_t)v * n + i];
        w_s[i * V + v] = scale ? x / s : x;
      }
      if (threadIdx.x == 0) {
        s_it[v] = 0;
        s_st[v] = bad ? MAPI_ENONFINITE : (!a.raw_start && !(s > 0.f)) ? MAPI_EZERONORM : MAPI_OK;
        s_done[v] = s_st[v] != MAPI_OK;
        s_dl[v] = NAN;
      }
    }
    __syncthreads();
    for (int t = 0; t < a.max_iters; ++t) {
      bool any = false;
#pragma unroll
      for (int v = 0; v < V; ++v) any |= !s_done[v];
      if (!any) break;
      cta_product<OP, ST, V, R>(it, w_s, y_s);
      __syncthreads();
      // Alg. 1 step 4 per vector: norm, divide, delta, stop test
#pragma unroll
      for (int v = 0; v < V; ++v) {
        if (s_done[v]) continue;  // uniform
        Kahan k;
        for (int i = threadIdx.x; i < n; i += kBatchThreads) {
          const float y = y_s[i * V + v];
          k.add(a.norm_l2 ? y * y : fabsf(y));
        }
        float L = block_sum<kBatchThreads>(k.value(), red);
        if (a.norm_l2) L = sqrtf(L);
        if (!(L > 0.f) || !isfinite(L)) {
          if (threadIdx.x == 0) {
            s_st[v] = (L == 0.f) ? MAPI_EZERONORM : MAPI_ENONFINITE;
            s_done[v] = 1;
          }
          __syncthreads();
          continue;
        }
        Kahan d;
        for (int i = threadIdx.x; i < n; i += kBatchThreads) {
          const float x = y_s[i * V + v] / L;
          d.add(fabsf(x - w_s[i * V + v]));
          w_s[i * V + v] = x;
        }
        const float D = block_sum<kBatchThreads>(d.value(), red);
        if (threadIdx.x == 0) {
          s_it[v] += 1;
          s_dl[v] = D;
          if (a.tol > 0.f && D < a.tol) s_done[v] = 1;
        }
        __syncthreads();
      }
    }
    // Alg. 1 step 6 (optional) and the results
    for (int v = 0; v < V; ++v) {
      float s = 1.f;
      if (a.final_l2 && s_st[v] == MAPI_OK) {
        Kahan k;
        for (int i = threadIdx.x; i < n; i += kBatchThreads) {
          const float x = w_s[i * V + v];
          k.add(x * x);
        }
        s = sqrtf(block_sum<kBatchThreads>(k.value(), red));
        if (!(s > 0.f)) s = 1.f;
      }
      for (int i = threadIdx.x; i < n; i += kBatchThreads)
        it.w_out[(int64_t)v * n + i] = (s == 1.f) ? w_s[i * V + v] : w_s[i * V + v] / s;
      if (threadIdx.x == 0) {
        it.res[2 * v] = s_it[v];
        it.res[2 * v + 1] = s_st[v];
        it.delta[v] = s_dl[v];
      }
    }
    __syncthreads();
  }
}

using BatchFn = void (*)(BatchArgs);

template <int OP, int ST, int V>
static BatchFn pick_r(int r) {
  switch (r) {
    case 1: return k_batched<OP, ST, V, 1>;
    case 2: return k_batched<OP, ST, V, 2>;
  }
  return nullptr;
}

template <int OP, int ST>
static BatchFn pick_v(int V, int r) {
  switch (V) {
    case 1: return pick_r<OP, ST, 1>(r);
    case 4: return pick_r<OP, ST, 4>(r);
  }
  return nullptr;
}

static BatchFn batched_fn(mapi_op op, mapi_storage st, int V, int r) {
  if (st == MAPI_ST_F32)
    return op == MAPI_OP_MIN1 ? pick_v<MAPI_OP_MIN1, kF32>(V, r)
         : op == MAPI_OP_MIN2 ? pick_v<MAPI_OP_MIN2, kF32>(V, r)
         : op == MAPI_OP_DOT  ? pick_v<MAPI_OP_DOT, kF32>(V, r)
                              : nullptr;
  if (st == MAPI_ST_BF16)
    return op == MAPI_OP_MIN1 ? pick_v<MAPI_OP_MIN1, kBF16>(V, r)
         : op == MAPI_OP_MIN2 ? pick_v<MAPI_OP_MIN2, kBF16>(V, r)
         : op == MAPI_OP_DOT  ? pick_v<MAPI_OP_DOT, kBF16>(V, r)
                              : nullptr;
  return nullptr;
}

static int pow2v(int nvec) { return nvec <= 1 ? 1 : 4; }

}  // namespace mapi

using namespace mapi;

namespace {

struct DeviceGuardB {
  int prev = -1;
  explicit DeviceGuardB(int dev) {
    cudaGetDevice(&prev);
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuardB() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

// Launch one persistent batched solve with rows-per-warp r (items and order
// already on the device).
mapi_status launch_batched(mapi_ctx* ctx, mapi_op op, mapi_storage st, int V, int r,
                           const BatchArgs& args, cudaStream_t s, double args_bytes,
                           double args_terms) {
  BatchFn fn = batched_fn(op, st, V, r);
  if (!fn) return fail(ctx, MAPI_EINVAL, "batched solve: op/storage/nvec not supported");
  const size_t smem = sizeof(float) * 2 * kBatchMaxN * V;
  MAPI_CUDA_TRY(ctx, cudaFuncSetAttribute((const void*)fn,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int occ = 0;
  MAPI_CUDA_TRY(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, (const void*)fn,
                                                                   kBatchThreads, smem));
  if (occ < 1) return fail(ctx, MAPI_ECUDA, "batched kernel does not fit");
  const int grid = std::min(args.count, occ * ctx->sm_count);
  MAPI_CUDA_TRY(ctx, cudaMemsetAsync(args.next, 0, sizeof(int), s));
  cudaEvent_t ev = prof_begin(ctx, s);
  fn<<<grid, kBatchThreads, smem, s>>>(args);
  MAPI_CUDA_TRY(ctx, cudaGetLastError());
  prof_end(ctx, s, ev, MAPI_KC_BATCHED, args_bytes, args_terms);
  count_launch(ctx);
  return MAPI_OK;
}

}  // namespace

extern "C" mapi_status mapi_iterate_batched(mapi_ctx* ctx, const mapi_batch_item* items,
                                            int count, mapi_op op, int nvec, int max_iters,
                                            double tol_l1, unsigned flags, int* iters_done,
                                            double* last_delta, int* statuses) {
  if (!ctx) return MAPI_EINVAL;
  if (!items || count < 1 || (nvec != 1 && nvec != 4) || max_iters < 0)
    return fail(ctx, MAPI_EINVAL, "bad batch arguments");
  if (op != MAPI_OP_MIN1 && op != MAPI_OP_MIN2 && op != MAPI_OP_DOT)
    return fail(ctx, MAPI_EINVAL, "batched solves take MIN1, MIN2 or DOT");
  DeviceGuardB g(ctx->device);
  mapi_storage st = MAPI_ST_F32;
  std::vector<BatchDev> host(count);
  std::vector<int64_t> work(count);
  for (int i = 0; i < count; ++i) {
    const mapi_mat* A = items[i].A;
    if (!A || !ctx->mats.count(const_cast<mapi_mat*>(A)) || !items[i].w0 || !items[i].w_out)
      return fail(ctx, MAPI_EINVAL, "batch item " + std::to_string(i) + ": bad pointers");
    if (A->rows != A->cols || A->rows > kBatchMaxN)
      return fail(ctx, MAPI_EINVAL, "batch items must be square with n <= 2048");
    if (i == 0) st = A->storage;
    if (A->storage != st || (st != MAPI_ST_F32 && st != MAPI_ST_BF16))
      return fail(ctx, MAPI_EINVAL, "one F32 or BF16 storage per batch");
    host[i].A = (const uint8_t*)A->data;
    host[i].row_bytes = A->ld * elem_bytes(A->storage);
    host[i].n = A->rows;
    host[i].chunks = (int)(host[i].row_bytes / 16);
    host[i].w0 = items[i].w0;
    host[i].w_out = items[i].w_out;
    work[i] = (int64_t)A->rows * A->rows;
  }
  const int V = pow2v(nvec);
  // largest instances first
  std::vector<int> order(count);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return work[x] > work[y]; });
  // device table: items, order, counter, results
  const size_t items_b = sizeof(BatchDev) * count, order_b = sizeof(int) * count;
  const size_t res_b = sizeof(int) * 2 * V * count, dl_b = sizeof(float) * V * count;
  const size_t total = items_b + order_b + 256 + res_b + dl_b + 1024;
  mapi_status s = ensure(ctx, ctx->batch, total);
  if (s != MAPI_OK) return s;
  char* base = (char*)ctx->batch.p;
  BatchDev* d_items = (BatchDev*)base;
  int* d_order = (int*)(base + items_b);
  int* d_next = (int*)(base + ((items_b + order_b + 255) / 256) * 256);
  int* d_res = d_next + 64;
  float* d_dl = (float*)(d_res + 2 * V * count);
  for (int i = 0; i < count; ++i) {
    host[i].res = d_res + 2 * V * i;
    host[i].delta = d_dl + V * i;
  }
  MAPI_CUDA_TRY(ctx, cudaMemcpyAsync(d_items, host.data(), items_b, cudaMemcpyHostToDevice,
                                     ctx->stream));
  MAPI_CUDA_TRY(ctx, cudaMemcpyAsync(d_order, order.data(), order_b, cudaMemcpyHostToDevice,
                                     ctx->stream));
  BatchArgs a;
  a.items = d_items;
  a.order = d_order;
  a.count = count;
  a.next = d_next;
  a.max_iters = max_iters;
  a.tol = (float)tol_l1;
  a.raw_start = (flags & MAPI_FLAG_RAW_START) ? 1 : 0;
  a.final_l2 = (flags & MAPI_FLAG_FINAL_L2) ? 1 : 0;
  a.norm_l2 = (op == MAPI_OP_DOT) ? 1 : 0;
  const int r = ctx->batch_rows_per_warp[st == MAPI_ST_F32 ? 0 : 1][V == 1 ? 0 : 1];
  // algorithmic work if every vector runs max_iters steps: each matrix read
  // once per step, n^2 terms per vector per step
  double bytes = 0.0, terms = 0.0;
  for (int i = 0; i < count; ++i) {
    bytes += (double)work[i] * elem_bytes(st) * max_iters;
    terms += (double)work[i] * V * max_iters;
  }
  if ((s = launch_batched(ctx, op, st, V, r > 0 ? r : 2, a, ctx->stream, bytes, terms)) != MAPI_OK)
    return s;
  std::vector<int> res(2 * V * count);
  std::vector<float> dl(V * count);
  MAPI_CUDA_TRY(ctx, cudaMemcpyAsync(res.data(), d_res, res_b, cudaMemcpyDeviceToHost, ctx->stream));
  MAPI_CUDA_TRY(ctx, cudaMemcpyAsync(dl.data(), d_dl, dl_b, cudaMemcpyDeviceToHost, ctx->stream));
  MAPI_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  prof_collect(ctx, ctx->pending, true);
  mapi_status result = MAPI_OK;
  for (int i = 0; i < count; ++i)
    for (int v = 0; v < V; ++v) {
      const int it = res[2 * (V * i + v)], stv = res[2 * (V * i + v) + 1];
      if (iters_done) iters_done[i * V + v] = it;
      if (last_delta) last_delta[i * V + v] = (double)dl[V * i + v];
      if (statuses) statuses[i * V + v] = stv;
      if (result == MAPI_OK && stv != MAPI_OK) result = (mapi_status)stv;
    }
  if (result != MAPI_OK) fail(ctx, result, "a batched vector stopped early with this status");
  return result;
}

extern "C" mapi_status mapi_autotune_batched(mapi_ctx* ctx, const mapi_batch_item* items,
                                             int count, mapi_op op, int nvec, int iters,
                                             int* chosen) {
  if (!ctx) return MAPI_EINVAL;
  if (!items || count < 1 || iters < 1) return fail(ctx, MAPI_EINVAL, "bad autotune arguments");
  DeviceGuardB g(ctx->device);
  const mapi_storage st = items[0].A ? items[0].A->storage : MAPI_ST_F32;
  const int V = pow2v(nvec);
  int* slot = &ctx->batch_rows_per_warp[st == MAPI_ST_F32 ? 0 : 1][V == 1 ? 0 : 1];
  cudaEvent_t e0, e1;
  MAPI_CUDA_TRY(ctx, cudaEventCreate(&e0));
  MAPI_CUDA_TRY(ctx, cudaEventCreate(&e1));
  float best = 1e30f;
  int best_r = 2;
  for (int r : {1, 2}) {
    *slot = r;
    mapi_status s = mapi_iterate_batched(ctx, items, count, op, nvec, 1, 0.0, MAPI_FLAG_RAW_START,
                                         nullptr, nullptr, nullptr);  // warm
    if (s != MAPI_OK && s != MAPI_EZERONORM) {
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      return s;
    }
    cudaEventRecord(e0, ctx->stream);
    mapi_iterate_batched(ctx, items, count, op, nvec, iters, 0.0, MAPI_FLAG_RAW_START, nullptr,
                         nullptr, nullptr);
    cudaEventRecord(e1, ctx->stream);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best) {
      best = ms;
      best_r = r;
    }
  }
  *slot = best_r;
  if (chosen) *chosen = best_r;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return MAPI_OK;
}
