// Batched MAPI: many independent instances, several start vectors each, in
// one persistent launch of 8-CTA clusters.  Large instances go first, one
// cluster each (every CTA streams 1/8 of the rows and keeps the whole
// iterate); when they are all claimed, every CTA claims small instances on
// its own.  Claims are largest first from atomic counters, the iterates and
// products of all vectors of an instance stay in shared memory, and each
// element of A read from memory serves every vector.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <type_traits>

#include <cooperative_groups.h>

#include "device_common.cuh"

namespace cg = cooperative_groups;

namespace mapi {

constexpr int kBatchThreads = 256;
constexpr int kBatchWarps = kBatchThreads / 32;
constexpr int kBatchIterFloats = 8192;  // iterate capacity: n_pad x V floats
constexpr int kBatchCluster = 8;        // CTAs per large instance
constexpr int kBatchLargeN = 1024;      // instances this large get a cluster
constexpr int kBatchRowFloats = kBatchIterFloats / kBatchCluster;  // a rank's products


struct BatchArgs {
  const BatchDev* items;
  const int* order;   // claim order (largest first; the nlarge large ones lead)
  int count;
  int nlarge;
  int* next;          // claim counters: next[0] large, next[32] small (zeroed)
  int norm_l2;
};

// y = A (+) w for V vectors in shared memory; a warp owns R rows at a time,
// its lanes stride over the row's 16-byte chunks, the next chunk of each row
// loading while the current one is consumed.
// w_s is [j][V] and zero past n up to the packed row length, so the zero
// padding of the packed rows contributes exact zeros; y_s is [i - rb][V].
// Half a 16-byte chunk (8 bytes), for the eight-row BF16 product: two
// buffers of eight full chunks do not fit the 128 registers two CTAs per SM
// allow (they spill).
template <int ST>
struct HalfChunk;
template <>
struct HalfChunk<kF32> {
  static constexpr int E = 2;
  uint2 raw;
  __device__ __forceinline__ float get(int e) const { return __uint_as_float(e ? raw.y : raw.x); }
};
template <>
struct HalfChunk<kBF16> {
  static constexpr int E = 4;
  uint2 raw;
  __device__ __forceinline__ float get(int e) const {
    const uint32_t wd = (e >> 1) ? raw.y : raw.x;
    return __uint_as_float((e & 1) ? (wd & 0xFFFF0000u) : (wd << 16));
  }
};
__device__ __forceinline__ uint2 ld_stream8(const void* p) {
  uint2 r;
  asm("ld.global.nc.L1::no_allocate.L2::256B.v2.u32 {%0,%1}, [%2];"
      : "=r"(r.x), "=r"(r.y)
      : "l"(p));
  return r;
}

template <int OP, int ST, int V, int R>
__device__ __forceinline__ void cta_product(const BatchDev& it, const float* __restrict__ w_s,
                                            float* __restrict__ y_s, int rb, int re) {
  // eight BF16 rows: 8-byte half chunks (twice as many, each half the
  // registers; measured 224.5 -> 221 ms per launch of the 4096-instance
  // workload).  FP32 keeps full chunks: its eight-row half-chunk variant lost
  // to the spilling full-chunk one.
  constexpr bool kHalf = R == 8 && ST == kBF16;
  using Ch = typename std::conditional<kHalf, HalfChunk<ST>, Chunk<ST>>::type;
  constexpr int E = Ch::E;
  constexpr int CB = kHalf ? 8 : 16;  // bytes per chunk
  const int nch = it.chunks * (16 / CB);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int row0 = rb + warp * R; row0 < re; row0 += kBatchWarps * R) {
    float acc[R][V];
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
      for (int v = 0; v < V; ++v) acc[r][v] = 0.f;
    const uint8_t* rowp[R];
#pragma unroll
    for (int r = 0; r < R; ++r)
      rowp[r] = it.A + (int64_t)min(row0 + r, re - 1) * it.row_bytes;  // rows past re repeat
    auto load = [&](Ch (&dst)[R], int c) {
#pragma unroll
      for (int r = 0; r < R; ++r) {
        if constexpr (kHalf)
          dst[r].raw = c < nch ? ld_stream8(rowp[r] + (int64_t)c * CB) : make_uint2(0, 0);
        else
          dst[r].raw = c < nch ? ld_stream(rowp[r] + (int64_t)c * CB) : make_uint4(0, 0, 0, 0);
      }
    };
    auto consume = [&](const Ch (&src)[R], int c) {
      // every iterate entry of the chunk's columns is read from shared memory
      // before the first is used, so the reads overlap
      float wv[E][V];
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const int j = c * E + e;
        if constexpr (V == 4) {
          const float4 q = *reinterpret_cast<const float4*>(w_s + j * 4);
          wv[e][0] = q.x;
          wv[e][1] = q.y;
          wv[e][2] = q.z;
          wv[e][3] = q.w;
        } else {
#pragma unroll
          for (int v = 0; v < V; ++v) wv[e][v] = w_s[j * V + v];
        }
      }
#pragma unroll
      for (int e = 0; e < E; ++e) {
#pragma unroll
        for (int v = 0; v < V; ++v) {
          const auto p = Op<OP>::prep(wv[e][v]);
#pragma unroll
          for (int r = 0; r < R; ++r) acc[r][v] = Op<OP>::term(src[r].get(e), p, acc[r][v]);
        }
      }
    };
    // software pipeline: the next chunks of every row are in flight while
    // the current one is consumed (two ahead for R <= 4, one for R = 8)
    if constexpr (R <= 4) {
      Ch b0[R], b1[R], b2[R];
      int c = lane;
      load(b0, c);
      load(b1, c + 32);
      for (; c < nch; c += 96) {
        load(b2, c + 64);
        consume(b0, c);
        if (c + 32 >= nch) break;
        load(b0, c + 96);
        consume(b1, c + 32);
        if (c + 64 >= nch) break;
        load(b1, c + 128);
        consume(b2, c + 64);
      }
    } else {
      Ch b0[R], b1[R];
      int c = lane;
      load(b0, c);
      for (; c < nch; c += 64) {
        load(b1, c + 32);
        consume(b0, c);
        if (c + 32 >= nch) break;
        load(b0, c + 64);
        consume(b1, c + 32);
      }
    }
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
      for (int v = 0; v < V; ++v) {
        float s = acc[r][v];
#pragma unroll
        for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0 && row0 + r < re) y_s[(row0 + r - rb) * V + v] = s;
      }
  }
}

// Per-CTA state of the instance in flight (static shared memory).
struct BatchShared {
  float red[kBatchWarps * 4];
  float part[4], dpart[4], L[4], D[4], dl[4];
  int idx, done[4], it[4], st[4];
};

// Sums V values over the CTA; every thread gets the totals (fixed order).
template <int V>
__device__ __forceinline__ void block_sum_vec(float (&x)[V], float* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int v = 0; v < V; ++v) {
#pragma unroll
    for (int o = 16; o; o >>= 1) x[v] += __shfl_xor_sync(0xffffffffu, x[v], o);
  }
  if (lane == 0) {
#pragma unroll
    for (int v = 0; v < V; ++v) red[warp * V + v] = x[v];
  }
  __syncthreads();
#pragma unroll
  for (int v = 0; v < V; ++v) {
    float t = 0.f;
#pragma unroll
    for (int q = 0; q < kBatchWarps; ++q) t += red[q * V + v];
    x[v] = t;
  }
  __syncthreads();
}

// Alg. 1 on one instance by CS CTAs of a cluster (CS = 1: this CTA alone).
// CTA `crank` owns rows [rb, re) and keeps the whole iterate w_s ([j][V],
// zero past n up to the packed row length); y_s holds its own rows' products.
// A step: products of the own rows; l1 (l2 for DOT) norm partials, summed over
// the cluster in rank order through DSMEM; then every CTA reads all ranks'
// products, divides them by the norm (the n divisions of §2.2) into its
// iterate, and sums the delta over its own rows, combined the same way.
template <int OP, int ST, int V, int R, int CS>
__device__ __forceinline__ void solve_one(const BatchArgs& a, const BatchDev& it, float* w_s,
                                          float* y_s, int crank, BatchShared& sh) {
  cg::cluster_group cluster = cg::this_cluster();
  auto csync = [&]() {
    if constexpr (CS > 1) cluster.sync();
    else __syncthreads();
  };
  auto csum = [&](float* slot) {
    float t = 0.f;
    if constexpr (CS > 1) {
#pragma unroll
      for (int q = 0; q < CS; ++q) t += *cluster.map_shared_rank(slot, q);
    } else {
      t = *slot;
    }
    return t;
  };
  const int n = it.n;
  const int npad = it.chunks * Chunk<ST>::E;
  const int rpc = (n + CS - 1) / CS;
  const int rb = min(n, crank * rpc), re = min(n, rb + rpc);
  // Alg. 1 step 1 per vector (every CTA, the whole vector)
  for (int v = 0; v < V; ++v) {
    Kahan k;
    int bad = 0;
    for (int i = threadIdx.x; i < n; i += kBatchThreads) {
      const float x = it.w0[(int64_t)v * n + i];
      bad |= !isfinite(x);
      k.add(x * x);
    }
    bad = __syncthreads_or(bad);
    const float s = sqrtf(block_sum<kBatchThreads>(k.value(), sh.red));
    const bool scale = !it.raw_start && s > 0.f && !bad;
    for (int i = threadIdx.x; i < n; i += kBatchThreads) {
      const float x = it.w0[(int64_t)v * n + i];
      w_s[i * V + v] = scale ? x / s : x;
    }
    for (int i = n + threadIdx.x; i < npad; i += kBatchThreads) w_s[i * V + v] = 0.f;
    if (threadIdx.x == 0) {
      sh.it[v] = 0;
      sh.st[v] = bad ? MAPI_ENONFINITE : (!it.raw_start && !(s > 0.f)) ? MAPI_EZERONORM : MAPI_OK;
      sh.done[v] = sh.st[v] != MAPI_OK;
      sh.dl[v] = NAN;
    }
  }
  __syncthreads();
  for (int t = 0; t < it.max_iters; ++t) {
    bool any = false;
#pragma unroll
    for (int v = 0; v < V; ++v) any |= !sh.done[v];
    if (!any) break;  // the same decision in every CTA of the cluster
    cta_product<OP, ST, V, R>(it, w_s, y_s, rb, re);
    __syncthreads();
    float p[V];
#pragma unroll
    for (int v = 0; v < V; ++v) p[v] = 0.f;
    for (int i = threadIdx.x; i < re - rb; i += kBatchThreads) {
#pragma unroll
      for (int v = 0; v < V; ++v) {
        const float y = y_s[i * V + v];
        p[v] += a.norm_l2 ? y * y : fabsf(y);
      }
    }
    block_sum_vec<V>(p, sh.red);
    if (threadIdx.x == 0) {
#pragma unroll
      for (int v = 0; v < V; ++v) sh.part[v] = p[v];
    }
    csync();  // norm partials of every rank visible
    if (threadIdx.x < V) {
      const float l = csum(&sh.part[threadIdx.x]);
      sh.L[threadIdx.x] = a.norm_l2 ? sqrtf(l) : l;
    }
    __syncthreads();
    float L[V], d[V];
    bool ok[V];
#pragma unroll
    for (int v = 0; v < V; ++v) {
      L[v] = sh.L[v];
      ok[v] = !sh.done[v] && L[v] > 0.f && isfinite(L[v]);
      d[v] = 0.f;
    }
    for (int q = 0; q < CS; ++q) {
      const float* src = y_s;
      if constexpr (CS > 1) src = cluster.map_shared_rank(y_s, q);
      const int qb = min(n, q * rpc), qe = min(n, qb + rpc);
      const bool own = q == crank;
      for (int i = threadIdx.x; i < qe - qb; i += kBatchThreads) {
        float y[V], w[V];
        if constexpr (V == 4) {
          const float4 y4 = reinterpret_cast<const float4*>(src)[i];
          const float4 w4 = reinterpret_cast<const float4*>(w_s)[qb + i];
          y[0] = y4.x, y[1] = y4.y, y[2] = y4.z, y[3] = y4.w;
          w[0] = w4.x, w[1] = w4.y, w[2] = w4.z, w[3] = w4.w;
        } else {
#pragma unroll
          for (int v = 0; v < V; ++v) y[v] = src[i * V + v], w[v] = w_s[(qb + i) * V + v];
        }
#pragma unroll
        for (int v = 0; v < V; ++v) {
          const float x = ok[v] ? y[v] / L[v] : w[v];
          if (own) d[v] += fabsf(x - w[v]);
          w[v] = x;
        }
        if constexpr (V == 4) {
          reinterpret_cast<float4*>(w_s)[qb + i] = make_float4(w[0], w[1], w[2], w[3]);
        } else {
#pragma unroll
          for (int v = 0; v < V; ++v) w_s[(qb + i) * V + v] = w[v];
        }
      }
    }
    block_sum_vec<V>(d, sh.red);
    if (threadIdx.x == 0) {
#pragma unroll
      for (int v = 0; v < V; ++v) sh.dpart[v] = d[v];
    }
    csync();  // every rank has read the products; delta partials visible
    if (threadIdx.x < V) sh.D[threadIdx.x] = csum(&sh.dpart[threadIdx.x]);
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
      for (int v = 0; v < V; ++v) {
        if (sh.done[v]) continue;
        if (!ok[v]) {
          sh.st[v] = (L[v] == 0.f) ? MAPI_EZERONORM : MAPI_ENONFINITE;
          sh.done[v] = 1;
          continue;
        }
        sh.it[v] += 1;
        sh.dl[v] = sh.D[v];
        if (it.tol > 0.f && sh.D[v] < it.tol) sh.done[v] = 1;
      }
    }
    __syncthreads();
  }
  // Alg. 1 step 6 (optional, once the solve ends) and the results (own rows)
  bool ends = it.last != 0;
  {
    bool all = true;
#pragma unroll
    for (int v = 0; v < V; ++v) all = all && sh.done[v];
    ends = ends || all;
  }
  for (int v = 0; v < V; ++v) {
    float s = 1.f;
    if (it.final_l2 && ends && sh.st[v] == MAPI_OK) {
      Kahan k;
      for (int i = threadIdx.x; i < n; i += kBatchThreads) {
        const float x = w_s[i * V + v];
        k.add(x * x);
      }
      s = sqrtf(block_sum<kBatchThreads>(k.value(), sh.red));
      if (!(s > 0.f)) s = 1.f;
    }
    for (int i = rb + threadIdx.x; i < re; i += kBatchThreads)
      it.w_out[(int64_t)v * n + i] = (s == 1.f) ? w_s[i * V + v] : w_s[i * V + v] / s;
    if (crank == 0 && threadIdx.x == 0) {
      it.res[2 * v] = sh.it[v];
      it.res[2 * v + 1] = sh.st[v];
      it.delta[v] = sh.dl[v];
    }
  }
  csync();  // no rank touches this instance's shared memory any more
}

// Phase 1: a cluster per large instance; phase 2: a CTA per small instance.
template <int OP, int ST, int V, int R>
__global__ void __launch_bounds__(kBatchThreads, 2) k_batched(BatchArgs a) {
  extern __shared__ float4 bsh4[];
  float* bsh = reinterpret_cast<float*>(bsh4);
  __shared__ BatchShared sh;
  cg::cluster_group cluster = cg::this_cluster();
  const int crank = (int)cluster.block_rank();
  for (;;) {
    if (crank == 0 && threadIdx.x == 0) {
      const int k = atomicAdd(&a.next[0], 1);
      const int idx = k < a.nlarge ? a.order[k] : -1;
#pragma unroll
      for (int q = 0; q < kBatchCluster; ++q) *cluster.map_shared_rank(&sh.idx, q) = idx;
    }
    cluster.sync();
    const int idx = sh.idx;
    if (idx < 0) break;
    // w_s: whole iterate; y_s: own rows
    solve_one<OP, ST, V, R, kBatchCluster>(a, a.items[idx], bsh, bsh + kBatchIterFloats, crank,
                                           sh);
  }
  const int nsmall = a.count - a.nlarge;
  for (;;) {
    __syncthreads();  // sh.idx of the previous claim has been read
    if (threadIdx.x == 0) {
      const int k = atomicAdd(&a.next[32], 1);
      sh.idx = k < nsmall ? a.order[a.nlarge + k] : -1;
    }
    __syncthreads();
    const int idx = sh.idx;
    if (idx < 0) return;
    // n < kBatchLargeN: w_s and y_s of kBatchLargeN x V each
    solve_one<OP, ST, V, R, 1>(a, a.items[idx], bsh, bsh + kBatchLargeN * V, 0, sh);
  }
}

using BatchFn = void (*)(BatchArgs);

template <int OP, int ST, int V>
static BatchFn pick_r(int r) {
  switch (r) {
    case 1: return k_batched<OP, ST, V, 1>;
    case 2: return k_batched<OP, ST, V, 2>;
    case 4: return k_batched<OP, ST, V, 4>;
    case 8: return k_batched<OP, ST, V, 8>;
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
  explicit DeviceGuardB(int d) {
    if (cudaGetDevice(&prev) == cudaSuccess && prev != d) cudaSetDevice(d);
  }
  ~DeviceGuardB() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

struct BatchLaunch {
  BatchFn fn = nullptr;
  int nclusters = 0;
};

// Attributes and grid of one batched launch (host queries; before any
// capture): as many 8-CTA clusters as fit, at most enough for the large
// instances plus a CTA per small one.
mapi_status plan_batched(mapi_ctx* ctx, mapi_op op, mapi_storage st, int V, int r,
                         const BatchArgs& args, BatchLaunch* bl) {
  bl->fn = batched_fn(op, st, V, r);
  if (!bl->fn) return fail(ctx, MAPI_EINVAL, "batched solve: op/storage/nvec not supported");
  // whole iterate + a cluster rank's rows; the small phase uses 2 x kBatchLargeN x V
  static_assert(2 * kBatchLargeN * 4 <= kBatchIterFloats + kBatchRowFloats, "small phase");
  const size_t smem = sizeof(float) * (kBatchIterFloats + kBatchRowFloats);
  MAPI_CUDA_TRY(ctx, cudaFuncSetAttribute((const void*)bl->fn,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = kBatchCluster;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.blockDim = dim3(kBatchThreads, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cfg.gridDim = dim3(kBatchCluster * ctx->sm_count, 1, 1);
  int nclusters = 0;
  MAPI_CUDA_TRY(ctx, cudaOccupancyMaxActiveClusters(&nclusters, (const void*)bl->fn, &cfg));
  if (nclusters < 1) return fail(ctx, MAPI_ECUDA, "batched kernel does not fit");
  const int want = args.nlarge + (args.count - args.nlarge + kBatchCluster - 1) / kBatchCluster;
  bl->nclusters = std::min(nclusters, std::max(1, want));
  return MAPI_OK;
}

// The claim counters' reset and the persistent launch, on stream s.
mapi_status enqueue_batched(mapi_ctx* ctx, const BatchLaunch& bl, const BatchArgs& args,
                            cudaStream_t s, double args_bytes, double args_terms) {
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = kBatchCluster;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.blockDim = dim3(kBatchThreads, 1, 1);
  cfg.dynamicSmemBytes = sizeof(float) * (kBatchIterFloats + kBatchRowFloats);
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cfg.gridDim = dim3(kBatchCluster * bl.nclusters, 1, 1);
  MAPI_CUDA_TRY(ctx, cudaMemsetAsync(args.next, 0, 64 * sizeof(int), s));
  cudaEvent_t ev = prof_begin(ctx, s);
  MAPI_CUDA_TRY(ctx, cudaLaunchKernelEx(&cfg, bl.fn, args));
  prof_end(ctx, s, ev, MAPI_KC_BATCHED, args_bytes, args_terms);
  count_launch(ctx);
  return MAPI_OK;
}

}  // namespace

namespace mapi {

// One launch over host-described instances (all of `st`, each with its own
// step count, stop rule and start mode); per-vector iterations, statuses and
// last deltas come back in res ([iters, status] per vector) and dl.
mapi_status batched_run(mapi_ctx* ctx, cudaStream_t stream, std::vector<BatchDev>& host,
                        mapi_op op, mapi_storage st, int V, std::vector<int>& res,
                        std::vector<float>& dl, bool use_graph) {
  // a cached graph is launched on the context's stream
  use_graph = use_graph && stream == ctx->stream;
  const int count = (int)host.size();
  std::vector<int64_t> work(count);
  for (int i = 0; i < count; ++i) work[i] = (int64_t)host[i].n * host[i].n;
  // largest instances first
  std::vector<int> order(count);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return work[x] > work[y]; });
  // device table: items, order, counters, results
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
  MAPI_CUDA_TRY(ctx, cudaMemcpyAsync(d_items, host.data(), items_b, cudaMemcpyHostToDevice, stream));
  MAPI_CUDA_TRY(ctx, cudaMemcpyAsync(d_order, order.data(), order_b, cudaMemcpyHostToDevice, stream));
  // instances of n >= kBatchLargeN (a cluster each) lead `order`
  int nlarge = 0;
  while (nlarge < count && host[order[nlarge]].n >= kBatchLargeN) ++nlarge;
  BatchArgs a;
  a.items = d_items;
  a.order = d_order;
  a.count = count;
  a.nlarge = nlarge;
  a.next = d_next;
  a.norm_l2 = (op == MAPI_OP_DOT) ? 1 : 0;
  const int r = ctx->batch_rows_per_warp[st == MAPI_ST_F32 ? 0 : 1][V == 1 ? 0 : 1];
  // algorithmic work if every vector runs all its steps: each matrix read
  // once per step, n^2 terms per vector per step
  double bytes = 0.0, terms = 0.0;
  for (int i = 0; i < count; ++i) {
    bytes += (double)work[i] * elem_bytes(st) * host[i].max_iters;
    terms += (double)work[i] * V * host[i].max_iters;
  }
  BatchLaunch bl;
  if ((s = plan_batched(ctx, op, st, V, r > 0 ? r : 2, a, &bl)) != MAPI_OK) return s;
  GraphEntry* ge = nullptr;
  if (use_graph) {
    // the counters' reset and the persistent launch as one cached graph,
    // replayed while the instance table keeps its shape (the table itself
    // is copied in ahead of it on the same stream)
    std::vector<int64_t> key = {3, (int64_t)op, (int64_t)st, V, r, count, nlarge,
                                bl.nclusters, (int64_t)(uintptr_t)ctx->batch.p,
                                (int64_t)ctx->prof_on};
    if (ctx->prof_on) {  // the work counted per launch feeds only the profile
      uint64_t bb, tb;
      std::memcpy(&bb, &bytes, 8);
      std::memcpy(&tb, &terms, 8);
      key.push_back((int64_t)bb);
      key.push_back((int64_t)tb);
    }
    s = launch_cached_graph(
        ctx, key, [&](cudaStream_t cs) { return enqueue_batched(ctx, bl, a, cs, bytes, terms); },
        &ge);
  } else {
    s = enqueue_batched(ctx, bl, a, stream, bytes, terms);
  }
  if (s != MAPI_OK) return s;
  res.assign(2 * V * count, 0);
  dl.assign(V * count, 0.f);
  MAPI_CUDA_TRY(ctx, cudaMemcpyAsync(res.data(), d_res, res_b, cudaMemcpyDeviceToHost, stream));
  MAPI_CUDA_TRY(ctx, cudaMemcpyAsync(dl.data(), d_dl, dl_b, cudaMemcpyDeviceToHost, stream));
  MAPI_CUDA_TRY(ctx, cudaStreamSynchronize(stream));
  if (ge) finish_graph(ctx, ge);
  else prof_collect(ctx, ctx->pending, true);
  return MAPI_OK;
}

int batched_max_n(int nvec) { return kBatchIterFloats / pow2v(nvec); }

}  // namespace mapi

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
  const int V = pow2v(nvec);
  const int nmax = batched_max_n(nvec);
  mapi_storage st = MAPI_ST_F32;
  std::vector<BatchDev> host(count);
  for (int i = 0; i < count; ++i) {
    const mapi_mat* A = items[i].A;
    if (!A || !ctx->mats.count(const_cast<mapi_mat*>(A)) || !items[i].w0 || !items[i].w_out)
      return fail(ctx, MAPI_EINVAL, "batch item " + std::to_string(i) + ": bad pointers");
    if (A->rows != A->cols || A->rows > nmax)
      return fail(ctx, MAPI_EINVAL,
                  "batch items must be square with n <= " + std::to_string(nmax));
    if (i == 0) st = A->storage;
    if (A->storage != st || (st != MAPI_ST_F32 && st != MAPI_ST_BF16))
      return fail(ctx, MAPI_EINVAL, "one F32 or BF16 storage per batch");
    BatchDev& h = host[i];
    h.A = (const uint8_t*)A->data;
    h.row_bytes = A->ld * elem_bytes(A->storage);
    h.n = A->rows;
    h.chunks = (int)(h.row_bytes / 16);
    h.w0 = items[i].w0;
    h.w_out = items[i].w_out;
    h.max_iters = max_iters;
    h.tol = (float)tol_l1;
    h.raw_start = (flags & MAPI_FLAG_RAW_START) ? 1 : 0;
    h.final_l2 = (flags & MAPI_FLAG_FINAL_L2) ? 1 : 0;
    h.last = 1;
  }
  std::vector<int> res;
  std::vector<float> dl;
  mapi_status s = batched_run(ctx, ctx->stream, host, op, st, V, res, dl, true);
  if (s != MAPI_OK) return s;
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

extern "C" mapi_status mapi_set_batched_rows(mapi_ctx* ctx, mapi_storage storage, int nvec,
                                             int rows_per_warp) {
  if (!ctx) return MAPI_EINVAL;
  if (storage != MAPI_ST_F32 && storage != MAPI_ST_BF16)
    return fail(ctx, MAPI_EINVAL, "batched rows: F32 or BF16 storage");
  if (nvec < 1 || nvec > 8) return fail(ctx, MAPI_EINVAL, "batched rows: nvec in [1, 8]");
  if (rows_per_warp != 1 && rows_per_warp != 2 && rows_per_warp != 4 && rows_per_warp != 8)
    return fail(ctx, MAPI_EINVAL, "batched rows: 1, 2, 4 or 8");
  const int V = pow2v(nvec);
  ctx->batch_rows_per_warp[storage == MAPI_ST_F32 ? 0 : 1][V == 1 ? 0 : 1] = rows_per_warp;
  return MAPI_OK;
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
  for (int r : {1, 2, 4, 8}) {
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
