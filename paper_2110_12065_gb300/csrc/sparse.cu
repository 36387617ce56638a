// MAPI-PageRank on the Google matrix of Eq. (11) without forming it (§3.3).
//
// Every entry of column j of G is one of a few values: the teleport value
// g0 = alpha * 0 + (1 - alpha)/n where j does not link to i, alpha * acc + g0
// where it does (acc = 1/d_j per link), and gd = alpha * (1/n) + g0 in a
// dangling column (all formed in FP64 in that order, then rounded to FP32:
// the values the dense FP32 copy of G holds).  Row i of G (+) w is therefore
//   S + sum over the in-links j of i of [ term(g_ij, w_j) - term(g0, w_j) ],
//   S = sum_j term(b_j, w_j),  b_j = gd (dangling j) or g0,
// which costs O(E + n) per step instead of O(n^2).
//
// Built once per call: the in-link lists (counting sort by target, each list
// sorted by source, repeated links merged into one entry with their value)
// and the list of long rows.  Per step, two kernels:
//   k_sp_form  (one thread per node): this step's iterate w_t = y / ||y||
//              from the last step (or the start vector), delta, stop test,
//              and the base sum S; the last CTA adds the block partials in
//              block order;
//   k_sp_rows  (one thread per short row, one warp per long row): y_i, and
//              the norm, again reduced in block order by the last CTA.
#include <algorithm>
#include <climits>
#include <cstring>

#include "device_common.cuh"

namespace mapi {
namespace {

constexpr int kSpThreads = 256;
constexpr int kSpLong = 32;        // rows with more in-links go to a warp
constexpr int kSpSortThread = 64;  // rows up to this many in-links sort in one thread
constexpr int kSpSortMax = 16384;  // longest in-link list sorted in shared memory
constexpr int kSpBatch = 8;        // in-links of a short row loaded together
constexpr int kSpHuge = 1024;      // rows with more in-links go to a whole CTA

struct SpCtl {
  unsigned counter_a, counter_b;
  int status, done, iters, bad;
  float delta, S, L, s2;
};

struct SpGraph {
  int n;
  const int* deg;     // out-degrees
  const int* inptr;   // n + 1
  const int* src;     // in-link sources (-1: merged into the previous entry)
  const float* val;   // entry values g_ij
  const int* longrows;  // rows with kSpLong < in-links <= kSpHuge, ascending
  int nlong;
  const int* hugerows;  // rows with more than kSpHuge in-links, ascending
  int nhuge;
  float g0, gd;
};

// ------------------------------------------------------------ construction
__global__ void k_sp_count(const int* __restrict__ indptr, const int* __restrict__ indices, int n,
                           int nnz, int* __restrict__ deg, int* __restrict__ incount,
                           SpCtl* ctl) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
    const int b = indptr[j], e = indptr[j + 1];
    if (b < 0 || e < b || e > nnz) {
      ctl->bad = 1;
      deg[j] = 0;
      continue;
    }
    deg[j] = e - b;
    for (int q = b; q < e; ++q) {
      const int i = indices[q];
      if (i < 0 || i >= n) {
        ctl->bad = 1;
        continue;
      }
      atomicAdd(&incount[i], 1);
    }
  }
}

// Exclusive scan of n counts into out (n + 1 entries), in three passes: the
// sum of each CTA's contiguous chunk; one CTA scans those sums; each CTA
// scans its chunk in tiles of kSpThreads from its offset.
__global__ void __launch_bounds__(kSpThreads) k_scan_sums(const int* __restrict__ cnt, int n,
                                                         int chunk, long long* __restrict__ bsum) {
  __shared__ long long sh[kSpThreads / 32];
  const long long b = (long long)blockIdx.x * chunk;
  const long long e = std::min<long long>(n, b + chunk);
  long long s = 0;
  for (long long i = b + threadIdx.x; i < e; i += kSpThreads) s += cnt[i];
#pragma unroll
  for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    long long t = 0;
    for (int q = 0; q < kSpThreads / 32; ++q) t += sh[q];
    bsum[blockIdx.x] = t;
  }
}

__global__ void __launch_bounds__(1024) k_scan_blocks(long long* __restrict__ bsum, int nb) {
  __shared__ long long part[1024];
  const int t = threadIdx.x;
  long long carry = 0;
  for (int base = 0; base < nb; base += 1024) {
    const long long v = base + t < nb ? bsum[base + t] : 0;
    part[t] = v;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
      const long long u = t >= o ? part[t - o] : 0;
      __syncthreads();
      part[t] += u;
      __syncthreads();
    }
    if (base + t < nb) bsum[base + t] = carry + part[t] - v;  // exclusive
    const long long tot = part[1023];
    __syncthreads();
    carry += tot;
  }
}

__global__ void __launch_bounds__(kSpThreads) k_scan_final(const int* __restrict__ cnt, int n,
                                                          int chunk,
                                                          const long long* __restrict__ bsum,
                                                          int* __restrict__ out) {
  __shared__ long long part[kSpThreads];
  const long long b = (long long)blockIdx.x * chunk;
  const long long e = std::min<long long>(n, b + chunk);
  long long carry = bsum[blockIdx.x];
  const int t = threadIdx.x;
  for (long long base = b; base < e; base += kSpThreads) {
    const long long v = base + t < e ? cnt[base + t] : 0;
    part[t] = v;
    __syncthreads();
    for (int o = 1; o < kSpThreads; o <<= 1) {
      const long long u = t >= o ? part[t - o] : 0;
      __syncthreads();
      part[t] += u;
      __syncthreads();
    }
    if (base + t < e) out[base + t] = (int)(carry + part[t] - v);
    const long long tot = part[kSpThreads - 1];
    __syncthreads();
    carry += tot;
  }
  if (e == n && b < e && t == 0) out[n] = (int)carry;
}

__global__ void k_sp_fill(const int* __restrict__ indptr, const int* __restrict__ indices, int n,
                          const int* __restrict__ inptr, int* __restrict__ fill,
                          int* __restrict__ src, const SpCtl* ctl) {
  if (ctl->bad) return;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
    for (int q = indptr[j]; q < indptr[j + 1]; ++q) {
      const int i = indices[q];
      src[inptr[i] + atomicAdd(&fill[i], 1)] = j;
    }
  }
}

// The entry value of a merged run of `cnt` links from j (FP64 as the dense
// builder forms it, then FP32).
__device__ __forceinline__ float sp_value(int cnt, int d, double alpha, double tele) {
  double acc = 0.0;
  for (int k = 0; k < cnt; ++k) acc += 1.0 / (double)d;
  return (float)(alpha * acc + tele);
}

// Sorted list [b, e) of sources: merge runs, write values.
__device__ __forceinline__ void sp_merge_run(int* src, float* val, int p, int e, const int* deg,
                                             double alpha, double tele) {
  const int j = src[p];
  int q = p + 1;
  while (q < e && src[q] == j) {
    src[q] = -1;
    ++q;
  }
  val[p] = sp_value(q - p, deg[j], alpha, tele);
}

// Short lists: one thread each (insertion sort); long ones are queued.
__global__ void k_sp_sort_short(int n, const int* __restrict__ inptr, int* __restrict__ src,
                                float* __restrict__ val, const int* __restrict__ deg,
                                double alpha, double tele, int* __restrict__ sortq, SpCtl* ctl) {
  if (ctl->bad) return;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int b = inptr[i], e = inptr[i + 1];
    if (e - b > kSpSortThread) {
      sortq[4 + atomicAdd(&sortq[0], 1)] = i;
      continue;
    }
    for (int p = b + 1; p < e; ++p) {
      const int x = src[p];
      int q = p - 1;
      while (q >= b && src[q] > x) {
        src[q + 1] = src[q];
        --q;
      }
      src[q + 1] = x;
    }
    for (int p = b; p < e; ++p)
      if (src[p] >= 0) sp_merge_run(src, val, p, e, deg, alpha, tele);
  }
}

// Row classes by in-link count: flags for the two ordered lists.
__global__ void k_sp_flags(int n, const int* __restrict__ inptr, int* __restrict__ fl,
                           int* __restrict__ fh) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int d = inptr[i + 1] - inptr[i];
    fl[i] = (d > kSpLong && d <= kSpHuge) ? 1 : 0;
    fh[i] = d > kSpHuge ? 1 : 0;
  }
}

// The rows of each class in ascending order (positions from the scans).
__global__ void k_sp_lists(int n, const int* __restrict__ inptr, const int* __restrict__ pl,
                           const int* __restrict__ ph, int* __restrict__ longrows,
                           int* __restrict__ hugerows) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int d = inptr[i + 1] - inptr[i];
    if (d > kSpLong && d <= kSpHuge) longrows[pl[i]] = i;
    if (d > kSpHuge) hugerows[ph[i]] = i;
  }
}

// Long lists: one CTA each, bitonic sort in shared memory.
__global__ void __launch_bounds__(1024) k_sp_sort_long(const int* __restrict__ inptr,
                                                       int* __restrict__ src,
                                                       float* __restrict__ val,
                                                       const int* __restrict__ deg, double alpha,
                                                       double tele, const int* __restrict__ sortq,
                                                       SpCtl* ctl) {
  extern __shared__ int key[];
  const int nq = sortq[0];
  for (int r = blockIdx.x; r < nq; r += gridDim.x) {
    const int i = sortq[4 + r];
    const int b = inptr[i], e = inptr[i + 1], len = e - b;
    if (len > kSpSortMax) {
      if (threadIdx.x == 0) ctl->bad = 2;
      continue;
    }
    int m = 1;
    while (m < len) m <<= 1;
    for (int p = threadIdx.x; p < m; p += blockDim.x) key[p] = p < len ? src[b + p] : INT_MAX;
    __syncthreads();
    for (int k = 2; k <= m; k <<= 1)
      for (int jj = k >> 1; jj > 0; jj >>= 1) {
        for (int p = threadIdx.x; p < m; p += blockDim.x) {
          const int q = p ^ jj;
          if (q > p) {
            const bool up = (p & k) == 0;
            const int a = key[p], c = key[q];
            if ((a > c) == up) {
              key[p] = c;
              key[q] = a;
            }
          }
        }
        __syncthreads();
      }
    for (int p = threadIdx.x; p < len; p += blockDim.x) src[b + p] = key[p];
    __syncthreads();
    // merge runs: a run starts where the source changes
    for (int p = threadIdx.x; p < len; p += blockDim.x) {
      if (p > 0 && key[p] == key[p - 1]) {
        src[b + p] = -1;
        continue;
      }
      int q = p + 1;
      while (q < len && key[q] == key[p]) ++q;
      val[b + p] = sp_value(q - p, deg[key[p]], alpha, tele);
    }
    __syncthreads();
  }
}

// --------------------------------------------------------------- iteration
// Step start: w_t and, per node, (w_j, term(g0, w_j)) for the row kernel;
// the base sum S; delta and the stop test.  t = 0 takes the scaled start
// vector.  final_pass: the last iterate, whose l2 norm (Alg. 1's optional
// last step) is also summed.
template <int OP>
__global__ void __launch_bounds__(kSpThreads)
    k_sp_form(SpGraph g, const float* __restrict__ y, const float* __restrict__ w_prev,
              float* __restrict__ w_out, float2* __restrict__ wt, float* __restrict__ part,
              int first, int final_pass, float tol, SpCtl* ctl) {
  if (*(volatile int*)&ctl->done) return;
  __shared__ float sh[33];
  const float L = first ? 1.f : ctl->L;
  Kahan ks, kd, k2;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < g.n; j += gridDim.x * blockDim.x) {
    const float x = first ? w_prev[j] : y[j] / L;  // the n divisions of §2.2
    if (!first) kd.add(fabsf(x - w_prev[j]));
    w_out[j] = x;
    const float b = g.deg[j] == 0 ? g.gd : g.g0;
    ks.add(Op<OP>::term(b, Op<OP>::prep(x), 0.f));
    wt[j] = make_float2(x, Op<OP>::term(g.g0, Op<OP>::prep(x), 0.f));
    if (final_pass) k2.add(x * x);
  }
  const float ps = block_sum<kSpThreads>(ks.value(), sh);
  const float pd = block_sum<kSpThreads>(kd.value(), sh);
  const float p2 = block_sum<kSpThreads>(k2.value(), sh);
  if (threadIdx.x == 0) {
    part[3 * blockIdx.x] = ps;
    part[3 * blockIdx.x + 1] = pd;
    part[3 * blockIdx.x + 2] = p2;
  }
  if (!elect_last_cta(&ctl->counter_a, gridDim.x)) return;
  Kahan s, d, q;
  for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) {
    s.add(__ldcg(&part[3 * b]));
    d.add(__ldcg(&part[3 * b + 1]));
    q.add(__ldcg(&part[3 * b + 2]));
  }
  const float S = block_sum<kSpThreads>(s.value(), sh);
  const float Dsum = block_sum<kSpThreads>(d.value(), sh);
  const float Q = block_sum<kSpThreads>(q.value(), sh);
  if (threadIdx.x == 0) {
    ctl->S = S;
    ctl->s2 = sqrtf(Q);
    if (!first) {
      ctl->iters += 1;
      ctl->delta = Dsum;
      if (tol > 0.f && Dsum < tol) ctl->done = 1;
    }
    ctl->counter_a = 0;
    __threadfence();
  }
}

// y_i = S + sum over the merged in-links (j, g_ij) of term(g_ij, w_j) -
// term(g0, w_j); then ||y||_1 (||y||_2 for DOT).
template <int OP>
__global__ void __launch_bounds__(kSpThreads)
    k_sp_rows(SpGraph g, const float2* __restrict__ wt, float* __restrict__ y,
              float* __restrict__ part, int norm_l2, SpCtl* ctl) {
  if (*(volatile int*)&ctl->done) return;
  __shared__ float sh[33];
  const float S = ctl->S;
  Kahan kn;
  // short rows: one thread each, in source order
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < g.n; i += gridDim.x * blockDim.x) {
    const int b = g.inptr[i], e = g.inptr[i + 1];
    if (e - b > kSpLong) continue;
    float c = 0.f;
    // kSpBatch in-links at a time: their sources and values, then their
    // gathers, all in flight before any is used (the order of the sum is
    // the in-link order)
    for (int q0 = b; q0 < e; q0 += kSpBatch) {
      int jv[kSpBatch];
      float gv[kSpBatch];
#pragma unroll
      for (int k = 0; k < kSpBatch; ++k) {
        jv[k] = q0 + k < e ? __ldg(&g.src[q0 + k]) : -1;
        gv[k] = q0 + k < e ? __ldg(&g.val[q0 + k]) : 0.f;
      }
      float2 wv[kSpBatch];
#pragma unroll
      for (int k = 0; k < kSpBatch; ++k) wv[k] = jv[k] >= 0 ? wt[jv[k]] : make_float2(0.f, 0.f);
#pragma unroll
      for (int k = 0; k < kSpBatch; ++k)
        if (jv[k] >= 0) c += Op<OP>::term(gv[k], Op<OP>::prep(wv[k].x), 0.f) - wv[k].y;
    }
    const float yi = S + c;
    y[i] = yi;
    kn.add(norm_l2 ? yi * yi : fabsf(yi));
  }
  // long rows: one warp each, lanes over the sources (four per lane in
  // flight), fixed butterfly
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  auto lane_sum = [&](int b, int e, int first, int stride) {
    float c = 0.f;
    for (int q0 = b + first; q0 < e; q0 += 4 * stride) {
      int jv[4];
      float gv[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int q = q0 + k * stride;
        jv[k] = q < e ? __ldg(&g.src[q]) : -1;
        gv[k] = q < e ? __ldg(&g.val[q]) : 0.f;
      }
      float2 wv[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) wv[k] = jv[k] >= 0 ? wt[jv[k]] : make_float2(0.f, 0.f);
#pragma unroll
      for (int k = 0; k < 4; ++k)
        if (jv[k] >= 0) c += Op<OP>::term(gv[k], Op<OP>::prep(wv[k].x), 0.f) - wv[k].y;
    }
    return c;
  };
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  for (int r = gw; r < g.nlong; r += nw) {
    const int i = g.longrows[r];
    float c = lane_sum(g.inptr[i], g.inptr[i + 1], lane, 32);
#pragma unroll
    for (int o = 16; o; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    const float yi = S + c;
    if (lane == 0) {
      y[i] = yi;
      kn.add(norm_l2 ? yi * yi : fabsf(yi));
    }
  }
  // huge rows: one CTA each, threads over the sources, warp then CTA sums in
  // a fixed order
  __shared__ float hw[kSpThreads / 32];
  for (int r = blockIdx.x; r < g.nhuge; r += gridDim.x) {
    const int i = g.hugerows[r];
    float c = lane_sum(g.inptr[i], g.inptr[i + 1], threadIdx.x, kSpThreads);
#pragma unroll
    for (int o = 16; o; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if (lane == 0) hw[warp] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
      float t = 0.f;
#pragma unroll
      for (int q = 0; q < kSpThreads / 32; ++q) t += hw[q];
      const float yi = S + t;
      y[i] = yi;
      kn.add(norm_l2 ? yi * yi : fabsf(yi));
    }
    __syncthreads();
  }
  const float pn = block_sum<kSpThreads>(kn.value(), sh);
  if (threadIdx.x == 0) part[blockIdx.x] = pn;
  if (!elect_last_cta(&ctl->counter_b, gridDim.x)) return;
  Kahan s;
  for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) s.add(__ldcg(&part[b]));
  float L = block_sum<kSpThreads>(s.value(), sh);
  if (norm_l2) L = sqrtf(L);
  if (threadIdx.x == 0) {
    ctl->L = L;
    if (!(L > 0.f) || !isfinite(L)) {
      ctl->status = (L == 0.f) ? MAPI_EZERONORM : MAPI_ENONFINITE;
      ctl->done = 1;
    }
    ctl->counter_b = 0;
    __threadfence();
  }
}

// Start vector: w0 / ||w0||_2 (Alg. 1 step 1), one CTA.
__global__ void __launch_bounds__(1024) k_sp_start(const float* __restrict__ w0, int n,
                                                   float* __restrict__ w, SpCtl* ctl) {
  __shared__ float sh[33];
  Kahan k;
  int bad = 0;
  for (int i = threadIdx.x; i < n; i += 1024) {
    const float x = w0[i];
    bad |= !isfinite(x);
    k.add(x * x);
  }
  bad = __syncthreads_or(bad);
  const float s = sqrtf(block_sum<1024>(k.value(), sh));
  const bool ok = !bad && s > 0.f;
  for (int i = threadIdx.x; i < n; i += 1024) w[i] = ok ? w0[i] / s : w0[i];
  if (threadIdx.x == 0) {
    ctl->status = bad ? MAPI_ENONFINITE : ok ? MAPI_OK : MAPI_EZERONORM;
    ctl->done = ok ? 0 : 1;
    ctl->iters = 0;
    ctl->delta = NAN;
  }
}

// Output: the final iterate scaled to unit l2 norm (skipped after a failure).
__global__ void k_sp_out(const float* __restrict__ w, int n, float* __restrict__ out,
                         const SpCtl* ctl) {
  const float s = (ctl->status == MAPI_OK && ctl->s2 > 0.f) ? ctl->s2 : 1.f;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    out[i] = (s == 1.f) ? w[i] : w[i] / s;
}

// Final pass when the solve stopped early: the l2 norm of the kept iterate.
__global__ void __launch_bounds__(1024) k_sp_norm2(const float* __restrict__ w, int n,
                                                   SpCtl* ctl) {
  __shared__ float sh[33];
  Kahan k;
  for (int i = threadIdx.x; i < n; i += 1024) k.add(w[i] * w[i]);
  const float s = sqrtf(block_sum<1024>(k.value(), sh));
  if (threadIdx.x == 0) ctl->s2 = s;
}

// out[0 .. n] = exclusive scan of cnt[0 .. n), out[n] the total.
mapi_status sp_scan(mapi_ctx* ctx, cudaStream_t s, const int* cnt, int n, int* out,
                    long long* bsum, int nb) {
  const int chunk = (n + nb - 1) / nb;
  const int used = (n + chunk - 1) / chunk;
  k_scan_sums<<<used, kSpThreads, 0, s>>>(cnt, n, chunk, bsum);
  MAPI_CUDA_TRY(ctx, cudaGetLastError());
  k_scan_blocks<<<1, 1024, 0, s>>>(bsum, used);
  MAPI_CUDA_TRY(ctx, cudaGetLastError());
  k_scan_final<<<used, kSpThreads, 0, s>>>(cnt, n, chunk, bsum, out);
  MAPI_CUDA_TRY(ctx, cudaGetLastError());
  count_launch(ctx, 3);
  return MAPI_OK;
}

template <int OP>
mapi_status sp_solve(mapi_ctx* ctx, cudaStream_t s, const SpGraph& g, float* wb0, float* wb1,
                     float* y, float2* wt, float* part, SpCtl* ctl, int grid, int max_iters,
                     float tol, int norm_l2, double step_bytes) {
  float* wb[2] = {wb0, wb1};
  // step t forms w_t into wb[t & 1] (t = 0: the scaled start vector in wb0)
  for (int t = 0; t <= max_iters; ++t) {
    const bool first = t == 0, last = t == max_iters;
    k_sp_form<OP><<<grid, kSpThreads, 0, s>>>(g, y, first ? wb[0] : wb[(t + 1) & 1], wb[t & 1],
                                              wt, part, first ? 1 : 0, last ? 1 : 0, tol, ctl);
    MAPI_CUDA_TRY(ctx, cudaGetLastError());
    count_launch(ctx);
    if (last) break;
    cudaEvent_t ev = prof_begin(ctx, s);
    k_sp_rows<OP><<<grid, kSpThreads, 0, s>>>(g, wt, y, part, norm_l2, ctl);
    MAPI_CUDA_TRY(ctx, cudaGetLastError());
    prof_end(ctx, s, ev, MAPI_KC_GEMV, step_bytes, 0.0);
    count_launch(ctx);
  }
  return MAPI_OK;
}

struct DeviceGuardS {
  int prev = -1;
  explicit DeviceGuardS(int d) {
    if (cudaGetDevice(&prev) == cudaSuccess && prev != d) cudaSetDevice(d);
  }
  ~DeviceGuardS() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

}  // namespace
}  // namespace mapi

using namespace mapi;

extern "C" mapi_status mapi_pagerank_sparse(mapi_ctx* ctx, const int* indptr, const int* indices,
                                            int n, double alpha, mapi_op op, const float* w0,
                                            int max_iters, double tol_l1, float* rank_out,
                                            int* iters_done, double* last_delta) {
  if (!ctx) return MAPI_EINVAL;
  if (!indptr || !w0 || !rank_out || n < 1 || max_iters < 0)
    return fail(ctx, MAPI_EINVAL, "bad argument");
  if (!(alpha >= 0.0 && alpha <= 1.0)) return fail(ctx, MAPI_EINVAL, "alpha outside [0, 1]");
  if (op != MAPI_OP_MIN1 && op != MAPI_OP_MIN2 && op != MAPI_OP_DOT)
    return fail(ctx, MAPI_EINVAL, "sparse PageRank takes MIN1, MIN2 or DOT");
  DeviceGuardS guard(ctx->device);
  cudaStream_t s = ctx->stream;
  int nnz = 0;
  MAPI_CUDA_TRY(ctx, cudaMemcpyAsync(&nnz, indptr + n, sizeof(int), cudaMemcpyDeviceToHost, s));
  MAPI_CUDA_TRY(ctx, cudaStreamSynchronize(s));
  if (nnz < 0) return fail(ctx, MAPI_EINVAL, "indptr[n] < 0");
  if (nnz > 0 && !indices) return fail(ctx, MAPI_EINVAL, "null indices");
  const int grid = std::max(1, std::min((n + kSpThreads - 1) / kSpThreads, 8 * ctx->sm_count));
  // one device block: ctl | deg | incount | inptr | fill | sortq | longrows |
  // hugerows | pos_long | pos_huge | src | val | wb0 | wb1 | y | wt | part
  auto al = [](size_t b) { return (b + 255) / 256 * 256; };
  const size_t E = (size_t)std::max(nnz, 1), N = (size_t)n;
  const size_t sizes[] = {al(sizeof(SpCtl)), al(4 * N),       al(4 * N),       al(4 * (N + 1)),
                          al(4 * N),         al(4 * (N + 4)), al(4 * N),       al(4 * N),
                          al(4 * (N + 1)),   al(4 * (N + 1)), al(4 * E),       al(4 * E),
                          al(4 * N),         al(4 * N),       al(4 * N),       al(8 * N),
                          al(4 * 3 * (size_t)grid),     al(8 * (size_t)grid)};
  size_t total = 0;
  for (size_t b : sizes) total += b;
  char* base = nullptr;
  if (cudaMallocAsync((void**)&base, total, s) != cudaSuccess) {
    cudaGetLastError();
    return fail(ctx, MAPI_ENOMEM, "sparse PageRank buffers");
  }
  char* p = base;
  auto take = [&](size_t i) {
    char* r = p;
    p += sizes[i];
    return r;
  };
  SpCtl* ctl = (SpCtl*)take(0);
  int* deg = (int*)take(1);
  int* incount = (int*)take(2);
  int* inptr = (int*)take(3);
  int* fill = (int*)take(4);
  int* sortq = (int*)take(5);
  int* longrows = (int*)take(6);
  int* hugerows = (int*)take(7);
  int* pos_long = (int*)take(8);
  int* pos_huge = (int*)take(9);
  int* src = (int*)take(10);
  float* val = (float*)take(11);
  float* wb0 = (float*)take(12);
  float* wb1 = (float*)take(13);
  float* y = (float*)take(14);
  float2* wt = (float2*)take(15);
  float* part = (float*)take(16);
  long long* bsum = (long long*)take(17);
  mapi_status st = MAPI_OK;
  auto run = [&]() -> mapi_status {
    MAPI_CUDA_TRY(ctx, cudaMemsetAsync(base, 0, (char*)longrows - base, s));  // ctl .. sortq
    k_sp_count<<<grid, kSpThreads, 0, s>>>(indptr, indices, n, nnz, deg, incount, ctl);
    MAPI_CUDA_TRY(ctx, cudaGetLastError());
    mapi_status r0 = sp_scan(ctx, s, incount, n, inptr, bsum, grid);
    if (r0 != MAPI_OK) return r0;
    k_sp_fill<<<grid, kSpThreads, 0, s>>>(indptr, indices, n, inptr, fill, src, ctl);
    MAPI_CUDA_TRY(ctx, cudaGetLastError());
    const double tele = (1.0 - alpha) / (double)n;
    k_sp_sort_short<<<grid, kSpThreads, 0, s>>>(n, inptr, src, val, deg, alpha, tele, sortq,
                                                ctl);
    MAPI_CUDA_TRY(ctx, cudaGetLastError());
    // ordered lists of the long and huge rows (flags in the spent count and
    // fill arrays, positions by scan)
    k_sp_flags<<<grid, kSpThreads, 0, s>>>(n, inptr, incount, fill);
    MAPI_CUDA_TRY(ctx, cudaGetLastError());
    if ((r0 = sp_scan(ctx, s, incount, n, pos_long, bsum, grid)) != MAPI_OK) return r0;
    if ((r0 = sp_scan(ctx, s, fill, n, pos_huge, bsum, grid)) != MAPI_OK) return r0;
    k_sp_lists<<<grid, kSpThreads, 0, s>>>(n, inptr, pos_long, pos_huge, longrows, hugerows);
    MAPI_CUDA_TRY(ctx, cudaGetLastError());
    const size_t lsm = sizeof(int) * kSpSortMax;
    MAPI_CUDA_TRY(ctx, cudaFuncSetAttribute((const void*)k_sp_sort_long,
                                            cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)lsm));
    k_sp_sort_long<<<ctx->sm_count, 1024, lsm, s>>>(inptr, src, val, deg, alpha, tele, sortq,
                                                   ctl);
    MAPI_CUDA_TRY(ctx, cudaGetLastError());
    count_launch(ctx, 9);
    int hq[2] = {0, 0};
    SpCtl hc;
    MAPI_CUDA_TRY(ctx, cudaMemcpyAsync(&hq[0], pos_long + n, sizeof(int), cudaMemcpyDeviceToHost, s));
    MAPI_CUDA_TRY(ctx, cudaMemcpyAsync(&hq[1], pos_huge + n, sizeof(int), cudaMemcpyDeviceToHost, s));
    MAPI_CUDA_TRY(ctx, cudaMemcpyAsync(&hc, ctl, sizeof(hc), cudaMemcpyDeviceToHost, s));
    MAPI_CUDA_TRY(ctx, cudaStreamSynchronize(s));
    if (hc.bad == 1) return fail(ctx, MAPI_EINVAL, "indptr or indices out of range");
    if (hc.bad == 2) return fail(ctx, MAPI_ENOTSUP, "a node has more than 16384 in-links");
    SpGraph g;
    g.n = n;
    g.deg = deg;
    g.inptr = inptr;
    g.src = src;
    g.val = val;
    g.longrows = longrows;
    g.nlong = hq[0];
    g.hugerows = hugerows;
    g.nhuge = hq[1];
    g.g0 = (float)(alpha * 0.0 + tele);
    g.gd = (float)(alpha * (1.0 / (double)n) + tele);
    k_sp_start<<<1, 1024, 0, s>>>(w0, n, wb0, ctl);
    MAPI_CUDA_TRY(ctx, cudaGetLastError());
    count_launch(ctx);
    const int norm_l2 = op == MAPI_OP_DOT ? 1 : 0;
    // algorithmic bytes of a row step: each in-link's source, value and
    // gathered (w_j, term(g0, w_j)); each row's extent and product
    const double step_bytes = 16.0 * nnz + 8.0 * n;
    mapi_status r2 = MAPI_OK;
    switch (op) {
      case MAPI_OP_MIN1:
        r2 = sp_solve<MAPI_OP_MIN1>(ctx, s, g, wb0, wb1, y, wt, part, ctl, grid, max_iters,
                                    (float)tol_l1, norm_l2, step_bytes);
        break;
      case MAPI_OP_MIN2:
        r2 = sp_solve<MAPI_OP_MIN2>(ctx, s, g, wb0, wb1, y, wt, part, ctl, grid, max_iters,
                                    (float)tol_l1, norm_l2, step_bytes);
        break;
      default:
        r2 = sp_solve<MAPI_OP_DOT>(ctx, s, g, wb0, wb1, y, wt, part, ctl, grid, max_iters,
                                   (float)tol_l1, norm_l2, step_bytes);
    }
    if (r2 != MAPI_OK) return r2;
    // the kept iterate: wb[iters & 1]; its l2 norm was summed by the last
    // form pass unless the solve ended before it
    MAPI_CUDA_TRY(ctx, cudaMemcpyAsync(&hc, ctl, sizeof(hc), cudaMemcpyDeviceToHost, s));
    MAPI_CUDA_TRY(ctx, cudaStreamSynchronize(s));
    const float* kept = (hc.iters & 1) ? wb1 : wb0;
    if (hc.done) {
      k_sp_norm2<<<1, 1024, 0, s>>>(kept, n, ctl);
      MAPI_CUDA_TRY(ctx, cudaGetLastError());
      count_launch(ctx);
    }
    k_sp_out<<<grid, kSpThreads, 0, s>>>(kept, n, rank_out, ctl);
    MAPI_CUDA_TRY(ctx, cudaGetLastError());
    count_launch(ctx);
    MAPI_CUDA_TRY(ctx, cudaMemcpyAsync(&hc, ctl, sizeof(hc), cudaMemcpyDeviceToHost, s));
    MAPI_CUDA_TRY(ctx, cudaStreamSynchronize(s));
    if (iters_done) *iters_done = hc.iters;
    if (last_delta) *last_delta = (double)hc.delta;
    if (hc.status != MAPI_OK) return fail(ctx, (mapi_status)hc.status, "the solve stopped early");
    return MAPI_OK;
  };
  st = run();
  cudaFreeAsync(base, s);
  cudaStreamSynchronize(s);
  return st;
}
