// MAPI iteration kernels (templated; instantiated per storage in k_iter_*.cu).
//
//   k_start_*   Alg. 1 step 1: w0 / ||w0||_2 (or as given; integer storage:
//               RNE(w0 2^q) then the integer l1 rule), zero padding, control
//               block reset.
//   k1_gemv_*   Alg. 1 steps 3-4 in one launch: y = A (+) w row by row (the
//               O(n^2) part, streamed once from HBM), then the last CTA to
//               finish normalises: w_new = y / ||y||_1 (Eq. (6); ||y||_2 for
//               DOT), delta = ||w_new - w_old||_1 and the stop test.
//   k_finish_*  Alg. 1 step 6 (optional): w_T / ||w_T||_2, written out.
#pragma once

#include <cooperative_groups.h>

#include "device_common.cuh"

namespace mapi {

namespace cgk = cooperative_groups;

// K1 on matrices of n >= 4096 runs in clusters of this many CTAs along the
// rows, and the cluster that finishes last runs the epilogue with all its
// threads (measured: BF16 112 -> 103 and FP8 88 -> 79 us per step at n =
// 16384; FP32 43 -> 37 at n = 4096, 69 -> 55 at 6144, unchanged at 16384;
// small matrices are slower in clusters and keep the one-CTA epilogue).
constexpr int kGemvCluster = 8;
constexpr int kGemvClusterMinRows = 4096;

struct GemvArgs {
  const uint8_t* A;     // rows_pad x ld elements, 16-byte rows
  int64_t row_bytes;    // ld * element size
  int chunks;           // 16-byte chunks per row
  int seg;              // chunks per column split (blockIdx.y)
  int n;                // logical rows (= cols)
  int rows_pad;
  const float* w;       // current iterates (nvec vectors, stride wst)
  float* w_next;        // next iterates
  int64_t wst;          // vector stride in elements (>= ld)
  float* ypart;         // [ksplit][nvec][rows_pad] partial products
  IterCtl* ctl;
  const float* row_mult;  // FP8: 2^(120 + k_i) per row; else unused
  int norm_l2;          // 1 for DOT (Eq. (1)), 0 for the MAVPs (Eq. (6))
  int clusters;         // 1: matrices of n >= kGemvClusterMinRows may run in clusters
};

constexpr int kEpiThreads = 256;

// Last-CTA epilogue for float storage.  NT threads.
template <int NT, int V>
__device__ void epilogue_float(const GemvArgs& g, int ks) {
  constexpr int kEpiU = 8;
  __shared__ float sh[33];
  for (int v = 0; v < V; ++v) {
    VecState* st = &g.ctl->v[v];
    if (*(volatile int*)&st->done) continue;  // uniform: written by earlier launches
    float* y0 = g.ypart + (int64_t)v * g.rows_pad;
    // kEpiU rows per thread in flight (the same order of additions as one at
    // a time): one CTA runs this for all n rows, so its loads must overlap
    Kahan acc;
    for (int i0 = threadIdx.x; i0 < g.n; i0 += NT * kEpiU) {
      float yv[kEpiU];
#pragma unroll
      for (int u = 0; u < kEpiU; ++u) {
        const int i = i0 + u * NT;
        yv[u] = i < g.n ? __ldcg(y0 + i) : 0.f;
      }
      for (int k = 1; k < ks; ++k) {
        const float* yk = g.ypart + ((int64_t)k * V + v) * g.rows_pad;
        float pk[kEpiU];
#pragma unroll
        for (int u = 0; u < kEpiU; ++u) {
          const int i = i0 + u * NT;
          pk[u] = i < g.n ? __ldcg(yk + i) : 0.f;
        }
#pragma unroll
        for (int u = 0; u < kEpiU; ++u) yv[u] += pk[u];
      }
#pragma unroll
      for (int u = 0; u < kEpiU; ++u) {
        const int i = i0 + u * NT;
        if (i < g.n) {
          if (ks > 1) y0[i] = yv[u];
          acc.add(g.norm_l2 ? yv[u] * yv[u] : fabsf(yv[u]));
        }
      }
    }
    float L = block_sum<NT>(acc.value(), sh);
    if (g.norm_l2) L = sqrtf(L);
    if (!(L > 0.f) || !isfinite(L)) {
      if (threadIdx.x == 0) {
        st->status = (L == 0.f) ? MAPI_EZERONORM : MAPI_ENONFINITE;
        st->done = 1;
      }
      continue;
    }
    const float* wo = g.w + (int64_t)v * g.wst;
    float* wn = g.w_next + (int64_t)v * g.wst;
    Kahan dl;
    for (int i0 = threadIdx.x; i0 < g.n; i0 += NT * kEpiU) {
      float yv[kEpiU], wv[kEpiU];
#pragma unroll
      for (int u = 0; u < kEpiU; ++u) {
        const int i = i0 + u * NT;
        yv[u] = i < g.n ? ((ks > 1) ? y0[i] : __ldcg(y0 + i)) : 0.f;
        wv[u] = i < g.n ? wo[i] : 0.f;
      }
#pragma unroll
      for (int u = 0; u < kEpiU; ++u) {
        const int i = i0 + u * NT;
        if (i < g.n) {
          const float x = yv[u] / L;  // the n divisions of §2.2
          dl.add(fabsf(x - wv[u]));
          wn[i] = x;
        }
      }
    }
    const float D = block_sum<NT>(dl.value(), sh);
    if (threadIdx.x == 0) {
      st->iters += 1;
      st->delta = D;
      st->norm = L;
      if (g.ctl->tol > 0.f && D < g.ctl->tol) st->done = 1;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int all = 1;
    for (int v = 0; v < V; ++v) all &= ((volatile int*)&g.ctl->v[v].done)[0];
    g.ctl->all_done = all;
    g.ctl->counter = 0;
    __threadfence();
  }
}

// The same epilogue run by all CS CTAs of the last cluster: thread t of CTA
// r takes rows r NT + t, r NT + t + CS NT, ... (kEpiU of them in flight) in
// both passes, so it reads back only what it wrote; the norm and delta are
// block sums added over the cluster in rank order.
template <int NT, int V, int CS>
__device__ void epilogue_float_cluster(const GemvArgs& g, int ks, cgk::cluster_group& cluster) {
  constexpr int kEpiU = 8;
  constexpr int NTC = NT * CS;
  __shared__ float sh[33];
  __shared__ float part[2];
  const int cr = (int)cluster.block_rank();
  const int tg = cr * NT + threadIdx.x;
  for (int v = 0; v < V; ++v) {
    VecState* st = &g.ctl->v[v];
    if (*(volatile int*)&st->done) continue;  // uniform: written by earlier launches
    float* y0 = g.ypart + (int64_t)v * g.rows_pad;
    Kahan acc;
    for (int i0 = tg; i0 < g.n; i0 += NTC * kEpiU) {
      float yv[kEpiU];
#pragma unroll
      for (int u = 0; u < kEpiU; ++u) {
        const int i = i0 + u * NTC;
        yv[u] = i < g.n ? __ldcg(y0 + i) : 0.f;
      }
      for (int k = 1; k < ks; ++k) {
        const float* yk = g.ypart + ((int64_t)k * V + v) * g.rows_pad;
        float pk[kEpiU];
#pragma unroll
        for (int u = 0; u < kEpiU; ++u) {
          const int i = i0 + u * NTC;
          pk[u] = i < g.n ? __ldcg(yk + i) : 0.f;
        }
#pragma unroll
        for (int u = 0; u < kEpiU; ++u) yv[u] += pk[u];
      }
#pragma unroll
      for (int u = 0; u < kEpiU; ++u) {
        const int i = i0 + u * NTC;
        if (i < g.n) {
          if (ks > 1) y0[i] = yv[u];
          acc.add(g.norm_l2 ? yv[u] * yv[u] : fabsf(yv[u]));
        }
      }
    }
    const float lp = block_sum<NT>(acc.value(), sh);
    if (threadIdx.x == 0) part[0] = lp;
    cluster.sync();
    float L = 0.f;
#pragma unroll
    for (int q = 0; q < CS; ++q) L += *cluster.map_shared_rank(&part[0], q);
    if (g.norm_l2) L = sqrtf(L);
    if (!(L > 0.f) || !isfinite(L)) {
      if (cr == 0 && threadIdx.x == 0) {
        st->status = (L == 0.f) ? MAPI_EZERONORM : MAPI_ENONFINITE;
        st->done = 1;
      }
      cluster.sync();  // part[0] is read by every rank before it changes
      continue;
    }
    const float* wo = g.w + (int64_t)v * g.wst;
    float* wn = g.w_next + (int64_t)v * g.wst;
    Kahan dl;
    for (int i0 = tg; i0 < g.n; i0 += NTC * kEpiU) {
      float yv[kEpiU], wv[kEpiU];
#pragma unroll
      for (int u = 0; u < kEpiU; ++u) {
        const int i = i0 + u * NTC;
        yv[u] = i < g.n ? ((ks > 1) ? y0[i] : __ldcg(y0 + i)) : 0.f;
        wv[u] = i < g.n ? wo[i] : 0.f;
      }
#pragma unroll
      for (int u = 0; u < kEpiU; ++u) {
        const int i = i0 + u * NTC;
        if (i < g.n) {
          const float x = yv[u] / L;  // the n divisions of §2.2
          dl.add(fabsf(x - wv[u]));
          wn[i] = x;
        }
      }
    }
    const float dp = block_sum<NT>(dl.value(), sh);
    if (threadIdx.x == 0) part[1] = dp;
    cluster.sync();
    if (cr == 0 && threadIdx.x == 0) {
      float D = 0.f;
#pragma unroll
      for (int q = 0; q < CS; ++q) D += *cluster.map_shared_rank(&part[1], q);
      st->iters += 1;
      st->delta = D;
      st->norm = L;
      if (g.ctl->tol > 0.f && D < g.ctl->tol) st->done = 1;
    }
    cluster.sync();  // part[] is read by rank 0 (and every rank) before it changes
  }
  if (cr == 0 && threadIdx.x == 0) {
    int all = 1;
    for (int v = 0; v < V; ++v) all &= ((volatile int*)&g.ctl->v[v].done)[0];
    g.ctl->all_done = all;
    g.ctl->counter = 0;
    __threadfence();
  }
}

// K1: y = A (+) w for V vectors, R rows per warp, WARPS warps per CTA; CL
// CTAs per cluster (1: the last CTA alone runs the epilogue).
template <int OP, int ST, int V, int R, int WARPS, int CL>
__global__ void __launch_bounds__(WARPS * 32)
    k1_gemv_float(GemvArgs g) {
  if (*(volatile int*)&g.ctl->all_done) return;
  using Ch = Chunk<ST>;
  constexpr int E = Ch::E;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // CTAs past the padded rows (the grid is a whole number of clusters) only
  // take part in the election
  const bool rows_here = blockIdx.x * WARPS * R < g.rows_pad;
  const int row0 = rows_here ? (blockIdx.x * WARPS + warp) * R : 0;
  const int ks = blockIdx.y;
  const int c_beg = ks * g.seg;
  const int c_end = rows_here ? min(g.chunks, c_beg + g.seg) : c_beg;

  float acc[R][V][2];
#pragma unroll
  for (int r = 0; r < R; ++r)
#pragma unroll
    for (int v = 0; v < V; ++v) acc[r][v][0] = acc[r][v][1] = 0.f;

  // FP8: the row scale 2^k (the stored factor 2^(120 + k) serves the
  // bit-placement decoder; the hardware conversion needs 2^-120 of it, exact)
  float mult[R];
#pragma unroll
  for (int r = 0; r < R; ++r) mult[r] = (ST == kFP8) ? g.row_mult[row0 + r] * 0x1p-120f : 1.f;

  const uint8_t* arow = g.A + (int64_t)row0 * g.row_bytes;

  auto consume = [&](const Ch (&ch)[R], int c) {
#pragma unroll
    for (int grp = 0; grp < E / 4; ++grp) {
#pragma unroll
      for (int v = 0; v < V; ++v) {
        const float4 wv = __ldg(reinterpret_cast<const float4*>(
            g.w + (int64_t)v * g.wst + (int64_t)c * E + grp * 4));
        const auto p0 = Op<OP>::prep(wv.x);
        const auto p1 = Op<OP>::prep(wv.y);
        const auto p2 = Op<OP>::prep(wv.z);
        const auto p3 = Op<OP>::prep(wv.w);
#pragma unroll
        for (int r = 0; r < R; ++r) {
          float a0, a1, a2, a3;
          if constexpr (ST == kFP8) {
            e4m3x4_values((&ch[r].raw.x)[grp], a0, a1, a2, a3);
          } else {
            a0 = ch[r].get(grp * 4 + 0);
            a1 = ch[r].get(grp * 4 + 1);
            a2 = ch[r].get(grp * 4 + 2);
            a3 = ch[r].get(grp * 4 + 3);
          }
          if (ST == kFP8) {
            a0 *= mult[r];
            a1 *= mult[r];
            a2 *= mult[r];
            a3 *= mult[r];
          }
          acc[r][v][0] = Op<OP>::term(a0, p0, acc[r][v][0]);
          acc[r][v][1] = Op<OP>::term(a1, p1, acc[r][v][1]);
          acc[r][v][0] = Op<OP>::term(a2, p2, acc[r][v][0]);
          acc[r][v][1] = Op<OP>::term(a3, p3, acc[r][v][1]);
        }
      }
    }
  };

  int c = c_beg + lane;
  // two chunks per row in flight per lane
  for (; c + 32 < c_end; c += 64) {
    Ch x[R], z[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      x[r].raw = ld_stream(arow + r * g.row_bytes + (int64_t)c * 16);
      z[r].raw = ld_stream(arow + r * g.row_bytes + (int64_t)(c + 32) * 16);
    }
    consume(x, c);
    consume(z, c + 32);
  }
  if (c < c_end) {
    Ch x[R];
#pragma unroll
    for (int r = 0; r < R; ++r) x[r].raw = ld_stream(arow + r * g.row_bytes + (int64_t)c * 16);
    consume(x, c);
  }

#pragma unroll
  for (int r = 0; r < R; ++r)
#pragma unroll
    for (int v = 0; v < V; ++v) {
      float s = acc[r][v][0] + acc[r][v][1];
#pragma unroll
      for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (lane == 0 && rows_here) g.ypart[((int64_t)ks * V + v) * g.rows_pad + row0 + r] = s;
    }

  if constexpr (CL == 1) {
    if (!elect_last_cta(&g.ctl->counter, gridDim.x * gridDim.y)) return;
    epilogue_float<WARPS * 32, V>(g, gridDim.y);
  } else {
    // last-cluster election: every CTA takes a ticket once its partials are
    // visible; the cluster holding the last ticket runs the epilogue
    cgk::cluster_group cluster = cgk::this_cluster();
    __shared__ int s_last;
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      const unsigned t = atomicAdd(&g.ctl->counter, 1u);
      s_last = (t == gridDim.x * gridDim.y - 1) ? 1 : 0;
    }
    cluster.sync();
    int last = 0;
#pragma unroll
    for (int q = 0; q < CL; ++q) last |= *cluster.map_shared_rank(&s_last, q);
    cluster.sync();  // every rank has read the tickets
    if (!last) return;
    __threadfence();
    epilogue_float_cluster<WARPS * 32, V, CL>(g, gridDim.y, cluster);
  }
}

// ------------------------------------------------------------ integer path
// w and y are INT32 in units of 2^-q; the w buffers are reinterpreted.
struct IGemvArgs {
  GemvArgs g;
  int q;
};

// Integer epilogue, run by the CS CTAs of the last cluster (CS = 1: the last
// CTA); thread t of CTA r takes rows r NT + t, r NT + t + CS NT, ...  Every
// sum is an exact INT64 sum, so the split changes no result.
template <int NT, int V, int CS>
__device__ void epilogue_int(const IGemvArgs& a, int ks) {
  constexpr int kEpiU = 8;  // rows per thread in flight (see epilogue_float)
  constexpr int NTC = NT * CS;
  const GemvArgs& g = a.g;
  __shared__ long long sh[33];
  __shared__ long long part[2];
  int cr = 0;
  if constexpr (CS > 1) cr = (int)cgk::this_cluster().block_rank();
  const int tg = cr * NT + threadIdx.x;
  // the CTA totals of slot k added over the cluster (after a cluster barrier)
  auto total = [&](int k, long long mine) {
    if constexpr (CS == 1) {
      return mine;
    } else {
      if (threadIdx.x == 0) part[k] = mine;
      cgk::cluster_group cl = cgk::this_cluster();
      cl.sync();
      long long t = 0;
#pragma unroll
      for (int q = 0; q < CS; ++q) t += *cl.map_shared_rank(&part[k], q);
      cl.sync();  // every rank has read part[k]
      return t;
    }
  };
  const int* ypart = reinterpret_cast<const int*>(g.ypart);
  for (int v = 0; v < V; ++v) {
    VecState* st = &g.ctl->v[v];
    if (*(volatile int*)&st->done) continue;
    int* y0 = reinterpret_cast<int*>(g.ypart) + (int64_t)v * g.rows_pad;
    long long s = 0;
    for (int i0 = tg; i0 < g.n; i0 += NTC * kEpiU) {
      int yv[kEpiU];
#pragma unroll
      for (int u = 0; u < kEpiU; ++u) {
        const int i = i0 + u * NTC;
        yv[u] = i < g.n ? __ldcg(y0 + i) : 0;
      }
      for (int k = 1; k < ks; ++k) {
        const int* yk = ypart + ((int64_t)k * V + v) * g.rows_pad;
        int pk[kEpiU];
#pragma unroll
        for (int u = 0; u < kEpiU; ++u) {
          const int i = i0 + u * NTC;
          pk[u] = i < g.n ? __ldcg(yk + i) : 0;
        }
#pragma unroll
        for (int u = 0; u < kEpiU; ++u) yv[u] += pk[u];
      }
#pragma unroll
      for (int u = 0; u < kEpiU; ++u) {
        const int i = i0 + u * NTC;
        if (i < g.n) {
          if (ks > 1) y0[i] = yv[u];
          s += (long long)abs(yv[u]);
        }
      }
    }
    const long long L = total(0, block_sum_i64<NT>(s, sh));
    if (L == 0) {
      if (cr == 0 && threadIdx.x == 0) {
        st->status = MAPI_EZERONORM;
        st->done = 1;
      }
      continue;
    }
    const int* wo = reinterpret_cast<const int*>(g.w) + (int64_t)v * g.wst;
    int* wn = reinterpret_cast<int*>(g.w_next) + (int64_t)v * g.wst;
    long long d = 0;
    const long long half = L / 2;
    // floor(N / L) for the n divisions: an FP32 estimate from one reciprocal
    // of L, made exact by whole steps of L on the remainder (the quotient is
    // at most 2^24 + 1, so the estimate is within a few units)
    const float rL = 1.f / (float)L;
    for (int i0 = tg; i0 < g.n; i0 += NTC * kEpiU) {
      int yv[kEpiU], wv[kEpiU];
#pragma unroll
      for (int u = 0; u < kEpiU; ++u) {
        const int i = i0 + u * NTC;
        yv[u] = i < g.n ? ((ks > 1) ? y0[i] : __ldcg(y0 + i)) : 0;
        wv[u] = i < g.n ? wo[i] : 0;
      }
#pragma unroll
      for (int u = 0; u < kEpiU; ++u) {
        const int i = i0 + u * NTC;
        if (i < g.n) {
          const long long N = ((long long)abs(yv[u]) << a.q) + half;
          long long m = (long long)((float)N * rL);
          long long rem = N - m * L;
          while (rem < 0) {
            --m;
            rem += L;
          }
          while (rem >= L) {
            ++m;
            rem -= L;
          }
          const int x = yv[u] < 0 ? -(int)m : (int)m;
          d += (long long)abs(x - wv[u]);
          wn[i] = x;
        }
      }
    }
    const long long D = total(1, block_sum_i64<NT>(d, sh));
    if (cr == 0 && threadIdx.x == 0) {
      st->iters += 1;
      st->idelta = D;
      st->delta = (float)D;
      if (g.ctl->itol > 0 && D < g.ctl->itol) st->done = 1;
    }
  }
  __syncthreads();
  if (cr == 0 && threadIdx.x == 0) {
    int all = 1;
    for (int v = 0; v < V; ++v) all &= ((volatile int*)&g.ctl->v[v].done)[0];
    g.ctl->all_done = all;
    g.ctl->counter = 0;
    __threadfence();
  }
}

template <int OP, int ST, int V, int R, int WARPS, int CL>
__global__ void __launch_bounds__(WARPS * 32)
    k1_gemv_int(IGemvArgs a) {
  const GemvArgs& g = a.g;
  if (*(volatile int*)&g.ctl->all_done) return;
  using Ch = Chunk<ST>;
  constexpr int E = Ch::E;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // CTAs past the padded rows (a whole number of clusters) only vote
  const bool rows_here = blockIdx.x * WARPS * R < g.rows_pad;
  const int row0 = rows_here ? (blockIdx.x * WARPS + warp) * R : 0;
  const int ks = blockIdx.y;
  const int c_beg = ks * g.seg;
  const int c_end = rows_here ? min(g.chunks, c_beg + g.seg) : c_beg;
  int acc[R][V];
#pragma unroll
  for (int r = 0; r < R; ++r)
#pragma unroll
    for (int v = 0; v < V; ++v) acc[r][v] = 0;
  const uint8_t* arow = g.A + (int64_t)row0 * g.row_bytes;
  const int* w = reinterpret_cast<const int*>(g.w);
  // int16 MIN1 / MIN2: two columns per 32-bit word at once, clamped with
  // packed 16-bit min/max (exact: the bounds are the iterate's entries
  // limited to +-32767, which changes no min against a stored int16) and
  // added with their signs by one two-way dot product into the INT32 sum
  constexpr bool kPacked = ST == kI16 && (OP == MAPI_OP_MIN1 || OP == MAPI_OP_MIN2);
  auto consume = [&](const Ch (&x)[R], int c) {
#pragma unroll
    for (int grp = 0; grp < E / 4; ++grp) {
#pragma unroll
      for (int v = 0; v < V; ++v) {
        const int4 wv = __ldg(reinterpret_cast<const int4*>(w + (int64_t)v * g.wst + (int64_t)c * E + grp * 4));
        if constexpr (kPacked) {
          uint32_t lo2[2], hi2[2], sg[2];
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int w0 = h ? wv.z : wv.x, w1 = h ? wv.w : wv.y;
            const auto p0 = IOp<OP>::prep(w0);
            const auto p1 = IOp<OP>::prep(w1);
            const int l0 = max(p0.lo, -32767), h0 = min(p0.hi, 32767);
            const int l1 = max(p1.lo, -32767), h1 = min(p1.hi, 32767);
            lo2[h] = ((uint32_t)l0 & 0xFFFFu) | ((uint32_t)l1 << 16);
            hi2[h] = ((uint32_t)h0 & 0xFFFFu) | ((uint32_t)h1 << 16);
            sg[h] = ((uint32_t)p0.s & 0xFFu) | (((uint32_t)p1.s & 0xFFu) << 8);
          }
#pragma unroll
          for (int r = 0; r < R; ++r) {
            int s = acc[r][v];
#pragma unroll
            for (int h = 0; h < 2; ++h)
              s = i16x2_clamp_dot(x[r].raw_word(grp * 2 + h), lo2[h], hi2[h], sg[h], s);
            acc[r][v] = s;
          }
        } else {
          const auto p0 = IOp<OP>::prep(wv.x);
          const auto p1 = IOp<OP>::prep(wv.y);
          const auto p2 = IOp<OP>::prep(wv.z);
          const auto p3 = IOp<OP>::prep(wv.w);
#pragma unroll
          for (int r = 0; r < R; ++r) {
            int s = acc[r][v];
            s = IOp<OP>::term(x[r].get(grp * 4 + 0), p0, s);
            s = IOp<OP>::term(x[r].get(grp * 4 + 1), p1, s);
            s = IOp<OP>::term(x[r].get(grp * 4 + 2), p2, s);
            s = IOp<OP>::term(x[r].get(grp * 4 + 3), p3, s);
            acc[r][v] = s;
          }
        }
      }
    }
  };
  int c = c_beg + lane;
  // two chunks per row in flight per lane
  for (; c + 32 < c_end; c += 64) {
    Ch x[R], z[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      x[r].raw = ld_stream(arow + r * g.row_bytes + (int64_t)c * 16);
      z[r].raw = ld_stream(arow + r * g.row_bytes + (int64_t)(c + 32) * 16);
    }
    consume(x, c);
    consume(z, c + 32);
  }
  if (c < c_end) {
    Ch x[R];
#pragma unroll
    for (int r = 0; r < R; ++r) x[r].raw = ld_stream(arow + r * g.row_bytes + (int64_t)c * 16);
    consume(x, c);
  }
#pragma unroll
  for (int r = 0; r < R; ++r)
#pragma unroll
    for (int v = 0; v < V; ++v) {
      int s = acc[r][v];
#pragma unroll
      for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (lane == 0 && rows_here)
        reinterpret_cast<int*>(g.ypart)[((int64_t)ks * V + v) * g.rows_pad + row0 + r] = s;
    }
  if constexpr (CL == 1) {
    if (!elect_last_cta(&g.ctl->counter, gridDim.x * gridDim.y)) return;
  } else {
    // last-cluster election (as in k1_gemv_float)
    cgk::cluster_group cluster = cgk::this_cluster();
    __shared__ int s_last;
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      const unsigned t = atomicAdd(&g.ctl->counter, 1u);
      s_last = (t == gridDim.x * gridDim.y - 1) ? 1 : 0;
    }
    cluster.sync();
    int last = 0;
#pragma unroll
    for (int q = 0; q < CL; ++q) last |= *cluster.map_shared_rank(&s_last, q);
    cluster.sync();  // every rank has read the tickets
    if (!last) return;
    __threadfence();
  }
  epilogue_int<WARPS * 32, V, CL>(a, gridDim.y);
}

// Launch table entry points (defined per storage file).
using LaunchFn = cudaError_t (*)(dim3 grid, cudaStream_t s, const GemvArgs& g, int q);

LaunchFn gemv_lookup_f32(int op, int V);
LaunchFn gemv_lookup_bf16(int op, int V);
LaunchFn gemv_lookup_fp8(int op, int V);
LaunchFn gemv_lookup_int(int st, int op, int V);

constexpr int kR = 2;      // rows per warp (FP32)
constexpr int kWarps = 8;  // warps per CTA

// Rows per warp by storage: every load of w serves R rows.  FP8 and the
// integer formats take 4 (w's L1 traffic was twice A's for FP8 at 2 rows;
// measured at n = 16384: FP8 98 -> 88 us, I16 120 -> 109 us per step); BF16
// stays at 2 (4 measured slower: 103 -> 115 us).
constexpr int kRowsNarrow = 4;
template <int ST>
constexpr int gemv_rows() { return (ST == kF32 || ST == kBF16) ? kR : kRowsNarrow; }
inline int gemv_rows_for(mapi_storage st) {
  return (st == MAPI_ST_F32 || st == MAPI_ST_BF16) ? kR : kRowsNarrow;
}

}  // namespace mapi

// Instantiate the float launch table for one storage tag.
#define MAPI_DEFINE_FLOAT_TABLE(FNNAME, ST)                                        \
  namespace mapi {                                                                \
  template <int OP, int V>                                                        \
  static cudaError_t launch_##FNNAME(dim3 grid, cudaStream_t s, const GemvArgs& g, \
                                     int) {                                       \
    if (g.n < kGemvClusterMinRows || !g.clusters) {                               \
      k1_gemv_float<OP, ST, V, gemv_rows<ST>(), kWarps, 1>                        \
          <<<grid, kWarps * 32, 0, s>>>(g);                                       \
      return cudaGetLastError();                                                  \
    }                                                                             \
    cudaLaunchConfig_t cfg = {};                                                  \
    cudaLaunchAttribute attr[1];                                                  \
    attr[0].id = cudaLaunchAttributeClusterDimension;                             \
    attr[0].val.clusterDim.x = kGemvCluster;                                      \
    attr[0].val.clusterDim.y = 1;                                                 \
    attr[0].val.clusterDim.z = 1;                                                 \
    cfg.gridDim = dim3((grid.x + kGemvCluster - 1) / kGemvCluster * kGemvCluster, \
                       grid.y, 1);                                                \
    cfg.blockDim = dim3(kWarps * 32, 1, 1);                                       \
    cfg.stream = s;                                                               \
    cfg.attrs = attr;                                                             \
    cfg.numAttrs = 1;                                                             \
    return cudaLaunchKernelEx(&cfg, k1_gemv_float<OP, ST, V, gemv_rows<ST>(), kWarps, \
                                                  kGemvCluster>, g);                              \
  }                                                                               \
  LaunchFn FNNAME(int op, int V) {                                                \
    switch (op * 16 + V) {                                                        \
      case MAPI_OP_MIN1 * 16 + 1: return launch_##FNNAME<MAPI_OP_MIN1, 1>;        \
      case MAPI_OP_MIN1 * 16 + 2: return launch_##FNNAME<MAPI_OP_MIN1, 2>;        \
      case MAPI_OP_MIN1 * 16 + 4: return launch_##FNNAME<MAPI_OP_MIN1, 4>;        \
      case MAPI_OP_MIN1 * 16 + 8: return launch_##FNNAME<MAPI_OP_MIN1, 8>;        \
      case MAPI_OP_MIN2 * 16 + 1: return launch_##FNNAME<MAPI_OP_MIN2, 1>;        \
      case MAPI_OP_MIN2 * 16 + 2: return launch_##FNNAME<MAPI_OP_MIN2, 2>;        \
      case MAPI_OP_MIN2 * 16 + 4: return launch_##FNNAME<MAPI_OP_MIN2, 4>;        \
      case MAPI_OP_MIN2 * 16 + 8: return launch_##FNNAME<MAPI_OP_MIN2, 8>;        \
      case MAPI_OP_DOT * 16 + 1: return launch_##FNNAME<MAPI_OP_DOT, 1>;          \
      case MAPI_OP_DOT * 16 + 2: return launch_##FNNAME<MAPI_OP_DOT, 2>;          \
      case MAPI_OP_DOT * 16 + 4: return launch_##FNNAME<MAPI_OP_DOT, 4>;          \
      case MAPI_OP_DOT * 16 + 8: return launch_##FNNAME<MAPI_OP_DOT, 8>;          \
      case MAPI_OP_DIAMOND * 16 + 1: return launch_##FNNAME<MAPI_OP_DIAMOND, 1>;  \
    }                                                                             \
    return nullptr;                                                               \
  }                                                                               \
  }
