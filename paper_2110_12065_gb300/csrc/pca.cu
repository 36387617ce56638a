// PCA by MAPI: min-covariance build (Eq. (5)), deflation (Alg. 2 step 6 with
// the sum form after Eq. (2)), the matrix-free pair step, and the top-k
// drivers for both modes.
#include <cooperative_groups.h>
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstring>

#include "device_common.cuh"

namespace cg = cooperative_groups;

namespace mapi {

// ======================================================================
// K2: C = (1/denom) X (+) X^T.  128 x 128 output tiles (upper triangle of
// tiles only), split over the samples (blockIdx.y) so that every SM has
// work; 256 threads, 8 x 8 register micro-tiles; the sample range is swept in
// chunks of 16 through two shared-memory buffers (k-major, padded rows), the
// next chunk prefetched into registers while the current one is consumed.
// Each split writes its partial tile; k_mincov_reduce sums the splits in a
// fixed order, divides by denom and mirrors the tile.
// ======================================================================
constexpr int kMcT = 128, kMcK = 16, kMcPad = 4;

template <int ST>
struct McStage;
template <>
struct McStage<kF32> {  // 128 rows x 16 floats = 512 float4, 2 per thread
  float4 v[2];
  __device__ __forceinline__ void load(const uint8_t* X, int64_t row_bytes, int rows_pad,
                                       int64_t k_end, int r0, int64_t k0) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int idx = threadIdx.x + h * 256;
      const int r = idx >> 2, cc = (idx & 3) * 4;
      v[h] = make_float4(0.f, 0.f, 0.f, 0.f);
      if (r0 + r < rows_pad && k0 + cc < k_end)
        v[h] = __ldg(reinterpret_cast<const float4*>(X + (int64_t)(r0 + r) * row_bytes +
                                                     (k0 + cc) * 4));
    }
  }
  __device__ __forceinline__ void store(float (*S)[kMcT + kMcPad]) const {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int idx = threadIdx.x + h * 256;
      const int r = idx >> 2, cc = (idx & 3) * 4;
      S[cc + 0][r] = v[h].x;
      S[cc + 1][r] = v[h].y;
      S[cc + 2][r] = v[h].z;
      S[cc + 3][r] = v[h].w;
    }
  }
};
template <>
struct McStage<kBF16> {  // 128 rows x 16 bf16 = 256 chunks of 8, 1 per thread
  Chunk<kBF16> c;
  __device__ __forceinline__ void load(const uint8_t* X, int64_t row_bytes, int rows_pad,
                                       int64_t k_end, int r0, int64_t k0) {
    const int r = threadIdx.x >> 1, cc = (threadIdx.x & 1) * 8;
    c.raw = make_uint4(0, 0, 0, 0);
    if (r0 + r < rows_pad && k0 + cc < k_end)
      c.raw = __ldg(reinterpret_cast<const uint4*>(X + (int64_t)(r0 + r) * row_bytes +
                                                   (k0 + cc) * 2));
  }
  __device__ __forceinline__ void store(float (*S)[kMcT + kMcPad]) const {
    const int r = threadIdx.x >> 1, cc = (threadIdx.x & 1) * 8;
#pragma unroll
    for (int e = 0; e < 8; ++e) S[cc + e][r] = c.get(e);
  }
};

__device__ __forceinline__ void mc_tile_of(int b, int T, int& tp, int& tq) {
  tp = 0;
  while (b >= T - tp) {
    b -= T - tp;
    ++tp;
  }
  tq = tp + b;
}

template <int OP, int ST>
__global__ void __launch_bounds__(256, 2)
    k_mincov(const uint8_t* __restrict__ X, int64_t row_bytes, int rows_pad, int64_t ld,
             int D, int64_t kseg, float* __restrict__ part) {
  __shared__ __align__(16) float As[2][kMcK][kMcT + kMcPad];
  __shared__ __align__(16) float Bs[2][kMcK][kMcT + kMcPad];
  const int T = (D + kMcT - 1) / kMcT;
  int tp, tq;
  mc_tile_of(blockIdx.x, T, tp, tq);
  const int p0 = tp * kMcT, q0 = tq * kMcT;
  const int64_t k_beg = (int64_t)blockIdx.y * kseg;
  const int64_t k_end = min(ld, k_beg + kseg);
  const int ty = threadIdx.x >> 4, tx = threadIdx.x & 15;
  float acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;

  McStage<ST> na, nb;
  int buf = 0;
  if (k_beg < k_end) {
    na.load(X, row_bytes, rows_pad, k_end, p0, k_beg);
    nb.load(X, row_bytes, rows_pad, k_end, q0, k_beg);
    na.store(As[0]);
    nb.store(Bs[0]);
  }
  __syncthreads();
  for (int64_t k0 = k_beg; k0 < k_end; k0 += kMcK) {
    const bool more = k0 + kMcK < k_end;
    if (more) {  // prefetch the next chunk into registers
      na.load(X, row_bytes, rows_pad, k_end, p0, k0 + kMcK);
      nb.load(X, row_bytes, rows_pad, k_end, q0, k0 + kMcK);
    }
#pragma unroll 4
    for (int k = 0; k < kMcK; ++k) {
      const float4 a0 = *reinterpret_cast<const float4*>(&As[buf][k][ty * 8]);
      const float4 a1 = *reinterpret_cast<const float4*>(&As[buf][k][ty * 8 + 4]);
      const float4 b0 = *reinterpret_cast<const float4*>(&Bs[buf][k][tx * 8]);
      const float4 b1 = *reinterpret_cast<const float4*>(&Bs[buf][k][tx * 8 + 4]);
      const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const auto p = Op<OP>::prep(bv[j]);
#pragma unroll
        for (int i = 0; i < 8; ++i) acc[i][j] = Op<OP>::term(a[i], p, acc[i][j]);
      }
    }
    if (more) {
      na.store(As[buf ^ 1]);
      nb.store(Bs[buf ^ 1]);
    }
    __syncthreads();
    buf ^= 1;
  }
  // partial tile: part[split][tile][128][128]
  float* out = part + ((int64_t)blockIdx.y * gridDim.x + blockIdx.x) * kMcT * kMcT;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    float4* o = reinterpret_cast<float4*>(out + (ty * 8 + i) * kMcT + tx * 8);
    o[0] = make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]);
    o[1] = make_float4(acc[i][4], acc[i][5], acc[i][6], acc[i][7]);
  }
}

// Sum the splits of each tile in order, divide by denom, write C and its
// mirror.  The tile goes through shared memory in 32 x 32 pieces so that the
// mirror's rows are written whole.
__global__ void __launch_bounds__(256)
    k_mincov_reduce(const float* __restrict__ part, int ntiles, int nsplit, int D, float denom,
                    float* __restrict__ C, int64_t ldc) {
  __shared__ float piece[32][33];
  const int T = (D + kMcT - 1) / kMcT;
  int tp, tq;
  mc_tile_of(blockIdx.x, T, tp, tq);
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (int pi = 0; pi < kMcT; pi += 32)
    for (int pj = 0; pj < kMcT; pj += 32) {
      // rows pi.., columns pj.. of the tile: direct copy, kept for the mirror
      for (int rr = ty; rr < 32; rr += 8) {
        const int e = (pi + rr) * kMcT + pj + tx;
        float sum = 0.f;
        for (int k = 0; k < nsplit; ++k)
          sum += part[((int64_t)k * ntiles + blockIdx.x) * kMcT * kMcT + e];
        const float v = sum / denom;
        piece[rr][tx] = v;
        const int p = tp * kMcT + pi + rr, q = tq * kMcT + pj + tx;
        if (p < D && q < D) C[(int64_t)p * ldc + q] = v;
      }
      __syncthreads();
      if (tp != tq) {
        // mirror: row q of C gets column q - tq*kMcT of the piece
        for (int rr = ty; rr < 32; rr += 8) {
          const int q = tq * kMcT + pj + rr, p = tp * kMcT + pi + tx;
          if (p < D && q < D) C[(int64_t)q * ldc + p] = piece[tx][rr];
        }
      }
      __syncthreads();
    }
}

// ======================================================================
// Deflation of an iterate without forming the outer products.  For
// P = wt (+) wt^T with c = |wt|, s = sign(wt) and z = s * y (min1):
//   (P y)_i = s_i [ sum_{c_j <= c_i} c_j z_j + c_i sum_{c_j > c_i} z_j ],
// which only needs wt sorted by c: two prefix sums over the sorted order.
// min2's outer product is half of (the min1 one + the same with every sign
// +1); dot's is w (w . y).  wt is the component at unit l1 norm for min1 /
// min2 (the unit of Eq. (8)'s iteration) and the kept unit-l2 component for
// dot; launch_outer_prep ranks a finished component once: perm[p] = index
// at sorted position p, wsort[p] = wt at that position (signed; its c is
// |wsort[p]|), ubi[i] = last sorted position whose c is <= c_i (ties
// included).
// ======================================================================
constexpr int kDeflMaxD = 1024;

struct DeflArgs {
  int nprev;          // finished components to deflate (0: none)
  int op;             // MAPI_OP_MIN1 / MIN2 / DOT
  const float* P;     // outer-product vectors wt, column m at P + m * ldp
  int64_t ldp;
  const int* perm;    // [m][D_pad] per component (launch_outer_prep)
  const float* wsort;
  const int* ubi;
  int64_t stride;     // elements between components in perm / wsort / ubi
};

// ======================================================================
// K4: pair step partials.  A cluster of 4 CTAs owns a stream of column
// tiles of X; CTA r of the cluster holds rows [r*RC, (r+1)*RC) of each tile
// (RC = 8 warps x RW rows).  Tiles arrive in shared memory through a
// S-stage TMA ring (one elected thread issues cp.async.bulk.tensor.2d with
// an mbarrier transaction count), so HBM reads run on while the warps
// compute and synchronise.  Lane = column (1 FP32 or 2 BF16 columns per
// 32-bit word; every row of a stage is 128 bytes, read conflict-free).
// Per tile:
//   t_n   = sum_d term(X_dn, w_d)   (column sums: warp -> CTA via shared
//           memory -> cluster via DSMEM, in a fixed order)
//   y_d  += sum_n term(X_dn, t_n)   (row sums kept per lane in registers)
// At the end each row's 32 lane partials are summed and written once per
// cluster: ypart[cluster][d].
// ======================================================================
constexpr int kPairWarps = 8, kPairCluster = 4, kPairStages = 3;

template <int ST>
struct PairCols;
template <>
struct PairCols<kF32> {
  static constexpr int CPL = 1;  // columns per lane
  static __device__ __forceinline__ void get(uint32_t raw, float (&v)[1]) {
    v[0] = __uint_as_float(raw);
  }
};
template <>
struct PairCols<kBF16> {
  static constexpr int CPL = 2;
  static __device__ __forceinline__ void get(uint32_t raw, float (&v)[2]) {
    v[0] = __uint_as_float(raw << 16);
    v[1] = __uint_as_float(raw & 0xFFFF0000u);
  }
};


// Sum over the cluster of one float per CTA (at `slot` in every CTA's shared
// memory), read in parallel by the lanes of one warp and added in a fixed
// butterfly order; every thread of the block gets the result.
__device__ __forceinline__ float cluster_sum(cg::cluster_group& cluster, float* slot, int CS,
                                             float* bcast) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (warp == 0) {
    float v = lane < CS ? cluster.map_shared_rank(slot, lane)[0] : 0.f;
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) *bcast = v;
  }
  __syncthreads();
  const float r = *bcast;
  __syncthreads();
  return r;
}

struct PairArgs {
  int D;          // logical rows
  int ntiles;     // column tiles
  int nclusters;
  const float* w;  // current iterate (D entries + zero padding)
  float* w_next;   // next iterate (written by the last cluster)
  float* ypart;    // [nclusters][D_pad] partial row sums, one row per cluster
  int D_pad;       // rows covered by one cluster (4 * 8 * RW)
  IterCtl* ctl;
  DeflArgs defl;
  int norm_l2;
  float denom;
  int reverse;    // walk this cluster's tiles last to first (odd steps), so a
                  // step starts on the tiles the previous one read last and
                  // that are still in L2
  int keep_tiles; // this many of a cluster's last tiles are kept in L2
  long long stall_ns;  // > 0: fault-detection test, see k_pair_partial
  PairPhases* phases;  // non-null: time stamps of the step's phases
};

// The phase stamps (%globaltimer, ns) of pair steps, summed over the steps
// that ran: a diagnostic of where a step's time goes.
__device__ __forceinline__ unsigned long long gtimer_u64() {
  return (unsigned long long)globaltimer_ns();
}

// Floats of shared memory the last cluster's epilogue needs: ys, u, wo (own
// rows), yfull and cbuf (D_pad each), four scan buffers and the component's
// w, sorted c, perm and ub (kDeflMaxD each).
// one padded array of the deflation: kDeflMaxD entries, one spare word per 32
constexpr int kDeflPadded = kDeflMaxD + kDeflMaxD / 8;
__host__ __device__ constexpr int pair_epi_floats(int rc, int d_pad) {
  return 3 * rc + 3 * d_pad + 2 * 8 * kDeflPadded;
}

constexpr int kPairMaxClusters = 80;  // partials per row the epilogue reads at once
constexpr int kEpiHalf = kPairWarps * 32 / 2;  // threads that load one component

// Index of sorted position p in a padded deflation array: the 32 lanes' runs
// of 8 positions [8 l, 8 l + 8) then fall on 32 different banks.
__device__ __forceinline__ int dpad(int p) { return p + (p >> 3); }

// Barrier of the 4 warps that deflate one component (named barriers 1, 2).
__device__ __forceinline__ void group_bar(int g) {
  asm volatile("bar.sync %0, %1;" ::"r"(1 + g), "r"(128) : "memory");
}

// Epilogue of one pair step, run by the last cluster to finish: CTA r owns
// rows [r*RS, (r+1)*RS) (the rows it streamed).  y = sum of the cluster
// partials (fixed order) / denom; u = y - sum_m P_m y (prefix-sum form; warps
// 0 and 1 of every CTA each take one earlier component, so up to 8 run at
// once, each scanned by one warp without block barriers); w_next =
// u / ||u||_1 (||u||_2 for DOT); delta and the stop test.  Shared memory: the
// (now idle) stage ring.
template <int RS>
__device__ void pair_epilogue(const PairArgs& a, cg::cluster_group& cluster, float* fsh) {
  constexpr int CS = kPairCluster;
  constexpr int NT = kPairWarps * 32;
  const int r = (int)cluster.block_rank();
  const int r0 = r * RS;
  const int D = a.D;
  const int h = threadIdx.x / kEpiHalf;  // half that loads component r + CS h
  const int th = threadIdx.x % kEpiHalf;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float* ys = fsh;
  float* u = ys + RS;
  float* wo = u + RS;
  float* yfull = wo + RS;
  float* cbuf = yfull + a.D_pad;  // [2][D_pad]: one per deflating warp
  auto arrays = [&](int g) { return cbuf + 2 * a.D_pad + g * 8 * kDeflPadded; };
  __shared__ float red[33];
  __shared__ float part[4];
  const bool dot = a.defl.op == MAPI_OP_DOT;

  // component m's vector, sorted |w| and the two index maps into group g's
  // padded arrays, loaded by the threads [t0, t0 + nt)
  // (nt = 128 threads, D <= 1024: at most 8 entries per thread, all loaded
  // before the first is stored)
  auto load_comp = [&](int m, int g, int t, int nt) {
    constexpr int PER = kDeflMaxD / kEpiHalf;
    const float* wm = a.defl.P + (int64_t)m * a.defl.ldp;
    float* wm_s = arrays(g) + 4 * kDeflPadded;
    float* cs_s = wm_s + kDeflPadded;
    int* perm_s = reinterpret_cast<int*>(cs_s + kDeflPadded);
    int* ub_s = perm_s + kDeflPadded;
    const int64_t o = (int64_t)m * a.defl.stride;
    float vw[PER], vc[PER];
    int vp[PER], vu[PER];
#pragma unroll
    for (int k = 0; k < PER; ++k) {
      const int i = t + k * nt;
      const bool in = i < D;
      vw[k] = in ? __ldcg(wm + i) : 0.f;
      vc[k] = (in && !dot) ? __ldcg(a.defl.wsort + o + i) : 0.f;
      vp[k] = (in && !dot) ? __ldcg(a.defl.perm + o + i) : 0;
      vu[k] = (in && !dot) ? __ldcg(a.defl.ubi + o + i) : 0;
    }
#pragma unroll
    for (int k = 0; k < PER; ++k) {
      const int i = t + k * nt;
      if (i < D) {
        wm_s[i] = vw[k];
        if (!dot) {
          cs_s[dpad(i)] = fabsf(vc[k]);
          perm_s[dpad(i)] = vp[k];
          ub_s[i] = vu[k];
        }
      }
    }
  };
  const bool stamp = a.phases && r == 0 && threadIdx.x == 0;
  unsigned long long t_elect = 0, t_reduce = 0, t_defl = 0;
  if (stamp) t_elect = gtimer_u64();
  // 0. prefetch: the first component of each deflating warp
  if (r + CS * h < a.defl.nprev) load_comp(r + CS * h, h, th, kEpiHalf);
  // 1. own rows of y: one row per thread; the row's cluster partials are all
  //    loaded before any is added (in cluster order)
  for (int i = threadIdx.x; i < RS; i += NT) {
    const int d = r0 + i;
    wo[i] = d < D ? a.w[d] : 0.f;
    // cluster-major partials: a warp's 32 rows of one cluster are 128
    // contiguous bytes
    const float* src = a.ypart + d;
    constexpr int B = kPairMaxClusters / 2;  // two batches of loads in flight
    float sum = 0.f;
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      float v[B];
#pragma unroll
      for (int g = 0; g < B; ++g)
        v[g] = b * B + g < a.nclusters ? __ldcg(src + (int64_t)(b * B + g) * a.D_pad) : 0.f;
#pragma unroll
      for (int g = 0; g < B; ++g)
        if (b * B + g < a.nclusters) sum += v[g];
    }
    ys[i] = d < D ? sum / a.denom : 0.f;
  }
  __syncthreads();
  if (stamp) t_reduce = gtimer_u64();
  // 2. deflation
  if (a.defl.nprev > 0) {
    cluster.sync();
    for (int i = threadIdx.x; i < a.D_pad; i += NT) {
      yfull[i] = cluster.map_shared_rank(ys, i / RS)[i % RS];
      cbuf[i] = 0.f;
      cbuf[a.D_pad + i] = 0.f;
    }
    __syncthreads();
    {
      // group g = warps 4g .. 4g + 3 deflates component r + CS g (and every
      // 2 CS-th after it); warp wq of the group scans sorted positions
      // [256 wq, 256 wq + 256), eight per lane.  Every sum is compensated
      // (TwoSum: hi + lo): the lane's eight terms, the scan over the lanes,
      // the warps' offsets; each prefix A_p = sum_{q <= p} c_q z_q and each
      // suffix S_p = sum_{q > p} z_q is rounded once, when it is stored.
      const int g = warp >> 2, wq = warp & 3, tg = threadIdx.x & 127;
      __shared__ float gtot[2][4][8];
      float* cb = cbuf + g * a.D_pad;
      float* sA = arrays(g);
      float* sS = sA + kDeflPadded;
      float* sA2 = sS + kDeflPadded;
      float* sS2 = sA2 + kDeflPadded;
      const float* wm_s = sS2 + kDeflPadded;
      const float* cs_s = wm_s + kDeflPadded;
      const int* perm_s = reinterpret_cast<const int*>(cs_s + kDeflPadded);
      const int* ub_s = perm_s + kDeflPadded;
      const bool two = a.defl.op == MAPI_OP_MIN2;
      for (int m = r + CS * g; m < a.defl.nprev; m += 2 * CS) {
        if (m >= 2 * CS) {  // more components than groups
          group_bar(g);
          load_comp(m, g, tg, 128);
        }
        group_bar(g);
        if (dot) {
          TwoSum pd;
          for (int i = tg; i < D; i += 128) pd.add_prod(wm_s[i], yfull[i]);
#pragma unroll
          for (int o = 16; o; o >>= 1) {
            TwoSum q;
            q.hi = __shfl_xor_sync(0xffffffffu, pd.hi, o);
            q.lo = __shfl_xor_sync(0xffffffffu, pd.lo, o);
            pd.add(q);
          }
          if (lane == 0) {
            gtot[g][wq][0] = pd.hi;
            gtot[g][wq][1] = pd.lo;
          }
          group_bar(g);
          TwoSum dv;
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            TwoSum e;
            e.hi = gtot[g][q][0];
            e.lo = gtot[g][q][1];
            dv.add(e);
          }
          const float d = dv.value();
          for (int i = tg; i < D; i += 128) cb[i] = fmaf(wm_s[i], d, cb[i]);
          group_bar(g);
          continue;
        }
        // sorted position p contributes c z to A and z to B (z = s y, with
        // c and s the magnitude and sign of the component there) and, for
        // min2, c y and y
        const int p0 = wq * 256 + lane * 8;
        // 1. this lane's totals
        TwoSum la, lb, la2, lb2;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          const int p = p0 + k;
          if (p < D) {
            const int i = perm_s[dpad(p)];
            const float y = yfull[i];
            const float c = cs_s[dpad(p)];
            const float z = sgnf(wm_s[i]) * y;
            la.add_prod(c, z);
            lb.add(z);
            if (two) {
              la2.add_prod(c, y);
              lb2.add(y);
            }
          }
        }
        // 2. inclusive scan of the lane totals over the warp
        TwoSum ia = la, ib = lb, ia2 = la2, ib2 = lb2;
        auto up = [&](TwoSum& v, int o) {
          TwoSum n;
          n.hi = __shfl_up_sync(0xffffffffu, v.hi, o);
          n.lo = __shfl_up_sync(0xffffffffu, v.lo, o);
          if (lane >= o) v.add(n);
        };
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          up(ia, o);
          up(ib, o);
          if (two) {
            up(ia2, o);
            up(ib2, o);
          }
        }
        if (lane == 31) {
          gtot[g][wq][0] = ia.hi;
          gtot[g][wq][1] = ia.lo;
          gtot[g][wq][2] = ib.hi;
          gtot[g][wq][3] = ib.lo;
          gtot[g][wq][4] = ia2.hi;
          gtot[g][wq][5] = ia2.lo;
          gtot[g][wq][6] = ib2.hi;
          gtot[g][wq][7] = ib2.lo;
        }
        group_bar(g);
        // 3. this lane's offset (everything before its first position) and
        //    the group's total of z (and y)
        auto neg = [](const TwoSum& v) {
          TwoSum n;
          n.hi = -v.hi;
          n.lo = -v.lo;
          return n;
        };
        TwoSum oa = ia, ob = ib, oa2 = ia2, ob2 = ib2;
        oa.add(neg(la));
        ob.add(neg(lb));
        oa2.add(neg(la2));
        ob2.add(neg(lb2));
        TwoSum totB, totB2;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          TwoSum ea, eb, ea2, eb2;
          ea.hi = gtot[g][q][0];
          ea.lo = gtot[g][q][1];
          eb.hi = gtot[g][q][2];
          eb.lo = gtot[g][q][3];
          ea2.hi = gtot[g][q][4];
          ea2.lo = gtot[g][q][5];
          eb2.hi = gtot[g][q][6];
          eb2.lo = gtot[g][q][7];
          if (q < wq) {
            oa.add(ea);
            ob.add(eb);
            if (two) {
              oa2.add(ea2);
              ob2.add(eb2);
            }
          }
          totB.add(eb);
          if (two) totB2.add(eb2);
        }
        // 4. walk the lane's positions again from its offset: the prefix
        //    A_p and the suffix S_p = totB - B_p, each rounded once
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          const int p = p0 + k;
          if (p < D) {
            const int i = perm_s[dpad(p)];
            const float y = yfull[i];
            const float c = cs_s[dpad(p)];
            const float z = sgnf(wm_s[i]) * y;
            oa.add_prod(c, z);
            ob.add(z);
            TwoSum sb = totB;
            sb.add(neg(ob));
            sA[dpad(p)] = oa.value();
            sS[dpad(p)] = sb.value();
            if (two) {
              oa2.add_prod(c, y);
              ob2.add(y);
              TwoSum sb2 = totB2;
              sb2.add(neg(ob2));
              sA2[dpad(p)] = oa2.value();
              sS2[dpad(p)] = sb2.value();
            }
          }
        }
        group_bar(g);
        for (int i = tg; i < D; i += 128) {
          const float wi = wm_s[i], ci = fabsf(wi);
          const int q = dpad(ub_s[i]);
          float v = sgnf(wi) * fmaf(ci, sS[q], sA[q]);
          if (two) v = 0.5f * (v + fmaf(ci, sS2[q], sA2[q]));
          cb[i] += v;
        }
      }
    }
    cluster.sync();
    const int nq = min(CS, a.defl.nprev);
    const bool second = a.defl.nprev > CS;  // some CTA's second warp holds a sum
    for (int i = threadIdx.x; i < RS; i += NT) {
      const int d = r0 + i;
      float v[2 * CS];
#pragma unroll
      for (int q = 0; q < CS; ++q) {
        const float* cq = cluster.map_shared_rank(cbuf, q);
        v[q] = q < nq ? cq[d] : 0.f;
        v[CS + q] = second ? cq[a.D_pad + d] : 0.f;
      }
      // u = y - sum_m P_m y, compensated, rounded once (the groups' sums in
      // the order of their first components m = 0, 1, ..., 2 CS - 1)
      TwoSum uc;
      uc.add(ys[i]);
#pragma unroll
      for (int q = 0; q < 2 * CS; ++q) uc.add(-v[q]);
      u[i] = d < D ? uc.value() : 0.f;
    }
  } else {
    for (int i = threadIdx.x; i < RS; i += NT) u[i] = ys[i];
  }
  __syncthreads();
  if (stamp) t_defl = gtimer_u64();
  // 3. norm over the cluster
  Kahan k;
  for (int i = threadIdx.x; i < RS; i += NT) {
    const float x = u[i];
    k.add(a.norm_l2 ? x * x : fabsf(x));
  }
  const float np = block_sum<NT>(k.value(), red);
  if (threadIdx.x == 0) part[0] = np;
  cluster.sync();
  float L = cluster_sum(cluster, &part[0], CS, &part[2]);
  if (a.norm_l2) L = sqrtf(L);
  const bool ok = (L > 0.f) && isfinite(L);
  // 4. normalise own rows; the delta only when a stop rule needs it
  const bool want_delta = a.ctl->tol > 0.f;
  Kahan dk;
  if (ok) {
    for (int i = threadIdx.x; i < RS; i += NT) {
      const int d = r0 + i;
      if (d >= D) continue;
      const float x = u[i] / L;  // the n divisions of §2.2
      if (want_delta) dk.add(fabsf(x - wo[i]));
      a.w_next[d] = x;
    }
  }
  float Dsum = 0.f;
  if (want_delta) {
    const float dp = block_sum<NT>(dk.value(), red);
    if (threadIdx.x == 0) part[1] = dp;
    cluster.sync();
    if (r == 0) Dsum = cluster_sum(cluster, &part[1], CS, &part[3]);
  }
  if (r == 0 && threadIdx.x == 0) {
    VecState* st = &a.ctl->v[0];
    if (!ok) {
      st->status = (L == 0.f) ? MAPI_EZERONORM : MAPI_ENONFINITE;
      st->done = 1;
    } else {
      st->iters += 1;
      if (want_delta) st->delta = Dsum;
      st->norm = L;
      if (want_delta && Dsum < a.ctl->tol) st->done = 1;
    }
    a.ctl->all_done = st->done;
    a.ctl->counter = 0;
    __threadfence();
  }
  if (stamp) {
    volatile PairPhases* ph = a.phases;
    const unsigned long long t_end = gtimer_u64();
    const unsigned long long t0 = ph->start_min;
    const unsigned long long lmin = ph->loop_min, lmax = ph->loop_max;
    if (ph->prev_end && t0 > ph->prev_end) ph->sum[0] += t0 - ph->prev_end;
    ph->sum[1] += lmin - t0;
    ph->sum[2] += lmax - t0;
    ph->sum[3] += t_elect - lmax;
    ph->sum[4] += t_reduce - t_elect;
    ph->sum[5] += t_defl - t_reduce;
    ph->sum[6] += t_end - t_defl;
    ph->sum[7] += 1;
    ph->prev_end = t_end;
    ph->start_min = ~0ull;
    ph->loop_min = ~0ull;
    ph->loop_max = 0;
    __threadfence();
  }
  cluster.sync();  // peers may still read this CTA's shared memory until here
}

template <int OP, int ST, int RW>
__global__ void __launch_bounds__(kPairWarps * 32, 2)
    k_pair_partial(const __grid_constant__ CUtensorMap xmap, PairArgs a) {
  using PC = PairCols<ST>;
  constexpr int CPL = PC::CPL;
  constexpr int TC = 32 * CPL;   // columns per tile
  constexpr int RC = kPairWarps * RW;
  constexpr unsigned kStageBytes = RC * 128;
  cg::cluster_group cluster = cg::this_cluster();
  const unsigned crank = cluster.block_rank();
  const int cid = blockIdx.x / kPairCluster;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int rbase = (int)crank * RC + warp * RW;  // first row of this warp

  extern __shared__ __align__(1024) uint32_t stage[];   // kPairStages x RC x 32 words
  __shared__ __align__(8) uint64_t full[kPairStages];   // TMA tile arrived
  // exchange slots of the column partials, by tile index mod 4: with phase B
  // one tile behind phase A, a peer can be at most three tiles ahead of this
  // CTA's reads (its push of tile j + 4 waits, through its phase B of tile
  // j + 2, for this CTA's push of tile j + 2, which follows this CTA's phase
  // B of tile j)
  __shared__ __align__(8) uint64_t tready[4];           // all 4 column partials arrived
  __shared__ float4 wp[RC];                 // (lo, hi, s, 0) per row of this CTA
  __shared__ float tbuf[2][kPairWarps][TC];  // per-warp column partials (by tile parity)
  __shared__ float tin[4][kPairCluster][TC];  // column partials pushed by each CTA
  __shared__ __align__(8) uint64_t never;  // nothing ever arrives here
  __shared__ int s_err;
  __shared__ int s_last;

  const int nmine = a.ntiles > cid ? (a.ntiles - cid + a.nclusters - 1) / a.nclusters : 0;
  if (threadIdx.x == 0) {
    s_err = 0;
    s_last = 0;
    for (int s = 0; s < kPairStages; ++s) mbar_init(&full[s], 1);
    for (int q = 0; q < 4; ++q) mbar_init(&tready[q], 1);
    mbar_init(&never, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  // Fault-detection test (stall_ns > 0, never in a normal solve): thread 0
  // waits on a barrier that nothing arrives at, through the same bounded
  // wait as every tile and exchange.  No copy or peer store is pending on
  // it, so the wait simply runs out; the step then computes as usual and
  // reports the expiry as MAPI_ETIMEOUT, which stops the solve.
  bool stalled = false;
  if (a.stall_ns > 0 && threadIdx.x == 0) stalled = !mbar_wait(&never, 0, a.stall_ns);
  // the tiles read last stay in L2 for the next step (which walks the other
  // way); the others leave L2 first
  const uint64_t pol_first = createpolicy_evict_first();
  const uint64_t pol_last = createpolicy_evict_last();
  auto issue = [&](int j) {
    const int s = j % kPairStages;
    const int tile = cid + (a.reverse ? nmine - 1 - j : j) * a.nclusters;
    mbar_expect_tx(&full[s], kStageBytes);
    tma_load_2d_hint(stage + (size_t)s * RC * 32, &xmap, tile * TC, (int)crank * RC, &full[s],
                     j >= nmine - a.keep_tiles ? pol_last : pol_first);
  };
  // X does not depend on the previous step: start streaming it before waiting
  // for that step (programmatic dependent launch)
  const int npre = nmine < kPairStages ? nmine : kPairStages;
  if (threadIdx.x == 0)
    for (int j = 0; j < npre; ++j) issue(j);
  // peers push into tin / tready only after every CTA of the cluster has
  // initialised its barriers; this wait needs nothing from the previous step
  cluster.sync();
  cudaGridDependencySynchronize();
  if (*(volatile const int*)&a.ctl->all_done) {
    // nothing left to do: let the copies already issued land, then leave
    if (threadIdx.x == 0)
      for (int j = 0; j < npre; ++j) mbar_wait(&full[j], 0);
    __syncthreads();
    return;
  }
  if (a.phases && threadIdx.x == 0) atomicMin(&a.phases->start_min, gtimer_u64());
  for (int r = threadIdx.x; r < RC; r += blockDim.x) {
    const int d = (int)crank * RC + r;
    const float wv = d < a.D ? a.w[d] : 0.f;
    const auto p = Op<OP>::prep(wv);
    if constexpr (OP == MAPI_OP_DOT) wp[r] = make_float4(p.w, 0.f, 0.f, 0.f);
    else wp[r] = make_float4(p.lo, p.hi, p.s, 0.f);
  }
  __syncthreads();

  float acc[RW];
#pragma unroll
  for (int j = 0; j < RW; ++j) acc[j] = 0.f;

  // Phase A of tile j: read this warp's rows of the stage into registers,
  // column partials -> tbuf[j & 1] -> (after the CTA barrier) warp 0 pushes
  // the CTA's partials to every CTA of the cluster.  The stage is refilled
  // as soon as every warp has read it.
  auto phase_a = [&](int j, uint32_t (&raw)[RW]) {
    const int s = j % kPairStages;
    const int par = j & 1;   // tbuf slot
    const int slot = j & 3;  // exchange slot
    if (!mbar_wait(&full[s], (unsigned)((j / kPairStages) & 1))) s_err = 1;
    const uint32_t* src = stage + (size_t)s * RC * 32 + (size_t)(warp * RW) * 32 + lane;
#pragma unroll
    for (int jj = 0; jj < RW; ++jj) raw[jj] = src[jj * 32];
    float tp[CPL];
#pragma unroll
    for (int c = 0; c < CPL; ++c) tp[c] = 0.f;
#pragma unroll
    for (int jj = 0; jj < RW; ++jj) {
      float x[CPL];
      PC::get(raw[jj], x);
      const float4 q = wp[warp * RW + jj];
      typename Op<OP>::P p;
      if constexpr (OP == MAPI_OP_DOT) p = {q.x};
      else p = {q.x, q.y, q.z};
#pragma unroll
      for (int c = 0; c < CPL; ++c) tp[c] = Op<OP>::term(x[c], p, tp[c]);
    }
#pragma unroll
    for (int c = 0; c < CPL; ++c) tbuf[par][warp][lane * CPL + c] = tp[c];
    __syncthreads();
    if (threadIdx.x == 0 && j + kPairStages < nmine && !s_err) issue(j + kPairStages);
    if (warp == 0) {
      if (lane == 0) mbar_expect_tx(&tready[slot], kPairCluster * TC * 4);
      __syncwarp();
#pragma unroll
      for (int c = 0; c < CPL; ++c) {
        float sum = 0.f;
#pragma unroll
        for (int w = 0; w < kPairWarps; ++w) sum += tbuf[par][w][lane * CPL + c];
        const uint32_t loc = smem_u32(&tin[slot][crank][lane * CPL + c]);
        const uint32_t bar = smem_u32(&tready[slot]);
#pragma unroll
        for (int q = 0; q < kPairCluster; ++q)
          st_async_f32(mapa_u32(loc, q), sum, mapa_u32(bar, q));
      }
    }
  };
  // Phase B of tile j: wait for the cluster's partials of its columns (they
  // were pushed while phase A of the next tile ran), then the row sums.
  auto phase_b = [&](int j, const uint32_t (&raw)[RW]) {
    const int slot = j & 3;
    if (!mbar_wait(&tready[slot], (unsigned)((j >> 2) & 1))) s_err = 1;
    typename Op<OP>::P tpar[CPL];
#pragma unroll
    for (int c = 0; c < CPL; ++c) {
      float t = 0.f;
#pragma unroll
      for (int r = 0; r < kPairCluster; ++r) t += tin[slot][r][lane * CPL + c];
      tpar[c] = Op<OP>::prep(t);
    }
#pragma unroll
    for (int jj = 0; jj < RW; ++jj) {
      float x[CPL];
      PC::get(raw[jj], x);
#pragma unroll
      for (int c = 0; c < CPL; ++c) acc[jj] = Op<OP>::term(x[c], tpar[c], acc[jj]);
    }
  };
  // two tiles in flight: A(j) overlaps the cluster exchange of tile j - 1
  uint32_t rawA[RW], rawB[RW];
  int j = 0;
#pragma unroll 1
  for (; j + 1 < nmine; j += 2) {
    phase_a(j, rawA);
    if (j > 0) phase_b(j - 1, rawB);
    phase_a(j + 1, rawB);
    phase_b(j, rawA);
  }
  if (j < nmine) {
    phase_a(j, rawA);
    if (j > 0) phase_b(j - 1, rawB);
    phase_b(j, rawA);
  } else if (nmine > 0) {
    phase_b(nmine - 1, rawB);
  }
  // row sums across the 32 lanes, written once per cluster: a transposing
  // butterfly halves the rows each lane holds at every level (31 shuffles
  // for 32 rows), so lane l ends with row l / (32 / RW)
  {
    constexpr int H = RW == 32 ? 5 : RW == 16 ? 4 : RW == 8 ? 3 : -1;
    static_assert(H > 0, "RW must be 8, 16 or 32");
#pragma unroll
    for (int lev = 0; lev < 5; ++lev) {
      const int o = 16 >> lev;
      if (lev < H) {
        const int half = RW >> (lev + 1);
        const bool upper = (lane & o) != 0;
#pragma unroll
        for (int k = 0; k < half; ++k) {
          const float send = upper ? acc[k] : acc[k + half];
          const float keep = upper ? acc[k + half] : acc[k];
          acc[k] = keep + __shfl_xor_sync(0xffffffffu, send, o);
        }
      } else {
        acc[0] += __shfl_xor_sync(0xffffffffu, acc[0], o);
      }
    }
    constexpr int grp = 32 / RW;
    if ((lane & (grp - 1)) == 0)
      a.ypart[(int64_t)cid * a.D_pad + rbase + lane / grp] = acc[0];
  }
  if (threadIdx.x == 0 && (s_err || stalled)) {
    // a tile or a peer's partials never arrived: report it; the solve stops
    a.ctl->v[0].status = MAPI_ETIMEOUT;
    a.ctl->v[0].done = 1;
  }
  if (a.phases && threadIdx.x == 0) {
    const unsigned long long t = gtimer_u64();
    atomicMin(&a.phases->loop_min, t);
    atomicMax(&a.phases->loop_max, t);
  }
  // the next step's kernel may launch now (it waits for this grid to finish
  // before it reads anything this step writes)
  cudaTriggerProgrammaticLaunchCompletion();
  // last-cluster election: every CTA takes a ticket once its partials are
  // visible; the cluster holding the last ticket runs the epilogue
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned t = atomicAdd(&a.ctl->counter, 1u);
    s_last = (t == (unsigned)(a.nclusters * kPairCluster) - 1) ? 1 : 0;
  }
  cluster.sync();
  int last = 0;
#pragma unroll
  for (int q = 0; q < kPairCluster; ++q) last |= *cluster.map_shared_rank(&s_last, q);
  if (!last) {
    cluster.sync();  // peers may still read this CTA's ticket until here
    return;
  }
  __threadfence();
  pair_epilogue<RC>(a, cluster, reinterpret_cast<float*>(stage));
}

// Copy a finished component's step count and status out of the control
// block; a failure sets the sticky abort flag that skips later components
// (their step count is recorded as 0 and their status as OK).
__global__ void k_record(const IterCtl* ctl, int* iters, int* status, int* abort, int c) {
  const int st = ctl->v[0].status;
  if (st == MAPI_ECANCELLED) {
    iters[c] = 0;
    status[c] = MAPI_OK;
    return;
  }
  iters[c] = ctl->v[0].iters;
  status[c] = st;
  if (st != MAPI_OK) *abort = 1;
}

// ---------------------------------------------------------------- host side

mapi_status launch_mincov_raw(mapi_ctx* ctx, const mapi_mat* X, mapi_op op, float denom,
                              float* C, int64_t ldc, cudaStream_t s) {
  const int T = (X->rows + kMcT - 1) / kMcT;
  const int nt = T * (T + 1) / 2;
  const int64_t rb = X->ld * elem_bytes(X->storage);
  const uint8_t* x = (const uint8_t*)X->data;
  // split the samples until there are about 4 CTAs per SM (2 resident)
  int nsplit = 1;
  while (nt * nsplit < 4 * ctx->sm_count && X->ld / (nsplit * 2) >= 4 * kMcK) nsplit *= 2;
  const int64_t kseg = ((X->ld + nsplit - 1) / nsplit + kMcK - 1) / kMcK * kMcK;
  mapi_status st = ensure(ctx, ctx->mcpart, sizeof(float) * (size_t)nsplit * nt * kMcT * kMcT);
  if (st != MAPI_OK) return st;
  float* part = (float*)ctx->mcpart.p;
  const dim3 grid(nt, nsplit);
  cudaEvent_t ev = prof_begin(ctx, s);
#define MC(OPV, STV) \
  k_mincov<OPV, STV><<<grid, 256, 0, s>>>(x, rb, X->rows_pad, X->ld, X->rows, kseg, part)
  if (X->storage == MAPI_ST_F32) {
    if (op == MAPI_OP_MIN1) MC(MAPI_OP_MIN1, kF32);
    else if (op == MAPI_OP_MIN2) MC(MAPI_OP_MIN2, kF32);
    else MC(MAPI_OP_DOT, kF32);
  } else if (X->storage == MAPI_ST_BF16) {
    if (op == MAPI_OP_MIN1) MC(MAPI_OP_MIN1, kBF16);
    else if (op == MAPI_OP_MIN2) MC(MAPI_OP_MIN2, kBF16);
    else MC(MAPI_OP_DOT, kBF16);
  } else {
    return fail(ctx, MAPI_EINVAL, "min-covariance supports F32 and BF16 storage");
  }
#undef MC
  MAPI_CUDA_TRY(ctx, cudaGetLastError());
  prof_end(ctx, s, ev, MAPI_KC_MINCOV, (double)X->rows * X->cols * elem_bytes(X->storage),
           (double)X->rows * (X->rows + 1) / 2 * X->cols);
  count_launch(ctx);
  k_mincov_reduce<<<nt, 256, 0, s>>>(part, nt, nsplit, X->rows, denom, C, ldc);
  MAPI_CUDA_TRY(ctx, cudaGetLastError());
  count_launch(ctx);
  return MAPI_OK;
}

struct PairLaunch {
  const void* fn = nullptr;
  int rw = 0;
  int clusters = 0;
  size_t smem = 0;
  CUtensorMap map;
};

template <int OP, int ST>
static const void* pair_fn(int rw) {
  switch (rw) {
    case 8: return (const void*)k_pair_partial<OP, ST, 8>;
    case 16: return (const void*)k_pair_partial<OP, ST, 16>;
    case 32: return (const void*)k_pair_partial<OP, ST, 32>;
  }
  return nullptr;
}

static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    else
      cudaGetLastError();
  }
  return fn;
}

static mapi_status plan_pair(mapi_ctx* ctx, const mapi_mat* X, mapi_op op, PairLaunch* pl) {
  const int D = X->rows;
  int rw = 8;
  while (kPairCluster * kPairWarps * rw < D && rw < 32) rw *= 2;
  if (kPairCluster * kPairWarps * rw < D)
    return fail(ctx, MAPI_EINVAL, "pair mode supports D <= 1024");
  const void* fn = nullptr;
  CUtensorMapDataType dt;
  int tc;
  if (X->storage == MAPI_ST_F32) {
    fn = op == MAPI_OP_MIN1 ? pair_fn<MAPI_OP_MIN1, kF32>(rw)
         : op == MAPI_OP_MIN2 ? pair_fn<MAPI_OP_MIN2, kF32>(rw)
                              : pair_fn<MAPI_OP_DOT, kF32>(rw);
    dt = CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    tc = 32;
  } else if (X->storage == MAPI_ST_BF16) {
    fn = op == MAPI_OP_MIN1 ? pair_fn<MAPI_OP_MIN1, kBF16>(rw)
         : op == MAPI_OP_MIN2 ? pair_fn<MAPI_OP_MIN2, kBF16>(rw)
                              : pair_fn<MAPI_OP_DOT, kBF16>(rw);
    dt = CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    tc = 64;
  } else {
    return fail(ctx, MAPI_EINVAL, "pair mode supports F32 and BF16 storage");
  }
  const int rc = kPairWarps * rw;
  const int d_pad = kPairCluster * rc;
  // the stage ring, reused by the last cluster's epilogue
  pl->smem = std::max((size_t)kPairStages * rc * 128,
                      (size_t)pair_epi_floats(rc, d_pad) * sizeof(float));
  MAPI_CUDA_TRY(ctx, cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)pl->smem));
  // the tensor map: X as [rows_pad][ld] with a (tc x rc) box; rows and
  // columns beyond the matrix read as zero
  PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
  if (!enc) return fail(ctx, MAPI_ECUDA, "cuTensorMapEncodeTiled unavailable");
  const int eb = elem_bytes(X->storage);
  cuuint64_t gdim[2] = {(cuuint64_t)X->ld, (cuuint64_t)X->rows_pad};
  cuuint64_t gstride[1] = {(cuuint64_t)X->ld * eb};
  cuuint32_t box[2] = {(cuuint32_t)tc, (cuuint32_t)rc};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(&pl->map, dt, 2, X->data, gdim, gstride, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(ctx, MAPI_ECUDA, "tensor map encoding failed");
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = kPairCluster;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3(kPairCluster * ctx->sm_count, 1, 1);
  cfg.blockDim = dim3(kPairWarps * 32, 1, 1);
  cfg.dynamicSmemBytes = pl->smem;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int nclusters = 0;
  MAPI_CUDA_TRY(ctx, cudaOccupancyMaxActiveClusters(&nclusters, fn, &cfg));
  if (nclusters < 1) return fail(ctx, MAPI_ECUDA, "pair kernel: no cluster fits");
  pl->fn = fn;
  pl->rw = rw;
  pl->clusters = std::min(nclusters, kPairMaxClusters);
  return MAPI_OK;
}

// Tiles per cluster whose lines are kept in L2 for the next step: together
// they fill about 60 % of L2 (the rest: stages, partials and the data of
// other streams).  When that covers all of a cluster's tiles, X stays in L2.
static int pair_keep_tiles(const mapi_ctx* ctx, const mapi_mat* X, const PairLaunch& pl) {
  const int TC = (X->storage == MAPI_ST_F32) ? 32 : 64;
  const double tile_bytes = (double)kPairCluster * kPairWarps * pl.rw * TC * elem_bytes(X->storage);
  const double keep = 0.6 * ctx->l2_bytes / (tile_bytes * pl.clusters);
  return keep < 0 ? 0 : (int)keep;
}

static mapi_status launch_pair_step(mapi_ctx* ctx, cudaStream_t s, const PairLaunch& pl,
                                    const mapi_mat* X, const float* w, float* w_next,
                                    float* ypart, const DeflArgs& defl, IterCtl* ctl,
                                    int norm_l2, float denom, int reverse) {
  PairArgs pa;
  pa.reverse = reverse;
  pa.keep_tiles = pair_keep_tiles(ctx, X, pl);
  pa.D = X->rows;
  const int TC = (X->storage == MAPI_ST_F32) ? 32 : 64;
  pa.ntiles = (int)((X->ld + TC - 1) / TC);
  pa.nclusters = pl.clusters;
  pa.w = w;
  pa.w_next = w_next;
  pa.ypart = ypart;
  pa.D_pad = kPairCluster * kPairWarps * pl.rw;
  pa.ctl = ctl;
  pa.defl = defl;
  pa.norm_l2 = norm_l2;
  pa.denom = denom;
  pa.stall_ns = ctx->stall_ns;
  pa.phases = ctx->phases_on ? (PairPhases*)ctx->pair_phases.p : nullptr;
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = kPairCluster;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  // the step may start streaming X while the previous one finishes
  attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[1].val.programmaticStreamSerializationAllowed = 1;
  cfg.gridDim = dim3(kPairCluster * pl.clusters, 1, 1);
  cfg.blockDim = dim3(kPairWarps * 32, 1, 1);
  cfg.dynamicSmemBytes = pl.smem;
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = 2;
  void* args[] = {(void*)&pl.map, &pa};
  cudaEvent_t ev = prof_begin(ctx, s);
  MAPI_CUDA_TRY(ctx, cudaLaunchKernelExC(&cfg, pl.fn, args));
  prof_end(ctx, s, ev, MAPI_KC_PAIR, (double)X->rows * X->cols * elem_bytes(X->storage),
           2.0 * X->rows * X->cols);
  count_launch(ctx);
  return MAPI_OK;
}

// Scratch of the min-covariance splits for X (the launcher grows it; callers
// that capture graphs size it first).
size_t mincov_scratch_bytes(const mapi_ctx* ctx, const mapi_mat* X) {
  const int T = (X->rows + kMcT - 1) / kMcT;
  const int nt = T * (T + 1) / 2;
  int nsplit = 1;
  while (nt * nsplit < 4 * ctx->sm_count && X->ld / (nsplit * 2) >= 4 * kMcK) nsplit *= 2;
  return sizeof(float) * (size_t)nsplit * nt * kMcT * kMcT;
}

namespace {

// Everything one PCA solve touches on the device, sized before capture.
struct PcaPlan {
  int D = 0, k = 0, mode = 0, iters = 0;
  mapi_op op = MAPI_OP_MIN1;
  double tol = 0, denom = 1;
  int64_t ldq = 0;
  int* rec = nullptr;    // [iters 64][status 64][abort]
  int* abort = nullptr;
  // min-covariance mode
  mapi_mat Cm, Ck;
  float* Q = nullptr;
  // pair mode
  PairLaunch pl;
  int D_pad = 0;
  int64_t wst = 0;
  void* defl = nullptr;
};

mapi_status pca_enqueue(mapi_ctx* ctx, cudaStream_t s, const mapi_mat* X, const PcaPlan& p,
                        const float* w0, float* P_out) {
  mapi_status st = MAPI_OK;
  const int D = p.D, k = p.k;
  MAPI_CUDA_TRY(ctx, cudaMemsetAsync(p.rec, 0, sizeof(int) * 129, s));
  if (p.mode == MAPI_PCA_MINCOV) {
    const size_t bytes = sizeof(float) * p.Cm.rows_pad * p.Cm.ld;
    MAPI_CUDA_TRY(ctx, cudaMemsetAsync(p.Cm.data, 0, bytes, s));
    MAPI_CUDA_TRY(ctx, cudaMemsetAsync(p.Ck.data, 0, bytes, s));
    if ((st = launch_mincov_raw(ctx, X, p.op, (float)p.denom, (float*)p.Cm.data, p.Cm.ld, s)) !=
        MAPI_OK)
      return st;
    for (int c = 0; c < k; ++c) {
      const mapi_mat* A = &p.Cm;
      if (c > 0) {
        // Alg. 2 step 6: C_c = C - sum_{m<c} P_m C (p.Q holds the transposed product)
        if ((st = launch_deflate_mincov(ctx, p.op, P_out, D, c, D, (const float*)p.Cm.data,
                                        p.ldq, p.Q, p.defl, k, outer_stride(D),
                                        (float*)p.Ck.data, s)) != MAPI_OK)
          return st;
        A = &p.Ck;
      }
      if ((st = enqueue_solve(ctx, s, A, p.op, 1, w0 + (int64_t)c * D, D, p.iters, p.tol,
                              MAPI_FLAG_FINAL_L2, P_out + (int64_t)c * D, D, p.abort)) != MAPI_OK)
        return st;
      k_record<<<1, 1, 0, s>>>((const IterCtl*)ctx->ctl.p, p.rec, p.rec + 64, p.abort, c);
      MAPI_CUDA_TRY(ctx, cudaGetLastError());
      count_launch(ctx);
    }
    return MAPI_OK;
  }
  // pair mode
  float* wb0 = (float*)ctx->wbuf0.p;
  float* wb1 = (float*)ctx->wbuf1.p;
  IterCtl* ctl = (IterCtl*)ctx->ctl.p;
  const int norm_l2 = (p.op == MAPI_OP_DOT) ? 1 : 0;
  const OuterSlot slot0 = outer_slot(p.defl, k, p.D_pad, 0);
  DeflArgs defl{};
  defl.op = p.op;
  // dot deflates with the kept unit-l2 components, min1 / min2 with their
  // unit-l1 copies (launch_outer_prep)
  defl.P = p.op == MAPI_OP_DOT ? P_out : slot0.wt;
  defl.ldp = p.op == MAPI_OP_DOT ? D : p.D_pad;
  defl.stride = p.D_pad;
  defl.perm = slot0.perm;
  defl.wsort = slot0.wsort;
  defl.ubi = slot0.ubi;
  for (int c = 0; c < k; ++c) {
    if (c > 0 && p.op != MAPI_OP_DOT) {
      if ((st = launch_outer_prep(ctx, p.op, P_out + (int64_t)(c - 1) * D, D,
                                  outer_slot(p.defl, k, p.D_pad, c - 1), s)) != MAPI_OK)
        return st;
    }
    defl.nprev = c;
    if ((st = launch_start_float(ctx, s, w0 + (int64_t)c * D, D, D, 1, wb0, wb1, p.wst, 0, ctl,
                                 (float)p.tol, p.abort)) != MAPI_OK)
      return st;
    for (int t = 0; t < p.iters; ++t) {
      const float* wc = (t & 1) ? wb1 : wb0;
      float* wn = (t & 1) ? wb0 : wb1;
      // the tile order alternates over all steps of all components
      if ((st = launch_pair_step(ctx, s, p.pl, X, wc, wn, (float*)ctx->ypart.p, defl, ctl,
                                 norm_l2, (float)p.denom, (c * p.iters + t) & 1)) != MAPI_OK)
        return st;
    }
    if ((st = launch_finish(ctx, s, wb0, wb1, p.wst, D, 1, ctl, 1, 0, 0, P_out + (int64_t)c * D,
                            D)) != MAPI_OK)
      return st;
    k_record<<<1, 1, 0, s>>>(ctl, p.rec, p.rec + 64, p.abort, c);
    MAPI_CUDA_TRY(ctx, cudaGetLastError());
    count_launch(ctx);
  }
  return MAPI_OK;
}

}  // namespace

mapi_status run_pca(mapi_ctx* ctx, const mapi_mat* X, int k, int mode, mapi_op op, int iters,
                    double tol, double denom, const float* w0, float* P_out, int* iters_done) {
  if (mode != MAPI_PCA_MINCOV && mode != MAPI_PCA_PAIR)
    return fail(ctx, MAPI_EINVAL, "mode must be MINCOV or PAIR");
  PcaPlan p;
  p.D = X->rows;
  p.k = k;
  p.mode = mode;
  p.op = op;
  p.iters = iters;
  p.tol = tol;
  p.denom = denom;
  p.ldq = (p.D + 3) / 4 * 4;
  mapi_status st;
  // ---- every allocation happens here, before any capture
  if ((st = ensure(ctx, ctx->aux, 64 + sizeof(int) * 129)) != MAPI_OK) return st;
  if (mode == MAPI_PCA_MINCOV) {
    p.Cm.rows = p.Cm.cols = p.D;
    p.Cm.rows_pad = (p.D + 63) / 64 * 64;
    p.Cm.ld = p.ldq;
    p.Cm.storage = MAPI_ST_F32;
    p.Cm.owner = ctx;
    p.Ck = p.Cm;
    const size_t bytes = sizeof(float) * p.Cm.rows_pad * p.Cm.ld;
    if ((st = ensure(ctx, ctx->pca_c0, bytes)) != MAPI_OK ||
        (st = ensure(ctx, ctx->pca_c1, bytes)) != MAPI_OK ||
        (st = ensure(ctx, ctx->mcpart, mincov_scratch_bytes(ctx, X))) != MAPI_OK)
      return st;
    if (k > 1) {
      if (p.D > kOuterMaxD)
        return fail(ctx, MAPI_ENOTSUP, "min-covariance deflation supports D <= 16384");
      if ((st = ensure(ctx, ctx->pca_q, sizeof(float) * p.D * p.ldq)) != MAPI_OK ||
          (st = ensure(ctx, ctx->pca_defl, outer_scratch_bytes(k, p.D))) != MAPI_OK)
        return st;
    }
    if ((st = prepare_solve(ctx, &p.Cm, 1)) != MAPI_OK) return st;
  } else {
    if ((st = plan_pair(ctx, X, op, &p.pl)) != MAPI_OK) return st;
    p.D_pad = kPairCluster * kPairWarps * p.pl.rw;
    p.wst = (p.D_pad + 15) / 16 * 16;
    if ((st = ensure(ctx, ctx->wbuf0, sizeof(float) * p.wst)) != MAPI_OK ||
        (st = ensure(ctx, ctx->wbuf1, sizeof(float) * p.wst)) != MAPI_OK ||
        (st = ensure(ctx, ctx->ypart,
                     sizeof(float) * (size_t)p.pl.clusters * p.D_pad)) != MAPI_OK ||
        (st = ensure(ctx, ctx->ctl, sizeof(IterCtl))) != MAPI_OK ||
        (st = ensure(ctx, ctx->pca_defl, sizeof(float) * 4 * (size_t)k * p.D_pad)) != MAPI_OK)
      return st;
  }
  if ((st = outer_prepare(ctx)) != MAPI_OK) return st;
  // addresses are final now (ensure may have moved buffers and dropped graphs)
  p.rec = (int*)((char*)ctx->aux.p + 64);
  p.abort = p.rec + 128;
  p.Cm.data = ctx->pca_c0.p;
  p.Ck.data = ctx->pca_c1.p;
  p.Q = (float*)ctx->pca_q.p;
  p.defl = ctx->pca_defl.p;

  uint64_t tb, db;
  std::memcpy(&tb, &tol, 8);
  std::memcpy(&db, &denom, 8);
  std::vector<int64_t> key = {2,
                              (int64_t)X->id,
                              k,
                              mode,
                              (int64_t)op,
                              iters,
                              (int64_t)tb,
                              (int64_t)db,
                              (int64_t)(uintptr_t)w0,
                              (int64_t)(uintptr_t)P_out,
                              (int64_t)ctx->prof_on,
                              (int64_t)(uintptr_t)ctx->aux.p,
                              (int64_t)(uintptr_t)ctx->wbuf0.p,
                              (int64_t)(uintptr_t)ctx->ypart.p,
                              (int64_t)(uintptr_t)ctx->pca_c0.p,
                              (int64_t)(uintptr_t)ctx->pca_defl.p,
                              (int64_t)ctx->stall_ns,
                              (int64_t)(ctx->phases_on ? (uintptr_t)ctx->pair_phases.p : 0)};
  GraphEntry* ge = nullptr;
  st = launch_cached_graph(
      ctx, key, [&](cudaStream_t cs) { return pca_enqueue(ctx, cs, X, p, w0, P_out); }, &ge);
  if (st != MAPI_OK) return st;
  MAPI_CUDA_TRY(ctx, cudaMemcpyAsync(ctx->rec_host, p.rec, sizeof(int) * 128,
                                     cudaMemcpyDeviceToHost, ctx->stream));
  MAPI_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  finish_graph(ctx, ge);
  mapi_status result = MAPI_OK;
  for (int c = 0; c < k; ++c) {
    if (iters_done) iters_done[c] = ctx->rec_host[c];
    if (result == MAPI_OK && ctx->rec_host[64 + c] != MAPI_OK)
      result = (mapi_status)ctx->rec_host[64 + c];
  }
  if (result != MAPI_OK) fail(ctx, result, "a component stopped early with this status");
  return result;
}

}  // namespace mapi
