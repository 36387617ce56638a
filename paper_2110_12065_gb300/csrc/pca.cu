// PCA by MAPI: min-covariance build (Eq. (5)), deflation (Alg. 2 step 6 with
// the sum form after Eq. (2)), the matrix-free pair step, and the top-k
// drivers for both modes.
#include <cooperative_groups.h>
#include <cuda.h>
#include <cudaTypedefs.h>

#include <cmath>

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

// Sum the splits of each tile in order, divide by denom, write C and its mirror.
__global__ void k_mincov_reduce(const float* __restrict__ part, int ntiles, int nsplit, int D,
                                float denom, float* __restrict__ C, int64_t ldc) {
  const int T = (D + kMcT - 1) / kMcT;
  int tp, tq;
  mc_tile_of(blockIdx.x, T, tp, tq);
  for (int e = threadIdx.x; e < kMcT * kMcT; e += blockDim.x) {
    const int i = e / kMcT, j = e % kMcT;
    const int p = tp * kMcT + i, q = tq * kMcT + j;
    if (p >= D || q >= D) continue;
    float s = 0.f;
    for (int k = 0; k < nsplit; ++k) s += part[((int64_t)k * ntiles + blockIdx.x) * kMcT * kMcT + e];
    const float v = s / denom;
    C[(int64_t)p * ldc + q] = v;
    if (tp != tq) C[(int64_t)q * ldc + p] = v;
  }
}

// ======================================================================
// Deflation operator Q = sum_{m<c} w_m (+) w_m^T (entry (i, j) =
// sum_m term(w_m[i], w_m[j])), from the finished l2-normalised components.
// ======================================================================
template <int OP>
__global__ void k_build_Q(const float* __restrict__ P, int64_t ldp, int c, int D,
                          float* __restrict__ Q, int64_t ldq) {
  const int64_t total = (int64_t)D * D;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(t / D), j = (int)(t % D);
    float s = 0.f;
    for (int m = 0; m < c; ++m) {
      const float wi = P[(int64_t)m * ldp + i], wj = P[(int64_t)m * ldp + j];
      s += (OP == MAPI_OP_DOT) ? wi * wj : Op<OP>::term(wi, Op<OP>::prep(wj), 0.f);
    }
    Q[(int64_t)i * ldq + j] = s;
  }
}

// C_c = C - Q C (ordinary FP32 product), 64 x 64 tiles, 4 x 4 micro-tiles.
__global__ void __launch_bounds__(256)
    k_deflate_gemm(const float* __restrict__ Cm, const float* __restrict__ Q, int D,
                   int64_t ld, float* __restrict__ Ck) {
  __shared__ float Qs[16][65];
  __shared__ float Cs[16][65];
  const int i0 = blockIdx.y * 64, j0 = blockIdx.x * 64;
  const int ty = threadIdx.x >> 4, tx = threadIdx.x & 15;
  float acc[4][4] = {};
  for (int l0 = 0; l0 < D; l0 += 16) {
    for (int e = threadIdx.x; e < 64 * 16; e += 256) {
      const int r = e >> 4, l = e & 15;
      Qs[l][r] = (i0 + r < D && l0 + l < D) ? Q[(int64_t)(i0 + r) * ld + l0 + l] : 0.f;
      const int l2 = e >> 6, c2 = e & 63;
      Cs[l2][c2] = (l0 + l2 < D && j0 + c2 < D) ? Cm[(int64_t)(l0 + l2) * ld + j0 + c2] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int l = 0; l < 16; ++l) {
      float a[4], bb[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = Qs[l][ty * 4 + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) bb[j] = Cs[l][tx * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], bb[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int r = i0 + ty * 4 + i, c = j0 + tx * 4 + j;
      if (r < D && c < D) Ck[(int64_t)r * ld + c] = Cm[(int64_t)r * ld + c] - acc[i][j];
    }
}

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
constexpr long long kWaitLimitNs = 2000000000LL;  // bounded waits: 2 s

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

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ long long globaltimer_ns() {
  long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
// Bounded wait on an mbarrier phase; false when the limit ran out.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity) {
  const uint32_t a = smem_u32(bar);
  long long t0 = 0;
  for (int i = 0;; ++i) {
    uint32_t ok;
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; "
        "selp.u32 %0, 1, 0, p; }"
        : "=r"(ok)
        : "r"(a), "r"(parity)
        : "memory");
    if (ok) return true;
    if (i == 0) t0 = globaltimer_ns();
    else if (globaltimer_ns() - t0 > kWaitLimitNs) return false;
  }
}
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes "
      "[%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst)),
      "l"(map), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

struct PairArgs {
  int D;          // logical rows
  int ntiles;     // column tiles
  int nclusters;
  const float* w;  // current iterate (D entries + zero padding)
  float* ypart;    // [nclusters][D_pad]
  int D_pad;       // rows covered by one cluster (4 * 8 * RW)
  IterCtl* ctl;
};

template <int OP, int ST, int RW>
__global__ void __launch_bounds__(kPairWarps * 32, 2)
    k_pair_partial(const __grid_constant__ CUtensorMap xmap, PairArgs a) {
  if (*(volatile const int*)&a.ctl->all_done) return;
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
  __shared__ __align__(8) uint64_t full[kPairStages];
  __shared__ float4 wp[RC];                 // (lo, hi, s, 0) per row of this CTA
  __shared__ float tbuf[kPairWarps][TC];    // per-warp column partials
  __shared__ float cpart[2][TC];            // CTA column partials (DSMEM-visible)
  __shared__ int s_err;

  const int nmine = a.ntiles > cid ? (a.ntiles - cid + a.nclusters - 1) / a.nclusters : 0;
  if (threadIdx.x == 0) {
    s_err = 0;
    for (int s = 0; s < kPairStages; ++s) mbar_init(&full[s], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  for (int r = threadIdx.x; r < RC; r += blockDim.x) {
    const int d = (int)crank * RC + r;
    const float wv = d < a.D ? a.w[d] : 0.f;
    const auto p = Op<OP>::prep(wv);
    if constexpr (OP == MAPI_OP_DOT) wp[r] = make_float4(p.w, 0.f, 0.f, 0.f);
    else wp[r] = make_float4(p.lo, p.hi, p.s, 0.f);
  }
  __syncthreads();
  auto issue = [&](int j) {
    const int s = j % kPairStages;
    const int tile = cid + j * a.nclusters;
    mbar_expect_tx(&full[s], kStageBytes);
    tma_load_2d(stage + (size_t)s * RC * 32, &xmap, tile * TC, (int)crank * RC, &full[s]);
  };
  if (threadIdx.x == 0)
    for (int j = 0; j < nmine && j < kPairStages; ++j) issue(j);

  float acc[RW];
#pragma unroll
  for (int j = 0; j < RW; ++j) acc[j] = 0.f;

  for (int j = 0; j < nmine; ++j) {
    const int s = j % kPairStages;
    const int par = j & 1;
    const bool ok = mbar_wait(&full[s], (unsigned)((j / kPairStages) & 1));
    if (!ok) s_err = 1;
    uint32_t raw[RW];
    const uint32_t* src = stage + (size_t)s * RC * 32 + (size_t)(warp * RW) * 32 + lane;
#pragma unroll
    for (int jj = 0; jj < RW; ++jj) raw[jj] = src[jj * 32];
    // column partials over this warp's rows
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
    for (int c = 0; c < CPL; ++c) tbuf[warp][lane * CPL + c] = tp[c];
    __syncthreads();
    // every warp has read stage s: refill it with tile j + S
    if (threadIdx.x == 0 && j + kPairStages < nmine && !s_err) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      issue(j + kPairStages);
    }
    if (warp == 0) {
#pragma unroll
      for (int c = 0; c < CPL; ++c) {
        float sum = 0.f;
#pragma unroll
        for (int w = 0; w < kPairWarps; ++w) sum += tbuf[w][lane * CPL + c];
        cpart[par][lane * CPL + c] = sum;
      }
    }
    cluster.sync();
    // t over the whole cluster, same order in every CTA
    typename Op<OP>::P tpar[CPL];
#pragma unroll
    for (int c = 0; c < CPL; ++c) {
      float t = 0.f;
#pragma unroll
      for (int r = 0; r < kPairCluster; ++r) {
        const float* rem = cluster.map_shared_rank(&cpart[par][0], r);
        t += rem[lane * CPL + c];
      }
      tpar[c] = Op<OP>::prep(t);
    }
#pragma unroll
    for (int jj = 0; jj < RW; ++jj) {
      float x[CPL];
      PC::get(raw[jj], x);
#pragma unroll
      for (int c = 0; c < CPL; ++c) acc[jj] = Op<OP>::term(x[c], tpar[c], acc[jj]);
    }
  }
  // row sums across the 32 lanes, written once per cluster
#pragma unroll
  for (int jj = 0; jj < RW; ++jj) {
    float sum = acc[jj];
#pragma unroll
    for (int o = 16; o; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    if (lane == 0) a.ypart[(int64_t)cid * a.D_pad + rbase + jj] = sum;
  }
  if (threadIdx.x == 0 && s_err) {
    // a tile never arrived: report it; later kernels of the solve stop
    a.ctl->v[0].status = MAPI_ETIMEOUT;
    a.ctl->v[0].done = 1;
    a.ctl->all_done = 1;
  }
  cluster.sync();  // no CTA leaves while a peer may still read its cpart
}

// ======================================================================
// Pair-step finish: one cluster of CS CTAs.  CTA r owns rows [r*RS,
// (r+1)*RS): it reduces the cluster partials (fixed order), deflates
// u = y - Q y (Q dense, optional), and after a cluster-wide norm normalises
// w_next = u / ||u||_1 (||u||_2 for DOT), computes delta and the stop test.
// ======================================================================
constexpr int kFinThreads = 256;

struct FinishArgs {
  const float* ypart;
  int nparts;
  int D, D_pad;
  const float* Q;  // D x D (ld = ldq) or null
  int64_t ldq;
  const float* w;
  float* w_next;
  IterCtl* ctl;
  int norm_l2;
  float denom;
};

__global__ void __launch_bounds__(kFinThreads) k_pair_finish(FinishArgs a) {
  if (*(volatile int*)&a.ctl->all_done) return;
  cg::cluster_group cluster = cg::this_cluster();
  const int CS = (int)cluster.num_blocks();
  const int r = (int)cluster.block_rank();
  const int RS = a.D_pad / CS;
  const int r0 = r * RS;
  extern __shared__ float fsh[];
  float* ys = fsh;               // RS    own rows of y (read by peers)
  float* u = fsh + RS;           // RS    own rows after deflation
  float* yfull = fsh + 2 * RS;   // D_pad gathered y
  __shared__ float red[33];
  __shared__ float part[4];      // [0] norm partial, [1] delta partial

  // 1. y for own rows: sum over partials in order; 4 threads per row
  for (int i = threadIdx.x >> 2; i < RS; i += kFinThreads / 4) {
    const int d = r0 + i;
    float s = 0.f;
    for (int g = (threadIdx.x & 3); g < a.nparts; g += 4) s += a.ypart[(int64_t)g * a.D_pad + d];
    s += __shfl_xor_sync(0xffffffffu, s, 1);
    s += __shfl_xor_sync(0xffffffffu, s, 2);
    if ((threadIdx.x & 3) == 0) ys[i] = (d < a.D) ? s / a.denom : 0.f;
  }
  cluster.sync();
  // 2. deflation u = y - Q y (needs the whole y)
  if (a.Q) {
    for (int i = threadIdx.x; i < a.D_pad; i += kFinThreads) {
      const float* rem = cluster.map_shared_rank(ys, i / RS);
      yfull[i] = rem[i % RS];
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = warp; i < RS; i += kFinThreads / 32) {
      const int d = r0 + i;
      float s = 0.f;
      if (d < a.D) {
        const float* qrow = a.Q + (int64_t)d * a.ldq;
        for (int j = lane; j < a.D; j += 32) s = fmaf(qrow[j], yfull[j], s);
      }
#pragma unroll
      for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (lane == 0) u[i] = (d < a.D) ? ys[i] - s : 0.f;
    }
    __syncthreads();
  } else {
    for (int i = threadIdx.x; i < RS; i += kFinThreads) u[i] = ys[i];
    __syncthreads();
  }
  // 3. norm partial of own rows
  Kahan k;
  for (int i = threadIdx.x; i < RS; i += kFinThreads) {
    const float x = u[i];
    k.add(a.norm_l2 ? x * x : fabsf(x));
  }
  const float np = block_sum<kFinThreads>(k.value(), red);
  if (threadIdx.x == 0) part[0] = np;
  cluster.sync();
  float L = 0.f;
  for (int q = 0; q < CS; ++q) L += cluster.map_shared_rank(part, q)[0];
  if (a.norm_l2) L = sqrtf(L);
  const bool ok = (L > 0.f) && isfinite(L);
  Kahan dk;
  if (ok) {
    for (int i = threadIdx.x; i < RS; i += kFinThreads) {
      const int d = r0 + i;
      if (d >= a.D) continue;
      const float x = u[i] / L;
      dk.add(fabsf(x - a.w[d]));
      a.w_next[d] = x;
    }
  }
  const float dp = block_sum<kFinThreads>(dk.value(), red);
  if (threadIdx.x == 0) part[1] = dp;
  cluster.sync();
  if (r == 0 && threadIdx.x == 0) {
    VecState* st = &a.ctl->v[0];
    if (!ok) {
      st->status = (L == 0.f) ? MAPI_EZERONORM : MAPI_ENONFINITE;
      st->done = 1;
    } else {
      float D = 0.f;
      for (int q = 0; q < CS; ++q) D += cluster.map_shared_rank(part, q)[1];
      st->iters += 1;
      st->delta = D;
      st->norm = L;
      if (a.ctl->tol > 0.f && D < a.ctl->tol) st->done = 1;
    }
    a.ctl->all_done = st->done;
  }
  cluster.sync();
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

static mapi_status launch_build_Q(mapi_ctx* ctx, mapi_op op, const float* P, int64_t ldp,
                                  int c, int D, float* Q, int64_t ldq, cudaStream_t s) {
  const int64_t total = (int64_t)D * D;
  const int g = (int)std::min<int64_t>((total + 255) / 256, (int64_t)ctx->sm_count * 16);
  if (op == MAPI_OP_MIN1) k_build_Q<MAPI_OP_MIN1><<<g, 256, 0, s>>>(P, ldp, c, D, Q, ldq);
  else if (op == MAPI_OP_MIN2) k_build_Q<MAPI_OP_MIN2><<<g, 256, 0, s>>>(P, ldp, c, D, Q, ldq);
  else k_build_Q<MAPI_OP_DOT><<<g, 256, 0, s>>>(P, ldp, c, D, Q, ldq);
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
  pl->smem = (size_t)kPairStages * rc * 128;
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
  pl->clusters = nclusters;
  return MAPI_OK;
}

static int finish_cluster_size(mapi_ctx* ctx, int D_pad) {
  static int cached = 0;
  if (cached) return cached;
  cudaFuncSetAttribute(k_pair_finish, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  for (int cs : {16, 8, 4}) {
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cs;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(cs, 1, 1);
    cfg.blockDim = dim3(kFinThreads, 1, 1);
    cfg.dynamicSmemBytes = (size_t)(2 * (D_pad / cs) + D_pad) * sizeof(float);
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, (const void*)k_pair_finish, &cfg) == cudaSuccess && n > 0) {
      cached = cs;
      return cs;
    }
    cudaGetLastError();
  }
  (void)ctx;
  return 0;
}

static mapi_status launch_pair_step(mapi_ctx* ctx, cudaStream_t s, const PairLaunch& pl,
                                    const mapi_mat* X, const float* w, float* w_next,
                                    float* ypart, const float* Q, int64_t ldq, int fcs,
                                    IterCtl* ctl, int norm_l2, float denom) {
  PairArgs pa;
  pa.D = X->rows;
  const int TC = (X->storage == MAPI_ST_F32) ? 32 : 64;
  pa.ntiles = (int)((X->ld + TC - 1) / TC);
  pa.nclusters = pl.clusters;
  pa.w = w;
  pa.ypart = ypart;
  pa.D_pad = kPairCluster * kPairWarps * pl.rw;
  pa.ctl = ctl;
  {
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = kPairCluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(kPairCluster * pl.clusters, 1, 1);
    cfg.blockDim = dim3(kPairWarps * 32, 1, 1);
    cfg.dynamicSmemBytes = pl.smem;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    void* args[] = {(void*)&pl.map, &pa};
    cudaEvent_t ev = prof_begin(ctx, s);
    MAPI_CUDA_TRY(ctx, cudaLaunchKernelExC(&cfg, pl.fn, args));
    prof_end(ctx, s, ev, MAPI_KC_PAIR, (double)X->rows * X->cols * elem_bytes(X->storage),
             2.0 * X->rows * X->cols);
    count_launch(ctx);
  }
  FinishArgs fa;
  fa.ypart = ypart;
  fa.nparts = pl.clusters;
  fa.D = X->rows;
  fa.D_pad = pa.D_pad;
  fa.Q = Q;
  fa.ldq = ldq;
  fa.w = w;
  fa.w_next = w_next;
  fa.ctl = ctl;
  fa.norm_l2 = norm_l2;
  fa.denom = denom;
  {
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = fcs;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(fcs, 1, 1);
    cfg.blockDim = dim3(kFinThreads, 1, 1);
    cfg.dynamicSmemBytes = (size_t)(2 * (pa.D_pad / fcs) + pa.D_pad) * sizeof(float);
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaEvent_t ev = prof_begin(ctx, s);
    MAPI_CUDA_TRY(ctx, cudaLaunchKernelEx(&cfg, k_pair_finish, fa));
    prof_end(ctx, s, ev, MAPI_KC_PAIR_FINISH, 4.0 * pl.clusters * pa.D_pad, 0.0);
    count_launch(ctx);
  }
  return MAPI_OK;
}

mapi_status run_pca(mapi_ctx* ctx, const mapi_mat* X, int k, int mode, mapi_op op,
                    int iters, double tol, double denom, const float* w0, float* P_out,
                    int* iters_done) {
  const int D = X->rows;
  cudaStream_t s = ctx->stream;
  mapi_status st;
  // device scratch: Q (D x D), two iterate buffers, counters
  const int64_t ldq = (D + 3) / 4 * 4;
  int* rec = nullptr;  // [iters k][status k]
  if ((st = ensure(ctx, ctx->aux, 64 + sizeof(int) * 2 * 64 + 64)) != MAPI_OK) return st;
  rec = (int*)((char*)ctx->aux.p + 64);
  int* abort = rec + 128;
  MAPI_CUDA_TRY(ctx, cudaMemsetAsync(rec, 0, sizeof(int) * 129, s));
  float* Q = nullptr;
  DevBuf qbuf;
  if (k > 1) {
    if (cudaMalloc(&qbuf.p, sizeof(float) * D * ldq) != cudaSuccess) {
      cudaGetLastError();
      return fail(ctx, MAPI_ENOMEM, "deflation buffer");
    }
    Q = (float*)qbuf.p;
  }
  auto cleanup = [&]() {
    if (qbuf.p) {
      cudaStreamSynchronize(s);
      cudaFree(qbuf.p);
    }
  };
  const float fdenom = (float)denom;
  if (mode == MAPI_PCA_MINCOV) {
    // C and C_c live in internal F32 matrices so that the K1 path iterates them
    mapi_mat Cm, Ck;
    Cm.rows = Cm.cols = D;
    Cm.rows_pad = (D + 63) / 64 * 64;
    Cm.ld = ldq;
    Cm.storage = MAPI_ST_F32;
    Cm.owner = ctx;
    Ck = Cm;
    const size_t bytes = sizeof(float) * Cm.rows_pad * Cm.ld;
    if (cudaMalloc(&Cm.data, bytes) != cudaSuccess || cudaMalloc(&Ck.data, bytes) != cudaSuccess) {
      cudaGetLastError();
      if (Cm.data) cudaFree(Cm.data);
      cleanup();
      return fail(ctx, MAPI_ENOMEM, "covariance buffers");
    }
    auto free_c = [&]() {
      cudaStreamSynchronize(s);
      cudaFree(Cm.data);
      cudaFree(Ck.data);
    };
    MAPI_CUDA_TRY(ctx, cudaMemsetAsync(Cm.data, 0, bytes, s));
    MAPI_CUDA_TRY(ctx, cudaMemsetAsync(Ck.data, 0, bytes, s));
    if ((st = launch_mincov_raw(ctx, X, op, fdenom, (float*)Cm.data, Cm.ld, s)) != MAPI_OK) {
      free_c();
      cleanup();
      return st;
    }
    if ((st = prepare_solve(ctx, &Cm, 1)) != MAPI_OK) {
      free_c();
      cleanup();
      return st;
    }
    for (int c = 0; c < k; ++c) {
      const mapi_mat* A = &Cm;
      if (c > 0) {
        if ((st = launch_build_Q(ctx, op, P_out, D, c, D, Q, ldq, s)) != MAPI_OK) break;
        dim3 g((D + 63) / 64, (D + 63) / 64);
        k_deflate_gemm<<<g, 256, 0, s>>>((const float*)Cm.data, Q, D, ldq, (float*)Ck.data);
        MAPI_CUDA_TRY(ctx, cudaGetLastError());
        count_launch(ctx);
        A = &Ck;
      }
      if ((st = enqueue_solve(ctx, s, A, op, 1, w0 + (int64_t)c * D, D, iters, tol,
                              MAPI_FLAG_FINAL_L2, P_out + (int64_t)c * D, D, abort)) != MAPI_OK)
        break;
      k_record<<<1, 1, 0, s>>>((const IterCtl*)ctx->ctl.p, rec, rec + 64, abort, c);
      count_launch(ctx);
    }
    free_c();
  } else if (mode == MAPI_PCA_PAIR) {
    PairLaunch pl;
    if ((st = plan_pair(ctx, X, op, &pl)) != MAPI_OK) {
      cleanup();
      return st;
    }
    const int D_pad = kPairCluster * kPairWarps * pl.rw;
    const int fcs = finish_cluster_size(ctx, D_pad);
    // every warp of the finish kernel covers 8 whole rows per pass
    if (fcs && (D_pad / fcs) % 8 != 0) {
      cleanup();
      return fail(ctx, MAPI_EINVAL, "unsupported pair-mode row count");
    }
    if (!fcs) {
      cleanup();
      return fail(ctx, MAPI_ECUDA, "finish kernel: no cluster fits");
    }
    const int64_t wst = (D_pad + 15) / 16 * 16;
    if ((st = ensure(ctx, ctx->wbuf0, sizeof(float) * wst)) != MAPI_OK ||
        (st = ensure(ctx, ctx->wbuf1, sizeof(float) * wst)) != MAPI_OK ||
        (st = ensure(ctx, ctx->ypart, sizeof(float) * (size_t)pl.clusters * D_pad)) != MAPI_OK ||
        (st = ensure(ctx, ctx->ctl, sizeof(IterCtl))) != MAPI_OK) {
      cleanup();
      return st;
    }
    float* wb0 = (float*)ctx->wbuf0.p;
    float* wb1 = (float*)ctx->wbuf1.p;
    IterCtl* ctl = (IterCtl*)ctx->ctl.p;
    const int norm_l2 = (op == MAPI_OP_DOT) ? 1 : 0;
    for (int c = 0; c < k; ++c) {
      if (c > 0) {
        if ((st = launch_build_Q(ctx, op, P_out, D, c, D, Q, ldq, s)) != MAPI_OK) break;
      }
      if ((st = launch_start_float(ctx, s, w0 + (int64_t)c * D, D, D, 1, wb0, wb1, wst, 0, ctl,
                                   (float)tol, abort)) != MAPI_OK)
        break;
      for (int t = 0; t < iters; ++t) {
        const float* wc = (t & 1) ? wb1 : wb0;
        float* wn = (t & 1) ? wb0 : wb1;
        if ((st = launch_pair_step(ctx, s, pl, X, wc, wn, (float*)ctx->ypart.p,
                                   c > 0 ? Q : nullptr, ldq, fcs, ctl, norm_l2, fdenom)) !=
            MAPI_OK)
          break;
      }
      if (st != MAPI_OK) break;
      if ((st = launch_finish(ctx, s, wb0, wb1, wst, D, 1, ctl, 1, 0, 0,
                              P_out + (int64_t)c * D, D)) != MAPI_OK)
        break;
      k_record<<<1, 1, 0, s>>>(ctl, rec, rec + 64, abort, c);
      count_launch(ctx);
    }
  } else {
    cleanup();
    return fail(ctx, MAPI_EINVAL, "mode must be MINCOV or PAIR");
  }
  if (st != MAPI_OK) {
    cleanup();
    return st;
  }
  int host[128];
  MAPI_CUDA_TRY(ctx, cudaMemcpyAsync(host, rec, sizeof(int) * 128, cudaMemcpyDeviceToHost, s));
  MAPI_CUDA_TRY(ctx, cudaStreamSynchronize(s));
  prof_collect(ctx, ctx->pending, true);
  cleanup();
  mapi_status result = MAPI_OK;
  for (int c = 0; c < k; ++c) {
    if (iters_done) iters_done[c] = host[c];
    if (result == MAPI_OK && host[64 + c] != MAPI_OK) result = (mapi_status)host[64 + c];
  }
  if (result != MAPI_OK) fail(ctx, result, "a component stopped early with this status");
  return result;
}

}  // namespace mapi
