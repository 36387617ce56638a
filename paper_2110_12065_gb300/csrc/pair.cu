// Matrix-free PCA "pair" step (the MAVP counterpart of X (X^T w) / N):
//   t_n = x_n^T (+) w,   y_d = sum_n X_dn (+) t_n / denom,
// then the deflation of Alg. 2 step 6 in the sum form of §1 applied to the
// iterate, u = y - sum_m P_m y, and the normalisation of Eq. (6),
// w' = u / ||u||_1 (||u||_2 for DOT).  Every step of one component runs in
// one persistent launch of 4-CTA clusters:
//
//   * streaming clusters (all but the last) read X once per step: a 3-stage
//     TMA ring of column tiles, column partials t exchanged across the
//     cluster through DSMEM, row sums in registers.  Their row sums are
//     added into a fixed-point accumulator in global memory (exact 64-bit
//     integer additions, so the sum does not depend on the order in which
//     clusters finish), then each CTA signals its arrival.  The ring keeps
//     streaming the next step's tiles while the step is finished elsewhere.
//   * the last cluster finishes every step: it waits for all arrivals, turns
//     the accumulated sums back into y, deflates, normalises, writes the new
//     iterate and publishes it; each streaming CTA then reads its rows of
//     the new iterate and goes on.  The earlier components it deflates by
//     stay in its shared memory for the whole launch.
//
// Every wait (tile copies, cluster exchanges, arrivals, the published
// iterate) is bounded by %globaltimer; when one runs out the solve stops
// with MAPI_ETIMEOUT.  All clusters must be resident at once: the launch is
// cooperative where the driver accepts that for a cluster launch, and the
// grid never exceeds the clusters the occupancy calculator allows.
#include <cooperative_groups.h>
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>

#include "device_common.cuh"

namespace cg = cooperative_groups;

namespace mapi {
namespace {

constexpr int kPairWarps = 8, kPairCluster = kPairClusterCtas, kPairStages = 3;
constexpr int kPairThreads = kPairWarps * 32;
constexpr int kDeflMaxD = 1024;               // largest order of the pair mode
constexpr int kDeflPadded = kDeflMaxD + kDeflMaxD / 8;
constexpr int kEpiHalf = kPairThreads / 2;    // threads that load one component
constexpr int kAccCopies = 4;                 // accumulator copies (spreads the atomics)
constexpr int kPairMaxStream = 96;            // streaming clusters at most

// Shared state of one launch in global memory (zeroed before it).
struct PairSync {
  unsigned arrivals;           // streaming CTAs that finished a step, all steps
  int err;                     // a bounded wait ran out somewhere
  unsigned pad_[kPairCluster];
  unsigned xmax;               // max |X| as FP32 bits (the fixed-point scale)
};

struct PairSolveArgs {
  int D;           // rows of X (the order of the iterate)
  int D_pad;       // rows covered by one cluster (4 x 8 x RW)
  int ncols;       // columns of X (samples)
  int ntiles;      // column tiles
  int nstream;     // streaming clusters (the epilogue cluster comes after them)
  int T;           // steps of this launch
  int dir0;        // walk direction of step 0 (alternates every step)
  int nround;      // tiles every streaming cluster takes
  int nfirst;      // clusters that take the remaining tiles (>= 1)
  int norm_l2;
  float denom;
  float* wb0;      // iterate of even steps (holds w_0 at the start)
  float* wb1;      // iterate of odd steps
  unsigned long long* acc;  // [2][kAccCopies][D_pad] fixed-point row sums
  PairSync* sync;
  IterCtl* ctl;
  DeflArgs defl;
  long long stall_ns;  // > 0: fault-detection test (mapi_debug_stall)
  PairPhases* phases;  // non-null: phase stamps (mapi_pair_phases)
  float* raw_out;      // non-null: one step, its y (no deflation or norm) written here
  unsigned long long* wpub;  // [D_pad] the published iterate: value bits | tag << 32
};

template <int ST>
struct PairCols;
template <>
struct PairCols<kF32> {
  static constexpr int CPL = 1;  // columns per lane
  static __device__ __forceinline__ void get(uint32_t raw, float (&v)[1]) {
    v[0] = __uint_as_float(raw);
  }
  static __device__ __forceinline__ void get_b(uint32_t raw, float (&v)[1]) { get(raw, v); }
};
template <>
struct PairCols<kBF16> {
  static constexpr int CPL = 2;
  static __device__ __forceinline__ void get(uint32_t raw, float (&v)[2]) {
    v[0] = __uint_as_float(raw << 16);
    v[1] = __uint_as_float(raw & 0xFFFF0000u);
  }
  // The same values by byte permutes, for phase B: written differently from
  // get() so the compiler cannot keep phase A's widened values alive until
  // phase B (64 floats instead of 32 packed words, which spilled).
  static __device__ __forceinline__ void get_b(uint32_t raw, float (&v)[2]) {
    uint32_t lo, hi;
    asm("prmt.b32 %0, %1, %2, 0x1044;" : "=r"(lo) : "r"(raw), "r"(0u));
    asm("prmt.b32 %0, %1, %2, 0x3244;" : "=r"(hi) : "r"(raw), "r"(0u));
    v[0] = __uint_as_float(lo);
    v[1] = __uint_as_float(hi);
  }
};

__device__ __forceinline__ unsigned long long gtimer_u64() {
  return (unsigned long long)globaltimer_ns();
}
__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_u32(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void st_release_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
// Bounded spin until the tag (high word) of *p is >= tag; the word, or 0
// when the limit ran out.
__device__ unsigned long long wait_tag(const unsigned long long* p, unsigned tag) {
  long long t0 = 0;
  for (int i = 0;; ++i) {
    const unsigned long long v = ld_acquire_u64(p);
    if ((unsigned)(v >> 32) >= tag) return v;
    if (i == 0) t0 = globaltimer_ns();
    else if (globaltimer_ns() - t0 > kWaitLimitNs) return 0;
    if (i > 4096) __nanosleep(32);
  }
}
__device__ __forceinline__ void red_release_add_u32(unsigned* p, unsigned v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
// Bounded spin until *p >= target (acquire); the value seen, or 0 when the
// limit ran out.
__device__ unsigned wait_geq(const unsigned* p, unsigned target) {
  long long t0 = 0;
  for (int i = 0;; ++i) {
    const unsigned v = ld_acquire_u32(p);
    if (v >= target) return v;
    if (i == 0) t0 = globaltimer_ns();
    else if (globaltimer_ns() - t0 > kWaitLimitNs) return 0;
    if (i > 4096) __nanosleep(32);
  }
}

// Exponent s of the fixed-point scale 2^s: every row sum of a step, and the
// sum of all of them, is below 2^60 2^-s.  For MIN1 / MIN2 a term is at most
// |X_dn| (the min takes one of its operands), so a row sum is below
// ncols max|X|; for DOT |t_n| <= max|X| ||w||_1 <= max|X| sqrt(D) (w at unit
// l2 norm) adds max|X| sqrt(D_pad).
__device__ __forceinline__ int acc_scale_exp(float xmax, int ncols, int D_pad, bool dot) {
  if (!(xmax > 0.f)) return 0;
  int e = ilogbf(xmax) + 1 + (31 - __clz(ncols)) + 1;
  if (dot) e += ilogbf(xmax) + 1 + ((31 - __clz(D_pad)) + 2) / 2;
  return min(120, max(-120, 60 - e));
}

// Sum over the cluster of one float per CTA (at `slot` in every CTA's shared
// memory), read in parallel by the lanes of one warp and added in a fixed
// butterfly order; every thread of the block gets the result.
__device__ __forceinline__ float cluster_sum(cg::cluster_group& cluster, float* slot,
                                             float* bcast) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (warp == 0) {
    float v = lane < kPairCluster ? cluster.map_shared_rank(slot, lane)[0] : 0.f;
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) *bcast = v;
  }
  __syncthreads();
  const float r = *bcast;
  __syncthreads();
  return r;
}

// Two such sums at once, in one pass: slot[0] and slot[1] of every CTA,
// each added in a fixed order; every thread of the block gets both.
__device__ __forceinline__ float2 cluster_sum2(cg::cluster_group& cluster, float* slot,
                                               float* bcast) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (warp == 0) {
    const int which = lane >> 2, rk = lane & 3;
    float v = which < 2 ? cluster.map_shared_rank(slot, rk)[which] : 0.f;
    v += __shfl_xor_sync(0xffffffffu, v, 1);
    v += __shfl_xor_sync(0xffffffffu, v, 2);
    if (lane == 0) bcast[0] = v;
    if (lane == 4) bcast[1] = v;
  }
  __syncthreads();
  const float2 r = make_float2(bcast[0], bcast[1]);
  __syncthreads();
  return r;
}

// Index of sorted position p in a padded deflation array: the 32 lanes' runs
// of 8 positions [8 l, 8 l + 8) then fall on 32 different banks.
__device__ __forceinline__ int dpad(int p) { return p + (p >> 3); }

// Barrier of the 4 warps that deflate one component (named barriers 1, 2).
__device__ __forceinline__ void group_bar(int g) {
  asm volatile("bar.sync %0, %1;" ::"r"(1 + g), "r"(128) : "memory");
}

// Floats of shared memory the epilogue cluster needs per CTA: ys, u, wo (own
// rows), yfull and cbuf[2] (D_pad each), and per warp group four scan arrays
// and the component's w, sorted |w|, perm and ub (kDeflPadded each).
__host__ __device__ constexpr int pair_epi_floats(int rc, int d_pad) {
  return 3 * rc + 3 * d_pad + 2 * 8 * kDeflPadded;
}

// ---------------------------------------------------------------- epilogue
// The last cluster: every step, y = the accumulated row sums / denom,
// u = y - sum_m P_m y (prefix-sum form of the MIN1 / MIN2 outer product, or
// the projection for DOT; CTA r's warp group g owns the earlier components
// m = r + 4 g (mod 8)), w' = u / ||u||, the stop test, and the publication
// of CTA r's rows of w' to the streaming CTAs of rank r.
template <int RS, int OP, bool STAMP>
__device__ void pair_epilogue(const PairSolveArgs& a, cg::cluster_group& cluster, float* fsh,
                              int s_exp) {
  constexpr int CS = kPairCluster;
  constexpr int NT = kPairThreads;
  const int r = (int)cluster.block_rank();
  const int r0 = r * RS;
  const int D = a.D, D_pad = a.D_pad;
  const int h = threadIdx.x / kEpiHalf;
  const int th = threadIdx.x % kEpiHalf;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float* u = fsh;
  float* wo = u + RS;
  float* ys = wo + RS;
  float* yfull = ys + RS;
  float* cbuf = yfull + D_pad;  // [2][D_pad]: one per warp group
  auto arrays = [&](int g) { return cbuf + 2 * D_pad + g * 8 * kDeflPadded; };
  __shared__ float red[33];
  __shared__ float part[8];
  __shared__ float gtot[2][4][8];
  // each CTA pushes its norm partial and error flag into every CTA's nin
  // (st.async, counted by nbar) instead of a cluster barrier and remote reads
  __shared__ __align__(8) uint64_t nbar;
  __shared__ float nin[2][CS];
  if (threadIdx.x == 0) {
    mbar_init(&nbar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();  // no peer pushes before the first step's cluster barrier
  // the deflation's operator is the iteration's (DeflArgs::op == OP)
  constexpr bool dot = OP == MAPI_OP_DOT;
  constexpr bool two = OP == MAPI_OP_MIN2;
  const int nprev = a.defl.nprev;
  // with at most 8 earlier components each group's arrays stay resident
  const bool resident = nprev <= 2 * CS;

  // component m's vector, sorted |w| and the two index maps into group g's
  // padded arrays, loaded by the threads [t0, t0 + nt) (at most 8 entries
  // per thread, all loaded before the first is stored)
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
  if (r + CS * h < nprev) load_comp(r + CS * h, h, th, kEpiHalf);
  for (int i = threadIdx.x; i < RS; i += NT) wo[i] = r0 + i < D ? __ldcg(a.wb0 + r0 + i) : 0.f;
  __syncthreads();
  const float inv = ldexpf(1.f, -s_exp);
  const bool want_delta = a.ctl->tol > 0.f;
  const bool stamp = STAMP && a.phases && r == 0 && threadIdx.x == 0;

  for (int t = 0; t < a.T; ++t) {
    // 1. every streaming CTA has added its row sums of step t
    if (threadIdx.x == 0 &&
        !wait_geq(&a.sync->arrivals, 4u * (unsigned)a.nstream * (unsigned)(t + 1)))
      atomicExch(&a.sync->err, 1);
    __syncthreads();
    unsigned long long t_seen = 0, t_reduce = 0, t_defl = 0;
    if (stamp) t_seen = gtimer_u64();
    // 2. y = (sum of the fixed-point row sums) 2^-s / denom, all rows (each
    //    copy and row read once; the integer sum is exact)
    unsigned long long* accb = a.acc + (size_t)(t & 1) * kAccCopies * D_pad;
    {
      // D_pad = 4 RS rows, RS / 64 per thread: every load in flight at once
      constexpr int PER = 4 * RS / NT;
      long long v[PER][kAccCopies];
#pragma unroll
      for (int k = 0; k < PER; ++k)
#pragma unroll
        for (int c = 0; c < kAccCopies; ++c)
          v[k][c] = (long long)__ldcg(accb + (size_t)c * D_pad + threadIdx.x + k * NT);
#pragma unroll
      for (int k = 0; k < PER; ++k) {
        const int i = threadIdx.x + k * NT;
        long long s = 0;
#pragma unroll
        for (int c = 0; c < kAccCopies; ++c) s += v[k][c];
        yfull[i] = i < D ? __ll2float_rn(s) * inv / a.denom : 0.f;
      }
    }
    for (int i = threadIdx.x; i < 2 * D_pad; i += NT) cbuf[i] = 0.f;
    __syncthreads();
    for (int i = threadIdx.x; i < RS; i += NT) ys[i] = yfull[r0 + i];
    if (stamp) t_reduce = gtimer_u64();
    if (a.raw_out) {  // one unnormalised pair product (a column shard's partial)
      for (int i = threadIdx.x; i < RS; i += NT)
        if (r0 + i < D) a.raw_out[r0 + i] = ys[i];
      if (r == 0 && threadIdx.x == 0) {
        VecState* st = &a.ctl->v[0];
        st->iters = 1;
        st->done = 1;
        if (*(volatile const int*)&a.sync->err) st->status = MAPI_ETIMEOUT;
        a.ctl->all_done = 1;
      }
      break;
    }
    // 3. deflation: group g = warps 4g .. 4g + 3 takes component r + CS g
    //    (and every 2 CS-th after it); warp wq of the group scans sorted
    //    positions [256 wq, 256 wq + 256), eight per lane.  Every sum is
    //    compensated (TwoSum: hi + lo); each prefix A_p = sum_{q <= p} c_q z_q
    //    and suffix S_p = sum_{q > p} z_q is rounded once, when stored.
    if (nprev > 0) {
      const int g = warp >> 2, wq = warp & 3, tg = threadIdx.x & 127;
      float* cb = cbuf + g * D_pad;
      float* sA = arrays(g);
      float* sS = sA + kDeflPadded;
      float* sA2 = sS + kDeflPadded;
      float* sS2 = sA2 + kDeflPadded;
      const float* wm_s = sS2 + kDeflPadded;
      const float* cs_s = wm_s + kDeflPadded;
      const int* perm_s = reinterpret_cast<const int*>(cs_s + kDeflPadded);
      const int* ub_s = perm_s + kDeflPadded;
      for (int m = r + CS * g; m < nprev; m += 2 * CS) {
        if (m >= 2 * CS || (!resident && t > 0)) {  // reload what a later one replaced
          group_bar(g);
          load_comp(m, g, tg, 128);
        }
        group_bar(g);
        if constexpr (dot) {
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
        // sorted position p contributes c z to A and z to B (z = s y, with c
        // and s the magnitude and sign of the component there) and, for
        // min2, c y and y
        const int p0 = wq * 256 + lane * 8;
        TwoSum la, lb, la2, lb2;  // this lane's totals
        float kc[8], kz[8], ky[8];  // the positions' c, z and y, kept for the second walk
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          const int p = p0 + k;
          const int i = p < D ? perm_s[dpad(p)] : 0;
          ky[k] = p < D ? yfull[i] : 0.f;
          kc[k] = p < D ? cs_s[dpad(p)] : 0.f;
          kz[k] = p < D ? sgnf(wm_s[i]) * ky[k] : 0.f;
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          if (p0 + k < D) {
            la.add_prod(kc[k], kz[k]);
            lb.add(kz[k]);
            if constexpr (two) {
              la2.add_prod(kc[k], ky[k]);
              lb2.add(ky[k]);
            }
          }
        }
        // inclusive scan of the lane totals over the warp
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
          if constexpr (two) {
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
        auto neg = [](const TwoSum& v) {
          TwoSum n;
          n.hi = -v.hi;
          n.lo = -v.lo;
          return n;
        };
        // this lane's offset (everything before its first position) and the
        // group's totals of z (and y)
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
            if constexpr (two) {
              oa2.add(ea2);
              ob2.add(eb2);
            }
          }
          totB.add(eb);
          if constexpr (two) totB2.add(eb2);
        }
        // walk the lane's positions again from its offset: A_p, and the
        // suffix S_p = totB - B_p, each rounded once
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          const int p = p0 + k;
          if (p < D) {
            const float y = ky[k], c = kc[k], z = kz[k];
            oa.add_prod(c, z);
            ob.add(z);
            TwoSum sb = totB;
            sb.add(neg(ob));
            sA[dpad(p)] = oa.value();
            sS[dpad(p)] = sb.value();
            if constexpr (two) {
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
        {
          // outputs i = tg + 128 k (D <= 1024: at most 8 per thread), each
          // stage's loads issued for all k before the next stage uses them
          constexpr int PO = kDeflMaxD / 128;
          float wi[PO];
          int qi[PO];
#pragma unroll
          for (int k = 0; k < PO; ++k) {
            const int i = tg + 128 * k;
            wi[k] = i < D ? wm_s[i] : 0.f;
            qi[k] = i < D ? dpad(ub_s[i]) : 0;
          }
          float va[PO], vs[PO], va2[PO], vs2[PO];
#pragma unroll
          for (int k = 0; k < PO; ++k) {
            va[k] = sA[qi[k]];
            vs[k] = sS[qi[k]];
            if constexpr (two) {
              va2[k] = sA2[qi[k]];
              vs2[k] = sS2[qi[k]];
            }
          }
#pragma unroll
          for (int k = 0; k < PO; ++k) {
            const int i = tg + 128 * k;
            if (i < D) {
              const float ci = fabsf(wi[k]);
              float v = sgnf(wi[k]) * fmaf(ci, vs[k], va[k]);
              if constexpr (two) v = 0.5f * (v + fmaf(ci, vs2[k], va2[k]));
              cb[i] += v;
            }
          }
        }
      }
    }
    // every CTA has read all rows of the accumulator and written its groups'
    // products: clear this CTA's rows for step t + 2, combine its own rows
    cluster.sync();
    for (int i = threadIdx.x; i < RS; i += NT)
#pragma unroll
      for (int c = 0; c < kAccCopies; ++c) accb[(size_t)c * D_pad + r0 + i] = 0ull;
    const int nq = min(CS, nprev);
    const bool second = nprev > CS;  // some CTA's second group holds a sum
    for (int i = threadIdx.x; i < RS; i += NT) {
      const int d = r0 + i;
      float v[2 * CS];
#pragma unroll
      for (int q = 0; q < CS; ++q) {
        const float* cq = cluster.map_shared_rank(cbuf, q);
        v[q] = q < nq ? cq[d] : 0.f;
        v[CS + q] = second ? cq[D_pad + d] : 0.f;
      }
      // u = y - sum_m P_m y, compensated and rounded once
      TwoSum uc;
      uc.add(ys[i]);
#pragma unroll
      for (int q = 0; q < 2 * CS; ++q) uc.add(-v[q]);
      u[i] = d < D ? uc.value() : 0.f;
    }
    __syncthreads();
    if (stamp) t_defl = gtimer_u64();
    // 4. norm over the cluster (and, through the same barrier, whether any
    //    wait ran out anywhere)
    Kahan k;
    for (int i = threadIdx.x; i < RS; i += NT) {
      const float x = u[i];
      k.add(a.norm_l2 ? x * x : fabsf(x));
    }
    const float np = block_sum<NT>(k.value(), red);
    // a CTA pushes its partial only after its combine above has read every
    // peer's cbuf, so once all partials are in, no peer reads this CTA's
    // cbuf any more (it is cleared again at the next step)
    if (threadIdx.x == 0) {
      const float ef = *(volatile const int*)&a.sync->err ? 1.f : 0.f;
      mbar_expect_tx(&nbar, 2 * CS * 4);
      const uint32_t bar = smem_u32(&nbar);
#pragma unroll
      for (int q = 0; q < CS; ++q) {
        st_async_f32(mapa_u32(smem_u32(&nin[0][r]), q), np, mapa_u32(bar, q));
        st_async_f32(mapa_u32(smem_u32(&nin[1][r]), q), ef, mapa_u32(bar, q));
      }
      const bool in = mbar_wait(&nbar, (unsigned)(t & 1), kWaitLimitNs);
      if (!in) atomicExch(&a.sync->err, 1);
      // in rank order, as (r0 + r1) + (r2 + r3)
      part[4] = (nin[0][0] + nin[0][1]) + (nin[0][2] + nin[0][3]);
      part[5] = !in || (nin[1][0] + nin[1][1]) + (nin[1][2] + nin[1][3]) > 0.f ? 1.f : 0.f;
    }
    __syncthreads();
    float L = part[4];
    const bool err = part[5] > 0.f;
    if (a.norm_l2) L = sqrtf(L);
    const bool ok = (L > 0.f) && isfinite(L);
    // 5. normalise own rows (the n divisions of §2.2), the delta when a stop
    //    rule needs it; the iterate stays in shared memory (the streaming
    //    CTAs take it from the publication below) and goes to global memory
    //    only after the last step
    Kahan dk;
    if (ok) {
      for (int i = threadIdx.x; i < RS; i += NT) {
        const int d = r0 + i;
        if (d >= D) continue;
        const float x = u[i] / L;
        if (want_delta) dk.add(fabsf(x - wo[i]));
        wo[i] = x;
      }
    }
    float Dsum = 0.f;
    if (want_delta) {
      const float dp = block_sum<NT>(dk.value(), red);
      if (threadIdx.x == 0) part[2] = dp;
      cluster.sync();
      Dsum = cluster_sum(cluster, &part[2], &part[6]);
    }
    const bool done = !ok || err || (want_delta && Dsum < a.ctl->tol) || t + 1 == a.T;
    if (done) {
      // the final iterate where the finish kernel reads it (by the parity of
      // the steps taken: this step's, or, when the norm failed, the last good
      // iterate under the previous step's parity)
      float* wfin = ok ? ((t & 1) ? a.wb0 : a.wb1) : ((t & 1) ? a.wb1 : a.wb0);
      for (int i = threadIdx.x; i < RS; i += NT)
        if (r0 + i < D) wfin[r0 + i] = wo[i];
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
        if (done) st->done = 1;
      }
      if (err) {
        st->status = MAPI_ETIMEOUT;
        st->done = 1;
      }
      a.ctl->all_done = done ? 1 : 0;
    }
    if (stamp) {
      volatile PairPhases* ph = a.phases;
      const unsigned long long t_pub = gtimer_u64();
      const unsigned long long t0 = ph->start_min;
      const unsigned long long lmin = ph->loop_min, lmax = ph->loop_max;
      if (ph->prev_end && t0 > ph->prev_end) ph->sum[0] += t0 - ph->prev_end;
      ph->sum[1] += lmin - t0;
      ph->sum[2] += lmax - t0;
      ph->sum[3] += t_seen - lmax;
      ph->sum[4] += t_reduce - t_seen;
      ph->sum[5] += t_defl - t_reduce;
      ph->sum[6] += t_pub - t_defl;
      ph->sum[7] += 1;
      ph->prev_end = t_pub;
      ph->start_min = ~0ull;
      ph->loop_min = ~0ull;
      ph->loop_max = 0;
    }
    // 6. publish this CTA's rows (and the stop bit) to the streaming CTAs of
    //    the same rank
    // each thread publishes its rows: value and tag 2 (t + 1) + stop in one
    // 64-bit word, released after this thread's writes of the step (its
    // rows of the iterate and of the cleared accumulator)
    const unsigned long long tag = (unsigned long long)(2u * (unsigned)(t + 1) + (done ? 1u : 0u));
    for (int i = threadIdx.x; i < RS; i += NT)
      st_release_u64(a.wpub + r0 + i, (tag << 32) | __float_as_uint(wo[i]));
    if (done) break;
  }
}

// ----------------------------------------------------------------- kernel
// STAMP: the variant that takes the phase stamps (mapi_pair_phases); the
// others carry no stamping code at all.
template <int OP, int ST, int RW, bool STAMP>
__global__ void __launch_bounds__(kPairThreads, 2)
    k_pair_solve(const __grid_constant__ CUtensorMap xmap, PairSolveArgs a) {
  using PC = PairCols<ST>;
  constexpr int CPL = PC::CPL;
  constexpr int TC = 32 * CPL;  // columns per tile
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
  __shared__ __align__(8) uint64_t tready[4];
  __shared__ __align__(8) uint64_t never;  // nothing ever arrives here
  using PT = OpReg<OP>;
  __shared__ typename PT::S wp[RC];         // the prepared iterate, per row of this CTA
  __shared__ float tbuf[2][kPairWarps][TC];  // per-warp column partials (by tile parity)
  __shared__ float tin[4][kPairCluster][TC];  // column partials pushed by each CTA
  __shared__ int s_err;
  __shared__ int s_stop;
  __shared__ unsigned long long s_t0;  // phase stamps: this step's start

  if (threadIdx.x == 0) {
    s_err = 0;
    s_stop = 0;
    for (int s = 0; s < kPairStages; ++s) mbar_init(&full[s], 1);
    for (int q = 0; q < 4; ++q) mbar_init(&tready[q], 1);
    mbar_init(&never, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  // Fault-detection test (stall_ns > 0, never in a normal solve): thread 0
  // waits on a barrier that nothing arrives at, through the same bounded
  // wait as every tile and exchange.  No copy or peer store is pending on
  // it, so the wait simply runs out; the solve then stops with
  // MAPI_ETIMEOUT after its first step.
  if (a.stall_ns > 0 && threadIdx.x == 0 && !mbar_wait(&never, 0, a.stall_ns))
    atomicExch(&a.sync->err, 1);
  // the solve failed to start (or an earlier component failed): nothing to do
  if (*(volatile const int*)&a.ctl->all_done) return;
  // peers push into tin / tready only after every CTA of the cluster has
  // initialised its barriers
  cluster.sync();
  const bool dot = OP == MAPI_OP_DOT;
  const int s_exp = acc_scale_exp(__uint_as_float(*(volatile const unsigned*)&a.sync->xmax),
                                  a.ncols, a.D_pad, dot);
  if (cid == a.nstream) {
    pair_epilogue<RC, OP, STAMP>(a, cluster, reinterpret_cast<float*>(stage), s_exp);
    cluster.sync();  // peers may still read this CTA's shared memory until here
    return;
  }

  // ---- streaming cluster
  // this cluster's tiles: nround rounds in which every streaming cluster
  // takes one (tile cid + j nstream), then the rest in rounds over the first
  // nfirst clusters only (their CTAs are placed first on their SMs and are
  // issued ahead of the others, so they run faster)
  const int extra = a.ntiles - a.nround * a.nstream;
  const int nmine =
      cid < a.nfirst ? a.nround + extra / a.nfirst + (cid < extra % a.nfirst ? 1 : 0) : a.nround;
  const unsigned total = (unsigned)a.T * (unsigned)nmine;  // tiles over all steps (< 2^31)
  const float scale = ldexpf(1.f, s_exp);
  // every tile is read once per step with the evict-first policy (the walk
  // reversal still finds the last tiles of a step in L2 at the start of the
  // next); marking a share of them evict-last measured slower
  const uint64_t pol_first = createpolicy_evict_first();
  unsigned issued = 0;  // thread 0: tiles issued (global order over the steps)
  auto issue_next = [&]() {
    const unsigned g = issued++;
    const int s = (int)(g % kPairStages);
    const int t = (int)(g / nmine), j = (int)(g % nmine);
    const int jj = ((a.dir0 + t) & 1) ? nmine - 1 - j : j;
    const int tile = jj < a.nround ? cid + jj * a.nstream
                                   : a.nround * a.nstream + (jj - a.nround) * a.nfirst + cid;
    mbar_expect_tx(&full[s], kStageBytes);
    tma_load_2d_hint(stage + (size_t)s * RC * 32, &xmap, tile * TC, (int)crank * RC, &full[s],
                     pol_first);
  };
  if (threadIdx.x == 0)
    while (issued < total && issued < kPairStages) issue_next();

  float acc[RW];
  // Phase A of tile g (global index over all steps): read this warp's rows of
  // the stage, column partials -> tbuf[g & 1] -> (after the CTA barrier) warp
  // 0 pushes the CTA's partials to every CTA of the cluster.  The stage is
  // refilled, with the next tile of this or a later step, as soon as every
  // warp has read it.
  auto phase_a = [&](unsigned g, uint32_t (&raw)[RW]) {
    const int s = (int)(g % kPairStages);
    const int par = (int)(g & 1);
    const int slot = (int)(g & 3);
    // after a wait has run out the others get 1 ms, so a failed solve ends soon
    if (!mbar_wait(&full[s], (unsigned)((g / kPairStages) & 1), s_err ? 1000000LL : kWaitLimitNs))
      s_err = 1;
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
      const typename PT::P p = PT::load(wp[warp * RW + jj]);
#pragma unroll
      for (int c = 0; c < CPL; ++c) tp[c] = PT::term(x[c], p, tp[c]);
    }
#pragma unroll
    for (int c = 0; c < CPL; ++c) tbuf[par][warp][lane * CPL + c] = tp[c];
    __syncthreads();
    if (threadIdx.x == 0 && issued < total && !s_err) issue_next();
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
  // Phase B of tile g: wait for the cluster's partials of its columns (they
  // were pushed while phase A of the next tile ran), then the row sums.
  auto phase_b = [&](unsigned g, const uint32_t (&raw)[RW]) {
    const int slot = (int)(g & 3);
    if (!mbar_wait(&tready[slot], (unsigned)((g >> 2) & 1), s_err ? 1000000LL : kWaitLimitNs))
      s_err = 1;
    typename PT::P tpar[CPL];
#pragma unroll
    for (int c = 0; c < CPL; ++c) {
      float tt = 0.f;
#pragma unroll
      for (int q = 0; q < kPairCluster; ++q) tt += tin[slot][q][lane * CPL + c];
      tpar[c] = PT::prep(tt);
    }
#pragma unroll
    for (int jj = 0; jj < RW; ++jj) {
      float x[CPL];
      PC::get_b(raw[jj], x);
#pragma unroll
      for (int c = 0; c < CPL; ++c) acc[jj] = PT::term(x[c], tpar[c], acc[jj]);
    }
  };

  unsigned gbase = 0;  // global index of this step's first tile
  for (int t = 0; t < a.T; ++t) {
    if (t > 0) {
      // the epilogue's rows of w_t for this rank, each in a tagged word
      // (and whether to stop, the tag's low bit): thread 0 waits for the
      // first row, then every thread takes its own (already there, or soon)
      if (threadIdx.x == 0 && wait_tag(a.wpub + (int)crank * RC, 2u * (unsigned)t) == 0ull) {
        s_err = 1;
        atomicExch(&a.sync->err, 1);
        s_stop = 1;
      }
      __syncthreads();
      for (int r = threadIdx.x; r < RC && !s_stop; r += blockDim.x) {
        const unsigned long long v = wait_tag(a.wpub + (int)crank * RC + r, 2u * (unsigned)t);
        if (v == 0ull) {
          s_err = 1;
          atomicExch(&a.sync->err, 1);
          s_stop = 1;
        } else {
          if ((v >> 32) & 1ull) s_stop = 1;
          wp[r] = PT::store(__uint_as_float((unsigned)v));
        }
      }
      __syncthreads();
      if (s_stop) break;
    } else {
      // w_0 from the start kernel
      for (int r = threadIdx.x; r < RC; r += blockDim.x) {
        const int d = (int)crank * RC + r;
        const float wv = d < a.D ? __ldcg(a.wb0 + d) : 0.f;
        wp[r] = PT::store(wv);
      }
      __syncthreads();
    }
    if (STAMP && a.phases && threadIdx.x == 0) {
      s_t0 = gtimer_u64();
      atomicMin(&a.phases->start_min, s_t0);
    }
#pragma unroll
    for (int j = 0; j < RW; ++j) acc[j] = 0.f;
    // two tiles in flight: A(j) overlaps the cluster exchange of tile j - 1
    uint32_t rawA[RW], rawB[RW];
    int j = 0;
#pragma unroll 1
    for (; j + 1 < nmine; j += 2) {
      phase_a(gbase + j, rawA);
      if (j > 0) phase_b(gbase + j - 1, rawB);
      phase_a(gbase + j + 1, rawB);
      phase_b(gbase + j, rawA);
    }
    if (j < nmine) {
      phase_a(gbase + j, rawA);
      if (j > 0) phase_b(gbase + j - 1, rawB);
      phase_b(gbase + j, rawA);
    } else if (nmine > 0) {
      phase_b(gbase + nmine - 1, rawB);
    }
    gbase += nmine;
    // row sums across the 32 lanes: a transposing butterfly halves the rows
    // each lane holds at every level (31 shuffles for 32 rows), so lane l
    // ends with row l / (32 / RW); the row sum goes into the fixed-point
    // accumulator (64-bit integer addition: exact and order-independent)
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
      if ((lane & (grp - 1)) == 0 && nmine > 0) {
        const long long v = __float2ll_rn(acc[0] * scale);
        atomicAdd(a.acc + ((size_t)(t & 1) * kAccCopies + (cid & (kAccCopies - 1))) * a.D_pad +
                      rbase + lane / grp,
                  (unsigned long long)v);
      }
    }
    if (threadIdx.x == 0) {
      if (s_err) atomicExch(&a.sync->err, 1);
      if (STAMP && a.phases) {
        const unsigned long long tn = gtimer_u64();
        atomicMin(&a.phases->loop_min, tn);
        atomicMax(&a.phases->loop_max, tn);
        if (cid < kPairPhaseClusters) atomicAdd(&a.phases->cl_ns[cid], tn - s_t0);
      }
    }
    // arrival: this CTA's row sums are in (the release, cumulative over what
    // thread 0 has seen through the block barrier, orders every thread's
    // additions before the count)
    __syncthreads();
    if (threadIdx.x == 0) red_release_add_u32(&a.sync->arrivals, 1u);
  }
  // tiles issued ahead for steps that did not run: let them land
  if (threadIdx.x == 0)
    for (unsigned g = gbase; g < issued; ++g)
      mbar_wait(&full[g % kPairStages], (unsigned)((g / kPairStages) & 1),
                s_err ? 1000000LL : kWaitLimitNs);
  __syncthreads();
  cluster.sync();  // peers may still push into this CTA's slots until here
}

// max |X| over the packed matrix, as FP32 bits (non-negative floats order
// like their bit patterns); BF16 values are exact in FP32.
template <int ST>
__global__ void k_pair_xmax(const void* __restrict__ X, int64_t elems, unsigned* out) {
  float m = 0.f;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  if (ST == kF32) {
    const float4* p = reinterpret_cast<const float4*>(X);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < elems / 4; i += stride) {
      const float4 v = __ldcs(p + i);
      m = fmaxf(m, fmaxf(fmaxf(fabsf(v.x), fabsf(v.y)), fmaxf(fabsf(v.z), fabsf(v.w))));
    }
  } else {
    const uint4* p = reinterpret_cast<const uint4*>(X);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < elems / 8; i += stride) {
      const uint4 v = __ldcs(p + i);
      const uint32_t wd[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        m = fmaxf(m, fabsf(__uint_as_float(wd[k] << 16)));
        m = fmaxf(m, fabsf(__uint_as_float(wd[k] & 0xFFFF0000u)));
      }
    }
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, __float_as_uint(m));
}

__global__ void k_coop_probe() {}

template <int OP, int ST, bool STAMP = false>
const void* solve_fn(int rw) {
  switch (rw) {
    case 8: return (const void*)k_pair_solve<OP, ST, 8, STAMP>;
    case 16: return (const void*)k_pair_solve<OP, ST, 16, STAMP>;
    case 32: return (const void*)k_pair_solve<OP, ST, 32, STAMP>;
  }
  return nullptr;
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
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

// Whether this device takes a cooperative launch of 4-CTA clusters (asked
// once per context with an empty kernel of the same grid).
bool coop_cluster_ok(mapi_ctx* ctx, int nclusters) {
  if (ctx->pair_coop >= 0) return ctx->pair_coop == 1;
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = kPairCluster;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  attr[1].id = cudaLaunchAttributeCooperative;
  attr[1].val.cooperative = 1;
  cfg.gridDim = dim3(kPairCluster * nclusters, 1, 1);
  cfg.blockDim = dim3(32, 1, 1);
  cfg.stream = ctx->stream;
  cfg.attrs = attr;
  cfg.numAttrs = 2;
  const cudaError_t e = cudaLaunchKernelEx(&cfg, k_coop_probe);
  if (e != cudaSuccess) cudaGetLastError();
  ctx->pair_coop = (e == cudaSuccess) ? 1 : 0;
  return ctx->pair_coop == 1;
}

}  // namespace

mapi_status plan_pair(mapi_ctx* ctx, const mapi_mat* X, mapi_op op, PairPlan* pl) {
  const int D = X->rows;
  int rw = 8;
  while (kPairCluster * kPairWarps * rw < D && rw < 32) rw *= 2;
  if (kPairCluster * kPairWarps * rw < D)
    return fail(ctx, MAPI_EINVAL, "pair mode supports D <= 1024");
  const void* fn = nullptr;
  CUtensorMapDataType dt;
  int tc;
  // the stamping variant exists for MIN1 (the benchmark's operator) only
  pl->fn_stamp = nullptr;
  if (X->storage == MAPI_ST_F32) {
    if (op == MAPI_OP_MIN1) pl->fn_stamp = solve_fn<MAPI_OP_MIN1, kF32, true>(rw);
    fn = op == MAPI_OP_MIN1 ? solve_fn<MAPI_OP_MIN1, kF32>(rw)
         : op == MAPI_OP_MIN2 ? solve_fn<MAPI_OP_MIN2, kF32>(rw)
                              : solve_fn<MAPI_OP_DOT, kF32>(rw);
    dt = CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    tc = 32;
  } else if (X->storage == MAPI_ST_BF16) {
    if (op == MAPI_OP_MIN1) pl->fn_stamp = solve_fn<MAPI_OP_MIN1, kBF16, true>(rw);
    fn = op == MAPI_OP_MIN1 ? solve_fn<MAPI_OP_MIN1, kBF16>(rw)
         : op == MAPI_OP_MIN2 ? solve_fn<MAPI_OP_MIN2, kBF16>(rw)
                              : solve_fn<MAPI_OP_DOT, kBF16>(rw);
    dt = CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    tc = 64;
  } else {
    return fail(ctx, MAPI_EINVAL, "pair mode supports F32 and BF16 storage");
  }
  const int rc = kPairWarps * rw;
  const int d_pad = kPairCluster * rc;
  // the stage ring of a streaming CTA, or the epilogue's arrays
  pl->smem = std::max((size_t)kPairStages * rc * 128,
                      (size_t)pair_epi_floats(rc, d_pad) * sizeof(float));
  MAPI_CUDA_TRY(ctx, cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)pl->smem));
  if (pl->fn_stamp)
    MAPI_CUDA_TRY(ctx, cudaFuncSetAttribute(pl->fn_stamp,
                                            cudaFuncAttributeMaxDynamicSharedMemorySize,
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
  cfg.blockDim = dim3(kPairThreads, 1, 1);
  cfg.dynamicSmemBytes = pl->smem;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int nclusters = 0;
  MAPI_CUDA_TRY(ctx, cudaOccupancyMaxActiveClusters(&nclusters, fn, &cfg));
  if (nclusters < 2) return fail(ctx, MAPI_ECUDA, "pair kernel: fewer than two clusters fit");
  pl->fn = fn;
  pl->rw = rw;
  pl->clusters = std::min(nclusters, kPairMaxStream + 1);
  pl->D_pad = d_pad;
  pl->coop = coop_cluster_ok(ctx, pl->clusters);
  return MAPI_OK;
}

// Scratch: accumulators [2][kAccCopies][D_pad], the published iterate
// [D_pad] (both 64-bit words), then PairSync.
size_t pair_scratch_bytes(const PairPlan& pl) {
  return sizeof(unsigned long long) * (2 * kAccCopies + 1) * (size_t)pl.D_pad + 256;
}

mapi_status launch_pair_prepare(mapi_ctx* ctx, cudaStream_t s, const PairPlan& pl,
                                const mapi_mat* X, void* scratch) {
  // the scale of the fixed-point sums comes from max |X|: zero the
  // accumulators and the shared state, then find max |X| (once per solve)
  MAPI_CUDA_TRY(ctx, cudaMemsetAsync(scratch, 0, pair_scratch_bytes(pl), s));
  PairSync* sync = reinterpret_cast<PairSync*>(
      (char*)scratch + sizeof(unsigned long long) * (2 * kAccCopies + 1) * (size_t)pl.D_pad);
  const int64_t elems = (int64_t)X->rows_pad * X->ld;
  const int blocks = 4 * ctx->sm_count;
  if (X->storage == MAPI_ST_F32)
    k_pair_xmax<kF32><<<blocks, 256, 0, s>>>(X->data, elems, &sync->xmax);
  else
    k_pair_xmax<kBF16><<<blocks, 256, 0, s>>>(X->data, elems, &sync->xmax);
  MAPI_CUDA_TRY(ctx, cudaGetLastError());
  count_launch(ctx);
  return MAPI_OK;
}

mapi_status launch_pair_solve(mapi_ctx* ctx, cudaStream_t s, const PairPlan& pl,
                              const mapi_mat* X, void* scratch, float* wb0, float* wb1,
                              const DeflArgs& defl, IterCtl* ctl, int T, int norm_l2,
                              float denom, int dir0, float* raw_out) {
  if (T <= 0) return MAPI_OK;
  const int TCc = (X->storage == MAPI_ST_F32) ? 32 : 64;
  const int64_t ntiles = (X->ld + TCc - 1) / TCc;
  // the tile split: a share of the tiles goes to the first half of the
  // streaming clusters only
  const int nstream = pl.clusters - 1;
  const int nfirst = std::max(1, nstream / 2);
  // (measured on GB300: the best share for FP32 X, whose loop is bound by
  // HBM, is 3 % of the tiles; for BF16, bound by issue, 26 %)
  const double skew = X->storage == MAPI_ST_BF16 ? 0.26 : 0.03;
  const int64_t nround = (int64_t)((double)ntiles * (1.0 - skew)) / nstream;
  const int64_t rest = ntiles - nround * nstream;
  const int64_t nmine_max = nround + (rest + nfirst - 1) / nfirst;
  if ((int64_t)T * nmine_max >= (1ll << 31))
    return fail(ctx, MAPI_EINVAL, "pair mode: max_iters x column tiles per cluster >= 2^31");
  const size_t acc_bytes = sizeof(unsigned long long) * (2 * kAccCopies + 1) * (size_t)pl.D_pad;
  PairSync* sync = reinterpret_cast<PairSync*>((char*)scratch + acc_bytes);
  // the accumulators and the shared state of the launch start at zero (max
  // |X| is kept)
  MAPI_CUDA_TRY(ctx, cudaMemsetAsync(scratch, 0, acc_bytes + offsetof(PairSync, xmax), s));
  PairSolveArgs a;
  a.D = X->rows;
  a.D_pad = pl.D_pad;
  a.ncols = X->cols;
  const int TC = (X->storage == MAPI_ST_F32) ? 32 : 64;
  a.ntiles = (int)((X->ld + TC - 1) / TC);
  a.nstream = pl.clusters - 1;
  a.T = T;
  a.dir0 = dir0 & 1;
  a.nround = (int)nround;
  a.nfirst = nfirst;
  a.norm_l2 = norm_l2;
  a.denom = denom;
  a.wb0 = wb0;
  a.wb1 = wb1;
  a.acc = reinterpret_cast<unsigned long long*>(scratch);
  a.sync = sync;
  a.ctl = ctl;
  a.defl = defl;
  a.stall_ns = ctx->stall_ns;
  const bool stamped = ctx->phases_on && ctx->pair_phases.p && pl.fn_stamp;
  a.phases = stamped ? (PairPhases*)ctx->pair_phases.p : nullptr;
  ctx->pair_nstream = a.nstream;
  a.raw_out = raw_out;
  a.wpub = reinterpret_cast<unsigned long long*>(scratch) + 2 * kAccCopies * (size_t)pl.D_pad;
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = kPairCluster;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  attr[1].id = cudaLaunchAttributeCooperative;
  attr[1].val.cooperative = 1;
  cfg.gridDim = dim3(kPairCluster * pl.clusters, 1, 1);
  cfg.blockDim = dim3(kPairThreads, 1, 1);
  cfg.dynamicSmemBytes = pl.smem;
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = pl.coop ? 2 : 1;
  void* args[] = {(void*)&pl.map, &a};
  cudaEvent_t ev = prof_begin(ctx, s);
  MAPI_CUDA_TRY(ctx, cudaLaunchKernelExC(&cfg, stamped ? pl.fn_stamp : pl.fn, args));
  prof_end(ctx, s, ev, MAPI_KC_PAIR, (double)T * X->rows * X->cols * elem_bytes(X->storage),
           2.0 * T * X->rows * X->cols, T);
  count_launch(ctx);
  return MAPI_OK;
}

}  // namespace mapi
