// Device-side helpers shared by the MAPI kernels: MAVP term functors,
// storage decoders, streaming loads and deterministic block reductions.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "mapi_internal.cuh"

namespace mapi {

// ------------------------------------------------------------- MAVP terms
//
// Every float term is evaluated as  s * clamp(a, lo, hi)  accumulated with one
// fused multiply-add, where (lo, hi, s) depend only on the vector entry w and
// are prepared once per w and shared by every row of A that meets it:
//
//   min1, Eq. (3): sign(a w) min(|a|, |w|) = sign(w) clamp(a, -|w|, |w|)
//                  -> lo = -|w|, hi = |w|, s = sign(w) (+1 for w = 0)
//   min2, Eq. (4): 1(sign a = sign w) min(|a|, |w|)
//                  = sign(w) clamp(a, min(w, 0), max(w, 0))
//
// The clamp returns min(|a|, |w|) with a's sign (or 0), the product by
// s = +-1 is exact and the sum is rounded once, so each term equals the
// definition exactly; only the order of the FP32 summation differs from a
// sequential sum.  Diamond (Eq. (7)) and dot (Eq. (1)) are plain arithmetic.

template <int OP>
struct Op;

template <>
struct Op<MAPI_OP_MIN1> {
  struct P {
    float lo, hi, s;
  };
  static __device__ __forceinline__ P prep(float w) {
    const float c = fabsf(w);
    return {-c, c, copysignf(1.f, w)};
  }
  static __device__ __forceinline__ float term(float a, const P& p, float acc) {
    return fmaf(fminf(fmaxf(a, p.lo), p.hi), p.s, acc);
  }
};

template <>
struct Op<MAPI_OP_MIN2> {
  struct P {
    float lo, hi, s;
  };
  static __device__ __forceinline__ P prep(float w) {
    return {fminf(w, 0.f), fmaxf(w, 0.f), w < 0.f ? -1.f : 1.f};
  }
  static __device__ __forceinline__ float term(float a, const P& p, float acc) {
    return fmaf(fminf(fmaxf(a, p.lo), p.hi), p.s, acc);
  }
};

__device__ __forceinline__ float sgnf(float x) {
  return (float)((x > 0.f) - (x < 0.f));
}

template <>
struct Op<MAPI_OP_DIAMOND> {
  struct P {
    float w, sw;
  };
  static __device__ __forceinline__ P prep(float w) { return {w, sgnf(w)}; }
  static __device__ __forceinline__ float term(float a, const P& p, float acc) {
    // sign(a) w + a sign(w)
    return fmaf(a, p.sw, fmaf(sgnf(a), p.w, acc));
  }
};

template <>
struct Op<MAPI_OP_DOT> {
  struct P {
    float w;
  };
  static __device__ __forceinline__ P prep(float w) { return {w}; }
  static __device__ __forceinline__ float term(float a, const P& p, float acc) {
    return fmaf(a, p.w, acc);
  }
};

// A vector entry's prepared form for loops that keep many of them in
// registers: Op's (lo, hi, s) by default; for MIN1 only (w, s), the bounds
// -|w| and |w| taken at each use (the same values as Op's lo and hi, so the
// terms are identical), one register per entry fewer.  S is the form kept
// in shared memory.
template <int OP>
struct OpReg {
  using P = typename Op<OP>::P;
  using S = float4;  // shared-memory form
  static __device__ __forceinline__ S store(float w) {
    const P p = Op<OP>::prep(w);
    return make_float4(p.lo, p.hi, p.s, 0.f);
  }
  static __device__ __forceinline__ P load(const S& q) { return {q.x, q.y, q.z}; }
  static __device__ __forceinline__ P prep(float w) { return Op<OP>::prep(w); }
  static __device__ __forceinline__ float term(float a, const P& p, float acc) {
    return Op<OP>::term(a, p, acc);
  }
};
template <>
struct OpReg<MAPI_OP_MIN1> {
  struct P {
    float w, s;
  };
  using S = float2;
  static __device__ __forceinline__ S store(float w) {
    return make_float2(w, copysignf(1.f, w));
  }
  static __device__ __forceinline__ P load(const S& q) { return {q.x, q.y}; }
  static __device__ __forceinline__ P prep(float w) { return {w, copysignf(1.f, w)}; }
  static __device__ __forceinline__ float term(float a, const P& p, float acc) {
    return fmaf(fminf(fmaxf(a, -fabsf(p.w)), fabsf(p.w)), p.s, acc);
  }
};
template <>
struct OpReg<MAPI_OP_DOT> {
  using P = Op<MAPI_OP_DOT>::P;
  using S = float;
  static __device__ __forceinline__ S store(float w) { return w; }
  static __device__ __forceinline__ P load(const S& q) { return {q}; }
  static __device__ __forceinline__ P prep(float w) { return {w}; }
  static __device__ __forceinline__ float term(float a, const P& p, float acc) {
    return fmaf(a, p.w, acc);
  }
};

// Integer terms (exact): the same clamp identity on INT32.
template <int OP>
struct IOp;

template <>
struct IOp<MAPI_OP_MIN1> {
  struct P {
    int lo, hi, s;
  };
  static __device__ __forceinline__ P prep(int w) {
    const int c = abs(w);
    return {-c, c, w < 0 ? -1 : 1};
  }
  static __device__ __forceinline__ int term(int a, const P& p, int acc) {
    return acc + p.s * min(max(a, p.lo), p.hi);
  }
};

template <>
struct IOp<MAPI_OP_MIN2> {
  struct P {
    int lo, hi, s;
  };
  static __device__ __forceinline__ P prep(int w) {
    return {min(w, 0), max(w, 0), w < 0 ? -1 : 1};
  }
  static __device__ __forceinline__ int term(int a, const P& p, int acc) {
    return acc + p.s * min(max(a, p.lo), p.hi);
  }
};

// --------------------------------------------------------- storage chunks
// A packed row is read in 16-byte chunks; Chunk<ST>::E elements per chunk.
template <int ST>
struct Chunk;

template <>
struct Chunk<kF32> {
  static constexpr int E = 4;
  uint4 raw;
  __device__ __forceinline__ float get(int e) const {
    return __uint_as_float((&raw.x)[e]);
  }
};

template <>
struct Chunk<kBF16> {
  static constexpr int E = 8;
  uint4 raw;
  __device__ __forceinline__ float get(int e) const {
    const uint32_t wd = (&raw.x)[e >> 1];
    return __uint_as_float((e & 1) ? (wd & 0xFFFF0000u) : (wd << 16));
  }
};

// E4M3 byte -> float without rounding: the 7 magnitude bits placed at the
// top of an FP32 exponent/mantissa field give 2^(e-127) (1.m) for normals and
// 2^-126 (0.m) for subnormals; a factor 2^120 then maps both onto the E4M3
// values 2^(e-7) (1.m) and 2^-6 (0.m).  The row scale 2^k is folded into the
// same (exact) power-of-two factor by the caller.
__device__ __forceinline__ float e4m3_bits_unscaled(uint32_t b) {
  return __uint_as_float(((b & 0x7Fu) << 20) | ((b & 0x80u) << 24));
}

// The four E4M3 bytes of a word (byte 0 first) as their exact values, by the
// hardware conversion of byte pairs to f16 pairs (every E4M3 value is an f16
// value) and of each half to f32.
__device__ __forceinline__ void e4m3x4_values(uint32_t wd, float& f0, float& f1, float& f2,
                                              float& f3) {
  uint32_t lo, hi;
  asm("{\n\t.reg .b16 l, h;\n\tmov.b32 {l, h}, %2;\n\t"
      "cvt.rn.f16x2.e4m3x2 %0, l;\n\tcvt.rn.f16x2.e4m3x2 %1, h;\n\t}"
      : "=r"(lo), "=r"(hi)
      : "r"(wd));
  f0 = __half2float(__ushort_as_half((unsigned short)(lo & 0xFFFFu)));
  f1 = __half2float(__ushort_as_half((unsigned short)(lo >> 16)));
  f2 = __half2float(__ushort_as_half((unsigned short)(hi & 0xFFFFu)));
  f3 = __half2float(__ushort_as_half((unsigned short)(hi >> 16)));
}

template <>
struct Chunk<kFP8> {
  static constexpr int E = 16;
  uint4 raw;
  __device__ __forceinline__ float get(int e) const {
    const uint32_t wd = (&raw.x)[e >> 2];
    return e4m3_bits_unscaled((wd >> ((e & 3) * 8)) & 0xFFu);
  }
};

template <>
struct Chunk<kI16> {
  static constexpr int E = 8;
  uint4 raw;
  __device__ __forceinline__ int get(int e) const {
    const uint32_t wd = (&raw.x)[e >> 1];
    return (e & 1) ? ((int)wd >> 16) : ((int)(wd << 16) >> 16);
  }
  // word k: elements 2k (low half) and 2k + 1 (high half)
  __device__ __forceinline__ uint32_t raw_word(int k) const { return (&raw.x)[k]; }
};

// acc + s0 clamp(a0, lo0, hi0) + s1 clamp(a1, lo1, hi1) for two int16
// columns packed in a word (element 0 in the low half): packed signed 16-bit
// max and min, then a two-way dot product of the clamped pair with the
// signs s0, s1 (+-1, the low two bytes of sg), accumulated in INT32.  Every
// operation is exact.
__device__ __forceinline__ int i16x2_clamp_dot(uint32_t a2, uint32_t lo2, uint32_t hi2,
                                               uint32_t sg, int acc) {
  uint32_t c;
  asm("max.s16x2 %0, %1, %2;" : "=r"(c) : "r"(a2), "r"(lo2));
  asm("min.s16x2 %0, %0, %1;" : "+r"(c) : "r"(hi2));
  int d;
  asm("dp2a.lo.s32.s32 %0, %1, %2, %3;" : "=r"(d) : "r"(c), "r"(sg), "r"(acc));
  return d;
}

template <>
struct Chunk<kI8> {
  static constexpr int E = 16;
  uint4 raw;
  __device__ __forceinline__ int get(int e) const {
    const uint32_t wd = (&raw.x)[e >> 2];
    return (int)(wd << (24 - (e & 3) * 8)) >> 24;
  }
};

// Streaming 16-byte load: read once per step, so it bypasses L1 and asks L2
// to fetch whole 256-byte sectors ahead.
__device__ __forceinline__ uint4 ld_stream(const void* p) {
  uint4 r;
  asm("ld.global.nc.L1::no_allocate.L2::256B.v4.u32 {%0,%1,%2,%3}, [%4];"
      : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
      : "l"(p));
  return r;
}

// ------------------------------------------------ async copies, mbarriers
constexpr long long kWaitLimitNs = 2000000000LL;  // bounded waits: 2 s

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
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity,
                                          long long limit_ns = kWaitLimitNs) {
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
    else if (globaltimer_ns() - t0 > limit_ns) return false;
  }
}
__device__ __forceinline__ uint32_t mapa_u32(uint32_t local, unsigned rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(local), "r"(rank));
  return r;
}
// 4-byte store into a peer CTA's shared memory that completes 4 bytes of the
// transaction count of the peer's mbarrier.
__device__ __forceinline__ void st_async_f32(uint32_t remote_addr, float v, uint32_t remote_bar) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.b32 [%0], %1, [%2];" ::"r"(
                   remote_addr),
               "r"(__float_as_uint(v)), "r"(remote_bar)
               : "memory");
}
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes "
      "[%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst)),
      "l"(map), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

// The same load with an L2 eviction-priority policy (createpolicy_*).
__device__ __forceinline__ void tma_load_2d_hint(void* dst, const CUtensorMap* map, int x, int y,
                                                 uint64_t* bar, uint64_t policy) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint "
      "[%0], [%1, {%2, %3}], [%4], %5;" ::"r"(smem_u32(dst)),
      "l"(map), "r"(x), "r"(y), "r"(smem_u32(bar)), "l"(policy)
      : "memory");
}
// L2 policy: lines that should leave first.
__device__ __forceinline__ uint64_t createpolicy_evict_first() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}

// 1-D bulk copy global -> shared (16-byte aligned, size a multiple of 16),
// completing `bytes` of the mbarrier's transaction count.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes,
                                         uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// Stream a block of RB consecutive rows of a row-major matrix, 16-byte
// chunks [c_beg, c_end), through an S-stage shared-memory ring of tiles of
// RB x kRingTileBytes.  One thread issues the bulk copies; every thread calls
// consume(tile, nchunks, first_chunk) for each tile in order, and the stage is
// refilled once all threads have returned from it.  `full` holds S mbarriers
// (initialised here); on a wait that times out `err` is set.
constexpr int kRingTileBytes = 2048;
constexpr int kRingTileChunks = kRingTileBytes / 16;

template <int RB, int S, class F>
__device__ __forceinline__ void stream_row_tiles(const uint8_t* A, int64_t row_bytes, int row0,
                                                 int c_beg, int c_end, uint8_t* stage,
                                                 uint64_t* full, int* err, F&& consume) {
  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) mbar_init(&full[s], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  const int ntiles = c_end > c_beg ? (c_end - c_beg + kRingTileChunks - 1) / kRingTileChunks : 0;
  auto issue = [&](int t) {
    const int s = t % S;
    const int cb = c_beg + t * kRingTileChunks;
    const int nch = min(kRingTileChunks, c_end - cb);
    const uint32_t bytes = (uint32_t)nch * 16;
    mbar_expect_tx(&full[s], RB * bytes);
    uint8_t* dst = stage + (size_t)s * RB * kRingTileBytes;
    const uint8_t* src = A + (int64_t)row0 * row_bytes + (int64_t)cb * 16;
    for (int r = 0; r < RB; ++r)
      bulk_g2s(dst + r * kRingTileBytes, src + (int64_t)r * row_bytes, bytes, &full[s]);
  };
  if (threadIdx.x == 0)
    for (int t = 0; t < ntiles && t < S; ++t) issue(t);
  for (int t = 0; t < ntiles; ++t) {
    const int s = t % S;
    if (!mbar_wait(&full[s], (unsigned)((t / S) & 1))) *err = 1;
    const int cb = c_beg + t * kRingTileChunks;
    consume(stage + (size_t)s * RB * kRingTileBytes, min(kRingTileChunks, c_end - cb), cb);
    __syncthreads();
    if (threadIdx.x == 0 && t + S < ntiles && !*err) issue(t + S);
  }
}

// ------------------------------------------------------ compensated sums
struct Kahan {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float x) {
    const float y = x - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
  }
  __device__ __forceinline__ float value() const { return s - c; }
};

// Compensated sum as an unevaluated pair hi + lo: every addition is made
// exact by Knuth's two-sum (the rounding error of hi + x is recovered and
// added into lo), and a product enters with its own rounding error
// recovered by a fused multiply-add.  The operations are written with the
// explicitly rounded intrinsics so that the compiler cannot fuse or reorder
// them.
struct TwoSum {
  float hi = 0.f, lo = 0.f;
  __device__ __forceinline__ void add(float x) {
    const float s = __fadd_rn(hi, x);
    const float bp = __fsub_rn(s, hi);
    const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bp)), __fsub_rn(x, bp));
    hi = s;
    lo = __fadd_rn(lo, e);
  }
  // hi + lo += a * b
  __device__ __forceinline__ void add_prod(float a, float b) {
    const float p = __fmul_rn(a, b);
    const float pe = fmaf(a, b, -p);
    add(p);
    lo = __fadd_rn(lo, pe);
  }
  __device__ __forceinline__ void add(const TwoSum& o) {
    add(o.hi);
    lo = __fadd_rn(lo, o.lo);
  }
  __device__ __forceinline__ float value() const { return __fadd_rn(hi, lo); }
};

// Deterministic block sum (fixed butterfly order); every thread gets the
// result.  `sh` needs 33 floats.  All threads of the block must call it.
template <int NT>
__device__ __forceinline__ float block_sum(float v, float* sh) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  if (warp == 0) {
    v = lane < NT / 32 ? sh[lane] : 0.f;
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) sh[32] = v;
  }
  __syncthreads();
  const float r = sh[32];
  __syncthreads();
  return r;
}

template <int NT>
__device__ __forceinline__ long long block_sum_i64(long long v, long long* sh) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  if (warp == 0) {
    v = lane < NT / 32 ? sh[lane] : 0;
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) sh[32] = v;
  }
  __syncthreads();
  const long long r = sh[32];
  __syncthreads();
  return r;
}

// Last-CTA election: every CTA calls this once after writing its outputs;
// exactly one CTA (the last to arrive) gets true, after a fence that makes
// every other CTA's writes visible to it.  No CTA waits for another.
__device__ __forceinline__ bool elect_last_cta(unsigned* counter, unsigned total) {
  __shared__ unsigned s_last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned t = atomicAdd(counter, 1u);
    s_last = (t == total - 1) ? 1u : 0u;
  }
  __syncthreads();
  const bool last = s_last != 0;
  if (last) __threadfence();
  return last;
}

}  // namespace mapi
