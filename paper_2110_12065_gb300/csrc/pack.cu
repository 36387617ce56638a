// Storage packing (once per matrix), read-back, and the Google matrix build.
#include "device_common.cuh"

namespace mapi {

__global__ void k_check_finite(const float* __restrict__ src, int rows, int cols,
                               int64_t ld, int* flag) {
  const int64_t total = (int64_t)rows * cols;
  int bad = 0;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t / cols, j = t % cols;
    bad |= !isfinite(src[i * ld + j]);
  }
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(flag, 1);
}

// max |a| as FP32 bits (non-negative floats order like their bit patterns).
__global__ void k_absmax(const float* __restrict__ src, int rows, int cols,
                         int64_t ld, unsigned* out) {
  const int64_t total = (int64_t)rows * cols;
  float m = 0.f;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t / cols, j = t % cols;
    m = fmaxf(m, fabsf(src[i * ld + j]));
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, __float_as_uint(m));
}

// Element-wise pack into the padded layout (rows_pad x ld, zeros outside).
template <int ST>
__global__ void k_pack(const float* __restrict__ src, int64_t ld_src, int rows,
                       int cols, int rows_pad, int64_t ld, void* dst, int q,
                       const int* __restrict__ row_exp) {
  const int64_t total = (int64_t)rows_pad * ld;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t / ld, j = t % ld;
    const float a = (i < rows && j < cols) ? src[i * ld_src + j] : 0.f;
    if (ST == kF32) {
      ((float*)dst)[t] = a;
    } else if (ST == kBF16) {
      ((__nv_bfloat16*)dst)[t] = __float2bfloat16_rn(a);
    } else if (ST == kFP8) {
      const int k = (i < rows) ? row_exp[i] : 0;
      ((__nv_fp8_storage_t*)dst)[t] =
          __nv_cvt_float_to_fp8(scalbnf(a, -k), __NV_SATFINITE, __NV_E4M3);
    } else if (ST == kI16) {
      ((int16_t*)dst)[t] = (int16_t)rintf(scalbnf(a, q));
    } else {
      ((int8_t*)dst)[t] = (int8_t)rintf(scalbnf(a, q));
    }
  }
}

// FP8 row exponent: smallest k with max_j |a_ij| <= 448 * 2^k.  With
// max = m 2^e (0.5 <= m < 1, exact frexp) and 448 = 0.875 * 2^9 this is
// k = e - 9 when m <= 0.875 and e - 8 otherwise; an all-zero row gets 0.
// row_mult = 2^(120 + k) undoes the decoder's bias and the scale together;
// it must stay finite, so k <= 7 (row maxima up to 448 * 2^7).
__global__ void k_fp8_rowexp(const float* __restrict__ src, int64_t ld_src, int rows,
                             int cols, int rows_pad, int* row_exp, float* row_mult,
                             int* flag) {
  const int lane = threadIdx.x & 31;
  const int warps = blockDim.x / 32;
  for (int i = blockIdx.x * warps + threadIdx.x / 32; i < rows_pad; i += gridDim.x * warps) {
    float m = 0.f;
    if (i < rows)
      for (int j = lane; j < cols; j += 32) m = fmaxf(m, fabsf(src[(int64_t)i * ld_src + j]));
#pragma unroll
    for (int o = 16; o; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0) {
      int k = 0;
      if (m > 0.f) {
        int e;
        const float f = frexpf(m, &e);
        k = (f <= 0.875f) ? e - 9 : e - 8;
      }
      if (k > 7) atomicOr(flag, 2);
      row_exp[i] = k;
      row_mult[i] = scalbnf(1.f, 120 + min(k, 7));
    }
  }
}

// Dequantised read-back (exact in FP32 for every storage).
template <int ST>
__global__ void k_unpack(const void* src, int rows, int cols, int64_t ld, int q,
                         const int* __restrict__ row_exp, float* dst) {
  const int64_t total = (int64_t)rows * cols;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t / cols, j = t % cols, s = i * ld + j;
    float v;
    if (ST == kF32) v = ((const float*)src)[s];
    else if (ST == kBF16) v = __bfloat162float(((const __nv_bfloat16*)src)[s]);
    else if (ST == kFP8)
      v = scalbnf(e4m3_bits_unscaled(((const uint8_t*)src)[s]), 120 + row_exp[i]);
    else if (ST == kI16) v = scalbnf((float)((const int16_t*)src)[s], -q);
    else v = scalbnf((float)((const int8_t*)src)[s], -q);
    dst[t] = v;
  }
}

// Google matrix, Eq. (11): G = alpha H + (1 - alpha)/n, H_ij = (#links j->i)/
// outdeg(j), dangling columns 1/n.  Entries are formed once in FP64 in the
// same order as their definition and rounded to FP32: every non-link entry is
// exactly tau; links add alpha * (1/d) per link.  One thread per column.
__global__ void k_google_fill(float* G, int64_t ld, int n, float tau_f) {
  const int64_t total = (int64_t)n * ld;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = t % ld;
    G[t] = (j < n) ? tau_f : 0.f;
  }
}

__global__ void k_google_links(const int* __restrict__ indptr,
                               const int* __restrict__ indices, int n, double alpha,
                               float* G, int64_t ld) {
  const double tele = (1.0 - alpha) / (double)n;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
    const int b = indptr[j], e = indptr[j + 1];
    const int d = e - b;
    if (d == 0) {
      const float v = (float)__dadd_rn(__dmul_rn(alpha, 1.0 / (double)n), tele);
      for (int i = 0; i < n; ++i) G[(int64_t)i * ld + j] = v;
      continue;
    }
    for (int k = b; k < e; ++k) {
      const int i = indices[k];
      if (i < 0 || i >= n) continue;  // out-of-range link: ignored, never written through
      // multiplicity of this link (targets of j are few; count them)
      int mult = 0;
      bool first = true;
      for (int k2 = b; k2 < e; ++k2) {
        if (indices[k2] == i) {
          if (k2 < k) first = false;
          ++mult;
        }
      }
      if (!first) continue;
      double h = 0.0;
      for (int r = 0; r < mult; ++r) h = __dadd_rn(h, 1.0 / (double)d);
      G[(int64_t)i * ld + j] = (float)__dadd_rn(__dmul_rn(alpha, h), tele);
    }
  }
}

// ---------------------------------------------------------------- launchers

static int grid_for(int64_t total, int threads, int sm) {
  int64_t g = (total + threads - 1) / threads;
  const int64_t cap = (int64_t)sm * 32;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return (int)g;
}

mapi_status launch_check_finite(mapi_ctx* ctx, const float* src, int rows, int cols,
                                int64_t ld, int* flag_dev) {
  k_check_finite<<<grid_for((int64_t)rows * cols, 256, ctx->sm_count), 256, 0,
                   ctx->stream>>>(src, rows, cols, ld, flag_dev);
  MAPI_CUDA_TRY(ctx, cudaGetLastError());
  count_launch(ctx);
  return MAPI_OK;
}

mapi_status launch_absmax(mapi_ctx* ctx, const float* src, int rows, int cols,
                          int64_t ld, unsigned* out_bits_dev) {
  k_absmax<<<grid_for((int64_t)rows * cols, 256, ctx->sm_count), 256, 0, ctx->stream>>>(
      src, rows, cols, ld, out_bits_dev);
  MAPI_CUDA_TRY(ctx, cudaGetLastError());
  count_launch(ctx);
  return MAPI_OK;
}

mapi_status launch_fp8_rowexp(mapi_ctx* ctx, const float* src, int64_t ld_src,
                              mapi_mat* m, int* flag_dev) {
  k_fp8_rowexp<<<grid_for((int64_t)m->rows_pad * 32, 256, ctx->sm_count), 256, 0,
                 ctx->stream>>>(src, ld_src, m->rows, m->cols, m->rows_pad, m->row_exp,
                                m->row_scale, flag_dev);
  MAPI_CUDA_TRY(ctx, cudaGetLastError());
  count_launch(ctx);
  return MAPI_OK;
}

mapi_status launch_pack(mapi_ctx* ctx, const float* src, int64_t ld_src, mapi_mat* m) {
  const int64_t total = (int64_t)m->rows_pad * m->ld;
  const int g = grid_for(total, 256, ctx->sm_count);
  switch (m->storage) {
    case MAPI_ST_F32:
      k_pack<kF32><<<g, 256, 0, ctx->stream>>>(src, ld_src, m->rows, m->cols, m->rows_pad,
                                                m->ld, m->data, m->q, m->row_exp);
      break;
    case MAPI_ST_BF16:
      k_pack<kBF16><<<g, 256, 0, ctx->stream>>>(src, ld_src, m->rows, m->cols, m->rows_pad,
                                                 m->ld, m->data, m->q, m->row_exp);
      break;
    case MAPI_ST_FP8E4M3_ROWPOW2:
      k_pack<kFP8><<<g, 256, 0, ctx->stream>>>(src, ld_src, m->rows, m->cols, m->rows_pad,
                                                m->ld, m->data, m->q, m->row_exp);
      break;
    case MAPI_ST_I16:
      k_pack<kI16><<<g, 256, 0, ctx->stream>>>(src, ld_src, m->rows, m->cols, m->rows_pad,
                                                m->ld, m->data, m->q, m->row_exp);
      break;
    case MAPI_ST_I8:
      k_pack<kI8><<<g, 256, 0, ctx->stream>>>(src, ld_src, m->rows, m->cols, m->rows_pad,
                                               m->ld, m->data, m->q, m->row_exp);
      break;
  }
  MAPI_CUDA_TRY(ctx, cudaGetLastError());
  count_launch(ctx);
  return MAPI_OK;
}

mapi_status launch_unpack_f32(mapi_ctx* ctx, const mapi_mat* m, float* dst) {
  const int g = grid_for((int64_t)m->rows * m->cols, 256, ctx->sm_count);
  switch (m->storage) {
    case MAPI_ST_F32:
      k_unpack<kF32><<<g, 256, 0, ctx->stream>>>(m->data, m->rows, m->cols, m->ld, m->q, m->row_exp, dst);
      break;
    case MAPI_ST_BF16:
      k_unpack<kBF16><<<g, 256, 0, ctx->stream>>>(m->data, m->rows, m->cols, m->ld, m->q, m->row_exp, dst);
      break;
    case MAPI_ST_FP8E4M3_ROWPOW2:
      k_unpack<kFP8><<<g, 256, 0, ctx->stream>>>(m->data, m->rows, m->cols, m->ld, m->q, m->row_exp, dst);
      break;
    case MAPI_ST_I16:
      k_unpack<kI16><<<g, 256, 0, ctx->stream>>>(m->data, m->rows, m->cols, m->ld, m->q, m->row_exp, dst);
      break;
    case MAPI_ST_I8:
      k_unpack<kI8><<<g, 256, 0, ctx->stream>>>(m->data, m->rows, m->cols, m->ld, m->q, m->row_exp, dst);
      break;
  }
  MAPI_CUDA_TRY(ctx, cudaGetLastError());
  count_launch(ctx);
  return MAPI_OK;
}

mapi_status launch_google(mapi_ctx* ctx, const int* indptr, const int* indices, int n,
                          double alpha, float* dst, int64_t ld) {
  const float tau_f = (float)((1.0 - alpha) / (double)n);
  k_google_fill<<<grid_for((int64_t)n * ld, 256, ctx->sm_count), 256, 0, ctx->stream>>>(
      dst, ld, n, tau_f);
  MAPI_CUDA_TRY(ctx, cudaGetLastError());
  count_launch(ctx);
  k_google_links<<<(n + 127) / 128, 128, 0, ctx->stream>>>(indptr, indices, n, alpha, dst, ld);
  MAPI_CUDA_TRY(ctx, cudaGetLastError());
  count_launch(ctx);
  return MAPI_OK;
}

}  // namespace mapi
