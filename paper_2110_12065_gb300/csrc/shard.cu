// Pieces of a partitioned solve (one shard of the data per process): the
// unnormalised product of a block of rows of A with w, y_i = a_i^T (+) w
// (the matrix-vector step of Alg. 1 before its normalisation).  Each rank
// of a row-partitioned solve computes its rows, the ranks gather y, and the
// l1 normalisation of Eq. (6) is applied to the whole vector.
#include "device_common.cuh"

namespace mapi {
namespace {

constexpr int kRowsWarps = 8;

// One warp per row: lanes stride the row's 16-byte chunks, each chunk's
// elements against the matching entries of w, then a warp butterfly.
template <int OP, int ST>
__global__ void __launch_bounds__(kRowsWarps * 32)
    k_rows_raw(const uint8_t* __restrict__ A, int64_t row_bytes, int n, int row_begin,
               int rows, const float* __restrict__ row_mult, const float* __restrict__ w,
               float* __restrict__ y) {
  const int lane = threadIdx.x & 31;
  const int r = blockIdx.x * kRowsWarps + (threadIdx.x >> 5);
  if (r >= rows) return;
  const int i = row_begin + r;
  constexpr int E = Chunk<ST>::E;
  const int chunks = (n + E - 1) / E;
  const float mult = (ST == kFP8) ? row_mult[i] : 1.f;
  const uint8_t* arow = A + (int64_t)i * row_bytes;
  float acc = 0.f;
  for (int c = lane; c < chunks; c += 32) {
    Chunk<ST> ch;
    ch.raw = ld_stream(arow + (int64_t)c * 16);
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int j = c * E + e;
      if (j < n) acc = Op<OP>::term(ch.get(e) * mult, Op<OP>::prep(w[j]), acc);
    }
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) y[r] = acc;
}

template <int OP>
const void* rows_fn(mapi_storage st) {
  switch (st) {
    case MAPI_ST_F32: return (const void*)k_rows_raw<OP, kF32>;
    case MAPI_ST_BF16: return (const void*)k_rows_raw<OP, kBF16>;
    case MAPI_ST_FP8E4M3_ROWPOW2: return (const void*)k_rows_raw<OP, kFP8>;
    default: return nullptr;
  }
}

}  // namespace

mapi_status launch_rows_raw(mapi_ctx* ctx, const mapi_mat* A, int row_begin, int rows,
                            mapi_op op, const float* w, float* y, cudaStream_t s) {
  const void* fn = op == MAPI_OP_MIN1   ? rows_fn<MAPI_OP_MIN1>(A->storage)
                   : op == MAPI_OP_MIN2 ? rows_fn<MAPI_OP_MIN2>(A->storage)
                   : op == MAPI_OP_DOT  ? rows_fn<MAPI_OP_DOT>(A->storage)
                                        : nullptr;
  if (!fn) return fail(ctx, MAPI_EINVAL, "row product: MIN1, MIN2 or DOT on F32, BF16 or FP8");
  if (rows == 0) return MAPI_OK;
  const uint8_t* a = (const uint8_t*)A->data;
  int64_t rb = A->ld * elem_bytes(A->storage);
  int n = A->cols;
  const float* rm = A->row_scale;
  void* args[] = {(void*)&a, (void*)&rb, (void*)&n, (void*)&row_begin, (void*)&rows,
                  (void*)&rm, (void*)&w, (void*)&y};
  MAPI_CUDA_TRY(ctx, cudaLaunchKernel(fn, dim3((rows + kRowsWarps - 1) / kRowsWarps),
                                      dim3(kRowsWarps * 32), args, 0, s));
  count_launch(ctx);
  return MAPI_OK;
}

}  // namespace mapi
