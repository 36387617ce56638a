// K1 MAVP-GEMV instantiations for integer storage (exact INT32 sums).
#include "k_iter.cuh"

namespace mapi {

template <int OP, int ST, int V>
static cudaError_t launch_int(dim3 grid, cudaStream_t s, const GemvArgs& g, int q) {
  IGemvArgs a{g, q};
  if (g.n < kGemvClusterMinRows || !g.clusters) {
    k1_gemv_int<OP, ST, V, gemv_rows<ST>(), kWarps, 1><<<grid, kWarps * 32, 0, s>>>(a);
    return cudaGetLastError();
  }
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = kGemvCluster;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3((grid.x + kGemvCluster - 1) / kGemvCluster * kGemvCluster, grid.y, 1);
  cfg.blockDim = dim3(kWarps * 32, 1, 1);
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k1_gemv_int<OP, ST, V, gemv_rows<ST>(), kWarps, kGemvCluster>, a);
}

template <int ST>
static LaunchFn lookup_st(int op, int V) {
  switch (op * 16 + V) {
    case MAPI_OP_MIN1 * 16 + 1: return launch_int<MAPI_OP_MIN1, ST, 1>;
    case MAPI_OP_MIN1 * 16 + 2: return launch_int<MAPI_OP_MIN1, ST, 2>;
    case MAPI_OP_MIN1 * 16 + 4: return launch_int<MAPI_OP_MIN1, ST, 4>;
    case MAPI_OP_MIN1 * 16 + 8: return launch_int<MAPI_OP_MIN1, ST, 8>;
    case MAPI_OP_MIN2 * 16 + 1: return launch_int<MAPI_OP_MIN2, ST, 1>;
    case MAPI_OP_MIN2 * 16 + 2: return launch_int<MAPI_OP_MIN2, ST, 2>;
    case MAPI_OP_MIN2 * 16 + 4: return launch_int<MAPI_OP_MIN2, ST, 4>;
    case MAPI_OP_MIN2 * 16 + 8: return launch_int<MAPI_OP_MIN2, ST, 8>;
  }
  return nullptr;
}

LaunchFn gemv_lookup_int(int st, int op, int V) {
  if (st == kI16) return lookup_st<kI16>(op, V);
  if (st == kI8) return lookup_st<kI8>(op, V);
  return nullptr;
}

}  // namespace mapi
