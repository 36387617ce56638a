// K1 MAVP-GEMV instantiations for BF16 storage.
#include "k_iter.cuh"
MAPI_DEFINE_FLOAT_TABLE(gemv_lookup_bf16, kBF16)
