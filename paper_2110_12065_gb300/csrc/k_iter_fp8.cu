// K1 MAVP-GEMV instantiations for FP8-E4M3 storage with power-of-two row scales.
#include "k_iter.cuh"
MAPI_DEFINE_FLOAT_TABLE(gemv_lookup_fp8, kFP8)
