// K1 MAVP-GEMV instantiations for FP32 storage.
#include "k_iter.cuh"
MAPI_DEFINE_FLOAT_TABLE(gemv_lookup_f32, kF32)
