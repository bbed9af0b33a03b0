// Fused update and auxiliary kernels for D2Q9 with f16 storage.
#include "tu_impl.cuh"
LBM_DEFINE_OPS(ops_d2q9_f16, D2Q9, StF16)
