// Fused update and auxiliary kernels for D2Q9 with bf16 storage.
#include "tu_impl.cuh"
LBM_DEFINE_OPS(ops_d2q9_bf16, D2Q9, StBF16)
