// Fused update and auxiliary kernels for D3Q27 with bf16 storage.
#include "tu_impl.cuh"
LBM_DEFINE_OPS(ops_d3q27_bf16, D3Q27, StBF16)
