// Fused update and auxiliary kernels for D3Q19 with bf16 storage.
#include "tu_impl.cuh"
LBM_DEFINE_OPS(ops_d3q19_bf16, D3Q19, StBF16)
