// Fused update and auxiliary kernels for D3Q27 with f16 storage.
#include "tu_impl.cuh"
LBM_DEFINE_OPS(ops_d3q27_f16, D3Q27, StF16)
