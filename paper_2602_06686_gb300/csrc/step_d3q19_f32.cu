// Fused update and auxiliary kernels for D3Q19 with f32 storage.
#include "tu_impl.cuh"
LBM_DEFINE_OPS(ops_d3q19_f32, D3Q19, StF32)
