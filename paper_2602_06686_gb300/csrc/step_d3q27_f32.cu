// Fused update and auxiliary kernels for D3Q27 with f32 storage.
#include "tu_impl.cuh"
LBM_DEFINE_OPS(ops_d3q27_f32, D3Q27, StF32)
