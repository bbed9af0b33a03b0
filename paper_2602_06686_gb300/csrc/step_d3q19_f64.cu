// Fused update and auxiliary kernels for D3Q19 with f64 storage.
#include "tu_impl.cuh"
LBM_DEFINE_OPS(ops_d3q19_f64, D3Q19, StF64)
