// Fused update and auxiliary kernels for D2Q9 with f64 storage.
#include "tu_impl.cuh"
LBM_DEFINE_OPS(ops_d2q9_f64, D2Q9, StF64)
