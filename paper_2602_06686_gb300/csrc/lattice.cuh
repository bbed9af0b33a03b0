// lattice.cuh -- compile-time lattice tables for the fused kernels.
//
// D2Q9 follows Eq. (D2Q9) of arXiv 2602.06686; D3Q19 uses 1 rest, 6 axial and
// 12 face-diagonal velocities (App. A.2) with the isotropic weights 1/3, 1/18,
// 1/36 in the order: rest, +x, -x, +y, -y, +z, -z, then the xy, xz, yz
// diagonals as (++, --, +-, -+); D3Q27 (App. D3Q27) continues D3Q19's order
// with the 8 body diagonals in inversion pairs (+++, ---), (++-, --+),
// (+-+, -+-), (-++, +--), weights the products of the D1Q3 weights
// (8/27, 2/27, 1/54, 1/216).  Weights are wnum(i) / kWDen.  Everything is a constexpr function of the
// velocity index so that, inside fully unrolled loops, every table access folds
// into an immediate and every zero velocity component removes its term.
#pragma once

namespace lbm {

struct D2Q9 {
  static constexpr int Q = 9;
  static constexpr int D = 2;
  static constexpr int NG = 1;
  __host__ __device__ static constexpr int cx(int i) {
    constexpr int v[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
    return v[i];
  }
  __host__ __device__ static constexpr int cy(int i) {
    constexpr int v[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
    return v[i];
  }
  __host__ __device__ static constexpr int cz(int) { return 0; }
  __host__ __device__ static constexpr int opp(int i) {
    constexpr int v[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
    return v[i];
  }
  static constexpr int kWDen = 36;
  __host__ __device__ static constexpr int wnum(int i) { return i == 0 ? 16 : (i <= 4 ? 4 : 1); }
  __host__ __device__ static constexpr double w(int i) { return wnum(i) / 36.0; }
};

struct D3Q19 {
  static constexpr int Q = 19;
  static constexpr int D = 3;
  static constexpr int NG = 3;
  __host__ __device__ static constexpr int cx(int i) {
    constexpr int v[19] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
    return v[i];
  }
  __host__ __device__ static constexpr int cy(int i) {
    constexpr int v[19] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1};
    return v[i];
  }
  __host__ __device__ static constexpr int cz(int i) {
    constexpr int v[19] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1};
    return v[i];
  }
  __host__ __device__ static constexpr int opp(int i) {
    constexpr int v[19] = {0, 2, 1, 4, 3, 6, 5, 8, 7, 10, 9, 12, 11, 14, 13, 16, 15, 18, 17};
    return v[i];
  }
  static constexpr int kWDen = 36;
  __host__ __device__ static constexpr int wnum(int i) {
    return i == 0 ? 12 : (i <= 6 ? 2 : 1);
  }
  __host__ __device__ static constexpr double w(int i) { return wnum(i) / 36.0; }
};

struct D3Q27 {
  static constexpr int Q = 27;
  static constexpr int D = 3;
  static constexpr int NG = 7;
  __host__ __device__ static constexpr int cx(int i) {
    constexpr int v[27] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0,
                           1, -1, 1, -1, 1, -1, -1, 1};
    return v[i];
  }
  __host__ __device__ static constexpr int cy(int i) {
    constexpr int v[27] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1,
                           1, -1, 1, -1, -1, 1, 1, -1};
    return v[i];
  }
  __host__ __device__ static constexpr int cz(int i) {
    constexpr int v[27] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1,
                           1, -1, -1, 1, 1, -1, 1, -1};
    return v[i];
  }
  __host__ __device__ static constexpr int opp(int i) {
    return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1);
  }
  static constexpr int kWDen = 216;
  __host__ __device__ static constexpr int wnum(int i) {
    return i == 0 ? 64 : (i <= 6 ? 16 : (i <= 18 ? 4 : 1));
  }
  __host__ __device__ static constexpr double w(int i) { return wnum(i) / 216.0; }
};

// Representative of each inversion pair: i < opp(i) (and the rest velocity).
template <class L>
__host__ __device__ constexpr bool is_pair_rep(int i) {
  return i < L::opp(i);
}

}  // namespace lbm
