// collide_v.cuh -- the per-node collision operators, generic over the
// arithmetic type V: float, double, or F2 (two FP32 nodes advanced together
// with the packed f32x2 instructions of sm_100+).
//
// Input and output are the shifted populations g_i = f_i - w_i rho0.  The
// operators (arXiv 2602.06686):
//   f* = f_eq + (1 - w+) R2 + (1 - w-) R3 + F_i/2 + (1 - w+/2) S+
//   TRT      R2 = fneq+                        R3 = fneq- + F_i/2
//   P-TRT    R2 = fneq+ - P_G fneq (Eq. PTRT)  R3 = fneq- + F_i/2 (Eq. R3_force)
//   TRT-RLB  R2 = P^(2) fneq, R3 = P^(3) fneq  (Eq. R2R3_hermite as w-orthogonal projections)
// with rho and the half-force velocity u of Eq. macro, the third-order
// equilibrium of Eq. feq, written per inversion pair (i, ibar) as
//   f_eq,i +- f_eq,ibar = 2 w [drho + rho (4.5 eu^2 - 1.5 u^2)]  +-  2 w rho eu (3 + 4.5 (eu^2 - u^2))
// (H3_i : uuu = (e_i.u)^3 - 3 cs^2 u^2 (e_i.u) on any velocity set),
// F_i = 3 w e_i.F and S+ = w (9 eu eF - 3 u.F).  The force reading keeps the
// first-order term of Sec. 2.2 and the whole Guo source at (1 - w+/2), which
// makes the antisymmetric force content F_i/2 + (1-w-) R3 for every rate.
//
// Ghost modes (hand-derived, w-orthogonal, integer values G(k, i)):
//   D2Q9 : phi = (ex^2 - cs^2)(ey^2 - cs^2) = cs^4 G with G = 1 (rest), -2
//          (axial), 4 (diagonal) and norm 4 cs^8 (App. A.1, Eq. R2_D2Q9).
//   D3Q19: the printed products (e_a^2 - cs^2)(e_b^2 - cs^2) are neither mutually
//          orthogonal nor orthogonal to H2 on D3Q19; the ghost subspace (the
//          complement of span{1, H2} in the symmetric subspace, Eq. S_decomp) is
//          spanned by phi~_ab = (e_a^2 - cs^2)(e_b^2 - cs^2) + (cs^2/2)(e_c^2 - cs^2)
//          and diagonalised into g_e = phi~_xy + phi~_yz + phi~_zx (norm 9/2 cs^8),
//          g_1 = phi~_xy - phi~_yz (9 cs^8), g_2 = phi~_xy + phi~_yz - 2 phi~_zx
//          (27 cs^8) with values
//              g_e*6: rest 1, axial -2, diagonal 1
//              g_1*2: x pair -1, z pair 1, xy diagonals 1, yz diagonals -1
//              g_2*2: x pair 1, y pair -2, z pair 1, xy 1, yz 1, xz -2.
//   P_G fneq = sum_k w_i G(k,i) (s_k^2 / N_k) sum_j G(k,j) fneq_j, where the
//   ghost sums are taken over the (shifted) populations: the ghost vectors are
//   w-orthogonal to 1 and H2, which span the symmetric part of f_eq and the
//   shift, so sum_j G(k,j) fneq_j = sum_j G(k,j) g_j exactly.  TRT and P-TRT
//   then finish each inversion pair in one pass; TRT-RLB forms every fneq first.
// TRT-RLB on D3Q19: the third-order components m_ab = e_a (e_b^2 - cs^2) of the
// same odd axis a overlap (<m_ab, m_ac>_w = -cs^6); their sum (norm 2 cs^6) and
// difference (norm 6 cs^6) are w-orthogonal.
//
// Every operation is an explicitly rounded add / sub / mul / fma, so the scalar
// and packed paths give bit-identical results and the compiler cannot regroup.
// No inexact product feeds a separate addition: the optimiser fuses such pairs
// in the packed form (the scalar intrinsics are left alone), so every product
// that is summed is written as an fma here.
#pragma once
#include <string.h>

#include <type_traits>

#include "lattice.cuh"

namespace lbm {

enum { C_TRT = 0, C_TRT_RLB = 1, C_P_TRT = 2 };

struct alignas(8) F2 {
  float x, y;
};

template <typename V>
struct Ar;

#if defined(__CUDA_ARCH__)
template <>
struct Ar<float> {
  using S = float;
  __device__ __forceinline__ static float add(float a, float b) { return __fadd_rn(a, b); }
  __device__ __forceinline__ static float sub(float a, float b) { return __fsub_rn(a, b); }
  __device__ __forceinline__ static float mul(float a, float b) { return __fmul_rn(a, b); }
  __device__ __forceinline__ static float fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
  __device__ __forceinline__ static float rcp(float a) { return __frcp_rn(a); }
  __device__ __forceinline__ static float c(double v) { return float(v); }
  __device__ __forceinline__ static float c(float v) { return v; }
  __device__ __forceinline__ static unsigned bad(float rho, float usq) {
    return (!(rho > 0.f) || !(usq <= 1.f)) ? 1u : 0u;
  }
};
template <>
struct Ar<double> {
  using S = double;
  __device__ __forceinline__ static double add(double a, double b) { return __dadd_rn(a, b); }
  __device__ __forceinline__ static double sub(double a, double b) { return __dsub_rn(a, b); }
  __device__ __forceinline__ static double mul(double a, double b) { return __dmul_rn(a, b); }
  __device__ __forceinline__ static double fma(double a, double b, double c) { return __fma_rn(a, b, c); }
  __device__ __forceinline__ static double rcp(double a) { return __drcp_rn(a); }
  __device__ __forceinline__ static double c(double v) { return v; }
  __device__ __forceinline__ static unsigned bad(double rho, double usq) {
    return (!(rho > 0.0) || !(usq <= 1.0)) ? 1u : 0u;
  }
};
// The two floats travel as separate 32-bit operands and are packed into the
// 64-bit f32x2 operand inside the asm block (register-pair moves that the
// assembler coalesces), so no value ever round-trips through local memory.
template <>
struct Ar<F2> {
  using S = float;
  __device__ __forceinline__ static F2 add(F2 a, F2 b) {
    F2 r;
    asm("{\n\t.reg .b64 a, b, d;\n\t"
        "mov.b64 a, {%2, %3};\n\tmov.b64 b, {%4, %5};\n\t"
        "add.rn.f32x2 d, a, b;\n\tmov.b64 {%0, %1}, d;\n\t}"
        : "=f"(r.x), "=f"(r.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return r;
  }
  __device__ __forceinline__ static F2 sub(F2 a, F2 b) {
    F2 r;
    asm("{\n\t.reg .b64 a, b, d;\n\t"
        "mov.b64 a, {%2, %3};\n\tmov.b64 b, {%4, %5};\n\t"
        "sub.rn.f32x2 d, a, b;\n\tmov.b64 {%0, %1}, d;\n\t}"
        : "=f"(r.x), "=f"(r.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return r;
  }
  __device__ __forceinline__ static F2 mul(F2 a, F2 b) {
    F2 r;
    asm("{\n\t.reg .b64 a, b, d;\n\t"
        "mov.b64 a, {%2, %3};\n\tmov.b64 b, {%4, %5};\n\t"
        "mul.rn.f32x2 d, a, b;\n\tmov.b64 {%0, %1}, d;\n\t}"
        : "=f"(r.x), "=f"(r.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return r;
  }
  __device__ __forceinline__ static F2 fma(F2 a, F2 b, F2 c) {
    F2 r;
    asm("{\n\t.reg .b64 a, b, c, d;\n\t"
        "mov.b64 a, {%2, %3};\n\tmov.b64 b, {%4, %5};\n\tmov.b64 c, {%6, %7};\n\t"
        "fma.rn.f32x2 d, a, b, c;\n\tmov.b64 {%0, %1}, d;\n\t}"
        : "=f"(r.x), "=f"(r.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
    return r;
  }
  __device__ __forceinline__ static F2 rcp(F2 a) { return F2{__frcp_rn(a.x), __frcp_rn(a.y)}; }
  __device__ __forceinline__ static F2 c(double v) { return F2{float(v), float(v)}; }
  __device__ __forceinline__ static F2 c(float v) { return F2{v, v}; }
  __device__ __forceinline__ static unsigned bad(F2 rho, F2 usq) {
    return Ar<float>::bad(rho.x, usq.x) | (Ar<float>::bad(rho.y, usq.y) << 1);
  }
};
#else
// Host compilation (used only to check the arithmetic against the oracle on a CPU).
template <typename T>
struct ArHost {
  using S = T;
  static T add(T a, T b) { return a + b; }
  static T sub(T a, T b) { return a - b; }
  static T mul(T a, T b) { return a * b; }
  static T fma(T a, T b, T c) { return __builtin_fma(a, b, c); }
  static T rcp(T a) { return T(1) / a; }
  static T c(double v) { return T(v); }
  static T c(float v) { return T(v); }
  static unsigned bad(T rho, T usq) { return (!(rho > 0) || !(usq <= 1)) ? 1u : 0u; }
};
template <>
struct Ar<double> : ArHost<double> {};
template <>
struct Ar<float> : ArHost<float> {
  static float fma(float a, float b, float c) { return __builtin_fmaf(a, b, c); }
};
#endif

// Per-launch constants (computed on the host in FP64, stored in the arithmetic
// precision).  The force terms are compiled out when the force is zero
// (FORCE = false).  Per-direction entries are used at pair representatives.
constexpr int kQMax = 27;
template <typename S>
struct CoefV {
  S rho0;
  S cp;            // 1 - w+
  S cm;            // 1 - w-  (as run: BGK w- = w+, RLB w- = 1)
  S Fh[3];         // F / 2 (half-force velocity, Eq. macro)
  S F[3];          // F (for u.F)
  S fe[kQMax];     // 9 w_i (e_i.F) (1 - w+/2): coefficient of e_i.u in S+_i
  S fu[kQMax];     // -3 w_i (1 - w+/2): coefficient of u.F in S+_i
  S fa[kQMax];     // antisymmetric force content: F_i/2 (2 - w-) (TRT, P-TRT) or F_i/2 (TRT-RLB)
};

// ---- ghost tables (integer values and s_k^2 / N_k) ------------------------
template <class L>
struct GhostT;

template <>
struct GhostT<D2Q9> {
  static constexpr int NG = 1;
  __host__ __device__ static constexpr int G(int, int i) { return i == 0 ? 1 : (i <= 4 ? -2 : 4); }
  // phi = G/9, N = 4/81 -> s^2/N = 1/4
  __host__ __device__ static constexpr double coef(int) { return 0.25; }
};

// D3Q27 P-TRT takes the tensor projection (the hybrid), so its ghost table is
// never read; TRT, which shares the pair branch, needs only NG.
template <>
struct GhostT<D3Q27> {
  static constexpr int NG = 1;
  __host__ __device__ static constexpr int G(int, int) { return 0; }
  __host__ __device__ static constexpr double coef(int) { return 0.0; }
};

template <>
struct GhostT<D3Q19> {
  static constexpr int NG = 3;
  // class: 0 rest, 1/2/3 axial along x/y/z, 4 xy, 5 xz, 6 yz diagonal
  __host__ __device__ static constexpr int cls(int i) {
    return i == 0 ? 0 : (i <= 6 ? 1 + (i - 1) / 2 : 4 + (i - 7) / 4);
  }
  __host__ __device__ static constexpr int G(int k, int i) {
    constexpr int ge[7] = {1, -2, -2, -2, 1, 1, 1};
    constexpr int g1[7] = {0, -1, 0, 1, 1, 0, -1};
    constexpr int g2[7] = {0, 1, -2, 1, 1, -2, 1};
    return k == 0 ? ge[cls(i)] : (k == 1 ? g1[cls(i)] : g2[cls(i)]);
  }
  // g_e = G/6, N = 1/18 -> 1/2;  g_1 = G/2, N = 1/9 -> 9/4;  g_2 = G/2, N = 1/3 -> 3/4
  __host__ __device__ static constexpr double coef(int k) { return k == 0 ? 0.5 : (k == 1 ? 2.25 : 0.75); }
};

template <class L>
__host__ __device__ constexpr int ecomp(int i, int a) {
  return a == 0 ? L::cx(i) : (a == 1 ? L::cy(i) : L::cz(i));
}

// sum_a e_i,a v_a: the positive components are added first, then the negative
// ones subtracted (every pair representative has a +1 component).
template <class L, typename V>
__device__ __forceinline__ V edot(int i, const V (&v)[3]) {
  using A = Ar<V>;
  V acc = A::c(0.0);
  bool init = false;
#pragma unroll
  for (int a = 0; a < L::D; ++a)
    if (ecomp<L>(i, a) == 1) {
      acc = init ? A::add(acc, v[a]) : v[a];
      init = true;
    }
#pragma unroll
  for (int a = 0; a < L::D; ++a)
    if (ecomp<L>(i, a) == -1) acc = A::sub(acc, v[a]);
  return acc;
}

// x / den for the integer denominator of the weights.  In FP32 arithmetic the
// reciprocal is split into head + tail (head = 1/den rounded to FP32, tail =
// the rounding error of the head, itself rounded): fma(x, head, x * tail) is x/den
// to within the final rounding, with no common relative bias.
template <typename V>
__device__ __forceinline__ V wden_div(V x, int den) {
  using A = Ar<V>;
  if constexpr (std::is_same<typename A::S, float>::value) {
    const double inv = 1.0 / den;
    const float head = float(inv);
    const float tail = float(inv - double(head));
    return A::fma(x, A::c(head), A::mul(x, A::c(tail)));
  } else {
    return A::mul(x, A::c(1.0 / den));
  }
}

// The collision.  Returns a bit mask of the lanes (nodes) that are not finite,
// have rho <= 0 or |u| > 1.
template <class L, int COLL, bool FORCE, typename V>
__device__ __forceinline__ unsigned collide_v(V (&g)[L::Q], const CoefV<typename Ar<V>::S>& c) {
  using A = Ar<V>;
  constexpr int Q = L::Q;
  // ---- pair sums / differences, density and momentum
  V s[Q], d[Q];
  V drho = g[0];
#pragma unroll
  for (int i = 1; i < Q; ++i) {
    if (!is_pair_rep<L>(i)) continue;
    s[i] = A::add(g[i], g[L::opp(i)]);
    d[i] = A::sub(g[i], g[L::opp(i)]);
    drho = A::add(drho, s[i]);
  }
  V j[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    j[a] = A::c(0.0);
    if (a >= L::D) continue;
    bool init = false;
#pragma unroll
    for (int i = 1; i < Q; ++i) {
      if (!is_pair_rep<L>(i)) continue;
      const int e = ecomp<L>(i, a);
      if (e == 1) {
        j[a] = init ? A::add(j[a], d[i]) : d[i];
        init = true;
      }
    }
#pragma unroll
    for (int i = 1; i < Q; ++i) {
      if (!is_pair_rep<L>(i)) continue;
      if (ecomp<L>(i, a) == -1) j[a] = A::sub(j[a], d[i]);
    }
  }
  const V rho = A::add(A::c(c.rho0), drho);
  const V inv = A::rcp(rho);
  V u[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    if (a >= L::D) {
      u[a] = A::c(0.0);
      continue;
    }
    u[a] = FORCE ? A::mul(A::add(j[a], A::c(c.Fh[a])), inv) : A::mul(j[a], inv);
  }
  V usq = A::mul(u[0], u[0]);
  usq = A::fma(u[1], u[1], usq);
  if (L::D == 3) usq = A::fma(u[2], u[2], usq);
  const unsigned badmask = A::bad(rho, usq);

  // per-node scalars
  // rho w_i and drho w_i as (rho / kWDen) * wnum_i (one multiply less when wnum_i = 1).
  // 1/kWDen is not a binary fraction.  Multiplying by its rounded value would
  // scale every weight by the same (1 + d), so the equilibrium would carry
  // (1 + d) times the node's momentum, and the antisymmetric relaxation adds
  // w- d j to the momentum at every step: a drift that compounds over a run
  // (in FP32, d = 7.5e-9 gains 2.4e-8 of the kinetic energy per step at
  // w- = 1.6).  The quotient is therefore formed with the constant split into
  // its rounded head and the tail the rounding dropped, fma(x, head, x tail),
  // whose error is the final rounding alone (random from node to node).  In
  // FP64 the same bias is 1e-17 per step and the plain product is kept.
  const V rho36 = wden_div<V>(rho, L::kWDen);
  const V drho36 = wden_div<V>(drho, L::kWDen);
  const V musq15 = A::mul(usq, A::c(-1.5));
  const V k3 = A::fma(usq, A::c(-4.5), A::c(3.0));
  V uF = A::c(0.0);
  if (FORCE) {
    uF = A::mul(u[0], A::c(c.F[0]));
    uF = A::fma(u[1], A::c(c.F[1]), uF);
    if (L::D == 3) uF = A::fma(u[2], A::c(c.F[2]), uF);
  }

  // rest velocity: f_eq0 - w0 rho0 = w0 (drho - 1.5 rho u^2), with w0 taken as
  // wnum_0 / kWDen through the same scaled densities as the moving directions:
  // a separately rounded w0 would make the weights of the equilibrium sum to
  // 1 + (d0 - d) and move mass by (1 - w+)(d0 - d) w0 1.5 rho u^2 at every step.
  const V feq0 = A::mul(A::c(double(L::wnum(0))), A::fma(rho36, musq15, drho36));
  const V np0 = A::sub(g[0], feq0);

  // D3Q27 P-TRT is the hybrid of Eq. PTRT_D3Q27: the tensor projection for the
  // second-order term (N_G = 7 > M_2 = 6), fneq- for the third.  It shares the
  // one-pass pair branch: the second-order Hermite moments of fneq come from
  // the pair sums, A2_ab = sum_i e_a e_b g_i - rho u_a u_b - cs^2 drho delta_ab
  // (the second moment of f_eq is rho u u + rho cs^2 delta, that of the shift
  // rho0 cs^2 delta), and R2_i = 4.5 w_i H2_i : A2.
  constexpr bool kHybrid = COLL == C_P_TRT && L::Q == 27;
  if constexpr (COLL != C_TRT_RLB) {
    // TRT and P-TRT need no moment of fneq but the ghost moments, so each pair
    // is finished in one pass (few values live at once).  The ghost moments
    // are taken from the populations: the ghost vectors are w-orthogonal to
    // span{1, H2} (Eq. S_decomp), which holds the symmetric part of f_eq and
    // the shift w_i rho0, so sum_j G(k,j) fneq_j = sum_j G(k,j) g_j exactly
    // (up to rounding), with g_i + g_ibar = s_i.
    using Gh = GhostT<L>;
    constexpr int NG = (COLL == C_P_TRT && !kHybrid) ? Gh::NG : 1;
    V m[NG];
    V r20 = np0;
    V A2d[3], A2o[3];  // hybrid: diagonal xx, yy, zz and off-diagonal xy, xz, yz
    if constexpr (kHybrid) {
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        bool id = false;
        A2d[a] = A::c(0.0);
#pragma unroll
        for (int i = 1; i < Q; ++i) {
          if (!is_pair_rep<L>(i) || ecomp<L>(i, a) == 0) continue;
          A2d[a] = id ? A::add(A2d[a], s[i]) : s[i];
          id = true;
        }
        A2d[a] = A::fma(A::mul(A::c(-1.0), rho), A::mul(u[a], u[a]), A2d[a]);
        A2d[a] = A::fma(A::c(-1.0 / 3.0), drho, A2d[a]);
      }
#pragma unroll
      for (int o = 0; o < 3; ++o) {
        const int a = o == 2 ? 1 : 0, b = o == 0 ? 1 : 2;
        bool io = false;
        A2o[o] = A::c(0.0);
#pragma unroll
        for (int i = 1; i < Q; ++i) {
          if (!is_pair_rep<L>(i)) continue;
          const int eab = ecomp<L>(i, a) * ecomp<L>(i, b);
          if (eab == 0) continue;
          A2o[o] = io ? (eab > 0 ? A::add(A2o[o], s[i]) : A::sub(A2o[o], s[i]))
                      : (eab > 0 ? s[i] : A::sub(A::c(0.0), s[i]));
          io = true;
        }
        A2o[o] = A::fma(A::mul(A::c(-1.0), rho), A::mul(u[a], u[b]), A2o[o]);
      }
      r20 = A::mul(A::c(4.5 * L::w(0) * (-1.0 / 3.0)), A::add(A::add(A2d[0], A2d[1]), A2d[2]));
    }
    if constexpr (COLL == C_P_TRT && !kHybrid) {
#pragma unroll
      for (int k = 0; k < NG; ++k) {
        V acc = Gh::G(k, 0) == 0 ? A::c(0.0) : A::mul(A::c(double(Gh::G(k, 0))), g[0]);
        bool init = Gh::G(k, 0) != 0;
#pragma unroll
        for (int i = 1; i < Q; ++i) {
          if (!is_pair_rep<L>(i) || Gh::G(k, i) == 0) continue;
          acc = init ? A::fma(A::c(double(Gh::G(k, i))), s[i], acc)
                     : A::mul(A::c(double(Gh::G(k, i))), s[i]);
          init = true;
        }
        m[k] = acc;
      }
      // R2_i = np_i - sum_k w_i G(k,i) (s_k^2/N_k) m_k as one fma chain from np_i
#pragma unroll
      for (int k = 0; k < NG; ++k) {
        if (Gh::G(k, 0) == 0) continue;
        r20 = A::fma(A::c(-L::w(0) * Gh::G(k, 0) * Gh::coef(k)), m[k], r20);
      }
    }
    // rest: f*_0 = f_eq0 + (1 - w+) R2_0 + S+_0, S+_0 = hg w0 (-3 u.F)
    V g0 = A::fma(A::c(c.cp), r20, feq0);
    if (FORCE) g0 = A::fma(A::c(c.fu[0]), uF, g0);
    g[0] = g0;
#pragma unroll
    for (int i = 1; i < Q; ++i) {
      if (!is_pair_rep<L>(i)) continue;
      const int w36 = L::wnum(i);
      const V eu = edot<L, V>(i, u);
      const V q = A::mul(eu, eu);
      const V t = A::fma(A::c(4.5), q, musq15);
      const V t2 = A::fma(A::c(4.5), q, k3);
      const V wr = w36 == 1 ? rho36 : A::mul(rho36, A::c(double(w36)));
      const V wd = w36 == 1 ? drho36 : A::mul(drho36, A::c(double(w36)));
      const V fs = A::fma(wr, t, wd);              // symmetric part of the shifted f_eq
      const V fa = A::mul(A::mul(wr, eu), t2);     // antisymmetric part
      V r2 = A::sub(A::mul(A::c(0.5), s[i]), fs);  // fneq+
      if constexpr (kHybrid) {
        V h = A::mul(A::c(ecomp<L>(i, 0) * ecomp<L>(i, 0) - 1.0 / 3.0), A2d[0]);
#pragma unroll
        for (int a = 1; a < 3; ++a) h = A::fma(A::c(ecomp<L>(i, a) * ecomp<L>(i, a) - 1.0 / 3.0), A2d[a], h);
#pragma unroll
        for (int o = 0; o < 3; ++o) {
          const int a = o == 2 ? 1 : 0, b = o == 0 ? 1 : 2;
          const int eab = ecomp<L>(i, a) * ecomp<L>(i, b);
          if (eab != 0) h = A::fma(A::c(2.0 * eab), A2o[o], h);
        }
        r2 = A::mul(A::c(4.5 * L::w(i)), h);
      } else if constexpr (COLL == C_P_TRT) {
#pragma unroll
        for (int k = 0; k < NG; ++k) {
          if (Gh::G(k, i) == 0) continue;
          r2 = A::fma(A::c(-L::w(i) * Gh::G(k, i) * Gh::coef(k)), m[k], r2);
        }
      }
      const V nm = A::sub(A::mul(A::c(0.5), d[i]), fa);  // fneq-
      V sym = A::fma(A::c(c.cp), r2, fs);
      V anti = A::fma(A::c(c.cm), nm, fa);
      if (FORCE) {
        // S+_i = hg w (9 eu eF - 3 u.F); antisymmetric force F_i/2 + (1 - w-) F_i/2
        sym = A::fma(A::c(c.fe[i]), eu, sym);
        sym = A::fma(A::c(c.fu[i]), uF, sym);
        anti = A::add(anti, A::c(c.fa[i]));
      }
      g[i] = A::add(sym, anti);
      g[L::opp(i)] = A::sub(sym, anti);
    }
    return badmask;
  } else {

    // ---- TRT-RLB: the Hermite projections need every fneq first.
    // per pair: equilibrium parts, fneq+-
    V fs[Q], fa[Q], np[Q], nm[Q];
#pragma unroll
    for (int i = 1; i < Q; ++i) {
      if (!is_pair_rep<L>(i)) continue;
      const int w36 = L::wnum(i);
      const V eu = edot<L, V>(i, u);
      const V q = A::mul(eu, eu);
      const V t = A::fma(A::c(4.5), q, musq15);
      const V t2 = A::fma(A::c(4.5), q, k3);
      const V wr = w36 == 1 ? rho36 : A::mul(rho36, A::c(double(w36)));
      const V wd = w36 == 1 ? drho36 : A::mul(drho36, A::c(double(w36)));
      fs[i] = A::fma(wr, t, wd);
      fa[i] = A::mul(A::mul(wr, eu), t2);
      np[i] = A::sub(A::mul(A::c(0.5), s[i]), fs[i]);
      nm[i] = A::sub(A::mul(A::c(0.5), d[i]), fa[i]);
    }

    // ---- symmetric relaxation target R2
    V r2[Q];
    V r20;
    {
      // TRT-RLB: w-orthogonal projection onto span{H2}:
      // A2_ab = sum_i (e_a e_b - cs^2 d_ab) fneq_i; R2_i = 4.5 w_i [sum_a H2_i,aa A_aa + 2 sum_{a<b} e_a e_b A_ab]
      V Ad[3], Ao[3];  // diagonal xx, yy, zz and off-diagonal xy, xz, yz
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        Ad[a] = A::mul(A::c(-1.0 / 3.0), np0);
        Ao[a] = A::c(0.0);
      }
      bool oinit[3] = {false, false, false};
#pragma unroll
      for (int i = 1; i < Q; ++i) {
        if (!is_pair_rep<L>(i)) continue;
#pragma unroll
        for (int a = 0; a < L::D; ++a) {
          const int e = ecomp<L>(i, a);
          Ad[a] = A::fma(A::c(2.0 * (e * e - 1.0 / 3.0)), np[i], Ad[a]);
        }
#pragma unroll
        for (int o = 0; o < 3; ++o) {
          const int a = o == 2 ? 1 : 0, b = o == 0 ? 1 : 2;
          if (b >= L::D) continue;
          const int eab = ecomp<L>(i, a) * ecomp<L>(i, b);
          if (eab == 0) continue;
          Ao[o] = oinit[o] ? A::fma(A::c(2.0 * eab), np[i], Ao[o]) : A::mul(A::c(2.0 * eab), np[i]);
          oinit[o] = true;
        }
      }
      V tr = A::add(Ad[0], Ad[1]);
      if (L::D == 3) tr = A::add(tr, Ad[2]);
      r20 = A::mul(A::c(4.5 * L::w(0) * (-1.0 / 3.0)), tr);
#pragma unroll
      for (int i = 1; i < Q; ++i) {
        if (!is_pair_rep<L>(i)) continue;
        V h = A::mul(A::c(ecomp<L>(i, 0) * ecomp<L>(i, 0) - 1.0 / 3.0), Ad[0]);
#pragma unroll
        for (int a = 1; a < L::D; ++a) {
          const int e = ecomp<L>(i, a);
          h = A::fma(A::c(e * e - 1.0 / 3.0), Ad[a], h);
        }
#pragma unroll
        for (int o = 0; o < 3; ++o) {
          const int a = o == 2 ? 1 : 0, b = o == 0 ? 1 : 2;
          if (b >= L::D) continue;
          const int eab = ecomp<L>(i, a) * ecomp<L>(i, b);
          if (eab != 0) h = A::fma(A::c(2.0 * eab), Ao[o], h);
        }
        r2[i] = A::mul(A::c(4.5 * L::w(i)), h);
      }
    }

    // ---- antisymmetric relaxation target R3 and post-collision
    V r3[Q];
    if constexpr (L::Q == 27) {
      // D3Q27 TRT-RLB: the seven third-order modes m_ab = e_a (e_b^2 - cs^2)
      // (a != b, norm 2 cs^6) and m_xyz = e_x e_y e_z (norm cs^6) are
      // w-orthogonal on the tensor-product lattice; A_k = sum_i m_k,i fneq_i
      // = sum over pairs of 2 m_k,i nm_i, R3_i = w_i sum_k m_k,i A_k / N_k.
      constexpr int kModes = 7;
      auto mode = [](int k, int i) constexpr -> double {
        if (k == 6) return double(ecomp<L>(i, 0) * ecomp<L>(i, 1) * ecomp<L>(i, 2));
        const int a = k / 2, b = (a + 1 + (k & 1)) % 3;
        const int ea = ecomp<L>(i, a), eb = ecomp<L>(i, b);
        return ea * (eb * eb - 1.0 / 3.0);
      };
      V Am[kModes];
      bool ai[kModes];
#pragma unroll
      for (int k = 0; k < kModes; ++k) {
        Am[k] = A::c(0.0);
        ai[k] = false;
      }
#pragma unroll
      for (int i = 1; i < Q; ++i) {
        if (!is_pair_rep<L>(i)) continue;
#pragma unroll
        for (int k = 0; k < kModes; ++k) {
          const double m = mode(k, i);
          if (m == 0.0) continue;
          Am[k] = ai[k] ? A::fma(A::c(2.0 * m), nm[i], Am[k]) : A::mul(A::c(2.0 * m), nm[i]);
          ai[k] = true;
        }
      }
#pragma unroll
      for (int i = 1; i < Q; ++i) {
        if (!is_pair_rep<L>(i)) continue;
        V h = A::c(0.0);
        bool hi = false;
#pragma unroll
        for (int k = 0; k < kModes; ++k) {
          const double m = mode(k, i);
          if (m == 0.0) continue;
          const double cf = (k == 6 ? 27.0 : 13.5) * L::w(i) * m;
          h = hi ? A::fma(A::c(cf), Am[k], h) : A::mul(A::c(cf), Am[k]);
          hi = true;
        }
        r3[i] = h;
      }
    } else {
      // fneq_i - fneq_ibar = 2 nm_i; modes m_ab = e_a (e_b^2 - cs^2)
      auto mode = [](int a, int b, int i) constexpr -> double {
        const int ea = ecomp<L>(i, a), eb = ecomp<L>(i, b);
        return ea * (eb * eb - 1.0 / 3.0);
      };
      if constexpr (L::D == 2) {
        V Axyy = A::c(0.0), Axxy = A::c(0.0);
        bool i1 = false, i2 = false;
#pragma unroll
        for (int i = 1; i < Q; ++i) {
          if (!is_pair_rep<L>(i)) continue;
          if (mode(0, 1, i) != 0.0) {
            Axyy = i1 ? A::fma(A::c(2.0 * mode(0, 1, i)), nm[i], Axyy) : A::mul(A::c(2.0 * mode(0, 1, i)), nm[i]);
            i1 = true;
          }
          if (mode(1, 0, i) != 0.0) {
            Axxy = i2 ? A::fma(A::c(2.0 * mode(1, 0, i)), nm[i], Axxy) : A::mul(A::c(2.0 * mode(1, 0, i)), nm[i]);
            i2 = true;
          }
        }
#pragma unroll
        for (int i = 1; i < Q; ++i) {
          if (!is_pair_rep<L>(i)) continue;
          V h = A::c(0.0);
          bool hi = false;
          if (mode(0, 1, i) != 0.0) {
            h = A::mul(A::c(13.5 * L::w(i) * mode(0, 1, i)), Axyy);
            hi = true;
          }
          if (mode(1, 0, i) != 0.0)
            h = hi ? A::fma(A::c(13.5 * L::w(i) * mode(1, 0, i)), Axxy, h)
                   : A::mul(A::c(13.5 * L::w(i) * mode(1, 0, i)), Axxy);
          r3[i] = h;
        }
      } else {
        V As[3], Adf[3];
        bool is[3] = {false, false, false}, id[3] = {false, false, false};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          As[a] = A::c(0.0);
          Adf[a] = A::c(0.0);
        }
#pragma unroll
        for (int i = 1; i < Q; ++i) {
          if (!is_pair_rep<L>(i)) continue;
#pragma unroll
          for (int a = 0; a < 3; ++a) {
            const int b = a == 0 ? 1 : 0, cc = a == 2 ? 1 : 2;
            const double sv = mode(a, b, i) + mode(a, cc, i);
            const double dv = mode(a, b, i) - mode(a, cc, i);
            if (sv != 0.0) {
              As[a] = is[a] ? A::fma(A::c(2.0 * sv), nm[i], As[a]) : A::mul(A::c(2.0 * sv), nm[i]);
              is[a] = true;
            }
            if (dv != 0.0) {
              Adf[a] = id[a] ? A::fma(A::c(2.0 * dv), nm[i], Adf[a]) : A::mul(A::c(2.0 * dv), nm[i]);
              id[a] = true;
            }
          }
        }
#pragma unroll
        for (int i = 1; i < Q; ++i) {
          if (!is_pair_rep<L>(i)) continue;
          V h = A::c(0.0);
          bool hi = false;
#pragma unroll
          for (int a = 0; a < 3; ++a) {
            const int b = a == 0 ? 1 : 0, cc = a == 2 ? 1 : 2;
            const double sv = mode(a, b, i) + mode(a, cc, i);
            const double dv = mode(a, b, i) - mode(a, cc, i);
            if (sv != 0.0) {
              h = hi ? A::fma(A::c(13.5 * L::w(i) * sv), As[a], h) : A::mul(A::c(13.5 * L::w(i) * sv), As[a]);
              hi = true;
            }
            if (dv != 0.0) {
              h = hi ? A::fma(A::c(4.5 * L::w(i) * dv), Adf[a], h) : A::mul(A::c(4.5 * L::w(i) * dv), Adf[a]);
              hi = true;
            }
          }
          r3[i] = h;
        }
      }
    }

    // rest: f*_0 = f_eq0 + (1 - w+) R2_0 + S+_0, S+_0 = hg w0 (-3 u.F)
    V g0 = A::fma(A::c(c.cp), r20, feq0);
    if (FORCE) g0 = A::fma(A::c(c.fu[0]), uF, g0);
    g[0] = g0;
#pragma unroll
    for (int i = 1; i < Q; ++i) {
      if (!is_pair_rep<L>(i)) continue;
      V sym = A::fma(A::c(c.cp), r2[i], fs[i]);
      V anti = A::fma(A::c(c.cm), r3[i], fa[i]);
      if (FORCE) {
        // S+_i = hg w (9 eu eF - 3 u.F); antisymmetric force F_i/2 (R3 already
        // carries the first-order part)
        sym = A::fma(A::c(c.fe[i]), edot<L, V>(i, u), sym);
        sym = A::fma(A::c(c.fu[i]), uF, sym);
        anti = A::add(anti, A::c(c.fa[i]));
      }
      g[i] = A::add(sym, anti);
      g[L::opp(i)] = A::sub(sym, anti);
    }
    return badmask;
  }
}

}  // namespace lbm
