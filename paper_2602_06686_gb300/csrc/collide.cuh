// collide.cuh -- per-node collision operators in shifted variables.
//
// Input and output are the shifted populations g_i = f_i - w_i rho0.  The
// operators (arXiv 2602.06686):
//   f* = f_eq + (1 - w+) R2 + (1 - w-) R3 + F_i/2 + (1 - w+/2) S+
//   TRT      R2 = fneq+                        R3 = fneq- + F_i/2
//   P-TRT    R2 = fneq+ - P_G fneq (Eq. PTRT)  R3 = fneq- + F_i/2 (Eq. R3_force)
//   TRT-RLB  R2 = P^(2) fneq, R3 = P^(3) fneq  (Eq. R2R3_hermite as orthogonal projections)
// with rho, u from Eq. macro (half-force velocity), the third-order f_eq of
// Eq. feq written as w [drho + rho (3 eu + 4.5 eu^2 - 1.5 u^2 + 4.5 eu (eu^2 - u^2))]
// (H3_i : uuu = (e_i.u)^3 - 3 cs^2 |u|^2 (e_i.u) on any velocity set),
// F_i = 3 w e_i.F and S+ = w (9 eu eF - 3 u.F).  The force reading keeps the
// first-order term of Sec. 2.2 and the whole Guo source at (1 - w+/2), which
// makes the antisymmetric force content F_i/2 + (1-w-) R3 for every rate.
//
// Everything runs per inversion pair (i, ibar): s = g_i + g_ibar and
// d = g_i - g_ibar give the parity split of Eq. parity for free, and the
// symmetric / antisymmetric post-collision parts combine as
// g*_i = sym + anti, g*_ibar = sym - anti.
//
// Ghost modes (hand-derived, w-orthogonal, integer-scaled values G(k, i)):
//   D2Q9 : phi = (ex^2 - cs^2)(ey^2 - cs^2) = cs^4 G, G = 1 (rest), -2 (axial),
//          4 (diagonal), norm 4 cs^8 (App. A.1, Eq. R2_D2Q9).
//   D3Q19: the printed products (e_a^2 - cs^2)(e_b^2 - cs^2) are neither mutually
//          orthogonal nor orthogonal to H2 on D3Q19; the ghost subspace (the
//          complement of span{1, H2} in the symmetric subspace, Eq. S_decomp) is
//          spanned by phi~_ab = (e_a^2 - cs^2)(e_b^2 - cs^2) + (cs^2/2)(e_c^2 - cs^2)
//          and diagonalised into g_e = phi~_xy + phi~_yz + phi~_zx (norm 9/2 cs^8),
//          g_1 = phi~_xy - phi~_yz (9 cs^8), g_2 = phi~_xy + phi~_yz - 2 phi~_zx
//          (27 cs^8), with values
//              g_e*6: rest 1, axial -2, diagonal 1
//              g_1*2: -x axis pair -1, z pair 1, xy diagonals 1, yz diagonals -1
//              g_2*2: x pair 1, y pair -2, z pair 1, xy 1, yz 1, xz -2.
// P_G fneq = sum_k w_i G(k,i) (s_k^2 / N_k) sum_j G(k,j) fneq_j with s_k the
// scale of G and N_k the norm.
#pragma once
#include "lattice.cuh"

namespace lbm {

enum { C_TRT = 0, C_TRT_RLB = 1, C_P_TRT = 2 };

template <typename R>
struct Coef {
  R rho0;
  R cp;  // 1 - w+
  R cm;  // 1 - w-
  R hg;  // 1 - w+/2
  R F[3];
};

// ---- ghost tables (integer values and s_k^2 / N_k) -----------------------
template <class L>
struct Ghost;

template <>
struct Ghost<D2Q9> {
  static constexpr int NG = 1;
  __host__ __device__ static constexpr int G(int, int i) {
    return i == 0 ? 1 : (i <= 4 ? -2 : 4);
  }
  // s = 1/9 (phi = G/9), N = 4/81 -> s^2/N = 1/4
  __host__ __device__ static constexpr double coef(int) { return 0.25; }
};

template <>
struct Ghost<D3Q19> {
  static constexpr int NG = 3;
  // class of a velocity: 0 rest, 1/2/3 axial along x/y/z, 4 xy, 5 xz, 6 yz diagonal
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
  __host__ __device__ static constexpr double coef(int k) {
    return k == 0 ? 0.5 : (k == 1 ? 2.25 : 0.75);
  }
};

template <class L, int COLL, typename R>
__device__ __forceinline__ void collide(R (&g)[L::Q], const Coef<R>& c, bool& bad) {
  constexpr int Q = L::Q;
  R s[Q], d[Q];  // pair sums / differences at the pair representative
  R drho = g[0];
  R jx = R(0), jy = R(0), jz = R(0);
#pragma unroll
  for (int i = 1; i < Q; ++i) {
    if (!is_pair_rep<L>(i)) continue;
    const int o = L::opp(i);
    s[i] = g[i] + g[o];
    d[i] = g[i] - g[o];
    drho += s[i];
    if (L::cx(i) == 1) jx += d[i];
    if (L::cx(i) == -1) jx -= d[i];
    if (L::cy(i) == 1) jy += d[i];
    if (L::cy(i) == -1) jy -= d[i];
    if (L::cz(i) == 1) jz += d[i];
    if (L::cz(i) == -1) jz -= d[i];
  }
  const R rho = c.rho0 + drho;
  const R inv = R(1) / rho;
  const R ux = (jx + R(0.5) * c.F[0]) * inv;
  const R uy = (jy + R(0.5) * c.F[1]) * inv;
  const R uz = (L::D == 3) ? (jz + R(0.5) * c.F[2]) * inv : R(0);
  const R usq = ux * ux + uy * uy + uz * uz;
  bad = !(rho > R(0)) || !(usq <= R(1));
  const R uF = ux * c.F[0] + uy * c.F[1] + uz * c.F[2];
  const R usq15 = R(1.5) * usq;

  // rest velocity
  const R w0 = R(L::w(0));
  const R feq0 = w0 * (drho - rho * usq15);
  const R np0 = g[0] - feq0;
  R np[Q], nm[Q], fs[Q], fa[Q], src[Q], Fi[Q];
#pragma unroll
  for (int i = 1; i < Q; ++i) {
    if (!is_pair_rep<L>(i)) continue;
    const R w = R(L::w(i));
    const R eu = R(L::cx(i)) * ux + R(L::cy(i)) * uy + R(L::cz(i)) * uz;
    const R eF = R(L::cx(i)) * c.F[0] + R(L::cy(i)) * c.F[1] + R(L::cz(i)) * c.F[2];
    fs[i] = w * (drho + rho * (R(4.5) * eu * eu - usq15));
    fa[i] = w * rho * eu * (R(3) + R(4.5) * (eu * eu - usq));
    np[i] = R(0.5) * s[i] - fs[i];
    nm[i] = R(0.5) * d[i] - fa[i];
    src[i] = c.hg * w * (R(9) * eu * eF - R(3) * uF);
    Fi[i] = R(3) * w * eF;
  }
  const R src0 = c.hg * w0 * (-R(3) * uF);

  // ---- symmetric relaxation target R2 (per pair rep and rest)
  R r2[Q];
  R r20;
  if constexpr (COLL == C_TRT) {
    r20 = np0;
#pragma unroll
    for (int i = 1; i < Q; ++i)
      if (is_pair_rep<L>(i)) r2[i] = np[i];
  } else if constexpr (COLL == C_P_TRT) {
    using Gh = Ghost<L>;
    R m[Gh::NG];
#pragma unroll
    for (int k = 0; k < Gh::NG; ++k) {
      R acc = R(Gh::G(k, 0)) * np0;
#pragma unroll
      for (int i = 1; i < Q; ++i) {
        if (!is_pair_rep<L>(i)) continue;
        if (Gh::G(k, i) != 0) acc += R(2 * Gh::G(k, i)) * np[i];
      }
      m[k] = acc;
    }
    R pg0 = R(0);
#pragma unroll
    for (int k = 0; k < Gh::NG; ++k)
      if (Gh::G(k, 0) != 0) pg0 += R(L::w(0) * Gh::G(k, 0) * Gh::coef(k)) * m[k];
    r20 = np0 - pg0;
#pragma unroll
    for (int i = 1; i < Q; ++i) {
      if (!is_pair_rep<L>(i)) continue;
      R pg = R(0);
#pragma unroll
      for (int k = 0; k < Gh::NG; ++k)
        if (Gh::G(k, i) != 0) pg += R(L::w(i) * Gh::G(k, i) * Gh::coef(k)) * m[k];
      r2[i] = np[i] - pg;
    }
  } else {  // TRT-RLB: orthogonal projection onto span{H2}
    // A2_ab = sum_i (e_a e_b - cs^2 d_ab) fneq_i; fneq_i + fneq_ibar = 2 np_i
    R Axx = R(-1.0 / 3.0) * np0, Ayy = Axx, Azz = Axx, Axy = R(0), Axz = R(0), Ayz = R(0);
#pragma unroll
    for (int i = 1; i < Q; ++i) {
      if (!is_pair_rep<L>(i)) continue;
      const R t = R(2) * np[i];
      Axx += R(L::cx(i) * L::cx(i) - 1.0 / 3.0) * t;
      Ayy += R(L::cy(i) * L::cy(i) - 1.0 / 3.0) * t;
      if (L::D == 3) Azz += R(L::cz(i) * L::cz(i) - 1.0 / 3.0) * t;
      if (L::cx(i) * L::cy(i) != 0) Axy += R(L::cx(i) * L::cy(i)) * t;
      if (L::cx(i) * L::cz(i) != 0) Axz += R(L::cx(i) * L::cz(i)) * t;
      if (L::cy(i) * L::cz(i) != 0) Ayz += R(L::cy(i) * L::cz(i)) * t;
    }
    // R2_i = w_i / (2 cs^4) H2_i : A2 = 4.5 w_i [sum_a H2_aa A_aa + 2 sum_{a<b} e_a e_b A_ab]
    r20 = R(4.5 * L::w(0)) * (R(-1.0 / 3.0) * (Axx + Ayy + (L::D == 3 ? Azz : R(0))));
#pragma unroll
    for (int i = 1; i < Q; ++i) {
      if (!is_pair_rep<L>(i)) continue;
      R h = R(L::cx(i) * L::cx(i) - 1.0 / 3.0) * Axx + R(L::cy(i) * L::cy(i) - 1.0 / 3.0) * Ayy;
      if (L::D == 3) h += R(L::cz(i) * L::cz(i) - 1.0 / 3.0) * Azz;
      if (L::cx(i) * L::cy(i) != 0) h += R(2 * L::cx(i) * L::cy(i)) * Axy;
      if (L::cx(i) * L::cz(i) != 0) h += R(2 * L::cx(i) * L::cz(i)) * Axz;
      if (L::cy(i) * L::cz(i) != 0) h += R(2 * L::cy(i) * L::cz(i)) * Ayz;
      r2[i] = R(4.5 * L::w(i)) * h;
    }
  }

  // ---- antisymmetric relaxation target R3 (per pair rep)
  R r3[Q];
  if constexpr (COLL == C_TRT_RLB) {
    // third-order modes m_ab = e_a (e_b^2 - cs^2); fneq_i - fneq_ibar = 2 nm_i
    auto mode = [](int a, int b, int i) constexpr -> double {
      const int ea = a == 0 ? L::cx(i) : (a == 1 ? L::cy(i) : L::cz(i));
      const int eb = b == 0 ? L::cx(i) : (b == 1 ? L::cy(i) : L::cz(i));
      return ea * (eb * eb - 1.0 / 3.0);
    };
    if constexpr (L::D == 2) {
      // D2Q9: m_xy (xyy) and m_yx (xxy), w-orthogonal, norms 2 cs^6 -> 1/N = 13.5
      R Axyy = R(0), Axxy = R(0);
#pragma unroll
      for (int i = 1; i < Q; ++i) {
        if (!is_pair_rep<L>(i)) continue;
        const R t = R(2) * nm[i];
        if (mode(0, 1, i) != 0.0) Axyy += R(mode(0, 1, i)) * t;
        if (mode(1, 0, i) != 0.0) Axxy += R(mode(1, 0, i)) * t;
      }
#pragma unroll
      for (int i = 1; i < Q; ++i) {
        if (!is_pair_rep<L>(i)) continue;
        R h = R(0);
        if (mode(0, 1, i) != 0.0) h += R(mode(0, 1, i)) * Axyy;
        if (mode(1, 0, i) != 0.0) h += R(mode(1, 0, i)) * Axxy;
        r3[i] = R(13.5 * L::w(i)) * h;
      }
    } else {
      // D3Q19: per odd axis a with the other axes b < c, the modes m_ab and m_ac
      // overlap (<m_ab, m_ac>_w = -cs^6); their sum (norm 2 cs^6) and difference
      // (norm 6 cs^6) are w-orthogonal: 1/N = 13.5 and 4.5.
      R As[3], Ad[3];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        As[a] = R(0);
        Ad[a] = R(0);
      }
#pragma unroll
      for (int i = 1; i < Q; ++i) {
        if (!is_pair_rep<L>(i)) continue;
        const R t = R(2) * nm[i];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          const int b = a == 0 ? 1 : 0, cc = a == 2 ? 1 : 2;
          const double sv = mode(a, b, i) + mode(a, cc, i);
          const double dv = mode(a, b, i) - mode(a, cc, i);
          if (sv != 0.0) As[a] += R(sv) * t;
          if (dv != 0.0) Ad[a] += R(dv) * t;
        }
      }
#pragma unroll
      for (int i = 1; i < Q; ++i) {
        if (!is_pair_rep<L>(i)) continue;
        R h = R(0);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          const int b = a == 0 ? 1 : 0, cc = a == 2 ? 1 : 2;
          const double sv = mode(a, b, i) + mode(a, cc, i);
          const double dv = mode(a, b, i) - mode(a, cc, i);
          if (sv != 0.0) h += R(13.5 * sv) * As[a];
          if (dv != 0.0) h += R(4.5 * dv) * Ad[a];
        }
        r3[i] = R(L::w(i)) * h;
      }
    }
  } else {
#pragma unroll
    for (int i = 1; i < Q; ++i)
      if (is_pair_rep<L>(i)) r3[i] = nm[i] + R(0.5) * Fi[i];
  }

  // ---- post-collision
  g[0] = feq0 + c.cp * r20 + src0;
#pragma unroll
  for (int i = 1; i < Q; ++i) {
    if (!is_pair_rep<L>(i)) continue;
    const R sym = fs[i] + c.cp * r2[i] + src[i];
    const R anti = fa[i] + c.cm * r3[i] + R(0.5) * Fi[i];
    g[i] = sym + anti;
    g[L::opp(i)] = sym - anti;
  }
}

}  // namespace lbm
