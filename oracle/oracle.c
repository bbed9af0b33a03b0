/*
 * oracle.c -- plain, slow, FP64 CPU oracle of the Purified-TRT (P-TRT) lattice
 * Boltzmann update of Yu et al., "Purified Two-Relaxation-Time Lattice Boltzmann
 * Method" (arXiv 2602.06686), with the standard TRT and TRT-RLB comparators and
 * the BGK / RLB single-rate comparators.
 *
 * THIS FILE IS TEST INFRASTRUCTURE.  Only the test suite, the smoke check and
 * the CPU-baseline leg of the benchmark may load it.  The product path (the CUDA
 * library) shares no code, header, table or helper with it.
 *
 * Every table is built generically from its definition:
 *   - Hermite tensors H1, H2, H3 by loops over the velocity components (Eq. Hermite);
 *   - the ghost basis by weighted Gram-Schmidt of the paper's fourth-order products
 *     (e_a^2 - cs^2)(e_b^2 - cs^2) against span{1, H2} and against each other
 *     (Eq. S_decomp, Eq. ghost_proj, App. A.1 / A.2).
 * so that no hand simplification used by a fast kernel is inherited here.
 *
 * Per-node collision (all in FP64, step order of Sec. 2.1 / Eq. PTRT):
 *   1. rho = sum f, j = sum e f, u = (j + F/2)/rho                       (Eq. macro)
 *   2. feq = w rho [1 + H1.u/cs2 + H2:uu/(2cs4) + H3:uuu/(6cs6)]         (Eq. feq)
 *   3. fneq = f - feq,  fneq+- = (fneq_i +- fneq_ibar)/2                  (Eq. fneq_parity)
 *   4. R1 = w H1.A1/cs2 with A1 = sum e fneq (first-order Hermite part; equals -F_i/2)
 *   5. R2: TRT      fneq+
 *          P-TRT    fneq+ - P_G fneq                                      (Eq. PTRT, Thm 2nd)
 *          TRT-RLB  P^(2) fneq, projection onto span{H2}                  (Eq. R2R3_hermite)
 *   6. R3: TRT, P-TRT  fneq- + F_i/2,  F_i = w e.F/cs2                    (Eq. R3_force)
 *          TRT-RLB     P^(3) fneq, projection onto span{H3}               (Eq. R2R3_hermite)
 *   7. f* = feq + (1-w+) R2 + (1-w-) R3 + (1-w+) R1 + (1-w+/2) S_Guo
 *      with S_Guo = w[(e-u).F/cs2 + (e.u)(e.F)/cs4]                       (Eq. source_guo)
 *
 * Readings where the printed equations are not self-consistent (each is checked
 * by a test against what the mathematics fixes):
 *   (a) Eq. PTRT omits the first-order term (1-w+)R1 that Sec. 2.2 assigns to
 *       tau_s1 and that the order-eps CE equation (Eq. order1) carries.  It is kept.
 *   (b) Scheme I (Eq. source_guo) attaches the -u.F/cs2 term to (1 - 1/(2 tau_s2)),
 *       which breaks mass conservation whenever tau_s1 != tau_s2.  The whole Guo
 *       source is taken with (1 - w+/2); together with (a) the antisymmetric force
 *       content of f* is exactly F_i/2 + (1-w-) R3 for every rate, which is the
 *       textbook TRT-Guo scheme split by parity.
 *   (c) The D3Q19 ghost products printed in App. A.2 are neither mutually
 *       orthogonal nor orthogonal to H2; the ghost subspace is taken as the
 *       orthogonal complement of span{1, H2} in the symmetric subspace, which is
 *       what Eq. S_decomp defines, spanned by the orthogonalised products.
 *   (d) On D3Q19 the Hermite contraction w H3:A3/(6cs6) of Eq. R2R3_hermite is
 *       not a projection (H3_xyy and H3_xzz have w-inner product -cs6 there), so
 *       Thm 3rd, whose proof uses the orthogonal projection P^(3), would fail for
 *       it.  The TRT-RLB comparator uses the orthogonal projections P^(2), P^(3),
 *       which coincide with the printed contraction on D2Q9.
 *   (e) The D3Q19 weights and velocity order are not printed; w = 1/3, 1/18, 1/36
 *       (the unique isotropic choice) with the order rest, +-x, +-y, +-z, then the
 *       xy, xz, yz diagonals.
 *
 * Streaming (Sec. 3.3, halfway bounce-back): push f*_i(x) to x + e_i, wrapping
 * periodic axes; if x + e_i is solid or outside a non-periodic axis the
 * population returns to its own node as f_ibar(x, t+1) = f*_i(x).
 *
 * Storage layout of population arrays: f[q][z][y][x], x fastest, FP64, the
 * pre-collision state f(x, t).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_MAXQ 27
#define OR_MAXG 7
#define OR_CS2 (1.0 / 3.0)

enum { OR_D2Q9 = 0, OR_D3Q19 = 1, OR_D3Q27 = 2 };
enum { OR_TRT = 0, OR_TRT_RLB = 1, OR_P_TRT = 2, OR_BGK = 3, OR_RLB = 4 };

typedef struct {
  int D, Q;
  int e[OR_MAXQ][3];
  double w[OR_MAXQ];
  int opp[OR_MAXQ];
  double H1[OR_MAXQ][3];
  double H2[OR_MAXQ][3][3];
  double H3[OR_MAXQ][3][3][3];
  int NG;
  double phi[OR_MAXG][OR_MAXQ]; /* w-orthogonal ghost basis */
  double phinorm[OR_MAXG];      /* sum_i w_i phi_k,i^2 */
  /* w-orthogonal bases of span{H2_ab} and span{H3_abc} on this lattice */
  int n2, n3;
  double b2[6][OR_MAXQ], b2norm[6];
  double b3[10][OR_MAXQ], b3norm[10];
} or_lattice;

/* Parameters of one lattice run.  Layout must match oracle/__init__.py. */
typedef struct {
  int lattice;
  int nx, ny, nz;
  int collision;
  int periodic[3];
  double omega_plus;  /* 1/tau_s1 */
  double omega_minus; /* 1/tau_s2 */
  double force[3];
  const uint8_t* solid; /* nx*ny*nz, nonzero = solid; may be NULL */
} or_params;

/* ---------------------------------------------------------------- lattice */

static double dot_w(const or_lattice* L, const double* a, const double* b) {
  double s = 0.0;
  for (int i = 0; i < L->Q; ++i) s += L->w[i] * a[i] * b[i];
  return s;
}

/* Builds velocities, weights, opposites, Hermite tensors and the ghost basis. */
static int build_lattice(int which, or_lattice* L) {
  memset(L, 0, sizeof(*L));
  if (which == OR_D2Q9) {
    /* Eq. D2Q9: order 0, (1,0), (0,1), (-1,0), (0,-1), (1,1), (-1,1), (-1,-1), (1,-1). */
    static const int ex[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
    static const int ey[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
    L->D = 2;
    L->Q = 9;
    for (int i = 0; i < 9; ++i) {
      L->e[i][0] = ex[i];
      L->e[i][1] = ey[i];
      L->e[i][2] = 0;
      L->w[i] = (i == 0) ? 4.0 / 9.0 : (i <= 4 ? 1.0 / 9.0 : 1.0 / 36.0);
    }
  } else if (which == OR_D3Q19) {
    /* rest; +-x, +-y, +-z; xy (++, --, +-, -+); xz (same pattern); yz (same). */
    static const int v[19][3] = {{0, 0, 0},  {1, 0, 0},   {-1, 0, 0}, {0, 1, 0},   {0, -1, 0},
                                 {0, 0, 1},  {0, 0, -1},  {1, 1, 0},  {-1, -1, 0}, {1, -1, 0},
                                 {-1, 1, 0}, {1, 0, 1},   {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
                                 {0, 1, 1},  {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};
    L->D = 3;
    L->Q = 19;
    for (int i = 0; i < 19; ++i) {
      int n2 = 0;
      for (int a = 0; a < 3; ++a) {
        L->e[i][a] = v[i][a];
        n2 += v[i][a] * v[i][a];
      }
      L->w[i] = (n2 == 0) ? 1.0 / 3.0 : (n2 == 1 ? 1.0 / 18.0 : 1.0 / 36.0);
    }
  } else if (which == OR_D3Q27) {
    /* App. D3Q27: rest; +-x, +-y, +-z; the 12 face diagonals as for D3Q19; the
     * 8 body diagonals in inversion pairs (+++, ---), (++-, --+), (+-+, -+-),
     * (-++, +--).  Weights: products of the D1Q3 weights 2/3 (0) and 1/6 (+-1),
     * i.e. 8/27, 2/27, 1/54, 1/216 (not printed; the tensor-product lattice). */
    static const int v[27][3] = {
        {0, 0, 0},   {1, 0, 0},   {-1, 0, 0},  {0, 1, 0},   {0, -1, 0},  {0, 0, 1},   {0, 0, -1},
        {1, 1, 0},   {-1, -1, 0}, {1, -1, 0},  {-1, 1, 0},  {1, 0, 1},   {-1, 0, -1}, {1, 0, -1},
        {-1, 0, 1},  {0, 1, 1},   {0, -1, -1}, {0, 1, -1},  {0, -1, 1},  {1, 1, 1},   {-1, -1, -1},
        {1, 1, -1},  {-1, -1, 1}, {1, -1, 1},  {-1, 1, -1}, {-1, 1, 1},  {1, -1, -1}};
    L->D = 3;
    L->Q = 27;
    for (int i = 0; i < 27; ++i) {
      double w = 1.0;
      for (int a = 0; a < 3; ++a) {
        L->e[i][a] = v[i][a];
        w *= v[i][a] == 0 ? 2.0 / 3.0 : 1.0 / 6.0;
      }
      L->w[i] = w;
    }
  } else {
    return -1;
  }
  /* Opposite index: e_ibar = -e_i. */
  for (int i = 0; i < L->Q; ++i) {
    L->opp[i] = -1;
    for (int j = 0; j < L->Q; ++j)
      if (L->e[j][0] == -L->e[i][0] && L->e[j][1] == -L->e[i][1] && L->e[j][2] == -L->e[i][2])
        L->opp[i] = j;
    if (L->opp[i] < 0) return -1;
  }
  /* Hermite tensors, Eq. Hermite, over the D active axes. */
  const int D = L->D;
  for (int i = 0; i < L->Q; ++i) {
    const int* e = L->e[i];
    for (int a = 0; a < D; ++a) {
      L->H1[i][a] = e[a];
      for (int b = 0; b < D; ++b) {
        L->H2[i][a][b] = (double)e[a] * e[b] - OR_CS2 * (a == b);
        for (int c = 0; c < D; ++c)
          L->H3[i][a][b][c] = (double)e[a] * e[b] * e[c] -
                              OR_CS2 * (e[a] * (b == c) + e[b] * (c == a) + e[c] * (a == b));
      }
    }
  }
  /* Ghost basis.  Hydrodynamic symmetric modes: 1 and H2_ab (a <= b); build a
   * w-orthogonal basis of their span by modified Gram-Schmidt, then remove that
   * span from each candidate product (e_a^2 - cs2)(e_b^2 - cs2), a < b, and
   * orthogonalise the candidates among themselves. */
  double hyd[1 + 6][OR_MAXQ];
  int nh = 0;
  for (int i = 0; i < L->Q; ++i) hyd[0][i] = 1.0;
  nh = 1;
  for (int a = 0; a < D; ++a)
    for (int b = a; b < D; ++b) {
      for (int i = 0; i < L->Q; ++i) hyd[nh][i] = L->H2[i][a][b];
      ++nh;
    }
  for (int k = 0; k < nh; ++k) {
    for (int m = 0; m < k; ++m) {
      double c = dot_w(L, hyd[k], hyd[m]) / dot_w(L, hyd[m], hyd[m]);
      for (int i = 0; i < L->Q; ++i) hyd[k][i] -= c * hyd[m][i];
    }
  }
  /* Candidates: the fourth-order products for a < b; on D3Q27 also the
   * sixth-order product and the three shear-energy modes of App. D3Q27
   * (G4 = (ex2-cs2)(ey2-cs2)(ez2-cs2)/cs2, G5..G7 = e_a e_b (e_c^2 - cs2)). */
  const int ncand = (D * (D - 1)) / 2 + (L->Q == 27 ? 4 : 0);
  int ng = 0;
  for (int k = 0; k < ncand; ++k) {
      double cand[OR_MAXQ];
      for (int i = 0; i < L->Q; ++i) {
        const double q[3] = {(double)L->e[i][0] * L->e[i][0] - OR_CS2,
                             (double)L->e[i][1] * L->e[i][1] - OR_CS2,
                             (double)L->e[i][2] * L->e[i][2] - OR_CS2};
        if (k < (D * (D - 1)) / 2) {
          const int a = (k < D - 1) ? 0 : 1, b = (k < D - 1) ? k + 1 : 2;
          cand[i] = q[a] * q[b];
        } else if (k == 3) {
          cand[i] = q[0] * q[1] * q[2] / OR_CS2;
        } else {
          const int c = k - 4; /* G5: xy(z), G6: yz(x), G7: zx(y) */
          const int a = c == 0 ? 0 : (c == 1 ? 1 : 2), b = c == 0 ? 1 : (c == 1 ? 2 : 0);
          const int cc = 3 - a - b;
          cand[i] = (double)L->e[i][a] * L->e[i][b] * q[cc];
        }
      }
      for (int m = 0; m < nh; ++m) {
        double c = dot_w(L, cand, hyd[m]) / dot_w(L, hyd[m], hyd[m]);
        for (int i = 0; i < L->Q; ++i) cand[i] -= c * hyd[m][i];
      }
      for (int m = 0; m < ng; ++m) {
        double c = dot_w(L, cand, L->phi[m]) / L->phinorm[m];
        for (int i = 0; i < L->Q; ++i) cand[i] -= c * L->phi[m][i];
      }
      double nrm = dot_w(L, cand, cand);
      if (nrm < 1e-14) return -2; /* dependent candidate: would signal a wrong lattice */
      for (int i = 0; i < L->Q; ++i) L->phi[ng][i] = cand[i];
      L->phinorm[ng] = nrm;
      ++ng;
  }
  L->NG = ng;
  /* Orthogonal bases of the Hermite spans used by the "Hermite projections" of
   * Eq. R2R3_hermite, read as w-orthogonal projections onto span{H2_ab} and
   * span{H3_abc} (the projections P^(2), P^(3) of the proofs of Thm 2nd and
   * Thm 3rd).  Aliased components (H3_xxx, H3_xyz on D3Q19) drop out. */
  L->n2 = 0;
  for (int a = 0; a < D; ++a)
    for (int b = a; b < D; ++b) {
      double v[OR_MAXQ];
      for (int i = 0; i < L->Q; ++i) v[i] = L->H2[i][a][b];
      for (int m = 0; m < L->n2; ++m) {
        double c = dot_w(L, v, L->b2[m]) / L->b2norm[m];
        for (int i = 0; i < L->Q; ++i) v[i] -= c * L->b2[m][i];
      }
      double nrm = dot_w(L, v, v);
      if (nrm < 1e-14) continue;
      for (int i = 0; i < L->Q; ++i) L->b2[L->n2][i] = v[i];
      L->b2norm[L->n2++] = nrm;
    }
  L->n3 = 0;
  for (int a = 0; a < D; ++a)
    for (int b = a; b < D; ++b)
      for (int c = b; c < D; ++c) {
        double v[OR_MAXQ];
        for (int i = 0; i < L->Q; ++i) v[i] = L->H3[i][a][b][c];
        for (int m = 0; m < L->n3; ++m) {
          double k = dot_w(L, v, L->b3[m]) / L->b3norm[m];
          for (int i = 0; i < L->Q; ++i) v[i] -= k * L->b3[m][i];
        }
        double nrm = dot_w(L, v, v);
        if (nrm < 1e-14) continue;
        for (int i = 0; i < L->Q; ++i) L->b3[L->n3][i] = v[i];
        L->b3norm[L->n3++] = nrm;
      }
  return 0;
}

/* w-orthogonal projection of g onto span{basis}: out_i = w_i sum_k b_k,i <b_k, g> / |b_k|^2,
 * where <b, g> = sum_j b_j g_j (g is a population vector, already carrying w). */
static void project(const or_lattice* L, int nb, const double (*b)[OR_MAXQ], const double* bn,
                    const double* g, double* out) {
  for (int i = 0; i < L->Q; ++i) out[i] = 0.0;
  for (int k = 0; k < nb; ++k) {
    double m = 0.0;
    for (int j = 0; j < L->Q; ++j) m += b[k][j] * g[j];
    for (int i = 0; i < L->Q; ++i) out[i] += L->w[i] * b[k][i] / bn[k] * m;
  }
}

/* --------------------------------------------------------------- collision */

/* Eq. feq: third-order Hermite equilibrium. */
static void equilibrium(const or_lattice* L, double rho, const double* u, double* feq) {
  const double cs2 = OR_CS2, cs4 = cs2 * cs2, cs6 = cs4 * cs2;
  const int D = L->D;
  for (int i = 0; i < L->Q; ++i) {
    double t1 = 0.0, t2 = 0.0, t3 = 0.0;
    for (int a = 0; a < D; ++a) {
      t1 += L->H1[i][a] * u[a];
      for (int b = 0; b < D; ++b) {
        t2 += L->H2[i][a][b] * u[a] * u[b];
        for (int c = 0; c < D; ++c) t3 += L->H3[i][a][b][c] * u[a] * u[b] * u[c];
      }
    }
    feq[i] = L->w[i] * rho * (1.0 + t1 / cs2 + t2 / (2.0 * cs4) + t3 / (6.0 * cs6));
  }
}

/* Eq. macro: density and half-force velocity. */
static void moments(const or_lattice* L, const double* F, const double* f, double* rho,
                    double* u) {
  double r = 0.0, j[3] = {0.0, 0.0, 0.0};
  for (int i = 0; i < L->Q; ++i) {
    r += f[i];
    for (int a = 0; a < L->D; ++a) j[a] += L->e[i][a] * f[i];
  }
  *rho = r;
  for (int a = 0; a < 3; ++a) u[a] = (a < L->D) ? (j[a] + 0.5 * F[a]) / r : 0.0;
}

/* (P_G fneq)_i of Eq. ghost_proj with the w-orthogonal ghost basis. */
static void ghost_projection(const or_lattice* L, const double* fneq, double* pg) {
  for (int i = 0; i < L->Q; ++i) pg[i] = 0.0;
  for (int k = 0; k < L->NG; ++k) {
    double sg = 0.0; /* ghost scalar moment S_G,k */
    for (int j = 0; j < L->Q; ++j) sg += L->phi[k][j] * fneq[j];
    for (int i = 0; i < L->Q; ++i) pg[i] += L->w[i] * L->phi[k][i] / L->phinorm[k] * sg;
  }
}

/* One node's collision.  scheme 1: the Guo source (Eq. source_guo, reading (b));
 * scheme 2: the simplified projection source of Eq. source_simple,
 *   S_i = (1 - w+/2) F_i + G_i,
 *   G_i = -(1 - w+/2) w_i H2_i,ab (d_g Phi_abg) / (6 cs6)          (Eq. Gi)
 * with dphi[a][b] = d_g Phi_abg given by the caller (a non-local quantity). */
static void collide_scheme(const or_lattice* L, const or_params* p, const double* f, double* fs,
                           int scheme, const double (*dphi)[3]) {
  const double cs2 = OR_CS2, cs4 = cs2 * cs2;
  const int Q = L->Q, D = L->D;
  const double* F = p->force;
  double wp = p->omega_plus, wm = p->omega_minus;
  if (p->collision == OR_BGK || p->collision == OR_RLB) wm = wp;

  double rho, u[3];
  moments(L, F, f, &rho, u); /* step 1 */
  double feq[OR_MAXQ], fneq[OR_MAXQ], fp[OR_MAXQ], fm[OR_MAXQ];
  equilibrium(L, rho, u, feq); /* step 2 */
  for (int i = 0; i < Q; ++i) fneq[i] = f[i] - feq[i];
  for (int i = 0; i < Q; ++i) { /* step 3 */
    fp[i] = 0.5 * (fneq[i] + fneq[L->opp[i]]);
    fm[i] = 0.5 * (fneq[i] - fneq[L->opp[i]]);
  }

  /* First-order Hermite moment of fneq (R1 = w H1.A1/cs2; A1 = -F/2 by Eq. macro). */
  double A1[3] = {0, 0, 0};
  for (int j = 0; j < Q; ++j)
    for (int a = 0; a < D; ++a) A1[a] += L->H1[j][a] * fneq[j];

  /* Hermite projections of the RLB family: w-orthogonal projections of fneq onto
   * span{H2} and span{H3}.  On D2Q9 (and for H2 on D3Q19) the Hermite components
   * are w-orthogonal with norms 2cs4 / cs4 and 2cs6, so this is the tensor
   * contraction of Eq. R2R3_hermite; on D3Q19 the H3 components H3_xyy and H3_xzz
   * (and the two analogous pairs) overlap, and the projection takes that into
   * account (the literal contraction is oracle_hermite_contraction). */
  double R2h[OR_MAXQ], R3h[OR_MAXQ];
  project(L, L->n2, (const double(*)[OR_MAXQ])L->b2, L->b2norm, fneq, R2h);
  project(L, L->n3, (const double(*)[OR_MAXQ])L->b3, L->b3norm, fneq, R3h);

  double pg[OR_MAXQ];
  ghost_projection(L, fneq, pg);

  double uF = 0.0;
  for (int a = 0; a < D; ++a) uF += u[a] * F[a];

  for (int i = 0; i < Q; ++i) {
    double eu = 0.0, eF = 0.0, h1a1 = 0.0;
    for (int a = 0; a < D; ++a) {
      eu += L->e[i][a] * u[a];
      eF += L->e[i][a] * F[a];
      h1a1 += L->H1[i][a] * A1[a];
    }
    const double w = L->w[i];
    const double Fi = w * eF / cs2;   /* step 4 */
    const double R1 = w * h1a1 / cs2; /* first-order Hermite part */
    const double sguo = w * ((eF - uF) / cs2 + eu * eF / cs4); /* Eq. source_guo, one rate */
    double R2, R3;
    switch (p->collision) {
      case OR_TRT:
      case OR_BGK:
        R2 = fp[i];
        R3 = fm[i] + 0.5 * Fi;
        break;
      case OR_P_TRT:
        if (Q == 27) {
          /* Eq. PTRT_D3Q27, the hybrid: N_G = 7 > M_2 = 6, so the second-order
           * term is the tensor (Hermite) projection, the third-order term the
           * antisymmetric approximation (fifth-order residual kept). */
          R2 = R2h[i];
        } else {
          R2 = fp[i] - pg[i];
        }
        R3 = fm[i] + 0.5 * Fi;
        break;
      case OR_TRT_RLB:
        R2 = R2h[i];
        R3 = R3h[i];
        break;
      case OR_RLB: /* regularised to second order, single rate: no third-order part */
        R2 = R2h[i];
        R3 = 0.0;
        break;
      default:
        R2 = R3 = 0.0;
    }
    if (scheme == 1) {
      fs[i] = feq[i] + (1.0 - wp) * R2 + (1.0 - wm) * R3 + (1.0 - wp) * R1 +
              (1.0 - 0.5 * wp) * sguo;
    } else {
      double h2d = 0.0; /* H2_i : d_g Phi */
      for (int a = 0; a < D; ++a)
        for (int b = 0; b < D; ++b) h2d += L->H2[i][a][b] * dphi[a][b];
      const double Gi = -(1.0 - 0.5 * wp) * w * h2d / (6.0 * cs4 * cs2); /* Eq. Gi */
      fs[i] = feq[i] + (1.0 - wp) * R2 + (1.0 - wm) * R3 + (1.0 - wp) * R1 +
              (1.0 - 0.5 * wp) * Fi + Gi; /* Eq. source_simple */
    }
  }
}

static void collide_node(const or_lattice* L, const or_params* p, const double* f, double* fs) {
  collide_scheme(L, p, f, fs, 1, NULL);
}

/* ------------------------------------------------------------- public API */

int oracle_lattice_info(int lattice, int* D, int* Q, int* NG, int* e /* Q*3 */, double* w,
                        int* opp, double* phi /* NG*Q */, double* phinorm) {
  or_lattice L;
  int rc = build_lattice(lattice, &L);
  if (rc) return rc;
  if (D) *D = L.D;
  if (Q) *Q = L.Q;
  if (NG) *NG = L.NG;
  for (int i = 0; i < L.Q; ++i) {
    if (e)
      for (int a = 0; a < 3; ++a) e[3 * i + a] = L.e[i][a];
    if (w) w[i] = L.w[i];
    if (opp) opp[i] = L.opp[i];
  }
  for (int k = 0; k < L.NG; ++k) {
    if (phinorm) phinorm[k] = L.phinorm[k];
    if (phi)
      for (int i = 0; i < L.Q; ++i) phi[k * L.Q + i] = L.phi[k][i];
  }
  return 0;
}

/* Hermite tensors, full (3-index storage even in 2-D): H2[Q][3][3], H3[Q][3][3][3]. */
int oracle_hermite(int lattice, double* H2, double* H3) {
  or_lattice L;
  int rc = build_lattice(lattice, &L);
  if (rc) return rc;
  for (int i = 0; i < L.Q; ++i)
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) {
        H2[(i * 3 + a) * 3 + b] = L.H2[i][a][b];
        for (int c = 0; c < 3; ++c) H3[((i * 3 + a) * 3 + b) * 3 + c] = L.H3[i][a][b][c];
      }
  return 0;
}

/* Rates from the physical parameters: tau+ = 1/2 + nu/cs2 (Eq. viscosity) and
 * tau- = 1/2 + Lambda/(tau+ - 1/2) (magic parameter, Sec. 3.2).  Exactly one of
 * (nu, tau_plus) and one of (Lambda, tau_minus) must be positive. */
int oracle_rates(double nu, double tau_plus, double Lambda, double tau_minus, double* omega_plus,
                 double* omega_minus) {
  if ((nu > 0) == (tau_plus > 0)) return -1;
  if ((Lambda > 0) == (tau_minus > 0)) return -1;
  double tp = tau_plus > 0 ? tau_plus : 0.5 + nu / OR_CS2;
  if (tp <= 0.5) return -1;
  double tm = tau_minus > 0 ? tau_minus : 0.5 + Lambda / (tp - 0.5);
  if (tm <= 0.5) return -1;
  *omega_plus = 1.0 / tp;
  *omega_minus = 1.0 / tm;
  return 0;
}

int oracle_equilibrium(int lattice, double rho, const double* u3, double* feq) {
  or_lattice L;
  int rc = build_lattice(lattice, &L);
  if (rc) return rc;
  equilibrium(&L, rho, u3, feq);
  return 0;
}

/* One collision at one node: fstar = C(f). */
int oracle_collide(const or_params* p, const double* f, double* fstar) {
  or_lattice L;
  int rc = build_lattice(p->lattice, &L);
  if (rc) return rc;
  collide_node(&L, p, f, fstar);
  return 0;
}

/* Batch of independent node collisions: f and fstar are [n][Q] (node-major). */
int oracle_collide_many(const or_params* p, int n, const double* f, double* fstar) {
  or_lattice L;
  int rc = build_lattice(p->lattice, &L);
  if (rc) return rc;
  for (int k = 0; k < n; ++k) collide_node(&L, p, f + (size_t)k * L.Q, fstar + (size_t)k * L.Q);
  return 0;
}

static size_t nnodes(const or_params* p) { return (size_t)p->nx * p->ny * p->nz; }

/* f = feq(rho, u) on every node; rho [N], u [D][N] (component planes). */
int oracle_init_equilibrium(const or_params* p, const double* rho, const double* u, double* f) {
  or_lattice L;
  int rc = build_lattice(p->lattice, &L);
  if (rc) return rc;
  const size_t N = nnodes(p);
  for (size_t n = 0; n < N; ++n) {
    double uu[3] = {0, 0, 0}, feq[OR_MAXQ];
    for (int a = 0; a < L.D; ++a) uu[a] = u[a * N + n];
    equilibrium(&L, rho[n], uu, feq);
    for (int i = 0; i < L.Q; ++i) f[i * N + n] = feq[i];
  }
  return 0;
}

/* Push-stream the post-collision fs into f (Sec. 3.3): f*_i(x) moves to
 * x + e_i, wrapping periodic axes; a population that would enter a solid node
 * or leave through a non-periodic edge returns to x as f_ibar (halfway
 * bounce-back).  Solid nodes keep their values.  fn is scratch of f's size. */
static void push_stream(const or_lattice* L, const or_params* p, double* f, const double* fs,
                        double* fn) {
  const int Q = L->Q;
  const long nx = p->nx, ny = p->ny, nz = p->nz;
  const size_t N = nnodes(p);
  memcpy(fn, f, sizeof(double) * Q * N); /* solid nodes keep their values */
#pragma omp parallel for schedule(static)
  for (long n = 0; n < (long)N; ++n) {
    if (p->solid && p->solid[n]) continue;
    const long x = n % nx, y = (n / nx) % ny, z = n / (nx * ny);
    for (int i = 0; i < Q; ++i) {
      long d[3] = {x + L->e[i][0], y + L->e[i][1], z + L->e[i][2]};
      const long ext[3] = {nx, ny, nz};
      int bounce = 0;
      for (int a = 0; a < 3; ++a) {
        if (d[a] < 0 || d[a] >= ext[a]) {
          if (p->periodic[a])
            d[a] = (d[a] + ext[a]) % ext[a];
          else
            bounce = 1;
        }
      }
      size_t m = 0;
      if (!bounce) {
        m = (size_t)(d[2] * ny + d[1]) * nx + d[0];
        if (p->solid && p->solid[m]) bounce = 1;
      }
      if (bounce)
        fn[L->opp[i] * N + n] = fs[i * N + n];
      else
        fn[i * N + m] = fs[i * N + n];
    }
  }
  memcpy(f, fn, sizeof(double) * Q * N);
}

/* n time steps: collide every fluid node, then push-stream with bounce-back.
 * f is updated in place ([Q][N]); nthreads <= 0 uses the OpenMP default. */
int oracle_step(const or_params* p, double* f, int nsteps, int nthreads) {
  or_lattice L;
  int rc = build_lattice(p->lattice, &L);
  if (rc) return rc;
  const int Q = L.Q;
  const size_t N = nnodes(p);
  double* fs = (double*)malloc(sizeof(double) * Q * N);
  double* fn = (double*)malloc(sizeof(double) * Q * N);
  if (!fs || !fn) {
    free(fs);
    free(fn);
    return -3;
  }
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#else
  (void)nthreads;
#endif
  for (int s = 0; s < nsteps; ++s) {
#pragma omp parallel for schedule(static)
    for (long n = 0; n < (long)N; ++n) {
      double fl[OR_MAXQ], fo[OR_MAXQ];
      if (p->solid && p->solid[n]) {
        for (int i = 0; i < Q; ++i) fs[i * N + n] = f[i * N + n];
        continue;
      }
      for (int i = 0; i < Q; ++i) fl[i] = f[i * N + n];
      collide_node(&L, p, fl, fo);
      for (int i = 0; i < Q; ++i) fs[i * N + n] = fo[i];
    }
    push_stream(&L, p, f, fs, fn);
  }
  free(fs);
  free(fn);
  return 0;
}

/* ------------------------------- Scheme II forcing (Eq. source_simple, Eq. Gi)
 * The cubic-velocity correction G_i needs d_g Phi_abg, where Phi is zero but
 * for Phi_aaa = rho u_a^3 (on D3Q19 also Phi_zzz = rho u_z^3, the same defect
 * of the third moment of f_eq along the third axis).  Its only non-zero
 * entries are therefore d_a Phi_aaa, one per axis.  The paper does not say how
 * the derivative is taken; the reading here: at time t, from the pre-collision
 * rho and half-force u (Eq. macro) of the fluid nodes, by second-order central
 * differences along axis a, (Phi(x + e_a) - Phi(x - e_a)) / 2, where a
 * neighbour across a periodic axis wraps; where one neighbour is solid or
 * beyond a non-periodic edge, the one-sided first-order difference with the
 * other; where both are, zero. */

/* phi [D][N]: rho u_a^3 at every fluid node, 0 on solid nodes. */
static void cubic_flux(const or_lattice* L, const or_params* p, const double* f, double* phi) {
  const size_t N = nnodes(p);
  for (size_t n = 0; n < N; ++n) {
    double fl[OR_MAXQ], rho, u[3];
    if (p->solid && p->solid[n]) {
      for (int a = 0; a < L->D; ++a) phi[a * N + n] = 0.0;
      continue;
    }
    for (int i = 0; i < L->Q; ++i) fl[i] = f[i * N + n];
    moments(L, p->force, fl, &rho, u);
    for (int a = 0; a < L->D; ++a) phi[a * N + n] = rho * u[a] * u[a] * u[a];
  }
}

/* dphi [D][N]: d_a Phi_aaa at every fluid node (the reading above), 0 on solids. */
static void cubic_flux_gradient(const or_lattice* L, const or_params* p, const double* phi,
                                double* dphi) {
  const long nx = p->nx, ny = p->ny, nz = p->nz;
  const long ext[3] = {nx, ny, nz};
  const size_t N = nnodes(p);
  for (size_t n = 0; n < N; ++n) {
    const int solid = p->solid && p->solid[n];
    const long c[3] = {(long)(n % nx), (long)((n / nx) % ny), (long)(n / (nx * ny))};
    for (int a = 0; a < L->D; ++a) {
      if (solid) {
        dphi[a * N + n] = 0.0;
        continue;
      }
      double v[2];
      int ok[2];
      for (int s = 0; s < 2; ++s) {
        long q[3] = {c[0], c[1], c[2]};
        q[a] += s ? 1 : -1;
        ok[s] = 1;
        if (q[a] < 0 || q[a] >= ext[a]) {
          if (p->periodic[a])
            q[a] = (q[a] + ext[a]) % ext[a];
          else
            ok[s] = 0;
        }
        const size_t m = ok[s] ? (size_t)(q[2] * ny + q[1]) * nx + q[0] : 0;
        if (ok[s] && p->solid && p->solid[m]) ok[s] = 0;
        v[s] = ok[s] ? phi[a * N + m] : 0.0;
      }
      const double here = phi[a * N + n];
      double d = 0.0;
      if (ok[0] && ok[1])
        d = 0.5 * (v[1] - v[0]);
      else if (ok[1])
        d = v[1] - here;
      else if (ok[0])
        d = here - v[0];
      dphi[a * N + n] = d;
    }
  }
}

/* dphi [D][N] = d_a Phi_aaa of the pre-collision state f (for tests). */
int oracle_cubic_flux_gradient(const or_params* p, const double* f, double* dphi) {
  or_lattice L;
  int rc = build_lattice(p->lattice, &L);
  if (rc) return rc;
  const size_t N = nnodes(p);
  double* phi = (double*)malloc(sizeof(double) * L.D * N);
  if (!phi) return -3;
  cubic_flux(&L, p, f, phi);
  cubic_flux_gradient(&L, p, phi, dphi);
  free(phi);
  return 0;
}

/* One node's collision with the Scheme II source, dphi[3][3] = d_g Phi_abg. */
int oracle_collide_s2(const or_params* p, const double* f, const double* dphi, double* fstar) {
  or_lattice L;
  int rc = build_lattice(p->lattice, &L);
  if (rc) return rc;
  double t[3][3];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) t[a][b] = dphi[3 * a + b];
  collide_scheme(&L, p, f, fstar, 2, (const double(*)[3])t);
  return 0;
}

/* n time steps with the Scheme II source: Phi and its gradient from the
 * pre-collision state, then collide every fluid node and push-stream as
 * oracle_step. */
int oracle_step_s2(const or_params* p, double* f, int nsteps, int nthreads) {
  or_lattice L;
  int rc = build_lattice(p->lattice, &L);
  if (rc) return rc;
  const int Q = L.Q, D = L.D;
  const size_t N = nnodes(p);
  double* fs = (double*)malloc(sizeof(double) * Q * N);
  double* fn = (double*)malloc(sizeof(double) * Q * N);
  double* phi = (double*)malloc(sizeof(double) * D * N);
  double* dphi = (double*)malloc(sizeof(double) * D * N);
  if (!fs || !fn || !phi || !dphi) {
    free(fs);
    free(fn);
    free(phi);
    free(dphi);
    return -3;
  }
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#else
  (void)nthreads;
#endif
  for (int s = 0; s < nsteps; ++s) {
    cubic_flux(&L, p, f, phi);
    cubic_flux_gradient(&L, p, phi, dphi);
#pragma omp parallel for schedule(static)
    for (long n = 0; n < (long)N; ++n) {
      double fl[OR_MAXQ], fo[OR_MAXQ], t[3][3] = {{0}};
      if (p->solid && p->solid[n]) {
        for (int i = 0; i < Q; ++i) fs[i * N + n] = f[i * N + n];
        continue;
      }
      for (int i = 0; i < Q; ++i) fl[i] = f[i * N + n];
      for (int a = 0; a < D; ++a) t[a][a] = dphi[a * N + n];
      collide_scheme(&L, p, fl, fo, 2, (const double(*)[3])t);
      for (int i = 0; i < Q; ++i) fs[i * N + n] = fo[i];
    }
    push_stream(&L, p, f, fs, fn);
  }
  free(fs);
  free(fn);
  free(phi);
  free(dphi);
  return 0;
}

/* ------------------------------------------------ open boundaries (Sec. 3.4)
 * The square-cylinder benchmark of Sec. 3.4 on D2Q9: the left boundary imposes
 * the uniform velocity u_in by halfway bounce-back from a wall moving with
 * (u_in, 0), half a spacing left of x = 0:
 *   f_ibar(x, t+1) = f*_i(x, t) - 2 w_i rho_w (e_i . u_w) / cs^2
 * for every population f*_i leaving through it; the right boundary is a
 * constant-pressure outlet by the Zou-He scheme at the nodes x = nx - 1: after
 * streaming, the three populations that would enter from outside (e_x = -1) are
 * set so that the node has density rho_out and zero transverse velocity,
 *   u_x = (sum_{e_x = 0} f + 2 sum_{e_x = +1} f) / rho_out - 1,
 *   f_i = f_ibar + 2 w_i rho_out (e_i . u) / cs^2 - (e_iy / 2)(f_{+y} - f_{-y}),
 * which also keeps the non-equilibrium part of the normal pair antisymmetric.
 * y (and z) follow p->periodic; x must be non-periodic.  Plain and node by node:
 * collide every fluid node, push-stream as oracle_step, then the outlet. */
static int zou_he_outlet(const or_lattice* L, double rho_out, double* f /* Q values */) {
  double s0 = 0.0, sp = 0.0, fyp = 0.0, fym = 0.0;
  for (int i = 0; i < L->Q; ++i) {
    if (L->e[i][0] == 0) s0 += f[i];
    if (L->e[i][0] == 1) sp += f[i];
    if (L->e[i][0] == 0 && L->e[i][1] == 1) fyp = f[i];
    if (L->e[i][0] == 0 && L->e[i][1] == -1) fym = f[i];
  }
  const double ux = (s0 + 2.0 * sp) / rho_out - 1.0;
  for (int i = 0; i < L->Q; ++i) {
    if (L->e[i][0] != -1) continue;
    const double eu = L->e[i][0] * ux;
    f[i] = f[L->opp[i]] + 2.0 * L->w[i] * rho_out * eu / OR_CS2 - 0.5 * L->e[i][1] * (fyp - fym);
  }
  return 0;
}

int oracle_step_open(const or_params* p, double u_in, double rho_w, double rho_out, double* f,
                     int nsteps, int nthreads) {
  or_lattice L;
  int rc = build_lattice(p->lattice, &L);
  if (rc) return rc;
  if (p->lattice != OR_D2Q9 || p->periodic[0] || p->nx < 2 || !(rho_out > 0.0)) return -4;
  const int Q = L.Q;
  const long nx = p->nx, ny = p->ny, nz = p->nz;
  const size_t N = nnodes(p);
  double* fs = (double*)malloc(sizeof(double) * Q * N);
  double* fn = (double*)malloc(sizeof(double) * Q * N);
  if (!fs || !fn) {
    free(fs);
    free(fn);
    return -3;
  }
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#else
  (void)nthreads;
#endif
  for (int s = 0; s < nsteps; ++s) {
#pragma omp parallel for schedule(static)
    for (long n = 0; n < (long)N; ++n) {
      double fl[OR_MAXQ], fo[OR_MAXQ];
      if (p->solid && p->solid[n]) {
        for (int i = 0; i < Q; ++i) fs[i * N + n] = f[i * N + n];
        continue;
      }
      for (int i = 0; i < Q; ++i) fl[i] = f[i * N + n];
      collide_node(&L, p, fl, fo);
      for (int i = 0; i < Q; ++i) fs[i * N + n] = fo[i];
    }
    memcpy(fn, f, sizeof(double) * Q * N);
#pragma omp parallel for schedule(static)
    for (long n = 0; n < (long)N; ++n) {
      if (p->solid && p->solid[n]) continue;
      const long x = n % nx, y = (n / nx) % ny, z = n / (nx * ny);
      for (int i = 0; i < Q; ++i) {
        long d[3] = {x + L.e[i][0], y + L.e[i][1], z + L.e[i][2]};
        const long ext[3] = {nx, ny, nz};
        int bounce = 0, inlet = 0;
        for (int a = 0; a < 3; ++a) {
          if (d[a] < 0 || d[a] >= ext[a]) {
            if (p->periodic[a]) {
              d[a] = (d[a] + ext[a]) % ext[a];
            } else {
              bounce = 1;
              if (a == 0 && d[0] < 0) inlet = 1;
            }
          }
        }
        size_t m = 0;
        if (!bounce) {
          m = (size_t)(d[2] * ny + d[1]) * nx + d[0];
          if (p->solid && p->solid[m]) bounce = 1;
        }
        if (bounce) {
          double v = fs[i * N + n];
          if (inlet) v -= 2.0 * L.w[i] * rho_w * (L.e[i][0] * u_in) / OR_CS2; /* moving wall */
          fn[L.opp[i] * N + n] = v;
        } else {
          fn[i * N + m] = fs[i * N + n];
        }
      }
    }
    /* outlet: the populations entering from outside, by Zou-He */
#pragma omp parallel for schedule(static)
    for (long r = 0; r < ny * nz; ++r) {
      const size_t n = (size_t)r * nx + (nx - 1);
      if (p->solid && p->solid[n]) continue;
      double fl[OR_MAXQ];
      for (int i = 0; i < Q; ++i) fl[i] = fn[i * N + n];
      zou_he_outlet(&L, rho_out, fl);
      for (int i = 0; i < Q; ++i) fn[i * N + n] = fl[i];
    }
    memcpy(f, fn, sizeof(double) * Q * N);
  }
  free(fs);
  free(fn);
  return 0;
}

/* Force on the solid nodes by momentum exchange (Sec. 3.4): with halfway
 * bounce-back from resting solid nodes, every link from a fluid node x_f to a
 * solid neighbour x_f + e_i returns f*_i(x_f) as f_ibar(x_f), so the link
 * transfers 2 e_i f*_i(x_f, t); f*(t) is the collision of the given
 * pre-collision state f(t).  out[3]: the force summed over all such links. */
int oracle_momentum_exchange(const or_params* p, const double* f, double* out) {
  or_lattice L;
  int rc = build_lattice(p->lattice, &L);
  if (rc) return rc;
  const long nx = p->nx, ny = p->ny, nz = p->nz;
  const size_t N = nnodes(p);
  out[0] = out[1] = out[2] = 0.0;
  if (!p->solid) return 0;
  for (size_t n = 0; n < N; ++n) {
    if (p->solid[n]) continue;
    const long x = n % nx, y = (n / nx) % ny, z = n / (nx * ny);
    int near = 0;
    size_t nb[OR_MAXQ];
    for (int i = 0; i < L.Q; ++i) {
      long d[3] = {x + L.e[i][0], y + L.e[i][1], z + L.e[i][2]};
      const long ext[3] = {nx, ny, nz};
      int out_of = 0;
      for (int a = 0; a < 3; ++a) {
        if (d[a] < 0 || d[a] >= ext[a]) {
          if (p->periodic[a]) d[a] = (d[a] + ext[a]) % ext[a];
          else out_of = 1;
        }
      }
      nb[i] = out_of ? (size_t)-1 : (size_t)(d[2] * ny + d[1]) * nx + d[0];
      if (!out_of && p->solid[nb[i]]) near = 1;
    }
    if (!near) continue;
    double fl[OR_MAXQ], fo[OR_MAXQ];
    for (int i = 0; i < L.Q; ++i) fl[i] = f[i * N + n];
    collide_node(&L, p, fl, fo);
    for (int i = 0; i < L.Q; ++i) {
      if (nb[i] == (size_t)-1 || !p->solid[nb[i]]) continue;
      for (int a = 0; a < 3; ++a) out[a] += 2.0 * L.e[i][a] * fo[i];
    }
  }
  return 0;
}

/* Density and half-force velocity (Eq. macro) of the pre-collision state. */
int oracle_macros(const or_params* p, const double* f, double* rho, double* u) {
  or_lattice L;
  int rc = build_lattice(p->lattice, &L);
  if (rc) return rc;
  const size_t N = nnodes(p);
  for (size_t n = 0; n < N; ++n) {
    double fl[OR_MAXQ], r, uu[3];
    for (int i = 0; i < L.Q; ++i) fl[i] = f[i * N + n];
    moments(&L, p->force, fl, &r, uu);
    rho[n] = r;
    for (int a = 0; a < L.D; ++a) u[a * N + n] = uu[a];
  }
  return 0;
}

/* Integral diagnostics over fluid nodes, FP64:
 *   out[0] mass = sum rho, out[1..3] momentum = sum rho u (half-force u),
 *   out[4] kinetic energy = 1/2 sum rho |u|^2,
 *   out[5] enstrophy = 1/2 sum |curl u|^2, second-order central differences;
 *          the neighbour across a periodic axis wraps, across a non-periodic edge
 *          or on a solid node it counts as velocity 0,
 *   out[6] 1 if any rho or u is NaN/Inf or rho <= 0, else 0. */
int oracle_diagnostics(const or_params* p, const double* f, double* out) {
  or_lattice L;
  int rc = build_lattice(p->lattice, &L);
  if (rc) return rc;
  const long nx = p->nx, ny = p->ny, nz = p->nz;
  const size_t N = nnodes(p);
  double* rho = (double*)malloc(sizeof(double) * N);
  double* u = (double*)malloc(sizeof(double) * 3 * N);
  if (!rho || !u) {
    free(rho);
    free(u);
    return -3;
  }
  for (size_t k = 0; k < 3 * N; ++k) u[k] = 0.0;
  oracle_macros(p, f, rho, u);
  double mass = 0, mom[3] = {0, 0, 0}, ke = 0, ens = 0, bad = 0;
  const long ext[3] = {nx, ny, nz};
  for (size_t n = 0; n < N; ++n) {
    if (p->solid && p->solid[n]) continue;
    const long x = n % nx, y = (n / nx) % ny, z = n / (nx * ny);
    const long c[3] = {x, y, z};
    double u2 = 0;
    if (!isfinite(rho[n]) || rho[n] <= 0) bad = 1;
    for (int a = 0; a < 3; ++a) {
      if (!isfinite(u[a * N + n])) bad = 1;
      mom[a] += rho[n] * u[a * N + n];
      u2 += u[a * N + n] * u[a * N + n];
    }
    mass += rho[n];
    ke += 0.5 * rho[n] * u2;
    /* du[a][b] = d u_a / d x_b */
    double du[3][3] = {{0}};
    for (int b = 0; b < L.D; ++b) {
      double val[2][3];
      for (int s = 0; s < 2; ++s) {
        long q[3] = {c[0], c[1], c[2]};
        q[b] += s ? 1 : -1;
        int zero = 0;
        if (q[b] < 0 || q[b] >= ext[b]) {
          if (p->periodic[b])
            q[b] = (q[b] + ext[b]) % ext[b];
          else
            zero = 1;
        }
        size_t m = zero ? 0 : (size_t)(q[2] * ny + q[1]) * nx + q[0];
        if (!zero && p->solid && p->solid[m]) zero = 1;
        for (int a = 0; a < 3; ++a) val[s][a] = zero ? 0.0 : u[a * N + m];
      }
      for (int a = 0; a < 3; ++a) du[a][b] = 0.5 * (val[1][a] - val[0][a]);
    }
    const double wx = du[2][1] - du[1][2], wy = du[0][2] - du[2][0], wz = du[1][0] - du[0][1];
    ens += 0.5 * (wx * wx + wy * wy + wz * wz);
  }
  out[0] = mass;
  out[1] = mom[0];
  out[2] = mom[1];
  out[3] = mom[2];
  out[4] = ke;
  out[5] = ens;
  out[6] = bad;
  free(rho);
  free(u);
  return 0;
}

/* Relative L2 norm of Sec. 3: sqrt(sum (qn - qa)^2 / sum qa^2). */
double oracle_l2(long n, const double* qn, const double* qa) {
  double num = 0, den = 0;
  for (long k = 0; k < n; ++k) {
    num += (qn[k] - qa[k]) * (qn[k] - qa[k]);
    den += qa[k] * qa[k];
  }
  return sqrt(num / den);
}

/* P^(5) g on D3Q27 (App. D3Q27): the w-orthogonal projection onto the three
 * fifth-order antisymmetric modes psi^(5,x) = e_x (e_y^2 - cs2)(e_z^2 - cs2) and
 * its cyclic permutations, the part of fneq- outside span{H1, H3}.  For tests. */
int oracle_fifth_order_projection(int lattice, const double* g, double* out) {
  or_lattice L;
  int rc = build_lattice(lattice, &L);
  if (rc) return rc;
  if (L.Q != 27) return -4;
  double psi[3][OR_MAXQ], nrm[3];
  for (int a = 0; a < 3; ++a) {
    const int b = (a + 1) % 3, c = (a + 2) % 3;
    for (int i = 0; i < L.Q; ++i)
      psi[a][i] = L.e[i][a] * ((double)L.e[i][b] * L.e[i][b] - OR_CS2) *
                  ((double)L.e[i][c] * L.e[i][c] - OR_CS2);
    nrm[a] = dot_w(&L, psi[a], psi[a]);
  }
  project(&L, 3, (const double(*)[OR_MAXQ])psi, nrm, g, out);
  return 0;
}

/* The literal Hermite contractions of Eq. R2R3_hermite, for tests only:
 * r2 = w H2:A2/(2cs4), r3 = w H3:A3/(6cs6) with A_n = sum_j H_n,j g_j. */
int oracle_hermite_contraction(int lattice, const double* g, double* r2, double* r3) {
  or_lattice L;
  int rc = build_lattice(lattice, &L);
  if (rc) return rc;
  const double cs2 = OR_CS2, cs4 = cs2 * cs2, cs6 = cs4 * cs2;
  const int D = L.D, Q = L.Q;
  double A2[3][3] = {{0}}, A3[3][3][3] = {{{0}}};
  for (int j = 0; j < Q; ++j)
    for (int a = 0; a < D; ++a)
      for (int b = 0; b < D; ++b) {
        A2[a][b] += L.H2[j][a][b] * g[j];
        for (int c = 0; c < D; ++c) A3[a][b][c] += L.H3[j][a][b][c] * g[j];
      }
  for (int i = 0; i < Q; ++i) {
    double h2 = 0.0, h3 = 0.0;
    for (int a = 0; a < D; ++a)
      for (int b = 0; b < D; ++b) {
        h2 += L.H2[i][a][b] * A2[a][b];
        for (int c = 0; c < D; ++c) h3 += L.H3[i][a][b][c] * A3[a][b][c];
      }
    r2[i] = L.w[i] * h2 / (2.0 * cs4);
    r3[i] = L.w[i] * h3 / (6.0 * cs6);
  }
  return 0;
}

/* Number of independent Hermite modes of order 2 and 3 on the lattice (the
 * ranks of span{H2_ab} and span{H3_abc}). */
int oracle_hermite_ranks(int lattice, int* n2, int* n3) {
  or_lattice L;
  int rc = build_lattice(lattice, &L);
  if (rc) return rc;
  *n2 = L.n2;
  *n3 = L.n3;
  return 0;
}
