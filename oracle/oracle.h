/*
 * Plain FP64 CPU oracle for the periodic treecode force path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may include, link or
 * call this code: only tests/, __graft_entry__.smoke() and bench.py's CPU
 * baseline leg use it.  It shares no code, header or table with the CUDA
 * library under paper_1407_2600_gb300/csrc.
 *
 * Units: unit periodic box (positions in [0,1)), G = 1, accelerations are
 * those of unit-mass sources unless masses are given.  The method is the pure
 * treecode of Sec. 2.1 ("2HOT"): Morton keys, a key-implied oct-tree, a
 * truncated multipole expansion of cells, a multipole acceptance test,
 * grouped sinks and periodic boundaries.
 */
#ifndef ORACLE_H
#define ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- Ewald summation (unit cube, neutralising background) ---------------- */
typedef struct {
  double alpha;  /* splitting parameter */
  double rcut;   /* real-space cutoff on |r - n| */
  int h2max;     /* reciprocal-space cutoff on |h|^2 */
} or_ewald_cfg;

void or_ewald_default(or_ewald_cfg *c);
/* Periodic acceleration at separation r (sink - source) from a unit source,
 * with the uniform neutralising background (Hernquist, Bouchet & Suto 1991). */
void or_ewald_acc(const double r[3], const or_ewald_cfg *c, double a[3]);
/* Periodic potential, zero-mean convention. */
double or_ewald_pot(const double r[3], const or_ewald_cfg *c);
/* Derivatives of the smooth remainder potential
 *   phi~(r) = phi_E(r) + 1/|r| + (2 pi / 3)|r|^2
 * whose field C~ = -grad phi~ = a_E - a_N - (4 pi/3) r is the field of all
 * images n != 0 with the background removed.  out[0] = phi~, out[1..3] =
 * d_i, out[4..9] = d_ij (xx,xy,xz,yy,yz,zz), out[10..19] = d_ijk
 * (xxx,xxy,xxz,xyy,xyz,xzz,yyy,yyz,yzz,zzz). */
void or_phitilde(const double r[3], const or_ewald_cfg *c, double out[20]);

/* All derivatives d^m phi~ with |m| <= P (P <= 9), in multi-index order
 * (order-major; within an order nx descending, then ny descending). */
void or_phitilde_mi(const double r[3], const or_ewald_cfg *c, int P, double *out);
/* Exact phi~ derivatives (|m| <= P) at the lattice nodes (i,j,k) 2^-lg with
 * 0 <= i,j,k <= 2^(lg-1) + 1; nmom(P) values per node. */
int or_phitilde_lattice(int lg, int P, double *tab);
/* Value at a signed lattice point (parity folding). */
void or_phitilde_lattice_get(const double *tab, int lg, int P, const int64_t ir[3], double *out);

/* Accurate tricubic table of C~ only (3 values per node) for the direct
 * oracle; nodes from -h to 1/2 + 2h with h = 1/(2 n1). */
int or_ctilde_table_build(int n1, double *tab /* (n1+4)^3 * 3 */);
void or_ctilde_table_eval(const double *tab, int n1, const double r[3], double out[3]);
/* Same layout for the 6 second derivatives of phi~ (used by the adjoint). */
int or_ctilde_grad_table_build(int n1, double *tab /* (n1+4)^3 * 6 */);
void or_ctilde_grad_table_eval(const double *tab, int n1, const double r[3], double out[6]);

/* ---- softening -------------------------------------------------------------
 * Pair acceleration a_i = m_j (x_j - x_i) f(r) with r = |x_j - x_i|:
 *   kernel 0, Plummer:  f = (r^2 + eps^2)^(-3/2)
 *   kernel 1, Dehnen's compensating K1 kernel (the paper's choice): the field
 *   of the density rho(r) = 105/(64 pi eps^3) (1 - x^2)(5 - 9 x^2), x = r/eps
 *   < 1 (zero beyond), the quadratic F1 kernel 1 - x^2 times the factor that
 *   makes its second moment vanish.  Its enclosed mass is
 *   M(x) = (175/16) x^3 - (147/8) x^5 + (135/16) x^7 (M(1) = 1), so
 *   f = M(x)/r^3 = (175/16 - (147/8) x^2 + (135/16) x^4)/eps^3 for r < eps
 *   and f = 1/r^3 beyond. */
double or_soft_factor(double r2, double eps, int kernel);
/* the softened pair potential (unit masses): Plummer -(r^2 + eps^2)^-1/2;
 * K1 -(105/32 - (175/32) x^2 + (147/32) x^4 - (45/32) x^6)/eps inside eps
 * (the integral of its force), -1/r beyond */
double or_soft_pot(double r2, double eps, int kernel);

/* ---- O1: direct summation with Ewald images --------------------------------
 * a_i = sum_{j != i} m_j [ a_E(r_ij) - a_N(r*_ij) + a_P(r*_ij) ]
 * (Plummer softening for the minimum-image pair only).  ctab == NULL uses the
 * exact Ewald sum per pair; otherwise the tricubic C~ table.  targets == NULL
 * means all particles.  acc is SoA 3 x ntarget. */
int or_direct_forces(int64_t n, const double *pos, const double *mass, double eps,
                     int64_t ntarget, const int64_t *targets, const double *ctab,
                     int n1, double *acc);
/* The same with the softening kernel of or_soft_factor for the minimum-image
 * pair (kernel 0 is or_direct_forces). */
int or_direct_forces_k(int64_t n, const double *pos, const double *mass, double eps, int kernel,
                       int64_t ntarget, const int64_t *targets, const double *ctab, int n1,
                       double *acc);
/* O1's potential (see direct.c); ptab NULL: exact Ewald sum per pair */
int or_direct_pot(int64_t n, const double *pos, const double *mass, double eps, int kernel,
                  int64_t ntarget, const int64_t *targets, const double *ptab, int n1, double *pot);
int or_phitilde_table_build(int n1, double *tab /* (n1+4)^3 */);
void or_phitilde_table_eval(const double *tab, int n1, const double r[3], double *out);
/* Vector-Jacobian product of O1: given lam (3 x n SoA, cotangent of the
 * accelerations of all particles), out = (d a / d x)^T lam (3 x n SoA). */
int or_direct_vjp(int64_t n, const double *pos, const double *mass, double eps,
                  const double *gtab, int n1, const double *lam, double *out);

/* ---- O2: CPU tree ------------------------------------------------------- */
typedef struct {
  double eps;     /* Plummer softening, box units */
  double theta;   /* opening angle */
  int order;      /* multipole order p, 0..4 */
  int n_leaf;     /* a cell with more particles is split */
  int n_group;    /* sinks per group (consecutive in key order) */
  int n_direct;   /* accepted cells with <= n_direct particles use P2P */
  int lmax;       /* deepest level, <= 21 */
  int ewald;      /* 0: no periodic correction; else the order p_E of the
                     per-group local expansion of the image field */
  int ew_level;   /* level of the fixed source cells of the image field */
  int ew_grid;    /* expansion points snap to the lattice 2^-ew_grid */
  int mac;        /* distance d of the opening test: 0 from the cell centre to
                     the group box, 1 from the cell's boundary to the group box */
  int bg;         /* 0, or the highest order q (p < q <= 8) of the uniform
                     background terms: every cell used through its expansion
                     also gets the orders p+1..q of a cube of the mean density
                     filling it, with the Newtonian kernel (the higher moments
                     of the cell's uniform share, which dominate the expansion
                     error of a near-uniform state) */
  int kernel;     /* softening of direct pairs (or_soft_factor): 0 Plummer,
                     1 Dehnen K1.  With K1, whose field is Newtonian beyond
                     eps, cell expansions use the Newtonian kernel 1/|R| */
  int dual;       /* 1: cell-group (dual) interactions.  An accepted cell C
                     of side s_C whose centre lies farther than
                     (s_C + s_G)/theta from the centre z of the group box
                     (largest side s_G; integer units of 2^-23, threshold
                     floor(S^2/theta^2) in IEEE double) is not expanded at
                     every sink: its field joins a local (Taylor) expansion
                     of the group about z, L_k = sum_n ((-1)^|n|/n!) M_n
                     d^(n+k) g(z - c*), 1 <= |k|, |n| + |k| <= p + 1 (the
                     M2P's derivative orders), evaluated once per sink,
                     a_k = sum_{|m| <= p} (x - z)^m/m! L_(m + e_k).  Not with
                     bg. */
  int replicas;   /* W = 1 or 2: periodic images by explicit near replicas
                     and a far-lattice expansion (needs ewald = 0).  The walk
                     visits every cell at each of the (2W+1)^3 images n,
                     |n|_inf <= W, of the box (the acceptance test per image;
                     cells of any level may be accepted), and the images
                     beyond them act
                     through one local expansion of order 8 about the box
                     centre c0: L_k = sum_n ((-1)^|n|/n!) M_n T_(k+n),
                     |k| + |n| <= 8, M the box's moments about c0, T the
                     derivatives at 0 of the far-lattice potential
                     (or_lattice_tensor); a = -sum_{|u| <= 7} d^u/u!
                     L_(u + e_k), potential sum_{|k| <= 8} d^k/k! L_k,
                     d = x - c0. */
} or_tree_params;

/* T_m = d^m Phi_F(0), |m| <= P (P <= 9): the far-lattice potential
 * Phi_F(r) = phi~(r) - (2 pi/3)|r|^2 + sum_{0 < |n|_inf <= W} 1/|r - n|,
 * the periodic potential of a unit mass with the uniform background, less
 * the near images' -1/|r - n|, |n|_inf <= W (multi-index order) */
void or_lattice_tensor(int P, int W, double *T);

/* stats[0] = P2P pair interactions, stats[1] = M2P interactions,
 * stats[2] = Ewald (group, cell) terms, stats[3] = cells, stats[4] = groups walked,
 * stats[5] = sinks walked (every particle of a group that holds a target),
 * stats[6] = cell-group local expansions (dual) */
int or_tree_forces(int64_t n, const double *pos, const double *mass,
                   const or_tree_params *p, const double *tab, int64_t ntarget,
                   const int64_t *targets, double *acc, double *stats);
/* the same with the potential (pot nullable, ntarget values): the tree's
 * -Psi of every interaction (P2P softened, expansions -sum c_n M_n d^n g,
 * the dual form's cells as M2P), the image field's phi~ series and the
 * background's -(2 pi/3) sum m |x - x*|^2 (needs ewald = 0 or >= 2) */
int or_tree_forces_pot(int64_t n, const double *pos, const double *mass,
                       const or_tree_params *p, const double *tab, int64_t ntarget,
                       const int64_t *targets, double *acc, double *pot, double *stats);

/* Tree topology export for structural parity: cell placeholder keys
 * (1 << 3l | prefix), particle ranges, in breadth-first (level, key) order.
 * Returns the number of cells or -(needed) if cap is too small. */
int64_t or_tree_cells(int64_t n, const double *pos, int n_leaf, int lmax, int64_t cap,
                      uint64_t *key, int32_t *level, int64_t *start, int64_t *count);
/* Morton keys (63 bits) and the stable sort permutation. */
void or_morton_keys(int64_t n, const double *pos, uint64_t *keys);
void or_sort_perm(int64_t n, const uint64_t *keys, int64_t *perm);

/* Multipole helpers exposed for pins. */
int or_nmom(int p);
void or_p2m(int64_t n, const double *pos, const double *mass, const double c[3], int p, double *M);
void or_m2m(const double *Mc, const double c[3], const double cp[3], int p, double *Mp);
/* d^m g for |m| <= pmax of g = (|R|^2 + eps^2)^-1/2, Hermite-product form. */
void or_dtensor(const double R[3], double eps, int pmax, double *D);
/* acceleration at R from a cell with moments M (order p), softened */
void or_m2p(const double *M, int p, const double R[3], double eps, double a[3]);
/* the same with only the orders pmin..pmax of M (pmax <= 8) */
void or_m2p_orders(const double *M, int pmin, int pmax, const double R[3], double eps, double a[3]);
/* its potential form Psi = sum_{pmin <= |n| <= pmax} ((-1)^|n|/n!) M_n d^n g(R)
 * (a = grad Psi; the potential is -Psi) */
double or_m2p_pot_orders(const double *M, int pmin, int pmax, const double R[3], double eps);
/* cell-group interaction of the dual form: L (nmom(p + 1) values, index 0
 * unused) += the local expansion about z of a cell's field at R = z - c
 * (orders |n| + |k| <= p + 1), and the acceleration at offset d from z */
void or_m2l(const double *M, int p, const double R[3], double eps, double *L);
void or_l2p(const double *L, int p, const double d[3], double a[3]);
/* moments (order <= p) of a cube of side s and density rho about its centre */
void or_cube_moments(double s, double rho, int p, double *C);

#ifdef __cplusplus
}
#endif
#endif
