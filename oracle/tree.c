/*
 * Oracle O2: plain FP64 CPU treecode (TEST INFRASTRUCTURE ONLY; see oracle.h).
 *
 * Written from Sec. 2.1: particles get a Morton key (the key order maps space
 * to a line with locality), the keys imply the oct-tree (a cell is a key
 * prefix, its parent and daughters follow by bit operations), cells carry a
 * truncated multipole expansion so that one interaction replaces many bodies,
 * a multipole acceptance test decides between the expansion and opening the
 * cell, sinks are bundled into groups that share one interaction list, and
 * the cells near the leaves are handled by direct (particle-particle) sums.
 * The concrete definitions used here (readings of a paper that gives no
 * formulas) are:
 *
 *  keys     q_d = floor(x_d 2^21) mod 2^21, bit b of q_x/q_y/q_z goes to key
 *           bit 3b/3b+1/3b+2; a stable sort orders equal keys by index.
 *  tree     a cell with more than n_leaf particles and level < lmax is split
 *           into its non-empty octants.
 *  groups   runs of at most n_group consecutive particles in key order that
 *           never straddle a level-(ew_grid-1) cell; the group box is the
 *           integer bounding box of the particles' quantised cells.
 *  MAC      integer units of 2^-23: d2 = squared distance from the cell
 *           centre to the nearest image of the group box; a cell of level
 *           l >= 2 is accepted iff d2 > floor(s*s/(theta*theta)), s = 2^(23-l).
 *  images   every particle is used at the image of its level-ew_level
 *           ancestor cell nearest e, the centre of the group's
 *           level-(ew_grid-1) cell; a cell above that level is accepted only
 *           if all its level-ew_level descendants share one image (else it is
 *           opened), and the MAC distance uses that image.
 *  M2P      a_k = sum_{|n|<=p} ((-1)^|n|/n!) M_n d^{n+e_k} g(R), R = x - c*,
 *           g = (|R|^2 + eps^2)^-1/2, moments about the geometric centre.
 *  background (bg = q > p) a cell used through its expansion also adds the
 *           orders p+1..q of a_k for the moments C_n of a cube of the mean
 *           density (total mass / unit volume) filling the cell, with the
 *           Newtonian kernel g = 1/|R|: the truncation error of the uniform
 *           share of every cell, which is what subtracting the uniform
 *           background from every cell (and summing it exactly) removes.
 *  P2P      a += m_j r f(|r|), r = x_j* - x_i, j != i, f the softening of
 *           or_soft_factor: Plummer (|r|^2 + eps^2)^(-3/2), or Dehnen's K1
 *           kernel (kernel = 1), whose field is Newtonian beyond eps; with K1
 *           the cell expansions use the Newtonian kernel (eps = 0 in M2P).
 *  periodic a_E(r) = a_N(r) + (4 pi/3) r + C~(r) for any image r; the walk sums
 *           the Newton/Plummer part, the background term is summed exactly
 *           and the image field sum_j m_j C~(x_i - x_j*) = -grad sum_j m_j
 *           phi~(x_i - x_j*) is a per-group local expansion of order p_E about
 *           e (the centre of the group's level-(ew_grid-1) cell, a point of
 *           the lattice 2^-ew_grid) built from the moments of
 *           the fixed level-ew_level cells C at R0 = e - c*_C (exact Ewald
 *           derivatives of phi~ at lattice points), truncated at total order
 *           p_E + 1 in the potential.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "oracle.h"

static const double PI = 3.14159265358979323846264338327950288;
#define QBITS 21

/* ---- multi-index helpers --------------------------------------------------- */
int or_nmom(int p) { return (p + 1) * (p + 2) * (p + 3) / 6; }

static int mi_idx(int nx, int ny, int nz) {
  int o = nx + ny + nz, j = ny + nz;
  return o * (o + 1) * (o + 2) / 6 + j * (j + 1) / 2 + nz;
}

static void mi_list(int p, int (*L)[3]) {
  for (int o = 0; o <= p; o++)
    for (int nx = o; nx >= 0; nx--)
      for (int ny = o - nx; ny >= 0; ny--) {
        int nz = o - nx - ny;
        int id = mi_idx(nx, ny, nz);
        L[id][0] = nx;
        L[id][1] = ny;
        L[id][2] = nz;
      }
}

static double fact(int n) {
  double f = 1.0;
  for (int i = 2; i <= n; i++) f *= i;
  return f;
}

static double ipow(double x, int k) {
  double r = 1.0;
  for (int i = 0; i < k; i++) r *= x;
  return r;
}

void or_p2m(int64_t n, const double *pos, const double *mass, const double c[3], int p,
            double *M) {
  int nm = or_nmom(p);
  int (*L)[3] = malloc(sizeof(int[3]) * nm);
  mi_list(p, L);
  for (int t = 0; t < nm; t++) M[t] = 0.0;
  for (int64_t j = 0; j < n; j++) {
    double d[3] = {pos[j] - c[0], pos[n + j] - c[1], pos[2 * n + j] - c[2]};
    for (int t = 0; t < nm; t++)
      M[t] += mass[j] * ipow(d[0], L[t][0]) * ipow(d[1], L[t][1]) * ipow(d[2], L[t][2]);
  }
  free(L);
}

static double binom(int n, int k) { return fact(n) / (fact(k) * fact(n - k)); }

/* M_n(cp) = sum_{k <= n} C(n,k) (c - cp)^(n-k) M_k(c) */
void or_m2m(const double *Mc, const double c[3], const double cp[3], int p, double *Mp) {
  int nm = or_nmom(p);
  int (*L)[3] = malloc(sizeof(int[3]) * nm);
  mi_list(p, L);
  double s[3] = {c[0] - cp[0], c[1] - cp[1], c[2] - cp[2]};
  for (int t = 0; t < nm; t++) {
    double v = 0.0;
    for (int kx = 0; kx <= L[t][0]; kx++)
      for (int ky = 0; ky <= L[t][1]; ky++)
        for (int kz = 0; kz <= L[t][2]; kz++) {
          double b = binom(L[t][0], kx) * binom(L[t][1], ky) * binom(L[t][2], kz);
          v += b * ipow(s[0], L[t][0] - kx) * ipow(s[1], L[t][1] - ky) *
               ipow(s[2], L[t][2] - kz) * Mc[mi_idx(kx, ky, kz)];
        }
    Mp[t] = v;
  }
  free(L);
}

/* d^m g, |m| <= pmax, g(R) = (|R|^2+eps^2)^-1/2, explicit Hermite-product form:
 *   d^m g = sum_{k <= m/2} prod_d [m_d! / (k_d! (m_d - 2k_d)! 2^k_d)] R^(m-2k) F_{|m|-|k|}
 *   F_j = 2^j f^(j)(s) = (-1)^j (2j-1)!! s^(-1/2-j),  s = |R|^2 + eps^2.
 * The term list is enumerated once (orders <= 9). */
#define DT_PMAX 9
typedef struct {
  double cf;
  int e[3], j;
} hterm;
static hterm g_ht[4096];
static int g_hbeg[256], g_hend[256];
static int g_ml[256][3];

__attribute__((constructor)) static void hermite_init(void) {
  int nm = or_nmom(DT_PMAX), nt = 0;
  mi_list(DT_PMAX, g_ml);
  for (int t = 0; t < nm; t++) {
    int m0 = g_ml[t][0], m1 = g_ml[t][1], m2 = g_ml[t][2];
    g_hbeg[t] = nt;
    for (int k0 = 0; 2 * k0 <= m0; k0++)
      for (int k1 = 0; 2 * k1 <= m1; k1++)
        for (int k2 = 0; 2 * k2 <= m2; k2++) {
          hterm *h = &g_ht[nt++];
          h->cf = fact(m0) / (fact(k0) * fact(m0 - 2 * k0) * ipow(2.0, k0)) * fact(m1) /
                  (fact(k1) * fact(m1 - 2 * k1) * ipow(2.0, k1)) * fact(m2) /
                  (fact(k2) * fact(m2 - 2 * k2) * ipow(2.0, k2));
          h->e[0] = m0 - 2 * k0;
          h->e[1] = m1 - 2 * k1;
          h->e[2] = m2 - 2 * k2;
          h->j = m0 + m1 + m2 - k0 - k1 - k2;
        }
    g_hend[t] = nt;
  }
}

void or_dtensor(const double R[3], double eps, int pmax, double *D) {
  double s = R[0] * R[0] + R[1] * R[1] + R[2] * R[2] + eps * eps;
  double F[DT_PMAX + 1];
  double df = 1.0; /* (2j-1)!! */
  for (int j = 0; j <= pmax; j++) {
    if (j > 0) df *= (2 * j - 1);
    F[j] = ((j & 1) ? -1.0 : 1.0) * df * pow(s, -0.5 - j);
  }
  double pw[3][DT_PMAX + 1];
  for (int d = 0; d < 3; d++) {
    pw[d][0] = 1.0;
    for (int e = 1; e <= pmax; e++) pw[d][e] = pw[d][e - 1] * R[d];
  }
  int nm = or_nmom(pmax);
  for (int t = 0; t < nm; t++) {
    double v = 0.0;
    for (int h = g_hbeg[t]; h < g_hend[t]; h++) {
      const hterm *q = &g_ht[h];
      v += q->cf * pw[0][q->e[0]] * pw[1][q->e[1]] * pw[2][q->e[2]] * F[q->j];
    }
    D[t] = v;
  }
}

void or_m2p_orders(const double *M, int pmin, int pmax, const double R[3], double eps, double a[3]) {
  double D[256];
  or_dtensor(R, eps, pmax + 1, D);
  int nm = or_nmom(pmax);
  a[0] = a[1] = a[2] = 0.0;
  for (int t = pmin > 0 ? or_nmom(pmin - 1) : 0; t < nm; t++) {
    int nx = g_ml[t][0], ny = g_ml[t][1], nz = g_ml[t][2];
    int o = nx + ny + nz;
    double C = ((o & 1) ? -1.0 : 1.0) * M[t] / (fact(nx) * fact(ny) * fact(nz));
    a[0] += C * D[mi_idx(nx + 1, ny, nz)];
    a[1] += C * D[mi_idx(nx, ny + 1, nz)];
    a[2] += C * D[mi_idx(nx, ny, nz + 1)];
  }
}

/* Psi(R) = sum_{pmin <= |n| <= pmax} ((-1)^|n|/n!) M_n d^n g(R): the
 * expansion's potential up to sign (a = grad Psi, potential -Psi) */
double or_m2p_pot_orders(const double *M, int pmin, int pmax, const double R[3], double eps) {
  double D[256];
  or_dtensor(R, eps, pmax, D);
  int nm = or_nmom(pmax);
  double v = 0.0;
  for (int t = pmin > 0 ? or_nmom(pmin - 1) : 0; t < nm; t++) {
    int nx = g_ml[t][0], ny = g_ml[t][1], nz = g_ml[t][2];
    v += ((nx + ny + nz) & 1 ? -1.0 : 1.0) * M[t] / (fact(nx) * fact(ny) * fact(nz)) * D[t];
  }
  return v;
}

void or_m2p(const double *M, int p, const double R[3], double eps, double a[3]) {
  or_m2p_orders(M, 0, p, R, eps, a);
}

/* Local expansion of a cell's field about z: with Psi(x) = sum_n
 * ((-1)^|n|/n!) M_n d^n g(x - c) (a = grad Psi), L_k = d^k Psi(z) truncated
 * to the derivative orders of the M2P: |n| + |k| <= p + 1. */
void or_m2l(const double *M, int p, const double R[3], double eps, double *L) {
  int P = p + 1;
  double D[256];
  or_dtensor(R, eps, P, D);
  int nl = or_nmom(P), nm = or_nmom(p);
  for (int t = 1; t < nl; t++) {
    int k0 = g_ml[t][0], k1 = g_ml[t][1], k2 = g_ml[t][2];
    int ok = k0 + k1 + k2;
    for (int u = 0; u < nm; u++) {
      int n0 = g_ml[u][0], n1 = g_ml[u][1], n2 = g_ml[u][2];
      int on = n0 + n1 + n2;
      if (on + ok > P) continue;
      double cf = ((on & 1) ? -1.0 : 1.0) / (fact(n0) * fact(n1) * fact(n2));
      L[t] += cf * M[u] * D[mi_idx(n0 + k0, n1 + k1, n2 + k2)];
    }
  }
}

/* a_k(z + d) = sum_{|m| <= p} d^m/m! L_(m + e_k): the gradient of the
 * truncated Taylor series of Psi about z */
void or_l2p(const double *L, int p, const double d[3], double a[3]) {
  int nm = or_nmom(p);
  a[0] = a[1] = a[2] = 0.0;
  for (int u = 0; u < nm; u++) {
    int m0 = g_ml[u][0], m1 = g_ml[u][1], m2 = g_ml[u][2];
    double tay = ipow(d[0], m0) * ipow(d[1], m1) * ipow(d[2], m2) / (fact(m0) * fact(m1) * fact(m2));
    a[0] += tay * L[mi_idx(m0 + 1, m1, m2)];
    a[1] += tay * L[mi_idx(m0, m1 + 1, m2)];
    a[2] += tay * L[mi_idx(m0, m1, m2 + 1)];
  }
}

/* Moments about its centre of a cube of side s filled with density rho:
 * C_n = rho prod_d int_{-s/2}^{s/2} x^{n_d} dx, i.e. rho prod_d s^(n_d+1) /
 * ((n_d+1) 2^n_d) for even n_d and 0 for odd n_d. */
void or_cube_moments(double s, double rho, int p, double *C) {
  int nm = or_nmom(p);
  for (int t = 0; t < nm; t++) {
    double v = rho;
    for (int d = 0; d < 3; d++) {
      int k = g_ml[t][d];
      v *= (k & 1) ? 0.0 : ipow(s, k + 1) / ((double)(k + 1) * ipow(2.0, k));
    }
    C[t] = v;
  }
}

/* ---- keys and sort --------------------------------------------------------- */
static int64_t quant(double x) {
  int64_t q = (int64_t)floor(x * (double)(1 << QBITS));
  int64_t M = (int64_t)1 << QBITS;
  q %= M;
  if (q < 0) q += M;
  return q;
}

static uint64_t spread3(uint64_t v) {
  uint64_t r = 0;
  for (int b = 0; b < QBITS; b++) r |= ((v >> b) & 1ull) << (3 * b);
  return r;
}

void or_morton_keys(int64_t n, const double *pos, uint64_t *keys) {
  for (int64_t i = 0; i < n; i++) {
    uint64_t qx = (uint64_t)quant(pos[i]), qy = (uint64_t)quant(pos[n + i]),
             qz = (uint64_t)quant(pos[2 * n + i]);
    keys[i] = spread3(qx) | (spread3(qy) << 1) | (spread3(qz) << 2);
  }
}

static const uint64_t *g_sort_keys;
static int cmp_key_idx(const void *a, const void *b) {
  int64_t i = *(const int64_t *)a, j = *(const int64_t *)b;
  uint64_t ki = g_sort_keys[i], kj = g_sort_keys[j];
  if (ki != kj) return ki < kj ? -1 : 1;
  return i < j ? -1 : (i > j ? 1 : 0);
}

void or_sort_perm(int64_t n, const uint64_t *keys, int64_t *perm) {
  for (int64_t i = 0; i < n; i++) perm[i] = i;
  g_sort_keys = keys; /* single-threaded use only */
  qsort(perm, (size_t)n, sizeof(int64_t), cmp_key_idx);
}

/* ---- tree ---------------------------------------------------------------- */
typedef struct {
  int level, nchild;
  int64_t start, count;
  int64_t ix[3];   /* integer cell coordinates at its level */
  int64_t child[8];
} tcell;

typedef struct {
  tcell *c;
  int64_t n, cap;
  const uint64_t *skeys; /* keys in sorted order */
  int n_leaf, lmax;
} tbuild;

static int64_t new_cell(tbuild *b) {
  if (b->n == b->cap) {
    b->cap = b->cap ? 2 * b->cap : 1024;
    b->c = realloc(b->c, sizeof(tcell) * b->cap);
  }
  return b->n++;
}

static int64_t build_rec(tbuild *b, int level, int64_t start, int64_t count, int64_t ix,
                         int64_t iy, int64_t iz) {
  int64_t id = new_cell(b);
  tcell *c = &b->c[id];
  c->level = level;
  c->start = start;
  c->count = count;
  c->ix[0] = ix;
  c->ix[1] = iy;
  c->ix[2] = iz;
  c->nchild = 0;
  if (count > b->n_leaf && level < b->lmax) {
    int sh = 3 * (QBITS - (level + 1));
    int64_t s = start;
    for (int d = 0; d < 8; d++) {
      int64_t e = s;
      while (e < start + count && (int)((b->skeys[e] >> sh) & 7ull) == d) e++;
      if (e > s) {
        int64_t ch = build_rec(b, level + 1, s, e - s, 2 * ix + (d & 1), 2 * iy + ((d >> 1) & 1),
                               2 * iz + ((d >> 2) & 1));
        c = &b->c[id]; /* realloc may have moved the array */
        c->child[c->nchild++] = ch;
      }
      s = e;
    }
  }
  return id;
}

/* centre of a cell in units of 2^-22 */
static int64_t centre_u(int64_t i, int level) { return (2 * i + 1) << (QBITS - level); }

typedef struct {
  const or_tree_params *p;
  const tcell *cells;
  const double *mom; /* ncell x nmom */
  int nmom;
  const double *X, *Y, *Z, *Mass; /* sorted order */
  const uint64_t *skeys;
  double T[QBITS + 1];
  /* image field: fixed level-ew_level cells */
  int64_t nec;
  const int64_t *ec_ix; /* 3 per cell */
  const double *ec_mom; /* nmom(p_E) per cell */
  const double *lat;    /* phi~ lattice, orders 0..p_E+1 */
  double rho;           /* mean density: total mass over the unit box */
} walkctx;

typedef struct {
  int64_t start, count;
  int64_t g2[3], w2[3]; /* group box centre and half-width, units 2^-23 */
  int64_t cell2[3];     /* centre of the group's level-(ew_grid-1) cell, units 2^-23 */
} tgroup;

typedef struct {
  double p2p, m2p, ew, m2l;
} wstats;

static const int64_t PBOX = (int64_t)1 << 23; /* one box in units of 2^-23 */

/* image shift k (box units) of the point 2*cu (units 2^-23) nearest g2 */
static int64_t img_shift(int64_t c2, int64_t g2) {
  int64_t delta = c2 - g2;
  int64_t red = ((delta + (PBOX >> 1)) % PBOX + PBOX) % PBOX - (PBOX >> 1);
  return (delta - red) / PBOX;
}

/* image of a cell from its level-ew_level ancestor (or common descendant image) */
static int cell_image(const walkctx *w, const tgroup *G, int level, const int64_t ix[3],
                      int64_t k[3]) {
  int le = w->p->ew_level;
  for (int d = 0; d < 3; d++) {
    if (level >= le) {
      int64_t a = ix[d] >> (level - le);
      k[d] = img_shift(2 * centre_u(a, le), G->cell2[d]);
    } else {
      int64_t lo = ix[d] << (le - level), hi = ((ix[d] + 1) << (le - level)) - 1;
      int64_t klo = img_shift(2 * centre_u(lo, le), G->cell2[d]);
      int64_t khi = img_shift(2 * centre_u(hi, le), G->cell2[d]);
      if (klo != khi) return 0;
      k[d] = klo;
    }
  }
  return 1;
}

static int64_t quant(double x);

static void walk_rec(const walkctx *w, const tgroup *G, int64_t ci, double *acc /* 3 x count */,
                     double *Lg /* the group's local expansion (dual) */, double *pot /* nullable */,
                     wstats *st, const int64_t *kfix /* replicas: the image (c - k), else NULL */) {
  const tcell *c = &w->cells[ci];
  const or_tree_params *p = w->p;
  int64_t kimg[3];
  int consistent = 1;
  if (kfix)
    for (int d = 0; d < 3; d++) kimg[d] = kfix[d];
  else
    consistent = cell_image(w, G, c->level, c->ix, kimg);
  int64_t d2 = 0;
  for (int d = 0; d < 3; d++) {
    int64_t delta = 2 * centre_u(c->ix[d], c->level) - G->g2[d] - kimg[d] * PBOX;
    int64_t ad = delta < 0 ? -delta : delta;
    /* d is measured from the cell centre, or (mac = 1) from the cell's
       faces: the half side 2^(22 - level) in these units is taken off */
    int64_t dd = ad - G->w2[d] - (p->mac ? ((int64_t)1 << (22 - c->level)) : 0);
    if (dd < 0) dd = 0;
    d2 += dd * dd;
  }
  /* levels 0-1 are always opened, except with replicas (any level may be accepted) */
  int accept = consistent && c->level >= (kfix ? 0 : 2) && (double)d2 > w->T[c->level];
  int leaf = c->nchild == 0;
  if (!accept && !leaf) {
    for (int k = 0; k < c->nchild; k++) walk_rec(w, G, c->child[k], acc, Lg, pot, st, kfix);
    return;
  }
  double cs[3];
  for (int d = 0; d < 3; d++) cs[d] = ldexp((double)centre_u(c->ix[d], c->level), -22) - (double)kimg[d];
  const double *M = w->mom + ci * w->nmom;
  int use_m2p = accept && c->count > p->n_direct;
  int le = p->ew_level;
  if (use_m2p && p->dual) {
    /* cell-group test: centre-to-centre distance against (s_C + s_G)/theta */
    int64_t wmax = G->w2[0] > G->w2[1] ? G->w2[0] : G->w2[1];
    if (G->w2[2] > wmax) wmax = G->w2[2];
    int64_t S = ((int64_t)1 << (23 - c->level)) + 2 * wmax;
    double T = floor((double)S * (double)S / (p->theta * p->theta));
    int64_t dcc2 = 0;
    for (int d = 0; d < 3; d++) {
      int64_t delta = 2 * centre_u(c->ix[d], c->level) - G->g2[d] - kimg[d] * PBOX;
      dcc2 += delta * delta;
    }
    if ((double)dcc2 > T) {
      double R[3];
      for (int d = 0; d < 3; d++) R[d] = ldexp((double)G->g2[d], -23) - cs[d];
      or_m2l(M, p->order, R, p->kernel == 1 ? 0.0 : p->eps, Lg);
      st->m2l += 1.0;
      if (!pot) return;
      /* the potential is the M2P form's (below) also for such cells */
      for (int64_t s = 0; s < G->count; s++) {
        int64_t i = G->start + s;
        double Rs[3] = {w->X[i] - cs[0], w->Y[i] - cs[1], w->Z[i] - cs[2]};
        pot[s] -= or_m2p_pot_orders(M, 0, p->order, Rs, p->kernel == 1 ? 0.0 : p->eps);
      }
      return;
    }
  }
  for (int64_t s = 0; s < G->count; s++) {
    int64_t i = G->start + s;
    double xi[3] = {w->X[i], w->Y[i], w->Z[i]};
    double a[3] = {0.0, 0.0, 0.0};
    if (use_m2p) {
      double R[3] = {xi[0] - cs[0], xi[1] - cs[1], xi[2] - cs[2]};
      or_m2p(M, p->order, R, p->kernel == 1 ? 0.0 : p->eps, a);
      if (pot) pot[s] -= or_m2p_pot_orders(M, 0, p->order, R, p->kernel == 1 ? 0.0 : p->eps);
      if (p->bg > p->order) {
        /* the cell's share of the uniform background (a cube of the mean
           density filling the cell) beyond order p, Newtonian kernel */
        double C[256], ab[3];
        or_cube_moments(ldexp(1.0, -c->level), w->rho, p->bg, C);
        or_m2p_orders(C, p->order + 1, p->bg, R, 0.0, ab);
        for (int d = 0; d < 3; d++) a[d] += ab[d];
        if (pot) pot[s] -= or_m2p_pot_orders(C, p->order + 1, p->bg, R, 0.0);
      }
      st->m2p += 1.0;
    } else {
      for (int64_t j = c->start; j < c->start + c->count; j++) {
        int64_t kj[3];
        if (kfix) {
          /* replicas: the whole cell at its image; only the sink itself in the central box is skipped */
          if (j == i && kfix[0] == 0 && kfix[1] == 0 && kfix[2] == 0) continue;
          for (int d = 0; d < 3; d++) kj[d] = kfix[d];
        } else {
          if (j == i) continue;
          /* per-particle image from its level-ew_level ancestor */
          int64_t jx[3] = {quant(w->X[j]) >> (QBITS - le), quant(w->Y[j]) >> (QBITS - le),
                           quant(w->Z[j]) >> (QBITS - le)};
          for (int d = 0; d < 3; d++) kj[d] = img_shift(2 * centre_u(jx[d], le), G->cell2[d]);
        }
        double r[3] = {w->X[j] - (double)kj[0] - xi[0], w->Y[j] - (double)kj[1] - xi[1],
                       w->Z[j] - (double)kj[2] - xi[2]};
        double r2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
        double f = w->Mass[j] * or_soft_factor(r2, p->eps, p->kernel);
        if (pot) pot[s] += w->Mass[j] * or_soft_pot(r2, p->eps, p->kernel);
        a[0] += f * r[0];
        a[1] += f * r[1];
        a[2] += f * r[2];
        st->p2p += 1.0;
      }
    }
    acc[s] += a[0];
    acc[G->count + s] += a[1];
    acc[2 * G->count + s] += a[2];
  }
}

/* per-group image field: local expansion about e from the level-ew_level cells */
static void periodic_group(const walkctx *w, const tgroup *G, double *acc, double *pot, wstats *st) {
  const or_tree_params *p = w->p;
  int pe = p->ewald, P = pe + 1, le = p->ew_level;
  int nl = or_nmom(P), ne = or_nmom(pe);
  int64_t step = (int64_t)1 << (23 - p->ew_grid);
  const int64_t *e2 = G->cell2; /* expansion point: centre of the group's cell */
  double e[3];
  for (int d = 0; d < 3; d++) e[d] = ldexp((double)e2[d], -23);
  double L[128], Dv[128], V[3] = {0.0, 0.0, 0.0}, Mt = 0.0, W = 0.0;
  for (int t = 0; t < nl; t++) L[t] = 0.0;
  for (int64_t ci = 0; ci < w->nec; ci++) {
    const int64_t *ix = w->ec_ix + 3 * ci;
    const double *M = w->ec_mom + ci * ne;
    int64_t k[3], ir[3];
    double cst[3];
    for (int d = 0; d < 3; d++) {
      int64_t c2 = 2 * centre_u(ix[d], le);
      k[d] = img_shift(c2, e2[d]);
      ir[d] = (e2[d] - (c2 - k[d] * PBOX)) / step;
      cst[d] = ldexp((double)c2, -23) - (double)k[d];
    }
    or_phitilde_lattice_get(w->lat, p->ew_grid, P, ir, Dv);
    for (int t = pot ? 0 : 1; t < nl; t++) {
      int m0 = g_ml[t][0], m1 = g_ml[t][1], m2 = g_ml[t][2];
      int om = m0 + m1 + m2;
      for (int u = 0; u < ne; u++) {
        int n0 = g_ml[u][0], n1 = g_ml[u][1], n2 = g_ml[u][2];
        int on = n0 + n1 + n2;
        if (om + on > P) continue;
        double cf = ((on & 1) ? -1.0 : 1.0) / (fact(n0) * fact(n1) * fact(n2));
        L[t] += cf * M[u] * Dv[mi_idx(m0 + n0, m1 + n1, m2 + n2)];
      }
    }
    double mc = M[0];
    V[0] += mc * (cst[0] - e[0]) + M[mi_idx(1, 0, 0)];
    V[1] += mc * (cst[1] - e[1]) + M[mi_idx(0, 1, 0)];
    V[2] += mc * (cst[2] - e[2]) + M[mi_idx(0, 0, 1)];
    Mt += mc;
    if (pot) {
      /* sum over the cell of m |x_j* - e|^2, about its centre r = c* - e */
      double r[3] = {cst[0] - e[0], cst[1] - e[1], cst[2] - e[2]};
      W += mc * (r[0] * r[0] + r[1] * r[1] + r[2] * r[2]) +
           2.0 * (r[0] * M[mi_idx(1, 0, 0)] + r[1] * M[mi_idx(0, 1, 0)] + r[2] * M[mi_idx(0, 0, 1)]) +
           M[mi_idx(2, 0, 0)] + M[mi_idx(0, 2, 0)] + M[mi_idx(0, 0, 2)];
    }
    st->ew += 1.0;
  }
  for (int64_t s = 0; s < G->count; s++) {
    int64_t i = G->start + s;
    double dd[3] = {w->X[i] - e[0], w->Y[i] - e[1], w->Z[i] - e[2]};
    double a[3];
    for (int k = 0; k < 3; k++) a[k] = (4.0 * PI / 3.0) * (Mt * dd[k] - V[k]);
    for (int u = 0; u < ne; u++) {
      int n0 = g_ml[u][0], n1 = g_ml[u][1], n2 = g_ml[u][2];
      double tay = ipow(dd[0], n0) * ipow(dd[1], n1) * ipow(dd[2], n2) /
                   (fact(n0) * fact(n1) * fact(n2));
      a[0] -= tay * L[mi_idx(n0 + 1, n1, n2)];
      a[1] -= tay * L[mi_idx(n0, n1 + 1, n2)];
      a[2] -= tay * L[mi_idx(n0, n1, n2 + 1)];
    }
    acc[s] += a[0];
    acc[G->count + s] += a[1];
    acc[2 * G->count + s] += a[2];
    if (pot) {
      /* -(2 pi/3) sum_j m_j |x - x_j*|^2 + sum_j m_j phi~(x - x_j*), the latter
         as the truncated Taylor series of the local expansion about e */
      double v = -(2.0 * PI / 3.0) *
                 (Mt * (dd[0] * dd[0] + dd[1] * dd[1] + dd[2] * dd[2]) -
                  2.0 * (dd[0] * V[0] + dd[1] * V[1] + dd[2] * V[2]) + W);
      for (int t = 0; t < nl; t++) {
        int m0 = g_ml[t][0], m1 = g_ml[t][1], m2 = g_ml[t][2];
        v += ipow(dd[0], m0) * ipow(dd[1], m1) * ipow(dd[2], m2) / (fact(m0) * fact(m1) * fact(m2)) * L[t];
      }
      pot[s] += v;
    }
  }
}

static int build_tree(int64_t n, const double *pos, int n_leaf, int lmax, int64_t *perm,
                      uint64_t *skeys, tbuild *b) {
  uint64_t *keys = malloc(sizeof(uint64_t) * (n > 0 ? n : 1));
  or_morton_keys(n, pos, keys);
  or_sort_perm(n, keys, perm);
  for (int64_t i = 0; i < n; i++) skeys[i] = keys[perm[i]];
  free(keys);
  memset(b, 0, sizeof(*b));
  b->skeys = skeys;
  b->n_leaf = n_leaf;
  b->lmax = lmax;
  build_rec(b, 0, 0, n, 0, 0, 0);
  return 0;
}

int64_t or_tree_cells(int64_t n, const double *pos, int n_leaf, int lmax, int64_t cap,
                      uint64_t *key, int32_t *level, int64_t *start, int64_t *count) {
  int64_t *perm = malloc(sizeof(int64_t) * n);
  uint64_t *skeys = malloc(sizeof(uint64_t) * n);
  tbuild b;
  build_tree(n, pos, n_leaf, lmax, perm, skeys, &b);
  int64_t nc = b.n;
  if (nc > cap) {
    free(perm);
    free(skeys);
    free(b.c);
    return -nc;
  }
  /* breadth-first order: by level, then by start (= key order within a level) */
  int64_t out = 0;
  for (int l = 0; l <= lmax; l++)
    for (int64_t i = 0; i < nc; i++) {
      /* cells of one level appear in start order in the preorder array */
      if (b.c[i].level != l) continue;
      uint64_t pre = skeys[b.c[i].start] >> (3 * (QBITS - l));
      key[out] = ((uint64_t)1 << (3 * l)) | pre;
      level[out] = l;
      start[out] = b.c[i].start;
      count[out] = b.c[i].count;
      out++;
    }
  free(perm);
  free(skeys);
  free(b.c);
  return nc;
}

#define LAT_P 8 /* order of the far-lattice expansion */

void or_lattice_tensor(int P, int W, double *T) {
  or_ewald_cfg cfg;
  or_ewald_default(&cfg);
  double zero[3] = {0.0, 0.0, 0.0}, D[256];
  int nm = or_nmom(P);
  or_phitilde_mi(zero, &cfg, P, T);
  /* the background's -(2 pi/3)|r|^2 */
  T[mi_idx(2, 0, 0)] -= 4.0 * PI / 3.0;
  T[mi_idx(0, 2, 0)] -= 4.0 * PI / 3.0;
  T[mi_idx(0, 0, 2)] -= 4.0 * PI / 3.0;
  /* the near images' +1/|r - n|, 0 < |n|_inf <= W (derivatives at r = 0: R = -n) */
  const int S1 = 2 * W + 1;
  for (int r = 0; r < S1 * S1 * S1; r++) {
    double R[3] = {-(double)(r % S1 - W), -(double)((r / S1) % S1 - W), -(double)(r / (S1 * S1) - W)};
    if (R[0] == 0.0 && R[1] == 0.0 && R[2] == 0.0) continue;
    or_dtensor(R, 0.0, P, D);
    for (int t = 0; t < nm; t++) T[t] += D[t];
  }
}

int or_tree_forces(int64_t n, const double *pos, const double *mass, const or_tree_params *p,
                   const double *tab, int64_t ntarget, const int64_t *targets, double *acc,
                   double *stats) {
  return or_tree_forces_pot(n, pos, mass, p, tab, ntarget, targets, acc, NULL, stats);
}

int or_tree_forces_pot(int64_t n, const double *pos, const double *mass, const or_tree_params *p,
                       const double *tab, int64_t ntarget, const int64_t *targets, double *acc,
                       double *pot, double *stats) {
  if (n <= 0) return 0;
  if (pot && p->ewald > 0 && p->ewald < 2) return -1; /* the background potential needs second moments */
  if (p->order < 0 || p->order > 4 || p->lmax < 2 || p->lmax > QBITS || p->n_leaf < 1 ||
      p->n_group < 1 || p->n_direct > p->n_leaf || p->ewald < 0 || p->ewald > 5 ||
      (p->ewald > 0 && !tab) || p->ew_level < 1 || p->ew_level > 8 ||
      p->ew_grid < p->ew_level + 1 || p->ew_grid > 10 || p->bg < 0 || p->bg > 8 || p->kernel < 0 ||
      p->kernel > 1 || p->dual < 0 || p->dual > 1 || (p->dual && p->bg > p->order) || p->replicas < 0 ||
      p->replicas > 2 || (p->replicas && p->ewald != 0))
    return -1;
  int64_t *perm = malloc(sizeof(int64_t) * n);
  uint64_t *skeys = malloc(sizeof(uint64_t) * n);
  tbuild b;
  build_tree(n, pos, p->n_leaf, p->lmax, perm, skeys, &b);
  int64_t nc = b.n;
  /* sorted particle arrays */
  double *S = malloc(sizeof(double) * 4 * n);
  double *X = S, *Y = S + n, *Z = S + 2 * n, *Ms = S + 3 * n;
  for (int64_t i = 0; i < n; i++) {
    int64_t j = perm[i];
    X[i] = pos[j];
    Y[i] = pos[n + j];
    Z[i] = pos[2 * n + j];
    Ms[i] = mass ? mass[j] : 1.0 / (double)n;
  }
  /* moments about geometric centres, direct from particles */
  int nm = or_nmom(p->order);
  double *mom = malloc(sizeof(double) * nm * nc);
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t ci = 0; ci < nc; ci++) {
    const tcell *c = &b.c[ci];
    double cc[3];
    for (int d = 0; d < 3; d++) cc[d] = ldexp((double)centre_u(c->ix[d], c->level), -22);
    int64_t m = c->count;
    double *tmp = malloc(sizeof(double) * 3 * m);
    for (int64_t k = 0; k < m; k++) {
      tmp[k] = X[c->start + k];
      tmp[m + k] = Y[c->start + k];
      tmp[2 * m + k] = Z[c->start + k];
    }
    or_p2m(m, tmp, Ms + c->start, cc, p->order, mom + ci * nm);
    free(tmp);
  }
  /* fixed level-ew_level cells (key prefixes) and their moments of order p_E */
  int le = p->ew_level, ne = or_nmom(p->ewald);
  int64_t nec = 0;
  int64_t *ec_ix = malloc(sizeof(int64_t) * 3 * (n + 1));
  int64_t *ec_rng = malloc(sizeof(int64_t) * 2 * (n + 1));
  for (int64_t i = 0; i < n;) {
    uint64_t pre = skeys[i] >> (3 * (QBITS - le));
    int64_t j = i;
    while (j < n && (skeys[j] >> (3 * (QBITS - le))) == pre) j++;
    int64_t ix[3] = {0, 0, 0};
    for (int bb = 0; bb < le; bb++)
      for (int d = 0; d < 3; d++) ix[d] |= (int64_t)((pre >> (3 * bb + d)) & 1ull) << bb;
    for (int d = 0; d < 3; d++) ec_ix[3 * nec + d] = ix[d];
    ec_rng[2 * nec] = i;
    ec_rng[2 * nec + 1] = j - i;
    nec++;
    i = j;
  }
  double *ec_mom = malloc(sizeof(double) * ne * (nec > 0 ? nec : 1));
  for (int64_t ci = 0; ci < nec; ci++) {
    double cc[3];
    for (int d = 0; d < 3; d++) cc[d] = ldexp((double)centre_u(ec_ix[3 * ci + d], le), -22);
    int64_t s0 = ec_rng[2 * ci], m = ec_rng[2 * ci + 1];
    double *tmp = malloc(sizeof(double) * 3 * m);
    for (int64_t k = 0; k < m; k++) {
      tmp[k] = X[s0 + k];
      tmp[m + k] = Y[s0 + k];
      tmp[2 * m + k] = Z[s0 + k];
    }
    or_p2m(m, tmp, Ms + s0, cc, p->ewald, ec_mom + ci * ne);
    free(tmp);
  }
  walkctx w;
  w.p = p;
  w.cells = b.c;
  w.mom = mom;
  w.nmom = nm;
  w.X = X;
  w.Y = Y;
  w.Z = Z;
  w.Mass = Ms;
  w.skeys = skeys;
  w.nec = nec;
  w.ec_ix = ec_ix;
  w.ec_mom = ec_mom;
  w.lat = tab;
  w.rho = 0.0;
  for (int64_t i = 0; i < n; i++) w.rho += Ms[i];
  for (int l = 0; l <= QBITS; l++) {
    double s = ldexp(1.0, 23 - l);
    w.T[l] = floor((s * s) / (p->theta * p->theta));
  }
  /* far lattice (replicas): box moments about c0, the lattice tensor, L */
  double Lfar[256];
  for (int t = 0; t < 256; t++) Lfar[t] = 0.0;
  if (p->replicas) {
    int nl = or_nmom(LAT_P);
    double Mb[256], T[256];
    double c0[3] = {0.5, 0.5, 0.5};
    or_p2m(n, S, Ms, c0, LAT_P, Mb);
    or_lattice_tensor(LAT_P, p->replicas, T);
    for (int t = 0; t < nl; t++) {
      int k0 = g_ml[t][0], k1 = g_ml[t][1], k2 = g_ml[t][2];
      int ok = k0 + k1 + k2;
      for (int u = 0; u < nl; u++) {
        int n0 = g_ml[u][0], n1 = g_ml[u][1], n2 = g_ml[u][2];
        int on = n0 + n1 + n2;
        if (on + ok > LAT_P) continue;
        double cf = ((on & 1) ? -1.0 : 1.0) / (fact(n0) * fact(n1) * fact(n2));
        Lfar[t] += cf * Mb[u] * T[mi_idx(n0 + k0, n1 + k1, n2 + k2)];
      }
    }
  }
  /* groups: runs of <= n_group consecutive particles inside one level-ls cell */
  int ls = p->ew_grid - 1;
  int64_t *gstart = malloc(sizeof(int64_t) * (n + 1));
  int64_t ng = 0;
  for (int64_t i = 0; i < n;) {
    uint64_t pre = skeys[i] >> (3 * (QBITS - ls));
    int64_t j = i;
    while (j < n && (skeys[j] >> (3 * (QBITS - ls))) == pre) j++;
    for (int64_t s = i; s < j; s += p->n_group) gstart[ng++] = s;
    i = j;
  }
  gstart[ng] = n;
  int64_t *gid = malloc(sizeof(int64_t) * n);
  for (int64_t g = 0; g < ng; g++)
    for (int64_t i = gstart[g]; i < gstart[g + 1]; i++) gid[i] = g;
  char *need = calloc((size_t)ng, 1);
  int64_t *where = malloc(sizeof(int64_t) * n); /* original index -> sorted position */
  for (int64_t i = 0; i < n; i++) where[perm[i]] = i;
  int64_t nt = targets ? ntarget : n;
  for (int64_t t = 0; t < nt; t++) {
    int64_t orig = targets ? targets[t] : t;
    need[gid[where[orig]]] = 1;
  }
  double *sacc = calloc((size_t)(3 * n), sizeof(double));
  double *spot = pot ? calloc((size_t)n, sizeof(double)) : NULL;
  double sp2p = 0.0, sm2p = 0.0, sew = 0.0, sgroups = 0.0, ssinks = 0.0, sm2l = 0.0;
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : sp2p, sm2p, sew, sgroups, ssinks, sm2l)
  for (int64_t gi = 0; gi < ng; gi++) {
    if (!need[gi]) continue;
    tgroup G;
    G.start = gstart[gi];
    G.count = gstart[gi + 1] - gstart[gi];
    int64_t lo[3] = {INT64_MAX, INT64_MAX, INT64_MAX}, hi[3] = {INT64_MIN, INT64_MIN, INT64_MIN};
    for (int64_t s = 0; s < G.count; s++) {
      int64_t i = G.start + s;
      int64_t q[3] = {quant(X[i]), quant(Y[i]), quant(Z[i])};
      for (int d = 0; d < 3; d++) {
        if (2 * q[d] < lo[d]) lo[d] = 2 * q[d];
        if (2 * q[d] + 2 > hi[d]) hi[d] = 2 * q[d] + 2;
      }
      if (s == 0)
        for (int d = 0; d < 3; d++) G.cell2[d] = 2 * centre_u(q[d] >> (QBITS - ls), ls);
    }
    for (int d = 0; d < 3; d++) {
      G.g2[d] = lo[d] + hi[d];
      G.w2[d] = hi[d] - lo[d];
    }
    double *ga = calloc((size_t)(3 * G.count), sizeof(double));
    double *gp = spot ? calloc((size_t)G.count, sizeof(double)) : NULL;
    wstats st = {0.0, 0.0, 0.0, 0.0};
    double Lg[128];
    for (int t = 0; t < 128; t++) Lg[t] = 0.0;
    if (p->replicas) {
      /* the near replicas |n|_inf <= W, each a walk from the root at image n (k = -n) */
      const int W = p->replicas, S1 = 2 * W + 1;
      for (int r = 0; r < S1 * S1 * S1; r++) {
        int64_t kf[3] = {-(r % S1 - W), -((r / S1) % S1 - W), -(r / (S1 * S1) - W)};
        walk_rec(&w, &G, 0, ga, Lg, gp, &st, kf);
      }
    } else {
      walk_rec(&w, &G, 0, ga, Lg, gp, &st, NULL);
    }
    if (p->dual && st.m2l > 0.0)
      for (int64_t s = 0; s < G.count; s++) {
        int64_t i = G.start + s;
        double d[3] = {X[i] - ldexp((double)G.g2[0], -23), Y[i] - ldexp((double)G.g2[1], -23),
                       Z[i] - ldexp((double)G.g2[2], -23)};
        double a[3];
        or_l2p(Lg, p->order, d, a);
        for (int k = 0; k < 3; k++) ga[k * G.count + s] += a[k];
      }
    if (p->ewald > 0) periodic_group(&w, &G, ga, gp, &st);
    if (p->replicas) {
      /* the far lattice: local expansion of order LAT_P about the box centre */
      for (int64_t s = 0; s < G.count; s++) {
        int64_t i = G.start + s;
        double d[3] = {X[i] - 0.5, Y[i] - 0.5, Z[i] - 0.5};
        double a[3], v = 0.0;
        or_l2p(Lfar, LAT_P - 1, d, a);
        for (int k = 0; k < 3; k++) ga[k * G.count + s] -= a[k];
        if (gp) {
          for (int t = 0; t < or_nmom(LAT_P); t++) {
            int m0 = g_ml[t][0], m1 = g_ml[t][1], m2 = g_ml[t][2];
            v += ipow(d[0], m0) * ipow(d[1], m1) * ipow(d[2], m2) / (fact(m0) * fact(m1) * fact(m2)) * Lfar[t];
          }
          gp[s] += v;
        }
      }
    }
    for (int64_t s = 0; s < G.count; s++)
      for (int d = 0; d < 3; d++) sacc[d * n + G.start + s] = ga[d * G.count + s];
    if (gp)
      for (int64_t s = 0; s < G.count; s++) spot[G.start + s] = gp[s];
    free(gp);
    free(ga);
    sp2p += st.p2p;
    sm2p += st.m2p;
    sew += st.ew;
    sgroups += 1.0;
    ssinks += (double)G.count;
    sm2l += st.m2l;
  }
  for (int64_t t = 0; t < nt; t++) {
    int64_t orig = targets ? targets[t] : t;
    int64_t sidx = where[orig];
    for (int d = 0; d < 3; d++) acc[d * nt + t] = sacc[d * n + sidx];
    if (pot) pot[t] = spot[sidx];
  }
  free(spot);
  if (stats) {
    stats[0] = sp2p;
    stats[1] = sm2p;
    stats[2] = sew;
    stats[3] = (double)nc;
    stats[4] = sgroups;
    stats[5] = ssinks;
    stats[6] = sm2l;
  }
  free(sacc);
  free(where);
  free(need);
  free(gid);
  free(gstart);
  free(ec_ix);
  free(ec_rng);
  free(ec_mom);
  free(mom);
  free(S);
  free(b.c);
  free(perm);
  free(skeys);
  return 0;
}
