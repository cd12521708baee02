/*
 * Oracle: Ewald summation for the unit periodic cube (TEST INFRASTRUCTURE ONLY;
 * see oracle.h).
 *
 * Sec. 2.1 states that 2HOT treats periodic boundaries with a high-order
 * expansion of the image field; the build replaces it by the classical Ewald
 * split (Hernquist, Bouchet & Suto 1991).  For a unit source with the uniform
 * neutralising background, in a unit box with G = 1,
 *
 *   phi_E(r) = - sum_n erfc(a|r-n|)/|r-n|
 *              - (1/pi) sum_{h != 0} exp(-pi^2 h^2 / a^2) / h^2 cos(2 pi h.r)
 *              + pi / a^2,
 *   a_E(r)   = - grad phi_E.
 *
 * Radial screened functions obey the ladder  d_i B_l = -r_i B_{l+1}  with
 *   B_0 = erfc(a r)/r,
 *   B_l = [ (2l-1) B_{l-1} + (2a^2)^l / (a sqrt(pi)) exp(-a^2 r^2) ] / r^2,
 * and the n = 0 image combined with +1/r gives the smooth E_l = I_l - B_l,
 * I_l = (2l-1)!! / r^(2l+1), expanded in a power series for small a r.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>

static const double PI = 3.14159265358979323846264338327950288;

void or_ewald_default(or_ewald_cfg *c) {
  c->alpha = 2.0;
  c->rcut = 3.0;  /* erfc(6) ~ 2e-17 */
  c->h2max = 15;  /* exp(-pi^2 15 / 4) ~ 9e-17 */
}

/* screened ladder B_0..B_lmax at distance rho */
static void bseq(double rho, double alpha, int lmax, double *B) {
  double r2 = rho * rho;
  double ex = exp(-alpha * alpha * r2);
  double pw = 1.0;
  B[0] = erfc(alpha * rho) / rho;
  for (int l = 1; l <= lmax; l++) {
    pw *= 2.0 * alpha * alpha;
    B[l] = ((2 * l - 1) * B[l - 1] + pw / (alpha * sqrt(PI)) * ex) / r2;
  }
}

/* smooth ladder E_l of erf(a r)/r, E_0 = erf(a r)/r, d_i E_l = -r_i E_{l+1} */
static void eseq(double r, double alpha, int lmax, double *E) {
  if (alpha * r > 1.0) {
    double Bv[16];
    bseq(r, alpha, lmax, Bv);
    double inv2 = 1.0 / (r * r);
    double I = 1.0 / r;
    for (int l = 0; l <= lmax; l++) {
      E[l] = I - Bv[l];
      I *= (2 * l + 1) * inv2;
    }
    return;
  }
  /* E_l(s) = (2a/sqrt(pi)) (2a^2)^l sum_m (-a^2 s)^m / (m! (2(l+m)+1)), s = r^2 */
  double s = r * r;
  double x = -alpha * alpha * s;
  double pref = 2.0 * alpha / sqrt(PI);
  for (int l = 0; l <= lmax; l++) {
    double t = 1.0, sum = 0.0;
    for (int m = 0; m < 60; m++) {
      sum += t / (2 * (l + m) + 1);
      t *= x / (m + 1);
    }
    E[l] = pref * sum;
    pref *= 2.0 * alpha * alpha;
  }
}

/* symmetric index tables */
static const int I2[6][2] = {{0, 0}, {0, 1}, {0, 2}, {1, 1}, {1, 2}, {2, 2}};
static const int I3[10][3] = {{0, 0, 0}, {0, 0, 1}, {0, 0, 2}, {0, 1, 1}, {0, 1, 2},
                              {0, 2, 2}, {1, 1, 1}, {1, 1, 2}, {1, 2, 2}, {2, 2, 2}};

static inline double kd(int i, int j) { return i == j ? 1.0 : 0.0; }

/* add s * (derivatives of a radial function with ladder psi[0..3] at rho) */
static void add_radial(const double rho[3], const double *psi, double s, double out[20]) {
  out[0] += s * psi[0];
  for (int i = 0; i < 3; i++) out[1 + i] += s * (-rho[i] * psi[1]);
  for (int t = 0; t < 6; t++) {
    int i = I2[t][0], j = I2[t][1];
    out[4 + t] += s * (-kd(i, j) * psi[1] + rho[i] * rho[j] * psi[2]);
  }
  for (int t = 0; t < 10; t++) {
    int i = I3[t][0], j = I3[t][1], k = I3[t][2];
    double v = (kd(i, j) * rho[k] + kd(i, k) * rho[j] + kd(j, k) * rho[i]) * psi[2] -
               rho[i] * rho[j] * rho[k] * psi[3];
    out[10 + t] += s * v;
  }
}

void or_phitilde(const double r[3], const or_ewald_cfg *c, double out[20]) {
  for (int t = 0; t < 20; t++) out[t] = 0.0;
  double alpha = c->alpha;
  int nm = (int)ceil(c->rcut) + 1;
  /* real space, n != 0: -B_0(|r - n|) */
  for (int nx = -nm; nx <= nm; nx++)
    for (int ny = -nm; ny <= nm; ny++)
      for (int nz = -nm; nz <= nm; nz++) {
        if (nx == 0 && ny == 0 && nz == 0) continue;
        double rho[3] = {r[0] - nx, r[1] - ny, r[2] - nz};
        double d = sqrt(rho[0] * rho[0] + rho[1] * rho[1] + rho[2] * rho[2]);
        if (d >= c->rcut) continue;
        double B[4];
        bseq(d, alpha, 3, B);
        add_radial(rho, B, -1.0, out);
      }
  /* n = 0 image plus the removed Newtonian 1/r: E_0 = erf(a r)/r */
  {
    double d = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
    double E[4];
    eseq(d, alpha, 3, E);
    add_radial(r, E, 1.0, out);
  }
  /* reciprocal space */
  int hm = (int)floor(sqrt((double)c->h2max));
  for (int hx = -hm; hx <= hm; hx++)
    for (int hy = -hm; hy <= hm; hy++)
      for (int hz = -hm; hz <= hm; hz++) {
        int h2 = hx * hx + hy * hy + hz * hz;
        if (h2 == 0 || h2 > c->h2max) continue;
        double h[3] = {(double)hx, (double)hy, (double)hz};
        double w = exp(-PI * PI * h2 / (alpha * alpha)) / h2;
        double th = 2.0 * PI * (h[0] * r[0] + h[1] * r[1] + h[2] * r[2]);
        double cs = cos(th), sn = sin(th);
        out[0] += -(1.0 / PI) * w * cs;
        for (int i = 0; i < 3; i++) out[1 + i] += 2.0 * w * h[i] * sn;
        for (int t = 0; t < 6; t++) out[4 + t] += 4.0 * PI * w * h[I2[t][0]] * h[I2[t][1]] * cs;
        for (int t = 0; t < 10; t++)
          out[10 + t] += -8.0 * PI * PI * w * h[I3[t][0]] * h[I3[t][1]] * h[I3[t][2]] * sn;
      }
  /* background: +(2 pi/3) r^2 and the zero-mean constant */
  double r2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
  out[0] += (2.0 * PI / 3.0) * r2 + PI / (alpha * alpha);
  for (int i = 0; i < 3; i++) out[1 + i] += (4.0 * PI / 3.0) * r[i];
  out[4 + 0] += 4.0 * PI / 3.0;
  out[4 + 3] += 4.0 * PI / 3.0;
  out[4 + 5] += 4.0 * PI / 3.0;
}

/* a_E written directly from the Ewald sums (independent of or_phitilde) */
void or_ewald_acc(const double r[3], const or_ewald_cfg *c, double a[3]) {
  double alpha = c->alpha;
  a[0] = a[1] = a[2] = 0.0;
  int nm = (int)ceil(c->rcut) + 1;
  for (int nx = -nm; nx <= nm; nx++)
    for (int ny = -nm; ny <= nm; ny++)
      for (int nz = -nm; nz <= nm; nz++) {
        double rho[3] = {r[0] - nx, r[1] - ny, r[2] - nz};
        double d = sqrt(rho[0] * rho[0] + rho[1] * rho[1] + rho[2] * rho[2]);
        if (d >= c->rcut || d == 0.0) continue;
        double f = (erfc(alpha * d) + 2.0 * alpha * d / sqrt(PI) * exp(-alpha * alpha * d * d)) /
                   (d * d * d);
        for (int i = 0; i < 3; i++) a[i] -= rho[i] * f;
      }
  int hm = (int)floor(sqrt((double)c->h2max));
  for (int hx = -hm; hx <= hm; hx++)
    for (int hy = -hm; hy <= hm; hy++)
      for (int hz = -hm; hz <= hm; hz++) {
        int h2 = hx * hx + hy * hy + hz * hz;
        if (h2 == 0 || h2 > c->h2max) continue;
        double w = exp(-PI * PI * h2 / (alpha * alpha)) / h2;
        double sn = sin(2.0 * PI * (hx * r[0] + hy * r[1] + hz * r[2]));
        a[0] -= 2.0 * w * hx * sn;
        a[1] -= 2.0 * w * hy * sn;
        a[2] -= 2.0 * w * hz * sn;
      }
}

double or_ewald_pot(const double r[3], const or_ewald_cfg *c) {
  double alpha = c->alpha, phi = 0.0;
  int nm = (int)ceil(c->rcut) + 1;
  for (int nx = -nm; nx <= nm; nx++)
    for (int ny = -nm; ny <= nm; ny++)
      for (int nz = -nm; nz <= nm; nz++) {
        double rho[3] = {r[0] - nx, r[1] - ny, r[2] - nz};
        double d = sqrt(rho[0] * rho[0] + rho[1] * rho[1] + rho[2] * rho[2]);
        if (d >= c->rcut || d == 0.0) continue;
        phi -= erfc(alpha * d) / d;
      }
  int hm = (int)floor(sqrt((double)c->h2max));
  for (int hx = -hm; hx <= hm; hx++)
    for (int hy = -hm; hy <= hm; hy++)
      for (int hz = -hm; hz <= hm; hz++) {
        int h2 = hx * hx + hy * hy + hz * hz;
        if (h2 == 0 || h2 > c->h2max) continue;
        double w = exp(-PI * PI * h2 / (alpha * alpha)) / h2;
        phi -= (1.0 / PI) * w * cos(2.0 * PI * (hx * r[0] + hy * r[1] + hz * r[2]));
      }
  return phi + PI / (alpha * alpha);
}

/* ---- phi~ derivatives of any order <= 9 ----------------------------------
 * For a radial function with ladder psi_l (d_i psi_l = -r_i psi_{l+1}),
 *   d^m psi = sum_{k <= m/2} prod_d [m_d!/(k_d!(m_d-2k_d)! 2^k_d)] r^(m-2k) (-1)^(|m|-|k|) psi_{|m|-|k|},
 * and d^m cos(2 pi h.r) = (2 pi)^|m| h^m cos(2 pi h.r + |m| pi/2). */
#define PX 9
static int ml_idx(int nx, int ny, int nz) {
  int o = nx + ny + nz, j = ny + nz;
  return o * (o + 1) * (o + 2) / 6 + j * (j + 1) / 2 + nz;
}
static int nmomP(int p) { return (p + 1) * (p + 2) * (p + 3) / 6; }
static int e_ml[256][3];
typedef struct {
  double cf;
  int e[3], j;
} eterm;
static eterm e_ht[2048];
static int e_hb[256], e_he[256];
static double factd(int n) {
  double f = 1.0;
  for (int i = 2; i <= n; i++) f *= i;
  return f;
}
__attribute__((constructor)) static void ewald_terms_init(void) {
  int nt = 0;
  for (int o = 0; o <= PX; o++)
    for (int nx = o; nx >= 0; nx--)
      for (int ny = o - nx; ny >= 0; ny--) {
        int nz = o - nx - ny, id = ml_idx(nx, ny, nz);
        e_ml[id][0] = nx;
        e_ml[id][1] = ny;
        e_ml[id][2] = nz;
      }
  for (int t = 0; t < nmomP(PX); t++) {
    int m0 = e_ml[t][0], m1 = e_ml[t][1], m2 = e_ml[t][2];
    e_hb[t] = nt;
    for (int k0 = 0; 2 * k0 <= m0; k0++)
      for (int k1 = 0; 2 * k1 <= m1; k1++)
        for (int k2 = 0; 2 * k2 <= m2; k2++) {
          eterm *h = &e_ht[nt++];
          h->cf = factd(m0) / (factd(k0) * factd(m0 - 2 * k0) * ldexp(1.0, k0)) * factd(m1) /
                  (factd(k1) * factd(m1 - 2 * k1) * ldexp(1.0, k1)) * factd(m2) /
                  (factd(k2) * factd(m2 - 2 * k2) * ldexp(1.0, k2));
          h->e[0] = m0 - 2 * k0;
          h->e[1] = m1 - 2 * k1;
          h->e[2] = m2 - 2 * k2;
          h->j = m0 + m1 + m2 - k0 - k1 - k2;
        }
    e_he[t] = nt;
  }
}

static void add_radial_mi(const double rho[3], const double *psi, double s, int P, double *out) {
  double pw[3][PX + 1];
  for (int d = 0; d < 3; d++) {
    pw[d][0] = 1.0;
    for (int e = 1; e <= P; e++) pw[d][e] = pw[d][e - 1] * rho[d];
  }
  for (int t = 0; t < nmomP(P); t++) {
    double v = 0.0;
    for (int h = e_hb[t]; h < e_he[t]; h++) {
      const eterm *q = &e_ht[h];
      v += q->cf * pw[0][q->e[0]] * pw[1][q->e[1]] * pw[2][q->e[2]] * ((q->j & 1) ? -psi[q->j] : psi[q->j]);
    }
    out[t] += s * v;
  }
}

void or_phitilde_mi(const double r[3], const or_ewald_cfg *c, int P, double *out) {
  int nm = nmomP(P);
  for (int t = 0; t < nm; t++) out[t] = 0.0;
  double alpha = c->alpha;
  int nmx = (int)ceil(c->rcut) + 1;
  for (int nx = -nmx; nx <= nmx; nx++)
    for (int ny = -nmx; ny <= nmx; ny++)
      for (int nz = -nmx; nz <= nmx; nz++) {
        if (nx == 0 && ny == 0 && nz == 0) continue;
        double rho[3] = {r[0] - nx, r[1] - ny, r[2] - nz};
        double d = sqrt(rho[0] * rho[0] + rho[1] * rho[1] + rho[2] * rho[2]);
        if (d >= c->rcut) continue;
        double B[PX + 1];
        bseq(d, alpha, P, B);
        add_radial_mi(rho, B, -1.0, P, out);
      }
  {
    double d = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
    double E[PX + 1];
    eseq(d, alpha, P, E);
    add_radial_mi(r, E, 1.0, P, out);
  }
  int hm = (int)floor(sqrt((double)c->h2max));
  for (int hx = -hm; hx <= hm; hx++)
    for (int hy = -hm; hy <= hm; hy++)
      for (int hz = -hm; hz <= hm; hz++) {
        int h2 = hx * hx + hy * hy + hz * hz;
        if (h2 == 0 || h2 > c->h2max) continue;
        double w = exp(-PI * PI * h2 / (alpha * alpha)) / h2;
        double th = 2.0 * PI * (hx * r[0] + hy * r[1] + hz * r[2]);
        double cs = cos(th), sn = sin(th);
        for (int t = 0; t < nm; t++) {
          int o = e_ml[t][0] + e_ml[t][1] + e_ml[t][2];
          double hp = pow(2.0 * PI, o);
          for (int q = 0; q < e_ml[t][0]; q++) hp *= hx;
          for (int q = 0; q < e_ml[t][1]; q++) hp *= hy;
          for (int q = 0; q < e_ml[t][2]; q++) hp *= hz;
          double ph = (o % 4 == 0) ? cs : (o % 4 == 1) ? -sn : (o % 4 == 2) ? -cs : sn;
          out[t] += -(1.0 / PI) * w * hp * ph;
        }
      }
  double r2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
  out[0] += (2.0 * PI / 3.0) * r2 + PI / (alpha * alpha);
  if (P >= 1)
    for (int i = 0; i < 3; i++) out[1 + i] += (4.0 * PI / 3.0) * r[i];
  if (P >= 2) {
    out[ml_idx(2, 0, 0)] += 4.0 * PI / 3.0;
    out[ml_idx(0, 2, 0)] += 4.0 * PI / 3.0;
    out[ml_idx(0, 0, 2)] += 4.0 * PI / 3.0;
  }
}

/* Lattice of phi~ derivatives at nodes (i,j,k) h, h = 2^-lg, 0 <= i,j,k <= 2^(lg-1)+1,
 * multi-index order 0..P (nmom(P) values per node). */
int or_phitilde_lattice(int lg, int P, double *tab) {
  if (lg < 1 || lg > 10 || P < 0 || P > PX) return -1;
  or_ewald_cfg c;
  or_ewald_default(&c);
  int m = (1 << (lg - 1)) + 2;
  int nm = nmomP(P);
  double h = ldexp(1.0, -lg);
  int64_t total = (int64_t)m * m * m;
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t id = 0; id < total; id++) {
    int i = (int)(id / ((int64_t)m * m)), j = (int)((id / m) % m), k = (int)(id % m);
    double r[3] = {i * h, j * h, k * h};
    or_phitilde_mi(r, &c, P, tab + id * nm);
  }
  return 0;
}

/* derivatives at the lattice point (ix,iy,iz) h (signed), by parity folding */
void or_phitilde_lattice_get(const double *tab, int lg, int P, const int64_t ir[3], double *out) {
  int m = (1 << (lg - 1)) + 2;
  int nm = nmomP(P);
  int64_t a[3];
  int neg[3];
  for (int d = 0; d < 3; d++) {
    neg[d] = ir[d] < 0;
    a[d] = neg[d] ? -ir[d] : ir[d];
  }
  const double *src = tab + ((a[0] * m + a[1]) * m + a[2]) * nm;
  for (int t = 0; t < nm; t++) {
    int s = 1;
    for (int d = 0; d < 3; d++)
      if (neg[d] && (e_ml[t][d] & 1)) s = -s;
    out[t] = s * src[t];
  }
}

/* parity of an order-1/2 component under r_d -> -r_d: (-1)^(count of d) */
static const int CNT[9][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}, {2, 0, 0}, {1, 1, 0},
                              {1, 0, 1}, {0, 2, 0}, {0, 1, 1}, {0, 0, 2}};

/* ---- tricubic tables for the direct oracle ------------------------------- */
static int tricubic_build(int n1, double *tab, int ncomp, int first) {
  if (n1 < 2) return -1;
  or_ewald_cfg c;
  or_ewald_default(&c);
  int m = n1 + 4;
  double h = 0.5 / n1;
  int64_t total = (int64_t)m * m * m;
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t id = 0; id < total; id++) {
    int i = (int)(id / ((int64_t)m * m)), j = (int)((id / m) % m), k = (int)(id % m);
    double r[3] = {(i - 1) * h, (j - 1) * h, (k - 1) * h};
    double out[20];
    or_phitilde(r, &c, out);
    for (int t = 0; t < ncomp; t++) tab[id * ncomp + t] = out[first + t];
  }
  return 0;
}

static void tricubic_eval(const double *tab, int n1, int ncomp, const int (*cnt)[3],
                          const double r[3], double *out) {
  double h = 0.5 / n1;
  int sgn[3], i0[3];
  double w[3][4];
  for (int d = 0; d < 3; d++) {
    double a = r[d];
    sgn[d] = a < 0.0 ? -1 : 1;
    a = fabs(a);
    double t = a / h;
    int i = (int)floor(t);
    if (i > n1 - 1) i = n1 - 1;
    if (i < 0) i = 0;
    double f = t - i;
    i0[d] = i; /* stencil nodes i-1..i+2 sit at table indices i..i+3 */
    w[d][0] = -f * (f - 1.0) * (f - 2.0) / 6.0;
    w[d][1] = (f + 1.0) * (f - 1.0) * (f - 2.0) / 2.0;
    w[d][2] = -(f + 1.0) * f * (f - 2.0) / 2.0;
    w[d][3] = (f + 1.0) * f * (f - 1.0) / 6.0;
  }
  int m = n1 + 4;
  for (int c = 0; c < ncomp; c++) out[c] = 0.0;
  for (int a = 0; a < 4; a++)
    for (int b = 0; b < 4; b++)
      for (int e = 0; e < 4; e++) {
        double ww = w[0][a] * w[1][b] * w[2][e];
        int64_t id = ((int64_t)(i0[0] + a) * m + (i0[1] + b)) * m + (i0[2] + e);
        for (int c = 0; c < ncomp; c++) out[c] += ww * tab[id * ncomp + c];
      }
  for (int c = 0; c < ncomp; c++) {
    int s = 1;
    for (int d = 0; d < 3; d++)
      if (sgn[d] < 0 && (cnt[c][d] & 1)) s = -s;
    out[c] *= s;
  }
}

/* C~ = -grad phi~ : store -d_i */
int or_ctilde_table_build(int n1, double *tab) {
  int rc = tricubic_build(n1, tab, 3, 1);
  if (rc) return rc;
  int64_t m = n1 + 4;
  for (int64_t i = 0; i < m * m * m * 3; i++) tab[i] = -tab[i];
  return 0;
}

void or_ctilde_table_eval(const double *tab, int n1, const double r[3], double out[3]) {
  tricubic_eval(tab, n1, 3, CNT, r, out);
}

/* phi~ itself on the same nodes (one value per node; even in every axis) */
int or_phitilde_table_build(int n1, double *tab) { return tricubic_build(n1, tab, 1, 0); }

void or_phitilde_table_eval(const double *tab, int n1, const double r[3], double *out) {
  static const int EVEN[1][3] = {{0, 0, 0}};
  tricubic_eval(tab, n1, 1, EVEN, r, out);
}

/* grad C~ = -d_ij phi~ : store -d_ij (xx,xy,xz,yy,yz,zz) */
int or_ctilde_grad_table_build(int n1, double *tab) {
  int rc = tricubic_build(n1, tab, 6, 4);
  if (rc) return rc;
  int64_t m = n1 + 4;
  for (int64_t i = 0; i < m * m * m * 6; i++) tab[i] = -tab[i];
  return 0;
}

void or_ctilde_grad_table_eval(const double *tab, int n1, const double r[3], double out[6]) {
  tricubic_eval(tab, n1, 6, CNT + 3, r, out);
}
