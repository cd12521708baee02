/*
 * Oracle O1: FP64 direct summation over all pairs with Ewald images
 * (TEST INFRASTRUCTURE ONLY; see oracle.h).
 *
 *   a_i = sum_{j != i} m_j [ a_E(r_ij) - a_N(r*_ij) + a_P(r*_ij) ]
 *
 * r_ij = x_i - x_j, r* its minimum image, a_N(r) = -r/|r|^3 (Newton),
 * a_P(r) = -r/(|r|^2 + eps^2)^(3/2) (Plummer).  The unsoftened periodic force
 * comes from Ewald; Plummer softening replaces Newton for the nearest image
 * only.  With the tricubic table, a_E(r) - a_N(r*) = (4 pi/3) r* + C~(r*).
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>

static const double PI = 3.14159265358979323846264338327950288;

static inline double min_image(double d) { return d - floor(d + 0.5); }

double or_soft_factor(double r2, double eps, int kernel) {
  if (kernel == 1) {
    double x2 = r2 / (eps * eps);
    if (x2 < 1.0) return (175.0 / 16.0 - (147.0 / 8.0) * x2 + (135.0 / 16.0) * x2 * x2) / (eps * eps * eps);
    return 1.0 / (r2 * sqrt(r2));
  }
  double s = r2 + eps * eps;
  return 1.0 / (s * sqrt(s));
}

double or_soft_pot(double r2, double eps, int kernel) {
  if (kernel == 1) {
    double x2 = r2 / (eps * eps);
    if (x2 < 1.0)
      return -(105.0 / 32.0 - (175.0 / 32.0) * x2 + (147.0 / 32.0) * x2 * x2 - (45.0 / 32.0) * x2 * x2 * x2) / eps;
    return -1.0 / sqrt(r2);
  }
  return -1.0 / sqrt(r2 + eps * eps);
}

/* phi_i = sum_{j != i} m_j [phi_E(r_ij) + 1/|r*| + s(r*)] + m_i phi~(0):
 * the Ewald potential (zero-mean convention) with the nearest image softened
 * (s the softened pair potential of or_soft_pot), plus each particle's
 * interaction with its own images and the background.  phi_E + 1/|r| =
 * phi~ - (2 pi/3)|r|^2 for the nearest image r*; phi~ from the exact Ewald
 * sum (ptab NULL) or the tricubic table of or_phitilde_table_build. */
int or_direct_pot(int64_t n, const double *pos, const double *mass, double eps, int kernel,
                  int64_t ntarget, const int64_t *targets, const double *ptab, int n1, double *pot) {
  if (n <= 0) return 0;
  if (kernel < 0 || kernel > 1) return -1;
  const double *X = pos, *Y = pos + n, *Z = pos + 2 * n;
  int64_t nt = targets ? ntarget : n;
  or_ewald_cfg cfg;
  or_ewald_default(&cfg);
  double zero[3] = {0.0, 0.0, 0.0}, d0[20];
  or_phitilde(zero, &cfg, d0);
#pragma omp parallel for schedule(dynamic, 4)
  for (int64_t t = 0; t < nt; t++) {
    int64_t i = targets ? targets[t] : t;
    double v = (mass ? mass[i] : 1.0 / (double)n) * d0[0];
    for (int64_t j = 0; j < n; j++) {
      if (j == i) continue;
      double mj = mass ? mass[j] : 1.0 / (double)n;
      double rs[3] = {min_image(X[i] - X[j]), min_image(Y[i] - Y[j]), min_image(Z[i] - Z[j])};
      double q2 = rs[0] * rs[0] + rs[1] * rs[1] + rs[2] * rs[2];
      double pt;
      if (ptab) {
        or_phitilde_table_eval(ptab, n1, rs, &pt);
      } else {
        double dd[20];
        or_phitilde(rs, &cfg, dd);
        pt = dd[0];
      }
      v += mj * (pt - (2.0 * PI / 3.0) * q2 + or_soft_pot(q2, eps, kernel));
    }
    pot[t] = v;
  }
  return 0;
}

int or_direct_forces(int64_t n, const double *pos, const double *mass, double eps,
                     int64_t ntarget, const int64_t *targets, const double *ctab, int n1,
                     double *acc) {
  return or_direct_forces_k(n, pos, mass, eps, 0, ntarget, targets, ctab, n1, acc);
}

int or_direct_forces_k(int64_t n, const double *pos, const double *mass, double eps, int kernel,
                       int64_t ntarget, const int64_t *targets, const double *ctab, int n1,
                       double *acc) {
  if (n <= 0) return 0;
  if (kernel < 0 || kernel > 1) return -1;
  const double *X = pos, *Y = pos + n, *Z = pos + 2 * n;
  int64_t nt = targets ? ntarget : n;
  or_ewald_cfg cfg;
  or_ewald_default(&cfg);
#pragma omp parallel for schedule(dynamic, 4)
  for (int64_t t = 0; t < nt; t++) {
    int64_t i = targets ? targets[t] : t;
    double ax = 0.0, ay = 0.0, az = 0.0;
    for (int64_t j = 0; j < n; j++) {
      if (j == i) continue;
      double mj = mass ? mass[j] : 1.0 / (double)n;
      double r[3] = {X[i] - X[j], Y[i] - Y[j], Z[i] - Z[j]};
      double rs[3] = {min_image(r[0]), min_image(r[1]), min_image(r[2])};
      double q2 = rs[0] * rs[0] + rs[1] * rs[1] + rs[2] * rs[2];
      double fp = or_soft_factor(q2, eps, kernel);
      double k[3];
      if (ctab) {
        double ct[3];
        or_ctilde_table_eval(ctab, n1, rs, ct);
        for (int d = 0; d < 3; d++) k[d] = -rs[d] * fp + (4.0 * PI / 3.0) * rs[d] + ct[d];
      } else {
        double ae[3];
        or_ewald_acc(r, &cfg, ae);
        double fn = 1.0 / (q2 * sqrt(q2));
        for (int d = 0; d < 3; d++) k[d] = ae[d] + rs[d] * fn - rs[d] * fp;
      }
      ax += mj * k[0];
      ay += mj * k[1];
      az += mj * k[2];
    }
    acc[t] = ax;
    acc[nt + t] = ay;
    acc[2 * nt + t] = az;
  }
  return 0;
}

/* out_j = sum_{i != j} grad K(r_ij) (m_i lam_j - m_j lam_i),
 * K(r) = a_P(r*) + (4 pi/3) r* + C~(r*), grad K symmetric and even in r.
 * grad C~ = -d_ij phi~ comes from the tricubic table gtab, or, with gtab
 * NULL, from the exact Ewald derivatives of phi~ at r*. */
int or_direct_vjp(int64_t n, const double *pos, const double *mass, double eps,
                  const double *gtab, int n1, const double *lam, double *out) {
  if (n <= 0) return 0;
  const double *X = pos, *Y = pos + n, *Z = pos + 2 * n;
  double e2 = eps * eps;
  or_ewald_cfg cfg;
  or_ewald_default(&cfg);
  static const int I2[6][2] = {{0, 0}, {0, 1}, {0, 2}, {1, 1}, {1, 2}, {2, 2}};
#pragma omp parallel for schedule(dynamic, 4)
  for (int64_t j = 0; j < n; j++) {
    double o[3] = {0.0, 0.0, 0.0};
    double mj = mass ? mass[j] : 1.0 / (double)n;
    double lj[3] = {lam[j], lam[n + j], lam[2 * n + j]};
    for (int64_t i = 0; i < n; i++) {
      if (i == j) continue;
      double mi = mass ? mass[i] : 1.0 / (double)n;
      double rs[3] = {min_image(X[i] - X[j]), min_image(Y[i] - Y[j]), min_image(Z[i] - Z[j])};
      double q2 = rs[0] * rs[0] + rs[1] * rs[1] + rs[2] * rs[2];
      double s = q2 + e2;
      double is3 = 1.0 / (s * sqrt(s)), is5 = is3 / s;
      double g6[6];
      if (gtab) {
        or_ctilde_grad_table_eval(gtab, n1, rs, g6);
      } else {
        double d10[10]; /* multi-indices |m| <= 2; 4..9 = xx, xy, xz, yy, yz, zz */
        or_phitilde_mi(rs, &cfg, 2, d10);
        for (int t = 0; t < 6; t++) g6[t] = -d10[4 + t];
      }
      double G[3][3];
      for (int t = 0; t < 6; t++) {
        int a = I2[t][0], b = I2[t][1];
        double v = -(a == b ? is3 : 0.0) + 3.0 * rs[a] * rs[b] * is5 + (a == b ? 4.0 * PI / 3.0 : 0.0) +
                   g6[t];
        G[a][b] = v;
        G[b][a] = v;
      }
      double li[3] = {lam[i], lam[n + i], lam[2 * n + i]};
      double v[3] = {mi * lj[0] - mj * li[0], mi * lj[1] - mj * li[1], mi * lj[2] - mj * li[2]};
      for (int a = 0; a < 3; a++) o[a] += G[a][0] * v[0] + G[a][1] * v[1] + G[a][2] * v[2];
    }
    out[j] = o[0];
    out[n + j] = o[1];
    out[2 * n + j] = o[2];
  }
  return 0;
}
