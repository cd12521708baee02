// Host-side check of the generated expansion kernels (compiled with T = double):
// each reverse-mode kernel against finite differences of its forward kernel
// or against the dot-product identity <J v, w> = <v, J^T w>.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <random>
#include <string>
#define __device__
#define __forceinline__ inline
#define __restrict__
static inline double nbody_rsqrt(double x) { return 1.0 / std::sqrt(x); }
static inline float nbody_rsqrt(float x) { return 1.0f / std::sqrt(x); }
static inline double nbody_rsqrt_pair(double x) { return 1.0 / std::sqrt(x); }
static inline float nbody_rsqrt_pair(float x) { return 1.0f / std::sqrt(x); }
using std::fma;
// host stand-ins for the packed FP32 pair operations (per component, round
// to nearest, as the device instructions are specified)
struct float2 {
  float x, y;
};
static inline float2 make_float2(float a, float b) { return float2{a, b}; }
static inline float2 __ffma2_rn(float2 a, float2 b, float2 c) {
  return float2{std::fma(a.x, b.x, c.x), std::fma(a.y, b.y, c.y)};
}
static inline float2 __fmul2_rn(float2 a, float2 b) { return float2{a.x * b.x, a.y * b.y}; }
static inline float2 __fadd2_rn(float2 a, float2 b) { return float2{a.x + b.x, a.y + b.y}; }
#include "../paper_1407_2600_gb300/csrc/m2p_gen.cuh"
#include "../paper_1407_2600_gb300/csrc/adj_gen.cuh"

static std::mt19937_64 rng(7);
static double U() { return std::uniform_real_distribution<double>(-1, 1)(rng); }
static double worst = 0;
static void check(const char* what, double got, double ref, double scale, double tol) {
  double e = std::fabs(got - ref) / (scale > 0 ? scale : 1.0);
  if (e > worst) worst = e;
  if (e > tol) {
    std::printf("FAIL %s got %.15g ref %.15g rel %.3g\n", what, got, ref, e);
    std::exit(1);
  }
}

template <int P> struct K;
#define KD(P)                                                                                         \
  template <> struct K<P> {                                                                            \
    static const int NB = kNB##P;                                                                      \
    static void fwd(const double* B, double x, double y, double z, double e, double& ax, double& ay, double& az) { \
      m2p_p##P<double>(B, x, y, z, e, ax, ay, az);                                                     \
    }                                                                                                  \
    static void self(const double* B, double x, double y, double z, double e, double lx, double ly, double lz, \
                     double& ox, double& oy, double& oz) {                                             \
      m2p_adj_self_p##P<double>(B, x, y, z, e, lx, ly, lz, ox, oy, oz);                                \
    }                                                                                                  \
    static void src(double x, double y, double z, double e, double lx, double ly, double lz, double* nu) { \
      m2p_adj_src_p##P<double>(x, y, z, e, lx, ly, lz, nu);                                            \
    }                                                                                                  \
    static void red(const double* M, double* B) { reduce_moments_p##P(M, B); }                         \
    static void p2m(double m, double x, double y, double z, double* M) { p2m_acc_p##P(m, x, y, z, M); } \
    static void padj(double m, double x, double y, double z, const double* nu, double& gx, double& gy, double& gz) { \
      p2m_adj_p##P(m, x, y, z, nu, gx, gy, gz);                                                        \
    }                                                                                                  \
    static void m2m(const double* Mc, double x, double y, double z, double* Mp) { m2m_acc_p##P(Mc, x, y, z, Mp); } \
    static double pot(const double* B, double x, double y, double z, double e) { return m2pot_p##P<double>(B, x, y, z, e); } \
    static void m2madj(const double* nup, double x, double y, double z, double* nuc) { m2m_adj_acc_p##P(nup, x, y, z, nuc); } \
  };
KD(0) KD(1) KD(2) KD(3) KD(4)

template <int P>
void fwd_scalar(const float* B, float x, float y, float z, float e, float& ax, float& ay, float& az);
template <int P> struct K2;
#define K2D(P)                                                                                               \
  template <> void fwd_scalar<P>(const float* B, float x, float y, float z, float e, float& ax, float& ay,    \
                                 float& az) {                                                               \
    m2p_p##P<float>(B, x, y, z, e, ax, ay, az);                                                             \
  }                                                                                                          \
  template <> struct K2<P> {                                                                                 \
    static void fwd2(const float2* B, float2 x, float2 y, float2 z, float2 e, float2& ax, float2& ay,        \
                     float2& az) {                                                                           \
      m2p2_p##P(B, x, y, z, e, ax, ay, az);                                                                  \
    }                                                                                                        \
    static void self1(const float* B, float x, float y, float z, float e, float lx, float ly, float lz,      \
                      float& ox, float& oy, float& oz) {                                                    \
      m2p_adj_self_p##P<float>(B, x, y, z, e, lx, ly, lz, ox, oy, oz);                                       \
    }                                                                                                        \
    static void self2(const float2* B, float2 x, float2 y, float2 z, float2 e, float2 lx, float2 ly,         \
                      float2 lz, float2& ox, float2& oy, float2& oz) {                                      \
      m2p2_adj_self_p##P(B, x, y, z, e, lx, ly, lz, ox, oy, oz);                                             \
    }                                                                                                        \
  };
K2D(0) K2D(1) K2D(2) K2D(3) K2D(4)

template <int P> void run_m2p() {
  const int NM = (P + 1) * (P + 2) * (P + 3) / 6;
  double M[NM], B[K<P>::NB];
  for (int t = 0; t < NM; t++) M[t] = U() * std::pow(0.1, t > 0);
  K<P>::red(M, B);
  double R[3] = {0.8 + 0.3 * U(), -0.6 + 0.2 * U(), 0.5 * U()}, e2 = 0.01, lam[3] = {U(), U(), U()};
  // self: J lam vs central differences of the forward acceleration along lam
  double o[3] = {0, 0, 0};
  K<P>::self(B, R[0], R[1], R[2], e2, lam[0], lam[1], lam[2], o[0], o[1], o[2]);
  double h = 1e-6, ap[3] = {0, 0, 0}, am[3] = {0, 0, 0};
  K<P>::fwd(B, R[0] + h * lam[0], R[1] + h * lam[1], R[2] + h * lam[2], e2, ap[0], ap[1], ap[2]);
  K<P>::fwd(B, R[0] - h * lam[0], R[1] - h * lam[1], R[2] - h * lam[2], e2, am[0], am[1], am[2]);
  double sc = std::fabs(o[0]) + std::fabs(o[1]) + std::fabs(o[2]);
  for (int k = 0; k < 3; k++) check("m2p_adj_self", o[k], (ap[k] - am[k]) / (2 * h), sc, 1e-7);
  // src: nu_n = d/dM_n (lam . a) through the reduction, by linearity in M
  double nu[NM];
  for (int t = 0; t < NM; t++) nu[t] = 0;
  K<P>::src(R[0], R[1], R[2], e2, lam[0], lam[1], lam[2], nu);
  // (lam . a) as a function of M is linear: derivative wrt M_n = lam . a(e_n) with the
  // moment C_n = (-1)^|n| M_n / n! folded in; nu excludes that factor
  for (int t = 0; t < NM; t++) {
    double Mt[NM], Bt[K<P>::NB], a[3] = {0, 0, 0};
    for (int q = 0; q < NM; q++) Mt[q] = (q == t);
    K<P>::red(Mt, Bt);
    K<P>::fwd(Bt, R[0], R[1], R[2], e2, a[0], a[1], a[2]);
    // undo (-1)^|n|/n!
    int o2 = 0, cnt = 0, nx = 0, ny = 0, nz = 0;
    for (int ord = 0; ord <= P; ord++)
      for (int ax = ord; ax >= 0; ax--)
        for (int ay = ord - ax; ay >= 0; ay--) {
          if (cnt == t) { o2 = ord; nx = ax; ny = ay; nz = ord - ax - ay; }
          cnt++;
        }
    double f = 1;
    for (int i = 2; i <= nx; i++) f *= i;
    for (int i = 2; i <= ny; i++) f *= i;
    for (int i = 2; i <= nz; i++) f *= i;
    double ref = (lam[0] * a[0] + lam[1] * a[1] + lam[2] * a[2]) * f * ((o2 & 1) ? -1 : 1);
    check("m2p_adj_src", nu[t], ref, 1.0 + std::fabs(ref), 1e-11);
  }
  // p2m transpose: g = d/dx (nu . M(x)) vs finite differences
  double d[3] = {0.1 * U(), 0.1 * U(), 0.1 * U()}, g[3] = {0, 0, 0}, m = 0.7;
  K<P>::padj(m, d[0], d[1], d[2], nu, g[0], g[1], g[2]);
  for (int k = 0; k < 3; k++) {
    double dp[3] = {d[0], d[1], d[2]}, dm[3] = {d[0], d[1], d[2]};
    dp[k] += h;
    dm[k] -= h;
    double Mp[NM], Mm[NM];
    for (int t = 0; t < NM; t++) Mp[t] = Mm[t] = 0;
    K<P>::p2m(m, dp[0], dp[1], dp[2], Mp);
    K<P>::p2m(m, dm[0], dm[1], dm[2], Mm);
    double ref = 0;
    for (int t = 0; t < NM; t++) ref += nu[t] * (Mp[t] - Mm[t]) / (2 * h);
    check("p2m_adj", g[k], ref, 1.0 + std::fabs(ref), 1e-7);
  }
  // m2m transpose: <m2m(Mc), w> = <Mc, m2m^T(w)>
  double Mc[NM], w[NM], Mp2[NM], adj[NM], s[3] = {0.05 * U(), 0.05 * U(), 0.05 * U()};
  for (int t = 0; t < NM; t++) {
    Mc[t] = U();
    w[t] = U();
    Mp2[t] = 0;
    adj[t] = 0;
  }
  K<P>::m2m(Mc, s[0], s[1], s[2], Mp2);
  K<P>::m2madj(w, s[0], s[1], s[2], adj);
  double l = 0, r = 0;
  for (int t = 0; t < NM; t++) {
    l += Mp2[t] * w[t];
    r += Mc[t] * adj[t];
  }
  check("m2m_adj", l, r, 1.0 + std::fabs(l), 1e-13);
}

template <int PE> struct F;
#define FD(PE)                                                                                       \
  template <> struct F<PE> {                                                                          \
    static const int NL = kNL##PE;                                                                    \
    static void m2l(const double* M, const double* D, double* L) { m2l_pe##PE<double>(M, D, L); }     \
    static void l2p(const double* L, double x, double y, double z, double& ax, double& ay, double& az) { \
      l2p_pe##PE<double>(L, x, y, z, ax, ay, az);                                                     \
    }                                                                                                 \
    static void hess(const double* L, double x, double y, double z, double lx, double ly, double lz, double& ox, \
                     double& oy, double& oz) {                                                        \
      l2p_hess_pe##PE<double>(L, x, y, z, lx, ly, lz, ox, oy, oz);                                    \
    }                                                                                                 \
    static void ladj(double x, double y, double z, double lx, double ly, double lz, double* Lb) {     \
      l2p_adj_pe##PE<double>(x, y, z, lx, ly, lz, Lb);                                                \
    }                                                                                                 \
    static void madj(const double* Lb, const double* D, double* nu) { m2l_adj_pe##PE<double>(Lb, D, nu); } \
    static double l0(const double* M, const double* D) { return m2l0_pe##PE<double>(M, D); }            \
    static double pot(double L0, const double* L, double x, double y, double z) {                      \
      return l2pot_pe##PE<double>(L0, L, x, y, z);                                                    \
    }                                                                                                 \
  };
FD(1) FD(2) FD(3) FD(4) FD(5)

template <int PE> void run_field() {
  const int NL = F<PE>::NL, NE = (PE + 1) * (PE + 2) * (PE + 3) / 6, NP = (PE + 2) * (PE + 3) * (PE + 4) / 6;
  double L[NL], d[3] = {0.02 * U(), 0.02 * U(), 0.02 * U()}, lam[3] = {U(), U(), U()}, h = 1e-6;
  for (int t = 0; t < NL; t++) L[t] = U();
  double o[3] = {0, 0, 0}, ap[3] = {0, 0, 0}, am[3] = {0, 0, 0};
  F<PE>::hess(L, d[0], d[1], d[2], lam[0], lam[1], lam[2], o[0], o[1], o[2]);
  F<PE>::l2p(L, d[0] + h * lam[0], d[1] + h * lam[1], d[2] + h * lam[2], ap[0], ap[1], ap[2]);
  F<PE>::l2p(L, d[0] - h * lam[0], d[1] - h * lam[1], d[2] - h * lam[2], am[0], am[1], am[2]);
  for (int k = 0; k < 3; k++) check("l2p_hess", o[k], (ap[k] - am[k]) / (2 * h), 1.0, 1e-7);
  // cotangent of L: lam . l2p(L) is linear in L
  double Lb[NL];
  for (int t = 0; t < NL; t++) Lb[t] = 0;
  F<PE>::ladj(d[0], d[1], d[2], lam[0], lam[1], lam[2], Lb);
  for (int t = 0; t < NL; t++) {
    double E[NL], a[3] = {0, 0, 0};
    for (int q = 0; q < NL; q++) E[q] = (q == t);
    F<PE>::l2p(E, d[0], d[1], d[2], a[0], a[1], a[2]);
    check("l2p_adj", Lb[t], lam[0] * a[0] + lam[1] * a[1] + lam[2] * a[2], 1.0, 1e-13);
  }
  // transposed M2L: <m2l(M), Lb> = <M, m2l^T(Lb)>
  double M[NE], D[NP], L2[NL], nu[NE];
  for (int t = 0; t < NE; t++) { M[t] = U(); nu[t] = 0; }
  for (int t = 0; t < NP; t++) D[t] = U();
  for (int t = 0; t < NL; t++) L2[t] = 0;
  F<PE>::m2l(M, D, L2);
  F<PE>::madj(Lb, D, nu);
  double l = 0, r = 0;
  for (int t = 0; t < NL; t++) l += L2[t] * Lb[t];
  for (int t = 0; t < NE; t++) r += M[t] * nu[t];
  check("m2l_adj", l, r, 1.0 + std::fabs(l), 1e-12);
}

// the packed two-cell M2P gives, per half, the scalar FP32 M2P bit for bit
template <int P>
void run_m2p2() {
  constexpr int NB = K<P>::NB;
  float B0[NB], B1[NB];
  float2 B2[NB];
  for (int t = 0; t < NB; t++) {
    B0[t] = (float)U();
    B1[t] = (float)U();
    B2[t] = make_float2(B0[t], B1[t]);
  }
  const float x0 = (float)(2 * U()), y0 = (float)(2 * U()), z0 = (float)(2 * U());
  const float x1 = (float)(2 * U()), y1 = (float)(2 * U()), z1 = (float)(2 * U());
  const float e0 = 0.01f, e1 = 0.02f;
  float ax0 = 0.25f, ay0 = -0.5f, az0 = 0.125f, ax1 = 0.25f, ay1 = -0.5f, az1 = 0.125f;
  float2 ax = make_float2(ax0, ax1), ay = make_float2(ay0, ay1), az = make_float2(az0, az1);
  fwd_scalar<P>(B0, x0, y0, z0, e0, ax0, ay0, az0);
  fwd_scalar<P>(B1, x1, y1, z1, e1, ax1, ay1, az1);
  K2<P>::fwd2(B2, make_float2(x0, x1), make_float2(y0, y1), make_float2(z0, z1), make_float2(e0, e1), ax, ay, az);
  if (ax.x != ax0 || ay.x != ay0 || az.x != az0 || ax.y != ax1 || ay.y != ay1 || az.y != az1) {
    std::printf("FAIL m2p2_p%d differs from m2p_p%d\n", P, P);
    std::exit(1);
  }
  // the packed reverse-mode sink term likewise (two cells, one sink's lambda)
  const float lx = (float)U(), ly = (float)U(), lz = (float)U();
  float ox0 = 0.5f, oy0 = 0.25f, oz0 = -1.0f, ox1 = 0.5f, oy1 = 0.25f, oz1 = -1.0f;
  float2 ox = make_float2(ox0, ox1), oy = make_float2(oy0, oy1), oz = make_float2(oz0, oz1);
  K2<P>::self1(B0, x0, y0, z0, e0, lx, ly, lz, ox0, oy0, oz0);
  K2<P>::self1(B1, x1, y1, z1, e1, lx, ly, lz, ox1, oy1, oz1);
  K2<P>::self2(B2, make_float2(x0, x1), make_float2(y0, y1), make_float2(z0, z1), make_float2(e0, e1),
               make_float2(lx, lx), make_float2(ly, ly), make_float2(lz, lz), ox, oy, oz);
  if (ox.x != ox0 || oy.x != oy0 || oz.x != oz0 || ox.y != ox1 || oy.y != oy1 || oz.y != oz1) {
    std::printf("FAIL m2p2_adj_self_p%d differs from m2p_adj_self_p%d\n", P, P);
    std::exit(1);
  }
}

// uniform-background terms: the Hessian-vector products against central
// differences of the forward terms, and the packed FP32 terms bit for bit per
// lane against the scalar FP32 terms
template <int L> struct BG;
#define BGD(L)                                                                                       \
  template <> struct BG<L> {                                                                          \
    template <typename T> static void f(T q, T x, T y, T z, T& ax, T& ay, T& az) {                    \
      cube_bg_l##L<T>(q, x, y, z, ax, ay, az);                                                        \
    }                                                                                                 \
    static void f2(float2 q, float2 x, float2 y, float2 z, float2& ax, float2& ay, float2& az) {      \
      cube_bg2_l##L(q, x, y, z, ax, ay, az);                                                          \
    }                                                                                                 \
    static void hvp(double q, double x, double y, double z, double lx, double ly, double lz, double& ox, \
                    double& oy, double& oz) {                                                         \
      cube_bg_hvp_l##L<double>(q, x, y, z, lx, ly, lz, ox, oy, oz);                                   \
    }                                                                                                 \
  };
BGD(4)
BGD(6)

template <int L> void run_bg() {
  double R[3];
  do {  // outside the unit cube's circumscribed sphere, where the series holds
    for (int d = 0; d < 3; d++) R[d] = 3 * U();
  } while (R[0] * R[0] + R[1] * R[1] + R[2] * R[2] < 1.0);
  const double q = 1.0 + 0.5 * U(), lam[3] = {U(), U(), U()}, h = 1e-6;
  double o[3] = {0, 0, 0}, ap[3] = {0, 0, 0}, am[3] = {0, 0, 0};
  BG<L>::hvp(q, R[0], R[1], R[2], lam[0], lam[1], lam[2], o[0], o[1], o[2]);
  BG<L>::template f<double>(q, R[0] + h * lam[0], R[1] + h * lam[1], R[2] + h * lam[2], ap[0], ap[1], ap[2]);
  BG<L>::template f<double>(q, R[0] - h * lam[0], R[1] - h * lam[1], R[2] - h * lam[2], am[0], am[1], am[2]);
  const double scale = std::fabs(o[0]) + std::fabs(o[1]) + std::fabs(o[2]);
  for (int k = 0; k < 3; k++) check(L == 4 ? "bg_hvp_l4" : "bg_hvp_l6", o[k], (ap[k] - am[k]) / (2 * h), scale, 1e-6);
  float x[2], y[2], z[2], qq[2] = {(float)(1.0 + 0.5 * U()), (float)(1.0 + 0.5 * U())};
  for (int c = 0; c < 2; c++) {
    do {
      x[c] = (float)(3 * U());
      y[c] = (float)(3 * U());
      z[c] = (float)(3 * U());
    } while (x[c] * x[c] + y[c] * y[c] + z[c] * z[c] < 1.0f);
  }
  float a[2][3] = {{0.25f, -0.5f, 0.125f}, {0.25f, -0.5f, 0.125f}};
  for (int c = 0; c < 2; c++) BG<L>::template f<float>(qq[c], x[c], y[c], z[c], a[c][0], a[c][1], a[c][2]);
  float2 ax = make_float2(0.25f, 0.25f), ay = make_float2(-0.5f, -0.5f), az = make_float2(0.125f, 0.125f);
  BG<L>::f2(make_float2(qq[0], qq[1]), make_float2(x[0], x[1]), make_float2(y[0], y[1]), make_float2(z[0], z[1]),
            ax, ay, az);
  if (ax.x != a[0][0] || ay.x != a[0][1] || az.x != a[0][2] || ax.y != a[1][0] || ay.y != a[1][1] ||
      az.y != a[1][2]) {
    std::printf("FAIL cube_bg2_l%d differs from cube_bg_l%d\n", L, L);
    std::exit(1);
  }
}

// one case from stdin for a comparison with the oracle: "p k", then k lines
// "m dx dy dz" (particles relative to the cell centre), then "Rx Ry Rz eps
// sx sy sz"; prints the moments from p2m_acc, the acceleration of m2p on the
// reduced moments at R, and the moments shifted by m2m_acc with s = c_child
// - c_parent, one value per line
template <int P> void run_io() {
  const int NM = (P + 1) * (P + 2) * (P + 3) / 6;
  int k = 0;
  if (std::scanf("%d", &k) != 1) std::exit(2);
  double M[NM], Mp[NM], B[K<P>::NB];
  for (int t = 0; t < NM; t++) M[t] = Mp[t] = 0.0;
  for (int i = 0; i < k; i++) {
    double m, x, y, z;
    if (std::scanf("%lf %lf %lf %lf", &m, &x, &y, &z) != 4) std::exit(2);
    K<P>::p2m(m, x, y, z, M);
  }
  double R[3], eps, sh[3];
  if (std::scanf("%lf %lf %lf %lf %lf %lf %lf", &R[0], &R[1], &R[2], &eps, &sh[0], &sh[1], &sh[2]) != 7) std::exit(2);
  K<P>::red(M, B);
  double a[3] = {0, 0, 0};
  K<P>::fwd(B, R[0], R[1], R[2], eps * eps, a[0], a[1], a[2]);
  K<P>::m2m(M, sh[0], sh[1], sh[2], Mp);
  for (int t = 0; t < NM; t++) std::printf("%.17g\n", M[t]);
  for (int d = 0; d < 3; d++) std::printf("%.17g\n", a[d]);
  for (int t = 0; t < NM; t++) std::printf("%.17g\n", Mp[t]);
  std::printf("%.17g\n", K<P>::pot(B, R[0], R[1], R[2], eps * eps));
}

// one image-field case from stdin: NE source moments M (orders <= pe about
// the source centre), NP derivatives D of phi~ at R0 (orders <= pe + 1), the
// sink offset d from the expansion point; prints the L2P acceleration of the
// M2L local expansion, one value per line
template <int PE> void run_field_io() {
  const int NE = (PE + 1) * (PE + 2) * (PE + 3) / 6, NP = (PE + 2) * (PE + 3) * (PE + 4) / 6;
  double M[NE], D[NP], L[F<PE>::NL], d[3];
  for (int t = 0; t < NE; t++)
    if (std::scanf("%lf", &M[t]) != 1) std::exit(2);
  for (int t = 0; t < NP; t++)
    if (std::scanf("%lf", &D[t]) != 1) std::exit(2);
  for (int k = 0; k < 3; k++)
    if (std::scanf("%lf", &d[k]) != 1) std::exit(2);
  for (int t = 0; t < F<PE>::NL; t++) L[t] = 0.0;
  F<PE>::m2l(M, D, L);
  double a[3] = {0, 0, 0};
  F<PE>::l2p(L, d[0], d[1], d[2], a[0], a[1], a[2]);
  for (int k = 0; k < 3; k++) std::printf("%.17g\n", a[k]);
  std::printf("%.17g\n", F<PE>::pot(F<PE>::l0(M, D), L, d[0], d[1], d[2]));
}

// the dual form's cell-group interaction: moments (nmom(P)), R, eps and the
// sink offset d read from stdin; prints the derivative tensor of g at R
// (orders <= P + 1) and the acceleration at d of the local expansion about z
template <int P> void dtens(double x, double y, double z, double e2, double* D);
template <> void dtens<1>(double x, double y, double z, double e2, double* D) { dtensor_p2<double>(x, y, z, e2, D); }
template <> void dtens<2>(double x, double y, double z, double e2, double* D) { dtensor_p3<double>(x, y, z, e2, D); }
template <> void dtens<3>(double x, double y, double z, double e2, double* D) { dtensor_p4<double>(x, y, z, e2, D); }
template <> void dtens<4>(double x, double y, double z, double e2, double* D) { dtensor_p5<double>(x, y, z, e2, D); }
struct MAcc {
  const double* m;
  double operator[](int u) const { return m[u]; }
};
template <int P> void l2pd(const double* L, double x, double y, double z, double& ax, double& ay, double& az);
#define DUAL_DISPATCH(P)                                                                         \
  template <> void l2pd<P>(const double* L, double x, double y, double z, double& ax, double& ay, double& az) { \
    l2p_pe##P<double>(L, x, y, z, ax, ay, az);                                                    \
  }
DUAL_DISPATCH(1)
DUAL_DISPATCH(2)
DUAL_DISPATCH(3)
DUAL_DISPATCH(4)

template <int P> void run_dual_io() {
  const int NM = (P + 1) * (P + 2) * (P + 3) / 6, NP = (P + 2) * (P + 3) * (P + 4) / 6;
  double M[35], R[3], eps, d[3], D[56], L[55];
  for (int t = 0; t < NM; t++)
    if (std::scanf("%lf", &M[t]) != 1) std::exit(2);
  for (int k = 0; k < 3; k++)
    if (std::scanf("%lf", &R[k]) != 1) std::exit(2);
  if (std::scanf("%lf", &eps) != 1) std::exit(2);
  for (int k = 0; k < 3; k++)
    if (std::scanf("%lf", &d[k]) != 1) std::exit(2);
  dtens<P>(R[0], R[1], R[2], eps * eps, D);
  for (int t = 0; t < NP; t++) std::printf("%.17g\n", D[t]);
  for (int t = 0; t < NP; t++) D[t] = -D[t];  // the image-field L2P subtracts: feed it -d g
  for (int t = 0; t < NP - 1; t++) L[t] = 0.0;
  const MAcc acc{M};
  auto red = [&](int t, int, double v) { L[t] += v; };
  if constexpr (P == 1) m2l_red_p1<double>(acc, D, red);
  if constexpr (P == 2) m2l_red_p2<double>(acc, D, red);
  if constexpr (P == 3) m2l_red_p3<double>(acc, D, red);
  if constexpr (P == 4) m2l_red_p4<double>(acc, D, red);
  double a[3] = {0, 0, 0};
  l2pd<P>(L, d[0], d[1], d[2], a[0], a[1], a[2]);
  for (int k = 0; k < 3; k++) std::printf("%.17g\n", a[k]);
}

int main(int argc, char** argv) {
  if (argc > 1 && std::string(argv[1]) == "dual") {
    int p = -1;
    if (std::scanf("%d", &p) != 1) return 2;
    switch (p) {
      case 1: run_dual_io<1>(); break;
      case 2: run_dual_io<2>(); break;
      case 3: run_dual_io<3>(); break;
      case 4: run_dual_io<4>(); break;
      default: return 2;
    }
    return 0;
  }
  if (argc > 1 && std::string(argv[1]) == "field") {
    int pe = -1;
    if (std::scanf("%d", &pe) != 1) return 2;
    switch (pe) {
      case 1: run_field_io<1>(); break;
      case 2: run_field_io<2>(); break;
      case 3: run_field_io<3>(); break;
      case 4: run_field_io<4>(); break;
      case 5: run_field_io<5>(); break;
      default: return 2;
    }
    return 0;
  }
  if (argc > 1 && std::string(argv[1]) == "io") {
    int p = -1;
    if (std::scanf("%d", &p) != 1) return 2;
    switch (p) {
      case 0: run_io<0>(); break;
      case 1: run_io<1>(); break;
      case 2: run_io<2>(); break;
      case 3: run_io<3>(); break;
      case 4: run_io<4>(); break;
      default: return 2;
    }
    return 0;
  }
  if (argc > 1 && std::string(argv[1]) == "bg") {
    // the background terms of a unit cube of unit density at the points read
    // from stdin ("x y z" per line): order-4 and order-6 accelerations
    double x, y, z;
    while (std::scanf("%lf %lf %lf", &x, &y, &z) == 3) {
      double a4[3] = {0, 0, 0}, a6[3] = {0, 0, 0};
      cube_bg_l4<double>(1.0, x, y, z, a4[0], a4[1], a4[2]);
      cube_bg_l6<double>(1.0, x, y, z, a6[0], a6[1], a6[2]);
      std::printf("%.17g %.17g %.17g %.17g %.17g %.17g %.17g %.17g\n", a4[0], a4[1], a4[2], a6[0], a6[1], a6[2],
                  cube_bgpot_l4<double>(1.0, x, y, z), cube_bgpot_l6<double>(1.0, x, y, z));
    }
    return 0;
  }
  for (int rep = 0; rep < 50; rep++) {
    run_bg<4>();
    run_bg<6>();
  }
  for (int rep = 0; rep < 50; rep++) {
    run_m2p2<0>(); run_m2p2<1>(); run_m2p2<2>(); run_m2p2<3>(); run_m2p2<4>();
  }
  for (int rep = 0; rep < 20; rep++) {
    run_m2p<0>(); run_m2p<1>(); run_m2p<2>(); run_m2p<3>(); run_m2p<4>();
    run_field<1>(); run_field<2>(); run_field<3>(); run_field<4>(); run_field<5>();
  }
  std::printf("OK worst %.3g\n", worst);
  return 0;
}
