// Periodic images (Sec. 2.1: periodic boundary conditions through an
// expansion of the image field).
//
// For a source at any image r of a separation, the Ewald acceleration is
//   a_E(r) = a_N(r) + (4 pi/3) r + C~(r),   C~ = -grad phi~,
//   phi~(r) = phi_E(r) + 1/|r| + (2 pi/3)|r|^2,
// where phi_E is the Ewald potential of a unit source with the neutralising
// background (real-space erfc sum plus reciprocal-space sum).  The walk sums
// the Newton/Plummer part at the images it chose; the background term is
// summed exactly from the masses and dipoles of the fixed level-l_E cells at
// the same images; and sum_j m_j C~ is evaluated from a local expansion of
// phi~ about the group's expansion point e (a point of the lattice
// 2^-grid), built from those cells' moments at R0 = e - c* (lattice points,
// so the phi~ derivatives are exact table entries) and truncated at total
// order p_E + 1.
//
// phi~ derivatives at the lattice nodes are computed here in FP64 from the
// Ewald sums.  The Cartesian derivatives of each radial term come from the
// McMurchie-Davidson recurrence on its "ladder" f_j = ((1/r) d/dr)^j f:
// T^(j)_n = d^n f_j satisfies T^(j)_{n+e_a} = r_a T^(j+1)_n + n_a T^(j+1)_{n-e_a}
// (Leibniz on d_a f_j = r_a f_{j+1}), started from T^(j)_0 = f_j.
#include <math.h>

#include <mutex>
#include <vector>

#include "common.cuh"
#include "m2p_gen.cuh"

namespace {

constexpr int kPMax = 6;               // derivative orders in the lattice table
constexpr int kPFar = 8;               // orders of the far-lattice tensor (near-replica scheme)
constexpr int kNMMax = 165;            // multi-indices of order <= 8
// Ewald split used to build the table: screening alpha, real-space cut-off
// and reciprocal-space extent.  phi~ does not depend on the split; with these
// the neglected real-space images (alpha r >= 8.1) and wave vectors
// (|h|^2 > 27, weight e^(-pi^2 h^2 / alpha^2) < 2e-23) stay below 1e-14 of
// the order-6 derivatives.
constexpr double kAlpha = 2.5;
constexpr double kRcut = 3.25;
constexpr int kHMax = 5;
constexpr int kH2Max = 27;

__constant__ signed char c_mi[kNMMax][3];
// recurrence plan per multi-index n (order >= 1): the axis a lowered, the
// indices of n - e_a and n - 2 e_a (-1 if n_a < 2) and the order |n|
__constant__ signed char c_rax[kNMMax];
__constant__ short c_rd1[kNMMax], c_rd2[kNMMax];
__constant__ signed char c_rord[kNMMax];

// ladder of the screened image term f = erfc(alpha r)/r:
//   f_j = -((2j - 1) f_{j-1} + (2 alpha/sqrt(pi)) (-2 alpha^2)^(j-1) e^(-alpha^2 r^2)) / r^2
__device__ void screened_ladder(double r, int P, double* f) {
  const double r2 = r * r;
  const double ex = (2.0 * kAlpha / sqrt(M_PI)) * exp(-kAlpha * kAlpha * r2);
  double w = 1.0;
  f[0] = erfc(kAlpha * r) / r;
  for (int j = 1; j <= P; j++) {
    f[j] = -((2 * j - 1) * f[j - 1] + w * ex) / r2;
    w *= -2.0 * kAlpha * kAlpha;
  }
}

// ladder of the smooth n = 0 term u = erf(alpha r)/r: 1/r's ladder
// (-1)^j (2j-1)!!/r^(2j+1) minus the screened one for alpha r >= 1, else its
// power series u_j = (2 alpha/sqrt(pi)) (-2 alpha^2)^j
//                    sum_k (-alpha^2 r^2)^k / (k! (2k + 2j + 1)).
__device__ void smooth_ladder(double r, int P, double* u) {
  if (kAlpha * r >= 1.0) {
    screened_ladder(r, P, u);
    double nj = 1.0 / r;
    const double ir2 = 1.0 / (r * r);
    for (int j = 0; j <= P; j++) {
      u[j] = nj - u[j];
      nj *= -(2 * j + 1) * ir2;
    }
    return;
  }
  const double x = -kAlpha * kAlpha * r * r;
  double pre = 2.0 * kAlpha / sqrt(M_PI);
  for (int j = 0; j <= P; j++) {
    double sum = 0.0;
    for (int k = 29; k >= 0; k--) sum = sum * x / (k + 1) + 1.0 / (2 * k + 2 * j + 1);
    u[j] = pre * sum;
    pre *= -2.0 * kAlpha * kAlpha;
  }
}

// out[n] += s d^n f(|r|) for |n| <= P <= PM from the ladder f[0..P]
template <int PM>
__device__ void add_cartesian(const double r[3], const double* f, double s, int P, int nm, double* out) {
  constexpr int NM = (PM + 1) * (PM + 2) * (PM + 3) / 6;
  double T[PM + 1][NM];
  for (int j = 0; j <= P; j++) T[j][0] = f[j];
  for (int t = 1; t < nm; t++) {
    const int a = c_rax[t], d1 = c_rd1[t], d2 = c_rd2[t], o = c_rord[t];
    const double k = (double)(c_mi[t][a] - 1);
    for (int j = 0; j + o <= P; j++) T[j][t] = r[a] * T[j + 1][d1] + (d2 >= 0 ? k * T[j + 1][d2] : 0.0);
  }
  for (int t = 0; t < nm; t++) out[t] += s * T[0][t];
}

template <int PM>
__global__ void phitilde_table_kernel(int lg, int P, int nm, double* __restrict__ tab) {
  constexpr int NM = (PM + 1) * (PM + 2) * (PM + 3) / 6;
  const int m = (1 << (lg - 1)) + 2;
  const int total = m * m * m;
  const double h = ldexp(1.0, -lg);
  for (int id = blockIdx.x * blockDim.x + threadIdx.x; id < total; id += gridDim.x * blockDim.x) {
    const int i = id / (m * m), j = (id / m) % m, k = id % m;
    const double r[3] = {i * h, j * h, k * h};
    double out[NM];
    for (int t = 0; t < nm; t++) out[t] = 0.0;
    double f[PM + 1];
    // real space: every image n != 0 within the cut-off, screened
    const int nmax = (int)ceil(kRcut) + 1;
    for (int nx = -nmax; nx <= nmax; nx++)
      for (int ny = -nmax; ny <= nmax; ny++)
        for (int nz = -nmax; nz <= nmax; nz++) {
          if (nx == 0 && ny == 0 && nz == 0) continue;
          const double rho[3] = {r[0] - nx, r[1] - ny, r[2] - nz};
          const double d = sqrt(rho[0] * rho[0] + rho[1] * rho[1] + rho[2] * rho[2]);
          if (d >= kRcut) continue;
          screened_ladder(d, P, f);
          add_cartesian<PM>(rho, f, -1.0, P, nm, out);
        }
    // the n = 0 source enters as erf(alpha r)/r (1/r is not part of phi~)
    smooth_ladder(sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]), P, f);
    add_cartesian<PM>(r, f, 1.0, P, nm, out);
    // reciprocal space: -(1/pi) sum_h e^(-pi^2 h^2/alpha^2)/h^2 cos(2 pi h.r);
    // d^n cos(k.r) = k^n cos(k.r + |n| pi/2)
    for (int hx = -kHMax; hx <= kHMax; hx++)
      for (int hy = -kHMax; hy <= kHMax; hy++)
        for (int hz = -kHMax; hz <= kHMax; hz++) {
          const int h2 = hx * hx + hy * hy + hz * hz;
          if (h2 == 0 || h2 > kH2Max) continue;
          const double wgt = -exp(-M_PI * M_PI * h2 / (kAlpha * kAlpha)) / (M_PI * h2);
          double sn, cs;
          sincos(2.0 * M_PI * (hx * r[0] + hy * r[1] + hz * r[2]), &sn, &cs);
          const double kx = 2.0 * M_PI * hx, ky = 2.0 * M_PI * hy, kz = 2.0 * M_PI * hz;
          for (int t = 0; t < nm; t++) {
            double kn = wgt;
            for (int q = 0; q < c_mi[t][0]; q++) kn *= kx;
            for (int q = 0; q < c_mi[t][1]; q++) kn *= ky;
            for (int q = 0; q < c_mi[t][2]; q++) kn *= kz;
            const int o = (c_mi[t][0] + c_mi[t][1] + c_mi[t][2]) & 3;
            out[t] += kn * (o == 0 ? cs : o == 1 ? -sn : o == 2 ? -cs : sn);
          }
        }
    // the background and the split's constant: (2 pi/3)|r|^2 + pi/alpha^2
    out[0] += (2.0 * M_PI / 3.0) * (r[0] * r[0] + r[1] * r[1] + r[2] * r[2]) + M_PI / (kAlpha * kAlpha);
    if (P >= 1)
      for (int d = 0; d < 3; d++) out[1 + d] += (4.0 * M_PI / 3.0) * r[d];
    if (P >= 2) {
      out[4] += 4.0 * M_PI / 3.0;  // (2,0,0)
      out[7] += 4.0 * M_PI / 3.0;  // (0,2,0)
      out[9] += 4.0 * M_PI / 3.0;  // (0,0,2)
    }
    for (int t = 0; t < nm; t++) tab[(int64_t)id * nm + t] = out[t];
  }
}

__global__ void to_float_kernel(const double* __restrict__ a, float* __restrict__ b, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = (float)a[i];
}

// ---- per-group image field and scatter to caller order -------------------------
template <int PE> struct PE_;
#define NB_PE(PE)                                                                        \
  template <> struct PE_<PE> {                                                           \
    static constexpr int NL = kNL##PE;                                                   \
    static constexpr int NE = (PE + 1) * (PE + 2) * (PE + 3) / 6;                        \
    static constexpr int NP = (PE + 2) * (PE + 3) * (PE + 4) / 6;                        \
    template <typename T>                                                                \
    static __device__ __forceinline__ void m2l(const T* M, const T* D, T* L) {           \
      m2l_pe##PE<T>(M, D, L);                                                            \
    }                                                                                    \
    template <typename T>                                                                \
    static __device__ __forceinline__ void l2p(const T* L, T x, T y, T z, T& ax, T& ay, T& az) { \
      l2p_pe##PE<T>(L, x, y, z, ax, ay, az);                                             \
    }                                                                                    \
    template <typename T>                                                                \
    static __device__ __forceinline__ T l0(const T* M, const T* D) {                     \
      return m2l0_pe##PE<T>(M, D);                                                       \
    }                                                                                    \
    template <typename T>                                                                \
    static __device__ __forceinline__ T pot(T L0, const T* L, T x, T y, T z) {           \
      return l2pot_pe##PE<T>(L0, L, x, y, z);                                            \
    }                                                                                    \
  };
NB_PE(1)
NB_PE(2)
NB_PE(3)
NB_PE(4)
NB_PE(5)

template <typename T>
struct PerArgs {
  DevTree tr;
  const typename Vec4<T>::type* src;
  const double* fm;     // field moments (FP64), (box, cell, NE)
  const float* fm32;    // the same in FP32 (read by the FP32 M2L)
  const T* tab;         // phi~ table, nodes x NP
  int le, lg, pe;
  T* lbuf;              // per run: L (NL), V (3), M_total
  int lstride;
  const T* accw;        // walk accelerations, key order
  float* out;           // caller order
  unsigned long long* counter;
  double* out64;        // when set, FP64 output in caller order instead of out
  const T* potw;        // walk potential, key order, or null (no potential)
  float* pout;          // potential, caller order
};

__constant__ unsigned char c_par_mask[kNMMax];  // bit d set: multi-index odd in axis d

// One warp per run of groups sharing an expansion point e: the local
// expansion of the image field, the background term's V and the total mass.
// The warps step through the list of runs (not the groups), so that every
// resident warp has a run to work on.
template <typename T, int PE>
__global__ void __launch_bounds__(128) field_m2l_kernel(PerArgs<T> a) {
  constexpr int NL = PE_<PE>::NL, NE = PE_<PE>::NE, NP = PE_<PE>::NP;
  const int lane = threadIdx.x & 31;
  const DevTree& tr = a.tr;
  const int nrun = tr.cnt[2];
  const int ncp = 1 << (3 * a.le);
  const int m = (1 << (a.lg - 1)) + 2;
  const int step = 1 << (23 - a.lg);
  const T scale = (T)(1.0 / 8388608.0);
  for (int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < nrun; r += (gridDim.x * blockDim.x) >> 5) {
    const int g = NB_IDX(tr.runhead[r], tr.cnt[1], 501);
    const int4 ga = tr.gA[g];
    const int4 gd = tr.gD[g];
    const int box = ga.z;
    T L[NL];
#pragma unroll
    for (int t = 0; t < NL; t++) L[t] = (T)0;
    T vx = 0, vy = 0, vz = 0, mt = 0;
    T l0 = 0, wq = 0;  // potential only: L_0 and sum m |x* - e|^2
    unsigned long long nused = 0;
    for (int cell = lane; cell < ncp; cell += 32) {
      T M[NE];
      if constexpr (sizeof(T) == 4) {
        const float* Mc = a.fm32 + ((int64_t)box * ncp + cell) * NE;
        if (Mc[0] == 0.f) continue;
#pragma unroll
        for (int t = 0; t < NE; t++) M[t] = Mc[t];
      } else {
        const double* Mc = a.fm + ((int64_t)box * ncp + cell) * NE;
        if (Mc[0] == 0.0) continue;
#pragma unroll
        for (int t = 0; t < NE; t++) M[t] = Mc[t];
      }
      nused++;
      const int cx2 = cell_c2((int)compact3((uint64_t)cell), a.le);
      const int cy2 = cell_c2((int)compact3((uint64_t)cell >> 1), a.le);
      const int cz2 = cell_c2((int)compact3((uint64_t)cell >> 2), a.le);
      const int kx = img_shift(cx2, gd.x), ky = img_shift(cy2, gd.y), kz = img_shift(cz2, gd.z);
      const int ox = cx2 - kx * NB_PBOX - gd.x, oy = cy2 - ky * NB_PBOX - gd.y, oz = cz2 - kz * NB_PBOX - gd.z;
      // R0 = e - c* on the lattice
      const int irx = -ox / step, iry = -oy / step, irz = -oz / step;
      const int neg = (irx < 0 ? 1 : 0) | (iry < 0 ? 2 : 0) | (irz < 0 ? 4 : 0);
      const int node = NB_IDX((abs(irx) * m + abs(iry)) * m + abs(irz), m * m * m, 502);
      const T* src = a.tab + (int64_t)node * NP;
      T D[NP];
#pragma unroll
      for (int t = 0; t < NP; t++) {
        const T v = src[t];
        D[t] = (__popc(c_par_mask[t] & neg) & 1) ? -v : v;
      }
      PE_<PE>::template m2l<T>(M, D, L);
      vx += M[0] * ((T)ox * scale) + M[1];
      vy += M[0] * ((T)oy * scale) + M[2];
      vz += M[0] * ((T)oz * scale) + M[3];
      mt += M[0];
      if constexpr (PE >= 2) {
        if (a.potw) {
          // L_0, and the cell's sum of m |x* - e|^2 about its centre r = c* - e
          l0 += PE_<PE>::template l0<T>(M, D);
          const T rx = (T)ox * scale, ry = (T)oy * scale, rz = (T)oz * scale;
          wq += M[0] * fma(rx, rx, fma(ry, ry, rz * rz)) + (T)2 * fma(rx, M[1], fma(ry, M[2], rz * M[3])) +
                (M[4] + M[7] + M[9]);
        }
      }
    }
#pragma unroll
    for (int t = 0; t < NL; t++) {
      T v = L[t];
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      L[t] = v;
    }
    for (int o = 16; o > 0; o >>= 1) {
      vx += __shfl_xor_sync(0xffffffffu, vx, o);
      vy += __shfl_xor_sync(0xffffffffu, vy, o);
      vz += __shfl_xor_sync(0xffffffffu, vz, o);
      mt += __shfl_xor_sync(0xffffffffu, mt, o);
      nused += __shfl_xor_sync(0xffffffffu, nused, o);
      if (a.potw) {
        l0 += __shfl_xor_sync(0xffffffffu, l0, o);
        wq += __shfl_xor_sync(0xffffffffu, wq, o);
      }
    }
    T* dst = a.lbuf + (int64_t)NB_IDX(gd.w, tr.ngroup, 503) * a.lstride;
    for (int t = lane; t < NL; t += 32) {
      T v = L[0];
#pragma unroll
      for (int q = 1; q < NL; q++)
        if (q == t) v = L[q];
      dst[t] = v;
    }
    if (lane == 0) {
      dst[NL] = vx;
      dst[NL + 1] = vy;
      dst[NL + 2] = vz;
      dst[NL + 3] = mt;
      dst[NL + 4] = l0;
      dst[NL + 5] = wq;
      if (a.counter) atomicAdd(a.counter, nused);
    }
  }
}

// One warp per group, one sink per lane: walk acceleration + background term
// + image field, scattered to the caller's order.
template <typename T, int PE>
__global__ void __launch_bounds__(128) field_l2p_kernel(PerArgs<T> a) {
  using V4 = typename Vec4<T>::type;
  constexpr int NL = PE_<PE>::NL;
  const int lane = threadIdx.x & 31;
  const DevTree& tr = a.tr;
  const int ngroup = tr.cnt[1];
  const T scale = (T)(1.0 / 8388608.0);
  const T fourpi3 = (T)(4.0 * M_PI / 3.0);
  for (int g = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; g < ngroup; g += (gridDim.x * blockDim.x) >> 5) {
    if (tr.gact && !tr.gact[g]) continue;
    const int4 ga = tr.gA[g], gd = tr.gD[g];
    if (lane >= ga.y || !NB_IN(ga.x + lane, tr.n, 504)) continue;
    if (tr.sact && !tr.sact[ga.x + lane]) continue;
    const T* Lr = a.lbuf + (int64_t)NB_IDX(gd.w, tr.ngroup, 503) * a.lstride;
    T L[NL];
#pragma unroll
    for (int t = 0; t < NL; t++) L[t] = Lr[t];
    const T vx = Lr[NL], vy = Lr[NL + 1], vz = Lr[NL + 2], mt = Lr[NL + 3];
    const int i = ga.x + lane;
    const V4 o4 = a.src[i];
    const int4 la = tr.cA[NB_IDX(tr.sleaf[i], tr.cnt[0], 505)];
    const T dx = o4.x + (T)(la.x - gd.x) * scale;
    const T dy = o4.y + (T)(la.y - gd.y) * scale;
    const T dz = o4.z + (T)(la.z - gd.z) * scale;
    T ax = a.accw[i] + fourpi3 * (mt * dx - vx);
    T ay = a.accw[tr.n + i] + fourpi3 * (mt * dy - vy);
    T az = a.accw[2 * tr.n + i] + fourpi3 * (mt * dz - vz);
    PE_<PE>::template l2p<T>(L, dx, dy, dz, ax, ay, az);
    const uint32_t j = tr.perm[i];
    if (!NB_IN(j, tr.n, 506)) continue;
    if (a.potw) {
      // walk + image series + the background's -(2 pi/3) sum m |x - x*|^2
      const T d2 = fma(dx, dx, fma(dy, dy, dz * dz));
      const T bgq = fma(mt, d2, fma((T)-2, fma(dx, vx, fma(dy, vy, dz * vz)), Lr[NL + 5]));
      a.pout[j] = (float)(a.potw[i] + PE_<PE>::template pot<T>(Lr[NL + 4], L, dx, dy, dz) -
                          (T)(2.0 * M_PI / 3.0) * bgq);
    }
    if (a.out64) {
      a.out64[j] = (double)ax;
      a.out64[tr.n + j] = (double)ay;
      a.out64[2 * tr.n + j] = (double)az;
    } else {
      a.out[j] = (float)ax;
      a.out[tr.n + j] = (float)ay;
      a.out[2 * tr.n + j] = (float)az;
    }
  }
}

// plain scatter when there are no periodic images
template <typename T, typename O>
__global__ void scatter_kernel(int64_t n, const uint32_t* __restrict__ perm, const T* __restrict__ accw,
                               const uint8_t* __restrict__ sact, O* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    if (sact && !sact[i]) continue;
    const uint32_t j = perm[i];
    if (!NB_IN(j, n, 507)) continue;
    out[j] = (O)accw[i];
    out[n + j] = (O)accw[n + i];
    out[2 * n + j] = (O)accw[2 * n + i];
  }
}

// potential to the caller's order when there are no periodic images
template <typename T>
__global__ void scatter_pot_kernel(int64_t n, const uint32_t* __restrict__ perm, const T* __restrict__ potw,
                                   float* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    if (NB_IN(perm[i], n, 507)) out[perm[i]] = (float)potw[i];
}

// ---- the near-replica scheme's far lattice --------------------------------------------
// The walk covers the images |n|_inf <= W of every source; the images beyond
// act through one local expansion of order 8 about the box centre c0:
// L_k = sum_n ((-1)^|n|/n!) M_n T_(k+n), |k| + |n| <= 8, with the box's
// moments M about c0 and T = d^m Phi_F(0), Phi_F the periodic potential of a
// unit mass with the uniform background less its near images' -1/|r - n|.
constexpr int kNF = 165;       // multi-indices of order <= 8
constexpr int kLatParts = 512;  // slices per box of the moment sums
constexpr int kLatTile = 128;  // particles per shared-memory tile

// compensated (Kahan) addition of v to the pair (s, c)
__device__ __forceinline__ void kadd_t(float& s, float& c, float v) {
  const float y = v - c;
  const float t = s + y;
  c = (t - s) - y;
  s = t;
}

__device__ __forceinline__ int mi_idx_dev(int nx, int ny, int nz) {
  const int o = nx + ny + nz, j = ny + nz;
  return o * (o + 1) * (o + 2) / 6 + j * (j + 1) / 2 + nz;
}

// T = phi~'s derivatives at 0 (node0), the background's -(2 pi/3)|r|^2, and
// the near images' +1/|r - n| (ladder f_j = (-1)^j (2j-1)!! / r^(2j+1) at R = -n)
__global__ void lattice_tensor_kernel(const double* __restrict__ node0, int W, double* __restrict__ T) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double out[kNF];
  for (int t = 0; t < kNF; t++) out[t] = node0[t];
  out[4] -= 4.0 * M_PI / 3.0;
  out[7] -= 4.0 * M_PI / 3.0;
  out[9] -= 4.0 * M_PI / 3.0;
  double f[kPFar + 1];
  for (int nx = -W; nx <= W; nx++)
    for (int ny = -W; ny <= W; ny++)
      for (int nz = -W; nz <= W; nz++) {
        if (nx == 0 && ny == 0 && nz == 0) continue;
        const double R[3] = {(double)-nx, (double)-ny, (double)-nz};
        const double r2 = R[0] * R[0] + R[1] * R[1] + R[2] * R[2];
        f[0] = 1.0 / sqrt(r2);
        for (int j = 1; j <= kPFar; j++) f[j] = -(2 * j - 1) * f[j - 1] / r2;
        add_cartesian<kPFar>(R, f, 1.0, kPFar, kNF, out);
      }
  for (int t = 0; t < kNF; t++) T[t] = out[t];
}

// partial moments about c0 of slice blockIdx.x of box blockIdx.y; thread t
// (< 165) owns M_t and sums m x^a y^b z^c over tiles of particles whose
// coordinate powers are staged in shared memory.  T = float (the mixed
// precision mode) forms the terms in FP32 and sums them with compensation;
// T = double in FP64.
template <typename T>
__global__ void __launch_bounds__(192) lattice_moments_part_kernel(const int64_t* __restrict__ off, int64_t n,
                                                                  const double* __restrict__ spos,
                                                                  const float* __restrict__ smass,
                                                                  double* __restrict__ part) {
  __shared__ T s_p[3][kLatTile][kPFar + 1];
  __shared__ T s_m[kLatTile];
  const int b = blockIdx.y, pp = blockIdx.x, t = threadIdx.x;
  const int64_t lo = off[b], cnt = off[b + 1] - lo;
  const int64_t s0 = lo + cnt * pp / kLatParts, s1 = lo + cnt * (pp + 1) / kLatParts;
  const int a0 = t < kNF ? c_mi[t][0] : 0, a1 = t < kNF ? c_mi[t][1] : 0, a2 = t < kNF ? c_mi[t][2] : 0;
  T acc = 0, cmp = 0;
  for (int64_t i0 = s0; i0 < s1; i0 += kLatTile) {
    const int nt = (int)min((int64_t)kLatTile, s1 - i0);
    for (int k = t; k < nt; k += blockDim.x) {
      const int64_t i = i0 + k;
      s_m[k] = (T)smass[i];
      for (int d = 0; d < 3; d++) {
        const T x = (T)(spos[d * n + i] - 0.5);
        T w = 1;
        for (int e = 0; e <= kPFar; e++) {
          s_p[d][k][e] = w;
          w *= x;
        }
      }
    }
    __syncthreads();
    if (t < kNF) {
      if constexpr (sizeof(T) == 4) {
        for (int k = 0; k < nt; k++) kadd_t(acc, cmp, (s_m[k] * s_p[0][k][a0]) * (s_p[1][k][a1] * s_p[2][k][a2]));
      } else {
        for (int k = 0; k < nt; k++) acc = fma(s_m[k] * s_p[0][k][a0], s_p[1][k][a1] * s_p[2][k][a2], acc);
      }
    }
    __syncthreads();
  }
  if (t < kNF) part[((int64_t)b * kLatParts + pp) * kNF + t] = (double)acc - (double)cmp;
}

// box moments (slices summed in order: reproducible), then the local
// expansion about c0, in FP64 and in the walk's precision
template <typename T>
__global__ void lattice_m2l_kernel(const double* __restrict__ part, const double* __restrict__ Tf,
                                   double* __restrict__ M, double* __restrict__ Ld, T* __restrict__ Lt) {
  __shared__ double s_M[kNF];
  const int b = blockIdx.x, t = threadIdx.x;
  if (t < kNF) {
    double v = 0.0;
    for (int pp = 0; pp < kLatParts; pp++) v += part[((int64_t)b * kLatParts + pp) * kNF + t];
    s_M[t] = v;
    M[(int64_t)b * kNF + t] = v;
  }
  __syncthreads();
  if (t < kNF) {
    const int k0 = c_mi[t][0], k1 = c_mi[t][1], k2 = c_mi[t][2], ok = k0 + k1 + k2;
    double v = 0.0;
    for (int u = 0; u < kNF; u++) {
      const int n0 = c_mi[u][0], n1 = c_mi[u][1], n2 = c_mi[u][2], on = n0 + n1 + n2;
      if (on + ok > kPFar) continue;
      double fac = 1.0;
      for (int q = 2; q <= n0; q++) fac *= q;
      for (int q = 2; q <= n1; q++) fac *= q;
      for (int q = 2; q <= n2; q++) fac *= q;
      v += ((on & 1) ? -s_M[u] : s_M[u]) / fac * Tf[mi_idx_dev(n0 + k0, n1 + k1, n2 + k2)];
    }
    Ld[(int64_t)b * kNF + t] = v;
    Lt[(int64_t)b * kNF + t] = (T)v;
  }
}

// walk accelerations + the far lattice (a -= sum_{|u| <= 7} d^u/u! L_(u+e_k),
// d = x - c0), scattered to the caller's order; with the potential, the
// walk's plus sum_{|k| <= 8} d^k/k! L_k
template <typename T, bool POT>
__global__ void lattice_l2p_kernel(DevTree tr, const T* __restrict__ Lt, const T* __restrict__ accw,
                                   float* __restrict__ out, double* __restrict__ out64, const T* __restrict__ potw,
                                   float* __restrict__ pout) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < tr.n; i += (int64_t)gridDim.x * blockDim.x) {
    if (tr.sact && !tr.sact[i]) continue;
    const T* L = Lt + (int64_t)NB_IDX((int)tr.sbox[i], tr.nbox, 508) * kNF;
    const T dx = (T)(tr.spos[i] - 0.5), dy = (T)(tr.spos[tr.n + i] - 0.5), dz = (T)(tr.spos[2 * tr.n + i] - 0.5);
    T ax = accw[i], ay = accw[tr.n + i], az = accw[2 * tr.n + i];
    l2p_pe7<T>(L + 1, dx, dy, dz, ax, ay, az);
    const uint32_t j = tr.perm[i];
    if (!NB_IN(j, tr.n, 506)) continue;
    if (out64) {
      out64[j] = (double)ax;
      out64[tr.n + j] = (double)ay;
      out64[2 * tr.n + j] = (double)az;
    } else {
      out[j] = (float)ax;
      out[tr.n + j] = (float)ay;
      out[2 * tr.n + j] = (float)az;
    }
    if constexpr (POT) pout[j] = (float)(potw[i] + l2pot_pe7<T>(L[0], L + 1, dx, dy, dz));
  }
}

// ---- host side: term tables and cached device tables ------------------------------
int mi_index(int nx, int ny, int nz) {
  int o = nx + ny + nz, j = ny + nz;
  return o * (o + 1) * (o + 2) / 6 + j * (j + 1) / 2 + nz;
}

struct TableCache {
  int device = -1, lg = 0, P = 0;
  double* d64 = nullptr;
  float* d32 = nullptr;
};
std::mutex g_tab_mutex;
std::vector<TableCache> g_tabs;

// multi-index tables of the table build and of the image field, per device
cudaError_t upload_terms() {
  static bool done[64] = {false};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 64 && done[dev]) return cudaSuccess;
  signed char mi[kNMMax][3], rax[kNMMax], rord[kNMMax];
  short rd1[kNMMax], rd2[kNMMax];
  unsigned char pm[kNMMax];
  for (int o = 0; o <= kPFar; o++)
    for (int nx = o; nx >= 0; nx--)
      for (int ny = o - nx; ny >= 0; ny--) {
        const int nz = o - nx - ny, t = mi_index(nx, ny, nz);
        const int n[3] = {nx, ny, nz};
        mi[t][0] = (signed char)nx;
        mi[t][1] = (signed char)ny;
        mi[t][2] = (signed char)nz;
        pm[t] = (unsigned char)((nx & 1) | ((ny & 1) << 1) | ((nz & 1) << 2));
        rord[t] = (signed char)o;
        rax[t] = 0;
        rd1[t] = rd2[t] = -1;
        if (o == 0) continue;
        int a = 0;
        while (n[a] == 0) a++;
        int m1[3] = {n[0], n[1], n[2]};
        m1[a] -= 1;
        rax[t] = (signed char)a;
        rd1[t] = (short)mi_index(m1[0], m1[1], m1[2]);
        if (n[a] >= 2) {
          m1[a] -= 1;
          rd2[t] = (short)mi_index(m1[0], m1[1], m1[2]);
        }
      }
  cudaError_t e;
  if ((e = cudaMemcpyToSymbol(c_mi, mi, sizeof(mi)))) return e;
  if ((e = cudaMemcpyToSymbol(c_rax, rax, sizeof(rax)))) return e;
  if ((e = cudaMemcpyToSymbol(c_rd1, rd1, sizeof(rd1)))) return e;
  if ((e = cudaMemcpyToSymbol(c_rd2, rd2, sizeof(rd2)))) return e;
  if ((e = cudaMemcpyToSymbol(c_rord, rord, sizeof(rord)))) return e;
  if ((e = cudaMemcpyToSymbol(c_par_mask, pm, sizeof(pm)))) return e;
  if (dev < 64) done[dev] = true;
  return cudaSuccess;
}

}  // namespace

// phi~ table for (lg, P) on the current device (built once, cached until exit)
cudaError_t nb_phitilde_table(int lg, int P, const double** t64, const float** t32, cudaStream_t s) {
  std::lock_guard<std::mutex> lock(g_tab_mutex);
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e) return e;
  for (auto& c : g_tabs)
    if (c.device == dev && c.lg == lg && c.P == P) {
      *t64 = c.d64;
      *t32 = c.d32;
      return cudaSuccess;
    }
  if (P > kPMax || lg < 2 || lg > 9) return cudaErrorInvalidValue;
  if ((e = upload_terms())) return e;
  const int m = (1 << (lg - 1)) + 2;
  const int nm = (P + 1) * (P + 2) * (P + 3) / 6;
  const int64_t total = (int64_t)m * m * m * nm;
  TableCache c;
  c.device = dev;
  c.lg = lg;
  c.P = P;
  if ((e = cudaMalloc(&c.d64, sizeof(double) * total))) return e;
  if ((e = cudaMalloc(&c.d32, sizeof(float) * total))) {
    cudaFree(c.d64);
    return e;
  }
  const int nodes = m * m * m;
  phitilde_table_kernel<kPMax><<<(nodes + 63) / 64, 64, 0, s>>>(lg, P, nm, c.d64);
  to_float_kernel<<<(int)((total + 255) / 256 > 4096 ? 4096 : (total + 255) / 256), 256, 0, s>>>(c.d64, c.d32,
                                                                                                 total);
  if ((e = cudaGetLastError())) return e;
  if ((e = cudaStreamSynchronize(s))) return e;
  g_tabs.push_back(c);
  *t64 = c.d64;
  *t32 = c.d32;
  return cudaSuccess;
}

// per run of groups: L (nl), V (3), M_total, and for the potential L_0 and W
int nb_field_stride(int pe) {
  const int nl = (pe + 2) * (pe + 3) * (pe + 4) / 6 - 1;
  return (nl + 6 + 3) & ~3;
}

cudaError_t nb_periodic(const DevTree& tr, bool fp64, int pe, int le, int lg, const void* src, const double* fm,
                        const float* fm32,
                        const void* tab, void* lbuf, const void* accw, float* out, unsigned long long* counter,
                        double* out64, const void* potw, float* pout, cudaStream_t s) {
  if (pe == 0 && potw) {
    if (fp64) scatter_pot_kernel<double><<<1024, 256, 0, s>>>(tr.n, tr.perm, (const double*)potw, pout);
    else scatter_pot_kernel<float><<<1024, 256, 0, s>>>(tr.n, tr.perm, (const float*)potw, pout);
    nb_launch_counter += 1;
  }
  if (pe == 0) {
    if (out64) {
      if (fp64) scatter_kernel<double, double><<<1024, 256, 0, s>>>(tr.n, tr.perm, (const double*)accw, tr.sact, out64);
      else scatter_kernel<float, double><<<1024, 256, 0, s>>>(tr.n, tr.perm, (const float*)accw, tr.sact, out64);
    } else if (fp64) {
      scatter_kernel<double, float><<<1024, 256, 0, s>>>(tr.n, tr.perm, (const double*)accw, tr.sact, out);
    } else {
      scatter_kernel<float, float><<<1024, 256, 0, s>>>(tr.n, tr.perm, (const float*)accw, tr.sact, out);
    }
    nb_launch_counter += 1;
    return cudaGetLastError();
  }
  int grid = (int)(((int64_t)tr.ngroup * 32 + 127) / 128);
  if (grid > 152 * 64) grid = 152 * 64;
  if (grid < 1) grid = 1;
  const int ls = nb_field_stride(pe);
#define NB_PER(TT, PE)                                                                              \
  {                                                                                                 \
    PerArgs<TT> a{tr, (const typename Vec4<TT>::type*)src, fm, fm32, (const TT*)tab, le, lg, pe, (TT*)lbuf, ls, \
                  (const TT*)accw, out, counter, out64, (const TT*)potw, pout};                     \
    field_m2l_kernel<TT, PE><<<grid, 128, 0, s>>>(a);                                               \
    field_l2p_kernel<TT, PE><<<grid, 128, 0, s>>>(a);                                               \
    break;                                                                                          \
  }
  if (fp64) {
    switch (pe) {
      case 1: NB_PER(double, 1)
      case 2: NB_PER(double, 2)
      case 3: NB_PER(double, 3)
      case 4: NB_PER(double, 4)
      default: NB_PER(double, 5)
    }
  } else {
    switch (pe) {
      case 1: NB_PER(float, 1)
      case 2: NB_PER(float, 2)
      case 3: NB_PER(float, 3)
      case 4: NB_PER(float, 4)
      default: NB_PER(float, 5)
    }
  }
#undef NB_PER
  nb_launch_counter += 2;
  return cudaGetLastError();
}

// Local expansions of the image field only (one per run of groups), for the
// reverse mode, which needs them without evaluating the forces.
cudaError_t nb_field_local(const DevTree& tr, bool fp64, int pe, int le, int lg, const void* src, const double* fm,
                           const float* fm32,
                           const void* tab, void* lbuf, cudaStream_t s) {
  if (pe == 0) return cudaSuccess;
  int grid = (int)(((int64_t)tr.ngroup * 32 + 127) / 128);
  if (grid > 152 * 64) grid = 152 * 64;
  if (grid < 1) grid = 1;
  const int ls = nb_field_stride(pe);
#define NB_LOC(TT, PE)                                                                              \
  {                                                                                                 \
    PerArgs<TT> a{tr, (const typename Vec4<TT>::type*)src, fm, fm32, (const TT*)tab, le, lg, pe, (TT*)lbuf, ls, \
                  nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};                            \
    field_m2l_kernel<TT, PE><<<grid, 128, 0, s>>>(a);                                               \
    break;                                                                                          \
  }
  if (fp64) {
    switch (pe) {
      case 1: NB_LOC(double, 1)
      case 2: NB_LOC(double, 2)
      case 3: NB_LOC(double, 3)
      case 4: NB_LOC(double, 4)
      default: NB_LOC(double, 5)
    }
  } else {
    switch (pe) {
      case 1: NB_LOC(float, 1)
      case 2: NB_LOC(float, 2)
      case 3: NB_LOC(float, 3)
      case 4: NB_LOC(float, 4)
      default: NB_LOC(float, 5)
    }
  }
#undef NB_LOC
  nb_launch_counter += 1;
  return cudaGetLastError();
}

namespace {
struct LatticeCache {
  int device = -1, W = 0;
  double* T = nullptr;
};
std::mutex g_lat_mutex;
std::vector<LatticeCache> g_lats;
}  // namespace

// The far-lattice tensor for shell width W on the current device (built
// once: the order-8 derivatives of phi~ at 0, then the near images and the
// background taken out; cached until exit)
cudaError_t nb_lattice_tensor(int W, const double** out, cudaStream_t s) {
  std::lock_guard<std::mutex> lock(g_lat_mutex);
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e) return e;
  for (auto& c : g_lats)
    if (c.device == dev && c.W == W) {
      *out = c.T;
      return cudaSuccess;
    }
  if ((e = upload_terms())) return e;
  const int lg = 2, m = (1 << (lg - 1)) + 2, nodes = m * m * m;
  double* tab = nullptr;
  LatticeCache c;
  c.device = dev;
  c.W = W;
  if ((e = cudaMalloc(&tab, sizeof(double) * nodes * kNF))) return e;
  if ((e = cudaMalloc(&c.T, sizeof(double) * kNF))) {
    cudaFree(tab);
    return e;
  }
  phitilde_table_kernel<kPFar><<<1, 64, 0, s>>>(lg, kPFar, kNF, tab);  // node 0 is r = 0
  lattice_tensor_kernel<<<1, 32, 0, s>>>(tab, W, c.T);
  if (!(e = cudaGetLastError())) e = cudaStreamSynchronize(s);
  cudaFree(tab);
  if (e) {
    cudaFree(c.T);
    return e;
  }
  g_lats.push_back(c);
  *out = c.T;
  return cudaSuccess;
}

// Far lattice of the near-replica scheme after a walk: box moments (two
// fixed-order stages), the local expansion per box, and its evaluation at
// every particle added to the walk's accelerations on the way to the
// caller's order.  part: nbox * 512 * 165 doubles; mom, Ld: nbox * 165
// doubles; Lt: nbox * 165 in the walk's precision.
cudaError_t nb_lattice(const DevTree& tr, bool fp64, int W, const void* accw, float* out, double* out64,
                       const void* potw, float* pout, double* part, double* mom, double* Ld, void* Lt,
                       cudaStream_t s) {
  const double* T = nullptr;
  cudaError_t e = nb_lattice_tensor(W, &T, s);
  if (e) return e;
  if (fp64)
    lattice_moments_part_kernel<double><<<dim3(kLatParts, tr.nbox), 192, 0, s>>>(tr.off, tr.n, tr.spos, tr.smass, part);
  else
    lattice_moments_part_kernel<float><<<dim3(kLatParts, tr.nbox), 192, 0, s>>>(tr.off, tr.n, tr.spos, tr.smass, part);
  int grid = (int)((tr.n + 255) / 256);
  if (grid > 152 * 32) grid = 152 * 32;
#define NB_LAT_L2P(TT)                                                                                 \
  if (potw)                                                                                            \
    lattice_l2p_kernel<TT, true><<<grid, 256, 0, s>>>(tr, (const TT*)Lt, (const TT*)accw, out, out64,  \
                                                      (const TT*)potw, pout);                          \
  else                                                                                                 \
    lattice_l2p_kernel<TT, false><<<grid, 256, 0, s>>>(tr, (const TT*)Lt, (const TT*)accw, out, out64, \
                                                       nullptr, nullptr);
  if (fp64) {
    lattice_m2l_kernel<double><<<tr.nbox, 192, 0, s>>>(part, T, mom, Ld, (double*)Lt);
    NB_LAT_L2P(double)
  } else {
    lattice_m2l_kernel<float><<<tr.nbox, 192, 0, s>>>(part, T, mom, Ld, (float*)Lt);
    NB_LAT_L2P(float)
  }
#undef NB_LAT_L2P
  nb_launch_counter += 3;
  return cudaGetLastError();
}

// fault word of the debug build's bounds checks in this unit (debug build only)
NB_DBG_EXPORT(periodic)
