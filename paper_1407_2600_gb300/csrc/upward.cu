// Upward pass: cell multipole moments (Sec. 2.1: cells carry a truncated
// multipole expansion that stands in for their bodies).
//
// Moments M_n = sum_j m_j (x_j - c)^n, |n| <= p, about the geometric cell
// centre c, in FP64.  Leaves are formed directly from their particles (P2M);
// a parent is formed from its daughters by the binomial shift (M2M) by the
// thread whose daughter finishes last (an arrival counter per cell), so the
// whole pass is one launch with no waiting.  Each finished cell also stores
// its reduced M2P coefficients in the walk's precision.
//
// The image field uses the moments (order p_E) of the fixed level-l_E key
// prefixes of each box, formed here by one block per prefix.
#include "common.cuh"
#include "m2p_gen.cuh"

namespace {

template <int P> struct Ord;
#define NB_ORD(P)                                                                                  \
  template <> struct Ord<P> {                                                                      \
    static constexpr int NM = (P + 1) * (P + 2) * (P + 3) / 6;                                     \
    static constexpr int NB = kNB##P;                                                              \
    static constexpr int NBS = (kNB##P + 3) & ~3;                                                  \
    static __device__ __forceinline__ void p2m(double m, double x, double y, double z, double* M) { \
      p2m_acc_p##P(m, x, y, z, M);                                                                 \
    }                                                                                              \
    static __device__ __forceinline__ void m2m(const double* Mc, double x, double y, double z,     \
                                               double* Mp) {                                       \
      m2m_acc_p##P(Mc, x, y, z, Mp);                                                               \
    }                                                                                              \
    static __device__ __forceinline__ void reduce(const double* M, double* B) {                   \
      reduce_moments_p##P(M, B);                                                                   \
    }                                                                                              \
  };
NB_ORD(0)
NB_ORD(1)
NB_ORD(2)
NB_ORD(3)
NB_ORD(4)

// Reduced coefficients in the cell's own length unit h = 2^-level: with
// R' = R/h and eps' = eps/h the expansion terms are O(1) for every accepted
// cell (R' >= 1/theta), so FP32 intermediates cannot overflow however deep the
// cell; a = h^-2 sum(...) is folded into the coefficients as B'' =
// h^-2 B(M_n h^-|n|).  All scalings are exact powers of two.
template <int P, typename T>
__device__ __forceinline__ void finish_cell(int c, int level, const double* M, T* __restrict__ coef) {
  constexpr int NM = Ord<P>::NM;
  double Ms[NM];
  int t = 0;
#pragma unroll
  for (int o = 0; o <= P; o++) {
    const double sc = ldexp(1.0, level * o);
#pragma unroll
    for (int q = 0; q < (o + 1) * (o + 2) / 2; q++, t++) Ms[t] = M[t] * sc;
  }
  double B[Ord<P>::NB];
  Ord<P>::reduce(Ms, B);
  T* dst = coef + (int64_t)c * Ord<P>::NBS;
  const double s2 = ldexp(1.0, 2 * level);
#pragma unroll
  for (int q = 0; q < Ord<P>::NB; q++) dst[q] = (T)(B[q] * s2);
#pragma unroll
  for (int q = Ord<P>::NB; q < Ord<P>::NBS; q++) dst[q] = (T)0;
}

template <int P, typename T>
__global__ void __launch_bounds__(128)
upward_kernel(int ncell, const int4* __restrict__ cA, const int4* __restrict__ cB,
              const double* __restrict__ spos, const float* __restrict__ smass, int64_t n,
              double* __restrict__ mom, int* __restrict__ arrive, T* __restrict__ coef) {
  constexpr int NM = Ord<P>::NM;
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < ncell; b += gridDim.x * blockDim.x) {
    int4 a = cA[b];
    if ((a.w >> 8) != 0) continue;  // only leaves start a climb
    int4 r = cB[b];
    double M[NM];
#pragma unroll
    for (int t = 0; t < NM; t++) M[t] = 0.0;
    double cx = ldexp((double)a.x, -23), cy = ldexp((double)a.y, -23), cz = ldexp((double)a.z, -23);
    for (int j = r.x; j < r.x + r.y; j++)
      Ord<P>::p2m((double)smass[j], spos[j] - cx, spos[n + j] - cy, spos[2 * n + j] - cz, M);
    double* dst = mom + (int64_t)b * NM;
#pragma unroll
    for (int t = 0; t < NM; t++) dst[t] = M[t];
    finish_cell<P, T>(b, a.w & 0xff, M, coef);
    int c = b;
    while (true) {
      int par = cB[c].w;
      if (par < 0) break;
      __threadfence();
      int nch = cA[par].w >> 8;
      int old = atomicAdd(&arrive[par], 1);
      if (old != nch - 1) break;
      __threadfence();
      int4 pa = cA[par];
      int first = cB[par].z;
#pragma unroll
      for (int t = 0; t < NM; t++) M[t] = 0.0;
      for (int ch = first; ch < first + nch; ch++) {
        int4 ca = __ldcg(&cA[ch]);
        double Mc[NM];
        const double* src = mom + (int64_t)ch * NM;
#pragma unroll
        for (int t = 0; t < NM; t++) Mc[t] = __ldcg(src + t);
        Ord<P>::m2m(Mc, ldexp((double)(ca.x - pa.x), -23), ldexp((double)(ca.y - pa.y), -23),
                    ldexp((double)(ca.z - pa.z), -23), M);
      }
      double* pd = mom + (int64_t)par * NM;
#pragma unroll
      for (int t = 0; t < NM; t++) pd[t] = M[t];
      finish_cell<P, T>(par, pa.w & 0xff, M, coef);
      c = par;
    }
  }
}

// image-field source moments: one block per (box, level-le prefix)
template <int PE>
__global__ void __launch_bounds__(256)
field_moments_kernel(int le, const int64_t* __restrict__ off, const uint64_t* __restrict__ skeys,
                     const double* __restrict__ spos, const float* __restrict__ smass, int64_t n,
                     double* __restrict__ fm) {
  constexpr int NM = (PE + 1) * (PE + 2) * (PE + 3) / 6;
  const int ncp = 1 << (3 * le);
  const int box = blockIdx.y;
  const int cell = blockIdx.x;
  __shared__ int64_t s_rng[2];
  __shared__ double s_red[8][NM];
  if (threadIdx.x == 0) {
    int64_t lo = off[box], hi = off[box + 1];
    int sh = 3 * (NB_QBITS - le);
    uint64_t P = (uint64_t)cell;
    int64_t a = lo, b = hi;
    while (a < b) {
      int64_t m = (a + b) >> 1;
      if ((skeys[m] >> sh) < P) a = m + 1; else b = m;
    }
    int64_t s = a;
    a = s;
    b = hi;
    while (a < b) {
      int64_t m = (a + b) >> 1;
      if ((skeys[m] >> sh) <= P) a = m + 1; else b = m;
    }
    s_rng[0] = s;
    s_rng[1] = a;
  }
  __syncthreads();
  int ix = (int)compact3((uint64_t)cell), iy = (int)compact3((uint64_t)cell >> 1),
      iz = (int)compact3((uint64_t)cell >> 2);
  double cx = ldexp((double)cell_c2(ix, le), -23), cy = ldexp((double)cell_c2(iy, le), -23),
         cz = ldexp((double)cell_c2(iz, le), -23);
  double M[NM];
#pragma unroll
  for (int t = 0; t < NM; t++) M[t] = 0.0;
  for (int64_t j = s_rng[0] + threadIdx.x; j < s_rng[1]; j += blockDim.x) {
    double m = smass[j], dx = spos[j] - cx, dy = spos[n + j] - cy, dz = spos[2 * n + j] - cz;
    if constexpr (PE == 1) p2m_acc_p1(m, dx, dy, dz, M);
    if constexpr (PE == 2) p2m_acc_p2(m, dx, dy, dz, M);
    if constexpr (PE == 3) p2m_acc_p3(m, dx, dy, dz, M);
    if constexpr (PE == 4) p2m_acc_p4(m, dx, dy, dz, M);
    if constexpr (PE == 5) p2m_acc_p5(m, dx, dy, dz, M);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int t = 0; t < NM; t++) {
    double v = M[t];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) s_red[warp][t] = v;
  }
  __syncthreads();
  double* dst = fm + ((int64_t)box * ncp + cell) * NM;
  for (int t = threadIdx.x; t < NM; t += blockDim.x) {
    double v = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); w++) v += s_red[w][t];
    dst[t] = v;
  }
}

int gridc(int64_t n, int threads) {
  int64_t g = (n + threads - 1) / threads;
  if (g < 1) g = 1;
  if (g > 152 * 64) g = 152 * 64;
  return (int)g;
}

}  // namespace

int nb_coef_stride(int order) {
  switch (order) {
    case 0: return Ord<0>::NBS;
    case 1: return Ord<1>::NBS;
    case 2: return Ord<2>::NBS;
    case 3: return Ord<3>::NBS;
    default: return Ord<4>::NBS;
  }
}

cudaError_t nb_upward(int order, bool fp64, int ncell, const int4* cA, const int4* cB, const double* spos,
                      const float* smass, int64_t n, double* mom, int* arrive, void* coef, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(arrive, 0, sizeof(int) * ncell, s);
  if (e) return e;
  int g = gridc(ncell, 128);
#define NB_UP(P)                                                                                      \
  if (fp64)                                                                                           \
    upward_kernel<P, double><<<g, 128, 0, s>>>(ncell, cA, cB, spos, smass, n, mom, arrive, (double*)coef); \
  else                                                                                                \
    upward_kernel<P, float><<<g, 128, 0, s>>>(ncell, cA, cB, spos, smass, n, mom, arrive, (float*)coef);
  switch (order) {
    case 0: NB_UP(0) break;
    case 1: NB_UP(1) break;
    case 2: NB_UP(2) break;
    case 3: NB_UP(3) break;
    default: NB_UP(4) break;
  }
#undef NB_UP
  nb_launch_counter += 1;
  return cudaGetLastError();
}

cudaError_t nb_field_moments(int pe, int le, int nbox, const int64_t* off, const uint64_t* skeys,
                             const double* spos, const float* smass, int64_t n, double* fm, cudaStream_t s) {
  dim3 g(1u << (3 * le), nbox);
  switch (pe) {
    case 1: field_moments_kernel<1><<<g, 256, 0, s>>>(le, off, skeys, spos, smass, n, fm); break;
    case 2: field_moments_kernel<2><<<g, 256, 0, s>>>(le, off, skeys, spos, smass, n, fm); break;
    case 3: field_moments_kernel<3><<<g, 256, 0, s>>>(le, off, skeys, spos, smass, n, fm); break;
    case 4: field_moments_kernel<4><<<g, 256, 0, s>>>(le, off, skeys, spos, smass, n, fm); break;
    default: field_moments_kernel<5><<<g, 256, 0, s>>>(le, off, skeys, spos, smass, n, fm); break;
  }
  nb_launch_counter += 1;
  return cudaGetLastError();
}
