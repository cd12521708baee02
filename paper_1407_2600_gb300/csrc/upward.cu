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

// Exact scalings by powers of two run on the integer pipe (i2d_pow2 in
// common.cuh, mul_pow2 below): GB300's FP64 pipe is narrow, and these run
// once per moment of every cell.
// x * 2^k (exact unless the result under- or overflows); the exponent field
// is adjusted directly when x and the result are normal numbers
__device__ __forceinline__ double mul_pow2(double x, int k) {
  const long long b = __double_as_longlong(x);
  const int ex = (int)((b >> 52) & 0x7ff);
  if (ex > 0 && ex + k > 0 && ex + k < 0x7ff) return __longlong_as_double(b + ((long long)k << 52));
  if (ex == 0 && (b & 0x000fffffffffffffLL) == 0) return x;  // +-0
  return x * __longlong_as_double((long long)(1023 + k) << 52);
}

// order |n| of the moment at storage index t (orders are stored in sequence)
__host__ __device__ constexpr int order_of(int t) {
  int o = 0;
  while ((o + 1) * (o + 2) * (o + 3) / 6 <= t) o++;
  return o;
}

// Reduced coefficients in the cell's own length unit h = 2^-level: with
// R' = R/h and eps' = eps/h the expansion terms are O(1) for every accepted
// cell (R' >= 1/theta), so FP32 intermediates cannot overflow however deep the
// cell; a = h^-2 sum(...) is folded into the coefficients as B'' =
// h^-2 B(M_n h^-|n|).  All scalings are exact powers of two.
// The slot just past the coefficients (where the row has one) carries the
// weight rho 2^-level of the cell's uniform-background term (0 without it).
struct BgArgs {
  const uint16_t* cbox;  // box of each cell
  const double* rho;     // mean density of each box; nullptr: no background term
  float* mom32;          // nullptr, or the cells' moments in their own unit
                         // M_n h^-|n| in FP32 (kDualStride per cell), for
                         // the cell-group local expansions of the dual form
  const int* pncell;     // the build's cell count (bounds of the debug build)
};

template <int P, typename T>
__device__ __forceinline__ void finish_cell(int c, int level, const double* M, T* __restrict__ coef, BgArgs bg) {
  constexpr int NM = Ord<P>::NM;
  double Ms[NM];
#pragma unroll
  for (int t = 0; t < NM; t++) Ms[t] = mul_pow2(M[t], level * order_of(t));
  double B[Ord<P>::NB];
  Ord<P>::reduce(Ms, B);
  T* dst = coef + (int64_t)c * Ord<P>::NBS;
#pragma unroll
  for (int q = 0; q < Ord<P>::NB; q++) dst[q] = (T)mul_pow2(B[q], 2 * level);
#pragma unroll
  for (int q = Ord<P>::NB; q < Ord<P>::NBS; q++) dst[q] = (T)0;
  if constexpr (Ord<P>::NB < Ord<P>::NBS)
    if (bg.rho) dst[Ord<P>::NB] = (T)mul_pow2(bg.rho[bg.cbox[c]], -level);
  if (bg.mom32) {
    float* m32 = bg.mom32 + (int64_t)c * kDualStride;
#pragma unroll
    for (int t = 0; t < NM; t++) m32[t] = (float)Ms[t];
  }
}

// Schedule of the upward pass.  Every cell gets an 8-bit key: leaves sort by
// particle count (0..63) and come first; cells with daughters follow by level,
// deepest first, and by daughter count within a level.  After a stable sort by
// this key, one launch forms all leaves (threads of a warp have similar
// counts) and one launch per level forms that level's parents from their
// finished daughters (similar daughter counts), so the FP64 work runs on
// full warps and no thread waits for another.  Slots past the cell count (a
// reserved capacity) get key 255, which no cell has and the schedule ignores.
__global__ void upkey_kernel(int cap, const int* __restrict__ pncell, const int4* __restrict__ cA,
                             const int4* __restrict__ cB, uint8_t* __restrict__ key) {
  const int ncell = *pncell;
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < cap; b += gridDim.x * blockDim.x) {
    if (b >= ncell) {
      key[b] = 255;
      continue;
    }
    const int4 a = cA[b];
    const int nch = a.w >> 8, lvl = a.w & 0xff;
    key[b] = nch == 0 ? (uint8_t)min(cB[b].y, 63) : (uint8_t)(64 + (NB_QBITS - lvl) * 8 + (nch - 1));
  }
}

// r[0] = number of leaves; cells with daughters at level NB_QBITS - j occupy
// [r[j], r[j + 1]) of the sorted order, j = 0..NB_QBITS
__global__ void urange_kernel(const uint32_t* __restrict__ hist, int* __restrict__ r) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  int pos = 0;
  for (int k = 0; k < 64; k++) pos += (int)hist[k];
  r[0] = pos;
  for (int j = 0; j <= NB_QBITS; j++) {
    for (int k = 64 + 8 * j; k < 64 + 8 * (j + 1); k++) pos += (int)hist[k];
    r[j + 1] = pos;
  }
}

// P2M of the leaves
template <int P, typename T>
__global__ void __launch_bounds__(128)
leaf_moments_kernel(const uint32_t* __restrict__ order, const int* __restrict__ r, const int4* __restrict__ cA,
                    const int4* __restrict__ cB, const double* __restrict__ spos, const float* __restrict__ smass,
                    int64_t n, double* __restrict__ mom, T* __restrict__ coef, BgArgs bg) {
  constexpr int NM = Ord<P>::NM;
  const int nleaf = r[0];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nleaf; i += gridDim.x * blockDim.x) {
    const int b = NB_IDX((int)order[i], *bg.pncell, 401);
    const int4 a = cA[b];
    const int4 rg = cB[b];
    double M[NM];
#pragma unroll
    for (int t = 0; t < NM; t++) M[t] = 0.0;
    const double cx = i2d_pow2(a.x, -23), cy = i2d_pow2(a.y, -23), cz = i2d_pow2(a.z, -23);
    for (int j = rg.x; j < rg.x + rg.y; j++) {
      if (!NB_IN(j, n, 402)) break;
      Ord<P>::p2m((double)smass[j], spos[j] - cx, spos[n + j] - cy, spos[2 * n + j] - cz, M);
    }
    double* dst = mom + (int64_t)b * NM;
#pragma unroll
    for (int t = 0; t < NM; t++) dst[t] = M[t];
    finish_cell<P, T>(b, a.w & 0xff, M, coef, bg);
  }
}

// M2M of the parents of one level from their daughters (formed by earlier
// launches).  A wide level gives each parent one thread, which shifts its
// daughters one after another.  GB300's FP64 pipe takes a warp instruction
// at a time however few lanes are active, so on a narrow level (near the
// root, or the deep levels of a halo) that serial chain would set the time;
// there a warp takes four parents, one lane per daughter shifts its moments
// and the daughters' terms are summed across lanes.
constexpr int kWideLevel = 12288;

template <int P, typename T>
__global__ void __launch_bounds__(128)
level_moments_kernel(int j, const uint32_t* __restrict__ order, const int* __restrict__ r,
                     const int4* __restrict__ cA, const int4* __restrict__ cB, double* __restrict__ mom,
                     T* __restrict__ coef, BgArgs bg) {
  constexpr int NM = Ord<P>::NM;
  const int lo = r[j], hi = r[j + 1];
  if (hi - lo < kWideLevel) {
    const int lane = threadIdx.x & 31, slot = lane >> 3, d = lane & 7;
    const int nwarp = (gridDim.x * blockDim.x) >> 5;
    for (int i0 = lo + 4 * ((blockIdx.x * blockDim.x + threadIdx.x) >> 5); i0 < hi; i0 += 4 * nwarp) {
      const int i = i0 + slot;
      int b = -1, first = 0, nch = 0;
      int4 pa = make_int4(0, 0, 0, 0);
      if (i < hi) {
        b = NB_IDX((int)order[i], *bg.pncell, 403);
        pa = cA[b];
        first = cB[b].z;
        nch = pa.w >> 8;
      }
      double M[NM];
#pragma unroll
      for (int t = 0; t < NM; t++) M[t] = 0.0;
      if (d < nch) {
        const int ch = NB_IDX(first + d, *bg.pncell, 404);
        const int4 ca = cA[ch];
        double Mc[NM];
        const double* src = mom + (int64_t)ch * NM;
#pragma unroll
        for (int t = 0; t < NM; t++) Mc[t] = src[t];
        Ord<P>::m2m(Mc, i2d_pow2(ca.x - pa.x, -23), i2d_pow2(ca.y - pa.y, -23), i2d_pow2(ca.z - pa.z, -23), M);
      }
      // sum over the eight daughter lanes of each parent (fixed order)
#pragma unroll
      for (int t = 0; t < NM; t++) {
        double v = M[t];
        v += __shfl_xor_sync(0xffffffffu, v, 1);
        v += __shfl_xor_sync(0xffffffffu, v, 2);
        v += __shfl_xor_sync(0xffffffffu, v, 4);
        M[t] = v;
      }
      if (d == 0 && b >= 0) {
        double* pd = mom + (int64_t)b * NM;
#pragma unroll
        for (int t = 0; t < NM; t++) pd[t] = M[t];
        finish_cell<P, T>(b, pa.w & 0xff, M, coef, bg);
      }
    }
    return;
  }
  for (int i = lo + blockIdx.x * blockDim.x + threadIdx.x; i < hi; i += gridDim.x * blockDim.x) {
    const int b = NB_IDX((int)order[i], *bg.pncell, 403);
    const int4 pa = cA[b];
    const int first = cB[b].z, nch = pa.w >> 8;
    double M[NM];
#pragma unroll
    for (int t = 0; t < NM; t++) M[t] = 0.0;
    for (int ch = first; ch < first + nch; ch++) {
      if (!NB_IN(ch, *bg.pncell, 404)) break;
      const int4 ca = cA[ch];
      double Mc[NM];
      const double* src = mom + (int64_t)ch * NM;
#pragma unroll
      for (int t = 0; t < NM; t++) Mc[t] = src[t];
      Ord<P>::m2m(Mc, i2d_pow2(ca.x - pa.x, -23), i2d_pow2(ca.y - pa.y, -23), i2d_pow2(ca.z - pa.z, -23), M);
    }
    double* pd = mom + (int64_t)b * NM;
#pragma unroll
    for (int t = 0; t < NM; t++) pd[t] = M[t];
    finish_cell<P, T>(b, pa.w & 0xff, M, coef, bg);
  }
}

// Image-field source moments: one block per (box, level-le prefix).  When the
// prefix is a cell of the tree and the tree's moments reach order PE, they are
// the same moments (about the same centre, over the same particles): they are
// copied; otherwise (a prefix inside a leaf, or a lower tree order) they are
// formed from the prefix's particles.  An FP32 copy (fm32, same layout) feeds
// the mixed-precision image-field M2L, which would otherwise convert every
// moment from FP64 once per run on GB300's narrow FP64 pipe.
struct TreeMoments {
  const int* hval;
  const uint64_t* ckey;
  const uint16_t* cbox;
  uint64_t mask;
  const double* mom;  // nullptr: always from the particles
  int nm;             // moments per cell of the tree
};

template <int PE>
__global__ void __launch_bounds__(256)
field_moments_kernel(int le, const int64_t* __restrict__ off, const uint64_t* __restrict__ skeys,
                     const double* __restrict__ spos, const float* __restrict__ smass, int64_t n,
                     TreeMoments tm, double* __restrict__ fm, float* __restrict__ fm32) {
  constexpr int NM = (PE + 1) * (PE + 2) * (PE + 3) / 6;
  const int ncp = 1 << (3 * le);
  const int box = blockIdx.y;
  const int cell = blockIdx.x;
  __shared__ int s_tc;
  if (threadIdx.x == 0)
    s_tc = (tm.mom && tm.nm >= NM) ? hash_find(tm.hval, tm.ckey, tm.cbox, tm.mask,
                                               (1ull << (3 * le)) | (uint64_t)cell, box)
                                   : -1;
  __syncthreads();
  if (s_tc >= 0) {
    double* dst = fm + ((int64_t)box * ncp + cell) * NM;
    float* d32 = fm32 + ((int64_t)box * ncp + cell) * NM;
    for (int t = threadIdx.x; t < NM; t += blockDim.x) {
      const double v = tm.mom[(int64_t)s_tc * tm.nm + t];
      dst[t] = v;
      d32[t] = (float)v;
    }
    return;
  }
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
    if (!NB_IN(j, n, 405)) break;
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
  float* d32 = fm32 + ((int64_t)box * ncp + cell) * NM;
  for (int t = threadIdx.x; t < NM; t += blockDim.x) {
    double v = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); w++) v += s_red[w][t];
    dst[t] = v;
    d32[t] = (float)v;
  }
}

// mean density of each box (its mass over the unit volume) in two fixed-order
// stages, so that it is bitwise reproducible: kMassParts blocks per box sum
// contiguous slices (FP64), then one warp per box sums the slices in order
constexpr int kMassParts = 64;
__global__ void __launch_bounds__(256) box_mass_part_kernel(const int64_t* __restrict__ off,
                                                            const float* __restrict__ smass,
                                                            double* __restrict__ part) {
  __shared__ double s_red[8];
  const int box = blockIdx.y, k = blockIdx.x;
  const int64_t lo = off[box], n = off[box + 1] - lo;
  const int64_t a = lo + n * k / kMassParts, b = lo + n * (k + 1) / kMassParts;
  double m = 0.0;
  for (int64_t j = a + threadIdx.x; j < b; j += blockDim.x) m += (double)smass[j];
  for (int o = 16; o > 0; o >>= 1) m += __shfl_xor_sync(0xffffffffu, m, o);
  if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); w++) t += s_red[w];
    part[(int64_t)box * kMassParts + k] = t;
  }
}

__global__ void box_mass_sum_kernel(int nbox, const double* __restrict__ part, double* __restrict__ rho) {
  const int box = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (box >= nbox) return;
  double m = part[(int64_t)box * kMassParts + lane] + part[(int64_t)box * kMassParts + 32 + lane];
  for (int o = 16; o > 0; o >>= 1) m += __shfl_xor_sync(0xffffffffu, m, o);
  if (lane == 0) rho[box] = m;
}

int gridc(int64_t n, int threads) {
  int64_t g = (n + threads - 1) / threads;
  if (g < 1) g = 1;
  if (g > 152 * 64) g = 152 * 64;
  return (int)g;
}

}  // namespace

// part: kMassParts doubles of scratch per box
cudaError_t nb_box_mass(const int64_t* off, const float* smass, int nbox, double* rho, double* part,
                        cudaStream_t s) {
  box_mass_part_kernel<<<dim3(kMassParts, nbox), 256, 0, s>>>(off, smass, part);
  box_mass_sum_kernel<<<(nbox + 3) / 4, 128, 0, s>>>(nbox, part, rho);
  nb_launch_counter += 2;
  return cudaGetLastError();
}

int nb_coef_stride(int order) {
  switch (order) {
    case 0: return Ord<0>::NBS;
    case 1: return Ord<1>::NBS;
    case 2: return Ord<2>::NBS;
    case 3: return Ord<3>::NBS;
    default: return Ord<4>::NBS;
  }
}

cudaError_t nb_upward(int order, bool fp64, int ncell, const int* pncell, const int4* cA, const int4* cB,
                      const double* spos, const float* smass, int64_t n, double* mom, void* coef, uint8_t* ukey,
                      uint32_t* uorder, uint32_t* uhist, int* urange, const uint16_t* cbox, const double* rho,
                      float* mom32, SortScratch* sc, cudaStream_t s) {
  const BgArgs bg{cbox, rho, mom32, pncell};
  upkey_kernel<<<gridc(ncell, 256), 256, 0, s>>>(ncell, pncell, cA, cB, ukey);
  nb_launch_counter += 1;
  cudaError_t e = nb_sort_digit8(ukey, ncell, uorder, uhist, sc, s);
  if (e) return e;
  urange_kernel<<<1, 32, 0, s>>>(uhist, urange);
  nb_launch_counter += 1;
  const int g = gridc(ncell, 128);
  const int gl = g < 152 * 4 ? g : 152 * 4;
#define NB_UP(P, TT)                                                                                        \
  {                                                                                                         \
    leaf_moments_kernel<P, TT><<<g, 128, 0, s>>>(uorder, urange, cA, cB, spos, smass, n, mom, (TT*)coef, bg); \
    for (int j = 0; j <= NB_QBITS; j++)                                                                     \
      level_moments_kernel<P, TT><<<gl, 128, 0, s>>>(j, uorder, urange, cA, cB, mom, (TT*)coef, bg);       \
  }
#define NB_UPP(P) \
  if (fp64) NB_UP(P, double) else NB_UP(P, float)
  switch (order) {
    case 0: NB_UPP(0) break;
    case 1: NB_UPP(1) break;
    case 2: NB_UPP(2) break;
    case 3: NB_UPP(3) break;
    default: NB_UPP(4) break;
  }
#undef NB_UPP
#undef NB_UP
  nb_launch_counter += 2 + NB_QBITS;
  return cudaGetLastError();
}

cudaError_t nb_field_moments(int pe, int le, int nbox, const int64_t* off, const uint64_t* skeys,
                             const double* spos, const float* smass, int64_t n, const int* hval,
                             const uint64_t* ckey, const uint16_t* cbox, uint64_t hcap, const double* mom,
                             int order, double* fm, float* fm32, cudaStream_t s) {
  dim3 g(1u << (3 * le), nbox);
  const TreeMoments tm{hval, ckey, cbox, hcap - 1, mom, (order + 1) * (order + 2) * (order + 3) / 6};
  switch (pe) {
    case 1: field_moments_kernel<1><<<g, 256, 0, s>>>(le, off, skeys, spos, smass, n, tm, fm, fm32); break;
    case 2: field_moments_kernel<2><<<g, 256, 0, s>>>(le, off, skeys, spos, smass, n, tm, fm, fm32); break;
    case 3: field_moments_kernel<3><<<g, 256, 0, s>>>(le, off, skeys, spos, smass, n, tm, fm, fm32); break;
    case 4: field_moments_kernel<4><<<g, 256, 0, s>>>(le, off, skeys, spos, smass, n, tm, fm, fm32); break;
    default: field_moments_kernel<5><<<g, 256, 0, s>>>(le, off, skeys, spos, smass, n, tm, fm, fm32); break;
  }
  nb_launch_counter += 1;
  return cudaGetLastError();
}

// fault word of the debug build's bounds checks in this unit (debug build only)
NB_DBG_EXPORT(upward)
