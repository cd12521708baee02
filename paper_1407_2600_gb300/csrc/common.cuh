// Internal declarations shared by the CUDA translation units of libnbody.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/nbody.h"

#define NB_QBITS 21            // key bits per axis
#define NB_NLEV 22             // levels 0..21
#define NB_PBOX (1 << 23)      // one box in integer units of 2^-23
#define NB_MAX_NBOX 65535

// Bounds checks of the debug build (compiled with -DNB_DEBUG_BOUNDS into
// libnbody_dbg.so; the product library is built without them).
// NB_IN(i, n, site) is true when 0 <= i < n.  Otherwise it records the first
// failing check of this translation unit, (site << 48) | (i & (2^48 - 1)), in
// the unit's fault word and returns false, and the caller skips the access,
// so that a bad index is reported instead of read or written.  Each unit
// exports its word through nbody_dbg_fault_<unit> (NB_DBG_EXPORT); without
// NB_DEBUG_BOUNDS the check is the constant true and compiles away.
#ifdef NB_DEBUG_BOUNDS
static __device__ unsigned long long nb_dbg_fault;
__device__ __forceinline__ bool nb_in(long long i, long long n, unsigned site) {
  if (i >= 0 && i < n) return true;
  atomicCAS(&nb_dbg_fault, 0ull, ((unsigned long long)site << 48) | ((unsigned long long)i & 0xffffffffffffull));
  return false;
}
#define NB_IN(i, n, site) nb_in((long long)(i), (long long)(n), (unsigned)(site))
// an index to read at: i when the check passes, else 0 (n > 0 wherever used)
#define NB_IDX(i, n, site) (NB_IN(i, n, site) ? (i) : 0)
// fault word of this unit to *out (0: no check failed); reset clears it
#define NB_DBG_EXPORT(unit)                                                                   \
  extern "C" int nbody_dbg_fault_##unit(unsigned long long* out, int reset) {                \
    cudaError_t e = cudaMemcpyFromSymbol(out, nb_dbg_fault, sizeof(unsigned long long));     \
    if (e == cudaSuccess && reset) {                                                          \
      const unsigned long long z = 0;                                                         \
      e = cudaMemcpyToSymbol(nb_dbg_fault, &z, sizeof(z));                                    \
    }                                                                                         \
    return (int)e;                                                                            \
  }
#else
#define NB_IN(i, n, site) true
#define NB_IDX(i, n, site) (i)
#define NB_DBG_EXPORT(unit)
#endif

// device status bits (OR-ed into the tree's status word)
// floats per cell of the FP32 cell-unit moments of the dual form (orders <= 4)
constexpr int kDualStride = 36;
#define NB_ST_OVERFLOW 1u
#define NB_ST_TIMEOUT 2u
#define NB_ST_BADINPUT 4u

// bounded spin limit for decoupled look-back waits
#define NB_SPIN_LIMIT (1 << 22)

// The hardware's approximate 1/sqrt(s) with subnormal inputs flushed to zero
// (PTX rsqrt.approx.ftz.f32).  Every argument here is at least eps^2 or a
// sum of squares of order one in a cell's unit, far above the subnormal
// range, so the flush never changes a result; it spares the instructions
// that the subnormal-preserving form adds around each reciprocal root.  An
// argument of zero gives +inf either way.
__device__ __forceinline__ float nb_rsqrt_ftz(float s) {
  float r;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(s));
  return r;
}

// FP32 1/sqrt(s): the hardware approximation (good to about 2 ulp) refined
// by one Newton-Raphson step r + r (1 - s r^2)/2 whose residual is formed
// exactly, r^2 = p + p_lo being an exact FMA two-product, so that only the
// final rounding is left.  Interaction terms of the walk inherit the
// reciprocal's error several times over (r^3 for the monopole, r^11 at
// hexadecapole order), and on near-uniform boxes far cells' terms cancel to
// a force a thousand times smaller than their sum.  s > 0 and finite.
__device__ __forceinline__ float nbody_rsqrt(float s) {
  const float r = nb_rsqrt_ftz(s);
  const float p = r * r;
  const float plo = fmaf(r, r, -p);
  const float e = fmaf(-s, plo, fmaf(-s, p, 1.0f));
  return fmaf(0.5f * r, e, r);
}
__device__ __forceinline__ double nbody_rsqrt(double x) { return rsqrt(x); }
// the hardware approximation alone, for particle-particle terms: each pair's
// term is small next to the sum it joins, so the last ulp of 1/sqrt does not
// show in the result, while one more instruction per pair would
__device__ __forceinline__ float nbody_rsqrt_pair(float x) { return nb_rsqrt_ftz(x); }
__device__ __forceinline__ double nbody_rsqrt_pair(double x) { return rsqrt(x); }

struct __align__(32) dbl4 {
  double x, y, z, w;
};
template <typename T> struct Vec4;
template <> struct Vec4<float> { typedef float4 type; };
template <> struct Vec4<double> { typedef dbl4 type; };

// level-l cell centre in units of 2^-23 from its integer index at that level
__host__ __device__ __forceinline__ int cell_c2(int i, int level) {
  return (2 * i + 1) << (22 - level);
}

// image shift k (in boxes) of a point c2 (units 2^-23) nearest the point g2
__host__ __device__ __forceinline__ int img_shift(int c2, int g2) {
  int delta = c2 - g2;
  int red = ((delta + (NB_PBOX >> 1)) & (NB_PBOX - 1)) - (NB_PBOX >> 1);  // [-2^22, 2^22)
  return (delta - red) >> 23;
}

// 21-bit spreads for Morton interleaving (x in bit 3b, y in 3b+1, z in 3b+2)
__host__ __device__ __forceinline__ uint64_t spread3(uint64_t x) {
  x &= 0x1fffffull;
  x = (x | (x << 32)) & 0x1f00000000ffffull;
  x = (x | (x << 16)) & 0x1f0000ff0000ffull;
  x = (x | (x << 8)) & 0x100f00f00f00f00full;
  x = (x | (x << 4)) & 0x10c30c30c30c30c3ull;
  x = (x | (x << 2)) & 0x1249249249249249ull;
  return x;
}
__host__ __device__ __forceinline__ uint32_t compact3(uint64_t x) {
  x &= 0x1249249249249249ull;
  x = (x ^ (x >> 2)) & 0x10c30c30c30c30c3ull;
  x = (x ^ (x >> 4)) & 0x100f00f00f00f00full;
  x = (x ^ (x >> 8)) & 0x1f0000ff0000ffull;
  x = (x ^ (x >> 16)) & 0x1f00000000ffffull;
  x = (x ^ (x >> 32)) & 0x1fffffull;
  return (uint32_t)x;
}

// quantised coordinate floor(x 2^21) mod 2^21 (x is wrapped to [0,1) first)
__device__ __forceinline__ uint32_t quant21(double x) {
  double f = floor(x * 2097152.0);
  long long q = (long long)f;
  q %= 2097152LL;
  if (q < 0) q += 2097152LL;
  return (uint32_t)q;
}

// v * 2^e for |v| < 2^31, exact, on the integer pipe (GB300's FP64 pipe is
// narrow, and int-to-double conversions run on it)
__device__ __forceinline__ double i2d_pow2(int v, int e) {
  if (v == 0) return 0.0;
  const unsigned long long sgn = v < 0 ? 0x8000000000000000ULL : 0ULL;
  const unsigned u = v < 0 ? (unsigned)(-(long long)v) : (unsigned)v;
  const int msb = 31 - __clz(u);
  const unsigned long long mant = ((unsigned long long)u << (52 - msb)) & 0x000fffffffffffffULL;
  return __longlong_as_double((long long)(sgn | ((unsigned long long)(1023 + msb + e) << 52) | mant));
}

// two timing events destroyed on every exit path (the launch autotuners)
struct EventPair {
  cudaEvent_t a = nullptr, b = nullptr;
  cudaError_t create() {
    cudaError_t e = cudaEventCreate(&a);
    if (e == cudaSuccess) e = cudaEventCreate(&b);
    return e;
  }
  ~EventPair() {
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
  }
};

// ---- key hash of the cells (open addressing, linear probing) ------------------
__device__ __forceinline__ uint64_t hmix(uint64_t k) {
  k ^= k >> 33;
  k *= 0xff51afd7ed558ccdull;
  k ^= k >> 33;
  k *= 0xc4ceb9fe1a85ec53ull;
  k ^= k >> 33;
  return k;
}
__device__ __forceinline__ uint64_t hslot(uint64_t key, int box, uint64_t mask) {
  return hmix(key ^ ((uint64_t)box * 0x9e3779b97f4a7c15ull)) & mask;
}
// the cell with this placeholder key in this box, or -1 (slots hold cell
// indices, -1 = empty)
__device__ __forceinline__ int hash_find(const int* __restrict__ hval, const uint64_t* __restrict__ ckey,
                                         const uint16_t* __restrict__ cbox, uint64_t mask, uint64_t key, int box) {
  uint64_t h = hslot(key, box, mask);
  for (uint64_t probe = 0; probe <= mask; probe++) {
    const int v = hval[h];
    if (v < 0) return -1;
    if (ckey[v] == key && cbox[v] == box) return v;
    h = (h + 1) & mask;
  }
  return -1;
}

// ---- device-side tree description passed to kernels -------------------------
struct DevTree {
  int64_t n;
  int nbox;
  const int64_t* off;      // nbox+1 particle offsets (device)
  const uint64_t* skeys;   // sorted keys
  const uint32_t* perm;    // sorted -> original index
  const uint16_t* sbox;    // box id per sorted particle
  const double* spos;      // 3n sorted positions (SoA)
  const float* smass;      // sorted masses
  // ncell and ngroup are the capacities the launch grids and buffers are
  // sized for; the counts of the last build are on the device (cnt[0] cells,
  // cnt[1] groups, both <= the capacities) so that a build needs no read back
  // to the host and a whole step can be captured in a CUDA graph
  const int* cnt;
  int ncell;
  const int4* cA;          // c2x, c2y, c2z, level | nchild << 8
  const int4* cB;          // start, count, child, parent
  int ngroup;
  const int4* gA;          // start, count, box, 0
  const int4* gB;          // g2x, g2y, g2z, 0 (box centre, units 2^-23)
  const int4* gC;          // w2x, w2y, w2z, 0 (half widths, units 2^-23)
  const int4* gD;          // e2x, e2y, e2z, run (expansion point, units 2^-23)
  const int* runhead;      // first group of each run of groups sharing e (cnt[2] runs)
  const int* sleaf;        // leaf cell of each sorted particle
  // evaluation of a subset (block steps): per sorted particle and per group
  // a nonzero byte marks the sinks whose accelerations are computed and
  // written; nullptr = every particle
  const uint8_t* sact;
  const uint8_t* gact;
};

// The dual form's cell-group pairs: the walk emits each group's pairs in
// chunks of up to 32 (one group per chunk, linked in the walk's order), a
// separate pass forms each chunk's summed local expansion, and a third sums
// a group's chunks in list order and evaluates the expansion at its sinks.
struct NbDualBufs {
  int* cell;      // cap x 32 source cells
  int* img;       // cap x 32 image shifts, (kx + 2) | (ky + 2) << 3 | (kz + 2) << 6
  int4* head;     // cap: group, pair count, next chunk of the group (-1), 0
  int* first;     // per group: its first chunk, or -1
  int* ctr;       // chunks asked for (can exceed cap: the overflow is reported)
  float* L;       // cap x kDualLStride: each chunk's local coefficients, group unit
  int cap;
};
constexpr int kDualLStride = 56;  // local coefficients per chunk (orders 1..5)

// kernels launched by this thread through the library (benchmark accounting)
extern thread_local long long nb_launch_counter;

// ---- host launchers (each returns cudaError_t of the launch) ---------------------
cudaError_t nb_launch_keys(const double* pos, int64_t n, int64_t box_n0, uint64_t* keys,
                           uint32_t* vals, cudaStream_t s);
cudaError_t nb_launch_box_ids(const int64_t* off, int nbox, int64_t n, uint16_t* box_of,
                              cudaStream_t s);
// stable LSD onesweep radix sort of (key, val); sorts bits [bit0, bit1) of
// the key, then (if box_of != NULL and nbox > 1) by box id of the value.
struct SortScratch {
  uint64_t* keys_alt;
  uint32_t* vals_alt;
  uint32_t* hist;       // 16 passes x 256
  uint32_t* status;     // tiles x 256 x passes
  uint32_t* tile_ctr;   // passes
  int64_t tiles_cap;    // rows of 256 status words available (tiles x passes)
  unsigned* dstatus;    // error word
};
// passes of nb_radix_sort; an odd count leaves the result in the alternate buffers
int nb_radix_passes(int bit1, int nbox);
cudaError_t nb_radix_sort(uint64_t* keys, uint32_t* vals, int64_t n, int bit1,
                          const uint16_t* box_of_orig, int nbox, SortScratch* sc, cudaStream_t s,
                          int* result_in_alt);
// stable sort of a small-range 8-bit digit array (one pass), values = index
cudaError_t nb_sort_digit8(const uint8_t* digit, int64_t n, uint32_t* order_out, uint32_t* hist_out,
                           SortScratch* sc, cudaStream_t s);
int64_t nb_sort_tiles(int64_t n);

cudaError_t nb_exclusive_scan_i32(const int* in, int* out, int64_t n, int* total_dev, int* tmp,
                                  cudaStream_t s);
int64_t nb_scan_tmp_ints(int64_t n);
