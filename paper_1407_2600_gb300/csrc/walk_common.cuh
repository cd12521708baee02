// Cell classification shared by the forward walk and its adjoint, so that
// both take identical discrete decisions (image, acceptance, interaction type).
#pragma once

#include "common.cuh"

template <typename T>
__device__ __forceinline__ void kadd(T& s, T& c, T x) {
  T y = x - c;
  T t = s + y;
  c = (t - s) - y;
  s = t;
}

// kadd on both halves of an FP32 pair, in packed instructions
__device__ __forceinline__ void kadd2(float2& s, float2& c, float2 x) {
  const float2 y = __fadd2_rn(x, make_float2(-c.x, -c.y));
  const float2 t = __fadd2_rn(s, y);
  const float2 d = __fadd2_rn(t, make_float2(-s.x, -s.y));
  c = __fadd2_rn(d, make_float2(-y.x, -y.y));
  s = t;
}

// Error-free transformations of FP32 sums (Knuth's TwoSum; Dekker's
// Fast2Sum for |a| >= |b|): s + e equals a + b exactly.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  e = b - (s - a);
}

// Largest cells whose monopole term is formed in double-float arithmetic:
// level <= kDfLevel (side >= 1/16 of the box).
constexpr float kDfScale = 16.f;

// The monopole term b0 R f(R), f = -(|R|^2 + eps^2)^(-3/2), of a cell's
// expansion (R = x sc + o in the cell's unit, sc a power of two) in
// double-float arithmetic -- every value an unevaluated sum hi + lo of two
// FP32 numbers, sums and products made error-free by TwoSum and the FMA
// two-product -- added to the double-float accumulators (sh, sl).  On a
// nearly uniform box the largest cells' monopole terms are a thousand times
// the force they add up to, and in plain FP32 their few-ulp rounding sets the
// error of the result; this form leaves an error of order 2^-44 of each term.
__device__ __forceinline__ void mono_df(float x, float y, float z, float sc, float ox, float oy, float oz, float e2,
                                        float b0, float* sh, float* sl) {
  float Rh[3], Rl[3];
  two_sum(x * sc, ox, Rh[0], Rl[0]);  // x sc is exact
  two_sum(y * sc, oy, Rh[1], Rl[1]);
  two_sum(z * sc, oz, Rh[2], Rl[2]);
  // s = |R|^2 + eps^2
  float p[3], pe[3];
#pragma unroll
  for (int d = 0; d < 3; d++) {
    p[d] = Rh[d] * Rh[d];
    pe[d] = fmaf(Rh[d], Rh[d], -p[d]) + 2.f * Rh[d] * Rl[d];
  }
  float s1, t1, s2, t2, s3, t3;
  two_sum(p[0], p[1], s1, t1);
  two_sum(s1, p[2], s2, t2);
  two_sum(s2, e2, s3, t3);
  float shi, slo;
  fast_two_sum(s3, ((t1 + t2) + t3) + ((pe[0] + pe[1]) + pe[2]), shi, slo);
  // r = s^(-1/2): one Newton step from the hardware value, residual exact
  const float r0 = nb_rsqrt_ftz(shi);
  const float q = r0 * r0, ql = fmaf(r0, r0, -q);
  float res = fmaf(-shi, q, 1.f);
  res = fmaf(-shi, ql, res);
  res = fmaf(-slo, q, res);  // 1 - s r0^2
  // f = -r^3 = -r0^3 (1 + 3 res / 2), second order in res dropped (|res| < 1e-6)
  const float c = r0 * q, cl = fmaf(r0, q, -c) + r0 * ql;
  const float fh = -c, fl = -(cl + c * (1.5f * res));
  const float u = b0 * fh, ul = fmaf(b0, fh, -u) + b0 * fl;
#pragma unroll
  for (int d = 0; d < 3; d++) {
    const float v = u * Rh[d];
    const float vl = fmaf(u, Rh[d], -v) + (u * Rl[d] + ul * Rh[d]);
    float h, e;
    two_sum(sh[d], v, h, e);
    sh[d] = h;
    sl[d] += e + vl;
  }
}

// 16-byte asynchronous copy from global to shared memory (PTX cp.async,
// cached in L1 and L2); both addresses 16-byte aligned.  The copies a thread
// issued are complete and visible to it after cp_async_wait_all.
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

__device__ __forceinline__ int warp_excl_scan(int v, int lane) {
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  return x - v;
}

enum { NB_CELL_NONE = 0, NB_CELL_OPEN = 1, NB_CELL_M2P = 2, NB_CELL_P2P = 3, NB_CELL_M2L = 4 };

// term of the order-independent checksum (a sum modulo 2^64) of every
// (group, cell, decision) of a walk and of every group's members: any change
// of the tree, the groups or an acceptance decision changes the sum with
// overwhelming probability
__device__ __forceinline__ unsigned long long decision_mix(int g, int c, int cls) {
  unsigned long long h = (unsigned long long)(g + 1) * 0x9E3779B97F4A7C15ull;
  h ^= (unsigned long long)(c + 1) * 0xC2B2AE3D27D4EB4Full;
  h ^= (unsigned long long)cls * 0x165667B19E3779F9ull;
  h ^= h >> 29;
  return h * 0xBF58476D1CE4E5B9ull;
}

// Image of a cell from its level-le ancestor (or the common image of its
// level-le descendants) nearest the expansion point e; then the integer
// acceptance test against the group box (centre g2, half-widths w2), with
// the distance taken from the cell centre or, with mac_edge, its faces.
__device__ __forceinline__ int classify_cell(const int4 ca, const int4 cb, const int4 gb, const int4 gc,
                                             const int4 gd, int le, const long long* thr, int n_direct,
                                             int mac_edge, int& kx, int& ky, int& kz) {
  const int lvl = ca.w & 0xff, nch = ca.w >> 8;
  bool consistent = true;
  const int ix = ((ca.x >> (22 - lvl)) - 1) >> 1;
  const int iy = ((ca.y >> (22 - lvl)) - 1) >> 1;
  const int iz = ((ca.z >> (22 - lvl)) - 1) >> 1;
  if (lvl >= le) {
    const int sh = lvl - le;
    kx = img_shift(cell_c2(ix >> sh, le), gd.x);
    ky = img_shift(cell_c2(iy >> sh, le), gd.y);
    kz = img_shift(cell_c2(iz >> sh, le), gd.z);
  } else {
    const int sh = le - lvl;
    kx = img_shift(cell_c2(ix << sh, le), gd.x);
    ky = img_shift(cell_c2(iy << sh, le), gd.y);
    kz = img_shift(cell_c2(iz << sh, le), gd.z);
    consistent = kx == img_shift(cell_c2(((ix + 1) << sh) - 1, le), gd.x) &&
                 ky == img_shift(cell_c2(((iy + 1) << sh) - 1, le), gd.y) &&
                 kz == img_shift(cell_c2(((iz + 1) << sh) - 1, le), gd.z);
  }
  // d from the cell centre, or (mac_edge) from its faces: less the half side
  const int hs = mac_edge ? (1 << (22 - lvl)) : 0;
  const int dx = abs(ca.x - gb.x - kx * NB_PBOX) - gc.x - hs;
  const int dy = abs(ca.y - gb.y - ky * NB_PBOX) - gc.y - hs;
  const int dz = abs(ca.z - gb.z - kz * NB_PBOX) - gc.z - hs;
  const long long ddx = dx > 0 ? dx : 0, ddy = dy > 0 ? dy : 0, ddz = dz > 0 ? dz : 0;
  const long long d2 = ddx * ddx + ddy * ddy + ddz * ddz;
  const bool accept = consistent && lvl >= 2 && d2 > thr[lvl];
  if (accept && cb.y > n_direct) return NB_CELL_M2P;
  if (accept || nch == 0) return NB_CELL_P2P;
  return NB_CELL_OPEN;
}

// Near-replica scheme: the walk's stack entries carry the image n of the
// whole subtree, |n|_inf <= W, as code (nx + W) + S (ny + W) + S^2 (nz + W),
// S = 2W + 1, above the cell index.
constexpr int kReplShift = 25;
constexpr unsigned kReplCellMask = (1u << kReplShift) - 1u;

// classify_cell at a given image (k = -n): no consistency condition, and
// cells of any level may be accepted
__device__ __forceinline__ int classify_cell_at(const int4 ca, const int4 cb, const int4 gb, const int4 gc,
                                                const long long* thr, int n_direct, int mac_edge, unsigned code,
                                                int W, int& kx, int& ky, int& kz) {
  const int lvl = ca.w & 0xff, nch = ca.w >> 8, S = 2 * W + 1;
  kx = W - (int)(code % S);
  ky = W - (int)((code / S) % S);
  kz = W - (int)(code / (S * S));
  const int hs = mac_edge ? (1 << (22 - lvl)) : 0;
  const int dx = abs(ca.x - gb.x - kx * NB_PBOX) - gc.x - hs;
  const int dy = abs(ca.y - gb.y - ky * NB_PBOX) - gc.y - hs;
  const int dz = abs(ca.z - gb.z - kz * NB_PBOX) - gc.z - hs;
  const long long ddx = dx > 0 ? dx : 0, ddy = dy > 0 ? dy : 0, ddz = dz > 0 ? dz : 0;
  const long long d2 = ddx * ddx + ddy * ddy + ddz * ddz;
  const bool accept = d2 > thr[lvl];
  if (accept && cb.y > n_direct) return NB_CELL_M2P;
  if (accept || nch == 0) return NB_CELL_P2P;
  return NB_CELL_OPEN;
}

// Image of one source particle of a leaf above level le, from its own
// level-le ancestor key prefix.
__device__ __forceinline__ void particle_image(uint64_t key, int le, const int4 gd, int& kx, int& ky, int& kz) {
  const uint64_t pk = key >> (3 * (NB_QBITS - le));
  kx = img_shift(cell_c2((int)compact3(pk), le), gd.x);
  ky = img_shift(cell_c2((int)compact3(pk >> 1), le), gd.y);
  kz = img_shift(cell_c2((int)compact3(pk >> 2), le), gd.z);
}
