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

__device__ __forceinline__ int warp_excl_scan(int v, int lane) {
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  return x - v;
}

enum { NB_CELL_NONE = 0, NB_CELL_OPEN = 1, NB_CELL_M2P = 2, NB_CELL_P2P = 3 };

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

// Image of one source particle of a leaf above level le, from its own
// level-le ancestor key prefix.
__device__ __forceinline__ void particle_image(uint64_t key, int le, const int4 gd, int& kx, int& ky, int& kz) {
  const uint64_t pk = key >> (3 * (NB_QBITS - le));
  kx = img_shift(cell_c2((int)compact3(pk), le), gd.x);
  ky = img_shift(cell_c2((int)compact3(pk >> 1), le), gd.y);
  kz = img_shift(cell_c2((int)compact3(pk >> 2), le), gd.z);
}
