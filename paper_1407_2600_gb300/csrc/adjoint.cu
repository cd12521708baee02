// Reverse mode of the force evaluation (vector-Jacobian product).  Not in the
// paper: the adjoint differentiates the tree force with its discrete decisions
// (tree, groups, images, acceptance) held fixed, so it is the exact derivative
// of the accelerations the forward kernels compute.
//
// For cotangents lam of the accelerations, mu = (da/dx)^T lam collects
//  * per sink: the Hessian-vector products of every M2P expansion used by its
//    group, minus the P2P tidal terms, plus the image field's local Hessian;
//  * per source particle: the P2P tidal terms of every group that summed it
//    directly (a diagonal pairing over the warp, one atomic per source and group);
//  * through the moments: the cotangents of the scaled M2P expansions per cell
//    (atomics), carried down the tree by the transposed shifts (M2M^T) and
//    onto the particles (P2M^T); likewise the image field's cotangents onto
//    the level-3 cells and their particles.
#include <math.h>

#include <mutex>
#include <vector>

#include "common.cuh"
#include "m2p_gen.cuh"
#include "adj_gen.cuh"
#include "walk_common.cuh"

namespace {

template <int P> constexpr int kNBofP() {
  return P == 0 ? kNB0 : P == 1 ? kNB1 : P == 2 ? kNB2 : P == 3 ? kNB3 : kNB4;
}

template <int P> struct AOrd;
#define NB_AORD(P)                                                                                      \
  template <> struct AOrd<P> {                                                                          \
    static constexpr int NBS = (kNB##P + 3) & ~3;                                                       \
    static constexpr int NM = (P + 1) * (P + 2) * (P + 3) / 6;                                          \
    template <typename T>                                                                               \
    static __device__ __forceinline__ void self(const T* B, T x, T y, T z, T e2, T lx, T ly, T lz, T& ox, \
                                                T& oy, T& oz) {                                         \
      m2p_adj_self_p##P<T>(B, x, y, z, e2, lx, ly, lz, ox, oy, oz);                                     \
    }                                                                                                   \
    static __device__ __forceinline__ void self2(const float2* B, float2 x, float2 y, float2 z, float2 e2,  \
                                                 float2 lx, float2 ly, float2 lz, float2& ox, float2& oy,   \
                                                 float2& oz) {                                              \
      m2p2_adj_self_p##P(B, x, y, z, e2, lx, ly, lz, ox, oy, oz);                                       \
    }                                                                                                   \
    template <typename T>                                                                               \
    static __device__ __forceinline__ void src(T x, T y, T z, T e2, T lx, T ly, T lz, T* nu) {          \
      m2p_adj_src_p##P<T>(x, y, z, e2, lx, ly, lz, nu);                                                 \
    }                                                                                                   \
    static __device__ __forceinline__ void m2madj(const double* nup, double x, double y, double z,      \
                                                  double* nuc) {                                        \
      m2m_adj_acc_p##P(nup, x, y, z, nuc);                                                              \
    }                                                                                                   \
    static __device__ __forceinline__ void p2madj(double m, double x, double y, double z, const double* nu, \
                                                  double& gx, double& gy, double& gz) {                 \
      p2m_adj_p##P(m, x, y, z, nu, gx, gy, gz);                                                         \
    }                                                                                                   \
  };
NB_AORD(0)
NB_AORD(1)
NB_AORD(2)
NB_AORD(3)
NB_AORD(4)

// sink-side derivative of the uniform-background term (orders as in the walk);
// the term does not depend on the source particles' positions
template <int P> struct ABg {
  static constexpr bool has = false;
  template <typename T>
  static __device__ __forceinline__ void hvp(T, T, T, T, T, T, T, T&, T&, T&) {}
};
#define NB_ABG(P, L)                                                                                   \
  template <> struct ABg<P> {                                                                          \
    static constexpr bool has = true;                                                                  \
    template <typename T>                                                                              \
    static __device__ __forceinline__ void hvp(T q, T x, T y, T z, T lx, T ly, T lz, T& ox, T& oy, T& oz) { \
      cube_bg_hvp_l##L<T>(q, x, y, z, lx, ly, lz, ox, oy, oz);                                         \
    }                                                                                                  \
  };
NB_ABG(0, 4)
NB_ABG(2, 4)
NB_ABG(4, 6)

template <typename T>
struct AdjArgs {
  DevTree tr;
  const T* coef;
  const typename Vec4<T>::type* src;
  const T* eps2;
  long long thr[NB_NLEV];
  int n_direct, le, mac_edge, bg;
  int* stack;
  int stack_cap;
  int* group_ctr;
  const float* lam;  // 3n, key order
  double* mu;        // 3n, key order
  float* nuc;        // per cell NM, scaled cotangents of the moments
  unsigned* status;
};

constexpr double kScale = 1.0 / 8388608.0;

// The walk of one group, shared by the two reverse-mode kernels: the same
// traversal, classification and M2P queue as the forward walk, with the
// interactions handed to callbacks.  on_m2p(nmp) consumes the first nmp
// queued cells (s_midx, s_moff, s_meps); on_p2p(is_p2p, ca, cb, kx, ky, kz,
// lvl) is called by every lane for the cells of one pop.  Returns false on a
// stack overflow.
template <typename T, typename OnM2P, typename OnP2P>
__device__ __forceinline__ bool adj_walk_group(const DevTree& tr, int box, const int4 gb, const int4 gc, const int4 gd,
                                               int le, const long long* thr, int n_direct, int mac_edge, T eps2, int* stk,
                                               int stack_cap, int lane, int* s_midx,
                                               typename Vec4<T>::type* s_moff, T* s_meps, OnM2P on_m2p,
                                               OnP2P on_p2p) {
  using V4 = typename Vec4<T>::type;
  const unsigned FULL = 0xffffffffu;
  const unsigned ltmask = (1u << lane) - 1u;
  const T scale = (T)kScale;
  int qn = 0;
  int top = 1;
  if (lane == 0) stk[0] = box;
  __syncwarp();
  while (top > 0) {
    const int nb = min(32, top);
    const int base = top - nb;
    top = base;
    int c = -1;
    int4 ca = make_int4(0, 0, 0, 0), cb = make_int4(0, 0, 0, 0);
    if (lane < nb) {
      c = stk[base + lane];
      ca = tr.cA[NB_IDX(c, tr.cnt[0], 601)];
      cb = tr.cB[NB_IDX(c, tr.cnt[0], 601)];
    }
    __syncwarp();
    int cls = NB_CELL_NONE, kx = 0, ky = 0, kz = 0;
    const int lvl = ca.w & 0xff, nch = ca.w >> 8;
    if (lane < nb) cls = classify_cell(ca, cb, gb, gc, gd, le, thr, n_direct, mac_edge, kx, ky, kz);
    {
      const int nc = (cls == NB_CELL_OPEN) ? nch : 0;
      const int pre = warp_excl_scan(nc, lane);
      const int tot = __shfl_sync(FULL, pre + nc, 31);
      if (top + tot > stack_cap) return false;
      for (int q = 0; q < nc; q++) stk[top + pre + q] = cb.z + q;
      top += tot;
      __syncwarp();
    }
    const unsigned mm = __ballot_sync(FULL, cls == NB_CELL_M2P);
    if (mm) {
      if (cls == NB_CELL_M2P) {
        const int pos = qn + __popc(mm & ltmask);
        const T sc = (T)(1 << lvl);
        s_midx[pos] = c;
        V4 mo;
        mo.x = -((T)(ca.x - kx * NB_PBOX - gd.x) * scale) * sc;
        mo.y = -((T)(ca.y - ky * NB_PBOX - gd.y) * scale) * sc;
        mo.z = -((T)(ca.z - kz * NB_PBOX - gd.z) * scale) * sc;
        mo.w = sc;
        s_moff[pos] = mo;
        s_meps[pos] = eps2 * (sc * sc);
      }
      qn += __popc(mm);
      if (qn >= 32) {
        __syncwarp();
        on_m2p(32);
        if (lane < qn - 32) {
          s_midx[lane] = s_midx[32 + lane];
          s_moff[lane] = s_moff[32 + lane];
          s_meps[lane] = s_meps[32 + lane];
        }
        qn -= 32;
      }
      __syncwarp();
    }
    on_p2p(cls == NB_CELL_P2P, ca, cb, kx, ky, kz, lvl);
  }
  if (qn > 0) on_m2p(qn);
  return true;
}

// Sink side: per sink, the Hessian-vector products of every M2P expansion
// its group uses (PK: two cells per packed FP32 pair instruction) and the
// P2P tidal terms, both for the sink and, by a diagonal pairing over the
// warp, for the source particles (one atomic per source and chunk).
template <int P, int WARPS, int MINB, bool PK>
__global__ void __launch_bounds__(WARPS * 32, MINB) adj_sink_kernel(AdjArgs<float> w) {
  using T = float;
  using V4 = float4;
  constexpr int NBS = AOrd<P>::NBS;
  constexpr int C4 = NBS / 4;
  __shared__ __align__(16) T s_coef[WARPS][32 * NBS];
  __shared__ V4 s_src[WARPS][64];
  __shared__ int s_jidx[WARPS][64];
  __shared__ V4 s_moff[WARPS][64];
  __shared__ T s_meps[WARPS][64];
  __shared__ int s_midx[WARPS][64];
  __shared__ int s_pfx[WARPS][32], s_pst[WARPS][32], s_plev[WARPS][32];
  __shared__ T s_poff[WARPS][32][3];
  __shared__ int4 s_pcen[WARPS][32];

  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const unsigned FULL = 0xffffffffu;
  const DevTree& tr = w.tr;
  const int ngroup = tr.cnt[1];
  int* stk = w.stack + ((int64_t)blockIdx.x * WARPS + wid) * w.stack_cap;
  const T scale = (T)kScale;

  while (true) {
    int g = 0;
    if (lane == 0) g = atomicAdd(w.group_ctr, 1);
    g = __shfl_sync(FULL, g, 0);
    if (g >= ngroup) break;
    const int4 ga = tr.gA[g], gb = tr.gB[g], gc = tr.gC[g], gd = tr.gD[g];
    const int cnt = ga.y, box = ga.z;
    const T eps2 = w.eps2[box];
    const bool act = lane < cnt;
    const int i = ga.x + (act ? lane : 0);
    T xi, yi, zi, lx = 0, ly = 0, lz = 0;
    {
      V4 o = w.src[i];
      int4 la = tr.cA[tr.sleaf[i]];
      xi = o.x + (T)(la.x - gd.x) * scale;
      yi = o.y + (T)(la.y - gd.y) * scale;
      zi = o.z + (T)(la.z - gd.z) * scale;
      if (act) {
        lx = w.lam[i];
        ly = w.lam[tr.n + i];
        lz = w.lam[2 * tr.n + i];
      }
    }
    T mx = 0, my = 0, mz = 0;  // sink cotangent
    auto on_m2p = [&](int nmp) {
      const float4* gsrc = reinterpret_cast<const float4*>(w.coef);
      float4* sdst = reinterpret_cast<float4*>(&s_coef[wid][0]);
      if constexpr (PK) {
        const int npair = (nmp + 1) >> 1;
        for (int t = lane; t < npair * C4; t += 32) {
          const int q = t / C4, r = t - q * C4;
          const float4 c0 = gsrc[(int64_t)s_midx[wid][2 * q] * C4 + r];
          const float4 c1 = 2 * q + 1 < nmp ? gsrc[(int64_t)s_midx[wid][2 * q + 1] * C4 + r]
                                           : make_float4(0.f, 0.f, 0.f, 0.f);
          sdst[2 * (q * C4 + r)] = make_float4(c0.x, c1.x, c0.y, c1.y);
          sdst[2 * (q * C4 + r) + 1] = make_float4(c0.z, c1.z, c0.w, c1.w);
        }
        __syncwarp();
        if (act) {
          const float2* cf = reinterpret_cast<const float2*>(&s_coef[wid][0]);
          const float2 x2 = make_float2(xi, xi), y2 = make_float2(yi, yi), z2 = make_float2(zi, zi);
          const float2 l2x = make_float2(lx, lx), l2y = make_float2(ly, ly), l2z = make_float2(lz, lz);
          for (int q = 0; q < npair; q++) {
            const float4 m0 = s_moff[wid][2 * q];
            const bool two = 2 * q + 1 < nmp;
            const float4 m1 = two ? s_moff[wid][2 * q + 1] : make_float4(0.f, 0.f, 0.f, 1.f);
            const float2 sc = make_float2(m0.w, m1.w);
            const float2 e2 = make_float2(s_meps[wid][2 * q], two ? s_meps[wid][2 * q + 1] : 1.f);
            float2 ox = make_float2(0.f, 0.f), oy = ox, oz = ox;
            const float2 rx = __ffma2_rn(x2, sc, make_float2(m0.x, m1.x));
            const float2 ry = __ffma2_rn(y2, sc, make_float2(m0.y, m1.y));
            const float2 rz = __ffma2_rn(z2, sc, make_float2(m0.z, m1.z));
            AOrd<P>::self2(&cf[q * NBS], rx, ry, rz, e2, l2x, l2y, l2z, ox, oy, oz);
            if (ABg<P>::has && w.bg) {
              const float2 qb = cf[q * NBS + kNBofP<P>()];
              ABg<P>::template hvp<float>(qb.x, rx.x, ry.x, rz.x, lx, ly, lz, ox.x, oy.x, oz.x);
              if (two) ABg<P>::template hvp<float>(qb.y, rx.y, ry.y, rz.y, lx, ly, lz, ox.y, oy.y, oz.y);
            }
            // back to box units: times 2^level of each cell
            mx = fma(ox.x, m0.w, fma(ox.y, m1.w, mx));
            my = fma(oy.x, m0.w, fma(oy.y, m1.w, my));
            mz = fma(oz.x, m0.w, fma(oz.y, m1.w, mz));
          }
        }
      } else {
        for (int t = lane; t < nmp * C4; t += 32) {
          const int q = t / C4, r = t - q * C4;
          sdst[t] = gsrc[(int64_t)s_midx[wid][q] * C4 + r];
        }
        __syncwarp();
        if (act) {
          for (int q = 0; q < nmp; q++) {
            const V4 mo = s_moff[wid][q];
            T ox = 0, oy = 0, oz = 0;
            const T rx = fma(xi, mo.w, mo.x), ry = fma(yi, mo.w, mo.y), rz = fma(zi, mo.w, mo.z);
            AOrd<P>::template self<T>(&s_coef[wid][q * NBS], rx, ry, rz, s_meps[wid][q], lx, ly, lz, ox, oy, oz);
            if (ABg<P>::has && w.bg)
              ABg<P>::template hvp<T>(s_coef[wid][q * NBS + kNBofP<P>()], rx, ry, rz, lx, ly, lz, ox, oy, oz);
            mx = fma(ox, mo.w, mx);
            my = fma(oy, mo.w, my);
            mz = fma(oz, mo.w, mz);
          }
        }
      }
      __syncwarp();
    };
    // P2P sources are queued (up to 31 carried + 32 new) and summed 32 at a
    // time, so the diagonal pairing below runs on full chunks
    int qp = 0;
    auto p2p_chunk = [&](int nn) {
      // diagonal pairing: in round k lane l takes source (l+k) mod 32 and
      // passes the source-side term to the lane that owns that source
      T sx = 0, sy = 0, sz = 0;
      for (int k = 0; k < 32; k++) {
        const int q = (lane + k) & 31;
        T wx = 0, wy = 0, wz = 0;
        if (act && q < nn && s_jidx[wid][q] != i) {
          const V4 sv = s_src[wid][q];
          const T dx = sv.x - xi, dy = sv.y - yi, dz = sv.z - zi;
          const T r2 = fma(dx, dx, fma(dy, dy, fma(dz, dz, eps2)));
          const T inv = nbody_rsqrt_pair(r2);
          const T f = (inv * inv) * inv;
          const T g5 = f * (inv * inv) * (T)3;
          const T rl = fma(dx, lx, fma(dy, ly, dz * lz));
          const T a = sv.w * f, bb = sv.w * g5 * rl;
          wx = fma(a, lx, -bb * dx);
          wy = fma(a, ly, -bb * dy);
          wz = fma(a, lz, -bb * dz);
        }
        mx -= wx;
        my -= wy;
        mz -= wz;
        const int from = (lane - k) & 31;
        sx += __shfl_sync(FULL, wx, from);
        sy += __shfl_sync(FULL, wy, from);
        sz += __shfl_sync(FULL, wz, from);
      }
      if (lane < nn && NB_IN(s_jidx[wid][lane], tr.n, 602)) {
        const int j = s_jidx[wid][lane];
        atomicAdd(&w.mu[j], (double)sx);
        atomicAdd(&w.mu[tr.n + j], (double)sy);
        atomicAdd(&w.mu[2 * tr.n + j], (double)sz);
      }
      __syncwarp();
    };
    auto on_p2p = [&](bool mine, const int4 ca, const int4 cb, int kx, int ky, int kz, int lvl) {
      const unsigned pm = __ballot_sync(FULL, mine);
      if (!pm) return;
      const int ncl = mine ? cb.y : 0;
      const int pre = warp_excl_scan(ncl, lane);
      const int total = __shfl_sync(FULL, pre + ncl, 31);
      s_pfx[wid][lane] = pre;
      s_pst[wid][lane] = cb.x;
      s_plev[wid][lane] = lvl;
      s_pcen[wid][lane] = ca;
      s_poff[wid][lane][0] = (T)(ca.x - kx * NB_PBOX - gd.x) * scale;
      s_poff[wid][lane][1] = (T)(ca.y - ky * NB_PBOX - gd.y) * scale;
      s_poff[wid][lane][2] = (T)(ca.z - kz * NB_PBOX - gd.z) * scale;
      __syncwarp();
      for (int b0 = 0; b0 < total; b0 += 32) {
        const int t = b0 + lane;
        if (t < total) {
          int lo = 0, hi = 31;
          while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (s_pfx[wid][mid] <= t) lo = mid; else hi = mid - 1;
          }
          const int q = lo;
          const int j = NB_IDX(s_pst[wid][q] + (t - s_pfx[wid][q]), (int)tr.n, 603);
          V4 v = w.src[j];
          T ox = s_poff[wid][q][0], oy = s_poff[wid][q][1], oz = s_poff[wid][q][2];
          if (s_plev[wid][q] < w.le) {
            const int4 pc = s_pcen[wid][q];
            int jx, jy, jz;
            particle_image(tr.skeys[j], w.le, gd, jx, jy, jz);
            ox = (T)(pc.x - jx * NB_PBOX - gd.x) * scale;
            oy = (T)(pc.y - jy * NB_PBOX - gd.y) * scale;
            oz = (T)(pc.z - jz * NB_PBOX - gd.z) * scale;
          }
          v.x = v.x + ox;
          v.y = v.y + oy;
          v.z = v.z + oz;
          s_src[wid][qp + lane] = v;
          s_jidx[wid][qp + lane] = j;
        }
        qp += min(32, total - b0);
        __syncwarp();
        if (qp >= 32) {
          p2p_chunk(32);
          if (lane < qp - 32) {
            s_src[wid][lane] = s_src[wid][32 + lane];
            s_jidx[wid][lane] = s_jidx[wid][32 + lane];
          }
          qp -= 32;
          __syncwarp();
        }
      }
    };
    const bool ok = adj_walk_group<T>(tr, box, gb, gc, gd, w.le, w.thr, w.n_direct, w.mac_edge, eps2, stk, w.stack_cap, lane,
                                      s_midx[wid], s_moff[wid], s_meps[wid], on_m2p, on_p2p);
    if (!ok) {
      if (lane == 0) atomicOr(w.status, NB_ST_OVERFLOW);
      continue;
    }
    if (qp > 0) p2p_chunk(qp);
    if (act && NB_IN(i, tr.n, 604)) {
      atomicAdd(&w.mu[i], (double)mx);
      atomicAdd(&w.mu[tr.n + i], (double)my);
      atomicAdd(&w.mu[2 * tr.n + i], (double)mz);
    }
  }
}

// Source side: the cotangents of the scaled moments of every cell a group
// expands, summed over the group's sinks by the lane that owns the cell, added
// to the cell with 16-byte vector atomics (stride NMP = NM rounded up to 4).
template <int P, int WARPS, int MINB>
__global__ void __launch_bounds__(WARPS * 32, MINB) adj_src_kernel(AdjArgs<float> w) {
  using T = float;
  using V4 = float4;
  constexpr int NM = AOrd<P>::NM, NMP = (NM + 3) & ~3;
  __shared__ V4 s_moff[WARPS][64];
  __shared__ T s_meps[WARPS][64];
  __shared__ int s_midx[WARPS][64];
  __shared__ V4 s_sx[WARPS][32];  // sink position (xyz) and, in w, unused
  __shared__ V4 s_sl[WARPS][32];  // sink lambda

  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const unsigned FULL = 0xffffffffu;
  const DevTree& tr = w.tr;
  const int ngroup = tr.cnt[1];
  int* stk = w.stack + ((int64_t)blockIdx.x * WARPS + wid) * w.stack_cap;
  const T scale = (T)kScale;

  while (true) {
    int g = 0;
    if (lane == 0) g = atomicAdd(w.group_ctr, 1);
    g = __shfl_sync(FULL, g, 0);
    if (g >= ngroup) break;
    const int4 ga = tr.gA[g], gb = tr.gB[g], gc = tr.gC[g], gd = tr.gD[g];
    const int cnt = ga.y, box = ga.z;
    const T eps2 = w.eps2[box];
    const bool act = lane < cnt;
    const int i = ga.x + (act ? lane : 0);
    {
      V4 o = w.src[i];
      int4 la = tr.cA[tr.sleaf[i]];
      V4 x, l;
      x.x = o.x + (T)(la.x - gd.x) * scale;
      x.y = o.y + (T)(la.y - gd.y) * scale;
      x.z = o.z + (T)(la.z - gd.z) * scale;
      x.w = 0.f;
      l.x = act ? w.lam[i] : 0.f;
      l.y = act ? w.lam[tr.n + i] : 0.f;
      l.z = act ? w.lam[2 * tr.n + i] : 0.f;
      l.w = 0.f;
      s_sx[wid][lane] = x;
      s_sl[wid][lane] = l;
    }
    __syncwarp();
    auto on_m2p = [&](int nmp) {
      if (lane < nmp) {
        const V4 mo = s_moff[wid][lane];
        const T e2 = s_meps[wid][lane];
        T nu[NMP];
#pragma unroll
        for (int t = 0; t < NMP; t++) nu[t] = (T)0;
        for (int sk = 0; sk < cnt; sk++) {
          const V4 x = s_sx[wid][sk], l = s_sl[wid][sk];
          AOrd<P>::template src<T>(fma(x.x, mo.w, mo.x), fma(x.y, mo.w, mo.y), fma(x.z, mo.w, mo.z), e2, l.x,
                                   l.y, l.z, nu);
        }
        float4* dst = reinterpret_cast<float4*>(w.nuc + (int64_t)NB_IDX(s_midx[wid][lane], tr.cnt[0], 605) * NMP);
#pragma unroll
        for (int t = 0; t < NMP / 4; t++) atomicAdd(dst + t, make_float4(nu[4 * t], nu[4 * t + 1], nu[4 * t + 2], nu[4 * t + 3]));
      }
      __syncwarp();
    };
    auto on_p2p = [&](bool, const int4, const int4, int, int, int, int) {};
    const bool ok = adj_walk_group<T>(tr, box, gb, gc, gd, w.le, w.thr, w.n_direct, w.mac_edge, eps2, stk, w.stack_cap, lane,
                                      s_midx[wid], s_moff[wid], s_meps[wid], on_m2p, on_p2p);
    if (!ok && lane == 0) atomicOr(w.status, NB_ST_OVERFLOW);
  }
}

// ---- image field --------------------------------------------------------------------
template <int PE> struct AFE;
#define NB_AFE(PE)                                                                                  \
  template <> struct AFE<PE> {                                                                      \
    static constexpr int NL = kNL##PE;                                                              \
    static constexpr int NE = (PE + 1) * (PE + 2) * (PE + 3) / 6;                                   \
    static constexpr int NP = (PE + 2) * (PE + 3) * (PE + 4) / 6;                                   \
    template <typename T>                                                                           \
    static __device__ __forceinline__ void hess(const T* L, T x, T y, T z, T lx, T ly, T lz, T& ox, T& oy, \
                                                T& oz) {                                            \
      l2p_hess_pe##PE<T>(L, x, y, z, lx, ly, lz, ox, oy, oz);                                       \
    }                                                                                               \
    template <typename T>                                                                           \
    static __device__ __forceinline__ void ladj(T x, T y, T z, T lx, T ly, T lz, T* Lb) {           \
      l2p_adj_pe##PE<T>(x, y, z, lx, ly, lz, Lb);                                                   \
    }                                                                                               \
    template <typename T>                                                                           \
    static __device__ __forceinline__ void madj(const T* Lb, const T* D, T* nu) {                   \
      m2l_adj_pe##PE<T>(Lb, D, nu);                                                                 \
    }                                                                                               \
    static __device__ __forceinline__ void p2madj(double m, double x, double y, double z, const double* nu, \
                                                  double& gx, double& gy, double& gz) {             \
      p2m_adj_p##PE(m, x, y, z, nu, gx, gy, gz);                                                    \
    }                                                                                               \
  };
NB_AFE(1)
NB_AFE(2)
NB_AFE(3)
NB_AFE(4)

__constant__ unsigned char c_apar[84];  // bit d set: multi-index odd in axis d

template <typename T>
struct AFArgs {
  DevTree tr;
  const typename Vec4<T>::type* src;
  const double* fm;   // field moments (box, cell, NE)
  const T* tab;       // phi~ table
  int le, lg;
  const T* lbuf;      // forward per-run expansion (NL, V, Mt)
  int lstride;
  double* lbar;       // per run cotangents (NL + 3)
  int bstride;
  const float* lam;
  double* mu;
  double* nue;        // field-moment cotangents (box, cell, NE)
};

// per group, lane = sink: local Hessian (sink side) and the run's cotangents
template <typename T, int PE>
__global__ void __launch_bounds__(128) adj_field_local_kernel(AFArgs<T> a) {
  using V4 = typename Vec4<T>::type;
  constexpr int NL = AFE<PE>::NL;
  const int lane = threadIdx.x & 31;
  const DevTree& tr = a.tr;
  const int ngroup = tr.cnt[1];
  const T scale = (T)kScale;
  const T fourpi3 = (T)(4.0 * M_PI / 3.0);
  for (int g = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; g < ngroup; g += (gridDim.x * blockDim.x) >> 5) {
    const int4 ga = tr.gA[g], gd = tr.gD[g];
    const bool act = lane < ga.y;
    const T* Lr = a.lbuf + (int64_t)gd.w * a.lstride;
    T Lb[NL];
#pragma unroll
    for (int t = 0; t < NL; t++) Lb[t] = (T)0;
    T lx = 0, ly = 0, lz = 0;
    if (act) {
      const int i = ga.x + lane;
      lx = (T)a.lam[i];
      ly = (T)a.lam[tr.n + i];
      lz = (T)a.lam[2 * tr.n + i];
      const V4 o4 = a.src[i];
      const int4 la = tr.cA[tr.sleaf[i]];
      const T dx = o4.x + (T)(la.x - gd.x) * scale;
      const T dy = o4.y + (T)(la.y - gd.y) * scale;
      const T dz = o4.z + (T)(la.z - gd.z) * scale;
      T L[NL];
#pragma unroll
      for (int t = 0; t < NL; t++) L[t] = Lr[t];
      const T mt = Lr[NL + 3];
      T ox = fourpi3 * mt * lx, oy = fourpi3 * mt * ly, oz = fourpi3 * mt * lz;
      AFE<PE>::template hess<T>(L, dx, dy, dz, lx, ly, lz, ox, oy, oz);
      a.mu[i] += (double)ox;  // one thread per sink: plain adds after the walk's atomics
      a.mu[tr.n + i] += (double)oy;
      a.mu[2 * tr.n + i] += (double)oz;
      AFE<PE>::template ladj<T>(dx, dy, dz, lx, ly, lz, Lb);
    }
    double* dst = a.lbar + (int64_t)gd.w * a.bstride;
#pragma unroll
    for (int t = 0; t < NL; t++) {
      T v = Lb[t];
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0) atomicAdd(dst + t, (double)v);
    }
    T vx = -fourpi3 * lx, vy = -fourpi3 * ly, vz = -fourpi3 * lz;
    for (int o = 16; o > 0; o >>= 1) {
      vx += __shfl_xor_sync(0xffffffffu, vx, o);
      vy += __shfl_xor_sync(0xffffffffu, vy, o);
      vz += __shfl_xor_sync(0xffffffffu, vz, o);
    }
    if (lane == 0) {
      atomicAdd(dst + NL, (double)vx);
      atomicAdd(dst + NL + 1, (double)vy);
      atomicAdd(dst + NL + 2, (double)vz);
    }
  }
}

// per run (warps step through the list of runs), lane = level-le cell:
// transposed M2L onto the cells
template <typename T, int PE>
__global__ void __launch_bounds__(128) adj_field_m2l_kernel(AFArgs<T> a) {
  constexpr int NL = AFE<PE>::NL, NE = AFE<PE>::NE, NP = AFE<PE>::NP;
  const int lane = threadIdx.x & 31;
  const DevTree& tr = a.tr;
  const int nrun = tr.cnt[2];
  const int ncp = 1 << (3 * a.le);
  const int m = (1 << (a.lg - 1)) + 2;
  const int step = 1 << (23 - a.lg);
  for (int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < nrun; r += (gridDim.x * blockDim.x) >> 5) {
    const int g = tr.runhead[r];
    const int4 ga = tr.gA[g];
    const int4 gd = tr.gD[g];
    const int box = ga.z;
    const double* Lbr = a.lbar + (int64_t)gd.w * a.bstride;
    T Lb[NL];
#pragma unroll
    for (int t = 0; t < NL; t++) Lb[t] = (T)Lbr[t];
    const T vbx = (T)Lbr[NL], vby = (T)Lbr[NL + 1], vbz = (T)Lbr[NL + 2];
    for (int cell = lane; cell < ncp; cell += 32) {
      const double* Mc = a.fm + ((int64_t)box * ncp + cell) * NE;
      if (Mc[0] == 0.0) continue;
      const int cx2 = cell_c2((int)compact3((uint64_t)cell), a.le);
      const int cy2 = cell_c2((int)compact3((uint64_t)cell >> 1), a.le);
      const int cz2 = cell_c2((int)compact3((uint64_t)cell >> 2), a.le);
      const int kx = img_shift(cx2, gd.x), ky = img_shift(cy2, gd.y), kz = img_shift(cz2, gd.z);
      const int ox = cx2 - kx * NB_PBOX - gd.x, oy = cy2 - ky * NB_PBOX - gd.y, oz = cz2 - kz * NB_PBOX - gd.z;
      const int irx = -ox / step, iry = -oy / step, irz = -oz / step;
      const int neg = (irx < 0 ? 1 : 0) | (iry < 0 ? 2 : 0) | (irz < 0 ? 4 : 0);
      const int node = (abs(irx) * m + abs(iry)) * m + abs(irz);
      const T* srcp = a.tab + (int64_t)node * NP;
      T D[NP];
#pragma unroll
      for (int t = 0; t < NP; t++) {
        const T v = srcp[t];
        D[t] = (__popc(c_apar[t] & neg) & 1) ? -v : v;
      }
      T nu[NE];
#pragma unroll
      for (int t = 0; t < NE; t++) nu[t] = (T)0;
      AFE<PE>::template madj<T>(Lb, D, nu);
      nu[1] += vbx;  // the background term's dipole (V = sum m (c*-e) + D)
      nu[2] += vby;
      nu[3] += vbz;
      double* dst = a.nue + ((int64_t)box * ncp + cell) * NE;
#pragma unroll
      for (int t = 0; t < NE; t++) atomicAdd(dst + t, (double)nu[t]);
    }
  }
}

// one thread per particle: field-moment cotangents onto the particle
template <int PE>
__global__ void adj_field_p2m_kernel(DevTree tr, int le, const double* __restrict__ nue, double* __restrict__ mu) {
  constexpr int NE = AFE<PE>::NE;
  const int ncp = 1 << (3 * le);
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < tr.n; j += (int64_t)gridDim.x * blockDim.x) {
    const int box = tr.sbox[j];
    const int cell = (int)(tr.skeys[j] >> (3 * (NB_QBITS - le)));
    const double* nu = nue + ((int64_t)box * ncp + cell) * NE;
    double nl[NE];
#pragma unroll
    for (int t = 0; t < NE; t++) nl[t] = nu[t];
    const double cx = i2d_pow2(cell_c2((int)compact3((uint64_t)cell), le), -23);
    const double cy = i2d_pow2(cell_c2((int)compact3((uint64_t)cell >> 1), le), -23);
    const double cz = i2d_pow2(cell_c2((int)compact3((uint64_t)cell >> 2), le), -23);
    double gx = 0, gy = 0, gz = 0;
    AFE<PE>::p2madj((double)tr.smass[j], tr.spos[j] - cx, tr.spos[tr.n + j] - cy, tr.spos[2 * tr.n + j] - cz, nl,
                    gx, gy, gz);
    mu[j] += gx;
    mu[tr.n + j] += gy;
    mu[2 * tr.n + j] += gz;
  }
}

// ---- moments: unscale, down the tree, onto the particles --------------------------------
template <int P>
__global__ void adj_unscale_kernel(const int* __restrict__ pncell, const int4* __restrict__ cA,
                                   const float* __restrict__ nuc, double* __restrict__ nu) {
  constexpr int NM = AOrd<P>::NM, NMP = (NM + 3) & ~3;
  const int ncell = *pncell;
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < ncell; c += gridDim.x * blockDim.x) {
    const int lvl = cA[c].w & 0xff;
    int t = 0;
    for (int o = 0; o <= P; o++) {
      // nu_n = nu'_n (-1)^|n| / n! h^(-2-|n|), h = 2^-level
      const double sc = __longlong_as_double((long long)(1023 + lvl * (2 + o)) << 52) * ((o & 1) ? -1.0 : 1.0);
      for (int nx = o; nx >= 0; nx--)
        for (int ny = o - nx; ny >= 0; ny--, t++) {
          const int nz = o - nx - ny;
          double f = 1.0;
          for (int q = 2; q <= nx; q++) f *= q;
          for (int q = 2; q <= ny; q++) f *= q;
          for (int q = 2; q <= nz; q++) f *= q;
          nu[(int64_t)c * NM + t] = (double)nuc[(int64_t)c * NMP + t] * sc / f;
        }
    }
  }
}

template <int P>
__global__ void adj_down_kernel(const int* __restrict__ pncell, int level, const int4* __restrict__ cA,
                                const int4* __restrict__ cB, double* __restrict__ nu) {
  constexpr int NM = AOrd<P>::NM;
  const int ncell = *pncell;
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < ncell; c += gridDim.x * blockDim.x) {
    const int4 a = cA[c];
    if ((a.w & 0xff) != level) continue;
    const int par = cB[c].w;
    if (par < 0) continue;
    const int4 pa = cA[par];
    double nup[NM], nc[NM];
#pragma unroll
    for (int t = 0; t < NM; t++) {
      nup[t] = nu[(int64_t)par * NM + t];
      nc[t] = nu[(int64_t)c * NM + t];
    }
    AOrd<P>::m2madj(nup, i2d_pow2(a.x - pa.x, -23), i2d_pow2(a.y - pa.y, -23), i2d_pow2(a.z - pa.z, -23), nc);
#pragma unroll
    for (int t = 0; t < NM; t++) nu[(int64_t)c * NM + t] = nc[t];
  }
}

template <int P>
__global__ void adj_p2m_kernel(DevTree tr, const double* __restrict__ nu, double* __restrict__ mu) {
  constexpr int NM = AOrd<P>::NM;
  if (tr.cnt[0] <= 0) return;  // a build that overflowed its capacity formed no leaves
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < tr.n; j += (int64_t)gridDim.x * blockDim.x) {
    const int leaf = tr.sleaf[j];
    const int4 a = tr.cA[leaf];
    double nl[NM];
#pragma unroll
    for (int t = 0; t < NM; t++) nl[t] = nu[(int64_t)leaf * NM + t];
    double gx = 0, gy = 0, gz = 0;
    AOrd<P>::p2madj((double)tr.smass[j], tr.spos[j] - i2d_pow2(a.x, -23), tr.spos[tr.n + j] - i2d_pow2(a.y, -23),
                    tr.spos[2 * tr.n + j] - i2d_pow2(a.z, -23), nl, gx, gy, gz);
    mu[j] += gx;
    mu[tr.n + j] += gy;
    mu[2 * tr.n + j] += gz;
  }
}

__global__ void adj_prep_kernel(int64_t n, const uint32_t* __restrict__ perm, const float* __restrict__ lam,
                                float* __restrict__ lam_s, double* __restrict__ mu) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t j = perm[i];
    for (int d = 0; d < 3; d++) {
      lam_s[d * n + i] = lam[d * n + j];
      mu[d * n + i] = 0.0;
    }
  }
}

__global__ void adj_scatter_kernel(int64_t n, const uint32_t* __restrict__ perm, const double* __restrict__ mu,
                                   double* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t j = perm[i];
    for (int d = 0; d < 3; d++) out[d * n + j] = mu[d * n + i];
  }
}

int gridv(int64_t n, int threads) {
  int64_t g = (n + threads - 1) / threads;
  if (g < 1) g = 1;
  if (g > 152 * 32) g = 152 * 32;
  return (int)g;
}

bool g_apar_done[64] = {false};

}  // namespace

struct AdjBuffers {
  float* lam_s;
  double* mu;
  float* nuc;
  double* nu;
  double* lbar;
  double* nue;
  int* group_ctr;
};

int nb_adj_coef_nm(int order) { return (order + 1) * (order + 2) * (order + 3) / 6; }
int nb_adj_lbar_stride(int pe) { return pe > 0 ? ((pe + 2) * (pe + 3) * (pe + 4) / 6 - 1) + 3 : 0; }

namespace {

template <typename K>
int adj_grid(K kernel, int warps, int max_blocks, int nsm) {
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, warps * 32, 0) != cudaSuccess) occ = 1;
  int grid = nsm * (occ > 0 ? occ : 1);
  if (grid * warps > max_blocks * 8) grid = max_blocks * 8 / warps;
  return grid;
}

// sink-side variants: packed or scalar Hessian-vector products, 4 warps per
// block, 3 or 4 blocks per SM (the register budget follows)
template <int P>
cudaError_t launch_sink(int v, const AdjArgs<float>& a, int max_blocks, int nsm, cudaStream_t s) {
  switch (v) {
    case 0:
      adj_sink_kernel<P, 4, 3, true><<<adj_grid(adj_sink_kernel<P, 4, 3, true>, 4, max_blocks, nsm), 128, 0, s>>>(a);
      break;
    case 1:
      adj_sink_kernel<P, 4, 4, true><<<adj_grid(adj_sink_kernel<P, 4, 4, true>, 4, max_blocks, nsm), 128, 0, s>>>(a);
      break;
    case 2:
      adj_sink_kernel<P, 4, 3, false><<<adj_grid(adj_sink_kernel<P, 4, 3, false>, 4, max_blocks, nsm), 128, 0, s>>>(a);
      break;
    default:
      adj_sink_kernel<P, 4, 4, false><<<adj_grid(adj_sink_kernel<P, 4, 4, false>, 4, max_blocks, nsm), 128, 0, s>>>(a);
      break;
  }
  nb_launch_counter += 1;
  return cudaGetLastError();
}
constexpr int kSinkVariants = 4;
std::mutex g_sink_mutex;
struct SinkTune {
  int device, order, variant;
};
std::vector<SinkTune> g_sink_tune;

template <int P>
cudaError_t launch_adj(const AdjArgs<float>& a, const AdjBuffers& B, const DevTree& tr, const float* lam,
                       int max_blocks, int nsm, cudaStream_t s) {
  cudaError_t e;
  int dev = 0;
  cudaGetDevice(&dev);
  int variant = -1;
  {
    std::lock_guard<std::mutex> lock(g_sink_mutex);
    for (const auto& t : g_sink_tune)
      if (t.device == dev && t.order == P) variant = t.variant;
  }
  if (variant < 0) {
    // time every variant on this call's data; each trial starts from a zero
    // sink cotangent, which the final run below starts from again
    EventPair ev;
    if ((e = ev.create())) return e;
    cudaEvent_t e0 = ev.a, e1 = ev.b;
    float best = 1e30f;
    variant = 0;
    for (int v = 0; v < kSinkVariants; v++) {
      adj_prep_kernel<<<gridv(tr.n, 256), 256, 0, s>>>(tr.n, tr.perm, lam, B.lam_s, B.mu);
      nb_launch_counter += 1;
      if ((e = cudaMemsetAsync(B.group_ctr, 0, sizeof(int), s))) return e;
      cudaEventRecord(e0, s);
      if ((e = launch_sink<P>(v, a, max_blocks, nsm, s))) return e;
      cudaEventRecord(e1, s);
      if ((e = cudaEventSynchronize(e1))) return e;
      float ms = 0;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best) {
        best = ms;
        variant = v;
      }
    }
    std::lock_guard<std::mutex> lock(g_sink_mutex);
    g_sink_tune.push_back({dev, P, variant});
    adj_prep_kernel<<<gridv(tr.n, 256), 256, 0, s>>>(tr.n, tr.perm, lam, B.lam_s, B.mu);
    nb_launch_counter += 1;
  }
  if ((e = cudaMemsetAsync(B.group_ctr, 0, sizeof(int), s))) return e;
  adj_src_kernel<P, 4, 4><<<adj_grid(adj_src_kernel<P, 4, 4>, 4, max_blocks, nsm), 128, 0, s>>>(a);
  nb_launch_counter += 1;
  if ((e = cudaMemsetAsync(B.group_ctr, 0, sizeof(int), s))) return e;
  return launch_sink<P>(variant, a, max_blocks, nsm, s);
}

}  // namespace

cudaError_t nb_forces_vjp(const DevTree& tr, bool fp64, int order, int pe, int le, int lg, const void* coef,
                          const void* src, const void* eps2, const long long* thr, int n_direct, int* stack,
                          int stack_cap, int max_blocks, const double* fm, const void* tab, const void* lbuf,
                          int lstride, int max_level, const float* lam, double* out, const AdjBuffers& B,
                          unsigned* status, int nsm, int mac_edge, int bg, cudaStream_t s) {
  if (fp64) return cudaErrorNotSupported;  // the reverse mode runs the mixed-precision walk
  if (pe > 4) return cudaErrorNotSupported;
  cudaError_t e;
  const int NM = nb_adj_coef_nm(order);
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 64 && !g_apar_done[dev]) {
    unsigned char pm[84];
    for (int o = 0, t = 0; o <= 6; o++)
      for (int nx = o; nx >= 0; nx--)
        for (int ny = o - nx; ny >= 0; ny--, t++) pm[t] = (unsigned char)((nx & 1) | ((ny & 1) << 1) | (((o - nx - ny) & 1) << 2));
    if ((e = cudaMemcpyToSymbol(c_apar, pm, sizeof(pm)))) return e;
    g_apar_done[dev] = true;
  }
  adj_prep_kernel<<<gridv(tr.n, 256), 256, 0, s>>>(tr.n, tr.perm, lam, B.lam_s, B.mu);
  if ((e = cudaMemsetAsync(B.nuc, 0, sizeof(float) * (size_t)tr.ncell * ((NM + 3) & ~3), s))) return e;
  if ((e = cudaMemsetAsync(B.group_ctr, 0, sizeof(int), s))) return e;
  nb_launch_counter += 1;
  {
    AdjArgs<float> a;
    a.tr = tr;
    a.coef = (const float*)coef;
    a.src = (const float4*)src;
    a.eps2 = (const float*)eps2;
    for (int l = 0; l < NB_NLEV; l++) a.thr[l] = thr[l];
    a.n_direct = n_direct;
    a.mac_edge = mac_edge;
    a.bg = bg;
    a.le = le;
    a.stack = stack;
    a.stack_cap = stack_cap;
    a.group_ctr = B.group_ctr;
    a.lam = B.lam_s;
    a.mu = B.mu;
    a.nuc = B.nuc;
    a.status = status;
    // source side, then (group counter reset) sink side; the sink side's
    // launch variant is autotuned on the first call per (device, order)
    switch (order) {
      case 0: e = launch_adj<0>(a, B, tr, lam, max_blocks, nsm, s); break;
      case 1: e = launch_adj<1>(a, B, tr, lam, max_blocks, nsm, s); break;
      case 2: e = launch_adj<2>(a, B, tr, lam, max_blocks, nsm, s); break;
      case 3: e = launch_adj<3>(a, B, tr, lam, max_blocks, nsm, s); break;
      default: e = launch_adj<4>(a, B, tr, lam, max_blocks, nsm, s); break;
    }
    if (e) return e;
  }
  if ((e = cudaGetLastError())) return e;
  if (pe > 0) {
    const int ncp = 1 << (3 * le);
    if ((e = cudaMemsetAsync(B.lbar, 0, sizeof(double) * (size_t)tr.ngroup * nb_adj_lbar_stride(pe), s))) return e;
    const int NE = (pe + 1) * (pe + 2) * (pe + 3) / 6;
    if ((e = cudaMemsetAsync(B.nue, 0, sizeof(double) * (size_t)tr.nbox * ncp * NE, s))) return e;
    AFArgs<float> a{tr, (const float4*)src, fm, (const float*)tab, le, lg, (const float*)lbuf, lstride, B.lbar,
                    nb_adj_lbar_stride(pe), B.lam_s, B.mu, B.nue};
    int grid = (int)(((int64_t)tr.ngroup * 32 + 127) / 128);
    if (grid > 152 * 64) grid = 152 * 64;
    if (grid < 1) grid = 1;
#define NB_ADJF(PE)                                                                          \
  {                                                                                          \
    adj_field_local_kernel<float, PE><<<grid, 128, 0, s>>>(a);                               \
    adj_field_m2l_kernel<float, PE><<<grid, 128, 0, s>>>(a);                                 \
    adj_field_p2m_kernel<PE><<<gridv(tr.n, 128), 128, 0, s>>>(tr, le, B.nue, B.mu);          \
    break;                                                                                   \
  }
    switch (pe) {
      case 1: NB_ADJF(1)
      case 2: NB_ADJF(2)
      case 3: NB_ADJF(3)
      default: NB_ADJF(4)
    }
#undef NB_ADJF
    nb_launch_counter += 3;
    if ((e = cudaGetLastError())) return e;
  }
#define NB_ADJD(P)                                                                                   \
  {                                                                                                  \
    adj_unscale_kernel<P><<<gridv(tr.ncell, 128), 128, 0, s>>>(tr.cnt, tr.cA, B.nuc, B.nu);         \
    for (int l = 1; l <= max_level; l++)                                                             \
      adj_down_kernel<P><<<gridv(tr.ncell, 128), 128, 0, s>>>(tr.cnt, l, tr.cA, tr.cB, B.nu);       \
    adj_p2m_kernel<P><<<gridv(tr.n, 128), 128, 0, s>>>(tr, B.nu, B.mu);                               \
    break;                                                                                           \
  }
  switch (order) {
    case 0: NB_ADJD(0)
    case 1: NB_ADJD(1)
    case 2: NB_ADJD(2)
    case 3: NB_ADJD(3)
    default: NB_ADJD(4)
  }
#undef NB_ADJD
  nb_launch_counter += 2 + max_level;
  adj_scatter_kernel<<<gridv(tr.n, 256), 256, 0, s>>>(tr.n, tr.perm, B.mu, out);
  nb_launch_counter += 1;
  return cudaGetLastError();
}

// fault word of the debug build's bounds checks in this unit (debug build only)
NB_DBG_EXPORT(adjoint)
