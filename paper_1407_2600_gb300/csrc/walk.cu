// Group tree walk with P2P and M2P interactions (Sec. 2.1: sinks that share
// an interaction list are bundled and their m x n interaction block is
// evaluated together; a multipole acceptance test picks cell expansions or
// opens the cell; near-leaf interactions are direct sums).
//
// One warp per group of <= 32 sinks (one sink per lane).  The warp walks the
// tree cooperatively: it pops up to 32 cells from its stack, each lane tests
// one cell with the integer acceptance test, opened cells push their
// daughters, accepted cells join a queue of M2P interactions that is
// evaluated 32 cells at a time (coefficients staged in shared memory, every
// lane a sink), and leaves are flattened into chunks of 32 source particles
// staged in shared memory for the P2P loop.  Every chunk's partial sum is
// added with Kahan compensation.  The walk order is fixed, so results are
// bitwise reproducible.
//
// Acceptance: in integer units of 2^-23, with the cell at the image of its
// level-l_E ancestor nearest the group's expansion point e (the centre of
// its level-(grid-1) cell), d2 is the squared
// distance from the cell centre to the group box; a cell of level l >= 2
// whose level-l_E descendants share one image is accepted iff
// d2 > floor(s^2/theta^2), s = 2^(23-l).
#include <mutex>
#include <type_traits>
#include <vector>

#include "common.cuh"
#include "m2p_gen.cuh"
#include "walk_common.cuh"

namespace {

template <int P> struct WOrd;
#define NB_WORD(P)                                                                                    \
  template <> struct WOrd<P> {                                                                        \
    static constexpr int NB = kNB##P;                                                                 \
    static constexpr int NBS = (kNB##P + 3) & ~3;                                                     \
    template <typename T>                                                                             \
    static __device__ __forceinline__ void m2p(const T* B, T x, T y, T z, T e2, T& ax, T& ay, T& az) { \
      m2p_p##P<T>(B, x, y, z, e2, ax, ay, az);                                                        \
    }                                                                                                 \
    static __device__ __forceinline__ void m2p2(const float2* B, float2 x, float2 y, float2 z, float2 e2, \
                                                float2& ax, float2& ay, float2& az) {                 \
      m2p2_p##P(B, x, y, z, e2, ax, ay, az);                                                          \
    }                                                                                                 \
  };
NB_WORD(0)
NB_WORD(1)
NB_WORD(2)
NB_WORD(3)
NB_WORD(4)

// Uniform-background term of an expanded cell: order 4 after expansions of
// order 0 and 2, order 6 after order 4 (none at orders 1 and 3, whose
// coefficient rows have no spare slot).  Its weight q = rho h_cell is stored
// in the cell's coefficient row just past the expansion's coefficients.
template <int P> struct WBg {
  static constexpr bool has = false;
  template <typename T>
  static __device__ __forceinline__ void add(T, T, T, T, T&, T&, T&) {}
  static __device__ __forceinline__ void add2(float2, float2, float2, float2, float2&, float2&, float2&) {}
};
#define NB_WBG(P, L)                                                                                        \
  template <> struct WBg<P> {                                                                               \
    static constexpr bool has = true;                                                                       \
    template <typename T>                                                                                   \
    static __device__ __forceinline__ void add(T q, T x, T y, T z, T& ax, T& ay, T& az) {                   \
      cube_bg_l##L<T>(q, x, y, z, ax, ay, az);                                                              \
    }                                                                                                       \
    static __device__ __forceinline__ void add2(float2 q, float2 x, float2 y, float2 z, float2& ax, float2& ay, \
                                                float2& az) {                                               \
      cube_bg2_l##L(q, x, y, z, ax, ay, az);                                                                \
    }                                                                                                       \
  };
NB_WBG(0, 4)
NB_WBG(2, 4)
NB_WBG(4, 6)

template <typename T>
struct WalkArgs {
  DevTree tr;
  const T* coef;
  const typename Vec4<T>::type* src;
  const T* eps2;  // per box
  long long thr[NB_NLEV];
  int n_direct;
  int mac_edge;
  int bg;  // add the uniform-background term of every expanded cell
  int le;
  int* stack;
  int stack_cap;
  int* group_ctr;
  T* acc;  // 3n, key order
  unsigned long long* counters;  // [0] p2p, [1] m2p
  unsigned* status;
};

constexpr double kScale = 1.0 / 8388608.0;  // 2^-23

// PK selects how a chunk of queued M2P cells is evaluated: every lane is a
// sink and loops over the chunk's cells, whose coefficients are staged in
// shared memory and read as broadcasts, one cell at a time (PK = false) or
// two at a time in packed FP32 pairs (PK = true, FP32 only: the coefficients
// of cells 2q and 2q + 1 are staged interleaved and each pair instruction
// advances both expansions, halving the instructions issued per M2P; every
// cell's result is bitwise the scalar one).  The autotuner picks.
template <typename T, int P, int WARPS, int MINB, bool PK>
__global__ void __launch_bounds__(WARPS * 32, MINB) walk_kernel(WalkArgs<T> w) {
  using V4 = typename Vec4<T>::type;
  constexpr int NBS = WOrd<P>::NBS;
  constexpr int C16 = NBS * (int)sizeof(T) / 16;  // 16-byte pieces per cell's coefficients
  __shared__ __align__(16) T s_coef[WARPS][32 * NBS];
  __shared__ V4 s_src[WARPS][32];
  // M2P queue (up to 31 carried + 32 new): centre offset and, in .w, the
  // cell scale 2^level; eps^2 in the cell unit; cell index
  __shared__ V4 s_moff[WARPS][64];
  __shared__ int s_midx[WARPS][64];
  __shared__ T s_meps[WARPS][64];
  __shared__ int s_pfx[WARPS][32];
  __shared__ int s_pst[WARPS][32];
  __shared__ int s_plev[WARPS][32];
  __shared__ T s_poff[WARPS][32][3];
  __shared__ int4 s_pcen[WARPS][32];

  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const unsigned FULL = 0xffffffffu;
  const unsigned ltmask = (1u << lane) - 1u;
  const DevTree& tr = w.tr;
  const int ngroup = tr.cnt[1];
  int* stk = w.stack + ((int64_t)blockIdx.x * WARPS + wid) * w.stack_cap;
  const T scale = (T)kScale;

  while (true) {
    int g = 0;
    if (lane == 0) g = atomicAdd(w.group_ctr, 1);
    g = __shfl_sync(FULL, g, 0);
    if (g >= ngroup) break;
    if (tr.gact && !tr.gact[g]) continue;  // no sink of this group is evaluated
    const int4 ga = tr.gA[g], gb = tr.gB[g], gc = tr.gC[g], gd = tr.gD[g];
    const int cnt = ga.y, box = ga.z;
    const T eps2 = w.eps2[box];
    const bool act = lane < cnt;
    const int i = ga.x + (act ? lane : 0);
    T xi, yi, zi;
    {
      V4 o = w.src[i];
      int4 la = tr.cA[tr.sleaf[i]];
      xi = o.x + (T)(la.x - gd.x) * scale;
      yi = o.y + (T)(la.y - gd.y) * scale;
      zi = o.z + (T)(la.z - gd.z) * scale;
    }
    T ax = 0, ay = 0, az = 0, cx = 0, cy = 0, cz = 0;
    unsigned long long n_p2p = 0, n_m2p = 0;
    int qn = 0;  // queued M2P cells
    // checksum of this lane's (group, cell, decision, cell count) terms and of
    // the group's membership (its sinks' input indices)
    unsigned long long hsum = act ? decision_mix(g, -2 - (int)tr.perm[i], 0) : 0ull;
    // evaluate the first nmp queued M2P cells for every sink of the group
    auto m2p_chunk = [&](int nmp) {
      if constexpr (PK) {
        // stage pairs: cell 2q in .x, cell 2q + 1 in .y (zeros past nmp)
        const int npair = (nmp + 1) >> 1;
        constexpr int C4 = NBS / 4;
        const float4* gsrc = reinterpret_cast<const float4*>(w.coef);
        float4* sdst = reinterpret_cast<float4*>(&s_coef[wid][0]);
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
          float2 px = make_float2(0.f, 0.f), py = px, pz = px;
          const float2 x2 = make_float2(xi, xi), y2 = make_float2(yi, yi), z2 = make_float2(zi, zi);
          const float2* cf = reinterpret_cast<const float2*>(&s_coef[wid][0]);
          auto pairs = [&](auto bgc) {
            for (int q = 0; q < npair; q++) {
              const float4 m0 = s_moff[wid][2 * q];
              const bool two = 2 * q + 1 < nmp;
              const float4 m1 = two ? s_moff[wid][2 * q + 1] : make_float4(0.f, 0.f, 0.f, 1.f);
              const float2 sc = make_float2(m0.w, m1.w);
              const float2 e2 = make_float2(s_meps[wid][2 * q], two ? s_meps[wid][2 * q + 1] : 1.f);
              const float2 rx = __ffma2_rn(x2, sc, make_float2(m0.x, m1.x));
              const float2 ry = __ffma2_rn(y2, sc, make_float2(m0.y, m1.y));
              const float2 rz = __ffma2_rn(z2, sc, make_float2(m0.z, m1.z));
              WOrd<P>::m2p2(&cf[q * NBS], rx, ry, rz, e2, px, py, pz);
              // the padding cell of an odd chunk has weight 0 at R = (0, 0, 0) + offset 0: skip it
              if constexpr (decltype(bgc)::value) {
                const float2 qb = cf[q * NBS + WOrd<P>::NB];
                WBg<P>::add2(two ? qb : make_float2(qb.x, 0.f), rx, ry, two ? rz : make_float2(rz.x, 1.f), px, py,
                             pz);
              }
            }
          };
          if (WBg<P>::has && w.bg) pairs(std::true_type{});
          else pairs(std::false_type{});
          kadd(ax, cx, px.x + px.y);
          kadd(ay, cy, py.x + py.y);
          kadd(az, cz, pz.x + pz.y);
        }
        n_m2p += nmp;
        __syncwarp();
        return;
      }
      const int4* gsrc = reinterpret_cast<const int4*>(w.coef);
      int4* sdst = reinterpret_cast<int4*>(&s_coef[wid][0]);
      for (int t = lane; t < nmp * C16; t += 32) {
        const int q = t / C16, r = t - q * C16;
        sdst[t] = gsrc[(int64_t)s_midx[wid][q] * C16 + r];
      }
      __syncwarp();
      if (act) {
        T px = 0, py = 0, pz = 0;
        // each M2P runs in its cell's unit (coordinates times 2^level,
        // coefficients pre-scaled): see the upward pass
        auto cells = [&](auto bgc) {
          for (int q = 0; q < nmp; q++) {
            const V4 mo = s_moff[wid][q];
            const T rx = fma(xi, mo.w, mo.x), ry = fma(yi, mo.w, mo.y), rz = fma(zi, mo.w, mo.z);
            WOrd<P>::template m2p<T>(&s_coef[wid][q * NBS], rx, ry, rz, s_meps[wid][q], px, py, pz);
            if constexpr (decltype(bgc)::value)
              WBg<P>::template add<T>(s_coef[wid][q * NBS + WOrd<P>::NB], rx, ry, rz, px, py, pz);
          }
        };
        if (WBg<P>::has && w.bg) cells(std::true_type{});
        else cells(std::false_type{});
        kadd(ax, cx, px);
        kadd(ay, cy, py);
        kadd(az, cz, pz);
      }
      n_m2p += nmp;
      __syncwarp();
    };
    int top = 1;
    if (lane == 0) stk[0] = box;  // root of this box
    __syncwarp();
    bool overflow = false;
    while (top > 0) {
      const int nb = min(32, top);
      const int base = top - nb;
      top = base;
      int c = -1;
      int4 ca = make_int4(0, 0, 0, 0), cb = make_int4(0, 0, 0, 0);
      if (lane < nb) {
        c = stk[base + lane];
        ca = tr.cA[c];
        cb = tr.cB[c];
      }
      __syncwarp();
      int cls = NB_CELL_NONE;
      int kx = 0, ky = 0, kz = 0;
      const int lvl = ca.w & 0xff, nch = ca.w >> 8;
      if (lane < nb) {
        cls = classify_cell(ca, cb, gb, gc, gd, w.le, w.thr, w.n_direct, w.mac_edge, kx, ky, kz);
        hsum += decision_mix(g, c, cls | (cb.y << 2));
      }
      // push daughters of opened cells
      {
        const int nc = (cls == 1) ? nch : 0;
        const int pre = warp_excl_scan(nc, lane);
        const int tot = __shfl_sync(FULL, pre + nc, 31);
        if (top + tot > w.stack_cap) {
          overflow = true;
          break;
        }
        for (int q = 0; q < nc; q++) stk[top + pre + q] = cb.z + q;
        top += tot;
        __syncwarp();
      }
      // queue the accepted cells; evaluate whenever 32 are queued
      const unsigned mm = __ballot_sync(FULL, cls == NB_CELL_M2P);
      if (mm) {
        if (cls == NB_CELL_M2P) {
          const int pos = qn + __popc(mm & ltmask);
          s_midx[wid][pos] = c;
          // -(c* - e) 2^level and eps^2 4^level: the cell's unit (exact scalings)
          const T sc = (T)(1 << lvl);
          V4 mo;
          mo.x = -((T)(ca.x - kx * NB_PBOX - gd.x) * scale) * sc;
          mo.y = -((T)(ca.y - ky * NB_PBOX - gd.y) * scale) * sc;
          mo.z = -((T)(ca.z - kz * NB_PBOX - gd.z) * scale) * sc;
          mo.w = sc;
          s_moff[wid][pos] = mo;
          s_meps[wid][pos] = eps2 * (sc * sc);
        }
        qn += __popc(mm);
        if (qn >= 32) {
          __syncwarp();
          m2p_chunk(32);
          // carry the remainder to the front of the queue
          if (lane < qn - 32) {
            s_midx[wid][lane] = s_midx[wid][32 + lane];
            s_moff[wid][lane] = s_moff[wid][32 + lane];
            s_meps[wid][lane] = s_meps[wid][32 + lane];
          }
          qn -= 32;
        }
        __syncwarp();
      }
      // P2P chunks
      const unsigned pm = __ballot_sync(FULL, cls == 3);
      if (pm) {
        const int ncl = (cls == 3) ? cb.y : 0;
        const int pre = warp_excl_scan(ncl, lane);
        const int total = __shfl_sync(FULL, pre + ncl, 31);
        s_pfx[wid][lane] = pre;  // monotone: lanes without P2P add nothing
        s_pst[wid][lane] = cb.x;
        s_plev[wid][lane] = lvl;
        s_pcen[wid][lane] = ca;
        s_poff[wid][lane][0] = (T)(ca.x - kx * NB_PBOX - gd.x) * scale;
        s_poff[wid][lane][1] = (T)(ca.y - ky * NB_PBOX - gd.y) * scale;
        s_poff[wid][lane][2] = (T)(ca.z - kz * NB_PBOX - gd.z) * scale;
        __syncwarp();
        // source t of this pop's P2P cells at its image, relative to e; past
        // the end a massless source at the origin
        auto fetch = [&](int t) {
          V4 v;
          v.x = v.y = v.z = v.w = (T)0;
          if (t < total) {
            // last P2P lane q with pfx[q] <= t
            int lo = 0, hi = 31;
            while (lo < hi) {
              const int mid = (lo + hi + 1) >> 1;
              if (s_pfx[wid][mid] <= t) lo = mid; else hi = mid - 1;
            }
            const int q = lo;
            const int j = s_pst[wid][q] + (t - s_pfx[wid][q]);
            v = w.src[j];
            T ox = s_poff[wid][q][0], oy = s_poff[wid][q][1], oz = s_poff[wid][q][2];
            if (s_plev[wid][q] < w.le) {
              // leaf above the image level: image per particle from its own
              // level-l_E ancestor
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
          }
          return v;
        };
        // the next chunk's sources are fetched while this chunk is summed
        V4 v = fetch(lane);
        for (int b0 = 0; b0 < total; b0 += 32) {
          if constexpr (PK) {
            // pairs of sources interleaved: (x0, x1, y0, y1) then (z0, z1, m0, m1)
            float* pa = reinterpret_cast<float*>(&s_src[wid][0]);
            float* pb = reinterpret_cast<float*>(&s_src[wid][16]);
            const int pr = lane >> 1, hf = lane & 1;
            pa[4 * pr + hf] = v.x;
            pa[4 * pr + 2 + hf] = v.y;
            pb[4 * pr + hf] = v.z;
            pb[4 * pr + 2 + hf] = v.w;
          } else {
            s_src[wid][lane] = v;
          }
          __syncwarp();
          const int nn = min(32, total - b0);
          const V4 vnext = fetch(b0 + 32 + lane);
          if constexpr (PK) {
            if (act) {
              const float4* pa = reinterpret_cast<const float4*>(&s_src[wid][0]);
              const float4* pb = reinterpret_cast<const float4*>(&s_src[wid][16]);
              const float2 nx = make_float2(-xi, -xi), ny = make_float2(-yi, -yi), nz = make_float2(-zi, -zi);
              const float2 e2 = make_float2(eps2, eps2);
              float2 px = make_float2(0.f, 0.f), py = px, pz = px;
              for (int k = 0; k < ((nn + 1) >> 1); k++) {
                const float4 a = pa[k], b = pb[k];
                const float2 dx = __fadd2_rn(make_float2(a.x, a.y), nx);
                const float2 dy = __fadd2_rn(make_float2(a.z, a.w), ny);
                const float2 dz = __fadd2_rn(make_float2(b.x, b.y), nz);
                const float2 r2 = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, __ffma2_rn(dz, dz, e2)));
                const float2 inv = make_float2(nbody_rsqrt(r2.x), nbody_rsqrt(r2.y));
                const float2 f = __fmul2_rn(__fmul2_rn(make_float2(b.z, b.w), __fmul2_rn(inv, inv)), inv);
                px = __ffma2_rn(dx, f, px);
                py = __ffma2_rn(dy, f, py);
                pz = __ffma2_rn(dz, f, pz);
              }
              kadd(ax, cx, px.x + px.y);
              kadd(ay, cy, py.x + py.y);
              kadd(az, cz, pz.x + pz.y);
            }
          } else if (act) {
            T px = 0, py = 0, pz = 0;
            for (int k = 0; k < nn; k++) {
              const V4 s = s_src[wid][k];
              const T dx = s.x - xi, dy = s.y - yi, dz = s.z - zi;
              const T r2 = fma(dx, dx, fma(dy, dy, fma(dz, dz, eps2)));
              const T inv = nbody_rsqrt(r2);
              const T f = s.w * (inv * inv) * inv;
              px = fma(dx, f, px);
              py = fma(dy, f, py);
              pz = fma(dz, f, pz);
            }
            kadd(ax, cx, px);
            kadd(ay, cy, py);
            kadd(az, cz, pz);
          }
          __syncwarp();
          v = vnext;
        }
        n_p2p += (unsigned long long)total;
      }
    }
    if (overflow) {
      if (lane == 0) atomicOr(w.status, NB_ST_OVERFLOW);
      continue;
    }
    if (qn > 0) m2p_chunk(qn);
    if (act && (!tr.sact || tr.sact[i])) {
      w.acc[i] = ax - cx;
      w.acc[tr.n + i] = ay - cy;
      w.acc[2 * tr.n + i] = az - cz;
    }
    if (lane == 0) {
      atomicAdd(&w.counters[0], n_p2p * (unsigned long long)cnt);
      atomicAdd(&w.counters[1], n_m2p * (unsigned long long)cnt);
    }
    for (int o = 16; o > 0; o >>= 1) hsum += __shfl_xor_sync(FULL, hsum, o);
    if (lane == 0) {
      atomicAdd(&w.counters[3], hsum);
    }
  }
}

template <typename T, int P, int WARPS, int MINB, bool PK>
cudaError_t launch_walk(const WalkArgs<T>& a, int nsm, int max_blocks, cudaStream_t s) {
  // resident blocks per SM, queried once per variant (and so never while a
  // stream is being captured, after the first evaluation)
  static int occ = 0;
  if (occ == 0) {
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, walk_kernel<T, P, WARPS, MINB, PK>,
                                                                   WARPS * 32, 0);
    if (e) {
      occ = 0;
      return e;
    }
  }
  int grid = nsm * (occ > 0 ? occ : 1);
  if (grid > max_blocks) grid = max_blocks;
  walk_kernel<T, P, WARPS, MINB, PK><<<grid, WARPS * 32, 0, s>>>(a);
  nb_launch_counter += 1;
  return cudaGetLastError();
}

// launch variants (warps per block, minimum resident blocks per SM, M2P
// form); the register budget per thread follows from the first two.  The
// stack is sized for 8 warps per block.
template <typename T, int P>
cudaError_t launch_variant(int v, const WalkArgs<T>& a, int nsm, int max_blocks, cudaStream_t s) {
  if constexpr (sizeof(T) == 8) {
    return launch_walk<T, P, 4, 1, false>(a, nsm, max_blocks, s);
  } else {
    switch (v) {
      case 0: return launch_walk<T, P, 8, 2, false>(a, nsm, max_blocks, s);
      case 1: return launch_walk<T, P, 8, 3, false>(a, nsm, max_blocks, s);
      case 2: return launch_walk<T, P, 8, 2, true>(a, nsm, max_blocks, s);
      default: return launch_walk<T, P, 4, 5, true>(a, nsm, max_blocks, s);
    }
  }
}
constexpr int kVariants = 4;

struct TuneEntry {
  int device, order, fp64, variant;
  float ms[kVariants];  // the tuning run's time of each variant
};
std::mutex g_tune_mutex;
std::vector<TuneEntry> g_tune;

// Autotuner: the first walk of a (device, precision, order) times every
// variant on the real data and keeps the fastest; results do not depend on
// the variant (each group's walk is the same computation).
template <typename T, int P>
cudaError_t run_walk(const WalkArgs<T>& a, int nsm, int max_blocks, int forced, cudaStream_t s) {
  int dev = 0;
  cudaGetDevice(&dev);
  const int fp = sizeof(T) == 8;
  if (forced >= 0) return launch_variant<T, P>(fp ? 0 : forced, a, nsm, max_blocks, s);
  {
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    for (const auto& t : g_tune)
      if (t.device == dev && t.order == P && t.fp64 == fp) return launch_variant<T, P>(t.variant, a, nsm, max_blocks, s);
  }
  if (fp) {
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    g_tune.push_back({dev, P, fp, 0, {}});
    return launch_variant<T, P>(0, a, nsm, max_blocks, s);
  }
  EventPair ev;
  cudaError_t e;
  if ((e = ev.create())) return e;
  cudaEvent_t e0 = ev.a, e1 = ev.b;
  float best = 1e30f;
  int bv = 0;
  TuneEntry te{dev, P, fp, 0, {}};
  for (int v = 0; v < kVariants; v++) {
    if ((e = cudaMemsetAsync(a.group_ctr, 0, sizeof(int), s))) return e;
    if ((e = cudaMemsetAsync(a.counters, 0, 4 * sizeof(unsigned long long), s))) return e;
    cudaEventRecord(e0, s);
    if ((e = launch_variant<T, P>(v, a, nsm, max_blocks, s))) return e;
    cudaEventRecord(e1, s);
    if ((e = cudaEventSynchronize(e1))) return e;
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    te.ms[v] = ms;
    if (ms < best) {
      best = ms;
      bv = v;
    }
  }
  te.variant = bv;
  {
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    g_tune.push_back(te);
  }
  if ((e = cudaMemsetAsync(a.group_ctr, 0, sizeof(int), s))) return e;
  if ((e = cudaMemsetAsync(a.counters, 0, 4 * sizeof(unsigned long long), s))) return e;
  return launch_variant<T, P>(bv, a, nsm, max_blocks, s);
}

}  // namespace

// warps per block of the walk for a precision (stack slots are sized for the largest)
int nb_walk_warps(bool fp64) { return fp64 ? 4 : 8; }

// the variant the autotuner chose for (precision, order) on this device, or
// -1; ms (nullable, kWalkVariantsMax entries) receives each variant's time
// in the tuning run (0 for variants not timed)
int nb_walk_variant(bool fp64, int order, double* ms) {
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lock(g_tune_mutex);
  for (const auto& t : g_tune)
    if (t.device == dev && t.order == order && t.fp64 == (fp64 ? 1 : 0)) {
      if (ms)
        for (int v = 0; v < kVariants; v++) ms[v] = t.ms[v];
      return t.variant;
    }
  return -1;
}

cudaError_t nb_walk(const DevTree& tr, bool fp64, int order, const void* coef, const void* src,
                    const void* eps2, const long long* thr, int n_direct, int le, int* stack,
                    int stack_cap, int max_blocks, int* group_ctr, void* acc,
                    unsigned long long* counters, unsigned* status, int nsm, int forced_variant,
                    int mac_edge, int bg, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(group_ctr, 0, sizeof(int), s);
  if (e) return e;
#define NB_WALK(TT, P)                                                             \
  {                                                                                \
    WalkArgs<TT> a;                                                                \
    a.tr = tr;                                                                     \
    a.coef = (const TT*)coef;                                                      \
    a.src = (const typename Vec4<TT>::type*)src;                                   \
    a.eps2 = (const TT*)eps2;                                                      \
    for (int l = 0; l < NB_NLEV; l++) a.thr[l] = thr[l];                           \
    a.n_direct = n_direct;                                                         \
    a.mac_edge = mac_edge;                                                         \
    a.bg = bg;                                                                     \
    a.le = le;                                                                     \
    a.stack = stack;                                                               \
    a.stack_cap = stack_cap;                                                       \
    a.group_ctr = group_ctr;                                                       \
    a.acc = (TT*)acc;                                                              \
    a.counters = counters;                                                         \
    a.status = status;                                                             \
    return run_walk<TT, P>(a, nsm, max_blocks, forced_variant, s);                 \
  }
  if (fp64) {
    switch (order) {
      case 0: NB_WALK(double, 0)
      case 1: NB_WALK(double, 1)
      case 2: NB_WALK(double, 2)
      case 3: NB_WALK(double, 3)
      default: NB_WALK(double, 4)
    }
  } else {
    switch (order) {
      case 0: NB_WALK(float, 0)
      case 1: NB_WALK(float, 1)
      case 2: NB_WALK(float, 2)
      case 3: NB_WALK(float, 3)
      default: NB_WALK(float, 4)
    }
  }
#undef NB_WALK
}
