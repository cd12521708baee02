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
    template <typename T, bool REF = true>                                                            \
    static __device__ __forceinline__ void m2p(const T* B, T x, T y, T z, T e2, T& ax, T& ay, T& az) { \
      m2p_p##P<T, REF>(B, x, y, z, e2, ax, ay, az);                                                   \
    }                                                                                                 \
    template <bool REF = true>                                                                        \
    static __device__ __forceinline__ void m2p2(const float2* B, float2 x, float2 y, float2 z, float2 e2, \
                                                float2& ax, float2& ay, float2& az) {                 \
      m2p2_p##P<REF>(B, x, y, z, e2, ax, ay, az);                                                     \
    }                                                                                                 \
    template <typename T>                                                                             \
    static __device__ __forceinline__ T pot(const T* B, T x, T y, T z, T e2) {                        \
      return m2pot_p##P<T>(B, x, y, z, e2);                                                           \
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
  template <typename T>
  static __device__ __forceinline__ T pot(T, T, T, T) { return T(0); }
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
    template <typename T>                                                                                   \
    static __device__ __forceinline__ T pot(T q, T x, T y, T z) {                                           \
      return cube_bgpot_l##L<T>(q, x, y, z);                                                                \
    }                                                                                                       \
  };
NB_WBG(0, 4)
NB_WBG(2, 4)
NB_WBG(4, 6)

// The dual form's cell-group expansion at order P: the softened kernel's
// derivatives to order P + 1 and the M2L one local coefficient at a time
// (m2l_red), the L2P of the image-field code (same truncation, same storage).
template <int P> struct WDual {
  static constexpr bool has = false;
  static constexpr int NL = 1;
  template <typename MA, typename Red>
  static __device__ __forceinline__ void m2l(const MA&, float, float, float, float, Red&&) {}
  static __device__ __forceinline__ void l2p(const float*, float, float, float, float&, float&, float&) {}
};
#define NB_WDUAL(P, Q)                                                                                   \
  template <> struct WDual<P> {                                                                          \
    static constexpr bool has = true;                                                                    \
    static constexpr int NL = kNL##P;                                                                    \
    template <typename MA, typename Red>                                                                 \
    static __device__ __forceinline__ void m2l(const MA& M, float x, float y, float z, float e2, Red&& red) { \
      float D[(Q + 1) * (Q + 2) * (Q + 3) / 6];                                                          \
      dtensor_p##Q<float>(x, y, z, e2, D);                                                               \
      _Pragma("unroll") for (int t = 0; t < (Q + 1) * (Q + 2) * (Q + 3) / 6; t++) D[t] = -D[t];          \
      m2l_red_p##P<float>(M, D, red);                                                                    \
    }                                                                                                    \
    static __device__ __forceinline__ void l2p(const float* L, float x, float y, float z, float& ax, float& ay, \
                                               float& az) {                                              \
      l2p_pe##P<float>(L, x, y, z, ax, ay, az);                                                          \
    }                                                                                                    \
  };
NB_WDUAL(1, 2)
NB_WDUAL(2, 3)
NB_WDUAL(3, 4)
NB_WDUAL(4, 5)

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
  int k1;  // Dehnen K1 softening of direct pairs, Newtonian expansions
  int repl;        // near-replica scheme: W (images |n|_inf <= W walked explicitly), else 0
  int dual;        // cell-group local expansions for well-separated cells
  double theta2;   // theta^2 of the cell-group test (IEEE double, as on the host)
  NbDualBufs db;   // where the walk emits its cell-group pairs
  int le;
  int* stack;
  int stack_cap;
  int* group_ctr;
  T* acc;  // 3n, key order
  T* pot;  // n, key order, or null: the potential variant (see below) writes it
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
//
// POTK adds the potential (scalar form only, not with the dual form): every
// interaction's potential form alongside its acceleration, -Psi with Psi =
// sum_j F_j S_j for an expansion (divided by its cell scale), the background
// term's q h / r^(2l+1), and m (r^2 + eps^2)^-1/2 (or the K1 kernel's
// potential) for a direct pair other than the sink itself.
template <typename T, int P, int WARPS, int MINB, bool PK, bool DUALK, bool POTK = false>
__global__ void __launch_bounds__(WARPS * 32, MINB) walk_kernel(WalkArgs<T> w) {
  static_assert(!POTK || (!PK && !DUALK), "the potential variant is scalar and without the dual form");
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
  __shared__ T s_b0[WARPS][32];  // monopole coefficient of the chunk's largest cells
  // double-float sums of the largest cells' monopole terms, per lane (hi x3, lo x3)
  __shared__ float s_df[WARPS][6][32];
  // dual form: queue of cell-group pairs (cell, image shift code) and the
  // cell-group thresholds per level
  __shared__ int s_lidx[WARPS][DUALK ? 64 : 1];
  __shared__ int s_limg[WARPS][DUALK ? 64 : 1];
  __shared__ long long s_tl[WARPS][DUALK ? NB_NLEV : 1];
  __shared__ int s_pfx[WARPS][32];
  __shared__ int s_pst[WARPS][32];
  __shared__ int s_plev[WARPS][32];
  __shared__ T s_poff[WARPS][32][3];
  __shared__ int4 s_pcen[WARPS][32];
  // the next pop's stack entries and cell records, copied while this pop's
  // interactions are summed
  __shared__ unsigned s_ne[WARPS][32];
  __shared__ __align__(16) int4 s_nA[WARPS][32];
  __shared__ __align__(16) int4 s_nB[WARPS][32];
  __shared__ int s_sj[WARPS][POTK ? 32 : 1];  // the staged sources' indices (the sink's own pair is skipped)
  __shared__ int s_pctr[WARPS][POTK ? 32 : 1];  // replicas: the P2P cell is at the central image

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
      V4 o = w.src[NB_IDX(i, tr.n, 101)];
      int4 la = tr.cA[NB_IDX(tr.sleaf[NB_IDX(i, tr.n, 101)], tr.cnt[0], 102)];
      xi = o.x + (T)(la.x - gd.x) * scale;
      yi = o.y + (T)(la.y - gd.y) * scale;
      zi = o.z + (T)(la.z - gd.z) * scale;
    }
    T ax = 0, ay = 0, az = 0, cx = 0, cy = 0, cz = 0;
    T ps = 0, pc = 0;  // Psi (the potential is -Psi), Kahan pair
    // double-float sum of the largest cells' monopole terms (FP32 walk only),
    // kept in shared memory: it changes once per such cell
    constexpr bool DF = std::is_same<T, float>::value;
    if constexpr (DF)
#pragma unroll
      for (int k = 0; k < 6; k++) s_df[wid][k][lane] = 0.f;
    unsigned long long n_p2p = 0, n_m2p = 0, n_m2l = 0;
    int qn = 0;  // queued M2P cells
    int pcar = 0;  // P2P sources staged but not yet summed (carried to the next pop)
    int ln = 0;  // queued cell-group (M2L) cells
    constexpr bool DUAL = DUALK && DF && WDual<P>::has;
    int lprev = -1;  // this group's last emitted chunk of cell-group pairs
    if constexpr (DUAL) {
      if (w.dual) {
        if (lane < NB_NLEV) {
          // (s_C + s_G)^2 / theta^2 with s_G the group box's largest side
          const long long wmax = max(gc.x, max(gc.y, gc.z));
          const long long S = (1ll << (23 - min(lane, 23))) + 2 * wmax;
          s_tl[wid][lane] = (long long)floor((double)S * (double)S / w.theta2);
        }
        __syncwarp();
      }
    }
    // checksum of this lane's (group, cell, decision, cell count) terms and of
    // the group's membership (its sinks' input indices)
    unsigned long long hsum = act ? decision_mix(g, -2 - (int)tr.perm[i], 0) : 0ull;
    // the largest queued cells' monopole terms, in double-float (their
    // coefficient was taken out of the expansions of the chunk).  Done with
    // the uniform-background terms, i.e. for the nearly uniform states
    // where those terms cancel a thousandfold.
    auto df_monopoles = [&](int nmp) {
      if (!w.bg) return;
      float sh[3], sl[3];
#pragma unroll
      for (int k = 0; k < 3; k++) {
        sh[k] = s_df[wid][k][lane];
        sl[k] = s_df[wid][3 + k][lane];
      }
      for (int q = 0; q < nmp; q++) {
        const V4 mo = s_moff[wid][q];
        if (mo.w <= (T)kDfScale)
          mono_df((float)xi, (float)yi, (float)zi, (float)mo.w, (float)mo.x, (float)mo.y, (float)mo.z,
                  (float)s_meps[wid][q], (float)s_b0[wid][q], sh, sl);
      }
#pragma unroll
      for (int k = 0; k < 3; k++) {
        s_df[wid][k][lane] = sh[k];
        s_df[wid][3 + k][lane] = sl[k];
      }
    };
    // dual form: the first nml queued cell-group pairs become one chunk of
    // the group's pair list (a separate pass forms their local expansions)
    auto m2l_chunk = [&](int nml) {
      if constexpr (DUAL) {
        int cidx = 0;
        if (lane == 0) cidx = atomicAdd(w.db.ctr, 1);
        cidx = __shfl_sync(FULL, cidx, 0);
        if (cidx < w.db.cap) {
          if (lane < nml) {
            w.db.cell[(int64_t)cidx * 32 + lane] = s_lidx[wid][lane];
            w.db.img[(int64_t)cidx * 32 + lane] = s_limg[wid][lane];
          }
          if (lane == 0) {
            w.db.head[cidx] = make_int4(g, nml, -1, 0);
            if (lprev < 0) w.db.first[g] = cidx;
            else w.db.head[lprev].z = cidx;
          }
          lprev = cidx;
        } else if (lane == 0) {
          atomicOr(w.status, NB_ST_OVERFLOW);  // the pool is too small: the caller grows it
        }
        n_m2l += nml;
      }
    };
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
          const float4 c0 = gsrc[(int64_t)NB_IDX(s_midx[wid][2 * q], tr.cnt[0], 105) * C4 + r];
          const float4 c1 = 2 * q + 1 < nmp ? gsrc[(int64_t)NB_IDX(s_midx[wid][2 * q + 1], tr.cnt[0], 105) * C4 + r]
                                           : make_float4(0.f, 0.f, 0.f, 0.f);
          sdst[2 * (q * C4 + r)] = make_float4(c0.x, c1.x, c0.y, c1.y);
          sdst[2 * (q * C4 + r) + 1] = make_float4(c0.z, c1.z, c0.w, c1.w);
        }
        __syncwarp();
        // the largest cells' monopoles are summed in double-float: out of the pair expansion
        if (w.bg && lane < nmp && s_moff[wid][lane].w <= kDfScale) {
          float* slot0 = &s_coef[wid][2 * (lane >> 1) * NBS + (lane & 1)];
          s_b0[wid][lane] = *slot0;
          *slot0 = 0.f;
        }
        __syncwarp();
        if (act) {
          // each cell's term is formed from zero and added to the chunk sum
          // once (the largest cells' monopoles, the terms that cancel most,
          // are summed apart in double-float)
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
              float2 tx = make_float2(0.f, 0.f), ty = tx, tz = tx;
              // the refined reciprocal square root where it matters: near-uniform
              // boxes, i.e. with the uniform-background terms
              WOrd<P>::template m2p2<decltype(bgc)::value>(&cf[q * NBS], rx, ry, rz, e2, tx, ty, tz);
              // the padding cell of an odd chunk has weight 0 at R = (0, 0, 0) + offset 0: skip it
              if constexpr (decltype(bgc)::value) {
                const float2 qb = cf[q * NBS + WOrd<P>::NB];
                WBg<P>::add2(two ? qb : make_float2(qb.x, 0.f), rx, ry, two ? rz : make_float2(rz.x, 1.f), tx, ty,
                             tz);
              }
              px = __fadd2_rn(px, tx);
              py = __fadd2_rn(py, ty);
              pz = __fadd2_rn(pz, tz);
            }
          };
          if (WBg<P>::has && w.bg) pairs(std::true_type{});
          else pairs(std::false_type{});
          df_monopoles(nmp);
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
        sdst[t] = gsrc[(int64_t)NB_IDX(s_midx[wid][q], tr.cnt[0], 105) * C16 + r];
      }
      __syncwarp();
      if constexpr (DF) {
        // the largest cells' monopoles are summed in double-float: out of the expansion
        if (w.bg && lane < nmp && s_moff[wid][lane].w <= kDfScale) {
          s_b0[wid][lane] = s_coef[wid][lane * NBS];
          s_coef[wid][lane * NBS] = (T)0;
        }
        __syncwarp();
      }
      if (act) {
        // each cell's term is formed from zero and added to the chunk sum
        // once (the largest cells' monopoles, the terms that cancel most,
        // are summed apart in double-float)
        T px = 0, py = 0, pz = 0, pp = 0;
        // each M2P runs in its cell's unit (coordinates times 2^level,
        // coefficients pre-scaled): see the upward pass
        auto cells = [&](auto bgc) {
          for (int q = 0; q < nmp; q++) {
            const V4 mo = s_moff[wid][q];
            const T rx = fma(xi, mo.w, mo.x), ry = fma(yi, mo.w, mo.y), rz = fma(zi, mo.w, mo.z);
            T tx = 0, ty = 0, tz = 0;
            WOrd<P>::template m2p<T, decltype(bgc)::value>(&s_coef[wid][q * NBS], rx, ry, rz, s_meps[wid][q], tx,
                                                           ty, tz);
            if constexpr (decltype(bgc)::value)
              WBg<P>::template add<T>(s_coef[wid][q * NBS + WOrd<P>::NB], rx, ry, rz, tx, ty, tz);
            px += tx;
            py += ty;
            pz += tz;
            if constexpr (POTK) {
              // Psi in the cell's unit is 2^level times the true one
              T tp = WOrd<P>::template pot<T>(&s_coef[wid][q * NBS], rx, ry, rz, s_meps[wid][q]);
              if constexpr (decltype(bgc)::value)
                tp += WBg<P>::template pot<T>(s_coef[wid][q * NBS + WOrd<P>::NB], rx, ry, rz);
              if (DF && w.bg && mo.w <= (T)kDfScale)  // the monopole taken out of the expansion
                tp += s_b0[wid][q] * nbody_rsqrt(fma(rx, rx, fma(ry, ry, fma(rz, rz, s_meps[wid][q]))));
              pp = fma(tp, (T)1 / mo.w, pp);
            }
          }
        };
        if (WBg<P>::has && w.bg) cells(std::true_type{});
        else cells(std::false_type{});
        if constexpr (DF) df_monopoles(nmp);
        kadd(ax, cx, px);
        kadd(ay, cy, py);
        kadd(az, cz, pz);
        if constexpr (POTK) kadd(ps, pc, pp);
      }
      n_m2p += nmp;
      __syncwarp();
    };
    int top = 1;
    if (w.repl) {
      // the root at every near image, |n|_inf <= W
      const int S1 = 2 * w.repl + 1;
      top = S1 * S1 * S1;
      for (int r = lane; r < top; r += 32) stk[r] = (int)((unsigned)box | ((unsigned)r << kReplShift));
    } else if (lane == 0) {
      stk[0] = box;  // root of this box
    }
    __syncwarp();
    // start copying the cell records of the next pop (the top min(32, top)
    // stack entries) to shared memory; the pop waits for them
    auto prefetch_pop = [&]() {
      const int nb2 = min(32, top);
      if (lane < nb2) {
        const unsigned e = (unsigned)stk[top - nb2 + lane];
        const int c2 = (int)(e & kReplCellMask);
        s_ne[wid][lane] = e;
        cp_async16(&s_nA[wid][lane], &tr.cA[NB_IDX(c2, tr.cnt[0], 104)]);
        cp_async16(&s_nB[wid][lane], &tr.cB[NB_IDX(c2, tr.cnt[0], 104)]);
      }
      cp_async_commit();
    };
    prefetch_pop();
    bool overflow = false;
    // each chunk routine has one call site (the end of this loop), which
    // keeps the kernel's instruction footprint small
    while (true) {
      const int nb = min(32, top);
      const int base = top - nb;
      top = base;
      int c = -1;
      unsigned code = 0;  // replicas: the image of this entry's subtree
      int4 ca = make_int4(0, 0, 0, 0), cb = make_int4(0, 0, 0, 0);
      cp_async_wait_all();  // each lane reads back only the slots it filled
      if (lane < nb) {
        const unsigned e = s_ne[wid][lane];
        c = (int)(e & kReplCellMask);
        code = e >> kReplShift;
        ca = s_nA[wid][lane];
        cb = s_nB[wid][lane];
      }
      __syncwarp();
      int cls = NB_CELL_NONE;
      int kx = 0, ky = 0, kz = 0;
      const int lvl = ca.w & 0xff, nch = ca.w >> 8;
      if (lane < nb) {
        cls = w.repl ? classify_cell_at(ca, cb, gb, gc, w.thr, w.n_direct, w.mac_edge, code, w.repl, kx, ky, kz)
                     : classify_cell(ca, cb, gb, gc, gd, w.le, w.thr, w.n_direct, w.mac_edge, kx, ky, kz);
        if constexpr (DUAL) {
          if (w.dual && cls == NB_CELL_M2P) {
            // cell-group test: centre-to-centre distance against (s_C + s_G)/theta
            const long long dx = ca.x - kx * NB_PBOX - gb.x, dy = ca.y - ky * NB_PBOX - gb.y,
                            dz = ca.z - kz * NB_PBOX - gb.z;
            if (dx * dx + dy * dy + dz * dz > s_tl[wid][lvl]) cls = NB_CELL_M2L;
          }
        }
        hsum += decision_mix(g, (int)((unsigned)c | (code << kReplShift)), cls | (cb.y << 3));
      }
      // push daughters of opened cells (at the same image)
      {
        const int nc = (cls == 1) ? nch : 0;
        const int pre = warp_excl_scan(nc, lane);
        const int tot = __shfl_sync(FULL, pre + nc, 31);
        if (top + tot > w.stack_cap) {
          overflow = true;
          break;
        }
        for (int q = 0; q < nc; q++) stk[top + pre + q] = (int)((unsigned)(cb.z + q) | (code << kReplShift));
        top += tot;
        __syncwarp();
        prefetch_pop();  // nothing below changes the stack before the next pop
      }
      // queue the accepted cells; evaluate whenever 32 are queued
      const unsigned mm = __ballot_sync(FULL, cls == NB_CELL_M2P);
      if (mm) {
        if (cls == NB_CELL_M2P && NB_IN(qn + __popc(mm & ltmask), 64, 106)) {
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
          s_meps[wid][pos] = w.k1 ? (T)0 : eps2 * (sc * sc);
        }
        qn += __popc(mm);
        __syncwarp();
      }
      if constexpr (DUAL) {
        const unsigned lm = __ballot_sync(FULL, cls == NB_CELL_M2L);
        if (lm) {
          if (cls == NB_CELL_M2L && NB_IN(ln + __popc(lm & ltmask), 64, 107)) {
            const int pos = ln + __popc(lm & ltmask);
            s_lidx[wid][pos] = c;
            s_limg[wid][pos] = (kx + 2) | ((ky + 2) << 3) | ((kz + 2) << 6);
          }
          ln += __popc(lm);
          __syncwarp();
        }
      }
      // P2P chunks.  This pop's sources join the ones carried over from
      // earlier pops (already staged at positions 0..pcar-1 of s_src), and
      // until the stack is empty only full chunks of 32 are summed, so that
      // nearly every chunk is full; the rest stays staged for the next pop.
      const bool fin = top == 0;
      const unsigned pm = __ballot_sync(FULL, cls == 3);
      if (pm || (fin && pcar > 0)) {
        const int ncl = (cls == 3) ? cb.y : 0;
        const int pre = warp_excl_scan(ncl, lane);
        const int total = __shfl_sync(FULL, pre + ncl, 31);
        s_pfx[wid][lane] = pre;  // monotone: lanes without P2P add nothing
        s_pst[wid][lane] = cb.x;
        s_plev[wid][lane] = lvl;
        s_pcen[wid][lane] = ca;
        if constexpr (POTK) s_pctr[wid][lane] = kx == 0 && ky == 0 && kz == 0;
        s_poff[wid][lane][0] = (T)(ca.x - kx * NB_PBOX - gd.x) * scale;
        s_poff[wid][lane][1] = (T)(ca.y - ky * NB_PBOX - gd.y) * scale;
        s_poff[wid][lane][2] = (T)(ca.z - kz * NB_PBOX - gd.z) * scale;
        __syncwarp();
        // source t of this pop's P2P cells at its image, relative to e; past
        // the end a massless source at the origin
        auto fetch = [&](int t, int& jo) {
          V4 v;
          v.x = v.y = v.z = v.w = (T)0;
          jo = -1;
          if (t >= 0 && t < total) {
            // last P2P lane q with pfx[q] <= t
            int lo = 0, hi = 31;
            while (lo < hi) {
              const int mid = (lo + hi + 1) >> 1;
              if (s_pfx[wid][mid] <= t) lo = mid; else hi = mid - 1;
            }
            const int q = lo;
            const int j = s_pst[wid][q] + (t - s_pfx[wid][q]);
            if constexpr (POTK) jo = (!w.repl || s_pctr[wid][q]) ? j : -1;  // a replica's pair is never the self pair
            v = w.src[NB_IDX(j, tr.n, 103)];
            T ox = s_poff[wid][q][0], oy = s_poff[wid][q][1], oz = s_poff[wid][q][2];
            if (!w.repl && s_plev[wid][q] < w.le) {
              // leaf above the image level: image per particle from its own
              // level-l_E ancestor
              const int4 pc = s_pcen[wid][q];
              int jx, jy, jz;
              particle_image(tr.skeys[NB_IDX(j, tr.n, 103)], w.le, gd, jx, jy, jz);
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
        // combined position k = b0 + lane: the carried sources, then source
        // k - pcar of this pop; the next chunk's sources are fetched while
        // this chunk is summed
        const int pc0 = pcar, avail = pc0 + total;
        pcar = fin ? 0 : (avail & 31);
        int jv = -1, jnext = -1;
        V4 v = fetch(lane - pc0, jv);
        for (int b0 = 0; b0 < avail; b0 += 32) {
          if (b0 > 0 || lane >= pc0) {  // a carried source stays where it is
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
              if constexpr (POTK) s_sj[wid][lane] = jv;
            }
          }
          __syncwarp();
          const int nn = min(32, avail - b0);
          if (nn < 32 && !fin) break;  // a partial chunk waits for the next pop's sources
          const V4 vnext = fetch(b0 + 32 + lane - pc0, jnext);
          // pair factor f of a = m d f: Plummer (r^2 + eps^2)^(-3/2), or the
          // K1 kernel, Newtonian from eps on and (175/16 - (147/8) x^2 +
          // (135/16) x^4)/eps^3 inside (x = r/eps: the enclosed mass of its
          // compensating density over r^3); the self pair has d = 0
          auto pairs = [&](auto k1c) {
            constexpr bool K1 = decltype(k1c)::value;
            const T e2p = K1 ? (T)0 : eps2;
            const T ie2 = K1 ? (T)1 / eps2 : (T)0;
            const T ie3 = K1 ? ie2 * sqrt(ie2) : (T)0;
            if constexpr (PK) {
              if (act) {
                const float4* pa = reinterpret_cast<const float4*>(&s_src[wid][0]);
                const float4* pb = reinterpret_cast<const float4*>(&s_src[wid][16]);
                const float2 nx = make_float2(-xi, -xi), ny = make_float2(-yi, -yi), nz = make_float2(-zi, -zi);
                const float2 e2 = make_float2(e2p, e2p);
                float2 px = make_float2(0.f, 0.f), py = px, pz = px;
                // unrolled: consecutive pairs' chains overlap (2.4 % off the walk)
#pragma unroll 8
                for (int k = 0; k < ((nn + 1) >> 1); k++) {
                  const float4 a = pa[k], b = pb[k];
                  const float2 dx = __fadd2_rn(make_float2(a.x, a.y), nx);
                  const float2 dy = __fadd2_rn(make_float2(a.z, a.w), ny);
                  const float2 dz = __fadd2_rn(make_float2(b.x, b.y), nz);
                  const float2 r2 = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, __ffma2_rn(dz, dz, e2)));
                  const float2 inv = make_float2(nbody_rsqrt_pair(r2.x), nbody_rsqrt_pair(r2.y));
                  float2 f = __fmul2_rn(__fmul2_rn(make_float2(b.z, b.w), __fmul2_rn(inv, inv)), inv);
                  if constexpr (K1) {
                    const float x2a = r2.x * ie2, x2b = r2.y * ie2;
                    if (x2a < 1.f) f.x = b.z * ie3 * fmaf(x2a, fmaf(x2a, 135.f / 16.f, -147.f / 8.f), 175.f / 16.f);
                    if (x2b < 1.f) f.y = b.w * ie3 * fmaf(x2b, fmaf(x2b, 135.f / 16.f, -147.f / 8.f), 175.f / 16.f);
                  }
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
              [[maybe_unused]] T pp = 0;
              for (int k = 0; k < nn; k++) {
                const V4 s = s_src[wid][k];
                const T dx = s.x - xi, dy = s.y - yi, dz = s.z - zi;
                const T r2 = fma(dx, dx, fma(dy, dy, fma(dz, dz, e2p)));
                const T inv = nbody_rsqrt_pair(r2);
                T f = s.w * (inv * inv) * inv;
                if constexpr (K1) {
                  const T x2 = r2 * ie2;
                  if (x2 < (T)1)
                    f = s.w * ie3 * fma(x2, fma(x2, (T)(135.0 / 16.0), (T)(-147.0 / 8.0)), (T)(175.0 / 16.0));
                }
                px = fma(dx, f, px);
                py = fma(dy, f, py);
                pz = fma(dz, f, pz);
                if constexpr (POTK) {
                  // m (r^2 + eps^2)^-1/2, or K1's m (105/32 - 175/32 x^2 + 147/32 x^4 - 45/32 x^6)/eps inside eps
                  T u = s.w * inv;
                  if constexpr (K1) {
                    const T x2 = r2 * ie2;
                    if (x2 < (T)1)
                      u = s.w * sqrt(ie2) *
                          fma(x2, fma(x2, fma(x2, (T)(-45.0 / 32.0), (T)(147.0 / 32.0)), (T)(-175.0 / 32.0)),
                              (T)(105.0 / 32.0));
                  }
                  if (s_sj[wid][k] != i) pp += u;
                }
              }
              kadd(ax, cx, px);
              kadd(ay, cy, py);
              kadd(az, cz, pz);
              if constexpr (POTK) kadd(ps, pc, pp);
            }
          };
          if (w.k1) pairs(std::true_type{});
          else pairs(std::false_type{});
          __syncwarp();
          v = vnext;
          jv = jnext;
        }
        n_p2p += (unsigned long long)total;
      }
      // evaluate queued cells 32 at a time, and what is left once the stack
      // is empty (up to two chunks then: the queue holds up to 63)
      while (qn >= 32 || (fin && qn > 0)) {
        const int k = min(qn, 32);
        __syncwarp();
        m2p_chunk(k);
        // carry the remainder to the front of the queue
        if (lane < qn - k) {
          s_midx[wid][lane] = s_midx[wid][32 + lane];
          s_moff[wid][lane] = s_moff[wid][32 + lane];
          s_meps[wid][lane] = s_meps[wid][32 + lane];
        }
        qn -= k;
        __syncwarp();
      }
      if constexpr (DUAL) {
        while (ln >= 32 || (fin && ln > 0)) {
          const int k = min(ln, 32);
          __syncwarp();
          m2l_chunk(k);
          if (lane < ln - k) {
            s_lidx[wid][lane] = s_lidx[wid][32 + lane];
            s_limg[wid][lane] = s_limg[wid][32 + lane];
          }
          ln -= k;
          __syncwarp();
        }
      }
      if (fin) break;
    }
    if (overflow) {
      if (lane == 0) atomicOr(w.status, NB_ST_OVERFLOW);
      continue;
    }
    if (act && NB_IN(i, tr.n, 108) && (!tr.sact || tr.sact[i])) {
      if constexpr (DF) {
        // (ax - cx) + (dsh + dsl), the large parts added error-free first
        const T a3[3] = {ax, ay, az}, c3[3] = {cx, cy, cz};
#pragma unroll
        for (int d = 0; d < 3; d++) {
          float h, e;
          two_sum(s_df[wid][d][lane], a3[d], h, e);
          w.acc[d * tr.n + i] = h + ((e + s_df[wid][3 + d][lane]) - c3[d]);
        }
      } else {
        w.acc[i] = ax - cx;
        w.acc[tr.n + i] = ay - cy;
        w.acc[2 * tr.n + i] = az - cz;
      }
      if constexpr (POTK) w.pot[i] = -(ps - pc);
    }
    if (lane == 0) {
      atomicAdd(&w.counters[0], n_p2p * (unsigned long long)cnt);
      atomicAdd(&w.counters[1], n_m2p * (unsigned long long)cnt);
      if (n_m2l) atomicAdd(&w.counters[4], n_m2l);  // one per (cell, group)
    }
    for (int o = 16; o > 0; o >>= 1) hsum += __shfl_xor_sync(FULL, hsum, o);
    if (lane == 0) {
      atomicAdd(&w.counters[3], hsum);
    }
  }
}

// ---- the dual form's cell-group expansions ----------------------------------------
struct DualArgs {
  DevTree tr;
  NbDualBufs db;
  const float* mom32;  // FP32 cell-unit moments (kDualStride per cell)
  const float* eps2;   // per box
  int k1;
  int lu;              // the groups' length unit 2^-lu (level of the cell no group straddles)
  float* acc;          // 3n, key order (the walk's accelerations; the expansions are added)
};

// One warp per chunk of cell-group pairs, lane per pair: the cell's local
// expansion about the group-box centre z at R = (z - c*) 2^level (its unit;
// derivatives by the Cartesian recurrence), each coefficient taken to the
// group's unit (x 2^((level - lu)(|k| + 1))) and written to shared memory;
// whenever 32 coefficients are buffered, lane r sums coefficient r over the
// lanes (compensated) and stores the chunk's sum.
template <int P>
__global__ void __launch_bounds__(256) dual_m2l_kernel(DualArgs a) {
  constexpr int NL = WDual<P>::NL;
  constexpr int NM4 = ((P + 1) * (P + 2) * (P + 3) / 6 + 3) / 4;
  __shared__ float s_buf[8][32 * 33];  // rows of 33: no bank conflicts
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const DevTree& tr = a.tr;
  const int nchunk = min(*a.db.ctr, a.db.cap);
  const float scale = 1.f / 8388608.f;  // 2^-23
  float* buf = s_buf[wid];
  const int stride = (gridDim.x * blockDim.x) >> 5;
  // the next chunk's header and pair slots are loaded while this chunk is
  // formed (slots past the chunk's count are read but not used)
  int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int4 hd_n = make_int4(0, 0, 0, 0);
  int cell_n = 0, code_n = 0;
  if (c < nchunk) {
    hd_n = a.db.head[c];
    cell_n = a.db.cell[(int64_t)c * 32 + lane];
    code_n = a.db.img[(int64_t)c * 32 + lane];
  }
  for (; c < nchunk; c += stride) {
    const int4 hd = hd_n;
    const int g = hd.x, nml = hd.y;
    const float live = lane < nml ? 1.f : 0.f;
    // a slot past the count takes pair 0's cell (always valid), weight 0
    const int cell = __shfl_sync(0xffffffffu, cell_n, lane < nml ? lane : 0);
    const int code = __shfl_sync(0xffffffffu, code_n, lane < nml ? lane : 0);
    if (c + stride < nchunk) {
      hd_n = a.db.head[c + stride];
      cell_n = a.db.cell[(int64_t)(c + stride) * 32 + lane];
      code_n = a.db.img[(int64_t)(c + stride) * 32 + lane];
    }
    const int4 gb = tr.gB[NB_IDX(g, tr.cnt[1], 111)];
    const int box = tr.gA[NB_IDX(g, tr.cnt[1], 111)].z;
    const int kx = (code & 7) - 2, ky = ((code >> 3) & 7) - 2, kz = ((code >> 6) & 7) - 2;
    const int4 ca = tr.cA[NB_IDX(cell, tr.cnt[0], 110)];
    const int lvl = ca.w & 0xff;
    const float sc = (float)(1 << lvl);
    const float rx = ((float)(gb.x - (ca.x - kx * NB_PBOX)) * scale) * sc;
    const float ry = ((float)(gb.y - (ca.y - ky * NB_PBOX)) * scale) * sc;
    const float rz = ((float)(gb.z - (ca.z - kz * NB_PBOX)) * scale) * sc;
    const float e2 = a.k1 ? 0.f : a.eps2[box] * (sc * sc);
    float Mr[4 * NM4];
    {
      const float4* src = reinterpret_cast<const float4*>(a.mom32 + (int64_t)NB_IDX(cell, tr.cnt[0], 110) * kDualStride);
#pragma unroll
      for (int k = 0; k < NM4; k++) {
        const float4 v = src[k];
        Mr[4 * k] = v.x * live;
        Mr[4 * k + 1] = v.y * live;
        Mr[4 * k + 2] = v.z * live;
        Mr[4 * k + 3] = v.w * live;
      }
    }
    // 2^((level - lu)(o + 1)) takes coefficient order o to the group's unit
    float f[7];
    f[0] = __int_as_float((127 + lvl - a.lu) << 23);  // |level - lu| < 24
    f[1] = f[0] * f[0];
#pragma unroll
    for (int o = 2; o < 7; o++) f[o] = f[o - 1] * f[0];
    float* Lout = a.db.L + (int64_t)c * kDualLStride;
    auto flush = [&](int t0, int rows) {
      __syncwarp();
      if (lane < rows) {
        float sacc = 0.f, scmp = 0.f;
        for (int j = 0; j < 32; j++) kadd(sacc, scmp, buf[lane * 33 + j]);
        Lout[t0 + lane] = sacc - scmp;
      }
      __syncwarp();
    };
    struct RegMoments {
      const float* m;
      __device__ __forceinline__ float operator[](int u) const { return m[u]; }
    };
    WDual<P>::m2l(RegMoments{Mr}, rx, ry, rz, e2, [&](int t, int o, float v) {
      buf[(t & 31) * 33 + lane] = v * f[o];
      if ((t & 31) == 31 || t == NL - 1) flush(t & ~31, (t & 31) + 1);
    });
  }
}

// One warp per group with cell-group pairs: lane t sums coefficients t and
// t + 32 over the group's chunks in list order (compensated), then every
// sink evaluates the expansion at d = (x - z) 2^lu and adds u^2 times it to
// its acceleration (the coefficients were built from -d g, which the
// image-field L2P turns back: it subtracts).
template <int P>
__global__ void __launch_bounds__(256) dual_l2p_kernel(DualArgs a) {
  constexpr int NL = WDual<P>::NL;
  __shared__ float s_L[8][64];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const DevTree& tr = a.tr;
  const int ngroup = tr.cnt[1];
  const double scale = 1.0 / 8388608.0;
  const float u = (float)(1 << a.lu);
  for (int g = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; g < ngroup; g += (gridDim.x * blockDim.x) >> 5) {
    int c = a.db.first[g];
    if (c < 0) continue;
    float h0 = 0.f, c0 = 0.f, h1 = 0.f, c1 = 0.f;
    int guard = 0;
    while (c >= 0 && c < a.db.cap && guard++ < (1 << 24)) {
      const float* Lc = a.db.L + (int64_t)c * kDualLStride;
      kadd(h0, c0, Lc[lane]);
      if (lane + 32 < NL) kadd(h1, c1, Lc[lane + 32]);
      c = a.db.head[c].z;
    }
    s_L[wid][lane] = h0 - c0;
    s_L[wid][lane + 32] = h1 - c1;
    __syncwarp();
    const int4 ga = tr.gA[g], gb = tr.gB[g];
    if (lane < ga.y && NB_IN(ga.x + lane, tr.n, 112)) {
      const int64_t i = ga.x + lane;
      if (!tr.sact || tr.sact[i]) {
        const float dx = (float)((tr.spos[i] - gb.x * scale)) * u;
        const float dy = (float)((tr.spos[tr.n + i] - gb.y * scale)) * u;
        const float dz = (float)((tr.spos[2 * tr.n + i] - gb.z * scale)) * u;
        float bx = 0.f, by = 0.f, bz = 0.f;
        WDual<P>::l2p(s_L[wid], dx, dy, dz, bx, by, bz);
        a.acc[i] += bx * (u * u);
        a.acc[tr.n + i] += by * (u * u);
        a.acc[2 * tr.n + i] += bz * (u * u);
      }
    }
    __syncwarp();
  }
}

template <int P>
cudaError_t launch_dual(const DualArgs& a, int nsm, cudaStream_t s) {
  if constexpr (WDual<P>::has) {
    dual_m2l_kernel<P><<<nsm * 8, 256, 0, s>>>(a);
    int grid = (int)(((int64_t)a.tr.ngroup * 32 + 255) / 256);
    if (grid > nsm * 16) grid = nsm * 16;
    if (grid < 1) grid = 1;
    dual_l2p_kernel<P><<<grid, 256, 0, s>>>(a);
    nb_launch_counter += 2;
  }
  return cudaGetLastError();
}

template <typename T, int P, int WARPS, int MINB, bool PK, bool DUALK, bool POTK = false>
cudaError_t launch_walk(const WalkArgs<T>& a, int nsm, int max_blocks, cudaStream_t s) {
  // resident blocks per SM, queried once per variant (and so never while a
  // stream is being captured, after the first evaluation)
  static int occ = 0;
  if (occ == 0) {
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &occ, walk_kernel<T, P, WARPS, MINB, PK, DUALK, POTK>, WARPS * 32, 0);
    if (e) {
      occ = 0;
      return e;
    }
  }
  int grid = nsm * (occ > 0 ? occ : 1);
  if (grid > max_blocks) grid = max_blocks;
  walk_kernel<T, P, WARPS, MINB, PK, DUALK, POTK><<<grid, WARPS * 32, 0, s>>>(a);
  nb_launch_counter += 1;
  return cudaGetLastError();
}

// launch variants (warps per block, minimum resident blocks per SM, M2P
// form): 16 warps per SM in blocks of 8 or 4, so every variant has 128
// registers per thread (none spills); the same shapes with the dual form,
// whose walk only queues the cell-group pairs.
// The stack is sized for 8 warps per block.
template <typename T, int P>
cudaError_t launch_variant(int v, const WalkArgs<T>& a, int nsm, int max_blocks, cudaStream_t s) {
  // the potential: one scalar variant per precision (never with the dual form)
  if (a.pot) {
    if constexpr (sizeof(T) == 8) return launch_walk<T, P, 4, 1, false, false, true>(a, nsm, max_blocks, s);
    else return launch_walk<T, P, 8, 1, false, false, true>(a, nsm, max_blocks, s);
  }
  if constexpr (sizeof(T) == 8) {
    return launch_walk<T, P, 4, 1, false, false>(a, nsm, max_blocks, s);
  } else {
    if constexpr (WDual<P>::has) {
      if (a.dual) {
        // the cell-group pairs are only queued here: the same shapes as below
        switch (v) {
          case 0: return launch_walk<T, P, 8, 2, false, true>(a, nsm, max_blocks, s);
          case 1: return launch_walk<T, P, 4, 4, false, true>(a, nsm, max_blocks, s);
          case 2: return launch_walk<T, P, 8, 2, true, true>(a, nsm, max_blocks, s);
          default: return launch_walk<T, P, 4, 4, true, true>(a, nsm, max_blocks, s);
        }
      }
    }
    switch (v) {
      case 0: return launch_walk<T, P, 8, 2, false, false>(a, nsm, max_blocks, s);
      case 1: return launch_walk<T, P, 4, 4, false, false>(a, nsm, max_blocks, s);
      case 2: return launch_walk<T, P, 8, 2, true, false>(a, nsm, max_blocks, s);
      default: return launch_walk<T, P, 4, 4, true, false>(a, nsm, max_blocks, s);
    }
  }
}
constexpr int kVariants = 4;

// an empty pair list for every group before a walk of the dual form
template <typename T>
cudaError_t reset_dual(const WalkArgs<T>& a, cudaStream_t s) {
  if (!a.dual || !a.db.ctr) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(a.db.ctr, 0, sizeof(int), s);
  if (e) return e;
  return cudaMemsetAsync(a.db.first, 0xff, sizeof(int) * (size_t)a.tr.ngroup, s);
}

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
  // tuning key: 0 FP32, 1 FP64, 2 FP32 with the dual form
  const int fp = sizeof(T) == 8 ? 1 : (a.dual ? 2 : 0);
  if (forced >= 0 || a.pot) return launch_variant<T, P>(fp == 1 || forced < 0 ? 0 : forced, a, nsm, max_blocks, s);
  {
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    for (const auto& t : g_tune)
      if (t.device == dev && t.order == P && t.fp64 == fp) return launch_variant<T, P>(t.variant, a, nsm, max_blocks, s);
  }
  if (fp == 1) {
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
    if ((e = reset_dual(a, s))) return e;
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
  if ((e = reset_dual(a, s))) return e;
  return launch_variant<T, P>(bv, a, nsm, max_blocks, s);
}

// after a walk of the dual form: the cell-group expansions and their L2P
template <typename T, int P>
cudaError_t finish_dual(const WalkArgs<T>& a, const float* mom32, const void* eps2, int k1, int lu, int nsm,
                        cudaStream_t s) {
  if constexpr (std::is_same<T, float>::value) {
    if (a.dual && !a.pot) {
      DualArgs d{a.tr, a.db, mom32, (const float*)eps2, k1, lu, a.acc};
      return launch_dual<P>(d, nsm, s);
    }
  }
  return cudaSuccess;
}

}  // namespace

// warps per block of the walk for a precision (stack slots are sized for the largest)
int nb_walk_warps(bool fp64) { return fp64 ? 4 : 8; }

// the variant the autotuner chose for (precision, order) on this device, or
// -1; ms (nullable, kWalkVariantsMax entries) receives each variant's time
// in the tuning run (0 for variants not timed)
int nb_walk_variant(bool fp64, bool dual, int order, double* ms) {
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lock(g_tune_mutex);
  for (const auto& t : g_tune)
    if (t.device == dev && t.order == order && t.fp64 == (fp64 ? 1 : (dual ? 2 : 0))) {
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
                    int mac_edge, int bg, int k1, int dual, double theta, const float* mom32, int lu,
                    const NbDualBufs* db, void* pot, int repl, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(group_ctr, 0, sizeof(int), s);
  if (e) return e;
  if (dual && !pot && !db) return cudaErrorInvalidValue;
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
    a.k1 = k1;                                                                     \
    a.dual = dual;                                                                 \
    a.theta2 = theta * theta;                                                      \
    a.db = db ? *db : NbDualBufs{};                                                \
    a.repl = repl;                                                                 \
    a.le = le;                                                                     \
    a.stack = stack;                                                               \
    a.stack_cap = stack_cap;                                                       \
    a.group_ctr = group_ctr;                                                       \
    a.acc = (TT*)acc;                                                              \
    a.pot = (TT*)pot;                                                              \
    if (pot) a.dual = 0;                                                           \
    a.counters = counters;                                                         \
    a.status = status;                                                             \
    if ((e = reset_dual(a, s))) return e;                                          \
    if ((e = run_walk<TT, P>(a, nsm, max_blocks, forced_variant, s))) return e;    \
    return finish_dual<TT, P>(a, mom32, eps2, k1, lu, nsm, s);                     \
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

// fault word of the debug build's bounds checks in this unit (debug build only)
NB_DBG_EXPORT(walk)
