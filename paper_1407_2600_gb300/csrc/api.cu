// C ABI of the periodic treecode force path: tree handle, phase orchestration,
// kick-drift-kick step, inspection and error reporting.  The phases follow
// Sec. 2.1: keys and sort, key-implied tree with its hash, moments, grouped
// walk, periodic images; the integrator is the kick-drift-kick form of the
// symplectic integrator it cites.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "common.cuh"

// launchers from the other translation units
cudaError_t nb_gather(const double* pos, const float* mass, const uint32_t* perm, const uint16_t* box_of,
                      const int64_t* off, int64_t n, double* spos, float* smass, uint16_t* sbox, unsigned* status,
                      cudaStream_t s);
cudaError_t nb_count_cells(const uint64_t* skeys, const uint16_t* sbox, const int64_t* off, int64_t n, int n_leaf,
                           int lmax, int* ccount, int8_t* l0, cudaStream_t s);
cudaError_t nb_cap_check(int* cnt, int cell_cap, int group_cap, unsigned* err, cudaStream_t s);
cudaError_t nb_emit_cells(const uint64_t* skeys, const uint16_t* sbox, const int64_t* off, int64_t n, int n_leaf,
                          int lmax, const int* ccount, const int* coff, const int8_t* l0, const int* pncell,
                          uint8_t* plevel, int* pstart, int* pcount, int* pparent, cudaStream_t s);
cudaError_t nb_bfs_cells(const uint64_t* skeys, const uint16_t* sbox, int64_t n, int ncell, const int* pncell,
                         const uint32_t* bfs2pre, int* pre2bfs, const uint8_t* plevel, const int* pstart,
                         const int* pcount, const int* pparent, int4* cA, int4* cB, uint64_t* ckey, uint16_t* cbox,
                         cudaStream_t s);
cudaError_t nb_hash_build(int ncell, const int* pncell, const uint64_t* ckey, const uint16_t* cbox, int* hval,
                          uint64_t cap, unsigned* err, cudaStream_t s);
cudaError_t nb_hash_lookup(const uint64_t* q, int64_t nq, int box, const int* hval, const uint64_t* ckey,
                           const uint16_t* cbox, uint64_t cap, int* out, cudaStream_t s);
cudaError_t nb_leaves(int ncell, const int* pncell, const int4* cA, const int4* cB, const double* spos,
                      const float* smass, int64_t n, int* sleaf, void* src, bool fp64, cudaStream_t s);
cudaError_t nb_group_flags(const uint64_t* skeys, const uint16_t* sbox, const int64_t* off, int64_t n, int ls,
                           int n_group, int* flag, cudaStream_t s);
cudaError_t nb_group_runs(int ngroup, const int* pngroup, int4* gA, int4* gD, int* flag, int* excl, int* total,
                          int* tmp, int* runhead, cudaStream_t s);
cudaError_t nb_group_info(const uint64_t* skeys, const uint16_t* sbox, int64_t n, int ngroup, const int* pngroup,
                          int ls, const int* flag, const int* gid, int* gstart, const double* spos, int4* gA,
                          int4* gB, int4* gC, int4* gD, cudaStream_t s);
int nb_walk_variant(bool fp64, bool dual, int order, double* ms);
int nb_coef_stride(int order);
cudaError_t nb_upward(int order, bool fp64, int ncell, const int* pncell, const int4* cA, const int4* cB,
                      const double* spos, const float* smass, int64_t n, double* mom, void* coef, uint8_t* ukey,
                      uint32_t* uorder, uint32_t* uhist, int* urange, const uint16_t* cbox, const double* rho,
                      float* mom32, SortScratch* sc, cudaStream_t s);
cudaError_t nb_box_mass(const int64_t* off, const float* smass, int nbox, double* rho, double* part,
                        cudaStream_t s);
cudaError_t nb_field_moments(int pe, int le, int nbox, const int64_t* off, const uint64_t* skeys,
                             const double* spos, const float* smass, int64_t n, const int* hval,
                             const uint64_t* ckey, const uint16_t* cbox, uint64_t hcap, const double* mom,
                             int order, double* fm, float* fm32, cudaStream_t s);
int nb_walk_warps(bool fp64);
cudaError_t nb_walk(const DevTree& tr, bool fp64, int order, const void* coef, const void* src, const void* eps2,
                    const long long* thr, int n_direct, int le, int* stack, int stack_cap, int max_blocks,
                    int* group_ctr, void* acc, unsigned long long* counters, unsigned* status, int nsm,
                    int forced_variant, int mac_edge, int bg, int k1, int dual, double theta, const float* mom32, int lu,
                    const NbDualBufs* db, void* pot, int repl, cudaStream_t s);
cudaError_t nb_phitilde_table(int lg, int P, const double** t64, const float** t32, cudaStream_t s);
int nb_field_stride(int pe);
struct AdjBuffers {
  float* lam_s;
  double* mu;
  float* nuc;
  double* nu;
  double* lbar;
  double* nue;
  int* group_ctr;
};
int nb_adj_coef_nm(int order);
int nb_adj_lbar_stride(int pe);
cudaError_t nb_forces_vjp(const DevTree& tr, bool fp64, int order, int pe, int le, int lg, const void* coef,
                          const void* src, const void* eps2, const long long* thr, int n_direct, int* stack,
                          int stack_cap, int max_blocks, const double* fm, const void* tab, const void* lbuf,
                          int lstride, int max_level, const float* lam, double* out, const AdjBuffers& B,
                          unsigned* status, int nsm, int mac_edge, int bg, cudaStream_t s);
cudaError_t nb_field_local(const DevTree& tr, bool fp64, int pe, int le, int lg, const void* src, const double* fm, const float* fm32,
                           const void* tab, void* lbuf, cudaStream_t s);
cudaError_t nb_lattice(const DevTree& tr, bool fp64, int W, const void* accw, float* out, double* out64,
                       const void* potw, float* pout, double* part, double* mom, double* Ld, void* Lt,
                       cudaStream_t s);
cudaError_t nb_periodic(const DevTree& tr, bool fp64, int pe, int le, int lg, const void* src, const double* fm, const float* fm32,
                        const void* tab, void* lbuf, const void* accw, float* out, unsigned long long* counter,
                        double* out64, const void* potw, float* pout, cudaStream_t s);

namespace {

constexpr int kStackCap = 8192;  // cells per warp stack
constexpr int kRing = 64;        // timed builds / evaluations kept

struct Buf {
  void* p = nullptr;
  size_t cap = 0;
  cudaError_t ensure(size_t bytes) {
    if (bytes <= cap && p) return cudaSuccess;
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
    size_t want = bytes + bytes / 4 + 256;
    cudaError_t e = cudaMalloc(&p, want);
    if (e) {
      cudaGetLastError();
      return e;
    }
    cap = want;
    return cudaSuccess;
  }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
  }
  template <typename T> T* as() const { return (T*)p; }
};

}  // namespace

struct nbody_tree {
  nbody_params prm;
  int nbox = 0;
  int64_t n = 0;
  std::vector<int64_t> h_off;
  std::vector<double> h_eps;  // per box, in box units (the caller's eps / L)
  std::vector<double> h_len;  // per box side length L in the caller's units
  bool scaled = false;        // some L != 1: the tree works on pos / L (upos)
  Buf upos, lscale;           // scaled positions; per box 1/L, 1/L^2, 1/L^3 (FP64)
  const double* pos = nullptr;
  const float* mass = nullptr;
  int device = 0, nsm = 0;
  // particles
  Buf off, box_of, keys, vals, keys2, vals2, sbox, spos, smass, src, sleaf;
  // sort scratch
  Buf hist, sstatus, tilectr, status;
  // build scratch
  Buf ccount, coff, l0, plevel, pstart, pcount, pparent, bfs2pre, pre2bfs, lvlhist, scantmp, totals;
  // Cells and groups.  ncell / ngroup are the counts of the last build as the
  // host knows them; cell_cap / group_cap size the buffers and launch grids.
  // Without a reservation every build reads its counts back and the
  // capacities equal them; with one (fixed_cap) builds never read back, the
  // kernels take the counts from totals[0..1] on the device, and a count
  // above its capacity sets the overflow status instead.
  bool fixed_cap = false;
  int cell_cap = 0, group_cap = 0;
  int ncell = 0, max_level = 0;
  Buf cA, cB, ckey, cbox, hval, mom, uorder, coef, ukey, urng;
  Buf mom32;  // FP32 cell-unit moments for the dual form
  uint64_t hcap = 0;
  // groups
  int ngroup = 0;
  Buf gflag, gid, gstart, gA, gB, gC, gD, runhead;
  // image field
  Buf fm;
  Buf rho;  // mean density per box (background terms)
  // block steps: active sinks (sorted order), active groups, per-box rung factors
  Buf act_s, act_g, rungc;
  const double* tab64 = nullptr;
  const float* tab32 = nullptr;
  // walk
  Buf eps2, stack, gctr, accw, counters, lbuf;
  Buf potw;  // the walk's potential (key order), when one is asked for
  // the dual form's cell-group pair chunks (lc_cap chunks of 32 pairs)
  Buf lc_cell, lc_img, lc_head, lc_first, lc_ctr, lc_L;
  // the near-replica scheme's far lattice: moment slices, box moments, local expansions
  Buf lat_part, lat_mom, lat_Ld, lat_Lt;
  int64_t lc_cap = 0;
  bool lc_grew = false;  // the last status read grew the pool
  // reverse mode
  Buf a_lam, a_mu, a_nuc, a_nu, a_lbar, a_nue, a_x0, a_x1, a_ph, a_g, a_lg, a_lx, a_lp, a_out;
  // the KDK adjoint's kept product J(x0)^T lam_ph with its x0 and lam_p0
  Buf a_xc, a_lc, a_muc, a_eq;
  bool adj_cache = false;
  long long adj_steps = 0, adj_reused = 0;
  bool forces_valid = false;  // walk + image field of the last build evaluated
  bool field_valid = false;   // image-field local expansions of the last build formed
  nbody_tree* aux = nullptr;  // second tree of the KDK adjoint (state at the step's end)
  int walk_blocks = 0;
  long long thr[NB_NLEV];
  int64_t* pinned = nullptr;
  // timing ring: builds (sort start, sort end, build end, moments end) and
  // evaluations (walk start, walk end, periodic end)
  cudaEvent_t bev[kRing][4];
  cudaEvent_t fev[kRing][3];
  bool events = false;
  int64_t nb_log = 0, nf_log = 0;
  long long launches = 0;
  Buf tot;  // accumulated p2p, m2p, m2l counters
  cudaStream_t last_stream = nullptr;

  ~nbody_tree() {
    Buf* all[] = {&off, &box_of, &keys, &vals, &keys2, &vals2, &sbox, &spos, &smass, &src, &sleaf,
                  &hist, &sstatus, &tilectr, &status, &ccount, &coff, &l0, &plevel, &pstart, &pcount,
                  &pparent, &bfs2pre, &pre2bfs, &lvlhist, &scantmp, &totals, &cA, &cB, &ckey, &cbox,
                  &hval, &mom, &uorder, &coef, &ukey, &urng, &gflag, &gid, &gstart, &gA, &gB, &gC, &gD, &runhead, &fm,
                  &eps2, &stack, &gctr, &accw, &counters, &tot, &lbuf, &rho, &act_s, &act_g, &rungc,
                  &a_lam, &a_mu, &a_nuc, &a_nu, &a_lbar, &a_nue, &a_x0, &a_x1, &a_ph, &a_g, &a_lg,
                  &a_lx, &a_lp, &a_out, &a_xc, &a_lc, &a_muc, &a_eq, &upos, &lscale, &mom32, &potw,
                  &lc_cell, &lc_img, &lc_head, &lc_first, &lc_ctr, &lc_L, &lat_part, &lat_mom, &lat_Ld,
                  &lat_Lt};
    for (Buf* b : all) b->release();
    if (pinned) cudaFreeHost(pinned);
    delete aux;
    if (events)
      for (int r = 0; r < kRing; r++) {
        for (auto& e : bev[r]) cudaEventDestroy(e);
        for (auto& e : fev[r]) cudaEventDestroy(e);
      }
  }

  DevTree dev() const {
    DevTree t;
    t.n = n;
    t.nbox = nbox;
    t.off = off.as<int64_t>();
    t.skeys = keys.as<uint64_t>();
    t.perm = vals.as<uint32_t>();
    t.sbox = sbox.as<uint16_t>();
    t.spos = spos.as<double>();
    t.smass = smass.as<float>();
    t.cnt = totals.as<int>();
    t.ncell = cell_cap;
    t.cA = cA.as<int4>();
    t.cB = cB.as<int4>();
    t.ngroup = group_cap;
    t.gA = gA.as<int4>();
    t.gB = gB.as<int4>();
    t.gC = gC.as<int4>();
    t.gD = gD.as<int4>();
    t.runhead = runhead.as<int>();
    t.sleaf = sleaf.as<int>();
    t.sact = nullptr;
    t.gact = nullptr;
    return t;
  }
};

namespace {

#define NB_CU(x)                                 \
  do {                                           \
    cudaError_t _e = (x);                        \
    if (_e != cudaSuccess) return map_err(_e);   \
  } while (0)

int map_err(cudaError_t e) {
  if (e == cudaErrorMemoryAllocation) return NBODY_ENOMEM;
  return NBODY_ECUDA;
}

int status_to_code(unsigned st) {
  if (st & NB_ST_OVERFLOW) return NBODY_EOVERFLOW;
  if (st & NB_ST_TIMEOUT) return NBODY_ETIMEOUT;
  if (st & NB_ST_BADINPUT) return NBODY_EINVAL;
  return NBODY_OK;
}

int validate(const nbody_params* p) {
  if (!p) return NBODY_EINVAL;
  if (!(p->theta > 0.0) || !(p->eps > 0.0)) return NBODY_EINVAL;
  if (p->order < 0 || p->order > 4) return NBODY_EINVAL;
  if (p->n_leaf < 1 || p->n_leaf > 64) return NBODY_EINVAL;
  if (p->n_group < 1 || p->n_group > 32) return NBODY_EINVAL;
  if (p->n_direct < 0 || p->n_direct > p->n_leaf) return NBODY_EINVAL;
  if (p->lmax < 2 || p->lmax > NB_QBITS) return NBODY_EINVAL;
  if (p->ewald_order < 0 || p->ewald_order > 5) return NBODY_EINVAL;
  if (p->ewald_order > 0) {
    if (p->ewald_level < 1 || p->ewald_level > 4) return NBODY_EINVAL;
    if (p->ewald_grid < p->ewald_level + 1 || p->ewald_grid > 8) return NBODY_EINVAL;
  }
  if (p->precision != NBODY_MIXED && p->precision != NBODY_FP64) return NBODY_EINVAL;
  if (((p->flags >> 8) & 0xf) > 4) return NBODY_EINVAL;  // walk variant override 0..3
  if (p->flags &
      ~(NBODY_FLAG_ASYNC | NBODY_FLAG_MAC_EDGE | NBODY_FLAG_BACKGROUND | NBODY_FLAG_K1 | NBODY_FLAG_DUAL |
        NBODY_FLAG_REPLICAS | (0xf << 8)))
    return NBODY_EINVAL;  // unknown flag bits
  if (p->flags & NBODY_FLAG_REPLICAS) {
    // the near replicas replace the image field; ewald_grid still places the groups
    if (p->ewald_order != 0 || p->ewald_grid < 2 || p->ewald_grid > 8) return NBODY_EINVAL;
  }
  if ((p->flags & NBODY_FLAG_DUAL) &&
      (p->order < 1 || p->precision != NBODY_MIXED || (p->flags & NBODY_FLAG_BACKGROUND)))
    return NBODY_ENOTSUP;
  if ((p->flags & NBODY_FLAG_BACKGROUND) && (p->order == 1 || p->order == 3)) return NBODY_EINVAL;
  if (!(p->box_len >= 0.0) || p->box_len > 1e300) return NBODY_EINVAL;  // 0 = unit box
  return NBODY_OK;
}

// image level used by the walk even without periodic images
int image_level(const nbody_params& p) { return p.ewald_order > 0 ? p.ewald_level : 3; }

// the FP32 copy of the image field's source moments, stored after the FP64 ones
float* fm32_of(const nbody_tree* t) {
  const nbody_params& p = t->prm;
  const int ne = (p.ewald_order + 1) * (p.ewald_order + 2) * (p.ewald_order + 3) / 6;
  return (float*)(t->fm.as<double>() + (int64_t)t->nbox * (1 << (3 * p.ewald_level)) * ne);
}
int group_level(const nbody_params& p) {
  return (p.ewald_order > 0 || (p.flags & NBODY_FLAG_REPLICAS)) ? p.ewald_grid - 1 : 5;
}

__global__ void kick_kernel(int64_t n3, float* __restrict__ mom, const float* __restrict__ acc, float k) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n3; i += (int64_t)gridDim.x * blockDim.x)
    mom[i] = fmaf(k, acc[i], mom[i]);
}

__global__ void drift_kernel(int64_t n3, double* __restrict__ pos, const float* __restrict__ mom, double d) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n3; i += (int64_t)gridDim.x * blockDim.x) {
    double x = pos[i] + d * (double)mom[i];
    x -= floor(x);
    if (x >= 1.0) x = 0.0;
    pos[i] = x;
  }
}

__global__ void copy_u64_kernel(const uint64_t* __restrict__ a, uint64_t* __restrict__ b, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = a[i];
}

__global__ void export_cells_kernel(int ncell, const int4* __restrict__ cA, const int4* __restrict__ cB, int what,
                                    int* __restrict__ out) {
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < ncell; b += gridDim.x * blockDim.x) {
    if (what == NBODY_EXPORT_CELL_RANGE) {
      out[2 * b] = cB[b].x;
      out[2 * b + 1] = cB[b].y;
    } else {
      out[b] = cA[b].w & 0xff;
    }
  }
}

__global__ void export_groups_kernel(int ng, const int4* __restrict__ gA, int* __restrict__ out) {
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < ng; g += gridDim.x * blockDim.x) {
    out[2 * g] = gA[g].x;
    out[2 * g + 1] = gA[g].y;
  }
}

__global__ void eps2_kernel(int nbox, const double* __restrict__ eps, float* __restrict__ e32,
                            double* __restrict__ e64) {
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nbox; b += gridDim.x * blockDim.x) {
    e32[b] = (float)(eps[b] * eps[b]);
    e64[b] = eps[b] * eps[b];
  }
}

// out[d n + i] = in[d n + i] * f[b] for every particle i of box b (offsets
// off) and d < nc: positions to box units (f = 1/L) and accelerations,
// potentials or force VJPs back to the caller's length unit (f = 1/L^2, 1/L,
// 1/L^3)
template <typename T>
__global__ void box_scale_kernel(const int64_t* __restrict__ off, int nbox, int64_t n,
                                 const double* __restrict__ f, const T* in, T* out, int nc) {
  for (int b = blockIdx.y; b < nbox; b += gridDim.y) {
    const int64_t lo = off[b], hi = off[b + 1];
    const double fb = f[b];
    for (int64_t i = lo + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < hi;
         i += (int64_t)gridDim.x * blockDim.x)
      for (int d = 0; d < nc; d++) out[d * n + i] = (T)(in[d * n + i] * fb);
  }
}

// elementwise pieces of the KDK adjoint
__global__ void drift_from_kernel(int64_t n3, const double* __restrict__ x0, const float* __restrict__ p, double d,
                                  double* __restrict__ x1) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n3; i += (int64_t)gridDim.x * blockDim.x) {
    double x = x0[i] + d * (double)p[i];
    x -= floor(x);
    if (x >= 1.0) x = 0.0;
    x1[i] = x;
  }
}

// lam_x1' = lam_x1 + k2 mu1;  lam_ph = lam_p1 + d lam_x1' (FP64 and its FP32 rounding)
__global__ void adj_mid_kernel(int64_t n3, const double* __restrict__ lx1, const double* __restrict__ mu1,
                               const float* __restrict__ lp1, double k2, double d, double* __restrict__ lx,
                               double* __restrict__ lp, float* __restrict__ lp32) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n3; i += (int64_t)gridDim.x * blockDim.x) {
    const double x = lx1[i] + k2 * mu1[i];
    const double p = (double)lp1[i] + d * x;
    lx[i] = x;
    lp[i] = p;
    lp32[i] = (float)p;
  }
}

// lam_x0 = lam_x1' + k1 mu0;  lam_p0 = lam_ph
__global__ void adj_fin_kernel(int64_t n3, const double* __restrict__ lx, const double* __restrict__ mu0, double k1,
                               const float* __restrict__ lp32, double* __restrict__ lx0, float* __restrict__ lp0) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n3; i += (int64_t)gridDim.x * blockDim.x) {
    lx0[i] = lx[i] + k1 * mu0[i];
    lp0[i] = lp32[i];
  }
}

// *flag = 1 unless a == b and c == d bit for bit (n3 doubles, n3 floats)
__global__ void differ_kernel(int64_t n3, const unsigned long long* __restrict__ a,
                              const unsigned long long* __restrict__ b, const unsigned* __restrict__ c,
                              const unsigned* __restrict__ d, int* flag) {
  bool diff = false;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n3; i += (int64_t)gridDim.x * blockDim.x)
    diff |= (a[i] != b[i]) | (c[i] != d[i]);
  if (__any_sync(0xffffffffu, diff) && (threadIdx.x & 31) == 0) atomicOr(flag, 1);
}

__global__ void accumulate_kernel(const unsigned long long* __restrict__ c, unsigned long long* __restrict__ tot) {
  if (threadIdx.x < 5) tot[threadIdx.x] += c[threadIdx.x];
}

// ---- block steps ------------------------------------------------------------------
// rung of each particle (caller order): the smallest r in [0, rmax] with
// 4^r >= q = |g| c_box, c_box = dlna^2 / (eta^2 H0^2 eps_box); |g| and q in
// FP64, rounded at every operation (no contraction), from the FP32 g
__global__ void rung_kernel(int64_t n, const float* __restrict__ acc, const uint16_t* __restrict__ box_of,
                            const double* __restrict__ cbox, int rmax, int8_t* __restrict__ rung) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double gx = acc[i], gy = acc[n + i], gz = acc[2 * n + i];
    const double g2 = __dadd_rn(__dadd_rn(__dmul_rn(gx, gx), __dmul_rn(gy, gy)), __dmul_rn(gz, gz));
    const double q = __dmul_rn(__dsqrt_rn(g2), cbox[box_of[i]]);
    int r = 0;
    double f = 1.0;
    while (r < rmax && f < q) {
      r++;
      f *= 4.0;
    }
    rung[i] = (int8_t)r;
  }
}

// active sinks in key order: rung[perm[i]] >= rmin
__global__ void active_kernel(int64_t n, const uint32_t* __restrict__ perm, const int8_t* __restrict__ rung, int rmin,
                              uint8_t* __restrict__ sact) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    sact[i] = rung[perm[i]] >= rmin ? 1 : 0;
}

// a group is evaluated when any of its sinks is active
__global__ void group_active_kernel(const int* __restrict__ pngroup, const int4* __restrict__ gA,
                                    const uint8_t* __restrict__ sact, uint8_t* __restrict__ gact) {
  const int ngroup = *pngroup;
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < ngroup; g += gridDim.x * blockDim.x) {
    const int4 a = gA[g];
    uint8_t any = 0;
    for (int k = 0; k < a.y; k++) any |= sact[a.x + k];
    gact[g] = any;
  }
}

// kicks of the particles whose rung has a factor in this call (f[r] != 0)
struct RungKicks {
  float f[8];
};
__global__ void kick_rungs_kernel(int64_t n, float* __restrict__ mom, const float* __restrict__ acc,
                                  const int8_t* __restrict__ rung, RungKicks k) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float f = k.f[rung[i] & 7];
    if (f != 0.f)
      for (int d = 0; d < 3; d++) mom[d * n + i] = fmaf(f, acc[d * n + i], mom[d * n + i]);
  }
}

__global__ void max_level_kernel(int ncell, const int4* __restrict__ cA, int* out) {
  int m = 0;
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < ncell; b += gridDim.x * blockDim.x)
    m = max(m, cA[b].w & 0xff);
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, m);
}

int gridn(int64_t n, int threads) {
  int64_t g = (n + threads - 1) / threads;
  if (g < 1) g = 1;
  if (g > 152 * 32) g = 152 * 32;
  return (int)g;
}

// After an overflow: if the dual form's last walk asked for more pair chunks
// than its pool holds, size the pool for that many (and a quarter more) so
// that the next evaluation fits; true when it grew.
bool dual_regrow(nbody_tree* t, cudaStream_t s) {
  if (!(t->prm.flags & NBODY_FLAG_DUAL) || !t->lc_ctr.p) return false;
  int need = 0;
  if (cudaMemcpyAsync(&need, t->lc_ctr.p, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if ((int64_t)need <= t->lc_cap) return false;
  t->lc_cap = (int64_t)need + need / 4 + 1024;
  return true;
}

// the status word of the calls since the last read (and on an overflow the
// dual form's pair pool sized for the next evaluation)
int read_status(nbody_tree* t, cudaStream_t s) {
  unsigned st = 0;
  NB_CU(cudaMemcpyAsync(&st, t->status.p, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
  NB_CU(cudaStreamSynchronize(s));
  NB_CU(cudaMemsetAsync(t->status.p, 0, sizeof(unsigned), s));
  const int rc = status_to_code(st);
  t->lc_grew = rc == NBODY_EOVERFLOW && dual_regrow(t, s);
  return rc;
}



bool capturing(cudaStream_t s) {
  cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &st) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return st != cudaStreamCaptureStatusNone;
}

// box offsets and per-box squared softening on the device; once per set-up
int upload_boxes(nbody_tree* t, cudaStream_t s) {
  NB_CU(t->off.ensure(8 * (t->nbox + 1)));
  NB_CU(cudaMemcpyAsync(t->off.p, t->h_off.data(), 8 * (t->nbox + 1), cudaMemcpyHostToDevice, s));
  NB_CU(t->eps2.ensure(12 * t->nbox + 64));
  Buf tmp;
  NB_CU(tmp.ensure(8 * t->nbox));
  NB_CU(cudaMemcpyAsync(tmp.p, t->h_eps.data(), 8 * t->nbox, cudaMemcpyHostToDevice, s));
  float* e32 = t->eps2.as<float>();
  double* e64 = (double*)((char*)t->eps2.p + ((4 * t->nbox + 15) & ~15));
  eps2_kernel<<<gridn(t->nbox, 128), 128, 0, s>>>(t->nbox, tmp.as<double>(), e32, e64);
  NB_CU(cudaGetLastError());
  if (t->scaled) {
    std::vector<double> f(3 * t->nbox);
    for (int b = 0; b < t->nbox; b++) {
      const double il = 1.0 / t->h_len[b];
      f[b] = il;
      f[t->nbox + b] = il * il;
      f[2 * t->nbox + b] = il * il * il;
    }
    NB_CU(t->lscale.ensure(8 * f.size()));
    NB_CU(cudaMemcpyAsync(t->lscale.p, f.data(), 8 * f.size(), cudaMemcpyHostToDevice, s));
  }
  NB_CU(cudaStreamSynchronize(s));
  tmp.release();
  return NBODY_OK;
}

// arrays of the caller's (3, n) layout scaled per box by lscale[k * nbox + b]
// (k = 0: 1/L, 1: 1/L^2, 2: 1/L^3); a no-op for unit boxes
template <typename T>
int scale_boxes(const nbody_tree* t, int k, const T* in, T* out, cudaStream_t s, int nc = 3) {
  if (!t->scaled) return NBODY_OK;
  const int64_t per = (t->n + t->nbox - 1) / t->nbox;
  dim3 g((unsigned)std::min<int64_t>((per + 255) / 256, 1024), (unsigned)std::min(t->nbox, 65535));
  box_scale_kernel<T><<<g, 256, 0, s>>>(t->off.as<int64_t>(), t->nbox, t->n, t->lscale.as<double>() + k * t->nbox,
                                        in, out, nc);
  nb_launch_counter += 1;
  NB_CU(cudaGetLastError());
  return NBODY_OK;
}

// buffers of cells and groups for the given capacities
int size_cells(nbody_tree* t, int cell_cap, int group_cap) {
  const nbody_params& p = t->prm;
  const bool fp64 = p.precision == NBODY_FP64;
  const int cs = nb_coef_stride(p.order);
  const int nm = (p.order + 1) * (p.order + 2) * (p.order + 3) / 6;
  const int64_t nc = cell_cap, ng = group_cap;
  NB_CU(t->plevel.ensure(nc));
  NB_CU(t->pstart.ensure(4 * nc));
  NB_CU(t->pcount.ensure(4 * nc));
  NB_CU(t->pparent.ensure(4 * nc));
  NB_CU(t->bfs2pre.ensure(4 * nc));
  NB_CU(t->pre2bfs.ensure(4 * nc));
  NB_CU(t->cA.ensure(16 * nc));
  NB_CU(t->cB.ensure(16 * nc));
  NB_CU(t->ckey.ensure(8 * nc));
  NB_CU(t->cbox.ensure(2 * nc));
  NB_CU(t->mom.ensure(8 * nc * nm));
  NB_CU(t->uorder.ensure(4 * nc));
  NB_CU(t->coef.ensure((fp64 ? 8 : 4) * nc * cs));
  if (p.flags & NBODY_FLAG_DUAL) NB_CU(t->mom32.ensure(4 * nc * kDualStride));
  NB_CU(t->ukey.ensure(nc));
  NB_CU(t->urng.ensure(4 * (256 + 32)));
  uint64_t hc = 1;
  while (hc < 2 * (uint64_t)nc) hc <<= 1;
  t->hcap = hc;
  NB_CU(t->hval.ensure(4 * hc));
  NB_CU(t->gstart.ensure(4 * ng));
  NB_CU(t->gA.ensure(16 * ng));
  NB_CU(t->gB.ensure(16 * ng));
  NB_CU(t->gC.ensure(16 * ng));
  NB_CU(t->gD.ensure(16 * ng));
  NB_CU(t->runhead.ensure(4 * ng));
  // scratch of the sorts: the key sort's passes and the one-pass cell sorts
  const int64_t tiles = nb_sort_tiles(t->n) + 1, ctiles = nb_sort_tiles(nc) + 1;
  NB_CU(t->sstatus.ensure(4 * 256 * (tiles * 12 > ctiles ? tiles * 12 : ctiles)));
  t->cell_cap = cell_cap;
  t->group_cap = group_cap;
  return NBODY_OK;
}

// counts of the last build as the host sees them (a read back when builds
// run on reserved capacities and so do not make one)
int host_counts(const nbody_tree* t, int* nc, int* ng) {
  if (!t->fixed_cap) {
    *nc = t->ncell;
    *ng = t->ngroup;
    return NBODY_OK;
  }
  int c[2] = {0, 0};
  if (t->last_stream) NB_CU(cudaStreamSynchronize(t->last_stream));
  NB_CU(cudaMemcpy(c, t->totals.p, sizeof(c), cudaMemcpyDeviceToHost));
  *nc = c[0];
  *ng = c[1];
  return NBODY_OK;
}

int build_impl(nbody_tree* t, cudaStream_t s) {
  const nbody_params& p = t->prm;
  const int64_t n = t->n;
  const bool fp64 = p.precision == NBODY_FP64;
  // per-particle buffers
  NB_CU(t->keys.ensure(8 * n));
  NB_CU(t->vals.ensure(4 * n));
  NB_CU(t->keys2.ensure(8 * n));
  NB_CU(t->vals2.ensure(4 * n));
  NB_CU(t->box_of.ensure(2 * n));
  NB_CU(t->sbox.ensure(2 * n));
  NB_CU(t->spos.ensure(24 * n));
  NB_CU(t->smass.ensure(4 * n));
  NB_CU(t->src.ensure((fp64 ? 32 : 16) * n));
  NB_CU(t->sleaf.ensure(4 * n));
  NB_CU(t->ccount.ensure(4 * n));
  NB_CU(t->coff.ensure(4 * n));
  NB_CU(t->l0.ensure(n));
  NB_CU(t->gflag.ensure(4 * n));
  NB_CU(t->gid.ensure(4 * n));
  NB_CU(t->scantmp.ensure(4 * (nb_scan_tmp_ints(n) + 16)));
  NB_CU(t->totals.ensure(64));
  NB_CU(t->hist.ensure(4 * 256 * 16));
  NB_CU(t->tilectr.ensure(4 * 16));
  NB_CU(t->lvlhist.ensure(4 * 256));
  if (!t->fixed_cap) NB_CU(t->sstatus.ensure(4 * 256 * (nb_sort_tiles(n) + 1) * 12));
  // the keys start in whichever buffer makes the sort's last pass land in
  // keys / vals, so every build (and a captured one) leaves them in place
  const int np = nb_radix_passes(63, t->nbox);
  Buf& kin = (np & 1) ? t->keys2 : t->keys;
  Buf& vin = (np & 1) ? t->vals2 : t->vals;
  SortScratch sc;
  sc.keys_alt = ((np & 1) ? t->keys : t->keys2).as<uint64_t>();
  sc.vals_alt = ((np & 1) ? t->vals : t->vals2).as<uint32_t>();
  sc.hist = t->hist.as<uint32_t>();
  sc.status = t->sstatus.as<uint32_t>();
  sc.tile_ctr = t->tilectr.as<uint32_t>();
  sc.tiles_cap = (int64_t)(t->sstatus.cap / (4 * 256));
  sc.dstatus = t->status.as<unsigned>();

  const bool timed = !capturing(s);
  cudaEvent_t* be = t->bev[t->nb_log % kRing];
  t->last_stream = s;
  if (timed) NB_CU(cudaEventRecord(be[0], s));
  // A1 keys, A2 sort, A3 gather
  NB_CU(nb_launch_box_ids(t->off.as<int64_t>(), t->nbox, n, t->box_of.as<uint16_t>(), s));
  NB_CU(nb_launch_keys(t->pos, n, 0, kin.as<uint64_t>(), vin.as<uint32_t>(), s));
  int alt = 0;
  NB_CU(nb_radix_sort(kin.as<uint64_t>(), vin.as<uint32_t>(), n, 63, t->box_of.as<uint16_t>(), t->nbox, &sc, s,
                      &alt));
  if (alt != (np & 1)) return NBODY_ECUDA;
  NB_CU(nb_gather(t->pos, t->mass, t->vals.as<uint32_t>(), t->box_of.as<uint16_t>(), t->off.as<int64_t>(), n,
                  t->spos.as<double>(), t->smass.as<float>(), t->sbox.as<uint16_t>(), t->status.as<unsigned>(), s));
  if (timed) NB_CU(cudaEventRecord(be[1], s));
  // A4 tree: cells per particle, scan, groups flags + scan, counts
  NB_CU(nb_count_cells(t->keys.as<uint64_t>(), t->sbox.as<uint16_t>(), t->off.as<int64_t>(), n, p.n_leaf, p.lmax,
                       t->ccount.as<int>(), t->l0.as<int8_t>(), s));
  int* totals = t->totals.as<int>();
  NB_CU(nb_exclusive_scan_i32(t->ccount.as<int>(), t->coff.as<int>(), n, totals, t->scantmp.as<int>(), s));
  const int ls = group_level(p);
  NB_CU(nb_group_flags(t->keys.as<uint64_t>(), t->sbox.as<uint16_t>(), t->off.as<int64_t>(), n, ls, p.n_group,
                       t->gflag.as<int>(), s));
  NB_CU(nb_exclusive_scan_i32(t->gflag.as<int>(), t->gid.as<int>(), n, totals + 1, t->scantmp.as<int>(), s));
  if (!t->fixed_cap) {
    NB_CU(cudaMemcpyAsync(t->pinned, totals, 8, cudaMemcpyDeviceToHost, s));
    NB_CU(cudaStreamSynchronize(s));
    const int ncell = (int)((int*)t->pinned)[0];
    const int ngroup = (int)((int*)t->pinned)[1];
    if (ncell <= 0 || ngroup <= 0) return NBODY_EINVAL;
    t->ncell = ncell;
    t->ngroup = ngroup;
    int rc = size_cells(t, ncell, ngroup);
    if (rc) return rc;
    sc.status = t->sstatus.as<uint32_t>();
    sc.tiles_cap = (int64_t)(t->sstatus.cap / (4 * 256));
  } else {
    NB_CU(nb_cap_check(totals, t->cell_cap, t->group_cap, t->status.as<unsigned>(), s));
    // slots past the cell count take the largest level code and sort last
    NB_CU(cudaMemsetAsync(t->plevel.p, 0xff, (size_t)t->cell_cap, s));
  }
  const int nc = t->cell_cap, ng = t->group_cap;
  NB_CU(nb_emit_cells(t->keys.as<uint64_t>(), t->sbox.as<uint16_t>(), t->off.as<int64_t>(), n, p.n_leaf, p.lmax,
                      t->ccount.as<int>(), t->coff.as<int>(), t->l0.as<int8_t>(), totals, t->plevel.as<uint8_t>(),
                      t->pstart.as<int>(), t->pcount.as<int>(), t->pparent.as<int>(), s));
  NB_CU(nb_sort_digit8(t->plevel.as<uint8_t>(), nc, t->bfs2pre.as<uint32_t>(), t->lvlhist.as<uint32_t>(), &sc, s));
  NB_CU(nb_bfs_cells(t->keys.as<uint64_t>(), t->sbox.as<uint16_t>(), n, nc, totals, t->bfs2pre.as<uint32_t>(),
                     t->pre2bfs.as<int>(), t->plevel.as<uint8_t>(), t->pstart.as<int>(), t->pcount.as<int>(),
                     t->pparent.as<int>(), t->cA.as<int4>(), t->cB.as<int4>(), t->ckey.as<uint64_t>(),
                     t->cbox.as<uint16_t>(), s));
  NB_CU(nb_hash_build(nc, totals, t->ckey.as<uint64_t>(), t->cbox.as<uint16_t>(), t->hval.as<int>(), t->hcap,
                      t->status.as<unsigned>(), s));
  NB_CU(nb_leaves(nc, totals, t->cA.as<int4>(), t->cB.as<int4>(), t->spos.as<double>(), t->smass.as<float>(), n,
                  t->sleaf.as<int>(), t->src.p, fp64, s));
  NB_CU(nb_group_info(t->keys.as<uint64_t>(), t->sbox.as<uint16_t>(), n, ng, totals + 1, ls, t->gflag.as<int>(),
                      t->gid.as<int>(), t->gstart.as<int>(), t->spos.as<double>(), t->gA.as<int4>(), t->gB.as<int4>(),
                      t->gC.as<int4>(), t->gD.as<int4>(), s));
  NB_CU(nb_group_runs(ng, totals + 1, t->gA.as<int4>(), t->gD.as<int4>(), t->gflag.as<int>(), t->gid.as<int>(),
                      totals + 2, t->scantmp.as<int>(), t->runhead.as<int>(), s));
  if (timed) NB_CU(cudaEventRecord(be[2], s));
  // A5 moments (with the background weights when asked for)
  const double* rho = nullptr;
  if (p.flags & NBODY_FLAG_BACKGROUND) {
    NB_CU(t->rho.ensure(8 * (int64_t)t->nbox * 65));  // the densities, then 64 partial sums per box
    NB_CU(nb_box_mass(t->off.as<int64_t>(), t->smass.as<float>(), t->nbox, t->rho.as<double>(),
                      t->rho.as<double>() + t->nbox, s));
    rho = t->rho.as<double>();
  }
  NB_CU(nb_upward(p.order, fp64, nc, totals, t->cA.as<int4>(), t->cB.as<int4>(), t->spos.as<double>(),
                  t->smass.as<float>(), n, t->mom.as<double>(), t->coef.p, t->ukey.as<uint8_t>(),
                  t->uorder.as<uint32_t>(), t->urng.as<uint32_t>(), t->urng.as<int>() + 256,
                  t->cbox.as<uint16_t>(), rho, (p.flags & NBODY_FLAG_DUAL) ? t->mom32.as<float>() : nullptr, &sc,
                  s));
  if (p.ewald_order > 0) {
    const int ne = (p.ewald_order + 1) * (p.ewald_order + 2) * (p.ewald_order + 3) / 6;
    // FP64 moments, then their FP32 copy
    NB_CU(t->fm.ensure(12 * (int64_t)t->nbox * (1 << (3 * p.ewald_level)) * ne));
    NB_CU(nb_field_moments(p.ewald_order, p.ewald_level, t->nbox, t->off.as<int64_t>(), t->keys.as<uint64_t>(),
                           t->spos.as<double>(), t->smass.as<float>(), n, t->hval.as<int>(),
                           t->ckey.as<uint64_t>(), t->cbox.as<uint16_t>(), t->hcap, t->mom.as<double>(), p.order,
                           t->fm.as<double>(), fm32_of(t), s));
  }
  if (timed) {
    NB_CU(cudaEventRecord(be[3], s));
    t->nb_log++;
  }
  t->forces_valid = false;
  t->field_valid = false;
  return NBODY_OK;
}

// state shared by the walk and the reverse walk: thresholds, stacks, tables
int eval_prep(nbody_tree* t, cudaStream_t s) {
  const nbody_params& p = t->prm;
  const bool fp64 = p.precision == NBODY_FP64;
  NB_CU(t->counters.ensure(64));
  if (!t->tot.p) {
    NB_CU(t->tot.ensure(64));
    NB_CU(cudaMemsetAsync(t->tot.p, 0, 64, s));
  }
  NB_CU(t->gctr.ensure(64));
  const int warps = nb_walk_warps(fp64);
  if (t->walk_blocks == 0) t->walk_blocks = t->nsm * 8;
  NB_CU(t->stack.ensure(4 * (int64_t)t->walk_blocks * warps * kStackCap));
  for (int l = 0; l < NB_NLEV; l++) {
    double sl = ldexp(1.0, 23 - l);
    double T = floor((sl * sl) / (p.theta * p.theta));
    t->thr[l] = T > 4.0e18 ? (long long)4000000000000000000LL : (long long)T;
  }
  if (p.ewald_order > 0) {
    NB_CU(nb_phitilde_table(p.ewald_grid, p.ewald_order + 1, &t->tab64, &t->tab32, s));
    NB_CU(t->lbuf.ensure((fp64 ? 8 : 4) * (int64_t)t->group_cap * nb_field_stride(p.ewald_order)));
  }
  return NBODY_OK;
}

// image-field local expansions of the last build, without the walk
int field_impl(nbody_tree* t, cudaStream_t s) {
  const nbody_params& p = t->prm;
  const bool fp64 = p.precision == NBODY_FP64;
  int rc = eval_prep(t, s);
  if (rc) return rc;
  const void* tab = fp64 ? (const void*)t->tab64 : (const void*)t->tab32;
  if (p.ewald_order > 0)
    NB_CU(nb_field_local(t->dev(), fp64, p.ewald_order, p.ewald_level, p.ewald_grid, t->src.p,
                         t->fm.as<double>(), fm32_of(t), tab, t->lbuf.p, s));
  t->field_valid = true;
  return NBODY_OK;
}

int forces_impl(nbody_tree* t, float* acc, cudaStream_t s, double* acc64 = nullptr, const uint8_t* sact = nullptr,
                const uint8_t* gact = nullptr, float* pot = nullptr) {
  const nbody_params& p = t->prm;
  const bool fp64 = p.precision == NBODY_FP64;
  const int64_t n = t->n;
  NB_CU(t->accw.ensure((fp64 ? 24 : 12) * n));
  if (pot) NB_CU(t->potw.ensure((fp64 ? 8 : 4) * n));
  int rc = eval_prep(t, s);
  if (rc) return rc;
  if (t->fixed_cap) NB_CU(nb_cap_check(t->totals.as<int>(), t->cell_cap, t->group_cap, t->status.as<unsigned>(), s));
  NB_CU(cudaMemsetAsync(t->counters.p, 0, 64, s));
  const void* eps2 = fp64 ? (const void*)((char*)t->eps2.p + ((4 * t->nbox + 15) & ~15)) : t->eps2.p;
  cudaEvent_t* fe = t->fev[t->nf_log % kRing];
  t->last_stream = s;
  const bool timed = !capturing(s);
  if (timed) NB_CU(cudaEventRecord(fe[0], s));
  DevTree tr = t->dev();
  tr.sact = sact;
  tr.gact = gact;
  unsigned long long* ctr = t->counters.as<unsigned long long>();
  const bool dual = (p.flags & NBODY_FLAG_DUAL) != 0;
  const int repl = (p.flags & NBODY_FLAG_REPLICAS) ? 2 : 0;
  if (repl) {
    // the walk's stack entries hold the image above 25 bits of cell index
    if (t->cell_cap >= (1 << 25)) return NBODY_ENOTSUP;
    NB_CU(t->lat_part.ensure(8 * 512 * 165 * (int64_t)t->nbox));
    NB_CU(t->lat_mom.ensure(8 * 165 * (int64_t)t->nbox));
    NB_CU(t->lat_Ld.ensure(8 * 165 * (int64_t)t->nbox));
    NB_CU(t->lat_Lt.ensure((fp64 ? 8 : 4) * 165 * (int64_t)t->nbox));
  }
  NbDualBufs db{};
  if (dual) {
    // chunks of 32 cell-group pairs: 32 per group to begin with (1024 pairs;
    // the benchmark workload averages under 600), grown when a walk asks for
    // more (dual_regrow)
    if (t->lc_cap == 0) t->lc_cap = std::max<int64_t>(1024, (int64_t)t->group_cap * 32);
    const int64_t cap = t->lc_cap;
    NB_CU(t->lc_cell.ensure(4 * 32 * cap));
    NB_CU(t->lc_img.ensure(4 * 32 * cap));
    NB_CU(t->lc_head.ensure(16 * cap));
    NB_CU(t->lc_L.ensure(4 * (int64_t)kDualLStride * cap));
    NB_CU(t->lc_first.ensure(4 * (int64_t)t->group_cap + 64));
    NB_CU(t->lc_ctr.ensure(64));
    db = NbDualBufs{t->lc_cell.as<int>(), t->lc_img.as<int>(), t->lc_head.as<int4>(), t->lc_first.as<int>(),
                    t->lc_ctr.as<int>(), t->lc_L.as<float>(), (int)cap};
  }
  // with a potential: the potential variant of the walk (accelerations too);
  // with the dual form it gives the potential only, and the dual walk then
  // writes the accelerations (the potential of every accepted cell is its
  // expansion's, as in the oracle)
  for (int pass = pot ? 0 : 1; pass < 2; pass++) {
    if (pass == 1 && pot && !dual) break;
    if (pass == 1 && pot) NB_CU(cudaMemsetAsync(t->counters.p, 0, 64, s));
    NB_CU(nb_walk(tr, fp64, p.order, t->coef.p, t->src.p, eps2, t->thr, p.n_direct, image_level(p),
                  t->stack.as<int>(), kStackCap, t->walk_blocks, t->gctr.as<int>(), t->accw.p, ctr,
                  t->status.as<unsigned>(), t->nsm, ((p.flags >> 8) & 0xf) - 1,
                  (p.flags & NBODY_FLAG_MAC_EDGE) ? 1 : 0, (p.flags & NBODY_FLAG_BACKGROUND) ? 1 : 0,
                  (p.flags & NBODY_FLAG_K1) ? 1 : 0, dual ? 1 : 0, p.theta, t->mom32.as<float>(), group_level(p),
                  dual ? &db : nullptr, pass == 0 ? t->potw.p : nullptr, repl, s));
  }
  if (timed) NB_CU(cudaEventRecord(fe[1], s));
  const void* tab = fp64 ? (const void*)t->tab64 : (const void*)t->tab32;
  if (repl)
    NB_CU(nb_lattice(tr, fp64, repl, t->accw.p, acc, acc64, pot ? t->potw.p : nullptr, pot, t->lat_part.as<double>(),
                     t->lat_mom.as<double>(), t->lat_Ld.as<double>(), t->lat_Lt.p, s));
  else
    NB_CU(nb_periodic(tr, fp64, p.ewald_order, p.ewald_level, p.ewald_grid, t->src.p, t->fm.as<double>(), fm32_of(t), tab,
                      t->lbuf.p, t->accw.p, acc, ctr + 2, acc64, pot ? t->potw.p : nullptr, pot, s));
  if (timed) NB_CU(cudaEventRecord(fe[2], s));
  accumulate_kernel<<<1, 32, 0, s>>>(ctr, t->tot.as<unsigned long long>());
  nb_launch_counter += 1;
  if (timed) t->nf_log++;
  t->forces_valid = true;
  t->field_valid = true;
  return NBODY_OK;
}

// out = (d acc / d pos)^T lam for the tree as last built (forces refreshed if needed)
int vjp_impl(nbody_tree* t, const float* lam, double* out, cudaStream_t s) {
  const nbody_params& p = t->prm;
  if (p.precision != NBODY_MIXED || p.ewald_order > 4 ||
      (p.flags & (NBODY_FLAG_K1 | NBODY_FLAG_DUAL | NBODY_FLAG_REPLICAS)))
    return NBODY_ENOTSUP;
  const int64_t n = t->n;
  if (!t->field_valid) {
    int rc = field_impl(t, s);
    if (rc) return rc;
  }
  const int nm = nb_adj_coef_nm(p.order);
  NB_CU(t->a_lam.ensure(12 * n));
  NB_CU(t->a_mu.ensure(24 * n));
  NB_CU(t->a_nuc.ensure(4 * (int64_t)t->cell_cap * ((nm + 3) & ~3)));
  NB_CU(t->a_nu.ensure(8 * (int64_t)t->cell_cap * nm));
  if (p.ewald_order > 0) {
    const int ne = (p.ewald_order + 1) * (p.ewald_order + 2) * (p.ewald_order + 3) / 6;
    NB_CU(t->a_lbar.ensure(8 * (int64_t)t->group_cap * nb_adj_lbar_stride(p.ewald_order)));
    NB_CU(t->a_nue.ensure(8 * (int64_t)t->nbox * (1 << (3 * p.ewald_level)) * ne));
  }
  if (t->fixed_cap) NB_CU(nb_cap_check(t->totals.as<int>(), t->cell_cap, t->group_cap, t->status.as<unsigned>(), s));
  AdjBuffers B;
  B.lam_s = t->a_lam.as<float>();
  B.mu = t->a_mu.as<double>();
  B.nuc = t->a_nuc.as<float>();
  B.nu = t->a_nu.as<double>();
  B.lbar = t->a_lbar.as<double>();
  B.nue = t->a_nue.as<double>();
  B.group_ctr = t->gctr.as<int>();
  DevTree tr = t->dev();
  NB_CU(nb_forces_vjp(tr, false, p.order, p.ewald_order, p.ewald_level, p.ewald_grid, t->coef.p, t->src.p,
                      t->eps2.p, t->thr, p.n_direct, t->stack.as<int>(), kStackCap, t->walk_blocks,
                      t->fm.as<double>(), t->tab32, t->lbuf.p, nb_field_stride(p.ewald_order), p.lmax, lam, out,
                      B, t->status.as<unsigned>(), t->nsm, (p.flags & NBODY_FLAG_MAC_EDGE) ? 1 : 0,
                      (p.flags & NBODY_FLAG_BACKGROUND) ? 1 : 0, s));
  return NBODY_OK;
}

int make_tree(const nbody_params* params, int nbox, const int64_t* offsets, const double* eps_host,
              const double* len_host, const double* pos, const float* mass, nbody_tree** tree, cudaStream_t s) {
  if (!tree || !pos || !offsets || nbox < 1 || nbox > NB_MAX_NBOX) return NBODY_EINVAL;
  int rc = validate(params);
  if (rc) return rc;
  if (offsets[0] != 0) return NBODY_EINVAL;
  for (int b = 0; b < nbox; b++)
    if (offsets[b + 1] <= offsets[b]) return NBODY_EINVAL;
  const int64_t n = offsets[nbox];
  if (n <= 0 || n >= ((int64_t)1 << 30)) return NBODY_EINVAL;
  if (eps_host)
    for (int b = 0; b < nbox; b++)
      if (!(eps_host[b] > 0.0)) return NBODY_EINVAL;
  if (len_host)
    for (int b = 0; b < nbox; b++)
      if (!(len_host[b] > 0.0) || len_host[b] > 1e300) return NBODY_EINVAL;
  nbody_tree* t = *tree;
  bool fresh = false;
  if (!t) {
    t = new (std::nothrow) nbody_tree();
    if (!t) return NBODY_ENOMEM;
    fresh = true;
    if (cudaGetDevice(&t->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&t->nsm, cudaDevAttrMultiProcessorCount, t->device) != cudaSuccess ||
        cudaMallocHost(&t->pinned, 64) != cudaSuccess || t->status.ensure(64) != cudaSuccess) {
      cudaGetLastError();
      delete t;
      return NBODY_ECUDA;
    }
    cudaMemset(t->status.p, 0, 64);
    for (int r = 0; r < kRing; r++) {
      for (auto& e : t->bev[r]) cudaEventCreate(&e);
      for (auto& e : t->fev[r]) cudaEventCreate(&e);
    }
    t->events = true;
  }
  std::vector<int64_t> off_new(offsets, offsets + nbox + 1);
  std::vector<double> eps_new(nbox), len_new(nbox);
  bool scaled = false;
  for (int b = 0; b < nbox; b++) {
    len_new[b] = len_host ? len_host[b] : (params->box_len > 0.0 ? params->box_len : 1.0);
    scaled |= len_new[b] != 1.0;
    eps_new[b] = (eps_host ? eps_host[b] : params->eps) / len_new[b];
  }
  // a rebuild with the same boxes enqueues no host synchronisation (so that
  // it can be captured on reserved capacities)
  const bool same_boxes = !fresh && t->off.p && t->nbox == nbox && t->h_off == off_new && t->h_eps == eps_new &&
                          t->h_len == len_new;
  t->prm = *params;
  t->nbox = nbox;
  t->n = n;
  t->pos = pos;
  t->mass = mass;
  t->scaled = scaled;
  t->h_off.swap(off_new);
  t->h_eps.swap(eps_new);
  t->h_len.swap(len_new);
  const long long l0 = nb_launch_counter;
  rc = same_boxes ? NBODY_OK : upload_boxes(t, s);
  if (rc == NBODY_OK && scaled) {
    // the tree works in box units: its positions are the caller's / L
    rc = t->upos.ensure(24 * n) == cudaSuccess ? scale_boxes<double>(t, 0, pos, t->upos.as<double>(), s)
                                               : NBODY_ENOMEM;
    t->pos = t->upos.as<double>();
  }
  // parameters may have changed the per-cell sizes of reserved buffers
  if (rc == NBODY_OK && t->fixed_cap) rc = size_cells(t, t->cell_cap, t->group_cap);
  if (rc == NBODY_OK) rc = build_impl(t, s);
  t->launches += nb_launch_counter - l0;
  if (rc == NBODY_OK && !(params->flags & NBODY_FLAG_ASYNC)) rc = read_status(t, s);
  if (rc != NBODY_OK && fresh) {
    delete t;
    return rc;
  }
  *tree = t;
  return rc;
}

}  // namespace

extern "C" {

void nbody_default_params(nbody_params* p) {
  if (!p) return;
  memset(p, 0, sizeof(*p));
  p->eps = 1.0 / (30.0 * 128.0);
  p->theta = 0.6;
  p->order = 4;
  p->n_leaf = 16;
  p->n_group = 32;
  p->n_direct = 4;
  p->lmax = 21;
  p->ewald_order = 4;
  p->ewald_level = 3;
  p->ewald_grid = 6;
  p->precision = NBODY_MIXED;
  p->flags = 0;
  p->box_len = 1.0;
}

int nbody_build_tree(const nbody_params* params, int64_t n, const double* pos_dev, const float* mass_dev,
                     nbody_tree** tree, nbody_stream_t stream) {
  if (n <= 0) return NBODY_EINVAL;
  int64_t off[2] = {0, n};
  return make_tree(params, 1, off, nullptr, nullptr, pos_dev, mass_dev, tree, (cudaStream_t)stream);
}

int nbody_build_tree_batched(const nbody_params* params, int nbox, const int64_t* offsets_host,
                             const double* eps_host, const double* pos_dev, const float* mass_dev,
                             nbody_tree** tree, nbody_stream_t stream) {
  return make_tree(params, nbox, offsets_host, eps_host, nullptr, pos_dev, mass_dev, tree, (cudaStream_t)stream);
}

int nbody_forces_batched(const nbody_params* params, int nbox, const int64_t* offsets_host,
                         const double* box_len_host, const double* eps_host, const double* pos_dev,
                         const float* mass_dev, float* acc_dev, nbody_tree** tree, nbody_stream_t stream) {
  if (!acc_dev) return NBODY_EINVAL;
  int rc = make_tree(params, nbox, offsets_host, eps_host, box_len_host, pos_dev, mass_dev, tree,
                     (cudaStream_t)stream);
  if (rc) return rc;
  return nbody_forces(*tree, acc_dev, nullptr, nullptr, stream);
}

int nbody_forces64(nbody_tree* tree, double* acc_dev, nbody_stream_t stream) {
  if (!tree || !acc_dev) return NBODY_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  const long long l0 = nb_launch_counter;
  int rc = forces_impl(tree, nullptr, s, acc_dev);
  if (rc == NBODY_OK) rc = scale_boxes<double>(tree, 1, acc_dev, acc_dev, s);
  tree->launches += nb_launch_counter - l0;
  if (rc) return rc;
  if (tree->prm.flags & NBODY_FLAG_ASYNC) return NBODY_OK;
  return read_status(tree, s);
}

int nbody_forces(nbody_tree* tree, float* acc_dev, float* pot_dev, nbody_stats* stats, nbody_stream_t stream) {
  if (!tree || !acc_dev) return NBODY_EINVAL;
  // the background's potential needs the image cells' second moments
  if (pot_dev && tree->prm.ewald_order == 1) return NBODY_ENOTSUP;
  cudaStream_t s = (cudaStream_t)stream;
  int rc = NBODY_OK;
  // a walk of the dual form that outgrew its pair pool is redone once with a
  // pool of the size it asked for (when the call synchronises)
  for (int attempt = 0; attempt < 2; attempt++) {
    const long long l0 = nb_launch_counter;
    rc = forces_impl(tree, acc_dev, s, nullptr, nullptr, nullptr, pot_dev);
    if (rc == NBODY_OK) rc = scale_boxes<float>(tree, 1, acc_dev, acc_dev, s);
    if (rc == NBODY_OK && pot_dev) rc = scale_boxes<float>(tree, 0, pot_dev, pot_dev, s, 1);
    tree->launches += nb_launch_counter - l0;
    if (rc) return rc;
    if (tree->prm.flags & NBODY_FLAG_ASYNC) return NBODY_OK;
    rc = read_status(tree, s);
    if (rc != NBODY_EOVERFLOW || capturing(s) || !tree->lc_grew) break;
  }
  if (stats) {
    memset(stats, 0, sizeof(*stats));
    unsigned long long c[4] = {0, 0, 0, 0};
    if (cudaMemcpy(c, tree->counters.p, sizeof(c), cudaMemcpyDeviceToHost) == cudaSuccess) {
      stats->p2p = (double)c[0];
      stats->m2p = (double)c[1];
      stats->m2l = (double)c[2];
      stats->decision_hash = c[3];
    }
    int nc = 0, ng = 0;
    if (host_counts(tree, &nc, &ng) != NBODY_OK) nc = ng = 0;
    stats->ncells = nc;
    stats->ngroups = ng;
    stats->nbox = tree->nbox;
    int* ml = nullptr;
    if (nc > 0 && cudaMalloc(&ml, sizeof(int)) == cudaSuccess) {
      cudaMemsetAsync(ml, 0, sizeof(int), s);
      max_level_kernel<<<gridn(nc, 256), 256, 0, s>>>(nc, tree->cA.as<int4>(), ml);
      int v = 0;
      if (cudaMemcpyAsync(&v, ml, sizeof(int), cudaMemcpyDeviceToHost, s) == cudaSuccess &&
          cudaStreamSynchronize(s) == cudaSuccess)
        stats->max_level = v;
      cudaFree(ml);
    }
    float ms = 0;
    cudaEvent_t* be = tree->bev[(tree->nb_log + kRing - 1) % kRing];
    cudaEvent_t* fe = tree->fev[(tree->nf_log + kRing - 1) % kRing];
    if (tree->nb_log > 0) {
      if (cudaEventElapsedTime(&ms, be[0], be[1]) == cudaSuccess) stats->ms_sort = ms;
      if (cudaEventElapsedTime(&ms, be[1], be[2]) == cudaSuccess) stats->ms_build = ms;
      if (cudaEventElapsedTime(&ms, be[2], be[3]) == cudaSuccess) stats->ms_upward = ms;
    }
    if (cudaEventElapsedTime(&ms, fe[0], fe[1]) == cudaSuccess) stats->ms_walk = ms;
    if (cudaEventElapsedTime(&ms, fe[1], fe[2]) == cudaSuccess) stats->ms_periodic = ms;
    cudaGetLastError();
  }
  return rc;
}

int nbody_kdk_step(nbody_tree* tree, double* pos_dev, float* mom_dev, float* acc_dev, double a0, double a1,
                   nbody_stream_t stream) {
  if (!tree || !pos_dev || !mom_dev || !acc_dev || !(a0 > 0.0) || !(a1 > 0.0)) return NBODY_EINVAL;
  if (tree->scaled) return NBODY_ENOTSUP;  // the integrator works in box units
  cudaStream_t s = (cudaStream_t)stream;
  tree->pos = pos_dev;
  const double H0 = sqrt(8.0 * M_PI / 3.0);
  const double ah = sqrt(a0 * a1);
  const double K1 = 2.0 / H0 * (sqrt(ah) - sqrt(a0));
  const double K2 = 2.0 / H0 * (sqrt(a1) - sqrt(ah));
  const double D = 2.0 / H0 * (1.0 / sqrt(a0) - 1.0 / sqrt(a1));
  const int64_t n3 = 3 * tree->n;
  const long long l0 = nb_launch_counter;
  kick_kernel<<<gridn(n3, 256), 256, 0, s>>>(n3, mom_dev, acc_dev, (float)K1);
  drift_kernel<<<gridn(n3, 256), 256, 0, s>>>(n3, pos_dev, mom_dev, D);
  nb_launch_counter += 2;
  NB_CU(cudaGetLastError());
  int rc = build_impl(tree, s);
  if (rc) return rc;
  rc = forces_impl(tree, acc_dev, s);
  if (rc) return rc;
  kick_kernel<<<gridn(n3, 256), 256, 0, s>>>(n3, mom_dev, acc_dev, (float)K2);
  nb_launch_counter += 1;
  tree->launches += nb_launch_counter - l0;
  NB_CU(cudaGetLastError());
  if (tree->prm.flags & NBODY_FLAG_ASYNC) return NBODY_OK;
  return read_status(tree, s);
}

namespace {

// accelerations of the particles with rung >= rmin, the others' left as they are
int forces_active_impl(nbody_tree* t, const int8_t* rung, int rmin, float* acc, cudaStream_t s) {
  const int64_t n = t->n;
  NB_CU(t->act_s.ensure(n));
  NB_CU(t->act_g.ensure((int64_t)t->group_cap + 1));
  active_kernel<<<gridn(n, 256), 256, 0, s>>>(n, t->vals.as<uint32_t>(), rung, rmin, t->act_s.as<uint8_t>());
  group_active_kernel<<<gridn(t->group_cap, 256), 256, 0, s>>>(t->totals.as<int>() + 1, t->gA.as<int4>(),
                                                                t->act_s.as<uint8_t>(), t->act_g.as<uint8_t>());
  nb_launch_counter += 2;
  NB_CU(cudaGetLastError());
  return forces_impl(t, acc, s, nullptr, t->act_s.as<uint8_t>(), t->act_g.as<uint8_t>());
}

}  // namespace

int nbody_assign_rungs(nbody_tree* t, const float* acc_dev, double eta, double dlna, int rmax, int8_t* rung_dev,
                       nbody_stream_t stream) {
  if (!t || !acc_dev || !rung_dev || !(eta > 0.0) || !(dlna > 0.0) || rmax < 0 || rmax > 7) return NBODY_EINVAL;
  if (t->scaled) return NBODY_ENOTSUP;
  cudaStream_t s = (cudaStream_t)stream;
  const double H0 = sqrt(8.0 * M_PI / 3.0);
  std::vector<double> c(t->nbox);
  for (int b = 0; b < t->nbox; b++) c[b] = (dlna * dlna) / ((eta * eta) * (H0 * H0) * t->h_eps[b]);
  NB_CU(t->rungc.ensure(8 * (int64_t)t->nbox));
  NB_CU(cudaMemcpyAsync(t->rungc.p, c.data(), 8 * t->nbox, cudaMemcpyHostToDevice, s));
  rung_kernel<<<gridn(t->n, 256), 256, 0, s>>>(t->n, acc_dev, t->box_of.as<uint16_t>(), t->rungc.as<double>(), rmax,
                                               rung_dev);
  t->launches += 1;
  nb_launch_counter += 1;
  NB_CU(cudaGetLastError());
  NB_CU(cudaStreamSynchronize(s));
  return NBODY_OK;
}

int nbody_forces_active(nbody_tree* t, const int8_t* rung_dev, int rmin, float* acc_dev, nbody_stream_t stream) {
  if (!t || !rung_dev || !acc_dev || rmin < 0) return NBODY_EINVAL;
  if (t->scaled) return NBODY_ENOTSUP;
  cudaStream_t s = (cudaStream_t)stream;
  const long long l0 = nb_launch_counter;
  int rc = forces_active_impl(t, rung_dev, rmin, acc_dev, s);
  t->launches += nb_launch_counter - l0;
  if (rc) return rc;
  if (t->prm.flags & NBODY_FLAG_ASYNC) return NBODY_OK;
  return read_status(t, s);
}

int nbody_kdk_multistep(nbody_tree* t, double* pos_dev, float* mom_dev, float* acc_dev, const int8_t* rung_dev,
                        double a0, double a1, int rmax, nbody_stream_t stream) {
  if (!t || !pos_dev || !mom_dev || !acc_dev || !rung_dev || !(a0 > 0.0) || !(a1 > a0) || rmax < 0 || rmax > 7)
    return NBODY_EINVAL;
  if (t->scaled) return NBODY_ENOTSUP;
  cudaStream_t s = (cudaStream_t)stream;
  t->pos = pos_dev;
  const double H0 = sqrt(8.0 * M_PI / 3.0);
  const int T = 1 << rmax;
  const double L = log(a1 / a0);
  // expansion factor at half-tick j2 (tick j2 / 2), as the oracle forms it
  auto at = [&](int j2) { return a0 * exp(L * j2 / (2 * T)); };
  auto K = [&](double x, double y) { return 2.0 / H0 * (sqrt(y) - sqrt(x)); };
  auto D = [&](double x, double y) { return 2.0 / H0 * (1.0 / sqrt(x) - 1.0 / sqrt(y)); };
  const int64_t n = t->n, n3 = 3 * n;
  const long long l0 = nb_launch_counter;
  for (int k = 0; k < T; k++) {
    // opening half kicks of the steps that start at tick k
    RungKicks ko;
    for (int r = 0; r < 8; r++) ko.f[r] = 0.f;
    for (int r = 0; r <= rmax; r++) {
      const int st = 1 << (rmax - r);
      if (k % st == 0) ko.f[r] = (float)K(at(2 * k), at(2 * k + st));
    }
    kick_rungs_kernel<<<gridn(n, 256), 256, 0, s>>>(n, mom_dev, acc_dev, rung_dev, ko);
    drift_kernel<<<gridn(n3, 256), 256, 0, s>>>(n3, pos_dev, mom_dev, D(at(2 * k), at(2 * k + 2)));
    nb_launch_counter += 2;
    NB_CU(cudaGetLastError());
    int rc = build_impl(t, s);
    if (rc) return rc;
    // the steps that end at tick k + 1: rungs >= rmax - (trailing zeros of k + 1)
    int tz = 0;
    while (tz < rmax && ((k + 1) >> tz & 1) == 0) tz++;
    const int rmin = rmax - tz;
    if ((rc = forces_active_impl(t, rung_dev, rmin, acc_dev, s))) return rc;
    RungKicks kc;
    for (int r = 0; r < 8; r++) kc.f[r] = 0.f;
    for (int r = rmin; r <= rmax; r++) {
      const int st = 1 << (rmax - r);
      kc.f[r] = (float)K(at(2 * (k + 1) - st), at(2 * (k + 1)));
    }
    kick_rungs_kernel<<<gridn(n, 256), 256, 0, s>>>(n, mom_dev, acc_dev, rung_dev, kc);
    nb_launch_counter += 1;
    NB_CU(cudaGetLastError());
  }
  t->launches += nb_launch_counter - l0;
  if (t->prm.flags & NBODY_FLAG_ASYNC) return NBODY_OK;
  return read_status(t, s);
}

int nbody_forces_vjp(nbody_tree* t, const float* lam_dev, double* out_dev, nbody_stream_t stream) {
  if (!t || !lam_dev || !out_dev) return NBODY_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  const long long l0 = nb_launch_counter;
  int rc = vjp_impl(t, lam_dev, out_dev, s);
  if (rc == NBODY_OK) rc = scale_boxes<double>(t, 2, out_dev, out_dev, s);
  t->launches += nb_launch_counter - l0;
  if (rc) return rc;
  if (t->prm.flags & NBODY_FLAG_ASYNC) return NBODY_OK;
  return read_status(t, s);
}

namespace {

// second tree of the KDK adjoint (the step's end state), created on first use
int ensure_aux(nbody_tree* t, cudaStream_t s) {
  if (t->aux) return NBODY_OK;
  t->aux = new (std::nothrow) nbody_tree();
  if (!t->aux) return NBODY_ENOMEM;
  nbody_tree* x = t->aux;
  x->device = t->device;
  x->nsm = t->nsm;
  if (cudaMallocHost(&x->pinned, 64) != cudaSuccess || x->status.ensure(64) != cudaSuccess) {
    cudaGetLastError();
    return NBODY_ECUDA;
  }
  NB_CU(cudaMemsetAsync(x->status.p, 0, 64, s));
  for (int r = 0; r < kRing; r++) {
    for (auto& e : x->bev[r]) cudaEventCreate(&e);
    for (auto& e : x->fev[r]) cudaEventCreate(&e);
  }
  x->events = true;
  return NBODY_OK;
}

int kdk_adjoint_impl(nbody_tree* t, const double* pos0, const float* mom0, const float* acc0, double a0, double a1,
                     const double* lam_pos1, const float* lam_mom1, double* lam_pos0, float* lam_mom0,
                     cudaStream_t s) {
  if (!t || !pos0 || !mom0 || !lam_pos1 || !lam_mom1 || !lam_pos0 || !lam_mom0 || !(a0 > 0.0) || !(a1 > 0.0))
    return NBODY_EINVAL;
  if (t->scaled || (t->prm.flags & (NBODY_FLAG_K1 | NBODY_FLAG_DUAL | NBODY_FLAG_REPLICAS))) return NBODY_ENOTSUP;
  if (t->prm.precision != NBODY_MIXED || t->prm.ewald_order > 4) return NBODY_ENOTSUP;
  const long long l0 = nb_launch_counter;
  const int64_t n = t->n, n3 = 3 * n;
  const double H0 = sqrt(8.0 * M_PI / 3.0);
  const double ah = sqrt(a0 * a1);
  const double K1 = 2.0 / H0 * (sqrt(ah) - sqrt(a0));
  const double K2 = 2.0 / H0 * (sqrt(a1) - sqrt(ah));
  const double D = 2.0 / H0 * (1.0 / sqrt(a0) - 1.0 / sqrt(a1));
  NB_CU(t->a_x0.ensure(8 * n3));
  NB_CU(t->a_x1.ensure(8 * n3));
  NB_CU(t->a_ph.ensure(4 * n3));
  NB_CU(t->a_g.ensure(4 * n3));
  NB_CU(t->a_lg.ensure(4 * n3));
  NB_CU(t->a_lx.ensure(8 * n3));
  NB_CU(t->a_lp.ensure(8 * n3));
  NB_CU(t->a_out.ensure(8 * n3));
  NB_CU(t->a_xc.ensure(8 * n3));
  NB_CU(t->a_lc.ensure(4 * n3));
  NB_CU(t->a_muc.ensure(8 * n3));
  NB_CU(t->a_eq.ensure(64));
  double* X0 = t->a_x0.as<double>();
  double* X1 = t->a_x1.as<double>();
  float* PH = t->a_ph.as<float>();
  float* LG = t->a_lg.as<float>();
  double* LX = t->a_lx.as<double>();
  double* LP = t->a_lp.as<double>();
  NB_CU(cudaMemcpyAsync(X0, pos0, 8 * n3, cudaMemcpyDeviceToDevice, s));
  // forward recompute with the arithmetic of nbody_kdk_step: tree at x0,
  // g(x0), the FP32 half kick and the FP64 drift
  t->pos = X0;
  int rc = build_impl(t, s);
  if (rc) return rc;
  const float* G = acc0;
  if (!G) {
    if ((rc = forces_impl(t, t->a_g.as<float>(), s))) return rc;
    G = t->a_g.as<float>();
  }
  NB_CU(cudaMemcpyAsync(PH, mom0, 4 * n3, cudaMemcpyDeviceToDevice, s));
  kick_kernel<<<gridn(n3, 256), 256, 0, s>>>(n3, PH, G, (float)K1);
  drift_from_kernel<<<gridn(n3, 256), 256, 0, s>>>(n3, X0, PH, D, X1);
  nb_launch_counter += 2;
  // J(x1)^T lam_p1: the product kept by the previous call when it was taken at
  // this x1 with this cotangent, else from a tree at x1
  bool reuse = false;
  if (t->adj_cache) {
    int* eq = t->a_eq.as<int>();
    NB_CU(cudaMemsetAsync(eq, 0, sizeof(int), s));
    differ_kernel<<<gridn(n3, 256), 256, 0, s>>>(n3, (const unsigned long long*)X1,
                                                   t->a_xc.as<unsigned long long>(), (const unsigned*)lam_mom1,
                                                   t->a_lc.as<unsigned>(), eq);
    nb_launch_counter += 1;
    NB_CU(cudaMemcpyAsync(t->pinned, eq, sizeof(int), cudaMemcpyDeviceToHost, s));
    NB_CU(cudaStreamSynchronize(s));
    reuse = ((int*)t->pinned)[0] == 0;
  }
  const double* MU1 = t->a_muc.as<double>();
  if (!reuse) {
    if ((rc = ensure_aux(t, s))) return rc;
    nbody_tree* x = t->aux;
    x->prm = t->prm;
    x->n = t->n;
    x->pos = X1;
    x->mass = t->mass;
    if (x->nbox != t->nbox || x->h_off != t->h_off || x->h_eps != t->h_eps || !x->off.p) {
      x->nbox = t->nbox;
      x->h_off = t->h_off;
      x->h_eps = t->h_eps;
      if ((rc = upload_boxes(x, s))) return rc;
    }
    if ((rc = build_impl(x, s))) return rc;
    if ((rc = vjp_impl(x, lam_mom1, t->a_out.as<double>(), s))) return rc;
    MU1 = t->a_out.as<double>();
  }
  // lam_x1' = lam_x1 + K2 mu1;  lam_ph = lam_p1 + D lam_x1'
  adj_mid_kernel<<<gridn(n3, 256), 256, 0, s>>>(n3, lam_pos1, MU1, lam_mom1, K2, D, LX, LP, LG);
  nb_launch_counter += 1;
  // J(x0)^T lam_ph, kept for the next call (a_out is free once MU1 is used)
  double* MU0 = reuse ? t->a_out.as<double>() : t->a_muc.as<double>();
  if ((rc = vjp_impl(t, LG, MU0, s))) return rc;
  // lam_x0 = lam_x1' + K1 mu0;  lam_p0 = lam_ph (FP32)
  adj_fin_kernel<<<gridn(n3, 256), 256, 0, s>>>(n3, LX, MU0, K1, LG, lam_pos0, lam_mom0);
  nb_launch_counter += 1;
  NB_CU(cudaMemcpyAsync(t->a_lc.p, LG, 4 * n3, cudaMemcpyDeviceToDevice, s));
  if (reuse) std::swap(t->a_out, t->a_muc);
  std::swap(t->a_x0, t->a_xc);
  t->pos = t->a_xc.as<double>();
  t->adj_cache = true;
  t->adj_steps += 1;
  t->adj_reused += reuse ? 1 : 0;
  NB_CU(cudaGetLastError());
  t->launches += nb_launch_counter - l0;
  if (t->prm.flags & NBODY_FLAG_ASYNC) return NBODY_OK;
  if (!reuse && (rc = read_status(t->aux, s))) return rc;
  return read_status(t, s);
}

}  // namespace

int nbody_kdk_adjoint(nbody_tree* t, const double* pos0, const float* mom0, double a0, double a1,
                      const double* lam_pos1, const float* lam_mom1, double* lam_pos0, float* lam_mom0,
                      nbody_stream_t stream) {
  return kdk_adjoint_impl(t, pos0, mom0, nullptr, a0, a1, lam_pos1, lam_mom1, lam_pos0, lam_mom0,
                          (cudaStream_t)stream);
}

int nbody_kdk_adjoint_acc(nbody_tree* t, const double* pos0, const float* mom0, const float* acc0, double a0,
                          double a1, const double* lam_pos1, const float* lam_mom1, double* lam_pos0,
                          float* lam_mom0, nbody_stream_t stream) {
  if (!acc0) return NBODY_EINVAL;
  return kdk_adjoint_impl(t, pos0, mom0, acc0, a0, a1, lam_pos1, lam_mom1, lam_pos0, lam_mom0,
                          (cudaStream_t)stream);
}

// size of the image-field lattice table of the tree's parameters (elements)
static int64_t image_table_count(const nbody_params& p) {
  if (p.ewald_order <= 0) return NBODY_EINVAL;
  const int64_t m = (1 << (p.ewald_grid - 1)) + 2;
  const int P = p.ewald_order + 1;
  return m * m * m * ((P + 1) * (P + 2) * (P + 3) / 6);
}

int64_t nbody_tree_count(const nbody_tree* t, int what) {
  if (!t) return NBODY_EINVAL;
  if (what == NBODY_EXPORT_IMAGE_TABLE) return image_table_count(t->prm);
  int nc = 0, ng = 0;
  if (what != NBODY_EXPORT_SORTED_KEYS && what != NBODY_EXPORT_PERM) {
    int rc = host_counts(t, &nc, &ng);
    if (rc) return rc;
  }
  switch (what) {
    case NBODY_EXPORT_SORTED_KEYS:
    case NBODY_EXPORT_PERM: return t->n;
    case NBODY_EXPORT_CELL_KEYS:
    case NBODY_EXPORT_CELL_RANGE:
    case NBODY_EXPORT_CELL_LEVEL:
    case NBODY_EXPORT_MOMENTS: return nc;
    case NBODY_EXPORT_GROUPS: return ng;
    default: return NBODY_EINVAL;
  }
}

int nbody_tree_export(const nbody_tree* t, int what, void* dst, nbody_stream_t stream) {
  if (!t || !dst) return NBODY_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  if (what == NBODY_EXPORT_IMAGE_TABLE) {
    const int64_t cnt = image_table_count(t->prm);
    if (cnt < 0) return (int)cnt;
    const double* t64 = nullptr;
    const float* t32 = nullptr;
    NB_CU(nb_phitilde_table(t->prm.ewald_grid, t->prm.ewald_order + 1, &t64, &t32, s));
    NB_CU(cudaMemcpyAsync(dst, t64, 8 * cnt, cudaMemcpyDeviceToDevice, s));
    NB_CU(cudaStreamSynchronize(s));
    return NBODY_OK;
  }
  const int nm = (t->prm.order + 1) * (t->prm.order + 2) * (t->prm.order + 3) / 6;
  int nc = 0, ng = 0;
  int rc = host_counts(t, &nc, &ng);
  if (rc) return rc;
  switch (what) {
    case NBODY_EXPORT_SORTED_KEYS:
      NB_CU(cudaMemcpyAsync(dst, t->keys.p, 8 * t->n, cudaMemcpyDeviceToDevice, s));
      break;
    case NBODY_EXPORT_PERM: NB_CU(cudaMemcpyAsync(dst, t->vals.p, 4 * t->n, cudaMemcpyDeviceToDevice, s)); break;
    case NBODY_EXPORT_CELL_KEYS:
      NB_CU(cudaMemcpyAsync(dst, t->ckey.p, 8 * (int64_t)nc, cudaMemcpyDeviceToDevice, s));
      break;
    case NBODY_EXPORT_CELL_RANGE:
    case NBODY_EXPORT_CELL_LEVEL:
      export_cells_kernel<<<gridn(nc, 256), 256, 0, s>>>(nc, t->cA.as<int4>(), t->cB.as<int4>(), what, (int*)dst);
      break;
    case NBODY_EXPORT_MOMENTS:
      NB_CU(cudaMemcpyAsync(dst, t->mom.p, 8 * (int64_t)nc * nm, cudaMemcpyDeviceToDevice, s));
      break;
    case NBODY_EXPORT_GROUPS:
      export_groups_kernel<<<gridn(ng, 256), 256, 0, s>>>(ng, t->gA.as<int4>(), (int*)dst);
      break;
    default: return NBODY_EINVAL;
  }
  NB_CU(cudaGetLastError());
  NB_CU(cudaStreamSynchronize(s));
  return NBODY_OK;
}

int nbody_tree_lookup(const nbody_tree* t, const uint64_t* keys_dev, int64_t nkeys, int32_t* idx_dev,
                      nbody_stream_t stream) {
  if (!t || !keys_dev || !idx_dev || nkeys < 0) return NBODY_EINVAL;
  if (nkeys == 0) return NBODY_OK;
  cudaStream_t s = (cudaStream_t)stream;
  NB_CU(nb_hash_lookup(keys_dev, nkeys, 0, t->hval.as<int>(), t->ckey.as<uint64_t>(), t->cbox.as<uint16_t>(),
                       t->hcap, (int*)idx_dev, s));
  NB_CU(cudaStreamSynchronize(s));
  return NBODY_OK;
}

int nbody_timing_read(nbody_tree* t, nbody_timing* out, int reset) {
  if (!t || !out) return NBODY_EINVAL;
  memset(out, 0, sizeof(*out));
  NB_CU(cudaStreamSynchronize(t->last_stream));
  const int64_t nb = t->nb_log < kRing ? t->nb_log : kRing;
  const int64_t nf = t->nf_log < kRing ? t->nf_log : kRing;
  for (int64_t r = 0; r < nb; r++) {
    float a = 0, b = 0, c = 0;
    cudaEvent_t* e = t->bev[(t->nb_log - 1 - r) % kRing];
    NB_CU(cudaEventElapsedTime(&a, e[0], e[1]));
    NB_CU(cudaEventElapsedTime(&b, e[1], e[2]));
    NB_CU(cudaEventElapsedTime(&c, e[2], e[3]));
    out->ms_sort += a;
    out->ms_build += b;
    out->ms_upward += c;
  }
  for (int64_t r = 0; r < nf; r++) {
    float a = 0, b = 0;
    cudaEvent_t* e = t->fev[(t->nf_log - 1 - r) % kRing];
    NB_CU(cudaEventElapsedTime(&a, e[0], e[1]));
    NB_CU(cudaEventElapsedTime(&b, e[1], e[2]));
    out->ms_walk += a;
    out->ms_periodic += b;
  }
  out->builds = nb;
  out->evaluations = nf;
  out->launches = t->launches;
  out->walk_variant = nb_walk_variant(t->prm.precision == NBODY_FP64, (t->prm.flags & NBODY_FLAG_DUAL) != 0,
                                      t->prm.order, out->walk_tune_ms);
  out->adjoint_steps = t->adj_steps;
  out->adjoint_reused = t->adj_reused;
  if (t->tot.p) {
    unsigned long long c[5] = {0, 0, 0, 0, 0};
    NB_CU(cudaMemcpy(c, t->tot.p, sizeof(c), cudaMemcpyDeviceToHost));
    out->p2p = (double)c[0];
    out->m2p = (double)c[1];
    out->m2l = (double)c[2];
    out->decision_hash = c[3];
    out->m2l_dual = (double)c[4];
  }
  if (reset) {
    t->nb_log = 0;
    t->nf_log = 0;
    t->launches = 0;
    t->adj_steps = 0;
    t->adj_reused = 0;
    if (t->tot.p) NB_CU(cudaMemset(t->tot.p, 0, 64));
  }
  return NBODY_OK;
}

int nbody_reserve(nbody_tree* t, int64_t max_cells, int64_t max_groups, nbody_stream_t stream) {
  if (!t || max_cells < 0 || max_groups < 0 || (max_cells == 0) != (max_groups == 0)) return NBODY_EINVAL;
  if (max_cells > ((int64_t)1 << 30) || max_groups > ((int64_t)1 << 30)) return NBODY_EINVAL;
  // a group holds at least one particle, and the group scans run in
  // per-particle scratch
  if (max_groups > t->n) max_groups = t->n;
  cudaStream_t s = (cudaStream_t)stream;
  const long long l0 = nb_launch_counter;
  int rc = NBODY_OK;
  if (max_cells == 0) {
    t->fixed_cap = false;
  } else {
    NB_CU(cudaStreamSynchronize(s));
    if (t->last_stream) NB_CU(cudaStreamSynchronize(t->last_stream));
    if ((rc = size_cells(t, (int)max_cells, (int)max_groups))) return rc;
    t->fixed_cap = true;
  }
  // the buffers may have moved: rebuild from the positions of the last build
  rc = build_impl(t, s);
  t->launches += nb_launch_counter - l0;
  if (rc) return rc;
  rc = read_status(t, s);
  if (rc == NBODY_OK && t->fixed_cap) {
    int nc = 0, ng = 0;
    if ((rc = host_counts(t, &nc, &ng))) return rc;
    t->ncell = nc;
    t->ngroup = ng;
  }
  return rc;
}

int nbody_autotune(nbody_tree* t, nbody_tune* out, nbody_stream_t stream) {
  if (!t) return NBODY_EINVAL;
  if (t->fixed_cap) return NBODY_ENOTSUP;
  cudaStream_t s = (cudaStream_t)stream;
  if (capturing(s)) return NBODY_ENOTSUP;
  const long long l0 = nb_launch_counter;
  const nbody_params p0 = t->prm;
  static const int kGroups[3] = {16, 24, 32};
  static const int kDirect[4] = {2, 4, 8, 12};
  nbody_tune r;
  memset(&r, 0, sizeof(r));
  r.best = -1;
  Buf acc;
  NB_CU(acc.ensure(12 * t->n));
  EventPair ev;
  NB_CU(ev.create());
  int rc = NBODY_OK;
  for (int gi = 0; gi < 3 && rc == NBODY_OK; gi++)
    for (int di = 0; di < 4 && rc == NBODY_OK; di++) {
      if (kDirect[di] > p0.n_leaf) continue;
      t->prm.n_group = kGroups[gi];
      t->prm.n_direct = kDirect[di];
      // once untimed (buffers sized for this candidate), then timed
      if ((rc = build_impl(t, s)) || (rc = forces_impl(t, acc.as<float>(), s))) break;
      NB_CU(cudaEventRecord(ev.a, s));
      if ((rc = build_impl(t, s)) || (rc = forces_impl(t, acc.as<float>(), s))) break;
      NB_CU(cudaEventRecord(ev.b, s));
      NB_CU(cudaEventSynchronize(ev.b));
      if ((rc = read_status(t, s))) break;
      float ms = 0.f;
      NB_CU(cudaEventElapsedTime(&ms, ev.a, ev.b));
      const int k = r.ncand++;
      r.n_group[k] = kGroups[gi];
      r.n_direct[k] = kDirect[di];
      r.ms[k] = ms;
      if (r.best < 0 || ms < r.ms[r.best]) r.best = k;
    }
  t->prm = p0;
  if (rc == NBODY_OK && r.best >= 0) {
    t->prm.n_group = r.n_group[r.best];
    t->prm.n_direct = r.n_direct[r.best];
  }
  // the tree as the caller will use it: rebuilt with the kept tile sizes
  const int rb = build_impl(t, s);
  t->launches += nb_launch_counter - l0;
  if (rc == NBODY_OK) rc = rb;
  if (rc == NBODY_OK) rc = read_status(t, s);
  if (out) *out = r;
  return rc;
}

int nbody_check(nbody_tree* t, nbody_stream_t stream) {
  if (!t) return NBODY_EINVAL;
  return read_status(t, (cudaStream_t)stream);
}

void nbody_tree_free(nbody_tree* t) { delete t; }

const char* nbody_strerror(int code) {
  switch (code) {
    case NBODY_OK: return "success";
    case NBODY_EINVAL: return "invalid argument";
    case NBODY_ENOMEM: return "device memory allocation failed";
    case NBODY_ECUDA: return "CUDA runtime error";
    case NBODY_EOVERFLOW: return "fixed-capacity device buffer overflow";
    case NBODY_ETIMEOUT: return "bounded device wait ran out";
    case NBODY_ENOTSUP: return "not supported";
    case NBODY_ERANGE: return "size exceeds the fixed maximum of an allocation-free entry point";
    default: return "unknown error";
  }
}

}  // extern "C"
