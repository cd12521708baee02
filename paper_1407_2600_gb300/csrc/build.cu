// Oct-tree from sorted Morton keys (Sec. 2.1: the key order implicitly
// defines the tree; parent and daughter keys follow by bit operations; a hash
// table maps a cell key to its storage).
//
// A cell is a key prefix.  A level-l prefix exists as a cell iff l = 0 (the
// box root) or its parent prefix holds more than n_leaf particles and the
// parent's level is below lmax.  Every cell starts at the first particle of
// its prefix range, so the cells starting at particle i are the levels
// l0(i) .. l0(i)+c_i-1 with l0(i) = (common-prefix level with particle i-1)+1.
// Counting c_i per particle and scanning gives the cells in depth-first
// (pre-)order; one stable pass by level turns that into breadth-first order,
// in which the daughters of a cell are contiguous.
#include "common.cuh"

namespace {

__device__ __forceinline__ uint64_t prefix_of(uint64_t k, int level) {
  return level == 0 ? 0ull : (k >> (3 * (NB_QBITS - level)));
}

// first index in [lo, hi) whose level-l prefix is >= P
__device__ __forceinline__ int64_t lower_pref(const uint64_t* __restrict__ k, int64_t lo, int64_t hi,
                                              uint64_t P, int level) {
  while (lo < hi) {
    int64_t mid = (lo + hi) >> 1;
    if (prefix_of(k[mid], level) < P) lo = mid + 1; else hi = mid;
  }
  return lo;
}
// first index in [lo, hi) whose level-l prefix is > P
__device__ __forceinline__ int64_t upper_pref(const uint64_t* __restrict__ k, int64_t lo, int64_t hi,
                                              uint64_t P, int level) {
  while (lo < hi) {
    int64_t mid = (lo + hi) >> 1;
    if (prefix_of(k[mid], level) <= P) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// Galloping forms of the two searches for a prefix P that particle i itself
// has: the ranges they look for are usually short, so probing i +- 1, 2, 4, ...
// before bisecting touches a few nearby keys instead of O(log n) scattered ones.
// first index in (i, hi) whose level-l prefix is > P (hi if none)
__device__ __forceinline__ int64_t upper_pref_from(const uint64_t* __restrict__ k, int64_t i, int64_t hi,
                                                   uint64_t P, int level) {
  int64_t lo = i + 1, step = 1;
  while (true) {
    const int64_t probe = i + step;
    if (probe >= hi) break;
    if (prefix_of(k[probe], level) > P) {
      hi = probe;
      break;
    }
    lo = probe + 1;
    step <<= 1;
  }
  return upper_pref(k, lo, hi, P, level);
}
// first index in [lo, i] whose level-l prefix is >= P (the start of P's range)
__device__ __forceinline__ int64_t lower_pref_to(const uint64_t* __restrict__ k, int64_t lo, int64_t i,
                                                 uint64_t P, int level) {
  int64_t hi = i, step = 1;
  while (true) {
    const int64_t probe = i - step;
    if (probe < lo) break;
    if (prefix_of(k[probe], level) < P) {
      lo = probe + 1;
      break;
    }
    hi = probe;
    step <<= 1;
  }
  return lower_pref(k, lo, hi + 1, P, level);
}

__device__ __forceinline__ int first_level(const uint64_t* __restrict__ k, int64_t i, int64_t bb) {
  if (i == bb) return 0;
  uint64_t x = k[i - 1] ^ k[i];
  if (x == 0ull) return NB_NLEV;  // identical key: starts no cell
  return (__clzll((long long)x) - 1) / 3 + 1;
}

struct BuildArgs {
  const uint64_t* skeys;
  const uint16_t* sbox;
  const int64_t* off;
  int64_t n;
  int n_leaf, lmax;
};

__global__ void count_cells_kernel(BuildArgs a, int* __restrict__ ccount, int8_t* __restrict__ l0out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < a.n;
       i += (int64_t)gridDim.x * blockDim.x) {
    int b = a.sbox[i];
    int64_t bb = a.off[b], be = a.off[b + 1];
    int l0 = first_level(a.skeys, i, bb);
    int c = 0;
    if (l0 <= a.lmax) {
      uint64_t k = a.skeys[i];
      bool exists = true;
      if (l0 > 0) {
        uint64_t pp = prefix_of(k, l0 - 1);
        int64_t lo = lower_pref_to(a.skeys, bb, i, pp, l0 - 1);
        int64_t hi = upper_pref_from(a.skeys, i, be, pp, l0 - 1);
        exists = (hi - lo) > a.n_leaf;
      }
      if (exists) {
        int l = l0;
        while (true) {
          c++;
          int64_t hi = upper_pref_from(a.skeys, i, be, prefix_of(k, l), l);
          if (hi - i > a.n_leaf && l < a.lmax) l++; else break;
        }
      }
    }
    ccount[i] = c;
    l0out[i] = (int8_t)l0;
  }
}

__global__ void emit_cells_kernel(BuildArgs a, const int* __restrict__ ccount, const int* __restrict__ coff,
                                  const int8_t* __restrict__ l0in, const int* __restrict__ pncell,
                                  uint8_t* __restrict__ plevel, int* __restrict__ pstart,
                                  int* __restrict__ pcount, int* __restrict__ pparent) {
  const int ncell = *pncell;  // 0 when the count exceeded the buffers' capacity
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < a.n;
       i += (int64_t)gridDim.x * blockDim.x) {
    int c = ccount[i];
    if (c == 0) continue;
    int b = a.sbox[i];
    int64_t bb = a.off[b], be = a.off[b + 1];
    int l0 = l0in[i];
    uint64_t k = a.skeys[i];
    int p0 = coff[i];
    if (p0 + c > ncell) continue;
    for (int t = 0; t < c; t++) {
      int l = l0 + t, p = p0 + t;
      int64_t hi = upper_pref_from(a.skeys, i, be, prefix_of(k, l), l);
      plevel[p] = (uint8_t)l;
      pstart[p] = (int)i;
      pcount[p] = (int)(hi - i);
      int par;
      if (t > 0) par = p - 1;
      else if (l == 0) par = -1;
      else {
        int64_t s = NB_IDX(lower_pref_to(a.skeys, bb, i, prefix_of(k, l - 1), l - 1), a.n, 301);
        par = coff[s] + (l - 1 - (int)l0in[s]);
      }
      pparent[p] = par;
    }
  }
}

__global__ void bfs_fill_kernel(BuildArgs a, const int* __restrict__ pncell, const uint32_t* __restrict__ bfs2pre,
                                int* __restrict__ pre2bfs) {
  const int ncell = *pncell;
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < ncell; b += gridDim.x * blockDim.x)
    if (NB_IN(bfs2pre[b], ncell, 303)) pre2bfs[bfs2pre[b]] = b;
}

__global__ void bfs_cells_kernel(BuildArgs a, const int* __restrict__ pncell, const uint32_t* __restrict__ bfs2pre,
                                 const int* __restrict__ pre2bfs, const uint8_t* __restrict__ plevel,
                                 const int* __restrict__ pstart, const int* __restrict__ pcount,
                                 const int* __restrict__ pparent, int4* __restrict__ cA,
                                 int4* __restrict__ cB, uint64_t* __restrict__ ckey,
                                 uint16_t* __restrict__ cbox) {
  const int ncell = *pncell;
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < ncell; b += gridDim.x * blockDim.x) {
    int p = NB_IDX((int)bfs2pre[b], ncell, 304);
    int l = plevel[p];
    int s = NB_IDX(pstart[p], (int)a.n, 305);
    uint64_t pre = prefix_of(a.skeys[s], l);
    int ix = (int)compact3(pre), iy = (int)compact3(pre >> 1), iz = (int)compact3(pre >> 2);
    cA[b] = make_int4(cell_c2(ix, l), cell_c2(iy, l), cell_c2(iz, l), l);
    int par = pparent[p];
    cB[b] = make_int4(s, pcount[p], 0, par >= 0 ? pre2bfs[NB_IDX(par, ncell, 302)] : -1);
    ckey[b] = (1ull << (3 * l)) | pre;
    cbox[b] = a.sbox[s];
  }
}

// daughters of a cell are contiguous in breadth-first order
__global__ void children_kernel(const int* __restrict__ pncell, int4* __restrict__ cB) {
  const int ncell = *pncell;
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < ncell; b += gridDim.x * blockDim.x) {
    int par = cB[b].w;
    if (par < 0) continue;
    if ((b == 0 || cB[b - 1].w != par) && NB_IN(par, ncell, 306)) cB[par].z = b;  // first daughter
  }
}

__global__ void nchild_kernel(const int* __restrict__ pncell, int4* __restrict__ cA, const int4* __restrict__ cB) {
  const int ncell = *pncell;
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < ncell; b += gridDim.x * blockDim.x) {
    int par = cB[b].w;
    if (par < 0) continue;
    bool last = (b == ncell - 1) || (cB[b + 1].w != par);
    if (last && NB_IN(par, ncell, 307)) {
      int nch = b - cB[par].z + 1;
      cA[par].w = (cA[par].w & 0xff) | (nch << 8);
    }
  }
}

// ---- hash of cell keys (open addressing, linear probing) ------------------------
// slots hold cell indices (-1 = empty); a slot matches when the cell's key
// and box equal the query
__global__ void hash_insert_kernel(const int* __restrict__ pncell, const uint64_t* __restrict__ ckey,
                                   const uint16_t* __restrict__ cbox, int* __restrict__ hval,
                                   uint64_t mask, unsigned* err) {
  const int ncell = *pncell;
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < ncell; b += gridDim.x * blockDim.x) {
    uint64_t h = hslot(ckey[b], cbox[b], mask);
    bool done = false;
    for (uint64_t probe = 0; probe <= mask; probe++) {
      if (atomicCAS(&hval[h], -1, b) == -1) {
        done = true;
        break;
      }
      h = (h + 1) & mask;
    }
    if (!done) atomicOr(err, NB_ST_OVERFLOW);
  }
}

__global__ void hash_lookup_kernel(const uint64_t* __restrict__ q, int64_t nq, int box,
                                   const int* __restrict__ hval, const uint64_t* __restrict__ ckey,
                                   const uint16_t* __restrict__ cbox, uint64_t mask, int* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nq;
       i += (int64_t)gridDim.x * blockDim.x) {
    out[i] = hash_find(hval, ckey, cbox, mask, q[i], box);
  }
}

// ---- leaves: particle -> leaf and leaf-relative FP32/FP64 source records ----------
template <typename T>
__global__ void leaf_kernel(const int* __restrict__ pncell, const int4* __restrict__ cA,
                            const int4* __restrict__ cB, const double* __restrict__ spos,
                            const float* __restrict__ smass, int64_t n, int* __restrict__ sleaf,
                            typename Vec4<T>::type* __restrict__ src) {
  const int ncell = *pncell;
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < ncell; b += gridDim.x * blockDim.x) {
    int4 a = cA[b];
    if ((a.w >> 8) != 0) continue;  // not a leaf
    int4 r = cB[b];
    const double cx = i2d_pow2(a.x, -23), cy = i2d_pow2(a.y, -23), cz = i2d_pow2(a.z, -23);
    for (int j = r.x; j < r.x + r.y; j++) {
      if (!NB_IN(j, n, 309)) break;
      sleaf[j] = b;
      typename Vec4<T>::type v;
      v.x = (T)(spos[j] - cx);
      v.y = (T)(spos[n + j] - cy);
      v.z = (T)(spos[2 * n + j] - cz);
      v.w = (T)smass[j];
      src[j] = v;
    }
  }
}

// ---- groups: runs of <= n_group particles inside one level-ls cell -------------------
__global__ void group_flag_kernel(BuildArgs a, int ls, int n_group, int* __restrict__ flag) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < a.n;
       i += (int64_t)gridDim.x * blockDim.x) {
    int b = a.sbox[i];
    int64_t bb = a.off[b];
    uint64_t P = prefix_of(a.skeys[i], ls);
    int64_t rs = lower_pref_to(a.skeys, bb, i, P, ls);
    flag[i] = ((i - rs) % n_group) == 0 ? 1 : 0;
  }
}

__global__ void group_start_kernel(int64_t n, const int* __restrict__ flag, const int* __restrict__ gid,
                                   const int* __restrict__ pngroup, int* __restrict__ gstart) {
  const int ngroup = *pngroup;  // 0 when the count exceeded the buffers' capacity
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    if (flag[i] && gid[i] < ngroup && NB_IN(gid[i], ngroup, 310)) gstart[gid[i]] = (int)i;
}

// one warp per group: count, box, integer bounding box and expansion point
__global__ void group_info_kernel(BuildArgs a, const int* __restrict__ pngroup, int ls,
                                  const int* __restrict__ gstart, const double* __restrict__ spos,
                                  int4* __restrict__ gA, int4* __restrict__ gB, int4* __restrict__ gC,
                                  int4* __restrict__ gD) {
  const int lane = threadIdx.x & 31;
  const int ngroup = *pngroup;
  for (int g = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; g < ngroup;
       g += (gridDim.x * blockDim.x) >> 5) {
    int s = gstart[g];
    int e = (g + 1 < ngroup) ? gstart[g + 1] : (int)a.n;
    int cnt = e - s;
    int lo[3] = {INT_MAX, INT_MAX, INT_MAX}, hi[3] = {INT_MIN, INT_MIN, INT_MIN};
    if (lane < cnt && NB_IN(s + lane, a.n, 311)) {
      int i = s + lane;
      for (int d = 0; d < 3; d++) {
        int q = (int)quant21(spos[d * a.n + i]);
        lo[d] = 2 * q;
        hi[d] = 2 * q + 2;
      }
    }
    for (int o = 16; o > 0; o >>= 1)
      for (int d = 0; d < 3; d++) {
        lo[d] = min(lo[d], __shfl_xor_sync(0xffffffffu, lo[d], o));
        hi[d] = max(hi[d], __shfl_xor_sync(0xffffffffu, hi[d], o));
      }
    if (lane == 0 && NB_IN(s, a.n, 311)) {
      uint64_t P = prefix_of(a.skeys[s], ls);
      int ix = (int)compact3(P), iy = (int)compact3(P >> 1), iz = (int)compact3(P >> 2);
      gA[g] = make_int4(s, cnt, a.sbox[s], 0);
      gB[g] = make_int4(lo[0] + hi[0], lo[1] + hi[1], lo[2] + hi[2], 0);
      gC[g] = make_int4(hi[0] - lo[0], hi[1] - lo[1], hi[2] - lo[2], 0);
      gD[g] = make_int4(cell_c2(ix, ls), cell_c2(iy, ls), cell_c2(iz, ls), 0);
    }
  }
}

// groups sharing an expansion cell (same box, same level-(grid-1) cell) form
// a run; gA.w = 1 marks a run's first group, gD.w receives the run index and
// runhead[run] the run's first group.
// The flags are scanned over the whole capacity, so slots past the count get 0.
__global__ void run_flag_kernel(int cap, const int* __restrict__ pngroup, int4* __restrict__ gA,
                                const int4* __restrict__ gD, int* __restrict__ flag) {
  const int ngroup = *pngroup;
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < cap; g += gridDim.x * blockDim.x) {
    if (g >= ngroup) {
      flag[g] = 0;
      continue;
    }
    bool first = g == 0;
    if (!first) {
      const int4 a = gD[g], b = gD[g - 1];
      first = a.x != b.x || a.y != b.y || a.z != b.z || gA[g].z != gA[g - 1].z;
    }
    gA[g].w = first ? 1 : 0;
    flag[g] = first ? 1 : 0;
  }
}

__global__ void run_index_kernel(const int* __restrict__ pngroup, const int* __restrict__ flag,
                                 const int* __restrict__ excl, int4* __restrict__ gD, int* __restrict__ runhead) {
  const int ngroup = *pngroup;
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < ngroup; g += gridDim.x * blockDim.x) {
    gD[g].w = excl[g] + flag[g] - 1;
    if (flag[g] && NB_IN(excl[g], ngroup, 312)) runhead[excl[g]] = g;
  }
}

// Counts of a build whose buffers were sized beforehand (a reserved capacity):
// a count above its capacity sets the overflow status and both counts drop to
// zero, so every later kernel of the build and of the evaluation does nothing
// and no buffer is written past its end.  A built tree has at least one cell
// and one group, so zero counts (an overflowed build) set the status again
// when an evaluation checks them.
__global__ void cap_check_kernel(int* __restrict__ cnt, int cell_cap, int group_cap, unsigned* __restrict__ err) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  if (cnt[0] > cell_cap || cnt[1] > group_cap || cnt[0] <= 0 || cnt[1] <= 0) {
    atomicOr(err, NB_ST_OVERFLOW);
    cnt[0] = 0;
    cnt[1] = 0;
  }
}

// A position or mass that is not finite sets NB_ST_BADINPUT in `status` (the
// build then returns NBODY_EINVAL); the rest of the build runs on, since every
// index it derives from a position goes through the wrapped key.
__global__ void gather_kernel(const double* __restrict__ pos, const float* __restrict__ mass,
                              const uint32_t* __restrict__ perm, const uint16_t* __restrict__ sbox,
                              const int64_t* __restrict__ off, int64_t n, double* __restrict__ spos,
                              float* __restrict__ smass, unsigned* __restrict__ status) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    uint32_t j = NB_IDX(perm[i], (uint32_t)n, 313);
    bool bad = false;
    for (int d = 0; d < 3; d++) {
      double x = pos[d * n + j];
      bad |= !isfinite(x);
      x -= floor(x);  // wrap into [0,1)
      if (x >= 1.0) x = 0.0;
      spos[d * n + i] = x;
    }
    if (mass) {
      const float m = mass[j];
      bad |= !isfinite(m);
      smass[i] = m;
    } else {
      int b = sbox[i];
      smass[i] = (float)(1.0 / (double)(off[b + 1] - off[b]));
    }
    if (bad) atomicOr(status, NB_ST_BADINPUT);
  }
}

__global__ void sbox_kernel(const uint32_t* __restrict__ perm, const uint16_t* __restrict__ box_of,
                            int64_t n, uint16_t* __restrict__ sbox) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    sbox[i] = box_of[NB_IDX(perm[i], (uint32_t)n, 314)];
}

int gridn(int64_t n, int threads) {
  int64_t g = (n + threads - 1) / threads;
  if (g < 1) g = 1;
  if (g > 152 * 64) g = 152 * 64;
  return (int)g;
}

}  // namespace

// ---- host launchers --------------------------------------------------------
cudaError_t nb_gather(const double* pos, const float* mass, const uint32_t* perm, const uint16_t* box_of,
                      const int64_t* off, int64_t n, double* spos, float* smass, uint16_t* sbox,
                      unsigned* status, cudaStream_t s) {
  sbox_kernel<<<gridn(n, 256), 256, 0, s>>>(perm, box_of, n, sbox);
  gather_kernel<<<gridn(n, 256), 256, 0, s>>>(pos, mass, perm, sbox, off, n, spos, smass, status);
  nb_launch_counter += 2;
  return cudaGetLastError();
}

cudaError_t nb_count_cells(const uint64_t* skeys, const uint16_t* sbox, const int64_t* off, int64_t n,
                           int n_leaf, int lmax, int* ccount, int8_t* l0, cudaStream_t s) {
  BuildArgs a{skeys, sbox, off, n, n_leaf, lmax};
  count_cells_kernel<<<gridn(n, 256), 256, 0, s>>>(a, ccount, l0);
  nb_launch_counter += 1;
  return cudaGetLastError();
}

cudaError_t nb_cap_check(int* cnt, int cell_cap, int group_cap, unsigned* err, cudaStream_t s) {
  cap_check_kernel<<<1, 32, 0, s>>>(cnt, cell_cap, group_cap, err);
  nb_launch_counter += 1;
  return cudaGetLastError();
}

cudaError_t nb_emit_cells(const uint64_t* skeys, const uint16_t* sbox, const int64_t* off, int64_t n,
                          int n_leaf, int lmax, const int* ccount, const int* coff, const int8_t* l0,
                          const int* pncell, uint8_t* plevel, int* pstart, int* pcount, int* pparent,
                          cudaStream_t s) {
  BuildArgs a{skeys, sbox, off, n, n_leaf, lmax};
  emit_cells_kernel<<<gridn(n, 256), 256, 0, s>>>(a, ccount, coff, l0, pncell, plevel, pstart, pcount,
                                                  pparent);
  nb_launch_counter += 1;
  return cudaGetLastError();
}

cudaError_t nb_bfs_cells(const uint64_t* skeys, const uint16_t* sbox, int64_t n, int ncell, const int* pncell,
                         const uint32_t* bfs2pre, int* pre2bfs, const uint8_t* plevel, const int* pstart,
                         const int* pcount, const int* pparent, int4* cA, int4* cB, uint64_t* ckey,
                         uint16_t* cbox, cudaStream_t s) {
  BuildArgs a{skeys, sbox, nullptr, n, 0, 0};
  bfs_fill_kernel<<<gridn(ncell, 256), 256, 0, s>>>(a, pncell, bfs2pre, pre2bfs);
  bfs_cells_kernel<<<gridn(ncell, 256), 256, 0, s>>>(a, pncell, bfs2pre, pre2bfs, plevel, pstart, pcount,
                                                     pparent, cA, cB, ckey, cbox);
  children_kernel<<<gridn(ncell, 256), 256, 0, s>>>(pncell, cB);
  nchild_kernel<<<gridn(ncell, 256), 256, 0, s>>>(pncell, cA, cB);
  nb_launch_counter += 4;
  return cudaGetLastError();
}

cudaError_t nb_hash_build(int ncell, const int* pncell, const uint64_t* ckey, const uint16_t* cbox, int* hval,
                          uint64_t cap, unsigned* err, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(hval, 0xff, sizeof(int) * cap, s);
  if (e) return e;
  hash_insert_kernel<<<gridn(ncell, 256), 256, 0, s>>>(pncell, ckey, cbox, hval, cap - 1, err);
  nb_launch_counter += 1;
  return cudaGetLastError();
}

cudaError_t nb_hash_lookup(const uint64_t* q, int64_t nq, int box, const int* hval, const uint64_t* ckey,
                           const uint16_t* cbox, uint64_t cap, int* out, cudaStream_t s) {
  hash_lookup_kernel<<<gridn(nq, 256), 256, 0, s>>>(q, nq, box, hval, ckey, cbox, cap - 1, out);
  nb_launch_counter += 1;
  return cudaGetLastError();
}

cudaError_t nb_leaves(int ncell, const int* pncell, const int4* cA, const int4* cB, const double* spos,
                      const float* smass, int64_t n, int* sleaf, void* src, bool fp64, cudaStream_t s) {
  if (fp64)
    leaf_kernel<double><<<gridn(ncell, 128), 128, 0, s>>>(pncell, cA, cB, spos, smass, n, sleaf,
                                                          (dbl4*)src);
  else
    leaf_kernel<float><<<gridn(ncell, 128), 128, 0, s>>>(pncell, cA, cB, spos, smass, n, sleaf,
                                                         (float4*)src);
  nb_launch_counter += 1;
  return cudaGetLastError();
}

cudaError_t nb_group_runs(int ngroup, const int* pngroup, int4* gA, int4* gD, int* flag, int* excl, int* total,
                          int* tmp, int* runhead, cudaStream_t s) {
  run_flag_kernel<<<gridn(ngroup, 256), 256, 0, s>>>(ngroup, pngroup, gA, gD, flag);
  nb_launch_counter += 1;
  cudaError_t e = nb_exclusive_scan_i32(flag, excl, ngroup, total, tmp, s);
  if (e) return e;
  run_index_kernel<<<gridn(ngroup, 256), 256, 0, s>>>(pngroup, flag, excl, gD, runhead);
  nb_launch_counter += 1;
  return cudaGetLastError();
}

cudaError_t nb_group_flags(const uint64_t* skeys, const uint16_t* sbox, const int64_t* off, int64_t n,
                           int ls, int n_group, int* flag, cudaStream_t s) {
  BuildArgs a{skeys, sbox, off, n, 0, 0};
  group_flag_kernel<<<gridn(n, 256), 256, 0, s>>>(a, ls, n_group, flag);
  nb_launch_counter += 1;
  return cudaGetLastError();
}

cudaError_t nb_group_info(const uint64_t* skeys, const uint16_t* sbox, int64_t n, int ngroup, const int* pngroup,
                          int ls, const int* flag, const int* gid, int* gstart, const double* spos, int4* gA,
                          int4* gB, int4* gC, int4* gD, cudaStream_t s) {
  BuildArgs a{skeys, sbox, nullptr, n, 0, 0};
  group_start_kernel<<<gridn(n, 256), 256, 0, s>>>(n, flag, gid, pngroup, gstart);
  group_info_kernel<<<gridn((int64_t)ngroup * 32, 256), 256, 0, s>>>(a, pngroup, ls, gstart, spos, gA, gB,
                                                                      gC, gD);
  nb_launch_counter += 2;
  return cudaGetLastError();
}

// fault word of the debug build's bounds checks in this unit (debug build only)
NB_DBG_EXPORT(build)
