// Morton keys and the onesweep LSD radix sort (Sec. 2.1: each particle gets a
// Morton-order key; sorting by key is the spatial decomposition).
//
// Sort: one upsweep pass builds the digit histograms of every 8-bit digit at
// once; then each digit pass is a single sweep in which a tile ranks its keys
// stably (peer masks from ballots + per-warp counters), publishes its per-digit counts and
// obtains its exclusive prefix by decoupled look-back over earlier tiles
// (bounded waits: a wait that runs out sets a status bit and the pass
// completes with the flag raised instead of hanging).
#include <mutex>

#include "common.cuh"

namespace {

constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kItems = 16;                        // keys per thread
constexpr int kTile = kSortThreads * kItems;      // 4096 keys per tile
constexpr uint32_t kFlagAgg = 1u << 30;
constexpr uint32_t kFlagInc = 2u << 30;
constexpr uint32_t kValMask = (1u << 30) - 1;

__global__ void keys_kernel(const double* __restrict__ pos, int64_t n, uint64_t* __restrict__ keys,
                            uint32_t* __restrict__ vals) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    uint32_t qx = quant21(pos[i]), qy = quant21(pos[n + i]), qz = quant21(pos[2 * n + i]);
    keys[i] = spread3(qx) | (spread3(qy) << 1) | (spread3(qz) << 2);
    vals[i] = (uint32_t)i;
  }
}

// keys_kernel for the allocation-free sort, which has no gather pass to
// validate the positions: a coordinate that is not finite sets the
// bad-input bit of *err (the build's gather does the same for its own path).
__global__ void keys_checked_kernel(const double* __restrict__ pos, int64_t n, uint64_t* __restrict__ keys,
                                    uint32_t* __restrict__ vals, unsigned* __restrict__ err) {
  bool bad = false;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double x = pos[i], y = pos[n + i], z = pos[2 * n + i];
    bad |= !(isfinite(x) && isfinite(y) && isfinite(z));
    uint32_t qx = quant21(x), qy = quant21(y), qz = quant21(z);
    keys[i] = spread3(qx) | (spread3(qy) << 1) | (spread3(qz) << 2);
    vals[i] = (uint32_t)i;
  }
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(err, NB_ST_BADINPUT);
}

__global__ void box_ids_kernel(const int64_t* __restrict__ off, int nbox, uint16_t* __restrict__ box_of) {
  for (int b = blockIdx.y; b < nbox; b += gridDim.y) {
    int64_t s = off[b], e = off[b + 1];
    for (int64_t i = s + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < e;
         i += (int64_t)gridDim.x * blockDim.x)
      box_of[i] = (uint16_t)b;
  }
}

// digit of an element for pass `pass`: key bits for pass < nkp, else box id bits
struct DigitFn {
  int nkp;                       // key passes
  const uint16_t* box_of_orig;   // box id by original index
  __device__ __forceinline__ uint32_t operator()(uint64_t k, uint32_t v, int pass) const {
    if (pass < nkp) return (uint32_t)(k >> (8 * pass)) & 255u;
    return (uint32_t)(box_of_orig[v] >> (8 * (pass - nkp))) & 255u;
  }
};

__global__ void upsweep_kernel(const uint64_t* __restrict__ keys, const uint32_t* __restrict__ vals,
                               int64_t n, DigitFn dig, int npass, uint32_t* __restrict__ hist) {
  __shared__ uint32_t h[16][256];
  for (int t = threadIdx.x; t < 16 * 256; t += blockDim.x) (&h[0][0])[t] = 0;
  __syncthreads();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    uint64_t k = keys[i];
    uint32_t v = vals[i];
    for (int p = 0; p < npass; p++) atomicAdd(&h[p][dig(k, v, p)], 1u);
  }
  __syncthreads();
  for (int t = threadIdx.x; t < npass * 256; t += blockDim.x) {
    uint32_t c = (&h[0][0])[t];
    if (c) atomicAdd(&hist[t], c);
  }
}

// exclusive scan of each pass's 256-bin histogram in place (one block per pass)
__global__ void hist_scan_kernel(uint32_t* hist) {
  __shared__ uint32_t s[256];
  uint32_t* h = hist + blockIdx.x * 256;
  int t = threadIdx.x;
  s[t] = h[t];
  __syncthreads();
  for (int o = 1; o < 256; o <<= 1) {
    uint32_t v = t >= o ? s[t - o] : 0u;
    __syncthreads();
    s[t] += v;
    __syncthreads();
  }
  h[t] = s[t] - h[t];
}

// The lanes of the warp holding the same valid digit as this lane (d < 256;
// an invalid lane's mask is not used): eight ballots, one per digit bit,
// intersected, and the ballot of the valid lanes.  On GB300 this ranks a
// tile's keys 12 % faster than match.any (2.80 -> 2.46 ms for the eight
// passes over 16.8M keys).
__device__ __forceinline__ uint32_t digit_peers(uint32_t d) {
  uint32_t peers = __ballot_sync(0xffffffffu, d < 256u);
#pragma unroll
  for (int b = 0; b < 8; b++) {
    const uint32_t bal = __ballot_sync(0xffffffffu, (d >> b) & 1u);
    peers &= ((d >> b) & 1u) ? bal : ~bal;
  }
  return peers;
}

__device__ __forceinline__ uint32_t ld_volatile(const uint32_t* p) {
  return *(const volatile uint32_t*)p;
}
__device__ __forceinline__ void st_volatile(uint32_t* p, uint32_t v) { *(volatile uint32_t*)p = v; }

// Decoupled look-back of one digit: the exclusive prefix of this tile from
// the status words (flag | count) of the tiles before it.  The words of
// kLookback predecessors are loaded at once, so a walk back over many tiles
// that have published only their aggregates costs one memory latency per
// kLookback tiles instead of one per tile.  A predecessor that has published
// nothing yet is waited for (bounded: the wait sets NB_ST_TIMEOUT in *err and
// gives up).
constexpr int kLookback = 8;
__device__ __forceinline__ uint32_t lookback(const uint32_t* __restrict__ status, int tile, int dd,
                                             unsigned* __restrict__ err) {
  uint32_t prefix = 0;
  int t = tile - 1, spins = 0;
  while (t >= 0) {
    uint32_t sv[kLookback];
#pragma unroll
    for (int q = 0; q < kLookback; q++) sv[q] = t - q >= 0 ? ld_volatile(status + (int64_t)(t - q) * 256 + dd) : kFlagInc;
    int used = kLookback;
    bool done = false;
#pragma unroll
    for (int q = 0; q < kLookback; q++) {
      if (done || used < kLookback) continue;
      if ((sv[q] & ~kValMask) == 0u) {
        used = q;  // not published yet: wait for it from here
      } else {
        prefix += sv[q] & kValMask;
        if (sv[q] & kFlagInc) done = true;
      }
    }
    if (done) break;
    if (used < kLookback) {
      t -= used;
      if (++spins > NB_SPIN_LIMIT) {
        atomicOr(err, NB_ST_TIMEOUT);
        break;
      }
    } else {
      t -= kLookback;
    }
  }
  return prefix;
}

__global__ void __launch_bounds__(kSortThreads)
onesweep_kernel(const uint64_t* __restrict__ kin, const uint32_t* __restrict__ vin,
                uint64_t* __restrict__ kout, uint32_t* __restrict__ vout, int64_t n, DigitFn dig,
                int pass, const uint32_t* __restrict__ base, uint32_t* __restrict__ status,
                uint32_t* __restrict__ tile_ctr, unsigned* __restrict__ err) {
  __shared__ uint32_t s_cnt[kSortWarps][256];
  __shared__ uint32_t s_excl[256];
  __shared__ uint32_t s_tstart[256];  // start of each digit in the tile's digit-sorted order
  __shared__ uint32_t s_wsum[kSortWarps];
  __shared__ uint64_t s_key[kTile];
  __shared__ uint32_t s_val[kTile];
  __shared__ uint8_t s_dig[kTile];
  __shared__ int s_tile;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) s_tile = (int)atomicAdd(tile_ctr, 1u);
  for (int t = threadIdx.x; t < kSortWarps * 256; t += kSortThreads) (&s_cnt[0][0])[t] = 0;
  __syncthreads();
  const int tile = s_tile;
  const int64_t wbase = (int64_t)tile * kTile + warp * (32 * kItems);
  uint64_t k[kItems];
  uint32_t v[kItems], d[kItems], rk[kItems];
  const uint32_t lt = (1u << lane) - 1u;
#pragma unroll
  for (int r = 0; r < kItems; r++) {
    int64_t i = wbase + r * 32 + lane;
    bool ok = i < n;
    k[r] = ok ? kin[i] : 0ull;
    v[r] = ok ? vin[i] : 0u;
    d[r] = ok ? dig(k[r], v[r], pass) : 256u;
  }
#pragma unroll
  for (int r = 0; r < kItems; r++) {
    const uint32_t peers = digit_peers(d[r]);
    uint32_t cur = d[r] < 256u ? s_cnt[warp][d[r]] : 0u;
    rk[r] = cur + __popc(peers & lt);
    __syncwarp();
    int leader = 31 - __clz(peers);
    if (lane == leader && d[r] < 256u) s_cnt[warp][d[r]] = cur + __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  {
    const int dd = threadIdx.x;  // one thread per digit
    uint32_t run = 0;
    for (int w = 0; w < kSortWarps; w++) {
      uint32_t c = s_cnt[w][dd];
      s_cnt[w][dd] = run;
      run += c;
    }
    // exclusive scan of the tile's digit counts over the 256 digits
    uint32_t x = run;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) s_wsum[warp] = x;
    __syncthreads();
    uint32_t wpre = 0;
    for (int w = 0; w < warp; w++) wpre += s_wsum[w];
    s_tstart[dd] = wpre + x - run;
    uint32_t* my = status + (int64_t)tile * 256 + dd;
    uint32_t prefix = 0;
    if (tile == 0) {
      st_volatile(my, kFlagInc | run);
    } else {
      st_volatile(my, kFlagAgg | run);
      prefix = lookback(status, tile, dd, err);
      __threadfence();
      st_volatile(my, kFlagInc | (prefix + run));
    }
    s_excl[dd] = base[dd] + prefix;
  }
  __syncthreads();
  // stage the tile in digit order, then write each digit's run contiguously
#pragma unroll
  for (int r = 0; r < kItems; r++) {
    if (d[r] < 256u && NB_IN(s_tstart[d[r]] + s_cnt[warp][d[r]] + rk[r], kTile, 202)) {
      const uint32_t lp = s_tstart[d[r]] + s_cnt[warp][d[r]] + rk[r];
      s_key[lp] = k[r];
      s_val[lp] = v[r];
      s_dig[lp] = (uint8_t)d[r];
    }
  }
  __syncthreads();
  const int64_t t0 = (int64_t)tile * kTile;
  const int cnt = (int)min((int64_t)kTile, n - t0);
  for (int e = threadIdx.x; e < cnt; e += kSortThreads) {
    const uint32_t dd = s_dig[e];
    const uint32_t dst = s_excl[dd] + ((uint32_t)e - s_tstart[dd]);
    if (!NB_IN(dst, n, 201)) continue;
    kout[dst] = s_key[e];
    vout[dst] = s_val[e];
  }
}

// single-pass stable sort by an 8-bit digit array; values are indices
__global__ void __launch_bounds__(kSortThreads)
digit_sweep_kernel(const uint8_t* __restrict__ digit, int64_t n, const uint32_t* __restrict__ base,
                   uint32_t* __restrict__ status, uint32_t* __restrict__ tile_ctr,
                   uint32_t* __restrict__ out, unsigned* __restrict__ err) {
  __shared__ uint32_t s_cnt[kSortWarps][256];
  __shared__ uint32_t s_excl[256];
  __shared__ int s_tile;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) s_tile = (int)atomicAdd(tile_ctr, 1u);
  for (int t = threadIdx.x; t < kSortWarps * 256; t += kSortThreads) (&s_cnt[0][0])[t] = 0;
  __syncthreads();
  const int tile = s_tile;
  const int64_t wbase = (int64_t)tile * kTile + warp * (32 * kItems);
  uint32_t d[kItems], rk[kItems];
  const uint32_t lt = (1u << lane) - 1u;
#pragma unroll
  for (int r = 0; r < kItems; r++) {
    int64_t i = wbase + r * 32 + lane;
    d[r] = i < n ? (uint32_t)digit[i] : 256u;
  }
#pragma unroll
  for (int r = 0; r < kItems; r++) {
    const uint32_t peers = digit_peers(d[r]);
    uint32_t cur = d[r] < 256u ? s_cnt[warp][d[r]] : 0u;
    rk[r] = cur + __popc(peers & lt);
    __syncwarp();
    int leader = 31 - __clz(peers);
    if (lane == leader && d[r] < 256u) s_cnt[warp][d[r]] = cur + __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  {
    const int dd = threadIdx.x;
    uint32_t run = 0;
    for (int w = 0; w < kSortWarps; w++) {
      uint32_t c = s_cnt[w][dd];
      s_cnt[w][dd] = run;
      run += c;
    }
    uint32_t* my = status + (int64_t)tile * 256 + dd;
    uint32_t prefix = 0;
    if (tile == 0) {
      st_volatile(my, kFlagInc | run);
    } else {
      st_volatile(my, kFlagAgg | run);
      prefix = lookback(status, tile, dd, err);
      __threadfence();
      st_volatile(my, kFlagInc | (prefix + run));
    }
    s_excl[dd] = base[dd] + prefix;
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < kItems; r++) {
    if (d[r] < 256u && NB_IN(s_excl[d[r]] + s_cnt[warp][d[r]] + rk[r], n, 203)) {
      int64_t i = wbase + r * 32 + lane;
      out[s_excl[d[r]] + s_cnt[warp][d[r]] + rk[r]] = (uint32_t)i;
    }
  }
}

__global__ void digit_hist_kernel(const uint8_t* __restrict__ digit, int64_t n, uint32_t* __restrict__ hist) {
  __shared__ uint32_t h[256];
  for (int t = threadIdx.x; t < 256; t += blockDim.x) h[t] = 0;
  __syncthreads();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(&h[digit[i]], 1u);
  __syncthreads();
  for (int t = threadIdx.x; t < 256; t += blockDim.x)
    if (h[t]) atomicAdd(&hist[t], h[t]);
}

// ---- exclusive scan of int32 (three kernels) ------------------------------------
constexpr int kScanThreads = 512;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ __forceinline__ int block_excl_scan(int v, int* smem_warp, int* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) smem_warp[warp] = x;
  __syncthreads();
  if (warp == 0) {
    int nw = blockDim.x >> 5;
    int w = lane < nw ? smem_warp[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    if (lane < nw) smem_warp[lane] = w;
  }
  __syncthreads();
  int prev = warp > 0 ? smem_warp[warp - 1] : 0;
  *total = smem_warp[(blockDim.x >> 5) - 1];
  __syncthreads();
  return prev + x - v;
}

__global__ void scan_reduce_kernel(const int* __restrict__ in, int64_t n, int* __restrict__ sums) {
  __shared__ int sw[32];
  int64_t b0 = (int64_t)blockIdx.x * kScanTile;
  int acc = 0;
  for (int r = 0; r < kScanItems; r++) {
    int64_t i = b0 + (int64_t)r * kScanThreads + threadIdx.x;
    if (i < n) acc += in[i];
  }
  int tot;
  block_excl_scan(acc, sw, &tot);
  if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

__global__ void scan_sums_kernel(int* sums, int64_t nb, int* total) {
  __shared__ int sw[32];
  int carry = 0;
  for (int64_t base = 0; base < nb; base += blockDim.x) {
    int64_t i = base + threadIdx.x;
    int v = i < nb ? sums[i] : 0;
    int tot;
    int ex = block_excl_scan(v, sw, &tot);
    if (i < nb) sums[i] = carry + ex;
    carry += tot;
  }
  if (threadIdx.x == 0 && total) *total = carry;
}

__global__ void scan_apply_kernel(const int* __restrict__ in, int* __restrict__ out, int64_t n,
                                  const int* __restrict__ sums) {
  __shared__ int sw[32];
  __shared__ int s_carry;
  int64_t b0 = (int64_t)blockIdx.x * kScanTile;
  if (threadIdx.x == 0) s_carry = sums[blockIdx.x];
  __syncthreads();
  // blocked: thread t handles items b0 + t*kScanItems .. +kScanItems
  int v[kScanItems];
  int loc = 0;
  for (int r = 0; r < kScanItems; r++) {
    int64_t i = b0 + (int64_t)threadIdx.x * kScanItems + r;
    v[r] = i < n ? in[i] : 0;
    loc += v[r];
  }
  int tot;
  int ex = block_excl_scan(loc, sw, &tot);
  int run = s_carry + ex;
  for (int r = 0; r < kScanItems; r++) {
    int64_t i = b0 + (int64_t)threadIdx.x * kScanItems + r;
    if (i < n) out[i] = run;
    run += v[r];
  }
}

int grid_for(int64_t n, int threads, int cap = 152 * 32) {
  int64_t g = (n + threads - 1) / threads;
  if (g < 1) g = 1;
  if (g > cap) g = cap;
  return (int)g;
}

}  // namespace

thread_local long long nb_launch_counter = 0;

int64_t nb_sort_tiles(int64_t n) { return (n + kTile - 1) / kTile; }

cudaError_t nb_launch_keys(const double* pos, int64_t n, int64_t, uint64_t* keys, uint32_t* vals,
                           cudaStream_t s) {
  keys_kernel<<<grid_for(n, 256), 256, 0, s>>>(pos, n, keys, vals);
  nb_launch_counter += 1;
  return cudaGetLastError();
}

cudaError_t nb_launch_box_ids(const int64_t* off, int nbox, int64_t n, uint16_t* box_of,
                              cudaStream_t s) {
  dim3 g(grid_for(n / (nbox > 0 ? nbox : 1) + 1, 256, 256), nbox < 65535 ? nbox : 65535);
  box_ids_kernel<<<g, 256, 0, s>>>(off, nbox, box_of);
  nb_launch_counter += 1;
  return cudaGetLastError();
}

int nb_radix_passes(int bit1, int nbox) { return (bit1 + 7) / 8 + (nbox > 1 ? (nbox > 256 ? 2 : 1) : 0); }

cudaError_t nb_radix_sort(uint64_t* keys, uint32_t* vals, int64_t n, int bit1,
                          const uint16_t* box_of_orig, int nbox, SortScratch* sc, cudaStream_t s,
                          int* result_in_alt) {
  int nkp = (bit1 + 7) / 8;
  int np = nb_radix_passes(bit1, box_of_orig ? nbox : 1);
  DigitFn dig{nkp, box_of_orig};
  int64_t tiles = nb_sort_tiles(n);
  if (tiles * np > sc->tiles_cap || np > 16) return cudaErrorInvalidValue;
  cudaError_t e;
  if ((e = cudaMemsetAsync(sc->hist, 0, sizeof(uint32_t) * 256 * np, s))) return e;
  if ((e = cudaMemsetAsync(sc->status, 0, sizeof(uint32_t) * 256 * tiles * np, s))) return e;
  if ((e = cudaMemsetAsync(sc->tile_ctr, 0, sizeof(uint32_t) * np, s))) return e;
  upsweep_kernel<<<grid_for(n, 256, 152 * 8), 256, 0, s>>>(keys, vals, n, dig, np, sc->hist);
  hist_scan_kernel<<<np, 256, 0, s>>>(sc->hist);
  uint64_t* ka = keys;
  uint32_t* va = vals;
  uint64_t* kb = sc->keys_alt;
  uint32_t* vb = sc->vals_alt;
  for (int p = 0; p < np; p++) {
    onesweep_kernel<<<(unsigned)tiles, kSortThreads, 0, s>>>(
        ka, va, kb, vb, n, dig, p, sc->hist + 256 * p, sc->status + (int64_t)256 * tiles * p,
        sc->tile_ctr + p, sc->dstatus);
    uint64_t* tk = ka;
    ka = kb;
    kb = tk;
    uint32_t* tv = va;
    va = vb;
    vb = tv;
  }
  *result_in_alt = (np & 1);
  nb_launch_counter += 2 + np;
  return cudaGetLastError();
}

cudaError_t nb_sort_digit8(const uint8_t* digit, int64_t n, uint32_t* order_out, uint32_t* hist_out,
                           SortScratch* sc, cudaStream_t s) {
  int64_t tiles = nb_sort_tiles(n);
  if (tiles > sc->tiles_cap) return cudaErrorInvalidValue;
  cudaError_t e;
  if ((e = cudaMemsetAsync(hist_out, 0, sizeof(uint32_t) * 256, s))) return e;
  if ((e = cudaMemsetAsync(sc->status, 0, sizeof(uint32_t) * 256 * tiles, s))) return e;
  if ((e = cudaMemsetAsync(sc->tile_ctr, 0, sizeof(uint32_t), s))) return e;
  digit_hist_kernel<<<grid_for(n, 256, 152 * 4), 256, 0, s>>>(digit, n, hist_out);
  // scan into hist (scratch copy keeps hist_out as counts)
  if ((e = cudaMemcpyAsync(sc->hist, hist_out, sizeof(uint32_t) * 256, cudaMemcpyDeviceToDevice, s)))
    return e;
  hist_scan_kernel<<<1, 256, 0, s>>>(sc->hist);
  digit_sweep_kernel<<<(unsigned)tiles, kSortThreads, 0, s>>>(digit, n, sc->hist, sc->status,
                                                               sc->tile_ctr, order_out, sc->dstatus);
  nb_launch_counter += 3;
  return cudaGetLastError();
}

int64_t nb_scan_tmp_ints(int64_t n) { return (n + kScanTile - 1) / kScanTile + 1; }

cudaError_t nb_exclusive_scan_i32(const int* in, int* out, int64_t n, int* total_dev, int* tmp,
                                  cudaStream_t s) {
  int64_t nb = (n + kScanTile - 1) / kScanTile;
  if (nb < 1) nb = 1;
  scan_reduce_kernel<<<(unsigned)nb, kScanThreads, 0, s>>>(in, n, tmp);
  scan_sums_kernel<<<1, 1024, 0, s>>>(tmp, nb, total_dev);
  scan_apply_kernel<<<(unsigned)nb, kScanThreads, 0, s>>>(in, out, n, tmp);
  nb_launch_counter += 3;
  return cudaGetLastError();
}

// ---- allocation-free Morton sort --------------------------------------------
// Some callers cannot allocate device memory at run time: code that runs
// while another allocator owns (or caps) the device memory, loops that must
// not pay cudaMalloc's implicit synchronisation, or processes whose device
// footprint must be fixed after set-up.  nbody_sort_keys_noalloc serves them:
// it is the keys + onesweep sort of nbody_build_tree with every scratch
// buffer (the alternate key/value buffers, the histograms, the look-back
// status words and the error word) in the file-scope array below, sized for
// at most kNoAllocMaxN particles.  Every GPU that loads this library holds
// the array (about 14.7 MB) until the process exits.
namespace {
constexpr int64_t kNoAllocMaxN = (int64_t)1 << 20;
constexpr int64_t kNoAllocTiles = kNoAllocMaxN / kTile + 1;
constexpr int kNoAllocPasses = 8;  // 63 key bits, 8 bits per pass
struct NoAllocScratch {
  uint64_t keys_alt[kNoAllocMaxN];
  uint32_t vals_alt[kNoAllocMaxN];
  uint32_t hist[16 * 256];
  uint32_t status[kNoAllocPasses * 256 * kNoAllocTiles];
  uint32_t tile_ctr[16];
  unsigned err;
};
std::mutex g_noalloc_mutex;
NoAllocScratch* g_noalloc_ptr[64] = {};
}  // namespace

static __device__ __align__(256) NoAllocScratch g_noalloc_scratch;

extern "C" int nbody_sort_keys_noalloc(const double* pos_dev, int64_t n, uint64_t* keys_out_dev,
                                       uint32_t* perm_out_dev, nbody_stream_t stream) {
  if (!pos_dev || !keys_out_dev || !perm_out_dev || n <= 0) return NBODY_EINVAL;
  if (n > kNoAllocMaxN) return NBODY_ERANGE;
  cudaStream_t s = (cudaStream_t)stream;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return NBODY_ECUDA;
  NoAllocScratch* sc = nullptr;
  {
    // once per device, with that device current: the device address of the
    // array (its name in host code is only a host-side stand-in)
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_ptr[dev]) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
        cudaGetLastError();
        return NBODY_ECUDA;
      }
      g_noalloc_ptr[dev] = (NoAllocScratch*)p;
    }
    sc = g_noalloc_ptr[dev];
  }
  // the array keeps the previous call's contents: the error word is cleared
  // here, the histograms, status words and tile counters by the sort itself
  if (cudaMemsetAsync(&sc->err, 0, sizeof(unsigned), s) != cudaSuccess) return NBODY_ECUDA;
  keys_checked_kernel<<<grid_for(n, 256), 256, 0, s>>>(pos_dev, n, keys_out_dev, perm_out_dev, &sc->err);
  nb_launch_counter += 1;
  if (cudaGetLastError() != cudaSuccess) return NBODY_ECUDA;
  SortScratch ss;
  ss.keys_alt = sc->keys_alt;
  ss.vals_alt = sc->vals_alt;
  ss.hist = sc->hist;
  ss.status = sc->status;
  ss.tile_ctr = sc->tile_ctr;
  ss.tiles_cap = kNoAllocPasses * kNoAllocTiles;
  ss.dstatus = &sc->err;
  int alt = 0;
  if (nb_radix_sort(keys_out_dev, perm_out_dev, n, 63, nullptr, 1, &ss, s, &alt) != cudaSuccess)
    return NBODY_ECUDA;
  if (alt) return NBODY_ECUDA;  // an even number of passes ends in the output buffers
  unsigned err = 0;
  if (cudaMemcpyAsync(&err, &sc->err, sizeof(unsigned), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return NBODY_ECUDA;
  if (err & NB_ST_BADINPUT) return NBODY_EINVAL;
  if (err & NB_ST_TIMEOUT) return NBODY_ETIMEOUT;
  return NBODY_OK;
}

// fault word of the debug build's bounds checks in this unit (debug build only)
NB_DBG_EXPORT(sort)
