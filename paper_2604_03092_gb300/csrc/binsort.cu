// Tile binning and the device radix sorts.
//
// Binning (splat2d_bin_sort): every visible (view, surfel) record stands for
// one instance per tile of its tile rect, with key = (global tile) << 32 |
// FP32 depth bits and value = surfel index; the instances are ordered by key
// with ties in ascending surfel index (= record order within a view), i.e.
// exactly a stable sort of the keys in record order.  It is done as a radix
// sort whose most significant digit is the whole tile index (count, scan,
// scatter into per-tile buckets) followed by a least-significant-digit radix
// sort of each bucket's depth bits in shared memory.
//
// splat2d_sort_pairs: a general stable LSD radix sort of (u64 key, u32 value)
// pairs with 8-bit digits over the key bits in use.  Each pass is upsweep
// (per-block digit histograms) -> scan of the histograms -> downsweep (stable
// ranking of each 2048-key tile with warp-level match, then scatter); blocks
// own contiguous, ordered slices, so equal keys keep their input order.
#include <cuda_runtime.h>

#include "splat2d_internal.cuh"

namespace s2d {

// ---------------------------------------------------------------------------
// Binning by tile: count -> scan -> scatter -> per-tile sort
//
// The first radix digit of the (tile, depth) key is the whole tile index: a
// counting pass gives each tile's instance count (warp-aggregated atomics:
// neighbouring surfels of a keyframe land in the same tiles), an exclusive
// scan gives each tile's [start, end) range directly, and a scatter pass
// drops every instance into its tile's bucket as a 64-bit composite
// (depth bits << 32 | surfel index).  Then each tile's bucket is sorted on
// its own by an LSD radix sort of the depth bits in shared memory (in global
// memory for the rare buckets too large for shared memory), and equal depth
// bits are put in ascending surfel index.  The result is the (tile, depth)
// order with ties in surfel order -- the stable sort of the instance keys.
// ---------------------------------------------------------------------------
struct TileBinArgs {
  const uint32_t* ntiles;
  const float4* records;
  const DView* views;
  int32_t V;
  int64_t R;
  int32_t tile_w, tile_h;
  uint32_t* counts;  // per tile; the scan turns them into scatter cursors
  unsigned long long* bucket;
  const Header* hdr;
};

// Visit every (record, tile) instance; warp lanes hold consecutive records and
// walk their tile rects in step so equal tiles can be aggregated.
template <bool SCATTER>
__global__ void __launch_bounds__(256) k_tile_pass(const TileBinArgs A) {
  if (SCATTER && A.hdr->status != 0) return;
  const int lane = threadIdx.x & 31;
  const uint32_t lt_mask = (1u << lane) - 1u;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t r0 = (int64_t)blockIdx.x * blockDim.x; r0 < A.R; r0 += stride) {
    const int64_t r = r0 + threadIdx.x;
    const uint32_t nt = r < A.R ? __ldg(A.ntiles + r) : 0u;
    if (!__any_sync(0xffffffffu, nt != 0)) continue;
    int tx0 = 0, ty0 = 0, w = 1, tbase = 0, tilesx = 0;
    uint64_t comp = 0;
    if (nt) {
      const int v = find_view_by_record(A.views, A.V, r);
      const DView& vw = A.views[v];
      const float4 f4 = __ldg(A.records + r * REC_F4 + 4);
      const uint32_t q0 = __float_as_uint(f4.z), q1 = __float_as_uint(f4.w);
      tx0 = (int)(q0 & 0xffffu) / A.tile_w;
      ty0 = (int)(q0 >> 16) / A.tile_h;
      const int tx1 = (int)(q1 & 0xffffu) / A.tile_w;
      w = tx1 - tx0 + 1;
      tbase = vw.tile_base;
      tilesx = vw.tiles_x;
      comp = ((uint64_t)__float_as_uint(f4.y) << 32) | (uint64_t)(uint32_t)(vw.soff + (r - vw.rbase));
    }
    const uint32_t kmax = __reduce_max_sync(0xffffffffu, nt);
    for (uint32_t k = 0; k < kmax; k++) {
      const bool has = k < nt;
      const uint32_t t = has ? (uint32_t)(tbase + (ty0 + (int)k / w) * tilesx + tx0 + (int)k % w) : 0xffffffffu;
      const uint32_t peers = __match_any_sync(0xffffffffu, t);
      if (!has) continue;
      const int leader = __ffs(peers) - 1;
      if (!SCATTER) {
        if (lane == leader) atomicAdd(A.counts + t, (uint32_t)__popc(peers));
      } else {
        uint32_t base = 0;
        if (lane == leader) base = atomicAdd(A.counts + t, (uint32_t)__popc(peers));
        base = __shfl_sync(peers, base, leader);
        A.bucket[base + __popc(peers & lt_mask)] = comp;
      }
    }
  }
}

// One block: exclusive scan of the tile counts -> ranges, scatter cursors,
// total and the capacity check.
__global__ void __launch_bounds__(1024) k_tile_scan(uint32_t* __restrict__ counts, uint2* __restrict__ ranges,
                                                    int64_t T, Header* __restrict__ hdr, int64_t cap) {
  __shared__ unsigned long long s_w[32];
  __shared__ unsigned long long s_carry;
  if (threadIdx.x == 0) s_carry = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int64_t base = 0; base < T; base += 1024) {
    const int64_t i = base + threadIdx.x;
    const unsigned long long v = i < T ? counts[i] : 0ull;
    unsigned long long x = v;
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) s_w[wid] = x;
    __syncthreads();
    if (wid == 0) {
      unsigned long long w = s_w[lane];
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xffffffffu, w, o);
        if (lane >= o) w += y;
      }
      s_w[lane] = w;
    }
    __syncthreads();
    const unsigned long long incl = x + (wid > 0 ? s_w[wid - 1] : 0ull) + s_carry;
    const unsigned long long start = incl - v;
    if (i < T) {
      const bool fits = incl <= (unsigned long long)cap;
      ranges[i] = fits ? make_uint2((uint32_t)start, (uint32_t)incl) : make_uint2(0u, 0u);
      counts[i] = fits ? (uint32_t)start : 0u;
    }
    __syncthreads();
    if (threadIdx.x == 1023) s_carry = incl;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const unsigned long long total = s_carry;
    hdr->needed = total;
    if ((int64_t)total > cap) {
      hdr->status = SPLAT2D_ERR_CAPACITY;
      hdr->n_inst = 0;
    } else {
      hdr->n_inst = total;
    }
  }
}

// Stable LSD radix sort of `n` composite keys by their depth bits (high 32),
// 8 bits per pass, ping-ponging between a and b (generic pointers: shared or
// global memory), ranked per warp with match_any so that equal digits keep
// their order.  4 passes: the result ends in `a`.  Needs NWARPS*256 counters.
template <int NWARPS>
__device__ void block_sort_depth(unsigned long long* a, unsigned long long* b, int n, uint32_t* cnt) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const uint32_t lt_mask = (1u << lane) - 1u;
  const int per = (((n + NWARPS - 1) / NWARPS) + 31) & ~31;  // elements per warp, whole rounds
  const int lo = min(wid * per, n), hi = min(lo + per, n);
  for (int pass = 0; pass < 4; pass++) {
    const int shift = 32 + 8 * pass;
    unsigned long long* src = (pass & 1) ? b : a;
    unsigned long long* dst = (pass & 1) ? a : b;
    for (int i = threadIdx.x; i < NWARPS * 256; i += NWARPS * 32) cnt[i] = 0;
    __syncthreads();
    // per-warp digit counts
    for (int base = lo; base < hi; base += 32) {
      const int i = base + lane;
      const uint32_t d = i < hi ? (uint32_t)(src[i] >> shift) & 0xffu : 256u;
      const uint32_t peers = __match_any_sync(0xffffffffu, d);
      if (d < 256 && lane == __ffs(peers) - 1) cnt[wid * 256 + d] += __popc(peers);
      __syncwarp();
    }
    __syncthreads();
    // exclusive offsets, digit-major then warp
    if (threadIdx.x < 256) {
      uint32_t acc = 0;
      for (int w = 0; w < NWARPS; w++) {
        const uint32_t c = cnt[w * 256 + threadIdx.x];
        cnt[w * 256 + threadIdx.x] = acc;
        acc += c;
      }
      cnt[NWARPS * 256 + threadIdx.x] = acc;  // digit total
    }
    __syncthreads();
    if (threadIdx.x < 32) {
      // exclusive scan of the 256 digit totals, 8 per lane
      uint32_t v[8], s = 0;
      for (int k = 0; k < 8; k++) {
        v[k] = cnt[NWARPS * 256 + lane * 8 + k];
        s += v[k];
      }
      uint32_t x = s;
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
      }
      uint32_t run = x - s;
      for (int k = 0; k < 8; k++) {
        cnt[NWARPS * 256 + lane * 8 + k] = run;
        run += v[k];
      }
    }
    __syncthreads();
    if (threadIdx.x < 256) {
      const uint32_t dbase = cnt[NWARPS * 256 + threadIdx.x];
      for (int w = 0; w < NWARPS; w++) cnt[w * 256 + threadIdx.x] += dbase;
    }
    __syncthreads();
    // stable scatter
    for (int base = lo; base < hi; base += 32) {
      const int i = base + lane;
      const unsigned long long key = i < hi ? src[i] : 0ull;
      const uint32_t d = i < hi ? (uint32_t)(key >> shift) & 0xffu : 256u;
      const uint32_t peers = __match_any_sync(0xffffffffu, d);
      uint32_t pos = 0;
      if (d < 256) pos = cnt[wid * 256 + d];
      __syncwarp();
      if (d < 256) {
        if (lane == __ffs(peers) - 1) cnt[wid * 256 + d] = pos + __popc(peers);
        dst[pos + __popc(peers & lt_mask)] = key;
      }
      __syncwarp();
    }
    __syncthreads();
  }
  // equal depth bits: ascending surfel index (runs are short)
  for (int i = threadIdx.x; i < n; i += NWARPS * 32) {
    const uint32_t d = (uint32_t)(a[i] >> 32);
    const bool starts = (i == 0 || (uint32_t)(a[i - 1] >> 32) != d) && i + 1 < n && (uint32_t)(a[i + 1] >> 32) == d;
    if (!starts) continue;
    int e = i + 1;
    while (e + 1 < n && (uint32_t)(a[e + 1] >> 32) == d) e++;
    for (int x = i + 1; x <= e; x++) {
      const unsigned long long key = a[x];
      int y = x - 1;
      while (y >= i && a[y] > key) {
        a[y + 1] = a[y];
        y--;
      }
      a[y + 1] = key;
    }
  }
  __syncthreads();
}

constexpr int SEG_THREADS = 512;
constexpr int SEG_WARPS = SEG_THREADS / 32;
constexpr int SEG_SMEM_KEYS = 12288;  // keys per shared-memory bucket sort (two buffers)
constexpr size_t SEG_SMEM_BYTES = 2 * sizeof(unsigned long long) * SEG_SMEM_KEYS + sizeof(uint32_t) * (SEG_WARPS + 1) * 256;

struct SegArgs {
  const uint2* ranges;
  int64_t T;
  unsigned long long* bucket;   // scattered composites (sorted in place for the large buckets)
  unsigned long long* scratch;  // ping-pong space for the large buckets (same indexing as bucket)
  uint64_t* keys;               // out: (tile << 32) | depth bits
  uint32_t* vals;               // out: surfel index
  const Header* hdr;
  uint32_t* queue;              // work counter
};

__global__ void __launch_bounds__(SEG_THREADS) k_tile_sort(const SegArgs A) {
  extern __shared__ __align__(16) unsigned char smem[];
  unsigned long long* sa = reinterpret_cast<unsigned long long*>(smem);
  unsigned long long* sb = sa + SEG_SMEM_KEYS;
  uint32_t* cnt = reinterpret_cast<uint32_t*>(sb + SEG_SMEM_KEYS);
  __shared__ int s_t;
  if (A.hdr->status != 0) return;
  for (;;) {
    if (threadIdx.x == 0) s_t = (int)atomicAdd(A.queue, 1u);
    __syncthreads();
    const int t = s_t;
    __syncthreads();
    if (t >= A.T) break;
    const uint2 rg = A.ranges[t];
    const int n = (int)(rg.y - rg.x);
    if (n == 0) continue;
    unsigned long long* src;
    if (n <= SEG_SMEM_KEYS) {
      for (int i = threadIdx.x; i < n; i += SEG_THREADS) sa[i] = A.bucket[rg.x + i];
      __syncthreads();
      block_sort_depth<SEG_WARPS>(sa, sb, n, cnt);
      src = sa;
    } else {
      block_sort_depth<SEG_WARPS>(A.bucket + rg.x, A.scratch + rg.x, n, cnt);
      src = A.bucket + rg.x;
    }
    const uint64_t tile = (uint64_t)t << 32;
    for (int i = threadIdx.x; i < n; i += SEG_THREADS) {
      const unsigned long long key = src[i];
      A.keys[rg.x + i] = tile | (key >> 32);
      A.vals[rg.x + i] = (uint32_t)key;
    }
    __syncthreads();
  }
}

cudaError_t launch_bin_tiles(const Layout& L, const RastParams& P, char* ws, cudaStream_t st) {
  if (L.R <= 0 || L.T <= 0) return cudaSuccess;
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(k_tile_sort, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SEG_SMEM_BYTES);
    attr_set = true;
  }
  Header* hdr = reinterpret_cast<Header*>(ws + L.header);
  uint32_t* counts = reinterpret_cast<uint32_t*>(ws + L.tile_count);
  uint2* ranges = reinterpret_cast<uint2*>(ws + L.ranges);
  cudaError_t e = cudaMemsetAsync(counts, 0, sizeof(uint32_t) * (size_t)L.T, st);
  if (e != cudaSuccess) return e;
  TileBinArgs A;
  A.ntiles = reinterpret_cast<const uint32_t*>(ws + L.ntiles);
  A.records = reinterpret_cast<const float4*>(ws + L.records);
  A.views = reinterpret_cast<const DView*>(ws + L.views);
  A.V = L.V;
  A.R = L.R;
  A.tile_w = P.tile_w;
  A.tile_h = P.tile_h;
  A.counts = counts;
  A.bucket = reinterpret_cast<unsigned long long*>(ws + L.keys1);
  A.hdr = hdr;
  const int grid = (int)min64((L.R + 255) / 256, (int64_t)sm_count() * 16);
  k_tile_pass<false><<<grid, 256, 0, st>>>(A);
  count_launches(1);
  k_tile_scan<<<1, 1024, 0, st>>>(counts, ranges, L.T, hdr, L.cap);
  count_launches(1);
  k_tile_pass<true><<<grid, 256, 0, st>>>(A);
  count_launches(1);
  SegArgs S;
  S.ranges = ranges;
  S.T = L.T;
  S.bucket = A.bucket;
  S.scratch = reinterpret_cast<unsigned long long*>(ws + L.keys0);
  S.keys = reinterpret_cast<uint64_t*>(ws + L.keys0);
  S.vals = reinterpret_cast<uint32_t*>(ws + L.vals0);
  S.hdr = hdr;
  S.queue = reinterpret_cast<uint32_t*>(ws + L.tile_hist) + ORDER_BINS;
  e = cudaMemsetAsync(S.queue, 0, sizeof(uint32_t), st);
  if (e != cudaSuccess) return e;
  const int sgrid = (int)min64(L.T, (int64_t)sm_count());
  k_tile_sort<<<sgrid, SEG_THREADS, SEG_SMEM_BYTES, st>>>(S);
  count_launches(1);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// LSD radix sort
// ---------------------------------------------------------------------------
// Contiguous slice of the n keys owned by block b: whole 2048-key tiles.
__device__ __forceinline__ void sort_slice(int64_t n, int nb, int b, int64_t& lo, int64_t& hi) {
  const int64_t tiles = (n + SORT_TILE - 1) / SORT_TILE;
  const int64_t per = (tiles + nb - 1) / nb;
  lo = min64((int64_t)b * per * SORT_TILE, n);
  hi = min64(lo + per * SORT_TILE, n);
}

__global__ void __launch_bounds__(SORT_THREADS) k_sort_upsweep(const uint64_t* __restrict__ keys,
                                                               const unsigned long long* __restrict__ n_dev,
                                                               int64_t n_static, int shift,
                                                               uint32_t* __restrict__ hist) {
  __shared__ uint32_t s_h[8][256];
  const int64_t n = n_dev ? (int64_t)*n_dev : n_static;
  const int wid = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < 8 * 256; i += SORT_THREADS) (&s_h[0][0])[i] = 0;
  __syncthreads();
  int64_t lo, hi;
  sort_slice(n, gridDim.x, blockIdx.x, lo, hi);
  for (int64_t i = lo + threadIdx.x; i < hi; i += SORT_THREADS) {
    const uint32_t d = (uint32_t)(__ldg(keys + i) >> shift) & 0xffu;
    atomicAdd(&s_h[wid][d], 1u);
  }
  __syncthreads();
  uint32_t* totals = hist + 256 * (size_t)gridDim.x;
  for (int d = threadIdx.x; d < 256; d += SORT_THREADS) {
    uint32_t t = 0;
#pragma unroll
    for (int w = 0; w < 8; w++) t += s_h[w][d];
    hist[(size_t)d * gridDim.x + blockIdx.x] = t;
    if (t) atomicAdd(totals + d, t);
  }
}

// Exclusive scan over the digit-major histogram (256 x nb): block d scans row
// d (nb <= 1024 block counts) and adds the number of keys with smaller digits.
__global__ void __launch_bounds__(1024) k_sort_scan(uint32_t* __restrict__ hist, int nb) {
  __shared__ uint32_t s_w[32];
  const int d = blockIdx.x;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const uint32_t* totals = hist + 256 * (size_t)nb;
  // keys with a smaller digit
  uint32_t below = (threadIdx.x < (unsigned)d) ? totals[threadIdx.x] : 0u;
  for (int o = 16; o > 0; o >>= 1) below += __shfl_xor_sync(0xffffffffu, below, o);
  if (lane == 0) s_w[wid] = below;
  __syncthreads();
  uint32_t base = 0;
  for (int w = 0; w < 32; w++) base += s_w[w];
  __syncthreads();
  const int i = threadIdx.x;
  const uint32_t v = i < nb ? hist[(size_t)d * nb + i] : 0u;
  uint32_t x = v;
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_w[wid] = x;
  __syncthreads();
  uint32_t wpre = 0;
  for (int w = 0; w < wid; w++) wpre += s_w[w];
  if (i < nb) hist[(size_t)d * nb + i] = base + wpre + x - v;
}

// Stable scatter.  Warp w ranks keys [tile + 256 w, tile + 256 w + 256) in
// eight rounds of 32 (lane order within a round), so (warp, round, lane)
// order equals input order.
__global__ void __launch_bounds__(SORT_THREADS) k_sort_downsweep(
    const uint64_t* __restrict__ kin, const uint32_t* __restrict__ vin, uint64_t* __restrict__ kout,
    uint32_t* __restrict__ vout, const unsigned long long* __restrict__ n_dev, int64_t n_static, int shift,
    uint32_t* __restrict__ hist) {
  __shared__ uint32_t s_wcnt[8][256];  // per-warp digit counts, then warp prefixes
  __shared__ uint32_t s_run[256];      // running output offset per digit for this block
  __shared__ uint32_t s_tcnt[256];
  const int64_t n = n_dev ? (int64_t)*n_dev : n_static;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const uint32_t lt_mask = (1u << lane) - 1u;
  int64_t lo, hi;
  sort_slice(n, gridDim.x, blockIdx.x, lo, hi);
  for (int d = threadIdx.x; d < 256; d += SORT_THREADS) s_run[d] = hist[(size_t)d * gridDim.x + blockIdx.x];
  // the scan has consumed the digit totals: clear them for the next pass
  if (blockIdx.x == 0)
    for (int d = threadIdx.x; d < 256; d += SORT_THREADS) hist[256 * (size_t)gridDim.x + d] = 0u;
  for (int i = threadIdx.x; i < 8 * 256; i += SORT_THREADS) (&s_wcnt[0][0])[i] = 0;
  __syncthreads();
  for (int64_t tile = lo; tile < hi; tile += SORT_TILE) {
    uint64_t k[SORT_IPT];
    uint32_t val[SORT_IPT], dig[SORT_IPT], rank[SORT_IPT];
#pragma unroll
    for (int r = 0; r < SORT_IPT; r++) {
      const int64_t i = tile + wid * 256 + r * 32 + lane;
      const bool ok = i < hi;
      k[r] = ok ? kin[i] : 0ull;
      val[r] = ok ? vin[i] : 0u;
      dig[r] = ok ? (uint32_t)(k[r] >> shift) & 0xffu : 256u;
    }
#pragma unroll
    for (int r = 0; r < SORT_IPT; r++) {
      const uint32_t d = dig[r];
      const uint32_t peers = __match_any_sync(0xffffffffu, d);
      const uint32_t before = __popc(peers & lt_mask);
      const int leader = __ffs(peers) - 1;
      uint32_t base = 0;
      if (d < 256) base = s_wcnt[wid][d];
      __syncwarp();
      if (d < 256 && lane == leader) s_wcnt[wid][d] = base + __popc(peers);
      __syncwarp();
      rank[r] = base + before;
    }
    __syncthreads();
    // per digit: exclusive prefix over warps, and the tile total
    for (int d = threadIdx.x; d < 256; d += SORT_THREADS) {
      uint32_t acc = 0;
#pragma unroll
      for (int w = 0; w < 8; w++) {
        const uint32_t c = s_wcnt[w][d];
        s_wcnt[w][d] = acc;
        acc += c;
      }
      s_tcnt[d] = acc;
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < SORT_IPT; r++) {
      const uint32_t d = dig[r];
      if (d < 256) {
        const uint32_t pos = s_run[d] + s_wcnt[wid][d] + rank[r];
        kout[pos] = k[r];
        vout[pos] = val[r];
      }
    }
    __syncthreads();
    for (int d = threadIdx.x; d < 256; d += SORT_THREADS) {
      s_run[d] += s_tcnt[d];
#pragma unroll
      for (int w = 0; w < 8; w++) s_wcnt[w][d] = 0;
    }
    __syncthreads();
  }
}

cudaError_t launch_sort(uint64_t* keys0, uint32_t* vals0, uint64_t* keys1, uint32_t* vals1,
                        const unsigned long long* n_dev, int64_t n_max, int key_bits, uint32_t* hist,
                        int sort_blocks, int* final_buffer, cudaStream_t st) {
  *final_buffer = 0;
  if (n_max <= 0 || key_bits <= 0) return cudaSuccess;
  uint64_t* kb[2] = {keys0, keys1};
  uint32_t* vb[2] = {vals0, vals1};
  int cur = 0;
  for (int shift = 0; shift < key_bits; shift += 8) {
    k_sort_upsweep<<<sort_blocks, SORT_THREADS, 0, st>>>(kb[cur], n_dev, n_max, shift, hist);
    count_launches(1);
    k_sort_scan<<<256, 1024, 0, st>>>(hist, sort_blocks);
    count_launches(1);
    k_sort_downsweep<<<sort_blocks, SORT_THREADS, 0, st>>>(kb[cur], vb[cur], kb[cur ^ 1], vb[cur ^ 1], n_dev,
                                                           n_max, shift, hist);
    count_launches(1);
    cur ^= 1;
  }
  *final_buffer = cur;
  return cudaGetLastError();
}

// Work order for the persistent render kernels: tiles bucketed by
// floor(log2(list length)), longest first (a counting sort on the bucket).
__global__ void __launch_bounds__(256) k_order_hist(const uint2* __restrict__ ranges, int64_t T,
                                                    uint32_t* __restrict__ bins) {
  __shared__ uint32_t s_b[ORDER_BINS];
  for (int i = threadIdx.x; i < ORDER_BINS; i += blockDim.x) s_b[i] = 0;
  __syncthreads();
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < T; t += (int64_t)gridDim.x * blockDim.x) {
    const uint2 r = ranges[t];
    const uint32_t len = r.y - r.x;
    const int b = len ? 32 - __clz(len) : 0;  // 0..32, larger = longer
    atomicAdd(&s_b[ORDER_BINS - 1 - b], 1u);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < ORDER_BINS; i += blockDim.x)
    if (s_b[i]) atomicAdd(&bins[i], s_b[i]);
}

__global__ void k_order_scan(uint32_t* __restrict__ bins) {
  if (threadIdx.x == 0) {
    uint32_t acc = 0;
    for (int i = 0; i < ORDER_BINS; i++) {
      uint32_t c = bins[i];
      bins[i] = acc;
      acc += c;
    }
  }
}

__global__ void __launch_bounds__(256) k_order_scatter(const uint2* __restrict__ ranges, int64_t T,
                                                       uint32_t* __restrict__ bins, uint32_t* __restrict__ order) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < T; t += (int64_t)gridDim.x * blockDim.x) {
    const uint2 r = ranges[t];
    const uint32_t len = r.y - r.x;
    const int b = len ? 32 - __clz(len) : 0;
    const uint32_t pos = atomicAdd(&bins[ORDER_BINS - 1 - b], 1u);
    order[pos] = (uint32_t)t;
  }
}

cudaError_t launch_order(const Layout& L, char* ws, cudaStream_t st) {
  if (L.T <= 0) return cudaSuccess;
  const uint2* ranges = reinterpret_cast<const uint2*>(ws + L.ranges);
  uint32_t* bins = reinterpret_cast<uint32_t*>(ws + L.tile_hist);
  uint32_t* order = reinterpret_cast<uint32_t*>(ws + L.tile_order);
  cudaError_t e = cudaMemsetAsync(bins, 0, sizeof(uint32_t) * ORDER_BINS, st);
  if (e != cudaSuccess) return e;
  int g2 = (int)min64((L.T + 255) / 256, (int64_t)sm_count() * 4);
  if (g2 < 1) g2 = 1;
  k_order_hist<<<g2, 256, 0, st>>>(ranges, L.T, bins);
  count_launches(1);
  k_order_scan<<<1, 32, 0, st>>>(bins);
  count_launches(1);
  k_order_scatter<<<g2, 256, 0, st>>>(ranges, L.T, bins, order);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace s2d
