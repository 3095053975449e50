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
  const uint4* bins;  // per record: depth bits, rect x0 | y0 << 16, rect x1 | y1 << 16, tile count

  const DView* views;
  int32_t V;
  int64_t R;
  int32_t tile_w, tile_h;
  uint32_t* counts;   // per tile: instances (count pass) / next free bucket slot (scatter, from the scan)
  unsigned long long* bucket;
  int64_t cap;        // instance capacity (bucket length)
  Header* hdr;
};

// Visit every (record, tile) instance: the count pass adds them up per tile,
// the scatter pass puts each record's composite (depth bits << 32 | surfel)
// into its tiles' buckets.  Warp lanes hold consecutive records (neighbouring
// pixels of a keyframe) and walk their tile rects in step, so runs of lanes
// on one tile take one atomic.
// Steps of the scatter whose cursor atomics are in flight together.
constexpr int BIN_KB = 4;

template <bool SCATTER>
__global__ void __launch_bounds__(256) k_tile_bin(const TileBinArgs A) {
  if (SCATTER && A.hdr->status != 0) return;
  const int lane = threadIdx.x & 31;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  // this thread's records only increase: follow the owning view forward
  int v = find_view_by_record(A.views, A.V, min64((int64_t)blockIdx.x * blockDim.x + threadIdx.x, A.R - 1));
  for (int64_t r0 = (int64_t)blockIdx.x * blockDim.x; r0 < A.R; r0 += stride) {
    const int64_t r = r0 + threadIdx.x;
    // 16 contiguous bytes per record (the records themselves are 80 bytes
    // apart: reading their rects pulled most of each record from DRAM)
    const uint4 e = r < A.R ? __ldg(A.bins + r) : make_uint4(0u, 0u, 0u, 0u);
    const uint32_t nt = e.w;
    if (!__any_sync(0xffffffffu, nt != 0)) continue;
    // the rect's tiles in row-major order: t walks a row, then jumps to the
    // next row's first tile (no division per step)
    uint32_t t = 0, wrap = 0;
    int left = 0, w = 1;
    uint64_t comp = 0;
    if (nt) {
      while (v + 1 < A.V && __ldg(&A.views[v + 1].rbase) <= r) v++;
      const DView& vw = A.views[v];
      const uint32_t q0 = e.y, q1 = e.z;
      const int tx0 = (int)(q0 & 0xffffu) / A.tile_w, ty0 = (int)(q0 >> 16) / A.tile_h;
      w = (int)(q1 & 0xffffu) / A.tile_w - tx0 + 1;
      t = (uint32_t)(vw.tile_base + ty0 * vw.tiles_x + tx0);
      wrap = (uint32_t)(vw.tiles_x - w + 1);
      left = w;
      comp = ((uint64_t)e.x << 32) | (uint64_t)(uint32_t)(vw.soff + (r - vw.rbase));
    }
    const uint32_t kmax = __reduce_max_sync(0xffffffffu, nt);
    auto advance = [&]() {
      t += (--left == 0) ? wrap : 1u;
      left = left == 0 ? w : left;
    };
    if (!SCATTER) {
      for (uint32_t k = 0; k < kmax; k++, advance()) {
        const bool has = k < nt;
        const TileRun tr = tile_run(has ? t : 0xffffffffu, has, lane);
        if (tr.lead) atomicAdd(A.counts + t, tr.run);
      }
    } else {
      // the cursor atomics of BIN_KB steps are issued before any of their
      // results is used, so the warp waits on one L2 round trip per batch
      for (uint32_t k0 = 0; k0 < kmax; k0 += BIN_KB) {
        uint32_t base[BIN_KB];
        int leader[BIN_KB];
#pragma unroll
        for (int j = 0; j < BIN_KB; j++) {
          base[j] = 0u;
          leader[j] = -1;
          if (k0 + j < kmax) {
            const bool has = k0 + j < nt;
            const TileRun tr = tile_run(has ? t : 0xffffffffu, has, lane);
            if (tr.lead) base[j] = atomicAdd(A.counts + t, tr.run);
            leader[j] = has ? tr.leader : -1;
            advance();
          }
        }
#pragma unroll
        for (int j = 0; j < BIN_KB; j++) {
          if (k0 + j >= kmax) break;  // uniform across the warp
          const uint32_t b = __shfl_sync(0xffffffffu, base[j], leader[j] & 31);
          if (leader[j] >= 0 && s2d_check((int64_t)b + (lane - leader[j]) < A.cap, A.hdr))
            A.bucket[b + (uint32_t)(lane - leader[j])] = comp;
        }
      }
    }
  }
}

// Size classes of the per-tile bucket sorts (upper bounds, inclusive; longer
// buckets go with the last class).
constexpr int SORT_CLASSES = 6;
constexpr int SORT_CLASS_BOUND[SORT_CLASSES] = {1024, 2048, 4096, 6144, 8192, 12288};

__device__ __forceinline__ int sort_class(uint32_t n) {
  static_assert(SORT_CLASSES == 6, "one comparison per class bound");
  constexpr uint32_t b0 = SORT_CLASS_BOUND[0], b1 = SORT_CLASS_BOUND[1], b2 = SORT_CLASS_BOUND[2],
                     b3 = SORT_CLASS_BOUND[3], b4 = SORT_CLASS_BOUND[4];
  return n == 0 ? -1
                : (n <= b0 ? 0 : (n <= b1 ? 1 : (n <= b2 ? 2 : (n <= b3 ? 3 : (n <= b4 ? 4 : 5)))));
}

// One block: exclusive scan of the tile counts -> ranges, scatter cursors,
// total and the capacity check; every non-empty tile is appended to the list
// of its sort size class.  Each thread takes SCAN_ITEMS consecutive tiles per
// sweep, so a sweep covers 8192 tiles with one block-wide scan of the
// threads' sums (a 64-view batch of about 770 K tiles takes 95 sweeps).
constexpr int SCAN_ITEMS = 8;

__global__ void __launch_bounds__(1024) k_tile_scan(const uint32_t* __restrict__ counts,
                                                    uint32_t* __restrict__ cursors, uint2* __restrict__ ranges,
                                                    int64_t T, Header* __restrict__ hdr, int64_t cap,
                                                    uint32_t* __restrict__ class_list,
                                                    uint32_t* __restrict__ class_count) {
  __shared__ unsigned long long s_w[32];
  __shared__ unsigned long long s_carry;
  if (threadIdx.x == 0) s_carry = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const uint32_t lt_mask = (1u << lane) - 1u;
  for (int64_t base = 0; base < T; base += 1024 * SCAN_ITEMS) {
    const int64_t i0 = base + (int64_t)threadIdx.x * SCAN_ITEMS;
    uint32_t v[SCAN_ITEMS];
    unsigned long long sum = 0;
#pragma unroll
    for (int j = 0; j < SCAN_ITEMS; j++) {
      v[j] = i0 + j < T ? counts[i0 + j] : 0u;
      sum += v[j];
    }
    unsigned long long x = sum;
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
    unsigned long long incl = x - sum + (wid > 0 ? s_w[wid - 1] : 0ull) + s_carry;
#pragma unroll
    for (int j = 0; j < SCAN_ITEMS; j++) {
      const int64_t i = i0 + j;
      const unsigned long long start = incl;
      incl += v[j];
      const bool fits = incl <= (unsigned long long)cap;
      if (i < T) {
        ranges[i] = fits ? make_uint2((uint32_t)start, (uint32_t)incl) : make_uint2(0u, 0u);
        cursors[i] = fits ? (uint32_t)start : 0u;
      }
      // append the tile to its size class's list (order within a list is free)
      const int cls = (i < T && fits) ? sort_class(v[j]) : -1;
#pragma unroll
      for (int c = 0; c < SORT_CLASSES; c++) {
        const uint32_t m = __ballot_sync(0xffffffffu, cls == c);
        if (!m) continue;
        uint32_t at = 0;
        if (lane == 0) at = atomicAdd(&class_count[c], (uint32_t)__popc(m));
        at = __shfl_sync(0xffffffffu, at, 0);
        if (cls == c) class_list[(size_t)c * T + at + __popc(m & lt_mask)] = (uint32_t)i;
      }
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

// Number of bits needed to represent v (0 for v == 0).
__device__ __forceinline__ int bits_of(uint32_t v) { return v ? 32 - __clz(v) : 0; }

// Stable LSD radix sort of n composite keys (depth bits << 32 | surfel index)
// in place in `a` (b: scratch of the same size), 8-bit digits of
// key_of(x) = ((x >> 32) - dmin) << ishift | ((x & 0xffffffff) - imin) over
// `nbits` bits (ishift < 0: the depth part alone, key_of(x) = (x >> 32) - dmin); generic pointers (shared or global memory); ranked per warp
// with match_any so that equal digits keep their order.  `cnt` holds
// (NWARPS + 1) * 256 counters.  Returns with the result in `a`.
template <int NWARPS>
__device__ void block_radix_any(unsigned long long* a, unsigned long long* b, int n, uint32_t* cnt, uint32_t dmin,
                            uint32_t imin, int ishift, int nbits) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const uint32_t lt_mask = (1u << lane) - 1u;
  const int per = (((n + NWARPS - 1) / NWARPS) + 31) & ~31;  // elements per warp, whole rounds
  const int lo = min(wid * per, n), hi = min(lo + per, n);
  const int passes = (nbits + 7) >> 3;
  unsigned long long* src = a;
  unsigned long long* dst = b;
  auto digit = [&](unsigned long long x, int shift) -> uint32_t {
    const unsigned long long dk = (unsigned long long)((uint32_t)(x >> 32) - dmin);
    const unsigned long long k = ishift < 0 ? dk : ((dk << ishift) | (unsigned long long)((uint32_t)x - imin));
    return (uint32_t)(k >> shift) & 0xffu;
  };
  for (int pass = 0; pass < passes; pass++) {
    const int shift = 8 * pass;
    for (int i = threadIdx.x; i < NWARPS * 256; i += NWARPS * 32) cnt[i] = 0;
    __syncthreads();
    for (int base = lo; base < hi; base += 32) {
      const int i = base + lane;
      const uint32_t d = i < hi ? digit(src[i], shift) : 256u;
      const uint32_t peers = __match_any_sync(0xffffffffu, d);
      if (d < 256 && lane == __ffs(peers) - 1) cnt[wid * 256 + d] += __popc(peers);
      __syncwarp();
    }
    __syncthreads();
    if (threadIdx.x < 256) {
      uint32_t acc = 0;
      for (int w = 0; w < NWARPS; w++) {
        const uint32_t c = cnt[w * 256 + threadIdx.x];
        cnt[w * 256 + threadIdx.x] = acc;
        acc += c;
      }
      cnt[NWARPS * 256 + threadIdx.x] = acc;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
      uint32_t v[8], sum = 0;
      for (int k = 0; k < 8; k++) {
        v[k] = cnt[NWARPS * 256 + lane * 8 + k];
        sum += v[k];
      }
      uint32_t x = sum;
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
      }
      uint32_t run = x - sum;
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
    for (int base = lo; base < hi; base += 32) {
      const int i = base + lane;
      const unsigned long long key = i < hi ? src[i] : 0ull;
      const uint32_t d = i < hi ? digit(key, shift) : 256u;
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
    unsigned long long* tmp = src;
    src = dst;
    dst = tmp;
  }
  if (src != a) {
    for (int i = threadIdx.x; i < n; i += NWARPS * 32) a[i] = src[i];
    __syncthreads();
  }
}

// Sort one tile's bucket by (depth bits, surfel index).  The depth digits are
// taken relative to the bucket's smallest depth, so only the bits that vary
// are sorted; equal depths are then put in surfel order, and a bucket with a
// long run of equal depths is sorted once more on the full composite key.
template <int NWARPS>
__device__ void sort_bucket_any(unsigned long long* a, unsigned long long* b, int n, uint32_t* cnt, uint32_t* red) {
  // red[0..3]: min depth, max depth, min index, max index; red[4]: long-run flag
  if (threadIdx.x == 0) {
    red[0] = 0xffffffffu; red[1] = 0u; red[2] = 0xffffffffu; red[3] = 0u; red[4] = 0u;
  }
  __syncthreads();
  uint32_t dmn = 0xffffffffu, dmx = 0u, imn = 0xffffffffu, imx = 0u;
  for (int i = threadIdx.x; i < n; i += NWARPS * 32) {
    const unsigned long long x = a[i];
    const uint32_t d = (uint32_t)(x >> 32), s = (uint32_t)x;
    dmn = min(dmn, d); dmx = max(dmx, d); imn = min(imn, s); imx = max(imx, s);
  }
  dmn = __reduce_min_sync(0xffffffffu, dmn);
  dmx = __reduce_max_sync(0xffffffffu, dmx);
  imn = __reduce_min_sync(0xffffffffu, imn);
  imx = __reduce_max_sync(0xffffffffu, imx);
  if ((threadIdx.x & 31) == 0) {
    atomicMin(&red[0], dmn); atomicMax(&red[1], dmx); atomicMin(&red[2], imn); atomicMax(&red[3], imx);
  }
  __syncthreads();
  const uint32_t dmin = red[0], dbits = (uint32_t)bits_of(red[1] - red[0]);
  const uint32_t imin = red[2], ibits = (uint32_t)bits_of(red[3] - red[2]);
  block_radix_any<NWARPS>(a, b, n, cnt, dmin, 0u, -1, (int)dbits);
  // equal depth bits: ascending surfel index (short runs in place)
  for (int i = threadIdx.x; i < n; i += NWARPS * 32) {
    const uint32_t d = (uint32_t)(a[i] >> 32);
    const bool starts = (i == 0 || (uint32_t)(a[i - 1] >> 32) != d) && i + 1 < n && (uint32_t)(a[i + 1] >> 32) == d;
    if (!starts) continue;
    int e = i + 1;
    while (e + 1 < n && e - i < 64 && (uint32_t)(a[e + 1] >> 32) == d) e++;
    if (e + 1 < n && (uint32_t)(a[e + 1] >> 32) == d) {
      red[4] = 1u;  // a long run: handled below
      continue;
    }
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
  if (red[4]) block_radix_any<NWARPS>(a, b, n, cnt, dmin, imin, (int)ibits, (int)(dbits + ibits));
}

// Shared-memory radix sort of a bucket of at most NWARPS * 32 * ITEMS
// composites, the keys of each pass held in registers.  Warp w owns a
// contiguous slice of the array; per pass it ranks its keys round by round
// (a round = 32 consecutive keys) with a ballot multisplit: eight ballots, one
// per digit bit, give each lane the mask of lanes holding its digit, so the
// rank within the round is a population count, and the round's first lane of
// each digit advances the warp's 16-bit counter of that digit.  A block scan
// of the (digit, warp) counters in digit-major order turns them into output
// offsets, so equal digits keep their order (stable), and every key is then
// stored at its offset.  Digits are those of block_radix_any.  Returns the
// buffer holding the result (a or b).  a and b may be the same buffer: a
// pass loads all its keys into registers before a block barrier and
// scatters them after it.
template <int NWARPS>
struct RegSortSmem {
  static constexpr int CP = NWARPS + 2;  // padded counter row: conflict-free leader updates
  static constexpr size_t CNT_BYTES = sizeof(uint16_t) * 256 * CP;
  static constexpr size_t BYTES = ((CNT_BYTES + 15) & ~(size_t)15) + sizeof(uint32_t) * (32 + 8);
};

template <int NWARPS, int ITEMS>
__device__ unsigned long long* block_radix_reg(unsigned long long* a, unsigned long long* b, int n, uint16_t* cnt,
                                               uint32_t* tot, uint32_t dmin, uint32_t imin, int ishift, int nbits,
                                               int lsb = 0) {
  constexpr int NT = NWARPS * 32, CP = RegSortSmem<NWARPS>::CP;
  static_assert(NWARPS % 8 == 0, "the counter scan takes 8 counters per thread");
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const uint32_t lt_mask = (1u << lane) - 1u;
  const int per = (((n + NWARPS - 1) / NWARPS) + 31) & ~31;
  const int lo = min(wid * per, n), hi = min(lo + per, n);
  const int nr = (hi - lo + 31) >> 5;  // rounds of this warp (<= ITEMS)
  const int passes = (nbits + 7) >> 3;
  unsigned long long* src = a;
  unsigned long long* dst = b;
  auto digit = [&](unsigned long long key, int shift) -> uint32_t {
    const unsigned long long dk = (unsigned long long)((uint32_t)(key >> 32) - dmin);
    const unsigned long long kk = ishift < 0 ? dk : ((dk << ishift) | (unsigned long long)((uint32_t)key - imin));
    return (uint32_t)(kk >> (shift + lsb)) & 0xffu;
  };
  int first = 0;
  if (passes > 0) {
    // The first pass may leave equal digits in any order (the order it starts
    // from is arbitrary anyway): each key takes its slot within its digit from
    // one shared atomic on a 256-bin histogram, and only the 256 bins are
    // scanned.  The later passes keep the order of equal digits (below).
    uint32_t* hist = reinterpret_cast<uint32_t*>(cnt);  // 256 words of the counter space
    unsigned long long key[ITEMS];
    uint32_t off[ITEMS];
    for (int i = threadIdx.x; i < 256; i += NT) hist[i] = 0u;
#pragma unroll
    for (int k = 0; k < ITEMS; k++) {
      const int i = lo + k * 32 + lane;
      key[k] = (k < nr && i < hi) ? src[i] : 0ull;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < ITEMS; k++) {
      if (k < nr && lo + k * 32 + lane < hi) {
        const uint32_t d = digit(key[k], 0);
        off[k] = (d << 16) | atomicAdd(&hist[d], 1u);
      }
    }
    __syncthreads();
    uint32_t v = 0, x = 0;
    if (threadIdx.x < 256) {
      v = hist[threadIdx.x];
      x = v;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
      }
      if (lane == 31) tot[wid] = x;
    }
    __syncthreads();
    if (threadIdx.x < 256) {
      uint32_t before = 0;
      for (int w = 0; w < wid; w++) before += tot[w];
      hist[threadIdx.x] = before + x - v;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < ITEMS; k++)
      if (k < nr && lo + k * 32 + lane < hi) dst[hist[off[k] >> 16] + (off[k] & 0xffffu)] = key[k];
    __syncthreads();
    unsigned long long* t = src;
    src = dst;
    dst = t;
    first = 1;
  }
  for (int pass = first; pass < passes; pass++) {
    const int shift = 8 * pass;
    unsigned long long key[ITEMS];
    uint32_t off[ITEMS];
#pragma unroll
    for (int k = 0; k < ITEMS; k++) {
      const int i = lo + k * 32 + lane;
      key[k] = (k < nr && i < hi) ? src[i] : 0ull;
    }
    for (int i = threadIdx.x; i < 256 * CP / 2; i += NT) reinterpret_cast<uint32_t*>(cnt)[i] = 0u;
    __syncthreads();
#pragma unroll
    for (int k = 0; k < ITEMS; k++) {
      if (k < nr) {
        const bool valid = lo + k * 32 + lane < hi;
        const uint32_t d = valid ? digit(key[k], shift) : 0u;
        uint32_t peers = __ballot_sync(0xffffffffu, valid);
#pragma unroll
        for (int bit = 0; bit < 8; bit++) {
          const bool on = (d >> bit) & 1u;
          const uint32_t bal = __ballot_sync(0xffffffffu, on);
          peers &= on ? bal : ~bal;
        }
        const int leader = __ffs(peers) - 1;
        uint32_t pre = 0;
        if (valid && lane == leader) {
          pre = cnt[d * CP + wid];
          cnt[d * CP + wid] = (uint16_t)(pre + __popc(peers));
        }
        pre = __shfl_sync(0xffffffffu, pre, leader & 31);
        off[k] = (d << 16) | (pre + __popc(peers & lt_mask));
        __syncwarp();
      }
    }
    __syncthreads();
    {
      // exclusive scan of the counters in (digit, warp) order, 8 per thread
      const int f0 = 8 * threadIdx.x, d = f0 / NWARPS, w0 = f0 % NWARPS;
      uint32_t c[8], sum = 0;
#pragma unroll
      for (int j = 0; j < 8; j++) {
        c[j] = cnt[d * CP + w0 + j];
        sum += c[j];
      }
      uint32_t x = sum;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
      }
      if (lane == 31) tot[wid] = x;
      __syncthreads();
      if (wid == 0) {
        uint32_t y = lane < NWARPS ? tot[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const uint32_t z = __shfl_up_sync(0xffffffffu, y, o);
          if (lane >= o) y += z;
        }
        if (lane < NWARPS) tot[lane] = y;
      }
      __syncthreads();
      uint32_t ex = x - sum + (wid > 0 ? tot[wid - 1] : 0u);
#pragma unroll
      for (int j = 0; j < 8; j++) {
        cnt[d * CP + w0 + j] = (uint16_t)ex;
        ex += c[j];
      }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < ITEMS; k++) {
      if (k < nr && lo + k * 32 + lane < hi) {
        const uint32_t d = off[k] >> 16;
        dst[(uint32_t)cnt[d * CP + wid] + (off[k] & 0xffffu)] = key[k];
      }
    }
    __syncthreads();
    unsigned long long* t = src;
    src = dst;
    dst = t;
  }
  return src;
}

// Sort a bucket of at most NWARPS * 32 * ITEMS composites by (depth bits,
// surfel index) and write it out as (tile | depth bits) keys and surfel
// values: load it from global memory into shared memory (finding the
// bucket's depth and index ranges on the way), radix-sort the top 16 bits of
// the depth relative to the smallest depth (two passes where the depths span
// more), then write every entry out at its place: an entry that ties with no
// neighbour on those bits at its sorted position, an entry of a run of ties
// at the run's start plus the number of the run's composites below its own
// (the composites are distinct), so every run is put in (depth, surfel)
// order in parallel.  A run longer than 64 triggers one exact re-sort on the
// relative composite key instead, whose result is written over.
template <int NWARPS, int ITEMS>
__device__ void sort_bucket_reg(const unsigned long long* __restrict__ g, int n, unsigned long long* sa,
                                unsigned long long* sb, uint16_t* cnt, uint32_t* tot, uint32_t* red,
                                uint64_t tile, uint64_t* __restrict__ okeys, uint32_t* __restrict__ ovals) {
  constexpr int NT = NWARPS * 32;
  if (threadIdx.x == 0) {
    red[0] = 0xffffffffu; red[1] = 0u; red[2] = 0xffffffffu; red[3] = 0u; red[4] = 0u;
  }
  __syncthreads();
  uint32_t dmn = 0xffffffffu, dmx = 0u, imn = 0xffffffffu, imx = 0u;
  for (int i = threadIdx.x; i < n; i += NT) {
    const unsigned long long x = g[i];
    sa[i] = x;
    const uint32_t d = (uint32_t)(x >> 32), s = (uint32_t)x;
    dmn = min(dmn, d); dmx = max(dmx, d); imn = min(imn, s); imx = max(imx, s);
  }
  dmn = __reduce_min_sync(0xffffffffu, dmn);
  dmx = __reduce_max_sync(0xffffffffu, dmx);
  imn = __reduce_min_sync(0xffffffffu, imn);
  imx = __reduce_max_sync(0xffffffffu, imx);
  if ((threadIdx.x & 31) == 0) {
    atomicMin(&red[0], dmn); atomicMax(&red[1], dmx); atomicMin(&red[2], imn); atomicMax(&red[3], imx);
  }
  __syncthreads();
  const uint32_t dmin = red[0], dbits = (uint32_t)bits_of(red[1] - red[0]);
  const uint32_t imin = red[2], ibits = (uint32_t)bits_of(red[3] - red[2]);
  // radix passes over the top 16 bits of the relative depth only; entries
  // that tie there form runs, put in (depth, surfel) order as they are
  // written out below
  const int lsb = max((int)dbits - 16, 0);
  unsigned long long* r = block_radix_reg<NWARPS, ITEMS>(sa, sb, n, cnt, tot, dmin, 0u, -1, (int)dbits - lsb, lsb);
  const int lane = threadIdx.x & 31;
  auto top = [&](unsigned long long x) -> uint32_t { return ((uint32_t)(x >> 32) - dmin) >> lsb; };
  auto emit = [&](int p, unsigned long long key) {
    okeys[p] = tile | (key >> 32);
    ovals[p] = (uint32_t)key;
  };
  for (int i0 = 0; i0 < n; i0 += NT) {
    const int i = i0 + threadIdx.x;
    const bool in = i < n;
    const unsigned long long key = in ? r[i] : 0ull;
    const uint32_t d = top(key);
    // the neighbours' top bits: the adjacent lanes' entries, across warps a load
    uint32_t dp = __shfl_up_sync(0xffffffffu, d, 1), dn = __shfl_down_sync(0xffffffffu, d, 1);
    if (lane == 0 && in && i > 0) dp = top(r[i - 1]);
    if (lane == 31 && i + 1 < n) dn = top(r[i + 1]);
    if (!in) continue;
    if (!((i > 0 && dp == d) || (i + 1 < n && dn == d))) {
      emit(i, key);
      continue;
    }
    int s = i, e = i;
    while (s > 0 && i - s < 64 && top(r[s - 1]) == d) s--;
    while (e + 1 < n && e - i < 64 && top(r[e + 1]) == d) e++;
    if (e - s >= 64) {
      red[4] = 1u;
      continue;
    }
    int rank = 0;
    for (int y = s; y <= e; y++) rank += r[y] < key ? 1 : 0;
    emit(s + rank, key);
  }
  __syncthreads();
  if (red[4]) {
    const unsigned long long* x =
        block_radix_reg<NWARPS, ITEMS>(r, r == sa ? sb : sa, n, cnt, tot, dmin, imin, (int)ibits, (int)(dbits + ibits));
    for (int i = threadIdx.x; i < n; i += NT) emit(i, x[i]);
  }
}

// Per-tile bucket sorts in three size classes, each a persistent launch over
// its class's tile list with shared memory sized for the class (so short
// buckets run several CTAs per SM); the last class also takes the buckets
// longer than its capacity and sorts those in global memory.
struct SegArgs {
  const uint2* ranges;
  unsigned long long* bucket;   // scattered composites (sorted in place for the oversized buckets)
  unsigned long long* scratch;  // ping-pong space for the oversized buckets (same indexing as bucket)
  uint64_t* keys;               // out: (tile << 32) | depth bits
  uint32_t* vals;               // out: surfel index
  Header* hdr;
  int64_t cap;                  // instance capacity
  const uint32_t* list;         // this class's tiles
  const uint32_t* list_count;   // their number
  uint32_t* queue;              // this class's work counter
};

template <int NWARPS, int ITEMS>
struct SegClass {
  static constexpr int THREADS = NWARPS * 32;
  static constexpr int CAP = NWARPS * 32 * ITEMS;
  static constexpr size_t SMEM = sizeof(unsigned long long) * CAP + RegSortSmem<NWARPS>::BYTES;
};

template <int NWARPS, int ITEMS, bool LAST>
// The bucket is sorted in place in one shared buffer (each radix pass holds
// its keys in registers between its loads and its scatter, with block
// barriers in between), so the 1025..4096, 4097..6144 and 6145..8192 classes
// (41, 57 and 73 KB of shared memory) run 3 CTAs per SM under a 42-register
// bound: their keys spill, but the third CTA hides more of the barrier waits
// (binning 10.01 -> 9.82 ms for the first class, 9.82 -> 9.62 ms for the
// second, on the 32-keyframe submap; sorting the 6145..8192 buckets there
// instead of in the 1024-thread class at one CTA per SM: 9.63 -> 9.37 ms, and
// 9.46 ms at 2 CTAs per SM without the spills).  The <= 1024 and 1025..2048
// classes (256 threads, 13 and 21 KB) run 6 CTAs per SM, which matters where
// buckets are short (64 uneven submaps: binning 13.38 -> 11.37 ms for the
// first, and 11.62 -> 11.35 ms for taking the 1025..2048 buckets out of the
// 512-thread class).
__global__ void __launch_bounds__(NWARPS * 32, NWARPS == 16 ? 3 : (NWARPS == 8 ? 6 : 1)) k_tile_sort(const SegArgs A) {
  using C = SegClass<NWARPS, ITEMS>;
  extern __shared__ __align__(16) unsigned char smem[];
  unsigned long long* sa = reinterpret_cast<unsigned long long*>(smem);
  unsigned long long* sb = sa;  // in place: every pass holds its keys in registers
  static_assert(!LAST || sizeof(unsigned long long) * C::CAP >= sizeof(uint32_t) * ((NWARPS + 1) * 256 + 8),
                "the oversized-bucket counters fit in the key buffer");
  uint16_t* cnt = reinterpret_cast<uint16_t*>(sa + C::CAP);
  uint32_t* tot = reinterpret_cast<uint32_t*>(smem + sizeof(unsigned long long) * C::CAP +
                                              ((RegSortSmem<NWARPS>::CNT_BYTES + 15) & ~(size_t)15));
  uint32_t* red = tot + 32;
  __shared__ uint32_t s_q;
  if (A.hdr->status != 0) return;
  const uint32_t n_tiles = *A.list_count;
  for (;;) {
    if (threadIdx.x == 0) s_q = atomicAdd(A.queue, 1u);
    __syncthreads();
    const uint32_t q = s_q;
    __syncthreads();
    if (q >= n_tiles) break;
    const uint32_t t = A.list[q];
    const uint2 rg = A.ranges[t];
    if (!s2d_check(rg.x <= rg.y && (int64_t)rg.y <= A.cap, A.hdr)) continue;
    const int n = (int)(rg.y - rg.x);
    const uint64_t tile = (uint64_t)t << 32;
    if (!LAST || n <= C::CAP) {
      sort_bucket_reg<NWARPS, ITEMS>(A.bucket + rg.x, n, sa, sb, cnt, tot, red, tile, A.keys + rg.x, A.vals + rg.x);
    } else {
      uint32_t* c32 = reinterpret_cast<uint32_t*>(smem);
      sort_bucket_any<NWARPS>(A.bucket + rg.x, A.scratch + rg.x, n, c32, c32 + (NWARPS + 1) * 256);
      const unsigned long long* res = A.bucket + rg.x;
      for (int i = threadIdx.x; i < n; i += NWARPS * 32) {
        const unsigned long long key = res[i];
        A.keys[rg.x + i] = tile | (key >> 32);
        A.vals[rg.x + i] = (uint32_t)key;
      }
    }
    __syncthreads();
  }
}

template <int NWARPS, int ITEMS, bool LAST>
static cudaError_t launch_tile_sort_class(const SegArgs& S, cudaStream_t st) {
  using C = SegClass<NWARPS, ITEMS>;
  auto k = k_tile_sort<NWARPS, ITEMS, LAST>;
  static int per_sm = -1;
  if (per_sm < 0) {
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, C::THREADS, C::SMEM);
    if (per_sm < 1) per_sm = 1;
  }
  k<<<per_sm * sm_count(), C::THREADS, C::SMEM, st>>>(S);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_bin_tiles(const Layout& L, const RastParams& P, char* ws, cudaStream_t st) {
  if (L.R <= 0 || L.T <= 0) return cudaSuccess;
  Header* hdr = reinterpret_cast<Header*>(ws + L.header);
  uint32_t* counts = reinterpret_cast<uint32_t*>(ws + L.tile_count);
  uint32_t* cursors = reinterpret_cast<uint32_t*>(ws + L.tile_cursor);
  uint2* ranges = reinterpret_cast<uint2*>(ws + L.ranges);
  cudaError_t e = cudaMemsetAsync(counts, 0, sizeof(uint32_t) * (size_t)L.T, st);
  if (e != cudaSuccess) return e;
  TileBinArgs A;
  A.bins = reinterpret_cast<const uint4*>(ws + L.bins);
  A.views = reinterpret_cast<const DView*>(ws + L.views);
  A.V = L.V;
  A.R = L.R;
  A.tile_w = P.tile_w;
  A.tile_h = P.tile_h;
  A.counts = counts;
  A.bucket = reinterpret_cast<unsigned long long*>(ws + L.keys1);
  A.cap = L.cap;
  A.hdr = hdr;
  const int64_t blocks = (L.R + 255) / 256;
  const int grid0 = (int)min64(blocks, (int64_t)sm_count() * 16), grid1 = grid0;
  k_tile_bin<false><<<grid0, 256, 0, st>>>(A);
  count_launches(1);
  uint32_t* queues = reinterpret_cast<uint32_t*>(ws + L.tile_hist) + ORDER_BINS;  // per class: queue, list size
  uint32_t* class_list = reinterpret_cast<uint32_t*>(ws + L.tile_class);
  e = cudaMemsetAsync(queues, 0, 2 * SORT_CLASSES * sizeof(uint32_t), st);
  if (e != cudaSuccess) return e;
  k_tile_scan<<<1, 1024, 0, st>>>(counts, cursors, ranges, L.T, hdr, L.cap, class_list, queues + SORT_CLASSES);
  count_launches(1);
  A.counts = cursors;
  k_tile_bin<true><<<grid1, 256, 0, st>>>(A);
  count_launches(1);
  SegArgs S;
  S.ranges = ranges;
  S.bucket = A.bucket;
  S.scratch = reinterpret_cast<unsigned long long*>(ws + L.keys0);
  S.keys = reinterpret_cast<uint64_t*>(ws + L.keys0);
  S.vals = reinterpret_cast<uint32_t*>(ws + L.vals0);
  S.hdr = hdr;
  S.cap = L.cap;
  static_assert(SegClass<8, 4>::CAP == SORT_CLASS_BOUND[0] && SegClass<8, 8>::CAP == SORT_CLASS_BOUND[1] &&
                    SegClass<16, 8>::CAP == SORT_CLASS_BOUND[2] && SegClass<16, 12>::CAP == SORT_CLASS_BOUND[3] &&
                    SegClass<16, 16>::CAP == SORT_CLASS_BOUND[4] && SegClass<32, 12>::CAP == SORT_CLASS_BOUND[5],
                "class capacities match the class bounds");
  for (int c = 0; c < SORT_CLASSES; c++) {
    S.list = class_list + (size_t)c * L.T;
    S.list_count = queues + SORT_CLASSES + c;
    S.queue = queues + c;
    switch (c) {
      case 0: e = launch_tile_sort_class<8, 4, false>(S, st); break;
      case 1: e = launch_tile_sort_class<8, 8, false>(S, st); break;
      case 2: e = launch_tile_sort_class<16, 8, false>(S, st); break;
      case 3: e = launch_tile_sort_class<16, 12, false>(S, st); break;
      case 4: e = launch_tile_sort_class<16, 16, false>(S, st); break;
      default: e = launch_tile_sort_class<32, 12, true>(S, st); break;
    }
    if (e != cudaSuccess) return e;
  }
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
