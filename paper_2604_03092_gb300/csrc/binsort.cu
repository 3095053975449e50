// Tile binning and the device radix sort.
//
// Binning: every visible (view, surfel) record emits one instance per tile of
// its tile rect, in record order, with key = (global tile) << 32 | FP32 depth
// bits and value = surfel index.  Offsets come from an exclusive scan of the
// per-record tile counts (reduce -> scan of block sums -> scan + emit).
//
// Sort: least-significant-digit radix sort with 8-bit digits over the key bits
// in use (32 depth bits + enough bits for the global tile index).  Each pass is
// upsweep (per-block digit histograms) -> scan of the histograms -> downsweep
// (stable ranking of each 2048-key tile with warp-level match, then scatter).
// Blocks own contiguous, ordered slices of the input and every ranking step
// preserves input order among equal digits, so the whole sort is stable:
// instances with equal (tile, depth) keep ascending record order, i.e.
// ascending surfel index within a view.
#include <cuda_runtime.h>

#include "splat2d_internal.cuh"

namespace s2d {

// ---------------------------------------------------------------------------
// exclusive scan of tile counts, fused with the emission of instances
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_scan_reduce(const uint32_t* __restrict__ ntiles, int64_t R,
                                                      unsigned long long* __restrict__ part, int64_t n_tiles) {
  __shared__ unsigned long long s_w[8];
  for (int64_t b = blockIdx.x; b < n_tiles; b += gridDim.x) {
    const int64_t base = b * SCAN_TILE;
    unsigned long long sum = 0;
    for (int i = threadIdx.x; i < SCAN_TILE; i += 256) {
      int64_t r = base + i;
      if (r < R) sum += __ldg(ntiles + r);
    }
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = sum;
    __syncthreads();
    if (threadIdx.x == 0) {
      unsigned long long t = 0;
      for (int w = 0; w < 8; w++) t += s_w[w];
      part[b] = t;
    }
    __syncthreads();
  }
}

// One block: exclusive scan of the block sums; total -> header, capacity check.
__global__ void __launch_bounds__(1024) k_scan_partials(unsigned long long* __restrict__ part, int64_t n,
                                                        Header* __restrict__ hdr, int64_t cap) {
  __shared__ unsigned long long s_w[32];
  __shared__ unsigned long long s_carry;
  if (threadIdx.x == 0) s_carry = 0;
  __syncthreads();
  for (int64_t base = 0; base < n; base += 1024) {
    int64_t i = base + threadIdx.x;
    unsigned long long v = i < n ? part[i] : 0ull;
    unsigned long long x = v;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int o = 1; o < 32; o <<= 1) {
      unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) s_w[wid] = x;
    __syncthreads();
    if (wid == 0) {
      unsigned long long w = s_w[lane];
      for (int o = 1; o < 32; o <<= 1) {
        unsigned long long y = __shfl_up_sync(0xffffffffu, w, o);
        if (lane >= o) w += y;
      }
      s_w[lane] = w;
    }
    __syncthreads();
    unsigned long long incl = x + (wid > 0 ? s_w[wid - 1] : 0ull) + s_carry;
    if (i < n) part[i] = incl - v;
    __syncthreads();
    if (threadIdx.x == 1023) s_carry = incl;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    unsigned long long total = s_carry;
    hdr->needed = total;
    if ((int64_t)total > cap) {
      hdr->status = SPLAT2D_ERR_CAPACITY;
      hdr->n_inst = 0;
    } else {
      hdr->n_inst = total;
    }
  }
}

struct BinArgs {
  const uint32_t* ntiles;
  const float4* records;
  const unsigned long long* part;
  const DView* views;
  int32_t V;
  int64_t R;
  int64_t n_tiles;
  int32_t tile_w, tile_h;
  const Header* hdr;
  uint64_t* keys;
  uint32_t* vals;
};

// Each thread owns 16 consecutive records of a 4096-record scan tile.
__global__ void __launch_bounds__(256) k_bin(const BinArgs A) {
  __shared__ unsigned long long s_w[8];
  if (A.hdr->status != 0) return;  // overflow: emit nothing
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int64_t b = blockIdx.x; b < A.n_tiles; b += gridDim.x) {
    const int64_t r0 = b * SCAN_TILE + (int64_t)threadIdx.x * 16;
    uint32_t cnt[16];
    unsigned long long sum = 0;
    if (r0 + 16 <= A.R) {
      const uint4* p = reinterpret_cast<const uint4*>(A.ntiles + r0);
#pragma unroll
      for (int k = 0; k < 4; k++) {
        uint4 q = __ldg(p + k);
        cnt[4 * k] = q.x; cnt[4 * k + 1] = q.y; cnt[4 * k + 2] = q.z; cnt[4 * k + 3] = q.w;
      }
    } else {
#pragma unroll
      for (int k = 0; k < 16; k++) cnt[k] = (r0 + k < A.R) ? __ldg(A.ntiles + r0 + k) : 0u;
    }
#pragma unroll
    for (int k = 0; k < 16; k++) sum += cnt[k];
    // block exclusive scan of per-thread sums
    unsigned long long x = sum;
    for (int o = 1; o < 32; o <<= 1) {
      unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) s_w[wid] = x;
    __syncthreads();
    unsigned long long wpre = 0;
    for (int w = 0; w < wid; w++) wpre += s_w[w];
    unsigned long long off = A.part[b] + wpre + x - sum;
    __syncthreads();
    if (sum == 0) continue;
    int v = find_view_by_record(A.views, A.V, r0);
    for (int k = 0; k < 16; k++) {
      const uint32_t n = cnt[k];
      if (!n) continue;
      const int64_t r = r0 + k;
      while (v + 1 < A.V && A.views[v + 1].rbase <= r) v++;
      const DView& vw = A.views[v];
      const float4 f4 = __ldg(A.records + r * REC_F4 + 4);
      const uint32_t zb = __float_as_uint(f4.y);
      const uint32_t q0 = __float_as_uint(f4.z), q1 = __float_as_uint(f4.w);
      const int tx0 = (int)(q0 & 0xffffu) / A.tile_w, ty0 = (int)(q0 >> 16) / A.tile_h;
      const int tx1 = (int)(q1 & 0xffffu) / A.tile_w, ty1 = (int)(q1 >> 16) / A.tile_h;
      const uint32_t sidx = (uint32_t)(vw.soff + (r - vw.rbase));
      for (int ty = ty0; ty <= ty1; ty++) {
        for (int tx = tx0; tx <= tx1; tx++) {
          const uint64_t tile = (uint64_t)(vw.tile_base + ty * vw.tiles_x + tx);
          A.keys[off] = (tile << 32) | zb;
          A.vals[off] = sidx;
          off++;
        }
      }
    }
  }
}

cudaError_t launch_bin(const Layout& L, const RastParams& P, char* ws, cudaStream_t st) {
  if (L.R <= 0) return cudaSuccess;
  const uint32_t* ntiles = reinterpret_cast<const uint32_t*>(ws + L.ntiles);
  unsigned long long* part = reinterpret_cast<unsigned long long*>(ws + L.scan_part);
  Header* hdr = reinterpret_cast<Header*>(ws + L.header);
  int grid = (int)min64(L.n_scan_tiles, (int64_t)sm_count() * 8);
  k_scan_reduce<<<grid, 256, 0, st>>>(ntiles, L.R, part, L.n_scan_tiles);
  count_launches(1);
  k_scan_partials<<<1, 1024, 0, st>>>(part, L.n_scan_tiles, hdr, L.cap);
  count_launches(1);
  BinArgs A;
  A.ntiles = ntiles;
  A.records = reinterpret_cast<const float4*>(ws + L.records);
  A.part = part;
  A.views = reinterpret_cast<const DView*>(ws + L.views);
  A.V = L.V;
  A.R = L.R;
  A.n_tiles = L.n_scan_tiles;
  A.tile_w = P.tile_w;
  A.tile_h = P.tile_h;
  A.hdr = hdr;
  A.keys = reinterpret_cast<uint64_t*>(ws + L.keys0);
  A.vals = reinterpret_cast<uint32_t*>(ws + L.vals0);
  k_bin<<<grid, 256, 0, st>>>(A);
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

// ---------------------------------------------------------------------------
// tile ranges [start, end) in the sorted instance array
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_ranges(const uint64_t* __restrict__ keys,
                                                const unsigned long long* __restrict__ n_dev,
                                                uint2* __restrict__ ranges) {
  const int64_t n = (int64_t)*n_dev;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t t = (uint32_t)(keys[i] >> 32);
    if (i == 0 || (uint32_t)(keys[i - 1] >> 32) != t) ranges[t].x = (uint32_t)i;
    if (i == n - 1 || (uint32_t)(keys[i + 1] >> 32) != t) ranges[t].y = (uint32_t)(i + 1);
  }
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

cudaError_t launch_ranges(const Layout& L, const uint64_t* keys, char* ws, cudaStream_t st) {
  uint2* ranges = reinterpret_cast<uint2*>(ws + L.ranges);
  Header* hdr = reinterpret_cast<Header*>(ws + L.header);
  cudaError_t e = cudaMemsetAsync(ranges, 0, sizeof(uint2) * (size_t)L.T, st);
  if (e != cudaSuccess) return e;
  int grid = (int)min64((L.cap + 255) / 256, (int64_t)sm_count() * 8);
  if (grid < 1) grid = 1;
  k_ranges<<<grid, 256, 0, st>>>(keys, &hdr->n_inst, ranges);
  count_launches(1);
  uint32_t* bins = reinterpret_cast<uint32_t*>(ws + L.tile_hist);
  uint32_t* order = reinterpret_cast<uint32_t*>(ws + L.tile_order);
  e = cudaMemsetAsync(bins, 0, sizeof(uint32_t) * ORDER_BINS, st);
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
