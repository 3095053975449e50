// Per-tile compositing (forward) and its adjoint (backward).
//
// Both kernels are persistent: one CTA per tile-shaped block of pixels pulls
// (view, tile) work items from an atomic queue ordered longest list first,
// so many views of uneven size run in one launch.  A tile's sorted surfel
// list is staged through shared memory in chunks.  For each chunk every lane
// (one pixel) gets a bitmask of the chunk entries whose pixel rect holds its
// pixel, built with 12 ballots per 32 entries (which entries span each column
// and each row of the warp's 8x4 patch), and then walks only its own entries:
// surfels are a few pixels wide, so a lane-per-pixel walk over a shared entry
// sequence would leave most lanes idle, while here nearly every lane does a
// useful (pixel, surfel) evaluation on every step.
//
// Forward (Eq. 1): front to back per pixel, alpha = min(alpha_max, sigma*G),
// pairs below alpha_min skipped, stop before T would fall below t_min; the
// tile stops staging as soon as all its pixels have stopped.
// Backward: back to front per pixel from its last blended entry, T recovered
// by division, one scalar suffix sum per pixel (the upstream gradient dotted
// with the features of the entries behind), evaluated 32 (pixel, entry) pairs
// at a time with segmented warp scans; each lane adds its pair's gradient to
// the entry's shared-memory slot, and after the chunk one set of vector
// atomics per (tile, entry) moves the sums to the gradient record.
#include <cuda_runtime.h>

#include "splat2d_internal.cuh"

namespace s2d {

// Shared-memory copy of a chunk of render records, unpacked, stored field by
// field (structure of arrays) so that lanes reading different records hit
// consecutive 16-byte slots instead of colliding banks.
template <int CHUNK>
struct SRecs {
  float4 c[CHUNK];    // cx_hi, cy_hi, cx_lo, cy_lo
  float4 p[CHUNK];    // p00 p01 p10 p11
  float4 q[CHUNK];    // p20 p21 p22 opacity
  float4 col[CHUNK];  // r g b z
  float4 n[CHUNK];    // nx ny nz, and in .w the pixel rect clipped to the tile (see pack_tile_rect)
};

// A record's pixel rect clipped to the tile and made relative to its origin,
// one byte per bound: x0 | y0 << 8 | x1 << 16 | y1 << 24 (inclusive; an
// empty clip has x0 > x1).  Tiles are at most 32 pixels wide.
__device__ __forceinline__ uint32_t pack_tile_rect(int x0, int y0, int x1, int y1, int tx0, int ty0, int tw,
                                                   int th) {
  const int a0 = max(x0 - tx0, 0), a1 = min(x1 - tx0, tw - 1);
  const int b0 = max(y0 - ty0, 0), b1 = min(y1 - ty0, th - 1);
  if (a0 > a1 || b0 > b1) return 0xffu;  // x0 = 255 > x1 = 0
  return (uint32_t)a0 | (uint32_t)b0 << 8 | (uint32_t)a1 << 16 | (uint32_t)b1 << 24;
}

template <int CHUNK>
__device__ __forceinline__ void unpack_record(const float4* __restrict__ rec, SRecs<CHUNK>& o, int j, int tx0,
                                              int ty0, int tw, int th, float4* __restrict__ copy = nullptr) {
  const float4 f0 = __ldg(rec + 0), f1 = __ldg(rec + 1), f2 = __ldg(rec + 2), f3 = __ldg(rec + 3),
               f4 = __ldg(rec + 4);
  if (copy) {  // streaming stores: read back only by the backward, long after
    __stcs(copy + 0, f0);
    __stcs(copy + 1, f1);
    __stcs(copy + 2, f2);
    __stcs(copy + 3, f3);
    __stcs(copy + 4, f4);
  }
  const float2 lo = unpack_half2_scaled(__float_as_uint(f0.z));
  o.c[j] = make_float4(f0.x, f0.y, lo.x, lo.y);
  o.p[j] = f1;
  o.q[j] = make_float4(f2.x, f2.y, f2.z, f0.w);
  o.col[j] = make_float4(f2.w, f3.x, f3.y, f4.y);
  const uint32_t r0 = __float_as_uint(f4.z), r1 = __float_as_uint(f4.w);
  const int x0 = (int)(r0 & 0xffffu), y0 = (int)(r0 >> 16), x1 = (int)(r1 & 0xffffu), y1 = (int)(r1 >> 16);
  o.n[j] = make_float4(f3.z, f3.w, f4.x, __uint_as_float(pack_tile_rect(x0, y0, x1, y1, tx0, ty0, tw, th)));
}

// alpha of one (pixel, record) pair.  Written with explicit round-to-nearest
// intrinsics so the forward and the backward compute identical bits.
struct Pair {
  float alpha, G, a, b, rc, rho, dx, dy;
  bool obj, clamped;
};
__device__ __forceinline__ void eval_pair(const float4 c, const float4 p, const float4 q, float px, float py,
                                          float lp_scale, float alpha_max, Pair& e) {
  e.dx = __fsub_rn(__fsub_rn(px, c.x), c.z);
  e.dy = __fsub_rn(__fsub_rn(py, c.y), c.w);
  e.a = __fmaf_rn(p.x, e.dx, __fmul_rn(p.y, e.dy));
  e.b = __fmaf_rn(p.z, e.dx, __fmul_rn(p.w, e.dy));
  const float cc = __fmaf_rn(q.x, e.dx, __fmaf_rn(q.y, e.dy, q.z));
  e.rc = rcp_approx(cc);
  const float ua = __fmul_rn(e.a, e.rc), vb = __fmul_rn(e.b, e.rc);
  const float ro = __fmaf_rn(ua, ua, __fmul_rn(vb, vb));
  const float rl = __fmul_rn(lp_scale, __fmaf_rn(e.dx, e.dx, __fmul_rn(e.dy, e.dy)));
  e.obj = ro <= rl;  // false for NaN (c = 0): the low-pass term decides
  e.rho = e.obj ? ro : rl;
  e.G = ex2_approx(-e.rho);
  const float raw = __fmul_rn(q.w, e.G);
  e.clamped = raw > alpha_max;
  e.alpha = e.clamped ? alpha_max : raw;
}

// Depth a pair contributes to the depth output: the center's depth z
// (record), or with the ray option, where the object-space term decides, the
// depth of the ray-splat intersection.  The record's third row is the
// normalised plane normal: c = N n.d(x) with d(x) the pixel's ray (z = 1),
// and at the center c = p22 = N n.mu_c / z, so the plane depth n.mu_c / n.d(x)
// is z p22 / c.
__device__ __forceinline__ float pair_depth(const Pair& e, float z, float p22, int depth_ray) {
  return (depth_ray && e.obj) ? z * p22 * e.rc : z;
}

// Whether the tile-relative pixel (lx, ly) lies in a packed clipped rect.
__device__ __forceinline__ bool in_tile_rect(uint32_t r, int lx, int ly) {
  return lx >= (int)(r & 0xffu) && ly >= (int)((r >> 8) & 0xffu) && lx <= (int)((r >> 16) & 0xffu) &&
         ly <= (int)(r >> 24);
}

struct RenderArgs {
  const DView* views;
  int32_t V;
  int64_t T;
  const uint2* ranges;
  const uint32_t* order;
  const uint32_t* vals;
  const float4* records;
  float4* rcopy;  // records in sorted-list order (instance i at i * REC_F4)
  // Blended-pair masks: for tile t, word w of its list (entries range.x +
  // 32 w ...) and the pixel of forward thread k, the entries of the word the
  // forward blended there, at ((range.x / 32 + t + w) * NT + k).  Written by
  // the forward for every chunk it stages, read by the backward.
  uint32_t* bmask;
  int64_t bmask_words;
  float* rgrad;
  RastParams P;
  Header* hdr;
  float* rgb;
  float* depth;
  float* normal;
  float* alpha;
  float* tfinal;
  uint32_t* last;
  float* dist;          // depth distortion output (forward; null: not asked for)
  float* dfinal;        // per pixel depth sum D, kept for the distortion's adjoint
  const float* d_dist;  // upstream gradient of the distortion (backward; null: none)
  const float* d_rgb;
  const float* d_depth;
  const float* d_normal;
  const float* d_alpha;
};

// Copies entries [base, base + count) of the sorted list's records to shared
// memory (a dependent gather: list entry, then record), and with keep_copy
// also to the sorted-order copy the backward reads.  (An L2 prefetch of the
// next chunk's records issued here cost the forward 0.56 ms on the submap:
// the gather's requests compete with it.)
// The list entries come in `ent`: entry threadIdx.x + e * NT of the chunk in
// ent[e], read a chunk ahead (see load_entries), so the record loads issue
// without first waiting on the list.
template <int NT, int CHUNK>
__host__ __device__ constexpr int entries_per_thread() {
  return (CHUNK + NT - 1) / NT;
}
template <int NT, int CHUNK>
__device__ __forceinline__ void load_entries(const RenderArgs& A, int64_t base, int64_t end,
                                             uint32_t (&ent)[entries_per_thread<NT, CHUNK>()]) {
#pragma unroll
  for (int e = 0; e < entries_per_thread<NT, CHUNK>(); e++) {
    const int j = (int)threadIdx.x + e * NT;
    ent[e] = (j < CHUNK && base + j < end) ? __ldg(A.vals + base + j) : 0u;
  }
}
template <int NT, int CHUNK>
__device__ __forceinline__ void stage_chunk(const RenderArgs& A, const DView& vw, int tx0, int ty0, int tw, int th,
                                            int64_t base, int count, SRecs<CHUNK>& s_rec, bool keep_copy,
                                            const uint32_t (&ent)[entries_per_thread<NT, CHUNK>()]) {
#pragma unroll
  for (int e = 0; e < entries_per_thread<NT, CHUNK>(); e++) {
    const int j = (int)threadIdx.x + e * NT;
    if (j >= count) break;
    const uint32_t s = ent[e];
    if (s2d_check((int64_t)s >= vw.soff && (int64_t)s < vw.soff + vw.scnt, A.hdr)) {
      const int64_t rec = vw.rbase + ((int64_t)s - vw.soff);
      unpack_record<CHUNK>(A.records + rec * REC_F4, s_rec, j, tx0, ty0, tw, th,
                           keep_copy ? A.rcopy + (base + j) * REC_F4 : nullptr);
    }
  }
}

// Copies entries [base, base + count) from the sorted-order record copy the
// forward left (contiguous, so the loads coalesce and wait on nothing) and
// the record index of each entry (for the gradient records) from the list.
// (An L2 prefetch of the next chunk's records made no measurable difference.)
template <int NT, int CHUNK>
__device__ __forceinline__ void stage_chunk_seq(const RenderArgs& A, const DView& vw, int tx0, int ty0, int tw,
                                                int th, int64_t base, int count, SRecs<CHUNK>& s_rec,
                                                uint32_t* s_idx) {
  for (int j = threadIdx.x; j < count; j += NT) {
    const uint32_t s = __ldg(A.vals + base + j);
    if (!s2d_check((int64_t)s >= vw.soff && (int64_t)s < vw.soff + vw.scnt, A.hdr)) continue;
    unpack_record<CHUNK>(A.rcopy + (base + j) * REC_F4, s_rec, j, tx0, ty0, tw, th);
    s_idx[j] = (uint32_t)(vw.rbase + ((int64_t)s - vw.soff));
  }
}

// Per-lane visit masks.  Each warp owns an 8x4 pixel patch (lane = column
// (lane & 7), row (lane >> 3)).  For the 32 entries of word `wd` of the chunk,
// returns the bits of the entries whose pixel rect holds this lane's pixel:
// the warp ballots, per patch column and per patch row, which entries'
// rects span it, and each lane ANDs its column's and its row's ballot.
template <int CHUNK>
__device__ __forceinline__ uint32_t lane_word(const SRecs<CHUNK>& s_rec, int wd, int count, int px0, int py0,
                                              int lane) {
  const int j = wd * 32 + lane;
  uint32_t cm = 0, rm = 0;
  if (j < count) {
    // (px0, py0): the patch's offset in the tile
    const uint32_t r = __float_as_uint(s_rec.n[j].w);
    const int c0 = max((int)(r & 0xffu) - px0, 0), c1 = min((int)((r >> 16) & 0xffu) - px0, 7);
    const int r0 = max((int)((r >> 8) & 0xffu) - py0, 0), r1 = min((int)(r >> 24) - py0, 3);
    if (c0 <= c1 && r0 <= r1) {
      cm = ((2u << c1) - 1u) & ~((1u << c0) - 1u);
      rm = ((2u << r1) - 1u) & ~((1u << r0) - 1u);
    }
  }
  uint32_t colb[8], rowb[4];
#pragma unroll
  for (int c = 0; c < 8; c++) colb[c] = __ballot_sync(0xffffffffu, (cm >> c) & 1u);
#pragma unroll
  for (int r = 0; r < 4; r++) rowb[r] = __ballot_sync(0xffffffffu, (rm >> r) & 1u);
  const int mc = lane & 7, mr = lane >> 3;
  uint32_t cw = colb[0];
#pragma unroll
  for (int c = 1; c < 8; c++) cw = (mc == c) ? colb[c] : cw;
  uint32_t rw = rowb[0];
#pragma unroll
  for (int r = 1; r < 4; r++) rw = (mr == r) ? rowb[r] : rw;
  return cw & rw;
}

// Position of the r-th set bit (r >= 1, counted from bit 0) of a word that
// has at least r set bits: a binary search on population counts of halves.
__device__ __forceinline__ int nth_set_bit(uint32_t b, int r) {
  int pos = 0, c;
  c = __popc(b & 0xffffu);
  if (r > c) { r -= c; b >>= 16; pos += 16; }
  c = __popc(b & 0xffu);
  if (r > c) { r -= c; b >>= 8; pos += 8; }
  c = __popc(b & 0xfu);
  if (r > c) { r -= c; b >>= 4; pos += 4; }
  c = __popc(b & 0x3u);
  if (r > c) { r -= c; b >>= 2; pos += 2; }
  c = (int)(b & 1u);
  if (r > c) pos += 1;
  return pos;
}

// Sum 8 per-lane values over the warp and give every lane all 8 totals
// (a transposing butterfly: each level halves the values a lane keeps).
__device__ __forceinline__ void warp_sum8_all(float (&v)[8], int lane) {
#pragma unroll
  for (int i = 0; i < 4; i++) {
    const bool up = lane & 16;
    const float send = up ? v[i] : v[i + 4];
    const float keep = up ? v[i + 4] : v[i];
    v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
  }
#pragma unroll
  for (int i = 0; i < 2; i++) {
    const bool up = lane & 8;
    const float send = up ? v[i] : v[i + 2];
    const float keep = up ? v[i + 2] : v[i];
    v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
  }
  {
    const bool up = lane & 4;
    const float send = up ? v[0] : v[1];
    const float keep = up ? v[1] : v[0];
    v[0] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
  }
  v[0] += __shfl_xor_sync(0xffffffffu, v[0], 2);
  v[0] += __shfl_xor_sync(0xffffffffu, v[0], 1);
  // lane L now holds the total of value index (L >> 2) & 7
  const float t0 = v[0];
#pragma unroll
  for (int k = 0; k < 8; k++) v[k] = __shfl_sync(0xffffffffu, t0, k << 2);
}

// Warp-wide inclusive scans over lanes.
__device__ __forceinline__ float warp_scan_mul(float x, int lane) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const float y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x = __fmul_rn(x, y);
  }
  return x;
}
__device__ __forceinline__ float warp_scan_add(float x, int lane) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const float y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  return x;
}

// Per-pixel state of the forward while it is handed between warps.
struct FwdState {
  float T, C0, C1, C2, D, N0, N1, N2, Ds;
  uint32_t last, done;
};

// Dynamic shared memory of the forward kernel.
template <int NT, int CHUNK>
struct FwdSmem {
  SRecs<CHUNK> rec;
  uint32_t bits[NT / 32][CHUNK / 32][32];
  FwdState st[NT];
  uint16_t list[NT / 32][CHUNK];
  uint16_t apix[NT];
  int item, nact, next;
};

// Tail mode of the forward: once at most P.fwd_tail pixels of a tile per
// warp are still compositing, all warps share them, one pixel at a time.

// DIST: also the depth distortion 2 sum_i sum_{j<i} w_i w_j (z_i - z_j) (front to
// back: each blended pair adds 2 w (z A - D) with A = 1 - T and D the depth
// sum in front of it).
template <int TW, int TH, int CHUNK, bool DIST>
__global__ void __launch_bounds__(TW* TH, (TW * TH == 64) ? (CHUNK <= 64 ? 16 : 12) : 3) k_render_fwd(const RenderArgs A) {
  constexpr int NT = TW * TH, NW = NT / 32, WX = TW / 8;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  FwdSmem<NT, CHUNK>& S = *reinterpret_cast<FwdSmem<NT, CHUNK>*>(smem_raw);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const uint32_t lt_mask = (1u << lane) - 1u;
  const RastParams& P = A.P;
  uint32_t n_eval = 0, n_blend = 0;
  // a failed binning (instance capacity exceeded) leaves no valid lists
  if (A.hdr->status != 0) return;
  for (;;) {
    if (threadIdx.x == 0) S.item = (int)atomicAdd(&A.hdr->queue_fwd, 1u);
    __syncthreads();
    const int item = S.item;
    __syncthreads();
    if (item >= A.T) break;
    const int t = (int)__ldg(A.order + item);
    const int v = find_view_by_tile(A.views, A.V, t);
    const DView& vw = A.views[v];
    const int lt = t - vw.tile_base;
    const int tx0 = (lt % vw.tiles_x) * TW, ty0 = (lt / vw.tiles_x) * TH;
    const int bx = tx0 + (wid % WX) * 8, by = ty0 + (wid / WX) * 4;
    const int ipx = bx + (lane & 7), ipy = by + (lane >> 3);
    const bool inside = ipx < vw.W && ipy < vw.H;
    const float px = (float)ipx + 0.5f, py = (float)ipy + 0.5f;
    const uint2 range = __ldg(A.ranges + t);
    float T = 1.f, C0 = 0.f, C1 = 0.f, C2 = 0.f, D = 0.f, N0 = 0.f, N1 = 0.f, N2 = 0.f, Ds = 0.f;
    uint32_t last = range.x;
    bool done = !inside;
    // list entries of the chunk staged next, read one chunk ahead
    uint32_t ent[entries_per_thread<NT, CHUNK>()];
    load_entries<NT, CHUNK>(A, range.x, range.y, ent);
    for (int64_t base = range.x; base < range.y; base += CHUNK) {
      const int n_act = __syncthreads_count(!done);
      if (n_act == 0) break;
      const int count = (int)min64(CHUNK, (int64_t)range.y - base);
      const int nwd = (count + 31) >> 5;
      // this chunk's first blended-mask word (tile t's words start at range.x / 32 + t);
      // computed where it is written, so nothing of it stays live across the walk
      auto mask_word = [&]() { return (range.x >> 5) + (uint32_t)t + (uint32_t)((base - (int64_t)range.x) >> 5); };
      const bool bm_ok = s2d_check((int64_t)mask_word() + nwd <= A.bmask_words, A.hdr);
      if (threadIdx.x == 0) {
        S.nact = 0;
        S.next = 0;
      }
      {
        uint32_t cur[entries_per_thread<NT, CHUNK>()];
#pragma unroll
        for (int e = 0; e < entries_per_thread<NT, CHUNK>(); e++) cur[e] = ent[e];
        load_entries<NT, CHUNK>(A, base + CHUNK, range.y, ent);
        stage_chunk<NT, CHUNK>(A, vw, tx0, ty0, TW, TH, base, count, S.rec, true, cur);
      }
      __syncthreads();
      if (n_act > P.fwd_tail * NW) {
        // ---- bulk: each lane walks its own pixel's entries --------------------
        if (__all_sync(0xffffffffu, done)) {
          // streaming stores: read once, by the backward, long after
          uint32_t* bm = A.bmask + (size_t)mask_word() * NT + threadIdx.x;
          for (int w2 = 0; w2 < nwd && bm_ok; w2++) __stcs(bm + (size_t)w2 * NT, 0u);
          continue;
        }
        for (int wd = 0; wd < nwd; wd++) S.bits[wid][wd][lane] = lane_word(S.rec, wd, count, bx - tx0, by - ty0, lane);
        int wd = 0;
        uint32_t b = done ? 0u : S.bits[wid][0][lane];
        uint32_t bl = 0u;  // entries of word wd this pixel blended (word wd's slot takes them when the walk moves on)
        for (;;) {
          while (b == 0 && !done && wd + 1 < nwd) {
            S.bits[wid][wd][lane] = bl;
            bl = 0u;
            b = S.bits[wid][++wd][lane];
          }
          const bool has = b != 0 && !done;
          if (!__any_sync(0xffffffffu, has)) break;
          if (!has) continue;
          const int j = wd * 32 + __ffs(b) - 1;
          b &= b - 1;
          Pair e;
          eval_pair(S.rec.c[j], S.rec.p[j], S.rec.q[j], px, py, P.lp_scale, P.alpha_max, e);
          n_eval++;
          if (e.alpha < P.alpha_min) continue;
          const float Tn = __fmul_rn(T, __fsub_rn(1.f, e.alpha));
          if (Tn < P.t_min) {
            done = true;
            continue;
          }
          const float w = __fmul_rn(e.alpha, T);
          const float4 col = S.rec.col[j], nrm = S.rec.n[j];
          C0 = __fmaf_rn(w, col.x, C0);
          C1 = __fmaf_rn(w, col.y, C1);
          C2 = __fmaf_rn(w, col.z, C2);
          float zp = col.w;
          if (P.depth_ray) zp = pair_depth(e, col.w, S.rec.q[j].z, 1);
          if constexpr (DIST) Ds = __fmaf_rn(2.f * w, __fmaf_rn(zp, __fsub_rn(1.f, T), -D), Ds);
          D = __fmaf_rn(w, zp, D);
          N0 = __fmaf_rn(w, nrm.x, N0);
          N1 = __fmaf_rn(w, nrm.y, N1);
          N2 = __fmaf_rn(w, nrm.z, N2);
          T = Tn;
          last = (uint32_t)(base + j + 1);
          bl |= 1u << (j & 31);
          n_blend++;
        }
        S.bits[wid][wd][lane] = bl;
        for (int w2 = wd + 1; w2 < nwd; w2++) S.bits[wid][w2][lane] = 0u;
        uint32_t* bm = A.bmask + (size_t)mask_word() * NT + threadIdx.x;
        for (int w2 = 0; w2 < nwd && bm_ok; w2++) __stcs(bm + (size_t)w2 * NT, S.bits[wid][w2][lane]);
      } else {
        // ---- tail: warps pull the remaining pixels; a warp composites 32 of
        //      a pixel's entries per step with a prefix product of (1 - alpha)
        if (!done) {
          const int k = atomicAdd(&S.nact, 1);
          S.apix[k] = (uint16_t)threadIdx.x;
          S.st[threadIdx.x] = FwdState{T, C0, C1, C2, D, N0, N1, N2, Ds, last, 0u};
        }
        for (int w2 = 0; w2 < nwd; w2++) S.bits[wid][w2][lane] = 0u;  // blended entries, set below
        __syncthreads();
        for (;;) {
          int k = 0;
          if (lane == 0) k = atomicAdd(&S.next, 1);
          k = __shfl_sync(0xffffffffu, k, 0);
          if (k >= n_act) break;
          const int pth = S.apix[k];
          const int pw = pth >> 5, pl = pth & 31;
          const int qx = tx0 + (pw % WX) * 8 + (pl & 7), qy = ty0 + (pw / WX) * 4 + (pl >> 3);
          const float fx = (float)qx + 0.5f, fy = (float)qy + 0.5f;
          FwdState st = S.st[pth];
          float acc[8] = {st.C0, st.C1, st.C2, st.D, st.N0, st.N1, st.N2, st.Ds};
          float tt = st.T;
          uint32_t lst = st.last;
          bool dn = false;
          // this pixel's entries of the chunk, ascending
          int nrel = 0;
          for (int wd = 0; wd < (count + 31) >> 5; wd++) {
            const int j = wd * 32 + lane;
            const bool rel = j < count && in_tile_rect(__float_as_uint(S.rec.n[j].w), qx - tx0, qy - ty0);
            const uint32_t bb = __ballot_sync(0xffffffffu, rel);
            if (rel) S.list[wid][nrel + __popc(bb & lt_mask)] = (uint16_t)j;
            nrel += __popc(bb);
          }
          __syncwarp();
          for (int g = 0; g < nrel && !dn; g += 32) {
            const bool has = g + lane < nrel;
            const int j = has ? (int)S.list[wid][g + lane] : 0;
            Pair e;
            float alpha = 0.f;
            if (has) {
              eval_pair(S.rec.c[j], S.rec.p[j], S.rec.q[j], fx, fy, P.lp_scale, P.alpha_max, e);
              alpha = e.alpha;
            }
            const bool kept = has && alpha >= P.alpha_min;
            const float f = kept ? __fsub_rn(1.f, alpha) : 1.f;
            const float Pin = warp_scan_mul(f, lane);
            float Pex = __shfl_up_sync(0xffffffffu, Pin, 1);
            if (lane == 0) Pex = 1.f;
            const float Tb = __fmul_rn(tt, Pex), Ta = __fmul_rn(tt, Pin);
            const uint32_t stopb = __ballot_sync(0xffffffffu, kept && Ta < P.t_min);
            const int sl = stopb ? __ffs(stopb) - 1 : 32;
            const bool contrib = kept && lane < sl;
            const float w = contrib ? __fmul_rn(alpha, Tb) : 0.f;
            float vals[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            float zpair = 0.f;
            if (contrib) {
              const float4 col = S.rec.col[j], nrm = S.rec.n[j];
              zpair = pair_depth(e, col.w, S.rec.q[j].z, P.depth_ray);
              vals[0] = w * col.x; vals[1] = w * col.y; vals[2] = w * col.z;
              vals[3] = w * zpair;
              vals[4] = w * nrm.x; vals[5] = w * nrm.y; vals[6] = w * nrm.z;
            }
            if constexpr (DIST) {
              // depth sum in front of each pair: the pixel's so far, then the group's own terms before it
              const float wz = vals[3];
              const float Bb = acc[3] + (warp_scan_add(wz, lane) - wz);
              vals[7] = contrib ? 2.f * w * (zpair * (1.f - Tb) - Bb) : 0.f;
            }
            warp_sum8_all(vals, lane);
#pragma unroll
            for (int q = 0; q < 8; q++) acc[q] += vals[q];
            n_eval += (has && lane <= sl) ? 1u : 0u;
            n_blend += contrib ? 1u : 0u;
            if (contrib) atomicOr(&S.bits[pw][j >> 5][pl], 1u << (j & 31));
            const uint32_t cb = __ballot_sync(0xffffffffu, contrib);
            if (cb) lst = (uint32_t)(base + __shfl_sync(0xffffffffu, j, 31 - __clz(cb)) + 1);
            if (stopb) {
              tt = __shfl_sync(0xffffffffu, Tb, sl);
              dn = true;
            } else {
              tt = __shfl_sync(0xffffffffu, Ta, 31);
            }
          }
          if (lane == 0)
            S.st[pth] = FwdState{tt, acc[0], acc[1], acc[2], acc[3], acc[4], acc[5], acc[6], acc[7], lst, dn ? 1u : 0u};
          __syncwarp();
        }
        __syncthreads();
        uint32_t* bm = A.bmask + (size_t)mask_word() * NT + threadIdx.x;
        for (int w2 = 0; w2 < nwd && bm_ok; w2++) __stcs(bm + (size_t)w2 * NT, S.bits[wid][w2][lane]);
        if (!done) {
          const FwdState st = S.st[threadIdx.x];
          T = st.T; C0 = st.C0; C1 = st.C1; C2 = st.C2; D = st.D;
          N0 = st.N0; N1 = st.N1; N2 = st.N2; Ds = st.Ds;
          last = st.last;
          done = st.done != 0u;
        }
      }
    }
    if (inside) {
      const int64_t HW = (int64_t)vw.W * vw.H;
      const int64_t pix = (int64_t)ipy * vw.W + ipx;
      if (A.rgb) {
        float* o = A.rgb + 3 * vw.poff + pix;
        o[0] = __fmaf_rn(T, P.bg[0], C0);
        o[HW] = __fmaf_rn(T, P.bg[1], C1);
        o[2 * HW] = __fmaf_rn(T, P.bg[2], C2);
      }
      if (A.depth) A.depth[vw.poff + pix] = D;
      if (A.normal) {
        float* o = A.normal + 3 * vw.poff + pix;
        o[0] = N0;
        o[HW] = N1;
        o[2 * HW] = N2;
      }
      if (A.alpha) A.alpha[vw.poff + pix] = 1.f - T;
      if constexpr (DIST) A.dist[vw.poff + pix] = Ds;
      A.tfinal[vw.poff + pix] = T;
      A.last[vw.poff + pix] = last;
      A.dfinal[vw.poff + pix] = D;
    }
  }
  if (P.stats) {
    unsigned long long a = n_eval, bb = n_blend;
    for (int o = 16; o > 0; o >>= 1) {
      a += __shfl_xor_sync(0xffffffffu, a, o);
      bb += __shfl_xor_sync(0xffffffffu, bb, o);
    }
    if (lane == 0) {
      atomicAdd(&A.hdr->stat[STAT_FWD_EVAL], a);
      atomicAdd(&A.hdr->stat[STAT_FWD_BLEND], bb);
    }
  }
}

constexpr int SGRAD_STRIDE = 17;

template <bool B>
struct BoolTag {
  static constexpr bool value = B;
};

// Per-entry gradient sums of a chunk in shared memory are kept in fixed point
// (integer shared atomics run at several times the rate of float ones).  Each
// quantity q has, per tile and chunk, a power-of-two scale s_q: a term t is
// added as round(t s_q) when |t s_q| < 2^22 (so a slot, which takes one term
// per pixel of the tile, stays below 2^30), and otherwise straight to the
// gradient record in global memory as a float, so no term is ever clipped.
// The scale comes from an earlier chunk of the same tile (re-derived after
// every other chunk): 2^FIX_BITS over the geometric mean of its nonzero
// per-entry sums, or, where it had none, over the largest term that went to
// global memory.  A tile's first chunk has
// no previous one and accumulates in float; until a quantity has a scale, its
// terms go to global memory.  Scales are exact powers of two, so the only
// rounding is that of each term to the nearest multiple of 1 / s_q: relative
// to the typical entry sum of the tile, 2^-FIX_BITS.
constexpr int FIX_BITS = 15;
constexpr float FIX_LIMIT = 4194304.f;  // 2^22
constexpr float FIX_MAGIC = 12582912.f;  // 1.5 * 2^23: adding it rounds |u| < 2^22 to an integer in the low bits
constexpr int FIX_MAGIC_BITS = 0x4B400000;

// Gradient of one kept (pixel, entry) pair w.r.t. the 16 stored record
// quantities (G_* order) and the depth; `da` is dL/dalpha.  Written without
// branches (selects only): the clamped and the low-pass cases zero the terms
// they do not carry.
__device__ __forceinline__ void pair_grads(const Pair& e, const float4 pp, const float4 qq, float da, float w,
                                           float dC0, float dC1, float dC2, float dD, float dN0, float dN1,
                                           float dN2, float lp_scale, float (&g)[16], float& gz) {
  g[G_R] = w * dC0;
  g[G_G] = w * dC1;
  g[G_B] = w * dC2;
  gz = w * dD;
  g[G_NX] = w * dN0;
  g[G_NY] = w * dN1;
  g[G_NZ] = w * dN2;
  const float dal = e.clamped ? 0.f : da;  // alpha = alpha_max carries no geometry gradient
  g[G_OP] = dal * e.G;
  const float drho = -kLn2 * e.G * (dal * qq.w);
  // object-space branch (rho = (a^2 + b^2) / c^2); its terms are selected away
  // when the low-pass term decides (there c may be 0 and rc infinite)
  const float t2 = 2.f * drho * e.rc * e.rc;
  const float gA = e.obj ? t2 * e.a : 0.f, gB = e.obj ? t2 * e.b : 0.f;
  const float gC = e.obj ? -2.f * drho * e.rho * e.rc : 0.f;
  g[G_P00] = gA * e.dx;
  g[G_P01] = gA * e.dy;
  g[G_P10] = gB * e.dx;
  g[G_P11] = gB * e.dy;
  g[G_P20] = gC * e.dx;
  g[G_P21] = gC * e.dy;
  g[G_P22] = gC;
  const float lp2 = 2.f * lp_scale * drho;
  const float ddx = e.obj ? gA * pp.x + gB * pp.z + gC * qq.x : lp2 * e.dx;
  const float ddy = e.obj ? gA * pp.y + gB * pp.w + gC * qq.y : lp2 * e.dy;
  g[G_CX] = -ddx;
  g[G_CY] = -ddy;
}

// Depth-output terms of a pair under the ray option (where the object-space
// term decides): z' = z p22 / c with c = p20 dx + p21 dy + p22, so for
// dz' = dL/dz': dL/dz = dz' p22 / c, dL/dc = -dz' z' / c, and c carries it to
// p20, p21, p22 and (through dx = px - cx, dy = py - cy) to the center.
// Replaces the plain-depth term gz = w dD that pair_grads wrote.
__device__ __forceinline__ void pair_grads_ray_depth(const Pair& e, const float4 qq, float z, float zp, float dzp,
                                                     float (&g)[16], float& gz) {
  if (!e.obj) return;
  const float dc = -dzp * zp * e.rc;
  gz = dzp * qq.z * e.rc;
  g[G_P22] += dzp * z * e.rc + dc;
  g[G_P20] += dc * e.dx;
  g[G_P21] += dc * e.dy;
  g[G_CX] -= dc * qq.x;
  g[G_CY] -= dc * qq.y;
}

// Dynamic shared memory of the backward kernel (per-pixel arrays indexed by
// the pixel's slot, see k_render_bwd).
template <int NT, int CHUNK, bool DIST>
struct BwdSmem {
  SRecs<CHUNK> rec;
  float grad[CHUNK * SGRAD_STRIDE];
  uint32_t idx[CHUNK];
  uint32_t pbits[NT][CHUNK / 32];  // per pixel: chunk entries whose rect holds it, below its last
  uint16_t pcnt[NT][CHUNK / 32];   // per pixel: set bits in its mask words >= w (from the deepest word)
  float4 up[NT][2];                // per pixel: dC0 dC1 dC2 dD | dN0 dN1 dN2 dA*T_final
  float2 tq[NT];                   // per pixel: (T in front of the deepest unprocessed entry, Q behind it)
  // depth distortion only: per pixel, the sums of w and w z over the entries
  // behind the deepest unprocessed one, and (its upstream gradient, its depth sum D)
  float2 ab[DIST ? NT : 1];
  float2 gdz[DIST ? NT : 1];
  uint32_t gexp[(SGRAD_STRIDE + 1) / 2];  // per quantity, 16 bits: the upper half of this chunk's scale (+inf: none)
  float ginv[SGRAD_STRIDE];        // per quantity: inverse of the scale (0: none)
  uint32_t estat[SGRAD_STRIDE];    // per quantity: (sum of biased exponents of nonzero entry sums) << 10 | their number
  uint32_t ofl[SGRAD_STRIDE];      // per quantity: largest biased exponent of a term added outside the slots
  uint8_t own[NT / 32][32];        // per warp and step: lane of the pixel whose run starts at each position
  int item;
  uint32_t top;
};

// DIST: also the adjoint of the depth distortion D_s = 2 sum_i w_i (z_i A_{i-1}
// - B_{i-1}) (A, B the sums of w and w z in front of i): dD_s/dw_k = 2 (z_k
// A_{k-1} - B_{k-1} + Bsuf_k - z_k Asuf_k) joins the pair's upstream feature
// sum f (so the transmittance terms carry it to alpha), and dD_s/dz_k = 2 w_k
// (A_{k-1} - Asuf_k) its depth gradient; Asuf, Bsuf (the sums behind k) are
// two more segmented prefix sums along the pixel's run, B_{k-1} = D - w_k z_k
// - Bsuf_k with D the pixel's depth sum kept by the forward.
// The reverse pass streams (pixel, entry) pairs.  Per chunk, each warp
// builds its 8x4 patch's per-pixel entry masks with ballots.  Then each warp
// takes 32 pixels spread over the tile (a diagonal interleave, so the warps'
// loads match), one per lane, and lays their pairs end to end -- pixel by pixel,
// each pixel's entries deepest first -- at offsets given by a warp prefix sum
// of the mask population counts.  Every step takes the next 32 positions of
// that stream: a lane finds its pixel from the OR-reduced mask of the run
// starts in the step and its entry by selecting a set bit of the pixel's
// mask, so the stream is never materialised.  Within each pixel's run a
// segmented prefix product of 1/(1 - alpha) recovers the transmittance in
// front of each entry and a segmented prefix sum gives the sum behind it;
// every lane adds its own pair's gradient terms to the entry's shared-memory
// slot, and the last lane of each run stores the pixel's running (T, Q) for
// its next run.
template <int TW, int TH, int CHUNK, bool DIST>
__global__ void __launch_bounds__(TW* TH, (TW * TH == 64) ? (CHUNK <= 64 ? 16 : 8) : 2) k_render_bwd(const RenderArgs A) {
  constexpr int NT = TW * TH, NW = NT / 32, WX = TW / 8, NWD = CHUNK / 32;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  BwdSmem<NT, CHUNK, DIST>& S = *reinterpret_cast<BwdSmem<NT, CHUNK, DIST>*>(smem_raw);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const uint32_t le_mask = (2u << lane) - 1u;  // lanes <= this lane
  const RastParams& P = A.P;
  uint32_t n_eval = 0, n_blend = 0, n_outside = 0;
  uint8_t* own = S.own[wid];
  // a failed binning (instance capacity exceeded) leaves no valid lists
  if (A.hdr->status != 0) return;
  const bool want_n = A.d_normal != nullptr;  // normal terms only when their gradient is asked for
  // The pixel at tile-local (x, y) is laid out by warp (x + 3y) mod NW -- a
  // diagonal interleave, so every warp's 32 pixels spread over the whole tile
  // and the warps' loads match -- as that warp's pixel number
  // y * (TW / NW) + x / NW.  Per-pixel shared arrays are indexed by slot =
  // warp * 32 + number, so one warp's pixels sit in consecutive slots.
  constexpr int PR = TW / NW;  // pixels per row of one warp
  static_assert(TW % NW == 0 && PR * TH == 32, "each warp lays out 32 pixels");
  static_assert(NT <= 256, "a fixed-point slot takes one term below 2^22 per pixel and must stay below 2^30");
  const int lx = (wid % WX) * 8 + (lane & 7), ly = (wid / WX) * 4 + (lane >> 3);
  const int myslot = ((lx + 3 * ly) % NW) * 32 + ly * PR + lx / NW;  // slot of this thread's own pixel
  const int mine = wid * 32 + lane;                                  // slot of the pixel this lane lays out
  for (int i = threadIdx.x; i < CHUNK * SGRAD_STRIDE; i += NT) S.grad[i] = 0.f;
  for (;;) {
    if (threadIdx.x == 0) S.item = (int)atomicAdd(&A.hdr->queue_bwd, 1u);
    __syncthreads();
    const int item = S.item;
    if (item >= A.T) break;
    const int t = (int)__ldg(A.order + item);
    const int v = find_view_by_tile(A.views, A.V, t);
    const DView& vw = A.views[v];
    const int lt = t - vw.tile_base;
    const int tx0 = (lt % vw.tiles_x) * TW, ty0 = (lt / vw.tiles_x) * TH;
    const int bx = tx0 + (wid % WX) * 8, by = ty0 + (wid / WX) * 4;
    const int ipx = bx + (lane & 7), ipy = by + (lane >> 3);
    const bool inside = ipx < vw.W && ipy < vw.H;
    const uint2 range = __ldg(A.ranges + t);
    const int64_t HW = (int64_t)vw.W * vw.H;
    uint32_t my_last = range.x;
    float T = 1.f, Q = 0.f;
    float As = 0.f, Bs = 0.f;  // distortion: sums of w and w z behind the deepest unprocessed entry
    bool fixed = false;  // a tile's first chunk accumulates in float, every later one in fixed point
    bool restat = true;  // the scales are re-derived after every other chunk
    {
      float4 u0 = make_float4(0.f, 0.f, 0.f, 0.f), u1 = u0;
      if (inside) {
        const int64_t pix = (int64_t)ipy * vw.W + ipx;
        my_last = A.last[vw.poff + pix];
        T = A.tfinal[vw.poff + pix];
        if (A.d_rgb) {
          const float* g = A.d_rgb + 3 * vw.poff + pix;
          u0.x = g[0]; u0.y = g[HW]; u0.z = g[2 * HW];
        }
        if (A.d_depth) u0.w = A.d_depth[vw.poff + pix];
        if (A.d_normal) {
          const float* g = A.d_normal + 3 * vw.poff + pix;
          u1.x = g[0]; u1.y = g[HW]; u1.z = g[2 * HW];
        }
        if (A.d_alpha) u1.w = A.d_alpha[vw.poff + pix] * T;
        Q = T * (u0.x * P.bg[0] + u0.y * P.bg[1] + u0.z * P.bg[2]);
      }
      S.up[myslot][0] = u0;
      S.up[myslot][1] = u1;
      if constexpr (DIST) {
        const int64_t pix = (int64_t)ipy * vw.W + ipx;
        S.gdz[myslot] = inside ? make_float2(A.d_dist[vw.poff + pix], A.dfinal[vw.poff + pix]) : make_float2(0.f, 0.f);
      }
    }
    if (threadIdx.x == 0) S.top = range.x;
    if (threadIdx.x < (SGRAD_STRIDE + 1) / 2) S.gexp[threadIdx.x] = 0x7f807f80u;
    if (threadIdx.x < SGRAD_STRIDE) {
      S.ginv[threadIdx.x] = 0.f;
      S.estat[threadIdx.x] = 0u;
      S.ofl[threadIdx.x] = 0u;
    }
    __syncthreads();
    if (my_last > range.x) atomicMax(&S.top, my_last);
    __syncthreads();
    const uint32_t top = S.top;
    // chunks run back from the tile's largest `last`, rounded up to a whole
    // word of the forward's blended-pair masks (words start every 32 entries
    // from the tile's first), so every chunk covers whole words and all but
    // the front one are full (the deepest chunk sets the first fixed-point
    // scales); entries at or past `top` are blended nowhere and not staged
    const int64_t woff = (int64_t)(range.x >> 5) + t;
    const int64_t hi0 = (int64_t)range.x + (((int64_t)top - (int64_t)range.x + 31) & ~(int64_t)31);
    for (int64_t hi = hi0; hi > (int64_t)range.x; hi -= CHUNK) {
      const int64_t lo = max64((int64_t)range.x, hi - CHUNK);
      const int count = (int)(min64(hi, (int64_t)top) - lo);
      const int nwd = (count + 31) >> 5;
      const bool act = inside && (int64_t)my_last > lo;
      stage_chunk_seq<NT, CHUNK>(A, vw, tx0, ty0, TW, TH, lo, count, S.rec, S.idx);
      // per-pixel masks of this chunk: the entries the forward blended at the pixel
      {
        const int64_t w0 = woff + ((lo - (int64_t)range.x) >> 5);
        const bool bm_ok = s2d_check(w0 + nwd <= A.bmask_words, A.hdr);
        const uint32_t* bm = A.bmask + w0 * NT + threadIdx.x;
        int pc[NWD];
#pragma unroll
        for (int wd = 0; wd < NWD; wd++) {
          uint32_t m = 0;
          if (wd < nwd) {
            m = (act && bm_ok) ? __ldcs(bm + (int64_t)wd * NT) : 0u;  // read once
            S.pbits[myslot][wd] = m;
          }
          pc[wd] = __popc(m);
        }
        int acc = 0;
#pragma unroll
        for (int wd = NWD - 1; wd >= 0; wd--) {
          acc += pc[wd];
          S.pcnt[myslot][wd] = (uint16_t)acc;
        }
      }
      if (act) S.tq[myslot] = make_float2(T, Q);
      if constexpr (DIST)
        if (act) S.ab[myslot] = make_float2(As, Bs);
      __syncthreads();
      // this warp's stream: its pixels' pairs end to end
      const uint32_t cnt = S.pcnt[mine][0];
      uint32_t incl = cnt;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
      }
      const uint32_t myoff = incl - cnt;
      const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
      // the chunk's steps, compiled once per way of accumulating the sums
      auto steps = [&](auto fixed_tag) {
      constexpr bool FIXED = decltype(fixed_tag)::value;
      int carry = 0;  // lane of the pixel whose run reaches the previous step's last position
      uint32_t gexp[(SGRAD_STRIDE + 1) / 2];  // this chunk's scales, in registers
#pragma unroll
      for (int w = 0; w < (SGRAD_STRIDE + 1) / 2; w++) gexp[w] = FIXED ? S.gexp[w] : 0u;
      for (uint32_t base = 0; base < total; base += 32) {
        const bool starts_here = cnt > 0 && myoff >= base && myoff < base + 32;
        if (starts_here) own[myoff - base] = (uint8_t)lane;
        const uint32_t M = __reduce_or_sync(0xffffffffu, starts_here ? (1u << (myoff - base)) : 0u);
        __syncwarp();
        const bool has = base + lane < total;
        const uint32_t below = M & le_mask;
        const int ol = below ? (int)own[31 - __clz(below)] : carry;
        carry = __shfl_sync(0xffffffffu, ol, 31);
        const uint32_t ooff = __shfl_sync(0xffffffffu, myoff, ol);
        const int ps = wid * 32 + ol;  // the pixel's slot
        int j = 0;
        if (has) {
          // entry: the q-th set bit of the pixel's mask counted from the
          // deepest; its word is the last w with pcnt[w] > q
          const int q = (int)(base + lane - ooff);
          const uint32_t* pw32 = reinterpret_cast<const uint32_t*>(S.pcnt[ps]);
          int wd = -1, cin = 0;
#pragma unroll
          for (int h = 0; h < NWD / 2; h++) {
            const uint32_t two = pw32[h];
            const int c0 = (int)(two & 0xffffu), c1 = (int)(two >> 16);
            if (c0 > q) { wd = 2 * h; cin = c0; }
            if (c1 > q) { wd = 2 * h + 1; cin = c1; }
          }
          j = wd * 32 + nth_set_bit(S.pbits[ps][wd], cin - q);
        }
        const bool start = has && (lane == 0 || ((M >> lane) & 1u));
        const bool end = has && (lane == 31 || base + lane + 1 == total || ((M >> (lane + 1)) & 1u));
        const uint32_t starts = __ballot_sync(0xffffffffu, start);
        const int s0 = 31 - __clz(starts & le_mask);
        // lanes past the stream's end (last step only) evaluate a valid
        // dummy pair and are masked out by `kept`
        const float2 tq = S.tq[ps];
        const float4 u0 = S.up[ps][0], u1 = S.up[ps][1];
        const int qy = ol / PR, qx = ((wid - 3 * qy) % NW + NW) % NW + (ol % PR) * NW;
        Pair e;
        eval_pair(S.rec.c[j], S.rec.p[j], S.rec.q[j], (float)(tx0 + qx) + 0.5f, (float)(ty0 + qy) + 0.5f, P.lp_scale,
                  P.alpha_max, e);
        const float alpha = e.alpha;
        const bool kept = has && alpha >= P.alpha_min;
        const float iom = kept ? rcp_approx(__fsub_rn(1.f, alpha)) : 1.f;
        // segmented prefix product: transmittance in front of this entry
        float x = iom;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const float y = __shfl_up_sync(0xffffffffu, x, o);
          x = (lane - o >= s0) ? __fmul_rn(x, y) : x;
        }
        const float Tb = tq.x * x;
        const float w = kept ? alpha * Tb : 0.f;
        const float4 col = S.rec.col[j];
        const float4 qj = S.rec.q[j];
        const float zp = pair_depth(e, col.w, qj.z, P.depth_ray);
        float f = fmaf(u0.x, col.x, fmaf(u0.y, col.y, fmaf(u0.z, col.z, u0.w * zp)));
        if (want_n) {
          const float4 nrm = S.rec.n[j];
          f = fmaf(u1.x, nrm.x, fmaf(u1.y, nrm.y, fmaf(u1.z, nrm.z, f)));
        }
        // distortion only: its depth gradient; the run's sums of w and w z; the pixel's carried sums
        float dzd = 0.f;
        [[maybe_unused]] float sa = 0.f, sb = 0.f;
        [[maybe_unused]] float2 ab = make_float2(0.f, 0.f);
        if constexpr (DIST) {
          // segmented prefix sums of w and w z: with the pixel's carried
          // sums, those behind this pair
          sa = w;
          sb = w * zp;
#pragma unroll
          for (int o = 1; o < 32; o <<= 1) {
            const float ya = __shfl_up_sync(0xffffffffu, sa, o);
            const float yb = __shfl_up_sync(0xffffffffu, sb, o);
            const bool in = lane - o >= s0;
            sa = in ? sa + ya : sa;
            sb = in ? sb + yb : sb;
          }
          ab = S.ab[ps];
          const float2 gd = S.gdz[ps];
          const float Asuf = ab.x + (sa - w), Bsuf = ab.y + (sb - w * zp);
          const float Ap = 1.f - Tb, Bp = gd.y - w * zp - Bsuf;  // the sums in front of this pair
          f = fmaf(gd.x * 2.f, zp * Ap - Bp + Bsuf - zp * Asuf, f);
          dzd = gd.x * 2.f * w * (Ap - Asuf);
        }
        const float wf = w * f;
        // segmented prefix sum: the sum over entries behind this one
        float sum = wf;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const float y = __shfl_up_sync(0xffffffffu, sum, o);
          sum = (lane - o >= s0) ? sum + y : sum;
        }
        const float Qb = tq.y + (sum - wf);
        n_eval += has ? 1u : 0u;
        n_blend += kept ? 1u : 0u;
        const float da = Tb * f - (Qb - u1.w) * iom;
        float g[16];
        float gz;
        pair_grads(e, S.rec.p[j], qj, da, w, u0.x, u0.y, u0.z, u0.w, u1.x, u1.y, u1.z, P.lp_scale, g, gz);
        if constexpr (DIST) gz += dzd;
        if (P.depth_ray) pair_grads_ray_depth(e, qj, col.w, zp, w * u0.w + dzd, g, gz);
        if (kept) {
          float* sg = S.grad + j * SGRAD_STRIDE;
          [[maybe_unused]] float umax = 0.f;  // fixed point: the largest scaled term
#pragma unroll
          for (int q = 0; q < SGRAD_STRIDE; q++) {
            if (!want_n && q >= G_NX && q <= G_NZ) continue;  // no normal gradient requested
            const float t = q < 16 ? g[q] : gz;
            if constexpr (FIXED) {
              // no scale yet (+inf) makes u infinite (or NaN for t = 0).
              // Branch-free: a term outside this chunk's range adds zero here;
              // the pair's largest |u| tells whether any did (fmaxf drops NaN).
              const uint32_t w2 = gexp[q >> 1];
              const float u = t * __uint_as_float((q & 1) ? (w2 & 0xffff0000u) : (w2 << 16));
              const bool in = fabsf(u) < FIX_LIMIT;
              atomicAdd(reinterpret_cast<int*>(sg + q),
                        __float_as_int(__fadd_rn(in ? u : 0.f, FIX_MAGIC)) - FIX_MAGIC_BITS);
              umax = fmaxf(umax, fabsf(u));
            } else {
              if (t != 0.f) atomicAdd(sg + q, t);
            }
          }
          if constexpr (FIXED) {
            if (!(umax < FIX_LIMIT)) {  // some term outside this chunk's range (or not finite): added exactly
              float* dst = A.rgrad + (int64_t)S.idx[j] * GRAD_F;
#pragma unroll
              for (int q = 0; q < SGRAD_STRIDE; q++) {
                if (!want_n && q >= G_NX && q <= G_NZ) continue;
                const float t = q < 16 ? g[q] : gz;
                const uint32_t w2 = gexp[q >> 1];
                const float u = t * __uint_as_float((q & 1) ? (w2 & 0xffff0000u) : (w2 << 16));
                if (fabsf(u) < FIX_LIMIT || t == 0.f) continue;
                atomicAdd(dst + q, t);
                atomicMax(&S.ofl[q], (__float_as_uint(t) >> 23) & 0xffu);
                n_outside++;
              }
            }
          }
        }
        __syncwarp();
        if (end) S.tq[ps] = make_float2(Tb, tq.y + sum);
        if constexpr (DIST)
          if (end) S.ab[ps] = make_float2(ab.x + sa, ab.y + sb);
        __syncwarp();
      }
      };
      if (fixed)
        steps(BoolTag<true>{});
      else
        steps(BoolTag<false>{});
      __syncthreads();
      if (act) {
        const float2 tq = S.tq[myslot];
        T = tq.x;
        Q = tq.y;
        if constexpr (DIST) {
          As = S.ab[myslot].x;
          Bs = S.ab[myslot].y;
        }
      }
      // flush this chunk's per-entry sums (decoded from fixed point where the
      // chunk used it): one set of vector atomics per entry; then gather the
      // exponent statistics the next chunk's scales come from
      for (int j0 = 0; j0 < count; j0 += NT) {
        const int jj = j0 + (int)threadIdx.x;
        const bool valid = jj < count;
        uint32_t* sg = reinterpret_cast<uint32_t*>(S.grad) + (valid ? jj : 0) * SGRAD_STRIDE;
        float v[SGRAD_STRIDE];
        float acc = 0.f;
#pragma unroll
        for (int q = 0; q < SGRAD_STRIDE; q++) {
          const uint32_t raw = valid ? sg[q] : 0u;
          v[q] = fixed ? (float)(int)raw * S.ginv[q] : __uint_as_float(raw);
          acc += fabsf(v[q]);
        }
        if (valid && acc != 0.f) {
          float* dst = A.rgrad + (int64_t)S.idx[jj] * GRAD_F;
          red_add_v4(dst + 0, v[0], v[1], v[2], v[3]);
          red_add_v4(dst + 4, v[4], v[5], v[6], v[7]);
          red_add_v4(dst + 8, v[8], v[9], v[10], v[11]);
          red_add_v4(dst + 12, v[12], v[13], v[14], v[15]);
          atomicAdd(dst + 16, v[16]);
#pragma unroll
          for (int q = 0; q < SGRAD_STRIDE; q++) sg[q] = 0u;
        }
        if (restat) {
#pragma unroll
          for (int q = 0; q < SGRAD_STRIDE; q++) {
            const uint32_t e = v[q] != 0.f ? ((__float_as_uint(v[q]) >> 23) & 0xffu) << 10 | 1u : 0u;
            const uint32_t es = __reduce_add_sync(0xffffffffu, e);
            if (lane == 0 && es) atomicAdd(&S.estat[q], es);
          }
        }
      }
      __syncthreads();
      // next chunk's scales: 2^(FIX_BITS - e) for the mean unbiased exponent e
      // of this chunk's nonzero sums (or, with none, for the largest term that
      // went outside); a quantity with neither keeps its scale
      if (restat && threadIdx.x < SGRAD_STRIDE) {
        const uint32_t st = S.estat[threadIdx.x], c = st & 1023u, of = S.ofl[threadIdx.x];
        const int m = c ? (int)((st >> 10) / c) : (of ? (int)of : -1);
        if (m >= 0) {
          const int es = 254 + FIX_BITS - m, ei = m - FIX_BITS;
          const bool ok = es >= 1 && es <= 254 && ei >= 1 && ei <= 254;
          S.ginv[threadIdx.x] = ok ? __uint_as_float((uint32_t)ei << 23) : 0.f;
          reinterpret_cast<uint16_t*>(S.gexp)[threadIdx.x] = (uint16_t)((ok ? es : 255) << 7);
        }
        S.estat[threadIdx.x] = 0u;
        S.ofl[threadIdx.x] = 0u;
      }
      fixed = true;
      restat = !restat;
    }
  }
  if (P.stats) {
    unsigned long long a = n_eval, bb = n_blend;
    for (int o = 16; o > 0; o >>= 1) {
      a += __shfl_xor_sync(0xffffffffu, a, o);
      bb += __shfl_xor_sync(0xffffffffu, bb, o);
    }
    if (lane == 0) {
      atomicAdd(&A.hdr->stat[STAT_BWD_EVAL], a);
      atomicAdd(&A.hdr->stat[STAT_BWD_BLEND], bb);
    }
    unsigned long long o = n_outside;
    for (int sh = 16; sh > 0; sh >>= 1) o += __shfl_xor_sync(0xffffffffu, o, sh);
    if (lane == 0 && o) atomicAdd(&A.hdr->stat[STAT_BWD_OUTSIDE], o);
  }
}

// ---------------------------------------------------------------------------
// Error attribution for pruning (Sec. 4.3, "Map Fusion": primitives that
// contribute to pixels with high RGB or depth error are removed).  A surfel
// contributes to a pixel when the pixel blends it: an entry of the pixel's
// tile list before the pixel's `last` (left by the forward) whose alpha there
// is at least alpha_min.  For every such pair the surfel's attributed error
// is raised to the pixel's error.  Errors are compared as the bit patterns of
// non-negative floats (ordered like the values), first per tile in shared
// memory, then once per (tile, surfel) with a global atomicMax.
// ---------------------------------------------------------------------------
template <int TW, int TH>
__global__ void __launch_bounds__(TW* TH) k_max_error(const RenderArgs A, const float* __restrict__ err,
                                                      uint32_t* __restrict__ max_err) {
  constexpr int NT = TW * TH, WX = TW / 8, MCH = 256;  // entries per pass
  __shared__ uint32_t emax[MCH];  // per entry of the pass: largest error bits of a pixel that blends it
  __shared__ int s_item;
  __shared__ uint32_t s_top;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (A.hdr->status != 0) return;
  for (;;) {
    if (threadIdx.x == 0) s_item = (int)atomicAdd(&A.hdr->queue_aux, 1u);
    __syncthreads();
    const int item = s_item;
    if (item >= A.T) break;
    const int t = (int)__ldg(A.order + item);
    const int v = find_view_by_tile(A.views, A.V, t);
    const DView& vw = A.views[v];
    const int lt = t - vw.tile_base;
    const int tx0 = (lt % vw.tiles_x) * TW, ty0 = (lt / vw.tiles_x) * TH;
    const int ipx = tx0 + (wid % WX) * 8 + (lane & 7), ipy = ty0 + (wid / WX) * 4 + (lane >> 3);
    const bool inside = ipx < vw.W && ipy < vw.H;
    const uint2 range = __ldg(A.ranges + t);
    uint32_t my_last = range.x, ebits = 0u;
    if (inside) {
      const int64_t pix = vw.poff + (int64_t)ipy * vw.W + ipx;
      const float e = err[pix];
      ebits = e > 0.f ? __float_as_uint(e) : 0u;  // negative and NaN errors count as zero
      if (ebits) my_last = A.last[pix];
    }
    if (threadIdx.x == 0) s_top = range.x;
    __syncthreads();
    if (my_last > range.x) atomicMax(&s_top, my_last);
    __syncthreads();
    const uint32_t top = s_top;
    const int64_t woff = (int64_t)(range.x >> 5) + t;
    for (int64_t lo = range.x; lo < (int64_t)top; lo += MCH) {
      const int count = (int)min64(MCH, (int64_t)top - lo);
      const int nwd = (count + 31) >> 5;
      for (int j = threadIdx.x; j < count; j += NT) emax[j] = 0u;
      __syncthreads();
      const int64_t w0 = woff + ((lo - (int64_t)range.x) >> 5);
      if (ebits && s2d_check(w0 + nwd <= A.bmask_words, A.hdr)) {
        for (int wd = 0; wd < nwd; wd++) {
          uint32_t m = __ldg(A.bmask + (w0 + wd) * NT + threadIdx.x);
          while (m) {
            const int j = wd * 32 + __ffs(m) - 1;
            m &= m - 1;
            atomicMax(&emax[j], ebits);
          }
        }
      }
      __syncthreads();
      for (int j = threadIdx.x; j < count; j += NT) {
        const uint32_t m = emax[j];
        if (!m) continue;
        const uint32_t sj = __ldg(A.vals + lo + j);
        if (s2d_check((int64_t)sj >= vw.soff && (int64_t)sj < vw.soff + vw.scnt, A.hdr)) atomicMax(max_err + sj, m);
      }
      __syncthreads();
    }
  }
}

// ---------------------------------------------------------------------------
// launch
// ---------------------------------------------------------------------------
static RenderArgs make_args(const Layout& L, const RastParams& P, char* ws, const uint32_t* vals) {
  RenderArgs A;
  A.views = reinterpret_cast<const DView*>(ws + L.views);
  A.V = L.V;
  A.T = L.T;
  A.ranges = reinterpret_cast<const uint2*>(ws + L.ranges);
  A.order = reinterpret_cast<const uint32_t*>(ws + L.tile_order);
  A.vals = vals;
  A.records = reinterpret_cast<const float4*>(ws + L.records);
  A.rcopy = reinterpret_cast<float4*>(ws + L.rcopy);
  A.bmask = reinterpret_cast<uint32_t*>(ws + L.bmask);
  A.bmask_words = L.bmask_words;
  A.rgrad = reinterpret_cast<float*>(ws + L.rgrad);
  A.P = P;
  A.hdr = reinterpret_cast<Header*>(ws + L.header);
  A.tfinal = reinterpret_cast<float*>(ws + L.tfinal);
  A.last = reinterpret_cast<uint32_t*>(ws + L.last);
  A.dfinal = reinterpret_cast<float*>(ws + L.dfinal);
  A.rgb = A.depth = A.normal = A.alpha = A.dist = nullptr;
  A.d_rgb = A.d_depth = A.d_normal = A.d_alpha = A.d_dist = nullptr;
  return A;
}

template <typename K>
static int persistent_grid(K kernel, int threads, size_t smem, int64_t work) {
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem);
  if (per_sm < 1) per_sm = 1;
  int64_t g = (int64_t)per_sm * sm_count();
  if (g > work) g = work;
  return (int)(g < 1 ? 1 : g);
}

template <int TW, int TH, int CHUNK, bool DIST>
static cudaError_t run_fwd_k(const RenderArgs& A, cudaStream_t st) {
  auto k = k_render_fwd<TW, TH, CHUNK, DIST>;
  constexpr size_t smem = sizeof(FwdSmem<TW * TH, CHUNK>);
  static int grid = -1;
  static int64_t grid_T = -1;
  if (grid < 0) cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (grid < 0 || grid_T != A.T) {
    grid = persistent_grid(k, TW * TH, smem, A.T);
    grid_T = A.T;
  }
  k<<<grid, TW * TH, smem, st>>>(A);
  count_launches(1);
  return cudaGetLastError();
}
template <int TW, int TH, int CHUNK>
static cudaError_t run_fwd(const RenderArgs& A, cudaStream_t st) {
  return A.dist ? run_fwd_k<TW, TH, CHUNK, true>(A, st) : run_fwd_k<TW, TH, CHUNK, false>(A, st);
}
template <int TW, int TH, int CHUNK, bool DIST>
static cudaError_t run_bwd_k(const RenderArgs& A, cudaStream_t st) {
  auto k = k_render_bwd<TW, TH, CHUNK, DIST>;
  constexpr size_t smem = sizeof(BwdSmem<TW * TH, CHUNK, DIST>);
  static int grid = -1;
  static int64_t grid_T = -1;
  if (grid < 0) cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (grid < 0 || grid_T != A.T) {
    grid = persistent_grid(k, TW * TH, smem, A.T);
    grid_T = A.T;
  }
  k<<<grid, TW * TH, smem, st>>>(A);
  count_launches(1);
  return cudaGetLastError();
}
template <int TW, int TH, int CHUNK>
static cudaError_t run_bwd(const RenderArgs& A, cudaStream_t st) {
  return A.d_dist ? run_bwd_k<TW, TH, CHUNK, true>(A, st) : run_bwd_k<TW, TH, CHUNK, false>(A, st);
}

template <int TW, int TH>
static cudaError_t run_max_error(const RenderArgs& A, const float* err, uint32_t* max_err, cudaStream_t st) {
  auto k = k_max_error<TW, TH>;
  static int grid = -1;
  static int64_t grid_T = -1;
  if (grid < 0 || grid_T != A.T) {
    grid = persistent_grid(k, TW * TH, 0, A.T);
    grid_T = A.T;
  }
  k<<<grid, TW * TH, 0, st>>>(A, err, max_err);
  count_launches(1);
  return cudaGetLastError();
}

#define S2D_DISPATCH(FN, TWv, THv, CH, ...)                                   \
  do {                                                                        \
    if (TWv == 16 && THv == 16) {                                             \
      if (CH == 64) return FN<16, 16, 64>(__VA_ARGS__);                       \
      if (CH == 128) return FN<16, 16, 128>(__VA_ARGS__);                     \
      if (CH == 256) return FN<16, 16, 256>(__VA_ARGS__);                     \
      if (CH == 512) return FN<16, 16, 512>(__VA_ARGS__);                     \
    } else if (TWv == 8 && THv == 8) {                                        \
      if (CH == 64) return FN<8, 8, 64>(__VA_ARGS__);                         \
      if (CH == 128) return FN<8, 8, 128>(__VA_ARGS__);                       \
      if (CH == 256) return FN<8, 8, 256>(__VA_ARGS__);                       \
    } else if (TWv == 32 && THv == 8) {                                       \
      if (CH == 64) return FN<32, 8, 64>(__VA_ARGS__);                        \
      if (CH == 128) return FN<32, 8, 128>(__VA_ARGS__);                      \
      if (CH == 256) return FN<32, 8, 256>(__VA_ARGS__);                      \
      if (CH == 512) return FN<32, 8, 512>(__VA_ARGS__);                      \
    }                                                                         \
    return cudaErrorInvalidValue;                                             \
  } while (0)

cudaError_t launch_render_fwd(const Layout& L, const RastParams& P, int chunk, char* ws, const uint32_t* vals,
                              float* rgb, float* depth, float* normal, float* alpha, float* dist, cudaStream_t st) {
  if (L.T <= 0) return cudaSuccess;
  RenderArgs A = make_args(L, P, ws, vals);
  A.rgb = rgb;
  A.depth = depth;
  A.normal = normal;
  A.alpha = alpha;
  A.dist = dist;
  Header* hdr = reinterpret_cast<Header*>(ws + L.header);
  cudaError_t e = cudaMemsetAsync(&hdr->queue_fwd, 0, sizeof(uint32_t), st);
  if (e != cudaSuccess) return e;
  S2D_DISPATCH(run_fwd, P.tile_w, P.tile_h, chunk, A, st);
}

cudaError_t launch_render_bwd(const Layout& L, const RastParams& P, int chunk, char* ws, const uint32_t* vals,
                              const float* d_rgb, const float* d_depth, const float* d_normal,
                              const float* d_alpha, const float* d_dist, cudaStream_t st) {
  if (L.T <= 0) return cudaSuccess;
  RenderArgs A = make_args(L, P, ws, vals);
  A.d_rgb = d_rgb;
  A.d_depth = d_depth;
  A.d_normal = d_normal;
  A.d_alpha = d_alpha;
  A.d_dist = d_dist;
  Header* hdr = reinterpret_cast<Header*>(ws + L.header);
  cudaError_t e = cudaMemsetAsync(&hdr->queue_bwd, 0, sizeof(uint32_t), st);
  if (e != cudaSuccess) return e;
  S2D_DISPATCH(run_bwd, P.tile_w, P.tile_h, chunk, A, st);
}

cudaError_t launch_max_error(const Layout& L, const RastParams& P, int chunk, char* ws, const uint32_t* vals,
                             const float* err, float* max_err, cudaStream_t st) {
  if (L.T <= 0) return cudaSuccess;
  RenderArgs A = make_args(L, P, ws, vals);
  Header* hdr = reinterpret_cast<Header*>(ws + L.header);
  cudaError_t e = cudaMemsetAsync(&hdr->queue_aux, 0, sizeof(uint32_t), st);
  if (e != cudaSuccess) return e;
  uint32_t* m = reinterpret_cast<uint32_t*>(max_err);
  if (P.tile_w == 8 && P.tile_h == 8) return run_max_error<8, 8>(A, err, m, st);
  if (P.tile_w == 16 && P.tile_h == 16) return run_max_error<16, 16>(A, err, m, st);
  if (P.tile_w == 32 && P.tile_h == 8) return run_max_error<32, 8>(A, err, m, st);
  return cudaErrorInvalidValue;
}

}  // namespace s2d
