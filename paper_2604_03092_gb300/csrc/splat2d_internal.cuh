// Internal declarations shared by the CUDA translation units of libsplat2d.
// Not part of the public ABI (see include/splat2d.h).
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

#include "splat2d.h"

namespace s2d {

// ---------------------------------------------------------------------------
// Device-side tables (written into the workspace by splat2d_preprocess)
// ---------------------------------------------------------------------------

// One camera, 128 bytes.
struct DView {
  int32_t W, H;
  float fx, fy, cx, cy;
  float R[9];
  float t[3];
  int64_t soff;       // surfel range [soff, soff + scnt)
  int64_t scnt;
  int64_t poff;       // first pixel in the packed images
  int64_t rbase;      // first render record of this view
  int32_t tile_base;  // first global tile of this view
  int32_t tiles_x, tiles_y;
  int32_t group;
  float ifx, ify;  // 1 / fx and 1 / fy, IEEE quotients computed on the host
};
static_assert(sizeof(DView) == 128, "DView layout");

// Consecutive views that render the same surfel range: the preprocess runs
// one thread per surfel of the range and loops over these views, so the
// surfel's parameters are read once per group instead of once per view.
struct DGroup {
  int64_t soff, scnt;  // surfel range
  int64_t wbase;       // first work item of this group
  int32_t v0, v1;      // views [v0, v1)
};
static_assert(sizeof(DGroup) == 32, "DGroup layout");

// Status word and counters at the start of the workspace (256 bytes).
struct Header {
  int32_t status;           // SPLAT2D_OK or a device error code
  uint32_t timeout_where;
  unsigned long long needed;     // instances the binning needed
  unsigned long long n_inst;     // instances binned (0 after an overflow)
  unsigned long long n_visible;  // visible (view, surfel) pairs
  uint32_t queue_fwd, queue_bwd; // persistent work queues
  unsigned long long stat[8];    // pair counters, see STAT_*
  uint32_t queue_aux;            // work queue of the error-attribution pass
  uint32_t pad[31];
};
static_assert(sizeof(Header) <= 256, "Header layout");
enum { STAT_FWD_EVAL = 0, STAT_FWD_BLEND = 1, STAT_BWD_EVAL = 2, STAT_BWD_BLEND = 3, STAT_BWD_OUTSIDE = 4 };

// Render record: 80 bytes per visible (view, surfel).  Geometry is stored
// relative to the projected center c = (cx_hi + cx_lo, cy_hi + cy_lo), kept
// as a float-float pair so that pixel offsets dx = px - c are exact to
// ~1e-7 px.  For a pixel offset (dx, dy):
//    a = p00 dx + p01 dy,  b = p10 dx + p11 dy,  c = p22 + p20 dx + p21 dy
//    rho' = (a^2 + b^2) / c^2 = (u^2 + v^2) * log2(e) / 2
// so the object-space Gaussian is exp2(-rho').
//   f0 = (cx_hi, cy_hi, pack_half2(cx_lo, cy_lo) * 2^16 scaled, opacity)
//   f1 = (p00, p01, p10, p11)
//   f2 = (p20, p21, p22, r)
//   f3 = (g, b, nx, ny)
//   f4 = (nz, z, rect x0 | y0 << 16, rect x1 | y1 << 16)   (pixel rect, inclusive)
constexpr int REC_F4 = 5;
// Gradient record: 80 bytes per (view, surfel): the derivatives of the loss
// with respect to the stored quantities, in this order (17 used):
enum {
  G_P00 = 0, G_P01, G_P10, G_P11, G_P20, G_P21, G_P22, G_CX,
  G_CY, G_OP, G_R, G_G, G_B, G_NX, G_NY, G_NZ,  // 16 reduced together
  G_Z,                                          // the 17th, reduced separately
  G_USED
};
constexpr int GRAD_F = 20;  // floats per gradient record (5 float4)

constexpr float kLog2e = 1.4426950408889634f;
constexpr float kLn2 = 0.69314718055994531f;

// ---------------------------------------------------------------------------
// Workspace layout (identical on every call for the same problem)
// ---------------------------------------------------------------------------
struct Layout {
  size_t header, views, groups, ntiles, bins, records, rgrad, keys0, keys1, vals0, vals1, sort_hist, ranges,
      tile_count, tile_cursor, tile_order, tile_hist, tile_class, tfinal, last, dfinal, rcopy, bmask, total;
  int64_t bmask_words;  // 32-entry words of blended-pair masks (each holds one word per tile pixel)
  int64_t R, T, P, cap;
  int64_t n_work;     // sum over view groups of the surfel range sizes
  int32_t V, G;
  bool groups_overlap;  // some surfel belongs to two groups
  int32_t sort_blocks;
  int32_t key_bits;
};

constexpr int SORT_THREADS = 256;
constexpr int SORT_IPT = 8;
constexpr int SORT_TILE = SORT_THREADS * SORT_IPT;  // 2048 keys per tile
constexpr int SORT_MAX_BLOCKS = 1024;
constexpr int ORDER_BINS = 64;   // cost buckets of the work queue order

__host__ __device__ __forceinline__ int64_t min64(int64_t a, int64_t b) { return a < b ? a : b; }
__host__ __device__ __forceinline__ int64_t max64(int64_t a, int64_t b) { return a > b ? a : b; }

// Host helpers (api.cu)
bool compute_layout(const splat2d_config* cfg, const splat2d_problem* prob, Layout* L);
std::atomic<uint64_t>& launch_counter();

// Per-launch constants
struct RastParams {
  float alpha_min, alpha_max, t_min, z_near;
  float lp_scale;   // log2(e) / (2 sigma_lp^2), 0 if the low-pass term is off
  float lp_r;       // sigma_lp (pixels) for the extent
  float bg[3];
  int32_t tile_w, tile_h;
  int32_t stats;    // keep pair counters
  int32_t fwd_tail; // forward: share the tile's pixels across warps below this many active per warp
  int32_t depth_ray; // depth output from the ray-splat intersection (SPLAT2D_FLAG_DEPTH_RAY)
};

// ---------------------------------------------------------------------------
// Launch wrappers (defined in the .cu files)
// ---------------------------------------------------------------------------
cudaError_t launch_upload(const void* host_src, size_t bytes, void* dst, cudaStream_t st);
cudaError_t launch_preprocess(const splat2d_surfels* S, const Layout& L, const RastParams& P, char* ws,
                              cudaStream_t st);
cudaError_t launch_bin_tiles(const Layout& L, const RastParams& P, char* ws, cudaStream_t st);
cudaError_t launch_order(const Layout& L, char* ws, cudaStream_t st);
cudaError_t launch_sort(uint64_t* keys0, uint32_t* vals0, uint64_t* keys1, uint32_t* vals1,
                        const unsigned long long* n_dev, int64_t n_max, int key_bits, uint32_t* hist,
                        int sort_blocks, int* final_buffer, cudaStream_t st);
cudaError_t launch_render_fwd(const Layout& L, const RastParams& P, int chunk, char* ws, const uint32_t* vals,
                              float* rgb, float* depth, float* normal, float* alpha, float* dist, cudaStream_t st);
cudaError_t launch_render_bwd(const Layout& L, const RastParams& P, int chunk, char* ws, const uint32_t* vals,
                              const float* d_rgb, const float* d_depth, const float* d_normal,
                              const float* d_alpha, const float* d_dist, cudaStream_t st);
cudaError_t launch_max_error(const Layout& L, const RastParams& P, int chunk, char* ws, const uint32_t* vals,
                             const float* err, float* max_err, cudaStream_t st);
cudaError_t launch_accum_gate(const float* alpha, int64_t n, float tau, uint32_t* keep_idx, int64_t* n_keep,
                              void* tmp, cudaStream_t st);
size_t accum_gate_tmp_size(int64_t n);
size_t voxelize_tmp_size(int32_t W, int32_t H);
cudaError_t launch_voxelize(const splat2d_surfels& in, int32_t W, int32_t H, float tau_d,
                            const splat2d_surfel_buffers& out, int32_t* out_block, int64_t* n_out, void* tmp,
                            cudaStream_t st);
cudaError_t launch_sim3(int64_t n, float* means, float* quats, float* scales, const float* sim3, const int32_t* index,
                        cudaStream_t st);
cudaError_t launch_preprocess_bwd(const splat2d_surfels* S, const Layout& L, const RastParams& P, char* ws,
                                  const splat2d_grads* G, bool atomic_params, cudaStream_t st);
int sm_count();
void count_launches(int n);  // host-side tally of kernels enqueued

// ---------------------------------------------------------------------------
// Device helpers
// ---------------------------------------------------------------------------
#ifdef __CUDACC__

// Error-free transformations (Knuth's TwoSum; the FMA-based exact product).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e) {
  p = __fmul_rn(a, b);
  e = __fmaf_rn(a, b, -p);
}
// Compensated dot product r0*m0 + r1*m1 + r2*m2 + t (Ogita, Rump & Oishi's
// Dot2: as accurate as evaluating in twice the working precision), returned
// as a normalised float-float pair.
__device__ __forceinline__ void dot3_plus(float r0, float r1, float r2, float m0, float m1, float m2, float t,
                                          float& hi, float& lo) {
  float p, s, h, r, q;
  two_prod(r0, m0, p, s);
  two_prod(r1, m1, h, r);
  two_sum(p, h, p, q);
  s = __fadd_rn(s, __fadd_rn(q, r));
  two_prod(r2, m2, h, r);
  two_sum(p, h, p, q);
  s = __fadd_rn(s, __fadd_rn(q, r));
  two_sum(p, t, p, q);
  s = __fadd_rn(s, q);
  hi = __fadd_rn(p, s);
  lo = __fsub_rn(s, __fsub_rn(hi, p));
}

// Fast approximate reciprocal and base-2 exponential (PTX, <= 1-2 ulp).
__device__ __forceinline__ float rcp_approx(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Vector atomic add of four floats (sm_90+).
__device__ __forceinline__ void red_add_v4(float* addr, float a, float b, float c, float d) {
  asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(addr), "f"(a), "f"(b), "f"(c), "f"(d)
               : "memory");
}

__device__ __forceinline__ uint32_t pack_half2_scaled(float lo_x, float lo_y) {
  // the low parts of the center are below 2^-9 px for images < 65536 px;
  // scaled by 2^16 they fit half precision with ~2^-27 px resolution
  __half2 h = __floats2half2_rn(lo_x * 65536.0f, lo_y * 65536.0f);
  return *reinterpret_cast<uint32_t*>(&h);
}
__device__ __forceinline__ float2 unpack_half2_scaled(uint32_t u) {
  __half2 h = *reinterpret_cast<__half2*>(&u);
  float2 f = __half22float2(h);
  return make_float2(f.x * (1.0f / 65536.0f), f.y * (1.0f / 65536.0f));
}

// Index of the view owning global tile `t` (views sorted by tile_base).
__device__ __forceinline__ int find_view_by_tile(const DView* views, int V, int t) {
  int lo = 0, hi = V - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (__ldg(&views[mid].tile_base) <= t) lo = mid; else hi = mid - 1;
  }
  return lo;
}
// Index of the view owning render record `r` (views sorted by rbase).
__device__ __forceinline__ int find_view_by_record(const DView* views, int V, int64_t r) {
  int lo = 0, hi = V - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (__ldg(&views[mid].rbase) <= r) lo = mid; else hi = mid - 1;
  }
  return lo;
}
__device__ __forceinline__ int find_group(const DGroup* groups, int G, int64_t w) {
  int lo = 0, hi = G - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (__ldg(&groups[mid].wbase) <= w) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Runs of equal tiles across the lanes of a full warp: each lane offers tile
// t (has = false: none).  Neighbouring records (neighbouring pixels of a
// keyframe) mostly hit the same tile at the same step, so one atomic per run
// serves all its lanes.  `leader` is the lane starting the run that holds
// this lane, `run` its length on the leader (0 elsewhere).
struct TileRun {
  int leader;
  uint32_t run;
  bool lead;
};
__device__ __forceinline__ TileRun tile_run(uint32_t t, bool has, int lane) {
  const uint32_t lt_mask = (1u << lane) - 1u;
  const uint32_t prev = __shfl_up_sync(0xffffffffu, t, 1);
  const uint32_t next = __shfl_down_sync(0xffffffffu, t, 1);
  const uint32_t heads = __ballot_sync(0xffffffffu, has && (lane == 0 || prev != t));
  const uint32_t ends = __ballot_sync(0xffffffffu, has && (lane == 31 || next != t));
  TileRun r;
  r.leader = 31 - __clz(heads & (lt_mask | (1u << lane)));  // run start at or below this lane
  r.lead = has && r.leader == lane;
  r.run = r.lead ? (uint32_t)(__ffs(ends & ~lt_mask) - lane) : 0u;
  return r;
}

// Index checks of the checked build (compiled with S2D_CHECKS): a failed
// check records SPLAT2D_ERR_BOUNDS in the status word (unless an earlier
// status is there) and the caller skips the access; nothing traps.  In the
// normal build the checks compile away.
#ifdef S2D_CHECKS
__device__ __forceinline__ bool s2d_check(bool ok, Header* hdr) {
  if (!ok) atomicCAS(reinterpret_cast<int*>(&hdr->status), 0, (int)SPLAT2D_ERR_BOUNDS);
  return ok;
}
#else
__device__ __forceinline__ bool s2d_check(bool ok, Header*) { return true; }
#endif

#endif  // __CUDACC__

}  // namespace s2d
