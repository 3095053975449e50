// C ABI of libsplat2d: argument checks, workspace layout and the launch
// sequence of each call.  See include/splat2d.h for the contract.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <vector>

#include "splat2d_internal.cuh"

namespace s2d {

std::atomic<uint64_t>& launch_counter() {
  static std::atomic<uint64_t> c{0};
  return c;
}
void count_launches(int n) { launch_counter().fetch_add((uint64_t)n); }

int sm_count() {
  static int cached[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 1;
  if (dev < 0 || dev >= 64) dev = 0;
  if (!cached[dev]) {
    int n = 0;
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    cached[dev] = n > 0 ? n : 1;
  }
  return cached[dev];
}

static size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

static bool valid_config(const splat2d_config* c) {
  if (!c) return false;
  const bool tile_ok = (c->tile_w == 16 && c->tile_h == 16) || (c->tile_w == 8 && c->tile_h == 8) ||
                       (c->tile_w == 32 && c->tile_h == 8);
  auto chunk_valid = [&](int ch) {
    return ch == 64 || ch == 128 || ch == 256 || (ch == 512 && c->tile_w * c->tile_h == 256);
  };
  const bool chunk_ok = chunk_valid(c->chunk) && (c->bwd_chunk == 0 || chunk_valid(c->bwd_chunk));
  if (!tile_ok || !chunk_ok) return false;
  if (!(c->alpha_min > 0.f && c->alpha_min < 1.f)) return false;
  if (!(c->alpha_max >= c->alpha_min && c->alpha_max < 1.f)) return false;
  if (!(c->t_min > 0.f && c->t_min < 1.f)) return false;
  if (!(c->lowpass_sigma >= 0.f && std::isfinite(c->lowpass_sigma))) return false;
  if (!(c->z_near > 0.f && std::isfinite(c->z_near))) return false;
  return true;
}

// Number of key bits in use: 32 depth bits + bits of the largest tile index.
static int key_bits_for(int64_t T) {
  int b = 0;
  while (b < 40 && (int64_t(1) << b) < T) b++;
  return 32 + b;
}

struct HostTables {
  std::vector<DView> views;
  std::vector<DGroup> groups;
};

static bool build_tables(const splat2d_config* cfg, const splat2d_problem* prob, Layout* L, HostTables* H) {
  if (!cfg || !prob || !prob->views || prob->n_views < 1 || prob->n_views > 4096) return false;
  if (prob->n_surfels < 0 || prob->n_surfels > 0xffffffffll) return false;
  if (prob->instance_capacity < 0 || prob->instance_capacity > 0xffffffffll) return false;
  const int V = prob->n_views;
  if (H) {
    H->views.assign(V, DView{});
    H->groups.clear();
  }
  int64_t R = 0, T = 0, P = 0, work = 0;
  int G = 0;
  std::vector<std::pair<int64_t, int64_t>> ranges;
  for (int v = 0; v < V; v++) {
    const splat2d_view& sv = prob->views[v];
    if (sv.width < 1 || sv.height < 1 || sv.width > 32768 || sv.height > 32768) return false;
    if (!(sv.fx > 0.f) || !(sv.fy > 0.f) || !std::isfinite(sv.cx) || !std::isfinite(sv.cy)) return false;
    for (int k = 0; k < 12; k++)
      if (!std::isfinite(sv.Rt[k])) return false;
    if (sv.surfel_offset < 0 || sv.surfel_count < 0 || sv.surfel_offset + sv.surfel_count > prob->n_surfels)
      return false;
    if (sv.pixel_offset < 0) return false;
    const int tx = (sv.width + cfg->tile_w - 1) / cfg->tile_w;
    const int ty = (sv.height + cfg->tile_h - 1) / cfg->tile_h;
    const bool new_group = v == 0 || sv.surfel_offset != prob->views[v - 1].surfel_offset ||
                           sv.surfel_count != prob->views[v - 1].surfel_count;
    if (new_group) {
      if (H) {
        DGroup g;
        g.soff = sv.surfel_offset;
        g.scnt = sv.surfel_count;
        g.wbase = work;
        g.v0 = v;
        g.v1 = v + 1;
        H->groups.push_back(g);
      }
      ranges.push_back({sv.surfel_offset, sv.surfel_offset + sv.surfel_count});
      work += sv.surfel_count;
      G++;
    } else if (H) {
      H->groups.back().v1 = v + 1;
    }
    if (H) {
      DView& d = H->views[v];
      d.W = sv.width;
      d.H = sv.height;
      d.fx = sv.fx; d.fy = sv.fy; d.cx = sv.cx; d.cy = sv.cy;
      d.ifx = 1.0f / sv.fx;  // the same correctly rounded quotient the kernels took per pair
      d.ify = 1.0f / sv.fy;
      for (int r = 0; r < 3; r++) {
        for (int c = 0; c < 3; c++) d.R[r * 3 + c] = sv.Rt[r * 4 + c];
        d.t[r] = sv.Rt[r * 4 + 3];
      }
      d.soff = sv.surfel_offset;
      d.scnt = sv.surfel_count;
      d.poff = sv.pixel_offset;
      d.rbase = R;
      d.tile_base = (int32_t)T;
      d.tiles_x = tx;
      d.tiles_y = ty;
      d.group = G - 1;
    }
    R += sv.surfel_count;
    T += (int64_t)tx * ty;
    P = std::max<int64_t>(P, sv.pixel_offset + (int64_t)sv.width * sv.height);
  }
  if (R > 0xffffffffll || T > 0x7fffffffll) return false;
  std::sort(ranges.begin(), ranges.end());
  bool overlap = false;
  for (size_t i = 1; i < ranges.size(); i++)
    if (ranges[i].first < ranges[i - 1].second) overlap = true;

  L->V = V;
  L->G = G;
  L->R = R;
  L->T = T;
  L->P = P;
  L->cap = prob->instance_capacity;
  L->n_work = work;
  L->groups_overlap = overlap;
  L->sort_blocks = std::min(SORT_MAX_BLOCKS, 4 * sm_count());
  L->key_bits = key_bits_for(T);
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off = align256(off + bytes);
    return o;
  };
  L->header = take(256);
  L->views = take(sizeof(DView) * V);
  L->groups = take(sizeof(DGroup) * G);
  L->ntiles = take(sizeof(uint32_t) * R);
  L->bins = take(sizeof(uint4) * R);  // per record: depth bits, rect (2 words), tile count
  L->records = take(sizeof(float4) * REC_F4 * R);
  L->rgrad = take(sizeof(float) * GRAD_F * R);
  L->keys0 = take(sizeof(uint64_t) * L->cap);
  L->keys1 = take(sizeof(uint64_t) * L->cap);
  L->vals0 = take(sizeof(uint32_t) * L->cap);
  L->vals1 = take(sizeof(uint32_t) * L->cap);
  L->sort_hist = take(sizeof(uint32_t) * (256 * (size_t)L->sort_blocks + 256));
  L->ranges = take(sizeof(uint2) * T);
  L->tile_count = take(sizeof(uint32_t) * T);   // instances per tile (counted by the preprocess)
  L->tile_cursor = take(sizeof(uint32_t) * T);  // scatter cursors (from the tile scan)
  L->tile_order = take(sizeof(uint32_t) * T);
  L->tile_hist = take(sizeof(uint32_t) * (ORDER_BINS + 16));
  L->tile_class = take(sizeof(uint32_t) * 6 * (size_t)T);  // one list per bucket-sort size class
  L->tfinal = take(sizeof(float) * P);
  L->last = take(sizeof(uint32_t) * P);
  L->dfinal = take(sizeof(float) * P);  // per pixel: the depth sum D (the depth-distortion adjoint needs it)
  // the records in sorted-list order, written by the forward as it stages
  // them and read back contiguously by the backward
  L->rcopy = take(sizeof(float4) * REC_F4 * (size_t)L->cap);
  // per (32-entry word of a tile's list, pixel of the tile): the entries of
  // the word the forward blended at that pixel, read by the backward.  Tile
  // t's words start at range.x / 32 + t, so cap / 32 + T + 1 words cover
  // every tile whatever its range.
  L->bmask_words = L->cap / 32 + T + 1;
  L->bmask = take(sizeof(uint32_t) * (size_t)L->bmask_words * (size_t)cfg->tile_w * (size_t)cfg->tile_h);
  L->total = off;
  return true;
}

bool compute_layout(const splat2d_config* cfg, const splat2d_problem* prob, Layout* L) {
  if (!valid_config(cfg)) return false;
  return build_tables(cfg, prob, L, nullptr);
}

static RastParams make_params(const splat2d_config* c) {
  RastParams P;
  P.alpha_min = c->alpha_min;
  P.alpha_max = c->alpha_max;
  P.t_min = c->t_min;
  P.z_near = c->z_near;
  P.lp_r = c->lowpass_sigma;
  P.lp_scale = c->lowpass_sigma > 0.f ? kLog2e / (2.f * c->lowpass_sigma * c->lowpass_sigma) : 1e30f;
  P.bg[0] = c->bg[0]; P.bg[1] = c->bg[1]; P.bg[2] = c->bg[2];
  P.tile_w = c->tile_w;
  P.tile_h = c->tile_h;
  P.stats = (c->flags & SPLAT2D_FLAG_NO_STATS) ? 0 : 1;
  P.depth_ray = (c->flags & SPLAT2D_FLAG_DEPTH_RAY) ? 1 : 0;
  const int tail = (int)((c->flags >> SPLAT2D_FLAG_TAIL_SHIFT) & 0xffu);
  P.fwd_tail = tail == 0 ? 6 : (tail == 255 ? 1 << 20 : tail);
  return P;
}

static int check_common(const splat2d_config* cfg, const splat2d_problem* prob, void* ws, size_t ws_bytes,
                        Layout* L) {
  if (!valid_config(cfg)) return SPLAT2D_ERR_INVALID_ARG;
  if (!build_tables(cfg, prob, L, nullptr)) return SPLAT2D_ERR_INVALID_ARG;
  if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255)) return SPLAT2D_ERR_INVALID_ARG;
  if (ws_bytes < L->total) return SPLAT2D_ERR_WORKSPACE_TOO_SMALL;
  return SPLAT2D_OK;
}

// The binning leaves the sorted instances in buffer 0.
static int final_sorted_buffer(const Layout&) { return 0; }

}  // namespace s2d

using namespace s2d;

extern "C" {

void splat2d_default_config(splat2d_config* c) {
  if (!c) return;
  std::memset(c, 0, sizeof(*c));
  c->tile_w = 8;
  c->tile_h = 8;
  c->chunk = 128;
  c->bwd_chunk = 64;
  c->alpha_min = 1.0f / 255.0f;
  c->alpha_max = 0.99f;
  c->t_min = 1e-4f;
  c->lowpass_sigma = 0.70710678118654752f;
  c->z_near = 0.01f;
}

size_t splat2d_workspace_size(const splat2d_config* cfg, const splat2d_problem* prob) {
  Layout L;
  if (!compute_layout(cfg, prob, &L)) return 0;
  return L.total;
}

int splat2d_workspace_layout(const splat2d_config* cfg, const splat2d_problem* prob, splat2d_layout* out) {
  Layout L;
  if (!out || !compute_layout(cfg, prob, &L)) return SPLAT2D_ERR_INVALID_ARG;
  const int fb = final_sorted_buffer(L);
  out->records = L.records;
  out->ntiles = L.ntiles;
  out->keys = fb ? L.keys1 : L.keys0;
  out->vals = fb ? L.vals1 : L.vals0;
  out->ranges = L.ranges;
  out->tfinal = L.tfinal;
  out->last = L.last;
  out->total = L.total;
  out->n_records = L.R;
  out->n_tiles = L.T;
  out->n_pixels = L.P;
  return SPLAT2D_OK;
}

int splat2d_preprocess(const splat2d_config* cfg, const splat2d_problem* prob, const splat2d_surfels* surfels,
                       void* ws, size_t ws_bytes, splat2d_stream stream) {
  Layout L;
  int rc = check_common(cfg, prob, ws, ws_bytes, &L);
  if (rc) return rc;
  if (!surfels || surfels->n != prob->n_surfels) return SPLAT2D_ERR_INVALID_ARG;
  if (prob->n_surfels > 0 && (!surfels->means || !surfels->scales || !surfels->quats || !surfels->opacity ||
                              !surfels->rgb))
    return SPLAT2D_ERR_INVALID_ARG;
  if (reinterpret_cast<uintptr_t>(surfels->quats) & 15) return SPLAT2D_ERR_INVALID_ARG;
  HostTables H;
  build_tables(cfg, prob, &L, &H);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  char* w = static_cast<char*>(ws);
  if (cudaMemsetAsync(w + L.header, 0, 256, st) != cudaSuccess) return SPLAT2D_ERR_CUDA;
  if (launch_upload(H.views.data(), sizeof(DView) * H.views.size(), w + L.views, st) != cudaSuccess)
    return SPLAT2D_ERR_CUDA;
  if (!H.groups.empty() &&
      launch_upload(H.groups.data(), sizeof(DGroup) * H.groups.size(), w + L.groups, st) != cudaSuccess)
    return SPLAT2D_ERR_CUDA;
  RastParams P = make_params(cfg);
  if (launch_preprocess(surfels, L, P, w, st) != cudaSuccess) return SPLAT2D_ERR_CUDA;
  return SPLAT2D_OK;
}

int splat2d_bin_sort(const splat2d_config* cfg, const splat2d_problem* prob, void* ws, size_t ws_bytes,
                     splat2d_stream stream) {
  Layout L;
  int rc = check_common(cfg, prob, ws, ws_bytes, &L);
  if (rc) return rc;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  char* w = static_cast<char*>(ws);
  RastParams P = make_params(cfg);
  if (launch_bin_tiles(L, P, w, st) != cudaSuccess) return SPLAT2D_ERR_CUDA;
  if (launch_order(L, w, st) != cudaSuccess) return SPLAT2D_ERR_CUDA;
  return SPLAT2D_OK;
}

int splat2d_render_fwd_dist(const splat2d_config* cfg, const splat2d_problem* prob, void* ws, size_t ws_bytes,
                            float* rgb, float* depth, float* normal, float* alpha, float* dist,
                            splat2d_stream stream) {
  Layout L;
  int rc = check_common(cfg, prob, ws, ws_bytes, &L);
  if (rc) return rc;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  char* w = static_cast<char*>(ws);
  const uint32_t* vals = reinterpret_cast<const uint32_t*>(w + (final_sorted_buffer(L) ? L.vals1 : L.vals0));
  if (launch_render_fwd(L, make_params(cfg), cfg->chunk, w, vals, rgb, depth, normal, alpha, dist, st) !=
      cudaSuccess)
    return SPLAT2D_ERR_CUDA;
  return SPLAT2D_OK;
}

int splat2d_render_fwd(const splat2d_config* cfg, const splat2d_problem* prob, void* ws, size_t ws_bytes,
                       float* rgb, float* depth, float* normal, float* alpha, splat2d_stream stream) {
  return splat2d_render_fwd_dist(cfg, prob, ws, ws_bytes, rgb, depth, normal, alpha, nullptr, stream);
}

int splat2d_render_bwd_tiles_dist(const splat2d_config* cfg, const splat2d_problem* prob, void* ws,
                                  size_t ws_bytes, const float* d_rgb, const float* d_depth, const float* d_normal,
                                  const float* d_alpha, const float* d_dist, splat2d_stream stream) {
  Layout L;
  int rc = check_common(cfg, prob, ws, ws_bytes, &L);
  if (rc) return rc;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  char* w = static_cast<char*>(ws);
  const uint32_t* vals = reinterpret_cast<const uint32_t*>(w + (final_sorted_buffer(L) ? L.vals1 : L.vals0));
  if (launch_render_bwd(L, make_params(cfg), cfg->bwd_chunk ? cfg->bwd_chunk : cfg->chunk, w, vals, d_rgb,
                        d_depth, d_normal, d_alpha, d_dist, st) != cudaSuccess)
    return SPLAT2D_ERR_CUDA;
  return SPLAT2D_OK;
}

int splat2d_render_bwd_tiles(const splat2d_config* cfg, const splat2d_problem* prob, void* ws, size_t ws_bytes,
                             const float* d_rgb, const float* d_depth, const float* d_normal, const float* d_alpha,
                             splat2d_stream stream) {
  return splat2d_render_bwd_tiles_dist(cfg, prob, ws, ws_bytes, d_rgb, d_depth, d_normal, d_alpha, nullptr,
                                       stream);
}

int splat2d_preprocess_bwd(const splat2d_config* cfg, const splat2d_problem* prob, const splat2d_surfels* surfels,
                           void* ws, size_t ws_bytes, const splat2d_grads* grads, splat2d_stream stream) {
  Layout L;
  int rc = check_common(cfg, prob, ws, ws_bytes, &L);
  if (rc) return rc;
  if (!surfels || surfels->n != prob->n_surfels || !grads) return SPLAT2D_ERR_INVALID_ARG;
  if (prob->n_surfels > 0 && (!surfels->means || !surfels->scales || !surfels->quats || !surfels->opacity ||
                              !surfels->rgb))
    return SPLAT2D_ERR_INVALID_ARG;
  if (reinterpret_cast<uintptr_t>(surfels->quats) & 15) return SPLAT2D_ERR_INVALID_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (launch_preprocess_bwd(surfels, L, make_params(cfg), static_cast<char*>(ws), grads, L.groups_overlap, st) !=
      cudaSuccess)
    return SPLAT2D_ERR_CUDA;
  return SPLAT2D_OK;
}

int splat2d_max_error(const splat2d_config* cfg, const splat2d_problem* prob, void* ws, size_t ws_bytes,
                      const float* err, float* max_err, splat2d_stream stream) {
  Layout L;
  int rc = check_common(cfg, prob, ws, ws_bytes, &L);
  if (rc) return rc;
  if (!err || !max_err) return SPLAT2D_ERR_INVALID_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  char* w = static_cast<char*>(ws);
  const uint32_t* vals = reinterpret_cast<const uint32_t*>(w + (final_sorted_buffer(L) ? L.vals1 : L.vals0));
  if (launch_max_error(L, make_params(cfg), cfg->chunk, w, vals, err, max_err, st) != cudaSuccess)
    return SPLAT2D_ERR_CUDA;
  return SPLAT2D_OK;
}

size_t splat2d_accum_gate_tmp_size(int64_t n) { return n < 0 ? 0 : accum_gate_tmp_size(n); }

int splat2d_accum_gate(const float* alpha, int64_t n, float tau, uint32_t* keep_idx, int64_t* n_keep, void* tmp,
                       size_t tmp_bytes, splat2d_stream stream) {
  if (n < 0 || n > (int64_t)0xFFFFFFFFll || !n_keep) return SPLAT2D_ERR_INVALID_ARG;
  if (n > 0 && (!alpha || !keep_idx || !tmp)) return SPLAT2D_ERR_INVALID_ARG;
  if (n > 0 && tmp_bytes < accum_gate_tmp_size(n)) return SPLAT2D_ERR_WORKSPACE_TOO_SMALL;
  if (launch_accum_gate(alpha, n, tau, keep_idx, n_keep, tmp, reinterpret_cast<cudaStream_t>(stream)) != cudaSuccess)
    return SPLAT2D_ERR_CUDA;
  return SPLAT2D_OK;
}

size_t splat2d_voxelize_tmp_size(int32_t width, int32_t height) {
  return (width < 0 || height < 0) ? 0 : voxelize_tmp_size(width, height);
}

int splat2d_voxelize(const splat2d_surfels* in, int32_t width, int32_t height, float tau_d,
                     const splat2d_surfel_buffers* out, int32_t* out_block, int64_t* n_out, void* tmp,
                     size_t tmp_bytes, splat2d_stream stream) {
  if (!in || !out || !n_out || width < 0 || height < 0) return SPLAT2D_ERR_INVALID_ARG;
  if (in->n != (int64_t)width * height || (int64_t)width * height > (int64_t)0x7FFFFFFF) return SPLAT2D_ERR_INVALID_ARG;
  if (in->n > 0) {
    if (!in->means || !in->scales || !in->quats || !in->opacity || !in->rgb) return SPLAT2D_ERR_INVALID_ARG;
    if (!out->means || !out->scales || !out->quats || !out->opacity || !out->rgb || !tmp)
      return SPLAT2D_ERR_INVALID_ARG;
    if (tmp_bytes < voxelize_tmp_size(width, height)) return SPLAT2D_ERR_WORKSPACE_TOO_SMALL;
  }
  if (launch_voxelize(*in, width, height, tau_d, *out, out_block, n_out, tmp, reinterpret_cast<cudaStream_t>(stream)) !=
      cudaSuccess)
    return SPLAT2D_ERR_CUDA;
  return SPLAT2D_OK;
}

int splat2d_sim3_apply(int64_t n, float* means, float* quats, float* scales, const float* sim3,
                       const int32_t* index, splat2d_stream stream) {
  if (n < 0 || (n > 0 && !sim3)) return SPLAT2D_ERR_INVALID_ARG;
  if (launch_sim3(n, means, quats, scales, sim3, index, reinterpret_cast<cudaStream_t>(stream)) != cudaSuccess)
    return SPLAT2D_ERR_CUDA;
  return SPLAT2D_OK;
}

int splat2d_render_bwd_dist(const splat2d_config* cfg, const splat2d_problem* prob, const splat2d_surfels* surfels,
                            void* ws, size_t ws_bytes, const float* d_rgb, const float* d_depth,
                            const float* d_normal, const float* d_alpha, const float* d_dist,
                            const splat2d_grads* grads, splat2d_stream stream) {
  if (!surfels || !prob || surfels->n != prob->n_surfels || !grads) return SPLAT2D_ERR_INVALID_ARG;
  int rc = splat2d_render_bwd_tiles_dist(cfg, prob, ws, ws_bytes, d_rgb, d_depth, d_normal, d_alpha, d_dist, stream);
  if (rc) return rc;
  return splat2d_preprocess_bwd(cfg, prob, surfels, ws, ws_bytes, grads, stream);
}

int splat2d_render_bwd(const splat2d_config* cfg, const splat2d_problem* prob, const splat2d_surfels* surfels,
                       void* ws, size_t ws_bytes, const float* d_rgb, const float* d_depth, const float* d_normal,
                       const float* d_alpha, const splat2d_grads* grads, splat2d_stream stream) {
  return splat2d_render_bwd_dist(cfg, prob, surfels, ws, ws_bytes, d_rgb, d_depth, d_normal, d_alpha, nullptr,
                                 grads, stream);
}

uint64_t splat2d_launch_count(void) { return s2d::launch_counter().load(); }

int splat2d_stats(const void* ws, splat2d_stats_t* out, splat2d_stream stream) {
  if (!ws || !out) return SPLAT2D_ERR_INVALID_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (cudaStreamSynchronize(st) != cudaSuccess) return SPLAT2D_ERR_CUDA;
  Header h;
  if (cudaMemcpy(&h, ws, sizeof(Header), cudaMemcpyDeviceToHost) != cudaSuccess) return SPLAT2D_ERR_CUDA;
  std::memset(out, 0, sizeof(*out));
  out->status = h.status;
  out->needed_capacity = (int64_t)h.needed;
  out->n_instances = (int64_t)h.n_inst;
  out->n_visible = (int64_t)h.n_visible;
  out->fwd_pairs_evaluated = (int64_t)h.stat[STAT_FWD_EVAL];
  out->fwd_pairs_blended = (int64_t)h.stat[STAT_FWD_BLEND];
  out->bwd_pairs_evaluated = (int64_t)h.stat[STAT_BWD_EVAL];
  out->bwd_pairs_blended = (int64_t)h.stat[STAT_BWD_BLEND];
  out->bwd_terms_outside = (int64_t)h.stat[STAT_BWD_OUTSIDE];
  return h.status;
}

int splat2d_status(const void* ws, int64_t* needed_capacity, splat2d_stream stream) {
  splat2d_stats_t s;
  int rc = splat2d_stats(ws, &s, stream);
  if (rc == SPLAT2D_ERR_INVALID_ARG || rc == SPLAT2D_ERR_CUDA) return rc;
  if (needed_capacity) *needed_capacity = s.needed_capacity;
  return (int)s.status;
}

size_t splat2d_sort_tmp_size(int64_t n) {
  if (n < 0) return 0;
  return align256(sizeof(uint64_t) * (size_t)n) + align256(sizeof(uint32_t) * (size_t)n) +
         align256(sizeof(uint32_t) * (256 * (size_t)std::min(SORT_MAX_BLOCKS, 4 * sm_count()) + 256));
}

int splat2d_sort_pairs(uint64_t* keys, uint32_t* vals, int64_t n, int key_bits, void* tmp, size_t tmp_bytes,
                       splat2d_stream stream) {
  if (n < 0 || n > 0xffffffffll || key_bits < 1 || key_bits > 64) return SPLAT2D_ERR_INVALID_ARG;
  if (n == 0) return SPLAT2D_OK;
  if (!keys || !vals || !tmp || (reinterpret_cast<uintptr_t>(tmp) & 255)) return SPLAT2D_ERR_INVALID_ARG;
  if (tmp_bytes < splat2d_sort_tmp_size(n)) return SPLAT2D_ERR_WORKSPACE_TOO_SMALL;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  char* t = static_cast<char*>(tmp);
  uint64_t* k1 = reinterpret_cast<uint64_t*>(t);
  uint32_t* v1 = reinterpret_cast<uint32_t*>(t + align256(sizeof(uint64_t) * n));
  uint32_t* hist = reinterpret_cast<uint32_t*>(t + align256(sizeof(uint64_t) * n) + align256(sizeof(uint32_t) * n));
  const int nb = std::min(SORT_MAX_BLOCKS, 4 * sm_count());
  if (cudaMemsetAsync(hist + 256 * (size_t)nb, 0, 256 * sizeof(uint32_t), st) != cudaSuccess) return SPLAT2D_ERR_CUDA;
  int fb = 0;
  if (launch_sort(keys, vals, k1, v1, nullptr, n, key_bits, hist, nb, &fb, st) != cudaSuccess)
    return SPLAT2D_ERR_CUDA;
  if (fb) {
    if (cudaMemcpyAsync(keys, k1, sizeof(uint64_t) * n, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
      return SPLAT2D_ERR_CUDA;
    if (cudaMemcpyAsync(vals, v1, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
      return SPLAT2D_ERR_CUDA;
  }
  return SPLAT2D_OK;
}

const char* splat2d_strerror(int code) {
  switch (code) {
    case SPLAT2D_OK: return "ok";
    case SPLAT2D_ERR_INVALID_ARG: return "invalid argument";
    case SPLAT2D_ERR_WORKSPACE_TOO_SMALL: return "workspace too small";
    case SPLAT2D_ERR_CUDA: return "CUDA error";
    case SPLAT2D_ERR_CAPACITY: return "instance capacity exceeded";
    case SPLAT2D_ERR_TIMEOUT: return "bounded wait timed out";
    case SPLAT2D_ERR_NO_DEVICE: return "no CUDA device";
    case SPLAT2D_ERR_BOUNDS: return "index check failed (checked build)";
    default: return "unknown status";
  }
}

}  // extern "C"
