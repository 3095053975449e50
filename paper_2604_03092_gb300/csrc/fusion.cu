// Accumulation gate of map fusion (Sec. 4.3, "Map Fusion": new primitives
// are added only where the global map does not yet reconstruct the frame,
// found by rendering its accumulation map and comparing with a threshold).
//
// The accumulation map is the forward's alpha output A = 1 - T_final at the
// new keyframe's pose; the frame's new primitives are per pixel, so the gate
// is an ordered stream compaction: keep_idx lists, in ascending order, the
// pixels with A < tau.  Three launches: per-block counts, one block scanning
// the counts (which also writes the total), and a scatter in which each
// block ranks its kept pixels with warp ballots.
#include <cuda_runtime.h>

#include "splat2d_internal.cuh"

namespace s2d {

constexpr int GATE_THREADS = 256;
constexpr int GATE_PER_THREAD = 4;
constexpr int GATE_TILE = GATE_THREADS * GATE_PER_THREAD;  // pixels per block

__device__ __forceinline__ bool gate_keep(const float* alpha, int64_t i, int64_t n, float tau) {
  return i < n && alpha[i] < tau;  // false for NaN
}

__global__ void __launch_bounds__(GATE_THREADS) k_gate_count(const float* __restrict__ alpha, int64_t n, float tau,
                                                             uint32_t* __restrict__ block_count) {
  __shared__ uint32_t s_w[GATE_THREADS / 32];
  const int64_t base = (int64_t)blockIdx.x * GATE_TILE;
  uint32_t c = 0;
#pragma unroll
  for (int k = 0; k < GATE_PER_THREAD; k++) c += gate_keep(alpha, base + k * GATE_THREADS + threadIdx.x, n, tau);
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t t = 0;
    for (int w = 0; w < GATE_THREADS / 32; w++) t += s_w[w];
    block_count[blockIdx.x] = t;
  }
}

// One block: exclusive scan of the block counts in place; the total goes to *n_keep.
__global__ void __launch_bounds__(1024) k_gate_scan(uint32_t* __restrict__ block_count, int64_t nb,
                                                    int64_t* __restrict__ n_keep) {
  __shared__ unsigned long long s_w[32];
  __shared__ unsigned long long s_carry;
  if (threadIdx.x == 0) s_carry = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int64_t b0 = 0; b0 < nb; b0 += 1024) {
    const int64_t i = b0 + threadIdx.x;
    const unsigned long long v = i < nb ? block_count[i] : 0ull;
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
    if (i < nb) block_count[i] = (uint32_t)(incl - v);
    __syncthreads();
    if (threadIdx.x == 1023) s_carry = incl;
    __syncthreads();
  }
  if (threadIdx.x == 0) *n_keep = (int64_t)s_carry;
}

__global__ void __launch_bounds__(GATE_THREADS) k_gate_scatter(const float* __restrict__ alpha, int64_t n, float tau,
                                                               const uint32_t* __restrict__ block_offset,
                                                               uint32_t* __restrict__ keep_idx) {
  __shared__ uint32_t s_w[GATE_THREADS / 32];
  __shared__ uint32_t s_run;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const uint32_t lt = (1u << lane) - 1u;
  const int64_t base = (int64_t)blockIdx.x * GATE_TILE;
  if (threadIdx.x == 0) s_run = block_offset[blockIdx.x];
  __syncthreads();
  // rounds of GATE_THREADS consecutive pixels keep the output in ascending order
  for (int k = 0; k < GATE_PER_THREAD; k++) {
    const int64_t i = base + k * GATE_THREADS + threadIdx.x;
    const bool keep = gate_keep(alpha, i, n, tau);
    const uint32_t m = __ballot_sync(0xffffffffu, keep);
    if (lane == 0) s_w[wid] = __popc(m);
    __syncthreads();
    uint32_t before = s_run;
    for (int w = 0; w < wid; w++) before += s_w[w];
    if (keep) keep_idx[before + __popc(m & lt)] = (uint32_t)i;
    __syncthreads();
    if (threadIdx.x == 0) {
      uint32_t t = 0;
      for (int w = 0; w < GATE_THREADS / 32; w++) t += s_w[w];
      s_run += t;
    }
    __syncthreads();
  }
}

size_t accum_gate_tmp_size(int64_t n) {
  const int64_t nb = (n + GATE_TILE - 1) / GATE_TILE;
  return sizeof(uint32_t) * (size_t)(nb > 0 ? nb : 1);
}

cudaError_t launch_accum_gate(const float* alpha, int64_t n, float tau, uint32_t* keep_idx, int64_t* n_keep,
                              void* tmp, cudaStream_t st) {
  const int64_t nb = (n + GATE_TILE - 1) / GATE_TILE;
  if (nb == 0) return cudaMemsetAsync(n_keep, 0, sizeof(int64_t), st);
  uint32_t* counts = static_cast<uint32_t*>(tmp);
  k_gate_count<<<(unsigned)nb, GATE_THREADS, 0, st>>>(alpha, n, tau, counts);
  count_launches(1);
  k_gate_scan<<<1, 1024, 0, st>>>(counts, nb, n_keep);
  count_launches(1);
  k_gate_scatter<<<(unsigned)nb, GATE_THREADS, 0, st>>>(alpha, n, tau, counts, keep_idx);
  count_launches(1);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Adaptive voxelization (Sec. 4.3, "Adaptive Voxelization"): a keyframe's
// per-pixel map (primitive y * W + x) is cut into 2x2 blocks; each block
// becomes one primitive whose center, opacity, colour and scales are the
// block means and whose rotation is the normalised sum of its quaternions,
// each first turned to the hemisphere of the block's first one, unless the
// block's depth variation (largest minus smallest camera-frame depth of its
// primitives) exceeds tau_d, in which case its primitives are kept.  Output
// is ordered: blocks in row-major order, a kept block's primitives in
// row-major order.  One thread per block; the same count / scan / scatter
// scheme as the gate.
// ---------------------------------------------------------------------------
constexpr int VOX_THREADS = 256;

struct VoxIn {
  const float *means, *scales, *quats, *opacity, *rgb;
  int32_t W, H, bw;
  int64_t nb;
  float tau_d;
};

struct VoxOut {
  float *means, *scales, *quats, *opacity, *rgb;
  int32_t* block;
};

// Members of block b (row-major) and whether it merges.
__device__ __forceinline__ int vox_members(const VoxIn& I, int64_t b, int64_t (&idx)[4], bool& merge) {
  const int bx = (int)(b % I.bw), by = (int)(b / I.bw);
  int n = 0;
  for (int dy = 0; dy < 2; dy++)
    for (int dx = 0; dx < 2; dx++) {
      const int x = 2 * bx + dx, y = 2 * by + dy;
      if (x < I.W && y < I.H) idx[n++] = (int64_t)y * I.W + x;
    }
  float zmin = I.means[3 * idx[0] + 2], zmax = zmin;
  for (int k = 1; k < n; k++) {
    const float z = I.means[3 * idx[k] + 2];
    zmin = fminf(zmin, z);
    zmax = fmaxf(zmax, z);
  }
  merge = !(zmax - zmin > I.tau_d);
  return n;
}

__global__ void __launch_bounds__(VOX_THREADS) k_vox_count(const VoxIn I, uint32_t* __restrict__ block_count) {
  __shared__ uint32_t s_w[VOX_THREADS / 32];
  const int64_t b = (int64_t)blockIdx.x * VOX_THREADS + threadIdx.x;
  uint32_t c = 0;
  if (b < I.nb) {
    int64_t idx[4];
    bool merge;
    const int n = vox_members(I, b, idx, merge);
    c = merge ? 1u : (uint32_t)n;
  }
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t t = 0;
    for (int w = 0; w < VOX_THREADS / 32; w++) t += s_w[w];
    block_count[blockIdx.x] = t;
  }
}

__device__ __forceinline__ void vox_copy(const VoxIn& I, const VoxOut& O, int64_t i, int64_t o, int32_t b) {
  for (int k = 0; k < 3; k++) O.means[3 * o + k] = I.means[3 * i + k];
  for (int k = 0; k < 2; k++) O.scales[2 * o + k] = I.scales[2 * i + k];
  for (int k = 0; k < 4; k++) O.quats[4 * o + k] = I.quats[4 * i + k];
  O.opacity[o] = I.opacity[i];
  for (int k = 0; k < 3; k++) O.rgb[3 * o + k] = I.rgb[3 * i + k];
  if (O.block) O.block[o] = b;
}

__global__ void __launch_bounds__(VOX_THREADS) k_vox_scatter(const VoxIn I, const uint32_t* __restrict__ block_offset,
                                                             const VoxOut O) {
  __shared__ uint32_t s_w[VOX_THREADS / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t b = (int64_t)blockIdx.x * VOX_THREADS + threadIdx.x;
  int64_t idx[4] = {0, 0, 0, 0};
  bool merge = true;
  int n = 0;
  if (b < I.nb) n = vox_members(I, b, idx, merge);
  const uint32_t c = b < I.nb ? (merge ? 1u : (uint32_t)n) : 0u;
  uint32_t x = c;
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_w[wid] = x;
  __syncthreads();
  uint32_t before = block_offset[blockIdx.x];
  for (int w = 0; w < wid; w++) before += s_w[w];
  const int64_t o = (int64_t)before + (x - c);
  if (b >= I.nb) return;
  if (!merge) {
    for (int k = 0; k < n; k++) vox_copy(I, O, idx[k], o + k, (int32_t)b);
    return;
  }
  const float inv = 1.0f / (float)n;
  float m[3] = {0.f, 0.f, 0.f}, sc[2] = {0.f, 0.f}, q[4] = {0.f, 0.f, 0.f, 0.f}, op = 0.f, c3[3] = {0.f, 0.f, 0.f};
  const float* q1 = I.quats + 4 * idx[0];
  for (int k = 0; k < n; k++) {
    const int64_t i = idx[k];
    for (int j = 0; j < 3; j++) m[j] += I.means[3 * i + j];
    for (int j = 0; j < 2; j++) sc[j] += I.scales[2 * i + j];
    const float* qi = I.quats + 4 * i;
    const float d = qi[0] * q1[0] + qi[1] * q1[1] + qi[2] * q1[2] + qi[3] * q1[3];
    const float sg = d >= 0.f ? 1.f : -1.f;  // align to the block's first quaternion
    for (int j = 0; j < 4; j++) q[j] += sg * qi[j];
    op += I.opacity[i];
    for (int j = 0; j < 3; j++) c3[j] += I.rgb[3 * i + j];
  }
  const float qn = sqrtf(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
  for (int j = 0; j < 3; j++) O.means[3 * o + j] = m[j] * inv;
  for (int j = 0; j < 2; j++) O.scales[2 * o + j] = sc[j] * inv;
  for (int j = 0; j < 4; j++) O.quats[4 * o + j] = q[j] / qn;
  O.opacity[o] = op * inv;
  for (int j = 0; j < 3; j++) O.rgb[3 * o + j] = c3[j] * inv;
  if (O.block) O.block[o] = (int32_t)b;
}

size_t voxelize_tmp_size(int32_t W, int32_t H) {
  const int64_t nb = (int64_t)((W + 1) / 2) * ((H + 1) / 2);
  const int64_t g = (nb + VOX_THREADS - 1) / VOX_THREADS;
  return sizeof(uint32_t) * (size_t)(g > 0 ? g : 1);
}

cudaError_t launch_voxelize(const splat2d_surfels& in, int32_t W, int32_t H, float tau_d,
                            const splat2d_surfel_buffers& out, int32_t* out_block, int64_t* n_out, void* tmp,
                            cudaStream_t st) {
  VoxIn I;
  I.means = in.means; I.scales = in.scales; I.quats = in.quats; I.opacity = in.opacity; I.rgb = in.rgb;
  I.W = W; I.H = H; I.bw = (W + 1) / 2;
  I.nb = (int64_t)I.bw * ((H + 1) / 2);
  I.tau_d = tau_d;
  VoxOut O;
  O.means = out.means; O.scales = out.scales; O.quats = out.quats; O.opacity = out.opacity; O.rgb = out.rgb;
  O.block = out_block;
  if (I.nb == 0) return cudaMemsetAsync(n_out, 0, sizeof(int64_t), st);
  const int64_t g = (I.nb + VOX_THREADS - 1) / VOX_THREADS;
  uint32_t* counts = static_cast<uint32_t*>(tmp);
  k_vox_count<<<(unsigned)g, VOX_THREADS, 0, st>>>(I, counts);
  count_launches(1);
  k_gate_scan<<<1, 1024, 0, st>>>(counts, g, n_out);
  count_launches(1);
  k_vox_scatter<<<(unsigned)g, VOX_THREADS, 0, st>>>(I, counts, O);
  count_launches(1);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Sim(3) transforms of primitives ("Map Fusion": camera-to-world insertion,
// mu' = s R mu + t, r' = q r; "Loop Correction of Gaussian Map": a keyframe's
// Delta T = T_new T_old^-1 applied rigidly to its primitives).  Tangent
// scales are multiplied by s (a similarity scales the disks with the map).
// One thread per primitive, in place; transform rows are (qw, qx, qy, qz,
// tx, ty, tz, s), chosen per primitive by `index` (or row 0).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_sim3(int64_t n, float* __restrict__ means, float* __restrict__ quats,
                                              float* __restrict__ scales, const float* __restrict__ sim3,
                                              const int32_t* __restrict__ index) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float* T = sim3 + 8 * (index ? (int64_t)index[i] : 0);
  float qw = T[0], qx = T[1], qy = T[2], qz = T[3];
  const float qn = sqrtf(qw * qw + qx * qx + qy * qy + qz * qz);
  qw /= qn; qx /= qn; qy /= qn; qz /= qn;
  const float s = T[7];
  // rotation matrix of the unit quaternion
  const float R00 = 1.f - 2.f * (qy * qy + qz * qz), R01 = 2.f * (qx * qy - qw * qz), R02 = 2.f * (qx * qz + qw * qy);
  const float R10 = 2.f * (qx * qy + qw * qz), R11 = 1.f - 2.f * (qx * qx + qz * qz), R12 = 2.f * (qy * qz - qw * qx);
  const float R20 = 2.f * (qx * qz - qw * qy), R21 = 2.f * (qy * qz + qw * qx), R22 = 1.f - 2.f * (qx * qx + qy * qy);
  if (means) {
    const float x = means[3 * i], y = means[3 * i + 1], z = means[3 * i + 2];
    means[3 * i + 0] = s * (R00 * x + R01 * y + R02 * z) + T[4];
    means[3 * i + 1] = s * (R10 * x + R11 * y + R12 * z) + T[5];
    means[3 * i + 2] = s * (R20 * x + R21 * y + R22 * z) + T[6];
  }
  if (quats) {
    const float rw = quats[4 * i], rx = quats[4 * i + 1], ry = quats[4 * i + 2], rz = quats[4 * i + 3];
    quats[4 * i + 0] = qw * rw - qx * rx - qy * ry - qz * rz;
    quats[4 * i + 1] = qw * rx + qx * rw + qy * rz - qz * ry;
    quats[4 * i + 2] = qw * ry - qx * rz + qy * rw + qz * rx;
    quats[4 * i + 3] = qw * rz + qx * ry - qy * rx + qz * rw;
  }
  if (scales) {
    scales[2 * i] *= s;
    scales[2 * i + 1] *= s;
  }
}

cudaError_t launch_sim3(int64_t n, float* means, float* quats, float* scales, const float* sim3, const int32_t* index,
                        cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_sim3<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, means, quats, scales, sim3, index);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace s2d
