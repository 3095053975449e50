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

}  // namespace s2d
