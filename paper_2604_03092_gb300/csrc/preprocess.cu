// Per-surfel preprocess (forward) and its reverse (chain rule to surfel
// parameters and the per-view camera se(3) tangent).
//
// Forward, per (view, surfel) -- the camera-frame quantities of the 2DGS
// surfel primitive (Sec. 3): center mu_c = R mu + t, tangent vectors
// U = s_u R t_u, V = s_v R t_v, normal n_c = R n turned to face the camera.
// The ray r = ((px - cx)/fx, (py - cy)/fy, 1) through a pixel meets the
// surfel plane at
//     u = ((V x mu_c) . r) / ((U x V) . r),   v = ((mu_c x U) . r) / ((U x V) . r)
// (the rows of adj([U V mu_c]); the homography M = K [U V mu_c] of the
// ray-splat intersection up to the intrinsics).  Written relative to the
// projected center c (where r = mu_c / z) the numerators have no constant
// term, which is what the render record stores (see splat2d_internal.cuh).
// The screen extent is the AABB of the projected disk u^2 + v^2 <= k^2,
// k^2 = 2 ln(sigma / alpha_min) (every pixel with alpha >= alpha_min lies
// inside), united with the low-pass square c +- sigma_lp k, evaluated in a
// cancellation-free form of the dual conic M diag(k^2, k^2, -1) M^T.
#include <cuda_runtime.h>

#include "splat2d_internal.cuh"

namespace s2d {

// ---------------------------------------------------------------------------
// Table upload: copies a small host table into the workspace through the
// kernel's parameter space (no host memory is touched at run time, so the
// call can be captured in a CUDA graph).
// ---------------------------------------------------------------------------
constexpr int kUploadBytes = 16384;
struct UploadBlob {
  uint4 data[kUploadBytes / 16];
};

__global__ void k_upload(const UploadBlob blob, uint4* __restrict__ dst, int n16) {
  for (int i = threadIdx.x; i < n16; i += blockDim.x) dst[i] = blob.data[i];
}

cudaError_t launch_upload(const void* host_src, size_t bytes, void* dst, cudaStream_t st) {
  const char* src = static_cast<const char*>(host_src);
  UploadBlob blob;
  for (size_t off = 0; off < bytes; off += kUploadBytes) {
    size_t n = bytes - off < (size_t)kUploadBytes ? bytes - off : (size_t)kUploadBytes;
    size_t n16 = (n + 15) / 16;
    memset(&blob, 0, sizeof(blob));
    memcpy(&blob, src + off, n);
    k_upload<<<1, 256, 0, st>>>(blob, reinterpret_cast<uint4*>(static_cast<char*>(dst) + off), (int)n16);
    count_launches(1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// ---------------------------------------------------------------------------
// Shared math
// ---------------------------------------------------------------------------
struct Surfel {
  float mx, my, mz;
  float su, sv;
  float qh[4], qn;          // normalised quaternion and the norm of the input
  float tu[3], tv[3], nw[3];  // columns of R(q)
  float op;
  float k2, kk;  // 2 ln(op / alpha_min) and its square root (per surfel, for every view)
  bool valid;
};

__device__ __forceinline__ void load_surfel(const splat2d_surfels& S, int64_t s, Surfel& f) {
  f.mx = __ldg(S.means + 3 * s + 0);
  f.my = __ldg(S.means + 3 * s + 1);
  f.mz = __ldg(S.means + 3 * s + 2);
  f.su = __ldg(S.scales + 2 * s + 0);
  f.sv = __ldg(S.scales + 2 * s + 1);
  float4 q = __ldg(reinterpret_cast<const float4*>(S.quats) + s);
  f.op = __ldg(S.opacity + s);
  float n2 = q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w;
  f.valid = n2 > 0.f && isfinite(n2);
  f.qn = sqrtf(n2);
  float inv = f.valid ? 1.0f / f.qn : 0.f;
  float w = q.x * inv, x = q.y * inv, y = q.z * inv, z = q.w * inv;
  f.qh[0] = w; f.qh[1] = x; f.qh[2] = y; f.qh[3] = z;
  // R(q) columns: t_u, t_v, n
  f.tu[0] = 1.f - 2.f * (y * y + z * z);
  f.tu[1] = 2.f * (x * y + w * z);
  f.tu[2] = 2.f * (x * z - w * y);
  f.tv[0] = 2.f * (x * y - w * z);
  f.tv[1] = 1.f - 2.f * (x * x + z * z);
  f.tv[2] = 2.f * (y * z + w * x);
  f.nw[0] = 2.f * (x * z + w * y);
  f.nw[1] = 2.f * (y * z - w * x);
  f.nw[2] = 1.f - 2.f * (x * x + y * y);
}

__device__ __forceinline__ void rot3(const float* R, const float* a, float* o) {
  o[0] = fmaf(R[0], a[0], fmaf(R[1], a[1], R[2] * a[2]));
  o[1] = fmaf(R[3], a[0], fmaf(R[4], a[1], R[5] * a[2]));
  o[2] = fmaf(R[6], a[0], fmaf(R[7], a[1], R[8] * a[2]));
}
__device__ __forceinline__ void rot3T(const float* R, const float* a, float* o) {
  o[0] = fmaf(R[0], a[0], fmaf(R[3], a[1], R[6] * a[2]));
  o[1] = fmaf(R[1], a[0], fmaf(R[4], a[1], R[7] * a[2]));
  o[2] = fmaf(R[2], a[0], fmaf(R[5], a[1], R[8] * a[2]));
}
__device__ __forceinline__ void cross3(const float* a, const float* b, float* c) {
  c[0] = fmaf(a[1], b[2], -a[2] * b[1]);
  c[1] = fmaf(a[2], b[0], -a[0] * b[2]);
  c[2] = fmaf(a[0], b[1], -a[1] * b[0]);
}
__device__ __forceinline__ float dot3(const float* a, const float* b) {
  return fmaf(a[0], b[0], fmaf(a[1], b[1], a[2] * b[2]));
}

// ceil / floor of the float-float value h + l (exact for any pair).
__device__ __forceinline__ int ff_ceil(float h, float l) {
  float s, e;
  two_sum(h, l, s, e);
  float c = ceilf(s);
  if (c == s && e > 0.f) c += 1.f;
  return (int)fminf(fmaxf(c, -1.0e6f), 1.0e6f);
}
__device__ __forceinline__ int ff_floor(float h, float l) {
  float s, e;
  two_sum(h, l, s, e);
  float c = floorf(s);
  if (c == s && e < 0.f) c -= 1.f;
  return (int)fminf(fmaxf(c, -1.0e6f), 1.0e6f);
}

// ---------------------------------------------------------------------------
// Forward preprocess
// ---------------------------------------------------------------------------
struct PreArgs {
  splat2d_surfels S;
  const DView* views;
  const DGroup* groups;
  int32_t G;
  int64_t n_work;
  RastParams P;
  uint32_t* ntiles;
  uint4* bins;  // per record: the binning passes' 16 bytes (depth bits, rect, tile count)
  float4* records;
  float4* rgrad;
  Header* hdr;
};

__device__ __forceinline__ uint32_t project_one(const PreArgs& A, const DView& vw, const Surfel& f,
                                                float4* rec_out) {
  const RastParams& P = A.P;
  if (!f.valid || !(f.op >= P.alpha_min)) return 0;
  // camera frame; the center as float-float for the projected center
  float mxh, mxl, myh, myl, mzh, mzl;
  dot3_plus(vw.R[0], vw.R[1], vw.R[2], f.mx, f.my, f.mz, vw.t[0], mxh, mxl);
  dot3_plus(vw.R[3], vw.R[4], vw.R[5], f.mx, f.my, f.mz, vw.t[1], myh, myl);
  dot3_plus(vw.R[6], vw.R[7], vw.R[8], f.mx, f.my, f.mz, vw.t[2], mzh, mzl);
  // depth key: a fixed FP32 evaluation order, reproduced bit for bit by the checker
  const float z32 = __fmaf_rn(vw.R[8], f.mz, __fmaf_rn(vw.R[7], f.my, __fmaf_rn(vw.R[6], f.mx, vw.t[2])));
  float mc[3] = {mxh, myh, mzh};
  float U[3], V[3], nc[3];
  rot3(vw.R, f.tu, U);
  rot3(vw.R, f.tv, V);
  rot3(vw.R, f.nw, nc);
  for (int k = 0; k < 3; k++) {
    U[k] *= f.su;
    V[k] *= f.sv;
  }
  if (dot3(nc, mc) > 0.f) {
    nc[0] = -nc[0]; nc[1] = -nc[1]; nc[2] = -nc[2];
  }
  const float k2 = f.k2, kk = f.kk;
  const float zmin = mzh - kk * sqrtf(U[2] * U[2] + V[2] * V[2]);
  if (!(zmin > P.z_near)) return 0;

  // projected center c = (fx mx/mz + cx, fy my/mz + cy) as float-float
  float cxh, cxl, cyh, cyl;
  {
    float q = __fdiv_rn(mxh, mzh);
    float r = __fmaf_rn(-q, mzh, mxh) + (mxl - q * mzl);
    float ql = r / mzh;
    float p, e, s, e2;
    two_prod(vw.fx, q, p, e);
    e = __fmaf_rn(vw.fx, ql, e);
    two_sum(p, vw.cx, s, e2);
    e += e2;
    cxh = s + e;
    cxl = e - (cxh - s);
  }
  {
    float q = __fdiv_rn(myh, mzh);
    float r = __fmaf_rn(-q, mzh, myh) + (myl - q * mzl);
    float ql = r / mzh;
    float p, e, s, e2;
    two_prod(vw.fy, q, p, e);
    e = __fmaf_rn(vw.fy, ql, e);
    two_sum(p, vw.cy, s, e2);
    e += e2;
    cyh = s + e;
    cyl = e - (cyh - s);
  }

  // rows of adj([U V mu_c])
  float av[3], bv[3], nv[3];
  cross3(V, mc, av);
  cross3(mc, U, bv);
  cross3(U, V, nv);

  // extent: centre offset of the projected k-ellipse and its half widths
  const float D22 = k2 * (U[2] * U[2] + V[2] * V[2]) - mzh * mzh;  // < 0 past the near test
  const float inv_d = 1.0f / (-D22);
  const float dxq = fmaxf(k2 * (bv[1] * bv[1] + av[1] * av[1]) - k2 * k2 * nv[1] * nv[1], 0.f);
  const float dyq = fmaxf(k2 * (av[0] * av[0] + bv[0] * bv[0]) - k2 * k2 * nv[0] * nv[0], 0.f);
  const float half_x = vw.fx * sqrtf(dxq) * inv_d;
  const float half_y = vw.fy * sqrtf(dyq) * inv_d;
  const float off_x = -k2 * vw.fx * (U[2] * bv[1] - V[2] * av[1]) * inv_d / mzh;
  const float off_y = -k2 * vw.fy * (V[2] * av[0] - U[2] * bv[0]) * inv_d / mzh;
  const float rlp = P.lp_r * kk;
  const float lox = fminf(off_x - half_x, -rlp), hix = fmaxf(off_x + half_x, rlp);
  const float loy = fminf(off_y - half_y, -rlp), hiy = fmaxf(off_y + half_y, rlp);
  int x0 = ff_ceil(cxh - 0.5f, cxl + lox), x1 = ff_floor(cxh - 0.5f, cxl + hix);
  int y0 = ff_ceil(cyh - 0.5f, cyl + loy), y1 = ff_floor(cyh - 0.5f, cyl + hiy);
  x0 = max(x0, 0); y0 = max(y0, 0);
  x1 = min(x1, vw.W - 1); y1 = min(y1, vw.H - 1);
  if (x0 > x1 || y0 > y1) return 0;
  const uint32_t ntx = (uint32_t)(x1 / P.tile_w - x0 / P.tile_w + 1);
  const uint32_t nty = (uint32_t)(y1 / P.tile_h - y0 / P.tile_h + 1);

  // ray-splat intersection coefficients, normalised by N = |U x V| |mu_c| / z
  // (rho' is invariant to a common scale, so the scale is free)
  const float nn = sqrtf(dot3(nv, nv)) * sqrtf(dot3(mc, mc)) / mzh;
  float p00 = 0.f, p01 = 0.f, p10 = 0.f, p11 = 0.f, p20 = 0.f, p21 = 0.f, p22 = 0.f;
  if (nn > 0.f && isfinite(nn)) {
    const float iN = 1.0f / nn;
    const float sk = 0.84932180028801907f;  // sqrt(log2(e) / 2)
    const float ifx = vw.ifx, ify = vw.ify;
    p00 = sk * av[0] * ifx * iN;
    p01 = sk * av[1] * ify * iN;
    p10 = sk * bv[0] * ifx * iN;
    p11 = sk * bv[1] * ify * iN;
    p20 = nv[0] * ifx * iN;
    p21 = nv[1] * ify * iN;
    p22 = dot3(nv, mc) / mzh * iN;
  }
  const uint32_t r0 = (uint32_t)x0 | ((uint32_t)y0 << 16);
  const uint32_t r1 = (uint32_t)x1 | ((uint32_t)y1 << 16);
  rec_out[0] = make_float4(cxh, cyh, __uint_as_float(pack_half2_scaled(cxl, cyl)), f.op);
  rec_out[1] = make_float4(p00, p01, p10, p11);
  rec_out[2] = make_float4(p20, p21, p22, 0.f);  // .w = r, filled by the caller
  rec_out[3] = make_float4(0.f, 0.f, nc[0], nc[1]);
  rec_out[4] = make_float4(nc[2], z32, __uint_as_float(r0), __uint_as_float(r1));
  return ntx * nty;
}

__global__ void __launch_bounds__(256, 3) k_preprocess(const PreArgs A) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  unsigned long long vis = 0;
  for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < A.n_work; w += stride) {
    const int g = find_group(A.groups, A.G, w);
    const DGroup grp = A.groups[g];
    const int64_t s = grp.soff + (w - grp.wbase);
    Surfel f;
    load_surfel(A.S, s, f);
    // the extent's k^2 = 2 ln(op / alpha_min): the surfel's, whatever the view
    f.k2 = 2.0f * logf(f.op / A.P.alpha_min);
    f.kk = sqrtf(f.k2);
    const float cr = __ldg(A.S.rgb + 3 * s + 0), cg = __ldg(A.S.rgb + 3 * s + 1), cb = __ldg(A.S.rgb + 3 * s + 2);
    for (int v = grp.v0; v < grp.v1; v++) {
      const DView& vw = A.views[v];
      const int64_t rec = vw.rbase + (s - vw.soff);
      float4 r[REC_F4];
      uint32_t nt = project_one(A, vw, f, r);
      A.ntiles[rec] = nt;
      A.bins[rec] = nt ? make_uint4(__float_as_uint(r[4].y), __float_as_uint(r[4].z), __float_as_uint(r[4].w), nt)
                       : make_uint4(0u, 0u, 0u, 0u);
      if (nt) {
        r[2].w = cr;
        r[3].x = cg;
        r[3].y = cb;
        float4* dst = A.records + rec * REC_F4;
#pragma unroll
        for (int k = 0; k < REC_F4; k++) dst[k] = r[k];
        vis++;
      }
    }
  }
  // warp-aggregated count of visible pairs
  for (int o = 16; o > 0; o >>= 1) vis += __shfl_xor_sync(0xffffffffu, vis, o);
  if ((threadIdx.x & 31) == 0 && vis) atomicAdd(&A.hdr->n_visible, vis);
}

cudaError_t launch_preprocess(const splat2d_surfels* S, const Layout& L, const RastParams& P, char* ws,
                              cudaStream_t st) {
  const int64_t n_work = L.n_work;
  PreArgs A;
  A.S = *S;
  A.views = reinterpret_cast<const DView*>(ws + L.views);
  A.groups = reinterpret_cast<const DGroup*>(ws + L.groups);
  A.G = L.G;
  A.n_work = n_work;
  A.P = P;
  A.ntiles = reinterpret_cast<uint32_t*>(ws + L.ntiles);
  A.bins = reinterpret_cast<uint4*>(ws + L.bins);
  A.records = reinterpret_cast<float4*>(ws + L.records);
  A.rgrad = reinterpret_cast<float4*>(ws + L.rgrad);
  A.hdr = reinterpret_cast<Header*>(ws + L.header);
  if (n_work <= 0) return cudaSuccess;
  int64_t blocks = (n_work + 255) / 256;
  int64_t cap = (int64_t)sm_count() * 16;
  if (blocks > cap) blocks = cap;
  k_preprocess<<<(unsigned)blocks, 256, 0, st>>>(A);
  count_launches(1);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Reverse preprocess: record gradients -> surfel parameters, per-view pose
// ---------------------------------------------------------------------------
struct PreBwdArgs {
  splat2d_surfels S;
  const DView* views;
  const DGroup* groups;
  int32_t G, V;
  int64_t n_work;
  int64_t per_block;   // contiguous work items per block
  RastParams P;
  const uint32_t* ntiles;
  float4* rgrad;  // consumed and cleared: zero again when this kernel ends
  splat2d_grads out;
  int32_t atomic_params;
  const Header* hdr;
};

constexpr int kPoseSlots = 64;  // per-block pose accumulators (views)

__global__ void __launch_bounds__(256, 4) k_preprocess_bwd(const PreBwdArgs A) {
  __shared__ float s_pose[kPoseSlots][6];
  __shared__ int s_vfirst;
  // a failed binning (instance capacity exceeded): nothing was accumulated
  if (A.hdr->status != 0) return;
  const int64_t wlo = (int64_t)blockIdx.x * A.per_block;
  const int64_t whi = min(wlo + A.per_block, A.n_work);
  if (wlo >= whi) return;
  for (int i = threadIdx.x; i < kPoseSlots * 6; i += blockDim.x) (&s_pose[0][0])[i] = 0.f;
  if (threadIdx.x == 0) s_vfirst = A.groups[find_group(A.groups, A.G, wlo)].v0;
  __syncthreads();
  const int vfirst = s_vfirst;
  const int lane = threadIdx.x & 31;
  const float sk = 0.84932180028801907f;
  for (int64_t wb = wlo; wb < whi; wb += blockDim.x) {
    const int64_t w = wb + threadIdx.x;
    const bool live = w < whi;
    int g = live ? find_group(A.groups, A.G, w) : find_group(A.groups, A.G, whi - 1);
    const DGroup grp = A.groups[g];
    const int64_t s = live ? grp.soff + (w - grp.wbase) : 0;
    Surfel f;
    if (live) load_surfel(A.S, s, f);
    // world-frame accumulators over the views of this surfel
    float gm[3] = {0.f, 0.f, 0.f}, gsu = 0.f, gsv = 0.f, gop = 0.f, gc[3] = {0.f, 0.f, 0.f};
    float gtu[3] = {0.f, 0.f, 0.f}, gtv[3] = {0.f, 0.f, 0.f}, gnw[3] = {0.f, 0.f, 0.f};
    // all lanes of the warp walk the same number of views so the pose
    // reduction below can use full-warp shuffles
    int nv = live ? grp.v1 - grp.v0 : 0;
    int nv_max = nv;
    for (int o = 16; o > 0; o >>= 1) nv_max = max(nv_max, __shfl_xor_sync(0xffffffffu, nv_max, o));
    for (int k = 0; k < nv_max; k++) {
      const int v = (k < nv) ? grp.v0 + k : -1;
      float pose[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
      if (v >= 0) {
        const DView& vw = A.views[v];
        const int64_t rec = vw.rbase + (s - vw.soff);
        if (A.ntiles[rec]) {
          float4* gp = A.rgrad + rec * (GRAD_F / 4);
          const float4 q0 = gp[0], q1 = gp[1], q2 = gp[2], q3 = gp[3], q4 = gp[4];
          // leave the gradient record zero for the next reverse pass
          const bool touched = (q0.x != 0.f) | (q0.y != 0.f) | (q0.z != 0.f) | (q0.w != 0.f) | (q1.x != 0.f) |
                               (q1.y != 0.f) | (q1.z != 0.f) | (q1.w != 0.f) | (q2.x != 0.f) | (q2.y != 0.f) |
                               (q2.z != 0.f) | (q2.w != 0.f) | (q3.x != 0.f) | (q3.y != 0.f) | (q3.z != 0.f) |
                               (q3.w != 0.f) | (q4.x != 0.f);
          if (touched) {
            const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
            gp[0] = z; gp[1] = z; gp[2] = z; gp[3] = z; gp[4] = z;
          }
          const float gr[17] = {q0.x, q0.y, q0.z, q0.w, q1.x, q1.y, q1.z, q1.w, q2.x,
                                q2.y, q2.z, q2.w, q3.x, q3.y, q3.z, q3.w, q4.x};
          // camera frame (FP32 is enough for the chain rule)
          float mc[3];
          mc[0] = fmaf(vw.R[0], f.mx, fmaf(vw.R[1], f.my, fmaf(vw.R[2], f.mz, vw.t[0])));
          mc[1] = fmaf(vw.R[3], f.mx, fmaf(vw.R[4], f.my, fmaf(vw.R[5], f.mz, vw.t[1])));
          mc[2] = fmaf(vw.R[6], f.mx, fmaf(vw.R[7], f.my, fmaf(vw.R[8], f.mz, vw.t[2])));
          float Ur[3], Vr[3], nc[3], U[3], V[3];
          rot3(vw.R, f.tu, Ur);
          rot3(vw.R, f.tv, Vr);
          rot3(vw.R, f.nw, nc);
          for (int j = 0; j < 3; j++) {
            U[j] = Ur[j] * f.su;
            V[j] = Vr[j] * f.sv;
          }
          const float flip = dot3(nc, mc) > 0.f ? -1.f : 1.f;
          for (int j = 0; j < 3; j++) nc[j] *= flip;
          float av[3], bv[3], nv3[3];
          cross3(V, mc, av);
          cross3(mc, U, bv);
          cross3(U, V, nv3);
          const float iz = 1.0f / mc[2];
          const float nn = sqrtf(dot3(nv3, nv3)) * sqrtf(dot3(mc, mc)) * iz;
          float gU[3] = {0.f, 0.f, 0.f}, gV[3] = {0.f, 0.f, 0.f}, gmc[3] = {0.f, 0.f, 0.f};
          if (nn > 0.f && isfinite(nn)) {
            const float iN = 1.0f / nn;
            const float ifx = vw.ifx, ify = vw.ify;
            // d/d(rows of adj): the normalisation carries no gradient
            float ga[3] = {gr[G_P00] * sk * ifx * iN, gr[G_P01] * sk * ify * iN, 0.f};
            float gb[3] = {gr[G_P10] * sk * ifx * iN, gr[G_P11] * sk * ify * iN, 0.f};
            const float gS = gr[G_P22] * iN;
            const float S = dot3(nv3, mc) * iz;
            float gn[3] = {gr[G_P20] * ifx * iN + gS * mc[0] * iz, gr[G_P21] * ify * iN + gS * mc[1] * iz,
                           gS * mc[2] * iz};
            gmc[0] += gS * nv3[0] * iz;
            gmc[1] += gS * nv3[1] * iz;
            gmc[2] += gS * nv3[2] * iz - gS * S * iz;
            float t[3];
            // a = V x mu
            cross3(mc, ga, t); for (int j = 0; j < 3; j++) gV[j] += t[j];
            cross3(ga, V, t); for (int j = 0; j < 3; j++) gmc[j] += t[j];
            // b = mu x U
            cross3(U, gb, t); for (int j = 0; j < 3; j++) gmc[j] += t[j];
            cross3(gb, mc, t); for (int j = 0; j < 3; j++) gU[j] += t[j];
            // n = U x V
            cross3(V, gn, t); for (int j = 0; j < 3; j++) gU[j] += t[j];
            cross3(gn, U, t); for (int j = 0; j < 3; j++) gV[j] += t[j];
          }
          // projected center and depth
          gmc[0] += gr[G_CX] * vw.fx * iz;
          gmc[1] += gr[G_CY] * vw.fy * iz;
          gmc[2] += -(gr[G_CX] * vw.fx * mc[0] + gr[G_CY] * vw.fy * mc[1]) * iz * iz + gr[G_Z];
          const float gnc[3] = {gr[G_NX], gr[G_NY], gr[G_NZ]};
          // pose: d/drho = g_mu_c; d/dphi = sum X x g_X over X in {mu_c, U, V, n_c}
          float t[3];
          pose[0] = gmc[0]; pose[1] = gmc[1]; pose[2] = gmc[2];
          cross3(mc, gmc, t); pose[3] += t[0]; pose[4] += t[1]; pose[5] += t[2];
          cross3(U, gU, t); pose[3] += t[0]; pose[4] += t[1]; pose[5] += t[2];
          cross3(V, gV, t); pose[3] += t[0]; pose[4] += t[1]; pose[5] += t[2];
          cross3(nc, gnc, t); pose[3] += t[0]; pose[4] += t[1]; pose[5] += t[2];
          // back to world
          float w3[3];
          rot3T(vw.R, gmc, w3); for (int j = 0; j < 3; j++) gm[j] += w3[j];
          rot3T(vw.R, gU, w3);
          gsu += dot3(f.tu, w3);
          for (int j = 0; j < 3; j++) gtu[j] += f.su * w3[j];
          rot3T(vw.R, gV, w3);
          gsv += dot3(f.tv, w3);
          for (int j = 0; j < 3; j++) gtv[j] += f.sv * w3[j];
          rot3T(vw.R, gnc, w3);
          for (int j = 0; j < 3; j++) gnw[j] += flip * w3[j];
          gop += gr[G_OP];
          gc[0] += gr[G_R]; gc[1] += gr[G_G]; gc[2] += gr[G_B];
        }
      }
      // pose of view v: reduce across the warp when the warp agrees on v
      const int v0 = __shfl_sync(0xffffffffu, v, 0);
      const bool uniform = __all_sync(0xffffffffu, v == v0);
      if (uniform) {
        if (v0 >= 0) {
#pragma unroll
          for (int j = 0; j < 6; j++)
            for (int o = 16; o > 0; o >>= 1) pose[j] += __shfl_xor_sync(0xffffffffu, pose[j], o);
          if (lane < 6) {
            float val = pose[0];
#pragma unroll
            for (int j = 1; j < 6; j++) if (lane == j) val = pose[j];
            const int slot = v0 - vfirst;
            if (slot >= 0 && slot < kPoseSlots) atomicAdd(&s_pose[slot][lane], val);
            else if (A.out.pose) atomicAdd(A.out.pose + 6 * v0 + lane, val);
          }
        }
      } else if (v >= 0) {
        const int slot = v - vfirst;
        for (int j = 0; j < 6; j++) {
          if (pose[j] == 0.f) continue;
          if (slot >= 0 && slot < kPoseSlots) atomicAdd(&s_pose[slot][j], pose[j]);
          else if (A.out.pose) atomicAdd(A.out.pose + 6 * v + j, pose[j]);
        }
      }
    }
    if (!live) continue;
    // rotation: d R(q)/d q for the three columns, then through the normalisation
    const float qw = f.qh[0], qx = f.qh[1], qy = f.qh[2], qz = f.qh[3];
    float dq[4];
    // t_u = (1-2(y^2+z^2), 2(xy+wz), 2(xz-wy))
    // t_v = (2(xy-wz), 1-2(x^2+z^2), 2(yz+wx))
    // n   = (2(xz+wy), 2(yz-wx), 1-2(x^2+y^2))
    dq[0] = 2.f * (qz * gtu[1] - qy * gtu[2] - qz * gtv[0] + qx * gtv[2] + qy * gnw[0] - qx * gnw[1]);
    dq[1] = 2.f * (qy * gtu[1] + qz * gtu[2] + qy * gtv[0] - 2.f * qx * gtv[1] + qw * gtv[2] + qz * gnw[0] -
                   qw * gnw[1] - 2.f * qx * gnw[2]);
    dq[2] = 2.f * (-2.f * qy * gtu[0] + qx * gtu[1] - qw * gtu[2] + qx * gtv[0] + qz * gtv[2] + qw * gnw[0] +
                   qz * gnw[1] - 2.f * qy * gnw[2]);
    dq[3] = 2.f * (-2.f * qz * gtu[0] + qw * gtu[1] + qx * gtu[2] - qw * gtv[0] - 2.f * qz * gtv[1] + qy * gtv[2] +
                   qx * gnw[0] + qy * gnw[1]);
    const float dd = qw * dq[0] + qx * dq[1] + qy * dq[2] + qz * dq[3];
    const float iq = f.valid ? 1.0f / f.qn : 0.f;
    float gq[4];
    for (int j = 0; j < 4; j++) gq[j] = (dq[j] - f.qh[j] * dd) * iq;
    const splat2d_grads& O = A.out;
    if (A.atomic_params) {
      if (O.means) for (int j = 0; j < 3; j++) atomicAdd(O.means + 3 * s + j, gm[j]);
      if (O.scales) { atomicAdd(O.scales + 2 * s, gsu); atomicAdd(O.scales + 2 * s + 1, gsv); }
      if (O.quats) for (int j = 0; j < 4; j++) atomicAdd(O.quats + 4 * s + j, gq[j]);
      if (O.opacity) atomicAdd(O.opacity + s, gop);
      if (O.rgb) for (int j = 0; j < 3; j++) atomicAdd(O.rgb + 3 * s + j, gc[j]);
    } else {
      if (O.means) for (int j = 0; j < 3; j++) O.means[3 * s + j] += gm[j];
      if (O.scales) { O.scales[2 * s] += gsu; O.scales[2 * s + 1] += gsv; }
      if (O.quats) for (int j = 0; j < 4; j++) O.quats[4 * s + j] += gq[j];
      if (O.opacity) O.opacity[s] += gop;
      if (O.rgb) for (int j = 0; j < 3; j++) O.rgb[3 * s + j] += gc[j];
    }
  }
  __syncthreads();
  if (A.out.pose) {
    for (int i = threadIdx.x; i < kPoseSlots * 6; i += blockDim.x) {
      const int v = vfirst + i / 6;
      const float val = (&s_pose[0][0])[i];
      if (v < A.V && val != 0.f) atomicAdd(A.out.pose + 6 * v + (i % 6), val);
    }
  }
}

cudaError_t launch_preprocess_bwd(const splat2d_surfels* S, const Layout& L, const RastParams& P, char* ws,
                                  const splat2d_grads* G, bool atomic_params, cudaStream_t st) {
  const int64_t n_work = L.n_work;
  if (n_work <= 0) return cudaSuccess;
  PreBwdArgs A;
  A.S = *S;
  A.views = reinterpret_cast<const DView*>(ws + L.views);
  A.groups = reinterpret_cast<const DGroup*>(ws + L.groups);
  A.G = L.G;
  A.V = L.V;
  A.n_work = n_work;
  A.P = P;
  A.ntiles = reinterpret_cast<const uint32_t*>(ws + L.ntiles);
  A.rgrad = reinterpret_cast<float4*>(ws + L.rgrad);
  A.hdr = reinterpret_cast<const Header*>(ws + L.header);
  A.out = *G;
  A.atomic_params = atomic_params ? 1 : 0;
  int64_t blocks_cap = (int64_t)sm_count() * 8;
  int64_t per = (n_work + blocks_cap - 1) / blocks_cap;
  per = ((per + 255) / 256) * 256;
  if (per < 256) per = 256;
  A.per_block = per;
  int64_t blocks = (n_work + per - 1) / per;
  k_preprocess_bwd<<<(unsigned)blocks, 256, 0, st>>>(A);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace s2d
