// Front end of the tracker: the depth pyramid and the vertex / normal maps the
// coarse-to-fine ICP runs on (the KinectFusion preprocessing the paper builds
// on), and the model-map preparation. One launch covers every pair of a
// batch: blockIdx.z selects the pair.
#include "kf_internal.cuh"

namespace kf {
namespace {

constexpr int kTx = 32, kTy = 8;
// resident front-end blocks per SM the register budget is sized for
#ifndef KF_FE_MINB
#define KF_FE_MINB 7
#endif

__device__ __forceinline__ bool valid_depth(float z) { return isfinite(z) && z > 0.f; }

// Model level l = level-0 model maps at pixels (x 2^l, y 2^l), converted to
// planes; a pixel is a hole (NaN vertex and normal) when any component is
// non-finite or the normal is all zero.
template <class T>
__global__ void __launch_bounds__(kTx* kTy) k_model_prep(const PairDesc* d, const float* Vin,
                                                         const float* Nin, int w, int level) {
  const LevelMaps& L = d->lv[level];
  const int x = blockIdx.x * kTx + threadIdx.x, y = blockIdx.y * kTy + threadIdx.y;
  if (x >= L.mw || y >= L.mh) return;
  const long src = ((long)(y << level) * w + (x << level)) * 3;
  const float vx = Vin[src], vy = Vin[src + 1], vz = Vin[src + 2];
  const float nx = Nin[src], ny = Nin[src + 1], nz = Nin[src + 2];
  const bool ok = isfinite(vx) && isfinite(vy) && isfinite(vz) && isfinite(nx) && isfinite(ny) &&
                  isfinite(nz) && (nx != 0.f || ny != 0.f || nz != 0.f);
  const float nan = __int_as_float(0x7fc00000);
  const int n = L.mw * L.mh, i = y * L.mw + x;
  T* V = static_cast<T*>(L.mV);
  T* N = static_cast<T*>(L.mN);
  Store<T>::st(V, i, ok ? vx : nan);
  Store<T>::st(V, n + i, ok ? vy : nan);
  Store<T>::st(V, 2 * n + i, ok ? vz : nan);
  Store<T>::st(N, i, ok ? nx : nan);
  Store<T>::st(N, n + i, ok ? ny : nan);
  Store<T>::st(N, 2 * n + i, ok ? nz : nan);
}

// ---------------------------------------------------------------------------
// Fused front end: one block owns a 32 x 32 tile of level 0 and the matching
// (32 >> l)^2 tile of every coarser level. It loads the raw depth of its tile
// plus halo into shared memory once, filters a region large enough for every
// level's neighbours, downsamples it level by level in shared memory and
// writes depth, vertex and normal maps:
//  * bilateral (level 0): D'(u) = sum D(u+d) w / sum w over the (2r+1)^2
//    window, w = exp(-|d|^2 / 2 sigma_s^2 - (D(u+d) - D(u))^2 / 2 sigma_r^2),
//    valid neighbours inside the image only, 0 where D(u) is not valid;
//  * level l+1 depth: mean of the valid depths of the 2x2 block within
//    3 sigma_r of the first valid one in scan order (the test in float32:
//    |z - anchor| <= (float)(3 sigma_r)); 0 if the block is empty;
//  * vertex v = z K^-1 (u, v, 1); normal = normalise((v(x+1,y) - v) x
//    (v(x,y+1) - v)) flipped to face the camera; the vertex is stored as NaN
//    where it or its normal is invalid, so the ICP reads one map to decide
//    whether a frame pixel takes part.
// ---------------------------------------------------------------------------
constexpr int kTile = 32;
constexpr int kRMax = 40 + 2 * 4;  // largest raw region: 4 levels, bilateral radius 4

__device__ __forceinline__ int region0(int levels) {
  return ((kTile >> (levels - 1)) + 1) << (levels - 1);
}

// Calls f(lx, ly) for the cells t = tid, tid + nthr, ... of a w x h region
// in row-major order, stepping the coordinates instead of dividing t.
template <class F>
__device__ __forceinline__ void for_region(int w, int h, int tid, int nthr, F f) {
  const int q = nthr / w, r = nthr - q * w;
  int ly = tid / w, lx = tid - ly * w;
  while (ly < h) {
    f(lx, ly);
    lx += r;
    ly += q;
    if (lx >= w) {
      lx -= w;
      ++ly;
    }
  }
}

template <class T>
__device__ void write_maps(const LevelMaps& Lg, const float* Ds, int R, int ox, int oy, int tile) {
  // a local copy: the map stores below could alias the descriptor in global
  // memory, which would force its fields to be reloaded for every pixel
  const LevelMaps L = Lg;
  // Ds: level depth region of R x R whose origin is level pixel (ox, oy)
  const int n = L.fps;  // plane stride
  const float nan = __int_as_float(0x7fc00000);
  T* V = static_cast<T*>(L.fV);
  T* N = static_cast<T*>(L.fN);
  const float ifx = 1.f / L.ffx, ify = 1.f / L.ffy;
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  for_region(tile, tile, tid, blockDim.x * blockDim.y, [&](int lx, int ly) {
    const int x = ox + lx, y = oy + ly;
    if (x >= L.fw || y >= L.fh) return;
    // (u - c) for the pixel and its right / lower neighbour; (float)(x + 1)
    // is (float)x + 1 exactly for image coordinates
    const float fx0 = (float)x, fy0 = (float)y;
    const float ux0 = fx0 - L.fcx, ux1 = (fx0 + 1.f) - L.fcx;
    const float uy0 = fy0 - L.fcy, uy1 = (fy0 + 1.f) - L.fcy;
    auto bp = [&](float ux, float uy, int sx, int sy, float3& v) -> bool {
      const float z = Ds[sy * R + sx];
      if (!(z > 0.f)) return false;
      v.x = ux * z * ifx;
      v.y = uy * z * ify;
      v.z = z;
      return true;
    };
    float3 v, v10, v01, nn = make_float3(nan, nan, nan);
    const bool ok = bp(ux0, uy0, lx, ly, v);
    bool nok = false;
    if (ok && x + 1 < L.fw && y + 1 < L.fh && bp(ux1, uy0, lx + 1, ly, v10) &&
        bp(ux0, uy1, lx, ly + 1, v01)) {
      const float ax = v10.x - v.x, ay = v10.y - v.y, az = v10.z - v.z;
      const float bx = v01.x - v.x, by = v01.y - v.y, bz = v01.z - v.z;
      float cx = ay * bz - az * by, cy = az * bx - ax * bz, cz = ax * by - ay * bx;
      const float len2 = cx * cx + cy * cy + cz * cz;
      if (len2 > 0.f && isfinite(len2)) {
        const float inv = rsqrtf(len2);
        cx *= inv;
        cy *= inv;
        cz *= inv;
        if (cx * v.x + cy * v.y + cz * v.z > 0.f) {
          cx = -cx;
          cy = -cy;
          cz = -cz;
        }
        nn = make_float3(cx, cy, cz);
        nok = true;
      }
    }
    const int i = y * L.fw + x;
    const bool keep = ok && nok;
    L.fdepth[i] = Ds[ly * R + lx];
    Store<T>::st(V, i, keep ? v.x : nan);
    Store<T>::st(V, n + i, keep ? v.y : nan);
    Store<T>::st(V, 2 * n + i, keep ? v.z : nan);
    Store<T>::st(N, i, nn.x);
    Store<T>::st(N, n + i, nn.y);
    Store<T>::st(N, 2 * n + i, nn.z);
  });
}

__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Raw depth that is missing, invalid or outside the image is held as kNoDepth
// in shared memory: its range term (k 1e30 - k z)^2 overflows to +inf, so its
// weight 2^-inf is exactly +0 and it adds nothing (0 * 1e30 = 0), with no
// per-tap test.
constexpr float kNoDepth = 1e30f;

template <int R>
__device__ __forceinline__ float bilateral_at(const float* s_raw, int RR, int cx, int cy, float z,
                                              const KParams& P) {
  // exponent sw2 - c2 (zn - z)^2 as sw2 - s^2 with s = k zn - k z, k^2 = c2
  float num = 0.f, den = 0.f;
  const float kz = P.bil_k * z;
#pragma unroll
  for (int dy = -R; dy <= R; ++dy)
#pragma unroll
    for (int dx = -R; dx <= R; ++dx) {
      const float zn = s_raw[(cy + dy) * RR + cx + dx];
      const float sd = fmaf(zn, P.bil_k, -kz);
      const float wt = ex2_approx(fmaf(-sd, sd, P.bil_sw2[(dy + R) * (2 * R + 1) + dx + R]));
      num = fmaf(wt, zn, num);
      den += wt;
    }
  return __fdividef(num, den);
}

template <class T, int RB>  // RB: the bilateral radius (a template so each launch holds one window)
__global__ void __launch_bounds__(kTx* kTy, KF_FE_MINB) k_frontend_fused(DescList list, KParams P) {
  __shared__ float s_raw[kRMax * kRMax];
  __shared__ float s_d0[40 * 40];
  __shared__ float s_d1[20 * 20];
  __shared__ float s_d2[10 * 10];
  __shared__ float s_d3[5 * 5];
  const PairDesc* d = list.d[blockIdx.z];
  const int W = d->iw, H = d->ih;
  const int X0 = blockIdx.x * kTile, Y0 = blockIdx.y * kTile;
  if (X0 >= W || Y0 >= H) return;
  const int levels = d->levels;
  const int R0 = region0(levels);
  constexpr int r = RB;  // = P.bil_radius (the launch picks the instance)
  const int RR = R0 + 2 * r;
  const int nthr = blockDim.x * blockDim.y;
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  const float* D = list.depth[blockIdx.z];
  for_region(RR, RR, tid, nthr, [&](int lx, int ly) {
    const int x = X0 - r + lx, y = Y0 - r + ly;
    float z = kNoDepth;
    if (x >= 0 && x < W && y >= 0 && y < H) {
      z = __ldg(D + y * W + x);
      if (!valid_depth(z)) z = kNoDepth;
    }
    s_raw[ly * RR + lx] = z;
  });
  __syncthreads();
  // bilateral filter over the R0 x R0 region: w = 2^(sw2 - dz^2 c2), the
  // k_bilateral weight with the exponent pre-scaled by log2(e)
  for_region(R0, R0, tid, nthr, [&](int lx, int ly) {
    const int x = X0 + lx, y = Y0 + ly;
    const float z = s_raw[(ly + r) * RR + lx + r];
    float out = 0.f;
    if (x < W && y < H && z != kNoDepth) {
      out = RB > 0 ? bilateral_at<RB>(s_raw, RR, lx + r, ly + r, z, P) : z;
    }
    s_d0[ly * R0 + lx] = out;
  });
  __syncthreads();
  // pyramid: level l+1 from level l inside shared memory (same rule as k_downsample)
  float* lev[4] = {s_d0, s_d1, s_d2, s_d3};
  for (int l = 0; l + 1 < levels; ++l) {
    const int Rs = R0 >> l, Ro = R0 >> (l + 1);
    const LevelMaps& Lo = d->lv[l + 1];
    const int ox = X0 >> (l + 1), oy = Y0 >> (l + 1);
    const float* src = lev[l];
    float* dst = lev[l + 1];
    for_region(Ro, Ro, tid, nthr, [&](int lx, int ly) {
      float out = 0.f;
      if (ox + lx < Lo.fw && oy + ly < Lo.fh) {
        const float b[4] = {src[(2 * ly) * Rs + 2 * lx], src[(2 * ly) * Rs + 2 * lx + 1],
                            src[(2 * ly + 1) * Rs + 2 * lx], src[(2 * ly + 1) * Rs + 2 * lx + 1]};
        float anchor = 0.f;
        bool have = false;
#pragma unroll
        for (int i = 0; i < 4; ++i)
          if (!have && b[i] > 0.f) {
            anchor = b[i];
            have = true;
          }
        float s = 0.f;
        int c = 0;
#pragma unroll
        for (int i = 0; i < 4; ++i)
          if (have && b[i] > 0.f && fabsf(__fsub_rn(b[i], anchor)) <= P.thr3sr32) {
            s = __fadd_rn(s, b[i]);
            ++c;
          }
        out = c ? __fdiv_rn(s, (float)c) : 0.f;
      }
      dst[ly * Ro + lx] = out;
    });
    __syncthreads();
  }
  for (int l = 0; l < levels; ++l)
    write_maps<T>(d->lv[l], lev[l], R0 >> l, X0 >> l, Y0 >> l, kTile >> l);
}

dim3 grid_for(int w, int h, int n) { return dim3((w + kTx - 1) / kTx, (h + kTy - 1) / kTy, n); }

// blockIdx.y: frame; threads stride over its 16-byte groups, kCopyU per
// thread at a time (all loads issued before the stores); a source not on a
// 16-byte boundary, and the last count % 4 floats, go one float at a time.
constexpr int kCopyU = 4;
__global__ void __launch_bounds__(256) k_copy_frames(FrameCopyList list) {
  const int f = blockIdx.y;
  const float* src = list.src[f];
  float* dst = list.dst[f];
  const int count = list.count[f];
  const int stride = gridDim.x * blockDim.x;
  const int t0 = blockIdx.x * blockDim.x + threadIdx.x;
  if ((reinterpret_cast<uintptr_t>(src) & 15u) == 0 && (reinterpret_cast<uintptr_t>(dst) & 15u) == 0) {
    const int n4 = count / 4;
    const float4* s4 = reinterpret_cast<const float4*>(src);
    float4* d4 = reinterpret_cast<float4*>(dst);
    for (int base = t0; base < n4; base += kCopyU * stride) {
      float4 v[kCopyU];
#pragma unroll
      for (int u = 0; u < kCopyU; ++u) {
        const int i = base + u * stride;
        if (i < n4) v[u] = s4[i];
      }
#pragma unroll
      for (int u = 0; u < kCopyU; ++u) {
        const int i = base + u * stride;
        if (i < n4) d4[i] = v[u];
      }
    }
    for (int i = 4 * n4 + t0; i < count; i += stride) dst[i] = src[i];
  } else {
    for (int i = t0; i < count; i += stride) dst[i] = src[i];
  }
}

}  // namespace

cudaError_t launch_copy_frames(const FrameCopyList& list, int max_count, cudaStream_t s) {
  if (list.n <= 0) return cudaSuccess;
  const int per_block = 256 * 4 * kCopyU;  // floats per block per pass
  int bx = (max_count + per_block - 1) / per_block;
  bx = bx < 1 ? 1 : (bx > 1024 ? 1024 : bx);
  k_copy_frames<<<dim3(bx, list.n), 256, 0, s>>>(list);
  return cudaGetLastError();
}

cudaError_t launch_frontend(const DescList& list, int max_w, int max_h, int levels,
                            const KParams& P, cudaStream_t s) {
  (void)levels;  // 1..4 levels and radius 0..4 (checked at tracker creation)
  const dim3 blk(kTx, kTy);
  const dim3 g((max_w + kTile - 1) / kTile, (max_h + kTile - 1) / kTile, list.n);
  const bool h = P.precision == KF_FP16;
  switch (P.bil_radius) {
    case 0: h ? k_frontend_fused<__half, 0><<<g, blk, 0, s>>>(list, P) : k_frontend_fused<float, 0><<<g, blk, 0, s>>>(list, P); break;
    case 1: h ? k_frontend_fused<__half, 1><<<g, blk, 0, s>>>(list, P) : k_frontend_fused<float, 1><<<g, blk, 0, s>>>(list, P); break;
    case 2: h ? k_frontend_fused<__half, 2><<<g, blk, 0, s>>>(list, P) : k_frontend_fused<float, 2><<<g, blk, 0, s>>>(list, P); break;
    case 3: h ? k_frontend_fused<__half, 3><<<g, blk, 0, s>>>(list, P) : k_frontend_fused<float, 3><<<g, blk, 0, s>>>(list, P); break;
    default: h ? k_frontend_fused<__half, 4><<<g, blk, 0, s>>>(list, P) : k_frontend_fused<float, 4><<<g, blk, 0, s>>>(list, P); break;
  }
  return cudaGetLastError();
}

cudaError_t launch_model_prep(const PairDesc* d_desc, const float* V, const float* N, int w,
                              int h, int levels, const int* mw, const int* mh, int precision,
                              const LevelMaps* /*host_levels*/, cudaStream_t s) {
  (void)h;
  const dim3 blk(kTx, kTy);
  for (int l = 0; l < levels; ++l) {
    if (precision == KF_FP16)
      k_model_prep<__half><<<grid_for(mw[l], mh[l], 1), blk, 0, s>>>(d_desc, V, N, w, l);
    else
      k_model_prep<float><<<grid_for(mw[l], mh[l], 1), blk, 0, s>>>(d_desc, V, N, w, l);
  }
  return cudaGetLastError();
}

}  // namespace kf
