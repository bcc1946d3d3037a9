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
// bilateral filter: 1 two vertically adjacent pixels per thread step with
// packed FP32x2 arithmetic; 0 one pixel per step (the same bits either way)
#ifndef KF_FE_PAIRS
#define KF_FE_PAIRS 1
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
  const float ifx = __fdiv_rn(1.f, L.ffx), ify = __fdiv_rn(1.f, L.ffy);
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  for_region(tile, tile, tid, blockDim.x * blockDim.y, [&](int lx, int ly) {
    const int x = ox + lx, y = oy + ly;
    if (x >= L.fw || y >= L.fh) return;
    // (u - c) for the pixel and its right / lower neighbour; (float)(x + 1)
    // is (float)x + 1 exactly for image coordinates
    const float fx0 = (float)x, fy0 = (float)y;
    const float ux0 = __fsub_rn(fx0, L.fcx), ux1 = __fsub_rn(fx0 + 1.f, L.fcx);
    const float uy0 = __fsub_rn(fy0, L.fcy), uy1 = __fsub_rn(fy0 + 1.f, L.fcy);
    // vertex: x = (u_c z) / f as (u_c z) (1 / f), each product rounded
    auto bp = [&](float ux, float uy, int sx, int sy, float3& v) -> bool {
      const float z = Ds[sy * R + sx];
      if (!(z > 0.f)) return false;
      v.x = __fmul_rn(__fmul_rn(ux, z), ifx);
      v.y = __fmul_rn(__fmul_rn(uy, z), ify);
      v.z = z;
      return true;
    };
    float3 v, v10, v01, nn = make_float3(nan, nan, nan);
    const bool ok = bp(ux0, uy0, lx, ly, v);
    bool nok = false;
    if (ok && x + 1 < L.fw && y + 1 < L.fh && bp(ux1, uy0, lx + 1, ly, v10) &&
        bp(ux0, uy1, lx, ly + 1, v01)) {
      // the decisions (a normal exists; it faces the camera) are float32 with
      // every operation rounded in this order, no contraction: a = v10 - v,
      // b = v01 - v; c = a x b, products rounded, then the difference;
      // l2 = (cx cx + cy cy) + cz cz: a normal iff finite and > 0;
      // s = (cx vx + cy vy) + cz vz > 0 flips it (decided before normalising)
      const float ax = __fsub_rn(v10.x, v.x), ay = __fsub_rn(v10.y, v.y), az = __fsub_rn(v10.z, v.z);
      const float bx = __fsub_rn(v01.x, v.x), by = __fsub_rn(v01.y, v.y), bz = __fsub_rn(v01.z, v.z);
      const float cx = __fsub_rn(__fmul_rn(ay, bz), __fmul_rn(az, by));
      const float cy = __fsub_rn(__fmul_rn(az, bx), __fmul_rn(ax, bz));
      const float cz = __fsub_rn(__fmul_rn(ax, by), __fmul_rn(ay, bx));
      const float len2 = __fadd_rn(__fadd_rn(__fmul_rn(cx, cx), __fmul_rn(cy, cy)), __fmul_rn(cz, cz));
      if (len2 > 0.f && isfinite(len2)) {
        const float sd = __fadd_rn(__fadd_rn(__fmul_rn(cx, v.x), __fmul_rn(cy, v.y)), __fmul_rn(cz, v.z));
        const float inv = sd > 0.f ? -rsqrtf(len2) : rsqrtf(len2);
        nn = make_float3(cx * inv, cy * inv, cz * inv);
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

// The filter for two vertically adjacent pixels (cx, cy) and (cx, cy + 1) at
// once: s_pair[y RR + x] holds (D(x, y), D(x, y + 1)), so one 8-byte load
// brings both pixels' neighbour at a tap, and packed FP32x2 fused
// multiply-adds and additions (each lane the scalar operation of
// bilateral_at, in the same order: the same bits) weigh and sum them.
template <int R>
__device__ __forceinline__ float2 bilateral_pair(const float2* s_pair, int RR, int cx, int cy,
                                                 float2 z, const KParams& P) {
  float2 num = make_float2(0.f, 0.f), den = make_float2(0.f, 0.f);
  const float2 k2 = make_float2(P.bil_k, P.bil_k);
  const float2 mkz = make_float2(-(P.bil_k * z.x), -(P.bil_k * z.y));
#pragma unroll
  for (int dy = -R; dy <= R; ++dy)
#pragma unroll
    for (int dx = -R; dx <= R; ++dx) {
      const float2 zn = s_pair[(cy + dy) * RR + cx + dx];
      const float2 sd = __ffma2_rn(zn, k2, mkz);
      const float sw = P.bil_sw2[(dy + R) * (2 * R + 1) + dx + R];
      const float2 e = __ffma2_rn(make_float2(-sd.x, -sd.y), sd, make_float2(sw, sw));
      const float2 wt = make_float2(ex2_approx(e.x), ex2_approx(e.y));
      num = __ffma2_rn(wt, zn, num);
      den = __fadd2_rn(den, wt);
    }
  return make_float2(__fdividef(num.x, den.x), __fdividef(num.y, den.y));
}

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
#if KF_FE_PAIRS
  // raw depth as vertical pairs: s_pair[y RR + x] = (D(x, y), D(x, y + 1)),
  // the row below the region holding no depth
  __shared__ float2 s_pair[kRMax * kRMax];
#else
  __shared__ float s_raw[kRMax * kRMax];
#endif
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
#if KF_FE_PAIRS
    s_pair[ly * RR + lx].x = z;
    if (ly > 0) s_pair[(ly - 1) * RR + lx].y = z;
    if (ly == RR - 1) s_pair[ly * RR + lx].y = kNoDepth;
#else
    s_raw[ly * RR + lx] = z;
#endif
  });
  __syncthreads();
  // bilateral filter over the R0 x R0 region: w = 2^(sw2 - dz^2 c2), the
  // k_bilateral weight with the exponent pre-scaled by log2(e)
#if KF_FE_PAIRS
  // two vertically adjacent pixels per step (rows ly and ly + 1; a region
  // with an odd row count filters one row below it and drops the result)
  for_region(R0, (R0 + 1) >> 1, tid, nthr, [&](int lx, int py) {
    const int ly = 2 * py;
    const int x = X0 + lx, y = Y0 + ly;
    const float2 z = s_pair[(ly + r) * RR + lx + r];
    float2 out = RB > 0 ? bilateral_pair<RB>(s_pair, RR, lx + r, ly + r, z, P) : z;
    const bool xin = x < W;
    s_d0[ly * R0 + lx] = xin && y < H && z.x != kNoDepth ? out.x : 0.f;
    if (ly + 1 < R0) s_d0[(ly + 1) * R0 + lx] = xin && y + 1 < H && z.y != kNoDepth ? out.y : 0.f;
  });
#else
  for_region(R0, R0, tid, nthr, [&](int lx, int ly) {
    const int x = X0 + lx, y = Y0 + ly;
    const float z = s_raw[(ly + r) * RR + lx + r];
    float out = 0.f;
    if (x < W && y < H && z != kNoDepth) {
      out = RB > 0 ? bilateral_at<RB>(s_raw, RR, lx + r, ly + r, z, P) : z;
    }
    s_d0[ly * R0 + lx] = out;
  });
#endif
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

// ---------------------------------------------------------------------------
// Integral-image normals (Sec. 3.3; Holzer et al.): the average 3D gradient
// over a square window whose half-size follows the depth and stops short of
// depth edges. One block owns a 32 x 32 tile of one level of one frame (four
// rows per thread; blockIdx.x walks the tiles of every level, blockIdx.y is
// the frame) and does everything in shared memory:
//  * the level depth of the tile plus a halo of rmax + 1;
//  * edge flags over the tile plus rmax, one 64-bit mask per row (a warp per
//    row, ballots): no depth, or a 4-neighbour inside the image without depth
//    or with |z_w - z| > delta z (float32); pixels outside the image count as
//    edges too, which bounds the window exactly as the border distance does;
//  * fixed-point vertices Q = rint(v 2^20) (int64, round half to even), v the
//    front end's float32 vertex ((x - cx) z) (1/fx), ((y - cy) z) (1/fy), z,
//    0 without depth, and their local integral image (3 channels): window
//    sums are exact integers, the same however they are added;
//  * per pixel the chessboard distance to the nearest edge (the smallest
//    square around it holding an edge bit, from the row masks), the half-size
//    r = min(floor((a + b z) 2^-l), dist - 1, border distance, rmax),
//    g_h = S(right) - S(left), g_v = S(below) - S(above), and the normal
//    (g_h x g_v) / |g_h x g_v| in float32 with each operation rounded (g
//    scaled by 2^-20 exactly), flipped to face the camera; no normal unless
//    r >= 1 and the cross product is non-zero.
// Rewrites the level's vertex (NaN without a normal) and normal maps.
// ---------------------------------------------------------------------------
constexpr float kFix = 1048576.f;                // 2^20
constexpr float kFixInv = 9.5367431640625e-07f;  // 2^-20
constexpr int kIiRows = 4 * kTy;                 // output rows per block

// tiles of each level of the largest frame of a launch, and their prefix
struct IiGrid {
  int tx[KF_MAX_LEVELS];       // tiles per row
  int first[KF_MAX_LEVELS + 1];  // first tile of each level; first[levels] = total
  int levels;
};

// shared-memory layout of one tile for half-size cap rmax (<= 15: a row of
// the window region, 32 + 2 rmax <= 62 pixels, fits one 64-bit mask)
struct IiTile {
  int rw, rh;    // window region: tile plus rmax on each side
  int dw, dh;    // depth region: window region plus 1
  size_t ii, mask, depth, bytes;  // byte offsets and total
  __host__ __device__ IiTile(int rmax) {
    rw = kTx + 2 * rmax;
    rh = kIiRows + 2 * rmax;
    dw = rw + 2;
    dh = rh + 2;
    ii = 0;
    mask = ii + (size_t)3 * (rw + 1) * (rh + 1) * sizeof(long long);
    depth = mask + (size_t)rh * sizeof(unsigned long long);
    bytes = (depth + (size_t)dw * dh * sizeof(float) + 15) / 16 * 16;
  }
};

// chessboard distance from region pixel (x, y) to the nearest edge, capped
// at C: the smallest d whose square (rows y-d..y+d, columns x-d..x+d) holds
// an edge bit, grown one ring at a time (x - C + 1 >= 0 and the rows and
// columns up to distance C - 1 lie inside the region)
__device__ __forceinline__ int edge_distance(const unsigned long long* M, int x, int y, int C) {
  unsigned long long rows = 0;
  for (int d = 0; d < C; ++d) {
    rows |= M[y - d] | M[y + d];
    const unsigned long long win = (rows >> (x - d)) & ((2ull << (2 * d)) - 1ull);
    if (win) return d;
  }
  return C;
}

template <class T>
__global__ void __launch_bounds__(kTx * kTy) k_ii_normals(DescList list, IiGrid G, KParams P) {
  extern __shared__ __align__(16) unsigned char s_ii_raw[];
  int l = 0;
  while (l + 1 < G.levels && (int)blockIdx.x >= G.first[l + 1]) ++l;
  const int tile = blockIdx.x - G.first[l];
  const LevelMaps L = list.d[blockIdx.y]->lv[l];
  const int W = L.fw, H = L.fh;
  const int X0 = (tile % G.tx[l]) * kTx, Y0 = (tile / G.tx[l]) * kIiRows;
  if (X0 >= W || Y0 >= H) return;
  const int rmax = P.ii_rmax, C = rmax + 1;
  const IiTile tl(rmax);
  long long* sI = reinterpret_cast<long long*>(s_ii_raw + tl.ii);
  unsigned long long* sM = reinterpret_cast<unsigned long long*>(s_ii_raw + tl.mask);
  float* sD = reinterpret_cast<float*>(s_ii_raw + tl.depth);
  const int tid = threadIdx.y * kTx + threadIdx.x, nt = kTx * kTy;
  const int lane = threadIdx.x, warp = threadIdx.y;
  const float nan = __int_as_float(0x7fc00000);
  const float ifx = __fdiv_rn(1.f, L.ffx), ify = __fdiv_rn(1.f, L.ffy);
  // the front end's vertex, operation for operation
  auto vertex = [&](int x, int y, float z) {
    return make_float3(__fmul_rn(__fmul_rn(__fsub_rn((float)x, L.fcx), z), ifx),
                       __fmul_rn(__fmul_rn(__fsub_rn((float)y, L.fcy), z), ify), z);
  };
  const int iw = tl.rw + 1, ipl = (tl.rw + 1) * (tl.rh + 1);  // integral row stride, plane
  // 1. depth with halo rmax + 1 (NaN outside the image: no depth)
  for (int k = tid; k < tl.dw * tl.dh; k += nt) {
    const int gy = Y0 - rmax - 1 + k / tl.dw, gx = X0 - rmax - 1 + k % tl.dw;
    sD[k] = (gx >= 0 && gx < W && gy >= 0 && gy < H) ? L.fdepth[gy * W + gx] : nan;
  }
  for (int k = tid; k < 3 * iw; k += nt) sI[(k / iw) * ipl + k % iw] = 0;  // row 0
  for (int k = tid; k < 3 * (tl.rh + 1); k += nt)
    sI[(k / (tl.rh + 1)) * ipl + (k % (tl.rh + 1)) * iw] = 0;                // column 0
  __syncthreads();
  // 2. a warp per region row: edge mask and fixed-point vertices
  for (int ry = warp; ry < tl.rh; ry += kTy) {
    const int gy = Y0 - rmax + ry;
    unsigned long long m = 0;
#pragma unroll
    for (int half = 0; half < 2; ++half) {
      const int rx = lane + 32 * half;
      bool edge = true;
      long long q[3] = {0, 0, 0};
      if (rx < tl.rw) {
        const int gx = X0 - rmax + rx;
        const float* d = sD + (ry + 1) * tl.dw + (rx + 1);
        const float z = d[0];
        if (gx >= 0 && gx < W && gy >= 0 && gy < H && valid_depth(z)) {
          edge = false;
          const float thr = __fmul_rn(P.ii_delta, z);
          const float zn[4] = {d[1], d[-1], d[tl.dw], d[-tl.dw]};
          const bool inside[4] = {gx + 1 < W, gx > 0, gy + 1 < H, gy > 0};
#pragma unroll
          for (int k = 0; k < 4; ++k)
            if (inside[k] && (!valid_depth(zn[k]) || fabsf(__fsub_rn(zn[k], z)) > thr)) edge = true;
          const float3 v = vertex(gx, gy, z);
          q[0] = __float2ll_rn(__fmul_rn(v.x, kFix));
          q[1] = __float2ll_rn(__fmul_rn(v.y, kFix));
          q[2] = __float2ll_rn(__fmul_rn(v.z, kFix));
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) sI[c * ipl + (ry + 1) * iw + (rx + 1)] = q[c];
      }
      m |= (unsigned long long)__ballot_sync(0xffffffffu, edge && rx < tl.rw) << (32 * half);
    }
    if (lane == 0) sM[ry] = m;
  }
  __syncthreads();
  // 3. row prefix sums, then 4. column prefix sums
  for (int k = tid; k < 3 * tl.rh; k += nt) {
    long long* row = sI + (k / tl.rh) * ipl + (k % tl.rh + 1) * iw;
    long long acc = 0;
    for (int x = 1; x <= tl.rw; ++x) {
      acc += row[x];
      row[x] = acc;
    }
  }
  __syncthreads();
  for (int k = tid; k < 3 * tl.rw; k += nt) {
    long long* col = sI + (k / tl.rw) * ipl + (k % tl.rw + 1);
    long long acc = 0;
    for (int y = 1; y <= tl.rh; ++y) {
      acc += col[y * iw];
      col[y * iw] = acc;
    }
  }
  __syncthreads();
  // 5. four output pixels per thread
  T* V = static_cast<T*>(L.fV);
  T* N = static_cast<T*>(L.fN);
  const int ps = L.fps;
  const float lscale = ldexpf(1.f, -l);
#pragma unroll 1
  for (int part = 0; part < kIiRows / kTy; ++part) {
    const int oy = threadIdx.y + kTy * part;
    const int x = X0 + lane, y = Y0 + oy;
    if (x >= W || y >= H) continue;
    const int rx = lane + rmax, ry = oy + rmax;
    const float z = sD[(ry + 1) * tl.dw + (rx + 1)];
    const float3 v = vertex(x, y, z);
    const int dist = edge_distance(sM, rx, ry, C);
    float t = __fmul_rn(__fadd_rn(P.ii_a, __fmul_rn(P.ii_b, z)), lscale);
    if (!isfinite(t)) t = 0.f;
    const int rdd = (int)floorf(fminf(t, (float)rmax));
    const int rimg = min(min(x, W - 1 - x), min(y, H - 1 - y));
    const int r = min(min(rdd, dist - 1), min(rimg, rmax));
    float n[3] = {nan, nan, nan};
    bool ok = false;
    if (valid_depth(z) && r >= 1) {
      // sum of Q over region columns x0..x1, rows y0..y1 (inclusive), channel c
      auto S = [&](int c, int x0, int x1, int y0, int y1) -> long long {
        const long long* I = sI + c * ipl;
        return I[(y1 + 1) * iw + x1 + 1] - I[y0 * iw + x1 + 1] - I[(y1 + 1) * iw + x0] + I[y0 * iw + x0];
      };
      float gh[3], gv[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const long long h = S(c, rx + 1, rx + r, ry - r, ry + r) - S(c, rx - r, rx - 1, ry - r, ry + r);
        const long long w = S(c, rx - r, rx + r, ry + 1, ry + r) - S(c, rx - r, rx + r, ry - r, ry - 1);
        gh[c] = __fmul_rn(__ll2float_rn(h), kFixInv);
        gv[c] = __fmul_rn(__ll2float_rn(w), kFixInv);
      }
      const float cx = __fsub_rn(__fmul_rn(gh[1], gv[2]), __fmul_rn(gh[2], gv[1]));
      const float cy = __fsub_rn(__fmul_rn(gh[2], gv[0]), __fmul_rn(gh[0], gv[2]));
      const float cz = __fsub_rn(__fmul_rn(gh[0], gv[1]), __fmul_rn(gh[1], gv[0]));
      float n2 = __fadd_rn(__fmul_rn(cx, cx), __fmul_rn(cy, cy));
      n2 = __fadd_rn(n2, __fmul_rn(cz, cz));
      if (n2 > 0.f) {
        const float sn = __fsqrt_rn(n2);
        n[0] = __fdiv_rn(cx, sn);
        n[1] = __fdiv_rn(cy, sn);
        n[2] = __fdiv_rn(cz, sn);
        float dot = __fadd_rn(__fmul_rn(n[0], v.x), __fmul_rn(n[1], v.y));
        dot = __fadd_rn(dot, __fmul_rn(n[2], v.z));
        if (dot > 0.f) {
          n[0] = -n[0];
          n[1] = -n[1];
          n[2] = -n[2];
        }
        ok = true;
      }
    }
    const int i = y * W + x;
    Store<T>::st(V, i, ok ? v.x : nan);
    Store<T>::st(V, ps + i, ok ? v.y : nan);
    Store<T>::st(V, 2 * ps + i, ok ? v.z : nan);
    Store<T>::st(N, i, n[0]);
    Store<T>::st(N, ps + i, n[1]);
    Store<T>::st(N, 2 * ps + i, n[2]);
  }
}

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

cudaError_t launch_integral_normals(const DescList& list, int max_w, int max_h, int levels,
                                    const KParams& P, cudaStream_t s) {
  const IiTile tl(P.ii_rmax);
  IiGrid G;
  G.levels = levels;
  G.first[0] = 0;
  for (int l = 0; l < levels; ++l) {
    const int w = max_w >> l, h = max_h >> l;
    G.tx[l] = (w + kTx - 1) / kTx;
    G.first[l + 1] = G.first[l] + G.tx[l] * ((h + kIiRows - 1) / kIiRows);
  }
  const dim3 g(G.first[levels], list.n);
  cudaError_t e;
  if (P.precision == KF_FP16) {
    e = cudaFuncSetAttribute(k_ii_normals<__half>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tl.bytes);
    if (e != cudaSuccess) return e;
    k_ii_normals<__half><<<g, dim3(kTx, kTy), tl.bytes, s>>>(list, G, P);
  } else {
    e = cudaFuncSetAttribute(k_ii_normals<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tl.bytes);
    if (e != cudaSuccess) return e;
    k_ii_normals<float><<<g, dim3(kTx, kTy), tl.bytes, s>>>(list, G, P);
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
