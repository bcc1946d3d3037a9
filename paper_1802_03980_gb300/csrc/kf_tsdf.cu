// Model producer: TSDF integration of depth frames into a cube of voxels and
// raycasting of the model's world vertex and normal maps (KinectFusion's
// mapping half; the paper keeps a 512^3 cube of at most 6 m side, Sec. 4.4,
// and aligns each frame to "the model reconstructed so far", Sec. 3).
//
// Every result that decides something discrete (the pixel a voxel projects
// to, the truncation test, the cell of a sample, a zero crossing) is an
// explicitly rounded float32 operation in a fixed order, so that a float32
// re-evaluation elsewhere reproduces the decisions bit for bit.
#include <cmath>
#include <cstring>
#include <string>

#include "kf_internal.cuh"

namespace kf {
namespace {

struct VolGeom {
  int res;
  float s;           // voxel size: (float)side / (float)res
  float o[3];        // world position of the cube's lower corner
  float mu, w_max;
};

struct Cam32 {
  int w, h;
  float fx, fy, cx, cy;
};

__device__ __forceinline__ float rowv(const float* R, float t, float x, float y, float z) {
  float a = __fadd_rn(__fmul_rn(R[0], x), __fmul_rn(R[1], y));
  a = __fadd_rn(a, __fmul_rn(R[2], z));
  return __fadd_rn(a, t);
}

// world -> camera rows [R^T | -R^T t] (float32) for integration
struct Xf12 {
  float r[9];
  float t[3];
};

// one voxel: F <- (W F + f) / (W + 1), W <- min(W + 1, w_max)
__device__ __forceinline__ void integrate_voxel(float* F, float* W, const VolGeom& g, const float* D,
                                                const Cam32& cam, const Xf12& xf, int i, int j, int k) {
  const float x = __fadd_rn(g.o[0], __fmul_rn((float)i + 0.5f, g.s));
  const float y = __fadd_rn(g.o[1], __fmul_rn((float)j + 0.5f, g.s));
  const float z = __fadd_rn(g.o[2], __fmul_rn((float)k + 0.5f, g.s));
  const float px = rowv(xf.r + 0, xf.t[0], x, y, z);
  const float py = rowv(xf.r + 3, xf.t[1], x, y, z);
  const float pz = rowv(xf.r + 6, xf.t[2], x, y, z);
  if (!(pz > 0.f)) return;
  const float uf = __fadd_rn(__fdiv_rn(__fmul_rn(cam.fx, px), pz), cam.cx);
  const float vf = __fadd_rn(__fdiv_rn(__fmul_rn(cam.fy, py), pz), cam.cy);
  const float ur = rintf(uf), vr = rintf(vf);
  if (!(ur >= 0.f && ur <= (float)(cam.w - 1) && vr >= 0.f && vr <= (float)(cam.h - 1))) return;
  const float d = __ldg(D + (size_t)vr * cam.w + (size_t)ur);
  if (!(isfinite(d) && d > 0.f)) return;
  const float eta = __fsub_rn(d, pz);
  if (!(eta >= -g.mu)) return;
  const float f = fminf(1.f, __fdiv_rn(eta, g.mu));
  const size_t v = ((size_t)k * g.res + j) * g.res + i;
  const float w = W[v];
  F[v] = __fdiv_rn(__fadd_rn(__fmul_rn(w, F[v]), f), __fadd_rn(w, 1.f));
  W[v] = fminf(__fadd_rn(w, 1.f), g.w_max);
}

// Integration visits only the voxels of bricks (8^3 voxels) that can lie in
// the image frustum: a brick is dropped when its bounding sphere lies wholly
// behind the camera or wholly outside one side plane of the frustum taken one
// pixel wider than the image on every side (so the float32 rounding of a
// voxel's projection, a small fraction of a pixel at depths >= 1 cm, cannot
// bring a dropped voxel into the image); bricks reaching closer than 1 cm to
// the camera plane are always kept. Every voxel that passes the per-voxel
// tests lies in a kept brick, so the volume is the same as from a pass over
// every voxel.
constexpr int kBrick = 8;
struct Frustum {
  float n[4][3];  // unit normals of the side planes (camera frame), inside: n . p >= 0
};

__global__ void k_cull_bricks(VolGeom g, Xf12 xf, Frustum fr, int nb, int* list, unsigned* count) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nb * nb * nb) return;
  const int bi = b % nb, bj = (b / nb) % nb, bk = b / (nb * nb);
  const float h = 0.5f * kBrick * g.s;  // half the brick's edge
  const float cx = g.o[0] + (float)(bi * kBrick) * g.s + h;
  const float cy = g.o[1] + (float)(bj * kBrick) * g.s + h;
  const float cz = g.o[2] + (float)(bk * kBrick) * g.s + h;
  const float px = xf.r[0] * cx + xf.r[1] * cy + xf.r[2] * cz + xf.t[0];
  const float py = xf.r[3] * cx + xf.r[4] * cy + xf.r[5] * cz + xf.t[1];
  const float pz = xf.r[6] * cx + xf.r[7] * cy + xf.r[8] * cz + xf.t[2];
  const float R = 1.7320509f * h + 1e-3f;  // bounding sphere plus a rounding margin
  if (pz < -R) return;
  if (pz - R >= 0.01f) {
    for (int q = 0; q < 4; ++q)
      if (fr.n[q][0] * px + fr.n[q][1] * py + fr.n[q][2] * pz < -R) return;
  }
  list[atomicAdd(count, 1u)] = b;
}

// one block of 8^3 threads per kept brick, bricks taken in turn
__global__ void __launch_bounds__(kBrick * kBrick * kBrick) k_integrate_bricks(
    float* F, float* W, VolGeom g, const float* D, Cam32 cam, Xf12 xf, int nb, const int* list,
    const unsigned* count) {
  const unsigned n = *count;
  const int t = threadIdx.x;
  const int di = t % kBrick, dj = (t / kBrick) % kBrick, dk = t / (kBrick * kBrick);
  for (unsigned q = blockIdx.x; q < n; q += gridDim.x) {
    const int b = list[q];
    const int i = (b % nb) * kBrick + di, j = ((b / nb) % nb) * kBrick + dj, k = (b / (nb * nb)) * kBrick + dk;
    if (i < g.res && j < g.res && k < g.res) integrate_voxel(F, W, g, D, cam, xf, i, j, k);
  }
}

__global__ void k_reset(float* F, float* W, size_t n) {
  for (size_t v = blockIdx.x * (size_t)blockDim.x + threadIdx.x; v < n; v += (size_t)gridDim.x * blockDim.x) {
    F[v] = 1.f;
    W[v] = 0.f;
  }
}

// trilinear field value at world point q; false when the cell leaves the
// cube or has an unobserved corner (W = 0)
__device__ __forceinline__ bool sample(const float* F, const float* W, const VolGeom& g,
                                       float qx, float qy, float qz, float& out) {
  const float gx = __fsub_rn(__fdiv_rn(__fsub_rn(qx, g.o[0]), g.s), 0.5f);
  const float gy = __fsub_rn(__fdiv_rn(__fsub_rn(qy, g.o[1]), g.s), 0.5f);
  const float gz = __fsub_rn(__fdiv_rn(__fsub_rn(qz, g.o[2]), g.s), 0.5f);
  const float fx0 = floorf(gx), fy0 = floorf(gy), fz0 = floorf(gz);
  if (!(fx0 >= 0.f && fx0 <= (float)(g.res - 2) && fy0 >= 0.f && fy0 <= (float)(g.res - 2) &&
        fz0 >= 0.f && fz0 <= (float)(g.res - 2)))
    return false;
  const int x0 = (int)fx0, y0 = (int)fy0, z0 = (int)fz0;
  const float tx = __fsub_rn(gx, fx0), ty = __fsub_rn(gy, fy0), tz = __fsub_rn(gz, fz0);
  const size_t r = g.res, b = ((size_t)z0 * r + y0) * r + x0;
  const size_t o[8] = {b, b + 1, b + r, b + r + 1, b + r * r, b + r * r + 1, b + r * r + r, b + r * r + r + 1};
  float c[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    if (!(__ldg(W + o[q]) > 0.f)) return false;
    c[q] = __ldg(F + o[q]);
  }
  auto lerp = [](float a, float bb, float u) { return __fadd_rn(a, __fmul_rn(u, __fsub_rn(bb, a))); };
  const float c00 = lerp(c[0], c[1], tx), c10 = lerp(c[2], c[3], tx);
  const float c01 = lerp(c[4], c[5], tx), c11 = lerp(c[6], c[7], tx);
  out = lerp(lerp(c00, c10, ty), lerp(c01, c11, ty), tz);
  return true;
}

struct RayParams {
  float R[9];   // camera -> world rotation (float32)
  float c[3];   // camera centre (world)
  float zn, zf, dz;
  int steps;    // samples k = 0 .. steps - 1 (z_k <= zf)
};

// one thread per pixel: first front-to-back zero crossing of the field
__global__ void __launch_bounds__(256) k_raycast(const float* F, const float* W, VolGeom g,
                                                 Cam32 cam, RayParams rp, float* V, float* N) {
  const int u = blockIdx.x * blockDim.x + threadIdx.x, v = blockIdx.y;
  if (u >= cam.w) return;
  const float nan = __int_as_float(0x7fc00000);
  const float dcx = __fdiv_rn(__fsub_rn((float)u, cam.cx), cam.fx);
  const float dcy = __fdiv_rn(__fsub_rn((float)v, cam.cy), cam.fy);
  const float dx = rowv(rp.R + 0, 0.f, dcx, dcy, 1.f);
  const float dy = rowv(rp.R + 3, 0.f, dcx, dcy, 1.f);
  const float dzv = rowv(rp.R + 6, 0.f, dcx, dcy, 1.f);
  float out[6] = {nan, nan, nan, nan, nan, nan};
  bool have_prev = false;
  float zp = 0.f, fp = 0.f;
  for (int k = 0; k < rp.steps; ++k) {
    const float z = __fadd_rn(rp.zn, __fmul_rn((float)k, rp.dz));
    if (z > rp.zf) break;
    const float qx = __fadd_rn(rp.c[0], __fmul_rn(z, dx));
    const float qy = __fadd_rn(rp.c[1], __fmul_rn(z, dy));
    const float qz = __fadd_rn(rp.c[2], __fmul_rn(z, dzv));
    float f;
    if (!sample(F, W, g, qx, qy, qz, f)) {
      have_prev = false;
      continue;
    }
    if (have_prev && fp > 0.f && f <= 0.f) {
      const float zs = __fadd_rn(zp, __fmul_rn(rp.dz, __fdiv_rn(fp, __fsub_rn(fp, f))));
      const float vx = __fadd_rn(rp.c[0], __fmul_rn(zs, dx));
      const float vy = __fadd_rn(rp.c[1], __fmul_rn(zs, dy));
      const float vz = __fadd_rn(rp.c[2], __fmul_rn(zs, dzv));
      float a, b, gx, gy, gz;
      if (sample(F, W, g, __fadd_rn(vx, g.s), vy, vz, a) && sample(F, W, g, __fsub_rn(vx, g.s), vy, vz, b)) {
        gx = a - b;
        if (sample(F, W, g, vx, __fadd_rn(vy, g.s), vz, a) && sample(F, W, g, vx, __fsub_rn(vy, g.s), vz, b)) {
          gy = a - b;
          if (sample(F, W, g, vx, vy, __fadd_rn(vz, g.s), a) && sample(F, W, g, vx, vy, __fsub_rn(vz, g.s), b)) {
            gz = a - b;
            const float n2 = gx * gx + gy * gy + gz * gz;
            if (n2 > 0.f) {
              const float inv = 1.f / sqrtf(n2);
              out[0] = vx;
              out[1] = vy;
              out[2] = vz;
              out[3] = gx * inv;
              out[4] = gy * inv;
              out[5] = gz * inv;
            }
          }
        }
      }
      break;
    }
    if (have_prev && fp < 0.f && f > 0.f) break;  // a back face: no surface
    have_prev = true;
    zp = z;
    fp = f;
  }
  const size_t p = ((size_t)v * cam.w + u) * 3;
  V[p] = out[0];
  V[p + 1] = out[1];
  V[p + 2] = out[2];
  N[p] = out[3];
  N[p + 1] = out[4];
  N[p + 2] = out[5];
}

}  // namespace
}  // namespace kf

using namespace kf;

struct kf_volume {
  kf_volume_params p;
  VolGeom g;
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  float* F = nullptr;
  float* W = nullptr;
  float* depth = nullptr;   // staging for host frames (grown on demand)
  size_t depth_cap = 0;
  float* maps = nullptr;    // staging for host outputs (grown on demand)
  size_t maps_cap = 0;
  int nb = 0;               // bricks per edge
  int* bricks = nullptr;    // kept bricks of the current integration
  unsigned* brick_count = nullptr;
  int sms = 1;
  std::string err;
};

namespace {

kf_status vfail(kf_volume* v, kf_status s, const std::string& msg) {
  if (v) v->err = msg;
  return s;
}

kf_status vcuda(kf_volume* v, cudaError_t e, const char* where) {
  if (v) v->err = std::string(where) + ": " + cudaGetErrorString(e);
  return e == cudaErrorMemoryAllocation ? KF_ERR_OOM : KF_ERR_CUDA;
}

#define KV_CK(v, expr)                                    \
  do {                                                    \
    cudaError_t e_ = (expr);                              \
    if (e_ != cudaSuccess) return vcuda(v, e_, #expr);    \
  } while (0)

bool cam_ok(const kf_intrinsics* K) {
  return K && K->width > 0 && K->height > 0 && std::isfinite(K->fx) && std::isfinite(K->fy) &&
         std::isfinite(K->cx) && std::isfinite(K->cy) && K->fx != 0.0 && K->fy != 0.0;
}

Cam32 cam32(const kf_intrinsics* K) {
  return Cam32{K->width, K->height, (float)K->fx, (float)K->fy, (float)K->cx, (float)K->cy};
}

bool pose_ok(const double* T) {
  if (!T) return false;
  for (int i = 0; i < 16; ++i)
    if (!std::isfinite(T[i])) return false;
  return true;
}

kf_status grow(kf_volume* v, float** buf, size_t* cap, size_t bytes) {
  if (*cap >= bytes) return KF_OK;
  cudaFree(*buf);
  *buf = nullptr;
  *cap = 0;
  KV_CK(v, cudaMalloc(buf, bytes));
  *cap = bytes;
  return KF_OK;
}

}  // namespace

extern "C" {

kf_status kf_volume_default_params(kf_volume_params* p) {
  if (!p) return KF_ERR_INVALID_ARG;
  p->res = 512;
  p->side = 6.0f;
  p->origin[0] = -3.0f;
  p->origin[1] = -3.0f;
  p->origin[2] = -3.0f;
  p->mu = 0.05f;  // ~4 voxels: the band behind a surface must hold several samples
  p->w_max = 64.0f;
  return KF_OK;
}

kf_status kf_volume_create(const kf_volume_params* p, void* cuda_stream, kf_volume** out) {
  if (!p || !out) return KF_ERR_INVALID_ARG;
  *out = nullptr;
  if (p->res < 2 || p->res > 1024 || !(p->side > 0.f) || !std::isfinite(p->side) || !(p->mu > 0.f) ||
      !(p->w_max >= 1.f) || !std::isfinite(p->origin[0]) || !std::isfinite(p->origin[1]) ||
      !std::isfinite(p->origin[2]))
    return KF_ERR_INVALID_ARG;
  kf_volume* v = new (std::nothrow) kf_volume();
  if (!v) return KF_ERR_OOM;
  v->p = *p;
  v->g.res = p->res;
  v->g.s = p->side / (float)p->res;
  for (int a = 0; a < 3; ++a) v->g.o[a] = p->origin[a];
  v->g.mu = p->mu;
  v->g.w_max = p->w_max;
  cudaGetDevice(&v->device);
  cudaError_t e = cudaSuccess;
  if (cuda_stream) {
    v->stream = static_cast<cudaStream_t>(cuda_stream);
  } else {
    e = cudaStreamCreateWithFlags(&v->stream, cudaStreamNonBlocking);
    v->own_stream = e == cudaSuccess;
  }
  const size_t n = (size_t)p->res * p->res * p->res;
  v->nb = (p->res + kBrick - 1) / kBrick;
  if (e == cudaSuccess) e = cudaMalloc(&v->F, n * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&v->W, n * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&v->bricks, (size_t)v->nb * v->nb * v->nb * sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&v->brick_count, sizeof(unsigned));
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&v->sms, cudaDevAttrMultiProcessorCount, v->device);
  if (e != cudaSuccess) {
    kf_volume_destroy(v);
    return e == cudaErrorMemoryAllocation ? KF_ERR_OOM : KF_ERR_CUDA;
  }
  const kf_status st = kf_volume_reset(v);
  if (st != KF_OK) {
    kf_volume_destroy(v);
    return st;
  }
  *out = v;
  return KF_OK;
}

void kf_volume_destroy(kf_volume* v) {
  if (!v) return;
  if (v->stream) cudaStreamSynchronize(v->stream);
  cudaFree(v->F);
  cudaFree(v->W);
  cudaFree(v->bricks);
  cudaFree(v->brick_count);
  cudaFree(v->depth);
  cudaFree(v->maps);
  if (v->own_stream) cudaStreamDestroy(v->stream);
  delete v;
}

const char* kf_volume_last_error(const kf_volume* v) { return v ? v->err.c_str() : "null volume"; }

kf_status kf_volume_reset(kf_volume* v) {
  if (!v) return KF_ERR_INVALID_ARG;
  const size_t n = (size_t)v->g.res * v->g.res * v->g.res;
  k_reset<<<1216, 256, 0, v->stream>>>(v->F, v->W, n);
  KV_CK(v, cudaGetLastError());
  return KF_OK;
}

kf_status kf_volume_integrate(kf_volume* v, const float* depth, const kf_intrinsics* K,
                              const double pose[16], int is_device_ptr) {
  if (!v || !depth || !cam_ok(K) || !pose_ok(pose)) return vfail(v, KF_ERR_INVALID_ARG, "bad argument");
  const float* D = depth;
  if (!is_device_ptr) {
    const size_t bytes = (size_t)K->width * K->height * sizeof(float);
    kf_status st = grow(v, &v->depth, &v->depth_cap, bytes);
    if (st != KF_OK) return st;
    KV_CK(v, cudaMemcpyAsync(v->depth, depth, bytes, cudaMemcpyHostToDevice, v->stream));
    D = v->depth;
  }
  // rows of [R^T | -R^T t] in double, then rounded to float32
  Xf12 xf;
  for (int a = 0; a < 3; ++a) {
    double tt = 0.0;
    for (int b = 0; b < 3; ++b) {
      xf.r[a * 3 + b] = (float)pose[b * 4 + a];
      tt -= pose[b * 4 + a] * pose[b * 4 + 3];
    }
    xf.t[a] = (float)tt;
  }
  // side planes of the frustum one pixel wider than the image (u in
  // [-1.5, w + 0.5], v likewise); with a non-positive focal length nothing
  // is culled
  Frustum fr;
  memset(&fr, 0, sizeof(fr));
  if (K->fx > 0.0 && K->fy > 0.0) {
    const double nrm[4][3] = {{K->fx, 0.0, K->cx + 1.5},
                              {-K->fx, 0.0, K->width + 0.5 - K->cx},
                              {0.0, K->fy, K->cy + 1.5},
                              {0.0, -K->fy, K->height + 0.5 - K->cy}};
    for (int q = 0; q < 4; ++q) {
      const double l = std::sqrt(nrm[q][0] * nrm[q][0] + nrm[q][1] * nrm[q][1] + nrm[q][2] * nrm[q][2]);
      for (int a = 0; a < 3; ++a) fr.n[q][a] = (float)(nrm[q][a] / l);
    }
  }
  const int nb = v->nb;
  const int nbricks = nb * nb * nb;
  KV_CK(v, cudaMemsetAsync(v->brick_count, 0, sizeof(unsigned), v->stream));
  k_cull_bricks<<<(nbricks + 255) / 256, 256, 0, v->stream>>>(v->g, xf, fr, nb, v->bricks, v->brick_count);
  KV_CK(v, cudaGetLastError());
  k_integrate_bricks<<<v->sms * 4, kBrick * kBrick * kBrick, 0, v->stream>>>(v->F, v->W, v->g, D, cam32(K),
                                                                             xf, nb, v->bricks,
                                                                             v->brick_count);
  KV_CK(v, cudaGetLastError());
  if (!is_device_ptr) KV_CK(v, cudaStreamSynchronize(v->stream));
  return KF_OK;
}

kf_status kf_volume_raycast(kf_volume* v, const kf_intrinsics* K, const double pose[16],
                            float z_near, float z_far, float dz, float* vertex, float* normal,
                            int is_device_ptr) {
  if (!v || !cam_ok(K) || !pose_ok(pose) || !vertex || !normal || !(dz > 0.f) ||
      !(z_far >= z_near) || !std::isfinite(z_near) || !std::isfinite(z_far))
    return vfail(v, KF_ERR_INVALID_ARG, "bad argument");
  const double nsteps = std::floor(((double)z_far - (double)z_near) / (double)dz) + 2.0;
  if (nsteps > 1e6) return vfail(v, KF_ERR_INVALID_ARG, "more than 1e6 samples per ray");
  RayParams rp;
  for (int a = 0; a < 3; ++a) {
    for (int b = 0; b < 3; ++b) rp.R[a * 3 + b] = (float)pose[a * 4 + b];
    rp.c[a] = (float)pose[a * 4 + 3];
  }
  rp.zn = z_near;
  rp.zf = z_far;
  rp.dz = dz;
  rp.steps = (int)nsteps;  // the kernel also stops once z_k > z_far
  const size_t px = (size_t)K->width * K->height;
  float* Vd = vertex;
  float* Nd = normal;
  if (!is_device_ptr) {
    kf_status st = grow(v, &v->maps, &v->maps_cap, px * 6 * sizeof(float));
    if (st != KF_OK) return st;
    Vd = v->maps;
    Nd = v->maps + px * 3;
  }
  const dim3 grid((K->width + 127) / 128, K->height);
  k_raycast<<<grid, 128, 0, v->stream>>>(v->F, v->W, v->g, cam32(K), rp, Vd, Nd);
  KV_CK(v, cudaGetLastError());
  if (!is_device_ptr) {
    KV_CK(v, cudaMemcpyAsync(vertex, Vd, px * 3 * sizeof(float), cudaMemcpyDeviceToHost, v->stream));
    KV_CK(v, cudaMemcpyAsync(normal, Nd, px * 3 * sizeof(float), cudaMemcpyDeviceToHost, v->stream));
    KV_CK(v, cudaStreamSynchronize(v->stream));
  }
  return KF_OK;
}

kf_status kf_volume_read(kf_volume* v, float* F, float* W) {
  if (!v) return KF_ERR_INVALID_ARG;
  const size_t n = (size_t)v->g.res * v->g.res * v->g.res;
  KV_CK(v, cudaStreamSynchronize(v->stream));
  if (F) KV_CK(v, cudaMemcpy(F, v->F, n * sizeof(float), cudaMemcpyDeviceToHost));
  if (W) KV_CK(v, cudaMemcpy(W, v->W, n * sizeof(float), cudaMemcpyDeviceToHost));
  return KF_OK;
}

}  // extern "C"
