// ICP hot path: projective association + distance histogram (Sec. 3.2),
// median from the CDF and the inlier band (Sec. 3.3), filtered point-to-plane
// normal-equation reduction (Eq. 3), the regularised FP64 solve (Eq. 4, 5),
// the pose update and the median-driven convergence control (Sec. 3.4).
//
// Work is split into items of consecutive frame pixels of one pair at one
// level. An iteration of a pair is two stages over its items. The association
// pass reads each frame vertex and gathers its model vertex and normal once:
// it counts the distance histogram and, knowing where the band edge fell the
// iteration before, sums the rows of the pixels surely inside the band and
// records the rows of the pixels near the edge. The reduction pass then only
// adds the recorded rows that the new band keeps, or, when the edge moved out
// of that window, associates again with the band known. Each stage's per-pair
// epilogue (median and band after the histogram; solve and update after the
// reduction) runs in the pair's last block to finish, found with a per-pair
// arrival counter (no block ever waits for another).
#include "kf_internal.cuh"

// Tuning of the ICP kernels: minimum resident blocks per SM (register cap)
// and frame pixels per thread per batch of the association passes.
#ifndef KF_ASSOC_MINB
#define KF_ASSOC_MINB 2
#endif
#ifndef KF_ASSOC_U
#define KF_ASSOC_U 4
#endif
#ifndef KF_REDUCE_MINB
#define KF_REDUCE_MINB 2
#endif
#ifndef KF_SCHED_MINB
#define KF_SCHED_MINB 2
#endif
// Prefetch during an association batch: 0 none; 1 the warp's frame-vertex
// lines of its next batch into L2; 2 also the model lines its next batch is
// likely to gather (the warp's current match offset applied to the next
// pixels); 3 and 4 as 1 and 2, into L1
#ifndef KF_PREFETCH
#define KF_PREFETCH 1
#endif
// Per-thread sums: 0 plain float32 fused multiply-adds; 1 compensated
// (Kahan) summation, each sum carrying its lost low-order part in a second
// register (a measurement build: twice the sum registers)
#ifndef KF_KAHAN
#define KF_KAHAN 0
#endif
// Scheduled kernel: the pair's median epilogue also runs the reduction pass
// of a hit while the pairs still running number at least the launch's
// blocks / KF_FUSE_GRID_DIV (0: never; a large value: always). Measured at
// 640x480 on 304 blocks: 256 pairs 4.60 ms never, 4.39 ms from 64 pairs on;
// 64 pairs 1.45 ms never, 1.49 ms from 32 on.
#ifndef KF_FUSE_GRID_DIV
#define KF_FUSE_GRID_DIV 4
#endif
namespace kf {

#ifdef KF_CHECKED
__device__ long long g_fault[3];
__device__ void kf_fault(int code, long long a, long long b) {
  if (atomicCAS(reinterpret_cast<unsigned long long*>(&g_fault[0]), 0ull, (unsigned long long)code) == 0ull) {
    g_fault[1] = a;
    g_fault[2] = b;
  }
}
void checked_fault(long long out[3]) {
  cudaMemcpyFromSymbol(out, g_fault, sizeof(long long) * 3);
  const long long z[3] = {0, 0, 0};
  cudaMemcpyToSymbol(g_fault, z, sizeof(z));
}
#else
void checked_fault(long long out[3]) { out[0] = out[1] = out[2] = 0; }
#endif

namespace {

// ---------------------------------------------------------------------------
// float32 decision chain. Every operation is one explicitly rounded IEEE
// operation in a fixed order (a fused multiply-add where fmaf is written, no
// other contraction), so that a float32 re-evaluation elsewhere reproduces
// each decision bit for bit:
//   row(R, t, v) = fma(R2, v.z, fma(R1, v.y, fma(R0, v.x, t)))
// ---------------------------------------------------------------------------
__device__ __forceinline__ float row3(const float* R, float t, float x, float y, float z) {
  return fmaf(R[2], z, fmaf(R[1], y, fmaf(R[0], x, t)));
}

__device__ __forceinline__ float rot3(const float* R, float x, float y, float z) {
  return fmaf(R[2], z, fmaf(R[1], y, fmaf(R[0], x, 0.f)));
}

// Projective association (Sec. 3.2), split in two phases so that a thread
// can issue the model gathers of several pixels before using any of them.
//
// project(): frame vertex v -> model pixel index j (or -1) and world point p.
//   model-camera point m = T_rel v; reject unless m.z > 0;
//   (u, v)^ = rint(fma(f m.xy, 1 / m.z, c)), round half to even; reject
//   outside the image.
// bin_of(): with the gathered model vertex q, d = |p - q| (point-to-point);
//   reject unless d < d_max (NaN model holes fail too); bin = floor(d B / d_max).
// xf: Rw[9] tw[3] (camera -> world) Rr[9] tr[3] (camera -> model camera).
__device__ __forceinline__ int project(const LevelMaps& L, float vx, float vy, float vz,
                                       const float* xf, float* p) {
  const float mx = row3(xf + 12, xf[21], vx, vy, vz);
  const float my = row3(xf + 15, xf[22], vx, vy, vz);
  const float mz = row3(xf + 18, xf[23], vx, vy, vz);
  p[0] = row3(xf + 0, xf[9], vx, vy, vz);
  p[1] = row3(xf + 3, xf[10], vx, vy, vz);
  p[2] = row3(xf + 6, xf[11], vx, vy, vz);
  if (!(mz > 0.f)) return -1;  // also rejects invalid (NaN) frame vertices
  const float rz = __frcp_rn(mz);  // 1 / m.z, rounded once
  const float uf = fmaf(__fmul_rn(L.mfx, mx), rz, L.mcx);
  const float vf = fmaf(__fmul_rn(L.mfy, my), rz, L.mcy);
  const float ur = rintf(uf), vr = rintf(vf);
  if (!(ur >= 0.f && ur <= (float)(L.mw - 1) && vr >= 0.f && vr <= (float)(L.mh - 1))) return -1;
  return (int)vr * L.mw + (int)ur;
}

__device__ __forceinline__ int bin_of(const float* p, const float* q, const KParams& P) {
  const float dx = __fsub_rn(p[0], q[0]);
  const float dy = __fsub_rn(p[1], q[1]);
  const float dz = __fsub_rn(p[2], q[2]);
  const float d2 = fmaf(dz, dz, fmaf(dy, dy, __fmul_rn(dx, dx)));
  const float d = __fsqrt_rn(d2);
  if (!(d < P.d_max32)) return -1;
  const int k = (int)floorf(__fmul_rn(d, P.scale32));
  return k < P.bins - 1 ? k : P.bins - 1;
}

// Optional normal-angle gate: (R_cur n_frame) . n_model >= cos_min, float32.
__device__ __forceinline__ bool angle_ok(const float* xf, const float* nf, const float* nq,
                                         const KParams& P) {
  const float wx = rot3(xf + 0, nf[0], nf[1], nf[2]);
  const float wy = rot3(xf + 3, nf[0], nf[1], nf[2]);
  const float wz = rot3(xf + 6, nf[0], nf[1], nf[2]);
  float dot = __fadd_rn(__fmul_rn(wx, nq[0]), __fmul_rn(wy, nq[1]));
  dot = __fadd_rn(dot, __fmul_rn(wz, nq[2]));
  return dot >= P.cos_min32;
}

// Association variants (template bits): kAGate = the normal-angle gate,
// kAShoot = normal shooting instead of the projected pixel.
constexpr int kAGate = 1, kAShoot = 2;

// Normal shooting (Sec. 3.3): among the valid model pixels of the
// (2w+1)^2 window around the projected pixel jc, the one whose vertex q lies
// closest to the line through the world point p along the world frame normal
// n. Squared distance to the line, float32, each operation rounded in this
// order: e = q - p; s = (e.x n.x + e.y n.y) + e.z n.z;
// l2 = ((e.x^2 + e.y^2) + e.z^2) - s s. Candidates row by row, a strictly
// smaller l2 replaces the best (ties keep the first). Holes (NaN vertex)
// are skipped. Returns the chosen pixel (or -1) and its vertex in q.
template <class T>
__device__ __forceinline__ int shoot(const LevelMaps& L, const T* mV, int jc, const float* p,
                                     const float* n, int w, float* q) {
  constexpr int kRow = 9;  // 2 w + 1 for the largest window (w = 4)
  const int mn = L.mw * L.mh;
  const int cu = jc % L.mw, cv = jc / L.mw;
  const float nan = __int_as_float(0x7fc00000);
  float best = __int_as_float(0x7f800000);
  int bj = -1;
  for (int dy = -w; dy <= w; ++dy) {
    const int y = cv + dy;
    if (y < 0 || y >= L.mh) continue;
    // one row of candidates loaded together, then compared in order
    float cx[kRow], cy[kRow], cz[kRow];
#pragma unroll
    for (int k = 0; k < kRow; ++k) {
      const int x = cu - w + k;
      const bool in = k <= 2 * w && x >= 0 && x < L.mw;
      const int j = y * L.mw + (in ? x : cu);
      cx[k] = in ? Store<T>::ld(mV, j) : nan;
      cy[k] = in ? Store<T>::ld(mV, mn + j) : nan;
      cz[k] = in ? Store<T>::ld(mV, 2 * mn + j) : nan;
    }
#pragma unroll
    for (int k = 0; k < kRow; ++k) {
      if (isnan(cx[k])) continue;  // outside the window or the image, or a hole
      const float ex = __fsub_rn(cx[k], p[0]), ey = __fsub_rn(cy[k], p[1]), ez = __fsub_rn(cz[k], p[2]);
      float sd = __fadd_rn(__fmul_rn(ex, n[0]), __fmul_rn(ey, n[1]));
      sd = __fadd_rn(sd, __fmul_rn(ez, n[2]));
      float ee = __fadd_rn(__fmul_rn(ex, ex), __fmul_rn(ey, ey));
      ee = __fadd_rn(ee, __fmul_rn(ez, ez));
      const float l2 = __fsub_rn(ee, __fmul_rn(sd, sd));
      if (l2 < best) {
        best = l2;
        bj = y * L.mw + cu - w + k;
        q[0] = cx[k];
        q[1] = cy[k];
        q[2] = cz[k];
      }
    }
  }
  return bj;
}

// Entry o (0..23) of the float32 transforms: Rw[9] tw[3] are T_cur rounded to
// float32; Rr[9] tr[3] are the FP64 relative transform T_m^-1 T_cur, summed
// in the order k = 0, 1, 2 with explicitly rounded operations, then rounded.
__device__ __forceinline__ float xf_entry(const double* T, const double* Tm, int o) {
  if (o < 9) return __double2float_rn(T[(o / 3) * 4 + o % 3]);
  if (o < 12) return __double2float_rn(T[(o - 9) * 4 + 3]);
  if (o < 21) {
    const int i = (o - 12) / 3, j = (o - 12) % 3;
    double s = __dmul_rn(Tm[0 * 4 + i], T[0 * 4 + j]);
    s = __dadd_rn(s, __dmul_rn(Tm[1 * 4 + i], T[1 * 4 + j]));
    s = __dadd_rn(s, __dmul_rn(Tm[2 * 4 + i], T[2 * 4 + j]));
    return __double2float_rn(s);
  }
  const int i = o - 21;
  const double d0 = __dsub_rn(T[3], Tm[3]), d1 = __dsub_rn(T[7], Tm[7]), d2 = __dsub_rn(T[11], Tm[11]);
  double s = __dmul_rn(Tm[0 * 4 + i], d0);
  s = __dadd_rn(s, __dmul_rn(Tm[1 * 4 + i], d1));
  s = __dadd_rn(s, __dmul_rn(Tm[2 * 4 + i], d2));
  return __double2float_rn(s);
}

__device__ void compute_xf(const double* T, const double* Tm, float* xf) {
  for (int o = 0; o < 24; ++o) xf[o] = xf_entry(T, Tm, o);
}

// Median bin k_med = min{k : 2 C(k) >= N} from the pair's histogram and the
// band of bins around it (Sec. 3.3). Block-wide; the caller is the pair's last
// block of the histogram stage. Returns (in thread 0) 1 when the pair stops
// here (fewer than n_min valid pairs), else 0.
__device__ __noinline__ int median_and_band(const PairDesc* d, PairState* st, const KParams& P) {
  __shared__ unsigned s_wsum[kBlockWarps];
  __shared__ int s_kmed;
  const int B = P.bins;
  const int per = (B + kBlock - 1) / kBlock;
  const int b0 = threadIdx.x * per;
  const int b1 = min(b0 + per, B);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned local = 0;
  for (int b = b0; b < b1; ++b) local += __ldcg(d->hist + b);
  if (threadIdx.x == 0) s_kmed = 0;
  // inclusive scan of the threads' counts: within each warp by shuffles,
  // then over the warps' totals (exact integer sums)
  unsigned incl = local;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) s_wsum[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    unsigned w = lane < kBlockWarps ? s_wsum[lane] : 0u;
#pragma unroll
    for (int o = 1; o < kBlockWarps; o <<= 1) {
      const unsigned y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    if (lane < kBlockWarps) s_wsum[lane] = w;
  }
  __syncthreads();
  if (warp > 0) incl += s_wsum[warp - 1];
  const unsigned N = s_wsum[kBlockWarps - 1];
  const unsigned before = incl - local;
  if (N > 0 && 2ull * incl >= N && 2ull * before < N) {
    unsigned c = before;
    for (int b = b0; b < b1; ++b) {
      c += __ldcg(d->hist + b);
      if (2ull * c >= N) {
        s_kmed = b;
        break;
      }
    }
  }
  __syncthreads();
  int stop = 0;
  if (threadIdx.x == 0) {
    const int kmed = s_kmed;
    st->N = (int)N;
    st->kmed = kmed;
    if ((int)N < P.n_min) {
      st->status = KF_ERR_TOO_FEW_INLIERS;
      st->stopped = 1;
      stop = 1;
    }
    int klo = 0, khi = B - 1;
    if (P.flags & KF_USE_FILTER) {
      const double m = (double)kmed + 0.5;
      khi = (int)floor(__dmul_rn(__dadd_rn(1.0, P.kappa), m));
      klo = (int)ceil(__dmul_rn(__dsub_rn(1.0, P.kappa), m)) - 1;
      khi = khi < B - 1 ? khi : B - 1;
      klo = klo > 0 ? klo : 0;
    }
    st->klo = klo;
    st->khi = khi;
    // the association pass summed bins < w0 and recorded bins [w0, w1): the
    // band [0, khi] is complete from those when khi lies in [w0 - 1, w1 - 1]
    const int w0 = __ldcg(&st->w0), w1 = __ldcg(&st->w1);
    st->hit = (w0 >= 0 && klo == 0 && khi >= w0 - 1 && khi <= w1 - 1) ? 1 : 0;
  }
  return stop;
}

__device__ double lambda_of_n(int mode, double c, int n) {
  const double dn = (double)n;
  switch (mode) {
    case KF_LAMBDA_C_SQRT_N: return c / sqrt(dn);
    case KF_LAMBDA_C_N: return c / dn;
    case KF_LAMBDA_C_N2: return c / (dn * dn);
    case KF_LAMBDA_C_LOG_N: return c * log(dn);
    default: return c;
  }
}

__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

// The pair's state the solve reads, loaded by one thread at the start of the
// epilogue (every load in flight at once, before the partials are combined)
// instead of one after another at the end of the solve. The state was last
// written by other blocks (the histogram epilogue, earlier solves): every
// read goes through L2.
struct PairPre {
  double lambda_c;
  int kmed, N, klo, khi, w0, w1, it, tl, total, hl, status, has_prior;
  int kh[kMaxWindow];
};

__device__ __forceinline__ PairPre load_pre(const PairState* st, int level) {
  PairPre q;
  q.lambda_c = __ldcg(&st->lambda_c);
  q.kmed = __ldcg(&st->kmed);
  q.N = __ldcg(&st->N);
  q.klo = __ldcg(&st->klo);
  q.khi = __ldcg(&st->khi);
  q.w0 = __ldcg(&st->w0);
  q.w1 = __ldcg(&st->w1);
  q.it = __ldcg(&st->iters[level]);
  q.tl = __ldcg(&st->trace_len);
  q.total = __ldcg(&st->total_iters);
  q.hl = __ldcg(&st->hist_len);
  q.status = __ldcg(&st->status);
  q.has_prior = __ldcg(&st->has_prior);
#pragma unroll
  for (int i = 0; i < kMaxWindow; ++i) q.kh[i] = __ldcg(&st->kmed_hist[i]);
  return q;
}

// Eq. 5: (A^T A + 2 lambda n P^T P) x = A^T b, P = [I3 | 0]; Cholesky solve;
// T <- [Exp(alpha, beta, gamma) | t] T; convergence control (Sec. 3.4).
// FP64, run by one warp (the FP64 units are narrow on this part, so the
// dependent chain, not the operation count, sets the time): a right-looking
// Cholesky with one reciprocal square root per column and the trailing update
// spread over lanes, substitutions by multiplication with the pivots'
// inverses, and the pose composition and float32 transforms one entry per lane.
// sm: >= 96 doubles of shared memory. Returns (in lane 0) the level the pair
// iterates at next, or -1 when it has finished or stopped.
// pre: the pair's state from load_pre, valid in lane 0.
__device__ __noinline__ int solve_update_warp(const PairDesc* d, PairState* st, const double* S,
                                               int level, const KParams& P, double* sm, int passes,
                                               const PairPre& pre) {
  const int lane = threadIdx.x & 31;
  const unsigned long long t_start = globaltimer_ns();
  double* H = sm;           // 36: H
  double* g = sm + 42;      // 6: A^T b, then the increment x
  double* Tn = sm + 54;     // 12: new pose
  double* dR = sm + 66;     // 9
  double* misc = sm + 75;   // [0] lambda [1] A [2] B
  const int n = (int)S[27];
  if (n < P.n_min) {
    if (lane == 0) {
      st->status = KF_ERR_TOO_FEW_INLIERS;
      st->stopped = 1;
    }
    return -1;
  }
  if (lane == 0) misc[0] = lambda_of_n(P.lambda_mode, pre.lambda_c, n);
  __syncwarp();
  const double reg = (2.0 * misc[0]) * (double)n;
  if (lane < 21) {  // upper-triangle sum `lane` -> (r, c)
    int r = 0, k = lane;
    while (k >= 6 - r) {
      k -= 6 - r;
      ++r;
    }
    const int c = r + k;
    const double v = S[lane] + ((r == c && r < 3) ? reg : 0.0);
    H[r * 6 + c] = v;
    H[c * 6 + r] = v;
  }
  if (lane < 6) g[lane] = S[21 + lane];
  __syncwarp();
  if ((P.flags & KF_PRIOR_ANCHORED) && __shfl_sync(0xffffffffu, pre.has_prior, 0)) {
    // prior-anchored variant: g_rot -= 2 lambda n r, r = log(R R_prior^T):
    // M = R R_prior^T one entry per lane, then t = atan2(|v| / 2, (tr M - 1) / 2)
    // and r = t / (2 sin t) v, v = (M21 - M12, M02 - M20, M10 - M01)
    double* M = sm + 54;  // the new-pose scratch, free until the update
    if (lane < 9) {
      const int i = lane / 3, j = lane % 3;
      double m = 0.0;
      for (int k = 0; k < 3; ++k) m += __ldcg(&st->T[i * 4 + k]) * __ldcg(&st->prior_R[j * 3 + k]);
      M[lane] = m;
    }
    __syncwarp();
    if (lane == 0) {
      const double v0 = M[7] - M[5], v1 = M[2] - M[6], v2 = M[3] - M[1];
      const double sn = 0.5 * sqrt(v0 * v0 + v1 * v1 + v2 * v2);
      const double cs = 0.5 * (M[0] + M[4] + M[8] - 1.0);
      const double t = atan2(sn, cs);
      const double f = t < 1e-4 ? 0.5 * (1.0 + t * t / 6.0) : t / (2.0 * sn);
      g[0] -= reg * f * v0;
      g[1] -= reg * f * v1;
      g[2] -= reg * f * v2;
    }
    __syncwarp();
  }
  // Cholesky factorisation H = L L^T and the two triangular solves, by one
  // thread in registers (the loops unroll to fixed indices): a chain of
  // dependent FP64 operations costs ~64 cycles each here, and one thread
  // avoids a warp barrier and a shared-memory round trip per step. A pivot
  // not above 1e-12 of its own diagonal entry of H is degenerate.
  int degenerate = 0;
  if (lane == 0) {
    double Lm[6][6], x[6];
#pragma unroll
    for (int i = 0; i < 6; ++i)
#pragma unroll
      for (int c = 0; c <= i; ++c) Lm[i][c] = H[i * 6 + c];
#pragma unroll
    for (int i = 0; i < 6; ++i) x[i] = g[i];
    double r[6];
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      double a = Lm[j][j];
#pragma unroll
      for (int c = 0; c < j; ++c) a -= Lm[j][c] * Lm[j][c];
      if (!(a > 1e-12 * H[j * 7])) degenerate = 1;
      r[j] = rsqrt(a);
      Lm[j][j] = a * r[j];
#pragma unroll
      for (int i = j + 1; i < 6; ++i) {
        double v = Lm[i][j];
#pragma unroll
        for (int c = 0; c < j; ++c) v -= Lm[i][c] * Lm[j][c];
        Lm[i][j] = v * r[j];
      }
    }
#pragma unroll
    for (int k = 0; k < 6; ++k) {  // L y = g
      double v = x[k];
#pragma unroll
      for (int c = 0; c < k; ++c) v -= Lm[k][c] * x[c];
      x[k] = v * r[k];
    }
#pragma unroll
    for (int k = 5; k >= 0; --k) {  // L^T x = y
      double v = x[k];
#pragma unroll
      for (int c = k + 1; c < 6; ++c) v -= Lm[c][k] * x[c];
      x[k] = v * r[k];
    }
#pragma unroll
    for (int i = 0; i < 6; ++i) g[i] = x[i];
  }
  degenerate = __shfl_sync(0xffffffffu, degenerate, 0);
  if (degenerate) {
    if (lane == 0) {
      st->status = KF_ERR_DEGENERATE;
      st->stopped = 1;
    }
    return -1;
  }
  __syncwarp();
  // Rodrigues: dR = I + A [w]x + B [w]x^2, A = sin(t)/t, B = (1 - cos t)/t^2;
  // below t = 0.2 both from their Taylor series (truncation < 3e-15)
  if (lane == 0) {
    const double th2 = g[0] * g[0] + g[1] * g[1] + g[2] * g[2];
    if (th2 < 0.04) {
      // multiplications by the coefficients' reciprocals (an FP64 division
      // costs ~380 cycles here; the series is far from needing exact ones)
      misc[1] = 1.0 - th2 * (1.0 / 6.0) * (1.0 - th2 * (1.0 / 20.0) * (1.0 - th2 * (1.0 / 42.0) * (1.0 - th2 * (1.0 / 72.0))));
      misc[2] = 0.5 * (1.0 - th2 * (1.0 / 12.0) * (1.0 - th2 * (1.0 / 30.0) * (1.0 - th2 * (1.0 / 56.0) * (1.0 - th2 * (1.0 / 90.0)))));
    } else {
      const double th = sqrt(th2);
      double sn, cs;
      sincos(th, &sn, &cs);
      misc[1] = sn / th;
      misc[2] = (1.0 - cs) / th2;
    }
  }
  __syncwarp();
  if (lane < 9) {
    const int i = lane / 3, j = lane % 3;
    const double K[9] = {0.0, -g[2], g[1], g[2], 0.0, -g[0], -g[1], g[0], 0.0};
    double k2 = 0.0;
    for (int k = 0; k < 3; ++k) k2 += K[i * 3 + k] * K[k * 3 + j];
    dR[lane] = (i == j ? 1.0 : 0.0) + misc[1] * K[lane] + misc[2] * k2;
  }
  __syncwarp();
  if (lane < 12) {
    const int i = lane / 4, j = lane % 4;
    double v = 0.0;
    for (int k = 0; k < 3; ++k) v += dR[i * 3 + k] * __ldcg(&st->T[k * 4 + j]);
    if (j == 3) v += g[3 + i];
    Tn[lane] = v;
  }
  __syncwarp();
  if (lane < 12) st->T[lane] = Tn[lane];
  if (lane < 24) st->xf[lane] = xf_entry(Tn, d->Tm, lane);
  if (lane == 1) st->rms = sqrt(S[28] / (double)n);
  if (lane != 0) return -1;
  // bookkeeping (the state's fields from pre)
  const int kmed = pre.kmed, N = pre.N, it = pre.it, tl = pre.tl;
  if (tl < KF_TRACE_MAX) {
    kf_iter_record& r = st->trace[tl];
    st->trace_len = tl + 1;
    r.level = level;
    r.iter = it;
    r.N = N;
    r.kmed = kmed;
    r.klo = pre.klo;
    r.khi = pre.khi;
    r.n = n;
    r.passes = passes;
    r.w0 = pre.w0;
    r.w1 = pre.w1;
    r.pad = 0;
    r.lambda = misc[0];
    for (int i = 0; i < 6; ++i) r.x[i] = g[i];
    r.solve_ns = (int)(globaltimer_ns() - t_start);
  }
  st->iters[level] = it + 1;
  st->total_iters = pre.total + 1;
  st->median_bin[level] = kmed;
  st->valid_pairs = N;
  st->inliers = n;
  int hl = pre.hl;
  int kh[kMaxWindow];
  for (int i = 0; i < kMaxWindow; ++i) kh[i] = pre.kh[i];
  if (hl < kMaxWindow) {
    kh[hl++] = kmed;
  } else {
    for (int i = 0; i + 1 < kMaxWindow; ++i) kh[i] = kh[i + 1];
    kh[kMaxWindow - 1] = kmed;
  }
  bool conv = false;
  if ((P.flags & KF_USE_CONVERGENCE) && hl >= P.conv_window) {
    conv = true;
    for (int i = hl - P.conv_window; i < hl; ++i) conv = conv && kh[i] == kmed;
  }
  int cur = level;
  if (conv || it + 1 >= P.caps[level]) {
    if (level == 0 && (P.flags & KF_USE_CONVERGENCE) && !conv && pre.status == KF_OK)
      st->status = KF_NOT_CONVERGED;
    cur = level - 1;
    hl = 0;
  }
  st->cur_level = cur;
  st->hist_len = hl;
  for (int i = 0; i < kMaxWindow; ++i) st->kmed_hist[i] = kh[i];
  // the next iteration's band-edge window around this band edge
  int w0 = -1, w1 = -1;
  if (P.split_ok && cur >= 0) {
    const int below = cur == level ? P.win_same_below : P.win_next_below;
    const int above = cur == level ? P.win_same_above : P.win_next_above;
    w0 = max(0, pre.khi - below + 1);
    w1 = pre.khi + above + 1;
  }
  st->w0 = w0;
  st->w1 = w1;
  return cur;
}

// ---------------------------------------------------------------------------
// Active work list (see kf_internal.cuh for the layout).
// ---------------------------------------------------------------------------
__device__ __forceinline__ int items_of(const PairDesc* d, int level) {
  const int px = d->lv[level].fw * d->lv[level].fh;
  const int c = level_chunk(level);
  return (px + c - 1) / c;
}

// Block-wide exclusive scan of one int per thread (kBlock threads); returns the
// exclusive prefix and writes the block total to *total.
__device__ int block_exclusive_scan(int v, int* total) {
  __shared__ int s_buf[kBlock];
  s_buf[threadIdx.x] = v;
  __syncthreads();
  for (int off = 1; off < kBlock; off <<= 1) {
    const int t = threadIdx.x >= off ? s_buf[threadIdx.x - off] : 0;
    __syncthreads();
    s_buf[threadIdx.x] += t;
    __syncthreads();
  }
  const int incl = s_buf[threadIdx.x];
  *total = s_buf[kBlock - 1];
  __syncthreads();
  return incl - v;
}

// Build the list of pairs still iterating at `level` and their items. One
// block of kBlock threads; every pair's state must be final when it runs.
__device__ void build_active_list(const PairDesc* const* descs, int n, int level, int* list, int cap) {
  int* pairs = list + 4;
  int* prefix = list + 4 + cap;
  int npairs = 0, nitems = 0;
  for (int base = 0; base < n; base += kBlock) {
    const int p = base + threadIdx.x;
    int cnt = 0;
    if (p < n && level >= 0) {
      // other blocks of this launch wrote these fields: read them from L2
      const PairState* st = descs[p]->st;
      if (__ldcg(&st->cur_level) == level && !__ldcg(&st->stopped))
        cnt = items_of(descs[p], level);
    }
    int tot_flags, tot_items;
    const int slot = block_exclusive_scan(cnt > 0 ? 1 : 0, &tot_flags);
    const int off = block_exclusive_scan(cnt, &tot_items);
    if (cnt > 0) {
      KF_GUARD(npairs + slot < cap, 8, npairs + slot, cap) {
        pairs[npairs + slot] = p;
        prefix[npairs + slot] = nitems + off;
      }
    }
    npairs += tot_flags;
    nitems += tot_items;
  }
  if (threadIdx.x == 0) {
    KF_GUARD(npairs <= cap, 9, npairs, cap)
    prefix[npairs] = nitems;
    list[0] = nitems;
    list[1] = npairs;
    list[2] = level;
  }
  __syncthreads();
}

// Entry s with prefix[s] <= f < prefix[s+1] (binary search).
__device__ __forceinline__ int find_slot(const int* prefix, int npairs, int f) {
  int lo = 0, hi = npairs - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldcg(prefix + mid) <= f) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// Row of Eq. 3 for the pair (p, q, n): a = [(p x n)^T, n^T], b = n . (q - p),
// accumulated into the 29 sums (21 upper a a^T, 6 a b, n, b^2). Every
// operation is written out (products and fused multiply-adds explicitly), so
// that each kernel that inlines it rounds the same way.
__device__ __forceinline__ void ls_row(const float* p, const float* q, const float* n, float* a,
                                       float& b) {
  a[0] = fmaf(p[1], n[2], -__fmul_rn(p[2], n[1]));
  a[1] = fmaf(p[2], n[0], -__fmul_rn(p[0], n[2]));
  a[2] = fmaf(p[0], n[1], -__fmul_rn(p[1], n[0]));
  a[3] = n[0];
  a[4] = n[1];
  a[5] = n[2];
  b = fmaf(n[0], __fsub_rn(q[0], p[0]),
           fmaf(n[1], __fsub_rn(q[1], p[1]), __fmul_rn(n[2], __fsub_rn(q[2], p[2]))));
}

// Registers of a thread's running sums: the 29 sums, and with KF_KAHAN their
// 29 compensations after them.
constexpr int kSumRegs = KF_KAHAN ? 2 * kSums : kSums;

// Sum k += x y. Plain: one fused multiply-add. KF_KAHAN: compensated
// summation (Kahan, 1965); sum[kSums + k] holds c, the rounding error of the
// last addition, which the next term has subtracted before it is added
// (x y - c in one fused rounding); the sum's value is then sum[k] - c.
__device__ __forceinline__ void add_term(float* sum, int k, float x, float y) {
#if KF_KAHAN
  const float t = fmaf(x, y, -sum[kSums + k]);
  const float s = __fadd_rn(sum[k], t);
  sum[kSums + k] = __fsub_rn(__fsub_rn(s, sum[k]), t);
  sum[k] = s;
#else
  sum[k] = fmaf(x, y, sum[k]);
#endif
}

__device__ __forceinline__ void accumulate(const float* a, float b, float* sum) {
  int s = 0;
#pragma unroll
  for (int r = 0; r < 6; ++r)
#pragma unroll
    for (int c = r; c < 6; ++c) {
      add_term(sum, s, a[r], a[c]);
      ++s;
    }
#pragma unroll
  for (int r = 0; r < 6; ++r) add_term(sum, 21 + r, a[r], b);
  sum[27] = __fadd_rn(sum[27], 1.f);  // a count: exact below 2^24
  add_term(sum, 28, b, b);
}

constexpr int kPassHist = 0, kPassSplit = 1, kPassBand = 2;

// ---------------------------------------------------------------------------
// Association passes. A batch is kBatch = KF_ASSOC_U * kBlock consecutive
// frame pixels of one item; thread t takes pixels b0 + t + u kBlock
// (u < KF_ASSOC_U): its frame vertices (coalesced loads), their projections,
// then every model gather of the batch issued before any is used. Warps run
// their batches independently (no barrier inside an item). Measured on GB300
// at 640x480: four pixels per thread and no software pipeline across
// batches beat one or two pixels per thread with the next batch's gathers in
// flight (the pipeline's second batch of registers costs the pixels in flight
// that hide the gathers), and beat staging the frame vertices in shared
// memory with bulk copies (a block barrier per batch).
// ---------------------------------------------------------------------------
constexpr int kU = KF_ASSOC_U;
constexpr int kBatch = kU * kBlock;

// The 24 float32 transform entries, read from shared memory once per batch
// (volatile: the loads stay inside the batch, so the registers holding them
// are free again while the gathers are awaited and the sums accumulate).
// sxf must be a shared-memory array aligned to 16 bytes (vector loads).
__device__ __forceinline__ void load_xf(const float* sxf, float* x) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(sxf);
#pragma unroll
  for (int c = 0; c < 6; ++c)
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(x[4 * c]), "=f"(x[4 * c + 1]), "=f"(x[4 * c + 2]), "=f"(x[4 * c + 3])
                 : "r"(a + 16 * c));
}

struct Verts {  // one batch's frame vertices (NaN past the batch's end)
  float v[kU][3];
};

template <bool kGate>
struct Batch {  // one batch after association, its gathers in flight
  float p[kU][3], q[kU][3], nq[kU][3];
  float nf[kGate ? kU : 1][3];  // frame normals (angle gate)
  int j[kU];
};

__device__ __forceinline__ void prefetch_l2(const void* p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}
__device__ __forceinline__ void prefetch_l1(const void* p) {
  asm volatile("prefetch.global.L1 [%0];" ::"l"(p));
}
__device__ __forceinline__ void prefetch_line(const void* p) {
  if constexpr (KF_PREFETCH >= 3) prefetch_l1(p);
  else prefetch_l2(p);
}

// Hints for the warp's next batch [nb0, ne): its frame-vertex lines (lanes
// 0..3 u: one line of 32 pixels per plane each) and, with an offset `off`
// (model index minus frame index of a pixel this warp just matched), the
// model vertex and normal lines at that offset. Every address stays inside
// its plane.
template <class T>
__device__ __forceinline__ void prefetch_next(const LevelMaps& L, int nb0, int ne, int off) {
  if constexpr (KF_PREFETCH == 0) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int kLines = 3 * kU * (KF_PREFETCH == 2 || KF_PREFETCH == 4 ? 3 : 1);
  for (int q = lane; q < kLines; q += 32) {
    const int set = q / (3 * kU);  // 0: frame vertex, 1: model vertex, 2: model normal
    const int r = q - set * 3 * kU, c = r / kU, u = r - c * kU;
    const int i = nb0 + warp * 32 + u * kBlock;
    if (i >= ne) continue;
    if (set == 0) {
      prefetch_line(static_cast<const T*>(L.fV) + (size_t)c * L.fps + i);
    } else {
      const int mn = L.mw * L.mh;
      const int j = min(max(i + off, 0), mn - 1);
      prefetch_line(static_cast<const T*>(set == 1 ? L.mV : L.mN) + (size_t)c * mn + j);
    }
  }
}

template <class T>
__device__ __forceinline__ void load_verts(const LevelMaps& L, int b0, int e, Verts& V) {
  const T* fV = static_cast<const T*>(L.fV);
  const int fs = L.fps;
#pragma unroll
  for (int u = 0; u < kU; ++u) {
    const int i = b0 + threadIdx.x + u * kBlock;
    const bool in = i < e;
    const int ii = in ? i : 0;
    const float x = Store<T>::ld(fV, ii), y = Store<T>::ld(fV, fs + ii), z = Store<T>::ld(fV, 2 * fs + ii);
    V.v[u][0] = in ? x : __int_as_float(0x7fc00000);
    V.v[u][1] = y;
    V.v[u][2] = z;
  }
}

// Projective association (Sec. 3.2; normal shooting with kAShoot) of a batch:
// world points, matched model pixels, and the gathers of their model vertex
// (and normal, when the pass or the gate needs it) issued.
template <class T, int kA, int kPass>
__device__ __forceinline__ void associate_batch(const LevelMaps& L, int b0, const Verts& V,
                                                const float* sxf, const KParams& P,
                                                Batch<(kA & kAGate) != 0>& B) {
  constexpr bool kGate = (kA & kAGate) != 0;
  constexpr bool kNeedN = kGate || kPass != kPassHist;
  const int fs = L.fps, mn = L.mw * L.mh;
  const T* mV = static_cast<const T*>(L.mV);
  const T* mN = static_cast<const T*>(L.mN);
  float xf[24];
  load_xf(sxf, xf);
#pragma unroll
  for (int u = 0; u < kU; ++u) B.j[u] = project(L, V.v[u][0], V.v[u][1], V.v[u][2], xf, B.p[u]);
  if constexpr (kGate || (kA & kAShoot) != 0) {
    const T* fN = static_cast<const T*>(L.fN);
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int i = B.j[u] >= 0 ? b0 + threadIdx.x + u * kBlock : 0;
      const float nf[3] = {Store<T>::ld(fN, i), Store<T>::ld(fN, fs + i), Store<T>::ld(fN, 2 * fs + i)};
      if constexpr (kGate) {
        B.nf[u][0] = nf[0];
        B.nf[u][1] = nf[1];
        B.nf[u][2] = nf[2];
      }
      if constexpr ((kA & kAShoot) != 0) {
        if (B.j[u] >= 0) {
          const float nw[3] = {rot3(xf + 0, nf[0], nf[1], nf[2]), rot3(xf + 3, nf[0], nf[1], nf[2]),
                               rot3(xf + 6, nf[0], nf[1], nf[2])};
          B.j[u] = shoot(L, mV, B.j[u], B.p[u], nw, P.shoot_w, B.q[u]);
        }
      }
    }
  }
#pragma unroll
  for (int u = 0; u < kU; ++u) {
    const int jj = B.j[u] < 0 ? 0 : B.j[u];
    if constexpr ((kA & kAShoot) == 0) {
      B.q[u][0] = Store<T>::ld(mV, jj);
      B.q[u][1] = Store<T>::ld(mV, mn + jj);
      B.q[u][2] = Store<T>::ld(mV, 2 * mn + jj);
    }
    if constexpr (kNeedN) {
      B.nq[u][0] = Store<T>::ld(mN, jj);
      B.nq[u][1] = Store<T>::ld(mN, mn + jj);
      B.nq[u][2] = Store<T>::ld(mN, 2 * mn + jj);
    }
  }
}

// What an association pass does with a batch once its gathers have landed:
// the point-to-point distance, bin and gates, then
//  kPassHist   the distance histogram only (no band-edge window is known);
//  kPassSplit  the histogram, and the rows of the pixels with bin < lo (= w0)
//              summed in registers, the rows of the pixels with bin in
//              [lo, hi) (= [w0, w1)) written as 32-byte records, packed in
//              the warp's record region of the item (rbase; wc counts the
//              records the warp has written there, in pixel order);
//  kPassBand   no histogram: the rows of the pixels with bin in [lo, hi]
//              (= the band [klo, khi]) summed in registers.
// kMode 1 also writes the inspection outputs (model pixel and bin per pixel).
template <int kA, int kPass, int kMode>
__device__ __forceinline__ void finish_batch(const PairDesc* d, int b0, int e,
                                             const Batch<(kA & kAGate) != 0>& B, const float* sxf,
                                             const KParams& P, unsigned* sh_hist, int lo, int hi,
                                             float* sum, int rbase, int& wc) {
  constexpr bool kGate = (kA & kAGate) != 0;
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int u = 0; u < kU; ++u) {
    const int i = b0 + threadIdx.x + u * kBlock;
    int k = B.j[u] >= 0 ? bin_of(B.p[u], B.q[u], P) : -1;
    if constexpr (kGate) {
      if (k >= 0 && !angle_ok(sxf, B.nf[u], B.nq[u], P)) k = -1;
    }
    if constexpr (kPass != kPassBand) {
      if constexpr (kMode == 1) {
        if (i < e) {
          d->dbg_index[i] = k >= 0 ? B.j[u] : -1;
          d->dbg_bin[i] = k;
        }
      }
      if (k >= 0) atomicAdd(sh_hist + k, 1u);
    }
    if constexpr (kPass == kPassSplit) {
      bool win = false;
      float a[6], b;
      if (k >= 0 && k < hi) {
        ls_row(B.p[u], B.q[u], B.nq[u], a, b);
        if (k < lo) accumulate(a, b, sum);
        else win = true;
      }
      // the window pixels of these 32 lanes take the next places of the
      // warp's region, in lane order
      const unsigned m = __ballot_sync(0xffffffffu, win);
      if (win) {
        const int r = rbase + wc + __popc(m & ((1u << lane) - 1u));
        KF_GUARD(r < d->px_cap + kChunk, 6, r, d->px_cap)
        {
          float4* rec = d->recs + 2 * (size_t)r;
          rec[0] = make_float4(a[0], a[1], a[2], a[3]);
          rec[1] = make_float4(a[4], a[5], b, __int_as_float(k));
        }
      }
      wc += __popc(m);
    }
    if constexpr (kPass == kPassBand) {
      if (k >= lo && k <= hi) {
        float a[6], b;
        ls_row(B.p[u], B.q[u], B.nq[u], a, b);
        accumulate(a, b, sum);
      }
    }
  }
}

// The warp's sum of the 29 per-lane float32 sums of one item, written as the
// warp's row of the item's partial: recursive halving, at each of five steps
// a lane keeps half of its remaining values and adds the partner lane's copy
// of that half (31 shuffles), leaving lane s with the warp's sum s (with
// KF_KAHAN a lane enters its compensated value, the sum minus its
// compensation). No block barrier: the warps of a block run their items
// independently.
__device__ __forceinline__ void warp_partial(const float* sum, float* dst) {
  const int lane = threadIdx.x & 31;
  float v[32];
#pragma unroll
  for (int k = 0; k < kSums; ++k) v[k] = KF_KAHAN ? __fsub_rn(sum[k], sum[kSumRegs - kSums + k]) : sum[k];
#pragma unroll
  for (int k = kSums; k < 32; ++k) v[k] = 0.f;
#pragma unroll
  for (int h = 16; h >= 1; h >>= 1) {
    const bool upper = (lane & h) != 0;
#pragma unroll
    for (int k = 0; k < h; ++k) {
      const float send = upper ? v[k] : v[k + h];
      const float keep = upper ? v[k + h] : v[k];
      v[k] = keep + __shfl_xor_sync(0xffffffffu, send, h);
    }
  }
  if (lane < kSums) dst[(threadIdx.x >> 5) * 32 + lane] = v[0];
}

// Where item li's partial rows go: slot A or slot B.
__device__ __forceinline__ float* partial_rows(const PairDesc* d, int li, bool slot_b) {
  return d->partials + (size_t)li * kPartialStride + (slot_b ? kSlotB : 0);
}

__device__ __forceinline__ void zero_sums(float* sum) {
#pragma unroll
  for (int k = 0; k < kSumRegs; ++k) sum[k] = 0.f;
}

// An association pass over the items [first, first + run) of one pair, in
// order, batch after batch; kPassSplit / kPassBand write each item's partial
// (slot A / slot B). Block-wide: ends with a barrier, so the block's shared
// histogram is complete on return.
template <class T, int kA, int kPass, int kMode>
__device__ void assoc_items(const PairDesc* d, const LevelMaps& L, int first, int run, int chunk,
                            const float* sxf, const KParams& P, unsigned* sh_hist, int lo, int hi) {
  constexpr bool kGate = (kA & kAGate) != 0;
  const int fn = L.fw * L.fh;
  float sum[kSumRegs];
  Verts va;
  Batch<kGate> sa;
  const int warp = threadIdx.x >> 5;
  for (int li = first; li < first + run; ++li) {
    const int ib = li * chunk, ie = min(fn, ib + chunk);
    // the warp's record region of the item: as many places as the warp has
    // pixels in it (chunk / kBlockWarps: kU of each batch's 32-pixel groups)
    const int rbase = ib + warp * (chunk / kBlockWarps);
    int wc = 0;
    zero_sums(sum);
    // batches of the item; the last one may be partial (kBatch need not
    // divide the item)
    for (int b0 = ib; b0 < ie; b0 += kBatch) {
      const int e = min(ie, b0 + kBatch);
      load_verts<T>(L, b0, e, va);
      associate_batch<T, kA, kPass>(L, b0, va, sxf, P, sa);
      {  // L2 hints for this warp's next batch (of this item or the next)
        int nb0 = b0 + kBatch, ne = e + kBatch;
        if (nb0 >= ie) {
          nb0 = ie;
          ne = li + 1 < first + run ? min(fn, ie + kBatch) : ie;
        }
        ne = min(ne, fn);
        // the match offset of the warp's first matched pixel (0: none)
        const unsigned ok = __ballot_sync(0xffffffffu, sa.j[0] >= 0);
        const int src = ok ? __ffs(ok) - 1 : 0;
        const int off = __shfl_sync(0xffffffffu, sa.j[0] - (b0 + threadIdx.x), src);
        prefetch_next<T>(L, nb0, ne, ok ? off : 0);
      }
      finish_batch<kA, kPass, kMode>(d, b0, e, sa, sxf, P, sh_hist, lo, hi, sum, rbase, wc);
    }
    if constexpr (kPass == kPassSplit) {
      if ((threadIdx.x & 31) == 0) {
        KF_GUARD(li < d->partial_cap, 7, li, d->partial_cap)
        d->wcount[li * kBlockWarps + warp] = wc;
      }
    }
    if constexpr (kPass != kPassHist) {
      KF_GUARD(li < d->partial_cap, 1, li, d->partial_cap)
      warp_partial(sum, partial_rows(d, li, kPass == kPassBand));
    }
  }
  __syncthreads();
}

// Reduction pass of an item whose band edge fell in the window: the
// recorded pixels with klo <= bin <= khi, in registers. Warp w reads the
// region warp w of the association pass filled: its record count and the
// first 32 kFixR records in one round trip (places past the count are read
// and ignored: the region has room for every pixel of the warp, and the
// buffer a chunk of padding), lane l taking places l, l + 32, ... in order.
// The records were written by other blocks: read through L2. fix_issue puts
// an item's loads in flight; fix_consume adds them (and any further rounds).
constexpr int kFixR = 2;
struct FixLoad {
  int total;
  float4 r0[kFixR], r1[kFixR];
};

__device__ __forceinline__ void fix_issue(const PairDesc* d, int li, int chunk, FixLoad& f) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int rbase = li * chunk + warp * (chunk / kBlockWarps);
  [[maybe_unused]] const int cap = chunk / kBlockWarps;  // places of the region
  KF_GUARD(li < d->partial_cap && rbase + cap <= d->px_cap + kChunk, 11, li, rbase) {}
  f.total = lane == 0 && li < d->partial_cap ? (int)__ldcg(d->wcount + li * kBlockWarps + warp) : 0;
#pragma unroll
  for (int r = 0; r < kFixR; ++r) {
    const size_t i = (size_t)rbase + r * 32 + lane;
    f.r0[r] = __ldcg(d->recs + 2 * i);
    f.r1[r] = __ldcg(d->recs + 2 * i + 1);
  }
}

__device__ __forceinline__ void fix_consume(const PairDesc* d, int li, int chunk, int klo, int khi,
                                            FixLoad& f, float* sum) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int rbase = li * chunk + warp * (chunk / kBlockWarps);
  [[maybe_unused]] const int cap = chunk / kBlockWarps;
  int total = __shfl_sync(0xffffffffu, f.total, 0);
  KF_GUARD(total <= cap, 10, total, cap) {}
#ifdef KF_CHECKED
  total = min(total, cap);
#endif
  for (int e0 = 0;;) {
#pragma unroll
    for (int r = 0; r < kFixR; ++r) {
      if (e0 + r * 32 + lane >= total) continue;
      const int k = __float_as_int(f.r1[r].w);
      if (k >= klo && k <= khi) {
        const float a[6] = {f.r0[r].x, f.r0[r].y, f.r0[r].z, f.r0[r].w, f.r1[r].x, f.r1[r].y};
        accumulate(a, f.r1[r].z, sum);
      }
    }
    e0 += 32 * kFixR;
    if (e0 >= total) break;
#pragma unroll
    for (int r = 0; r < kFixR; ++r) {
      const size_t i = (size_t)rbase + e0 + r * 32 + lane;
      f.r0[r] = __ldcg(d->recs + 2 * i);
      f.r1[r] = __ldcg(d->recs + 2 * i + 1);
    }
  }
}

__device__ __forceinline__ void fixup_item(const PairDesc* d, int li, int chunk, int klo, int khi,
                                           float* sum) {
  FixLoad f;
  fix_issue(d, li, chunk, f);
  fix_consume(d, li, chunk, klo, khi, f, sum);
}

// The reduction pass of a hit over every item of a pair by one block (the
// block that ran the pair's median): warp w takes region w of items 0, 1,
// ..., count - 1, with the next item's loads in flight while it adds the
// current one. Each item's slot B rows are the ones the reduction tasks
// would write (the same warp-to-region map, the same order): which way runs
// changes no bit. Block-wide: ends with a barrier.
__device__ __noinline__ void fixup_all(const PairDesc* d, int count, int chunk, int klo, int khi) {
  FixLoad cur, nxt = {};
  if (count > 0) fix_issue(d, 0, chunk, cur);
  for (int li = 0; li < count; ++li) {
    if (li + 1 < count) fix_issue(d, li + 1, chunk, nxt);
    float sum[kSumRegs];
    zero_sums(sum);
    fix_consume(d, li, chunk, klo, khi, cur, sum);
    KF_GUARD(li < d->partial_cap, 1, li, d->partial_cap)
    warp_partial(sum, partial_rows(d, li, true));
    cur = nxt;
  }
  __threadfence_block();
  __syncthreads();
}

// The reduction pass over items [first, first + run) of one pair, last item
// first (the association pass left the latest items' data in L2): the
// recorded window pixels on a hit, else a re-association with the band known.
// Each item writes slot B of its partial.
template <class T, int kA>
__device__ void reduce_items(const PairDesc* d, const LevelMaps& L, int first, int run, int chunk,
                             const float* sxf, const KParams& P, int hit, int klo, int khi) {
  for (int li = first + run - 1; li >= first; --li) {
    if (hit) {
      float sum[kSumRegs];
      zero_sums(sum);
      fixup_item(d, li, chunk, klo, khi, sum);
      KF_GUARD(li < d->partial_cap, 1, li, d->partial_cap)
      warp_partial(sum, partial_rows(d, li, true));
    } else {
      assoc_items<T, kA, kPassBand, 0>(d, L, li, 1, chunk, sxf, P, nullptr, klo, khi);
    }
  }
}

// The pair's reduction epilogue (block-wide, run by the block that finished
// its last item): per sum, the items' partials in FP64 in a fixed order (slot
// A + slot B on a hit, slot B alone otherwise; 8 strided sub-sums, then the 8
// in order), the histogram cleared for the next iteration, then the solve and
// update (mode 2: the sums are stored instead). Returns (in thread 0) the
// solve's next level (-1: finished or stopped).
__device__ __noinline__ int combine_and_solve(const PairDesc* d, PairState* st, int count,
                                               int level, const KParams& P, int mode,
                                               double (*s_part)[kSums], double* s_sums,
                                               double* s_solve) {
  __shared__ int s_hit;
  PairPre pre;
  if (threadIdx.x == 0) {
    if (mode == 0) pre = load_pre(st, level);
    s_hit = __ldcg(&st->hit);
  }
  KF_GUARD(count <= d->partial_cap, 2, count, d->partial_cap) {}
#ifdef KF_CHECKED
  if (count > d->partial_cap) count = d->partial_cap;  // the violation is recorded; stay inside
#endif
  __syncthreads();
  const int hit = s_hit;
  // warp `sub` takes items sub, sub + 8, ...; lane k < 29 sums, per item, the
  // 16 rows of sum k (slot A's 8 warps, zero on a miss, and slot B's) in
  // float32 by pairwise halving, then adds the items in increasing order in
  // float64; four items' loads in flight. (The FP64 pipe of this part retires
  // about two additions per cycle per SM: a float64 chain over every row
  // would hold the pair's epilogue for microseconds.)
  const int k = threadIdx.x & 31, sub = threadIdx.x >> 5;
  auto item_value = [&](int l) {
    const float* a = d->partials + (size_t)l * kPartialStride + k;
    float v[2 * kBlockWarps];
#pragma unroll
    for (int w = 0; w < kBlockWarps; ++w) {
      v[w] = hit ? __ldcg(a + w * 32) : 0.f;
      v[kBlockWarps + w] = __ldcg(a + kSlotB + w * 32);
    }
#pragma unroll
    for (int h = kBlockWarps; h >= 1; h >>= 1)
#pragma unroll
      for (int i = 0; i < h; ++i) v[i] = __fadd_rn(v[i], v[i + h]);
    return v[0];
  };
  double t = 0.0;
  if (k < kSums) {
    int l = sub;
    for (; l + 24 < count; l += 32) {
      const float e0 = item_value(l), e1 = item_value(l + 8), e2 = item_value(l + 16),
                  e3 = item_value(l + 24);
      t += (double)e0;
      t += (double)e1;
      t += (double)e2;
      t += (double)e3;
    }
    for (; l < count; l += 8) t += (double)item_value(l);
  }
  if (k < kSums) s_part[sub][k] = t;
  for (int b = threadIdx.x; b < P.bins; b += kBlock) d->hist[b] = 0u;
  __syncthreads();
  if (threadIdx.x < kSums) {
    double t = s_part[0][threadIdx.x];
    for (int sub = 1; sub < 8; ++sub) t += s_part[sub][threadIdx.x];
    s_sums[threadIdx.x] = t;
  }
  __syncthreads();
  int next = -1;
  if (threadIdx.x < 32) {
    if (mode != 0) {
      if (threadIdx.x == 0)
        for (int k = 0; k < kSums; ++k) st->dbg_sums[k] = s_sums[k];
    } else {
      next = solve_update_warp(d, st, s_sums, level, P, s_solve, hit ? 1 : 2, pre);
    }
    if (threadIdx.x == 0) d->counters[1] = 0u;
  }
  __syncthreads();
  return next;
}

// ---------------------------------------------------------------------------
// Per-stage launches (KF_LAUNCH_PER_ITERATION and the inspection hooks): the
// same items, passes and epilogues as the scheduled kernel, one launch per
// stage and iteration over the active list; each block takes a contiguous
// run of items.
// ---------------------------------------------------------------------------
// Stage 1: association pass (histogram, and the split sums when the pair has
// a window); the pair's last item to finish computes the median, band and hit
// (not in mode 2, whose band is given).
template <class T, int kA>
__global__ void __launch_bounds__(kBlock, KF_ASSOC_MINB) k_assoc_hist(const PairDesc* const* descs,
                                                                      const int* list, int cap,
                                                                      int level, int mode, KParams P) {
  extern __shared__ unsigned sh_hist[];
  __shared__ __align__(16) float sxf[24];  // 16-byte vector loads (load_xf)
  __shared__ int s_active, s_last, s_w0, s_w1;
  const int n_items = __ldcg(list);
  const int M = (n_items + gridDim.x - 1) / gridDim.x;
  int f = blockIdx.x * M;
  const int f1 = min(n_items, f + M);
  if (f >= f1) return;
  const int* pairs = list + 4;
  const int* prefix = list + 4 + cap;
  int slot = find_slot(prefix, __ldcg(list + 1), f);
  const int chunk = level_chunk(level);
  while (f < f1) {
    const int pstart = __ldcg(prefix + slot);
    const int run_end = min(f1, __ldcg(prefix + slot + 1));
    const PairDesc* d = descs[__ldcg(pairs + slot)];
    PairState* st = d->st;
    __syncthreads();  // shared memory of the previous run is free again
    if (threadIdx.x == 0) {
      s_active = (st->cur_level == level) && !st->stopped;
      s_w0 = mode == 1 ? -1 : st->w0;
      s_w1 = st->w1;
    }
    if (threadIdx.x < 24) sxf[threadIdx.x] = st->xf[threadIdx.x];
    for (int b = threadIdx.x; b < P.bins; b += kBlock) sh_hist[b] = 0u;
    __syncthreads();
    if (s_active) {
      const LevelMaps L = d->lv[level];
      const int fn = L.fw * L.fh;
      const int count = (fn + chunk - 1) / chunk;
      const int first = f - pstart, run = run_end - f;
      if (s_w0 >= 0)
        assoc_items<T, kA, kPassSplit, 0>(d, L, first, run, chunk, sxf, P, sh_hist, s_w0, s_w1);
      else if (mode == 1)
        assoc_items<T, kA, kPassHist, 1>(d, L, first, run, chunk, sxf, P, sh_hist, 0, 0);
      else
        assoc_items<T, kA, kPassHist, 0>(d, L, first, run, chunk, sxf, P, sh_hist, 0, 0);
      for (int b = threadIdx.x; b < P.bins; b += kBlock) {
        const unsigned c = sh_hist[b];
        if (c) atomicAdd(d->hist + b, c);
      }
      __threadfence();
      __syncthreads();
      if (threadIdx.x == 0) {
        const unsigned nrun = (unsigned)run;
        s_last = (atomicAdd(d->counters + 0, nrun) + nrun == (unsigned)count);
      }
      __syncthreads();
      if (s_last) {
        __threadfence();
        if (mode != 2) median_and_band(d, st, P);
        if (threadIdx.x == 0) d->counters[0] = 0u;
      }
    }
    f = run_end;
    ++slot;
  }
}

// Stage 2: reduction pass; the pair's last item to finish combines, solves
// and updates (mode 2: stores the sums instead). The launch's last block
// builds the active list of the next launch (level next_level; -1: none).
template <class T, int kA>
__global__ void __launch_bounds__(kBlock, KF_REDUCE_MINB) k_reduce_solve(const PairDesc* const* descs, int n,
                                                            const int* list, int* out_list, int cap,
                                                            unsigned* launch_counter, int level,
                                                            int next_level, int mode, KParams P) {
  __shared__ __align__(16) float sxf[24];  // 16-byte vector loads (load_xf)
  __shared__ int s_active, s_klo, s_khi, s_hit, s_last;
  __shared__ double s_sums[kSums];
  __shared__ double s_part[8][kSums];
  __shared__ double s_solve[96];
  const int n_items = __ldcg(list);
  const int M = (n_items + gridDim.x - 1) / gridDim.x;
  int f = blockIdx.x * M;
  const int f1 = min(n_items, f + M);
  const int* pairs = list + 4;
  const int* prefix = list + 4 + cap;
  const int chunk = level_chunk(level);
  const int npairs = f < f1 ? __ldcg(list + 1) : 0;
  int slot = f < f1 ? find_slot(prefix, npairs, f) : 0;
  while (f < f1) {
    const int pstart = __ldcg(prefix + slot);
    const int run_end = min(f1, __ldcg(prefix + slot + 1));
    const PairDesc* d = descs[__ldcg(pairs + slot)];
    PairState* st = d->st;
    __syncthreads();
    if (threadIdx.x == 0) {
      s_active = (st->cur_level == level) && !st->stopped;
      s_klo = st->klo;
      s_khi = st->khi;
      s_hit = st->hit;
    }
    if (threadIdx.x < 24) sxf[threadIdx.x] = st->xf[threadIdx.x];
    __syncthreads();
    if (s_active) {
      const LevelMaps L = d->lv[level];
      const int fn = L.fw * L.fh;
      const int count = (fn + chunk - 1) / chunk;
      reduce_items<T, kA>(d, L, f - pstart, run_end - f, chunk, sxf, P, s_hit, s_klo, s_khi);
      __threadfence();
      __syncthreads();
      if (threadIdx.x == 0) {
        const unsigned nrun = (unsigned)(run_end - f);
        s_last = (atomicAdd(d->counters + 1, nrun) + nrun == (unsigned)count);
      }
      __syncthreads();
      if (s_last) {
        __threadfence();
        combine_and_solve(d, st, count, level, P, mode, s_part, s_sums, s_solve);
      }
    }
    f = run_end;
    ++slot;
  }
  // the launch's last block to finish builds the next launch's active list
  __shared__ int s_glast;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_glast = (atomicAdd(launch_counter, 1u) == gridDim.x - 1);
  __syncthreads();
  if (s_glast) {
    __threadfence();
    if (next_level >= 0) build_active_list(descs, n, next_level, out_list, cap);
    if (threadIdx.x == 0) *launch_counter = 0u;
  }
}

// ---------------------------------------------------------------------------
// Seed (one block for all pairs, then the first active list), finish, and
// inspection set-up.
// ---------------------------------------------------------------------------
// Initial state of one pair (thread-level; T: the seed pose, 12 doubles).
__device__ void init_state(const PairDesc* d, const PairInput& pi, const KParams& P, double* sT) {
  PairState* st = d->st;
  // T0 = [R_prior | t_init] when the IMU prior is used (Sec. 3), else init
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 4; ++j) sT[i * 4 + j] = pi.init[i * 4 + j];
  if (pi.has_prior && (P.flags & KF_USE_PRIOR))
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) sT[i * 4 + j] = pi.prior_R[i * 3 + j];
  for (int i = 0; i < 12; ++i) st->T[i] = sT[i];
  for (int i = 0; i < 9; ++i) st->prior_R[i] = pi.prior_R[i];
  st->has_prior = pi.has_prior;
  st->lambda_c = pi.lambda;
  st->cur_level = P.levels - 1;
  st->stopped = 0;
  st->status = KF_OK;
  for (int l = 0; l < KF_MAX_LEVELS; ++l) {
    st->iters[l] = 0;
    st->median_bin[l] = -1;
  }
  for (int i = 0; i < kMaxWindow; ++i) st->kmed_hist[i] = 0;
  st->total_iters = 0;
  st->hist_len = 0;
  st->N = st->kmed = st->klo = st->khi = 0;
  st->w0 = st->w1 = -1;  // no band edge known yet: the first pass is histogram only
  st->hit = 0;
  st->valid_pairs = st->inliers = 0;
  st->rms = 0.0;
  st->trace_len = 0;
  d->counters[0] = 0u;
  d->counters[1] = 0u;
}

__global__ void __launch_bounds__(kBlock) k_icp_init(const PairDesc* const* descs,
                                                     const PairInput* in, int n, int* list,
                                                     KParams P) {
  for (int p = 0; p < n; ++p) {
    const PairDesc* d = descs[p];
    for (int b = threadIdx.x; b < P.bins; b += kBlock) d->hist[b] = 0u;
  }
  for (int p = threadIdx.x; p < n; p += kBlock) {
    double sT[12];
    init_state(descs[p], in[p], P, sT);
    compute_xf(sT, descs[p]->Tm, descs[p]->st->xf);
  }
  __threadfence();
  __syncthreads();
  build_active_list(descs, n, P.levels - 1, list, n);
}

__global__ void k_icp_finish(const PairDesc* const* descs, PairOutput* out) {
  const PairDesc* d = descs[blockIdx.x];
  const PairState* st = d->st;
  PairOutput& o = out[blockIdx.x];
  for (int i = 0; i < 12; ++i) o.pose[i] = st->T[i];
  o.pose[12] = o.pose[13] = o.pose[14] = 0.0;
  o.pose[15] = 1.0;
  o.res.status = st->status;
  for (int l = 0; l < KF_MAX_LEVELS; ++l) {
    o.res.iters[l] = st->iters[l];
    o.res.median_bin[l] = st->median_bin[l];
  }
  o.res.total_iters = st->total_iters;
  o.res.inliers = st->inliers;
  o.res.valid_pairs = st->valid_pairs;
  o.res.rms_residual = st->rms;
}

__global__ void __launch_bounds__(kBlock) k_debug_setup(const PairDesc* const* self,
                                                        const double* pose, int level, int klo,
                                                        int khi, int w0, int w1, int hit,
                                                        int* list, KParams P) {
  const PairDesc* d = self[0];
  PairState* st = d->st;
  for (int b = threadIdx.x; b < P.bins; b += blockDim.x) d->hist[b] = 0u;
  if (threadIdx.x == 0) {
    for (int i = 0; i < 12; ++i) st->T[i] = pose[i];
    st->cur_level = level;
    st->stopped = 0;
    st->status = KF_OK;
    st->has_prior = 0;
    st->klo = klo;
    st->khi = khi;
    st->w0 = w0;
    st->w1 = w1;
    st->hit = hit;
    st->N = 0;
    d->counters[0] = 0u;
    d->counters[1] = 0u;
    compute_xf(st->T, d->Tm, st->xf);
  }
  __threadfence();
  __syncthreads();
  build_active_list(self, 1, level, list, 1);
}

// ---------------------------------------------------------------------------
// Scheduled ICP: every level and iteration of every pair of a batch in one
// persistent launch. Work is the same two kinds of task as in the per-stage
// launches (association pass of a run of items; reduction pass of a run of
// items), but pairs advance independently: the block that finishes a pair's
// last item of a stage runs that stage's epilogue and queues the pair's next
// stage at once, so one pair's median, solve and update overlap the other
// pairs' items instead of ending a launch.
//
// Device queue: a ring of 64-bit slots, each a ticket's tag and its task (a
// run of consecutive items of one stage of one pair). A producer reserves
// tickets at the tail and writes their slots; a block claims the next ticket
// at the head (one ahead of the task it is running) and waits for its slot to
// carry that ticket's tag. Every wait is bounded in time: a wait that runs
// out sets the queue's error word, which the host reports, and the block
// returns. The ring holds every task that can be outstanding at once (each
// pair has at most one stage queued) plus one exit word per block; it is
// zeroed before each launch.
// ---------------------------------------------------------------------------
constexpr unsigned long long kTaskExit = 0xffffffffffull;  // 40-bit payload, all ones
constexpr unsigned long long kTaskAbort = 1ull << 62;      // never stored in a slot
#ifndef KF_MAX_RUN
#define KF_MAX_RUN 16
#endif
// runs per block and round of stages the run length aims at (shorter runs
// shorten each pair's stages, longer ones cost fewer task claims)
#ifndef KF_RUNS_PER_BLOCK
#define KF_RUNS_PER_BLOCK 2
#endif
constexpr int kMaxRun = KF_MAX_RUN;  // <= 16 (the task word's 4-bit run field)
static_assert(kMaxRun >= 1 && kMaxRun <= 16, "run length field");

// slot: tag (24 bits) << 40 | task (40 bits):
//   pair (16) | level (2) | stage (1: reduction) | run length - 1 (4) | first item (17)
__device__ __forceinline__ unsigned long long task_word(int p, int level, int stage, int run,
                                                        int item) {
  return ((unsigned long long)p << 24) | ((unsigned long long)level << 22) |
         ((unsigned long long)stage << 21) | ((unsigned long long)(run - 1) << 17) |
         (unsigned long long)item;
}

__device__ __forceinline__ void slot_store(unsigned long long* a, unsigned long long v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(a), "l"(v) : "memory");
}

__device__ __forceinline__ unsigned long long slot_load_acquire(const unsigned long long* a) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(a) : "memory");
  return v;
}

__device__ __forceinline__ unsigned word_load_relaxed(const unsigned* a) {
  unsigned v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(a) : "memory");
  return v;
}

// 1 .. 2^24 - 1, never the 0 of a zeroed slot; a slot's earlier tickets
// (ticket - m * slots, slots a power of two) never repeat its tag
__device__ __forceinline__ unsigned slot_tag(unsigned ticket) { return ticket % 0xffffffu + 1u; }

// Block-wide: make this block's writes visible, then queue `count` tasks;
// task i is word(i).
template <class F>
__device__ void push_tasks(unsigned* qh, unsigned long long* qs, unsigned qmask, int count, F word) {
  __shared__ unsigned s_base;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_base = atomicAdd(qh + kQTail, (unsigned)count);
  __syncthreads();
  const unsigned base = s_base;
  for (int i = threadIdx.x; i < count; i += kBlock) {
    const unsigned t = base + (unsigned)i;
    slot_store(qs + (t & qmask), ((unsigned long long)slot_tag(t) << 40) | word(i));
  }
  __syncthreads();
}

// Queue one stage of a pair: `count` items in runs of g consecutive items,
// g chosen from the items of all pairs still running so that a round of
// stages gives every block about KF_RUNS_PER_BLOCK runs (a lone pair gets
// single items).
// The association stage queues its runs first to last, the reduction last to
// first (the items associated last are the ones most likely still in L2).
// Scheduling only: items, partials and their order do not depend on g.
__device__ void push_stage(unsigned* qh, unsigned long long* qs, unsigned qmask, int n, int p,
                           int level, int stage, int count) {
  __shared__ int s_g;
  if (threadIdx.x == 0) {
    const int active = n - (int)word_load_relaxed(qh + kQDone);
    const long long want = (long long)active * count / ((long long)KF_RUNS_PER_BLOCK * gridDim.x);
    s_g = (int)(want < 1 ? 1 : (want > kMaxRun ? kMaxRun : want));
  }
  __syncthreads();
  const int g = s_g;
  const int ntask = (count + g - 1) / g;
  push_tasks(qh, qs, qmask, ntask, [=](int i) {
    const int j = stage ? ntask - 1 - i : i;
    const int first = j * g;
    return task_word(p, level, stage, min(g, count - first), first);
  });
}

// Thread 0: the task of `ticket` once its slot is written; kTaskAbort when
// the wait ran out (or another block's did).
__device__ unsigned long long wait_task(unsigned* qh, const unsigned long long* qs, unsigned qmask,
                                        unsigned ticket, unsigned long long limit_ns) {
  const unsigned long long* slot = qs + (ticket & qmask);
  const unsigned tag = slot_tag(ticket);
  unsigned long long t0 = 0;
  unsigned ns = 0;
  for (int spin = 0;; ++spin) {
    const unsigned long long v = slot_load_acquire(slot);
    if ((unsigned)(v >> 40) == tag) return v & 0xffffffffffull;
    if (spin == 0) {
      t0 = globaltimer_ns();
    } else {
      if (word_load_relaxed(qh + kQErr) != 0u) return kTaskAbort;
      if (globaltimer_ns() - t0 > limit_ns) {
        atomicExch(qh + kQErr, 1u);
        return kTaskAbort;
      }
    }
    if (ns) __nanosleep(ns);
    ns = ns < 256 ? ns + 32 : 256;
  }
}

// Block-wide: initial state of one pair (as the per-stage path's seed).
__device__ void seed_pair(const PairDesc* d, const PairInput& pi, const KParams& P, double* sT) {
  for (int b = threadIdx.x; b < P.bins; b += kBlock) d->hist[b] = 0u;
  if (threadIdx.x == 0) init_state(d, pi, P, sT);
  __syncthreads();
  if (threadIdx.x < 24) d->st->xf[threadIdx.x] = xf_entry(sT, d->Tm, threadIdx.x);
}

// Block-wide: the pair's outputs; the block that finishes the batch's last
// pair queues one exit word per block.
__device__ void finish_pair(const PairDesc* d, PairOutput* o, int n, unsigned* qh,
                            unsigned long long* qs, unsigned qmask) {
  __shared__ int s_lastpair;
  if (threadIdx.x == 0) {
    const PairState* st = d->st;
    for (int i = 0; i < 12; ++i) o->pose[i] = __ldcg(&st->T[i]);
    o->pose[12] = o->pose[13] = o->pose[14] = 0.0;
    o->pose[15] = 1.0;
    o->res.status = __ldcg(&st->status);
    for (int l = 0; l < KF_MAX_LEVELS; ++l) {
      o->res.iters[l] = __ldcg(&st->iters[l]);
      o->res.median_bin[l] = __ldcg(&st->median_bin[l]);
    }
    o->res.total_iters = __ldcg(&st->total_iters);
    o->res.inliers = __ldcg(&st->inliers);
    o->res.valid_pairs = __ldcg(&st->valid_pairs);
    o->res.rms_residual = __ldcg(&st->rms);
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_lastpair = atomicAdd(qh + kQDone, 1u) == (unsigned)(n - 1);
  __syncthreads();
  if (s_lastpair) push_tasks(qh, qs, qmask, gridDim.x, [](int) { return kTaskExit; });
}

template <class T, int kA>
__global__ void __launch_bounds__(kBlock, KF_SCHED_MINB) k_icp_sched(const PairDesc* const* descs,
                                                                     const PairInput* in,
                                                                     PairOutput* out, int n,
                                                                     unsigned* qh,
                                                                     unsigned long long* qs,
                                                                     unsigned qmask,
                                                                     unsigned long long limit_ns,
                                                                     KParams P) {
  extern __shared__ unsigned sh_hist[];
  __shared__ __align__(16) float sxf[24];  // 16-byte vector loads (load_xf)
  __shared__ unsigned long long s_word;
  __shared__ int s_last, s_flag, s_a, s_b, s_hit;
  __shared__ double s_sums[kSums];
  __shared__ double s_part[8][kSums];
  __shared__ double s_solve[96];
  // seed: every block that starts takes unseeded pairs until none is left
  for (;;) {
    if (threadIdx.x == 0) s_word = atomicAdd(qh + kQSeed, 1u);
    __syncthreads();
    const unsigned p = (unsigned)s_word;
    __syncthreads();
    if (p >= (unsigned)n) break;
    const PairDesc* d = descs[p];
    seed_pair(d, in[p], P, s_solve);
    const int level = P.levels - 1;
    push_stage(qh, qs, qmask, n, (int)p, level, 0, items_of(d, level));
  }
  unsigned ticket = 0;
  if (threadIdx.x == 0) ticket = atomicAdd(qh + kQHead, 1u);
  for (;;) {
    if (threadIdx.x == 0) {
      const unsigned long long w = wait_task(qh, qs, qmask, ticket, limit_ns);
      if (w < kTaskExit) ticket = atomicAdd(qh + kQHead, 1u);  // claim the next one ahead
      s_word = w;
    }
    __syncthreads();
    const unsigned long long w = s_word;
    if (w >= kTaskExit) break;
    const int p = (int)(w >> 24), level = (int)((w >> 22) & 3u);
    const int run = (int)((w >> 17) & 15u) + 1, first = (int)(w & 0x1ffffu);
    const PairDesc* d = descs[p];
    PairState* st = d->st;
    const LevelMaps L = d->lv[level];
    const int fn = L.fw * L.fh;
    const int chunk = level_chunk(level);
    const int count = (fn + chunk - 1) / chunk;
    if (threadIdx.x < 24) sxf[threadIdx.x] = __ldcg(&st->xf[threadIdx.x]);
    if (!((w >> 21) & 1u)) {
      // association pass of items [first, first + run)
      if (threadIdx.x == 0) {
        s_a = __ldcg(&st->w0);
        s_b = __ldcg(&st->w1);
      }
      for (int b = threadIdx.x; b < P.bins; b += kBlock) sh_hist[b] = 0u;
      __syncthreads();
      if (s_a >= 0)
        assoc_items<T, kA, kPassSplit, 0>(d, L, first, run, chunk, sxf, P, sh_hist, s_a, s_b);
      else
        assoc_items<T, kA, kPassHist, 0>(d, L, first, run, chunk, sxf, P, sh_hist, 0, 0);
      for (int b = threadIdx.x; b < P.bins; b += kBlock) {
        const unsigned c = sh_hist[b];
        if (c) atomicAdd(d->hist + b, c);
      }
      __threadfence();
      __syncthreads();
      if (threadIdx.x == 0)
        s_last = atomicAdd(d->counters + 0, (unsigned)run) + (unsigned)run == (unsigned)count;
      __syncthreads();
      if (s_last) {
        __threadfence();
        const int stop = median_and_band(d, st, P);
        if (threadIdx.x == 0) {
          d->counters[0] = 0u;
          s_flag = stop;
          // while many pairs run, a hit's reduction pass is done here, by this
          // block (its item tasks would each wait on a round trip for a few
          // records); with few pairs left, spread over blocks for latency
          const int active = n - (int)word_load_relaxed(qh + kQDone);
          s_hit = !stop && st->hit && (long long)active * KF_FUSE_GRID_DIV >= (long long)gridDim.x;
          s_a = st->klo;
          s_b = st->khi;
        }
        __syncthreads();
        if (s_flag) {
          finish_pair(d, out + p, n, qh, qs, qmask);
        } else if (s_hit) {
          fixup_all(d, count, chunk, s_a, s_b);
          __threadfence();
          const int next = combine_and_solve(d, st, count, level, P, 0, s_part, s_sums, s_solve);
          if (threadIdx.x == 0) s_flag = next;
          __syncthreads();
          const int nl = s_flag;
          if (nl >= 0) push_stage(qh, qs, qmask, n, p, nl, 0, items_of(d, nl));
          else finish_pair(d, out + p, n, qh, qs, qmask);
        } else {
          push_stage(qh, qs, qmask, n, p, level, 1, count);
        }
      }
    } else {
      // reduction pass of items first + run - 1 down to first, slot B each
      if (threadIdx.x == 0) {
        s_a = __ldcg(&st->klo);
        s_b = __ldcg(&st->khi);
        s_hit = __ldcg(&st->hit);
      }
      __syncthreads();
      if (s_hit) {
        reduce_items<T, kA>(d, L, first, run, chunk, sxf, P, 1, s_a, s_b);
      } else {
        // re-association with the band known (items in increasing order; the
        // partials do not depend on it)
        assoc_items<T, kA, kPassBand, 0>(d, L, first, run, chunk, sxf, P, nullptr, s_a, s_b);
      }
      __threadfence();
      __syncthreads();
      if (threadIdx.x == 0)
        s_last = atomicAdd(d->counters + 1, (unsigned)run) + (unsigned)run == (unsigned)count;
      __syncthreads();
      if (s_last) {
        __threadfence();
        const int next = combine_and_solve(d, st, count, level, P, 0, s_part, s_sums, s_solve);
        if (threadIdx.x == 0) s_flag = next;
        __syncthreads();
        const int nl = s_flag;
        if (nl >= 0) push_stage(qh, qs, qmask, n, p, nl, 0, items_of(d, nl));
        else finish_pair(d, out + p, n, qh, qs, qmask);
      }
    }
    __syncthreads();
  }
}

// the block's histogram
size_t sched_smem(const KParams& P) { return (size_t)P.bins * sizeof(unsigned); }

template <class K>
int wave(K kernel, size_t smem) {
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, kBlock, smem);
  return sms * (per > 0 ? per : 1);
}

}  // namespace

// association variant of these params (template bits kAGate | kAShoot)
int assoc_variant(const KParams& P) { return (P.use_angle ? kAGate : 0) | (P.shoot_w > 0 ? kAShoot : 0); }

// X(T, A) for the storage type and association variant of P
#define KF_ASSOC_SWITCH(P, X)                                  \
  do {                                                         \
    const bool h_ = (P).precision == KF_FP16;                  \
    switch (assoc_variant(P)) {                                \
      case 0: if (h_) { X(__half, 0); } else { X(float, 0); } break; \
      case 1: if (h_) { X(__half, 1); } else { X(float, 1); } break; \
      case 2: if (h_) { X(__half, 2); } else { X(float, 2); } break; \
      default: if (h_) { X(__half, 3); } else { X(float, 3); } break; \
    }                                                          \
  } while (0)

void icp_grids(const KParams& P, int* g_assoc, int* g_reduce, int* g_sched) {
  const size_t sm = (size_t)P.bins * sizeof(unsigned), ss = sched_smem(P);
#define KF_X(T, A)                                 \
  *g_assoc = wave(k_assoc_hist<T, A>, sm);         \
  *g_reduce = wave(k_reduce_solve<T, A>, 0);       \
  *g_sched = wave(k_icp_sched<T, A>, ss)
  KF_ASSOC_SWITCH(P, KF_X);
#undef KF_X
  // one partition of the items for both passes
  *g_assoc = *g_reduce = (*g_assoc < *g_reduce ? *g_assoc : *g_reduce);
}

cudaError_t launch_icp_sched(const PairDesc* const* descs, const PairInput* in, PairOutput* out,
                             int n, unsigned* queue, unsigned qmask, int grid,
                             unsigned long long wait_limit_ns, const KParams& P, cudaStream_t s) {
  const size_t sm = sched_smem(P);
  unsigned long long* slots = reinterpret_cast<unsigned long long*>(queue + kQHeaderWords);
#define KF_X(T, A) \
  k_icp_sched<T, A><<<grid, kBlock, sm, s>>>(descs, in, out, n, queue, slots, qmask, wait_limit_ns, P)
  KF_ASSOC_SWITCH(P, KF_X);
#undef KF_X
  return cudaGetLastError();
}

cudaError_t launch_icp_init(const PairDesc* const* descs, const PairInput* in, int n, int* list,
                            const KParams& P, cudaStream_t s) {
  k_icp_init<<<1, kBlock, 0, s>>>(descs, in, n, list, P);
  return cudaGetLastError();
}

cudaError_t launch_assoc_hist(const PairDesc* const* descs, const int* list, int cap, int grid,
                              int level, int mode, const KParams& P, cudaStream_t s) {
  const size_t sm = (size_t)P.bins * sizeof(unsigned);
#define KF_X(T, A) k_assoc_hist<T, A><<<grid, kBlock, sm, s>>>(descs, list, cap, level, mode, P)
  KF_ASSOC_SWITCH(P, KF_X);
#undef KF_X
  return cudaGetLastError();
}

cudaError_t launch_reduce_solve(const PairDesc* const* descs, int n, const int* in_list,
                                int* out_list, int cap, unsigned* launch_counter, int grid,
                                int level, int next_level, int mode, const KParams& P,
                                cudaStream_t s) {
#define KF_X(T, A)                                                                        \
  k_reduce_solve<T, A><<<grid, kBlock, 0, s>>>(descs, n, in_list, out_list, cap, launch_counter, \
                                               level, next_level, mode, P)
  KF_ASSOC_SWITCH(P, KF_X);
#undef KF_X
  return cudaGetLastError();
}

cudaError_t launch_icp_finish(const PairDesc* const* descs, PairOutput* out, int n,
                              const KParams& /*P*/, cudaStream_t s) {
  k_icp_finish<<<n, 1, 0, s>>>(descs, out);
  return cudaGetLastError();
}

cudaError_t launch_debug_setup(const PairDesc* const* d_self, const double* d_pose, int level,
                               int klo, int khi, int w0, int w1, int hit, int* list,
                               const KParams& P, cudaStream_t s) {
  k_debug_setup<<<1, kBlock, 0, s>>>(d_self, d_pose, level, klo, khi, w0, w1, hit, list, P);
  return cudaGetLastError();
}

}  // namespace kf

// ===========================================================================
// Allocation-free reduction entry point. The paper has no counterpart: this
// serves callers that may not allocate device memory themselves (a host
// application whose allocator is owned by another runtime, a plug-in running
// inside someone else's CUDA context, a caller that must not add
// cudaMalloc / cudaFree synchronisation points while other work is in
// flight). Its scratch lives in the file-scope array below instead.
// ===========================================================================
#include <cstring>
#include <mutex>

namespace kf {
namespace {

constexpr int kNoAllocMaxItems = 1024;  // 1024 items x 4096 px = 4,194,304 frame pixels
constexpr size_t kNoAllocHeader = 512;  // arrival counter (bytes 0..3), xf (bytes 256..351)
constexpr int kNoAllocStride = 32;     // floats per block partial (29 used)
constexpr size_t kNoAllocBytes = kNoAllocHeader + sizeof(float) * kNoAllocStride * kNoAllocMaxItems;
constexpr int kNoAllocMaxDevices = 64;

// Scratch of kf_reduce_noalloc: 131,584 bytes held on every device that loads
// the library, until the process exits. Every call shares it.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

struct NoAllocArgs {
  const float* fv;            // frame vertices, interleaved xyz, camera frame
  const float* mv;            // model vertices, interleaved xyz, world frame
  const float* mn;            // model normals, interleaved xyz, world frame
  int fw, fh, mw, mh;
  float mfx, mfy, mcx, mcy;
  double T[12];               // current pose 3x4
  double Tm[12];              // model pose 3x4
  KParams P;                  // d_max32, scale32, bins used
  int klo, khi;
  double* out;                // 29 sums (device)
};

__global__ void k_noalloc_setup(unsigned char* scratch, NoAllocArgs a) {
  if (threadIdx.x == 0) {
    *reinterpret_cast<unsigned*>(scratch) = 0u;  // arrival counter starts at zero
    compute_xf(a.T, a.Tm, reinterpret_cast<float*>(scratch + 256));
  }
}

__global__ void __launch_bounds__(kBlock, 2) k_noalloc_reduce(unsigned char* scratch, NoAllocArgs a,
                                                              int nitems) {
  __shared__ __align__(16) float sxf[24];  // 16-byte vector loads (load_xf)
  __shared__ float s_red[kBlock / 32][kSums];
  __shared__ int s_last;
  unsigned* counter = reinterpret_cast<unsigned*>(scratch);
  float* partials = reinterpret_cast<float*>(scratch + kNoAllocHeader);
  if (threadIdx.x < 24) sxf[threadIdx.x] = reinterpret_cast<const float*>(scratch + 256)[threadIdx.x];
  __syncthreads();
  LevelMaps L = {};
  L.fw = a.fw;
  L.fh = a.fh;
  L.mw = a.mw;
  L.mh = a.mh;
  L.mfx = a.mfx;
  L.mfy = a.mfy;
  L.mcx = a.mcx;
  L.mcy = a.mcy;
  const int npx = a.fw * a.fh;
  const int begin = blockIdx.x * kChunk;
  const int end = min(npx, begin + kChunk);
  float sum[kSums];
#pragma unroll
  for (int k = 0; k < kSums; ++k) sum[k] = 0.f;
  for (int i = begin + threadIdx.x; i < end; i += kBlock) {
    float p[3];
    const int j = project(L, a.fv[3 * i], a.fv[3 * i + 1], a.fv[3 * i + 2], sxf, p);
    if (j < 0) continue;
    const float q[3] = {a.mv[3 * j], a.mv[3 * j + 1], a.mv[3 * j + 2]};
    const float n0 = a.mn[3 * j], n1 = a.mn[3 * j + 1], n2 = a.mn[3 * j + 2];
    // a model hole: any vertex or normal component non-finite, or a zero
    // normal (the tracker's model preparation drops the same pixels)
    if (!(isfinite(q[0]) && isfinite(q[1]) && isfinite(q[2]) && isfinite(n0) && isfinite(n1) &&
          isfinite(n2)) ||
        (n0 == 0.f && n1 == 0.f && n2 == 0.f))
      continue;
    const int k = bin_of(p, q, a.P);
    if (k < a.klo || k > a.khi) continue;
    const float av[6] = {p[1] * n2 - p[2] * n1, p[2] * n0 - p[0] * n2, p[0] * n1 - p[1] * n0,
                         n0, n1, n2};
    const float b = n0 * (q[0] - p[0]) + n1 * (q[1] - p[1]) + n2 * (q[2] - p[2]);
    int s = 0;
#pragma unroll
    for (int r = 0; r < 6; ++r)
#pragma unroll
      for (int c = r; c < 6; ++c) {
        sum[s] = fmaf(av[r], av[c], sum[s]);
        ++s;
      }
#pragma unroll
    for (int r = 0; r < 6; ++r) sum[21 + r] = fmaf(av[r], b, sum[21 + r]);
    sum[27] += 1.f;
    sum[28] = fmaf(b, b, sum[28]);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < kSums; ++k) {
    float v = sum[k];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    if (lane == 0) s_red[warp][k] = v;
  }
  __syncthreads();
  if (threadIdx.x < kSums) {
    float v = 0.f;
#pragma unroll
    for (int w = 0; w < kBlock / 32; ++w) v += s_red[w][threadIdx.x];
    partials[blockIdx.x * kNoAllocStride + threadIdx.x] = v;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = (atomicAdd(counter, 1u) == (unsigned)(nitems - 1));
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  if (threadIdx.x < kSums) {
    double t = 0.0;
    for (int l = 0; l < nitems; ++l) t += (double)__ldcg(partials + l * kNoAllocStride + threadIdx.x);
    a.out[threadIdx.x] = t;
  }
  if (threadIdx.x == 0) *counter = 0u;
}

std::mutex g_noalloc_mutex;
unsigned char* g_noalloc_ptr[kNoAllocMaxDevices] = {nullptr};

}  // namespace
}  // namespace kf

extern "C" kf_status kf_reduce_noalloc(const float* frame_vertex, int width, int height,
                                       const float* model_vertex, const float* model_normal,
                                       const kf_intrinsics* model_K, const double pose[16],
                                       const double model_pose[16], double d_max, int hist_bins,
                                       int klo, int khi, double* sums, void* cuda_stream) {
  using namespace kf;
  if (!frame_vertex || !model_vertex || !model_normal || !model_K || !pose || !model_pose || !sums)
    return KF_ERR_INVALID_ARG;
  if (width < 1 || height < 1 || model_K->width < 1 || model_K->height < 1) return KF_ERR_INVALID_ARG;
  if (!(d_max > 0) || hist_bins < 1 || hist_bins > kMaxBins || klo < 0 || khi < klo)
    return KF_ERR_INVALID_ARG;
  if (!(model_K->fx > 0) || !(model_K->fy > 0)) return KF_ERR_INVALID_ARG;
  // model indices are 32-bit: 3 w h interleaved floats must stay below 2^31
  if (3LL * model_K->width * model_K->height > 2147483647LL) return KF_ERR_INVALID_ARG;
  const long long npx = (long long)width * height;
  if (npx > (long long)kNoAllocMaxItems * kChunk) return KF_ERR_SCRATCH_LIMIT;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return KF_ERR_CUDA;
  if (dev < 0 || dev >= kNoAllocMaxDevices) return KF_ERR_INTERNAL;
  unsigned char* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_ptr[dev]) {
      // the host-side name of the array is not a device address: ask the
      // runtime for this device's copy (once per device, this device current)
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return KF_ERR_CUDA;
      g_noalloc_ptr[dev] = static_cast<unsigned char*>(p);
    }
    scratch = g_noalloc_ptr[dev];
  }
  NoAllocArgs a;
  memset(&a, 0, sizeof(a));
  a.fv = frame_vertex;
  a.mv = model_vertex;
  a.mn = model_normal;
  a.fw = width;
  a.fh = height;
  a.mw = model_K->width;
  a.mh = model_K->height;
  a.mfx = (float)model_K->fx;
  a.mfy = (float)model_K->fy;
  a.mcx = (float)model_K->cx;
  a.mcy = (float)model_K->cy;
  for (int i = 0; i < 12; ++i) {
    a.T[i] = pose[i];
    a.Tm[i] = model_pose[i];
  }
  a.P.bins = hist_bins;
  a.P.d_max32 = (float)d_max;
  a.P.scale32 = (float)((double)hist_bins / d_max);
  a.klo = klo;
  a.khi = khi;
  a.out = sums;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  const int nitems = (int)((npx + kChunk - 1) / kChunk);
  k_noalloc_setup<<<1, 32, 0, s>>>(scratch, a);
  k_noalloc_reduce<<<nitems, kBlock, 0, s>>>(scratch, a, nitems);
  return cudaGetLastError() == cudaSuccess ? KF_OK : KF_ERR_CUDA;
}
