// Internal device-side structures of the tracking library (not part of the ABI).
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "kf_track.h"

namespace kf {

constexpr int kSums = 29;           // 21 upper(A^T A) + 6 A^T b + n + sum b^2
// Work-item partial sums, one row of 32 floats (29 used) per warp of the
// block that ran the item, in two slots: slot A (offset 0) holds the
// association pass's sums of the pixels surely inside the band, slot B
// (offset kSlotB) the reduction pass's sums (the window pixels, or the whole
// band). Per-warp rows keep the passes free of block barriers; the combine
// adds them in a fixed order.
constexpr int kBlockWarps = 8;      // warps per block of the ICP kernels
constexpr int kSlotB = kBlockWarps * 32;
constexpr int kPartialStride = 2 * kSlotB;  // floats per work-item partial
constexpr int kBlock = kBlockWarps * 32;  // threads per block of the ICP kernels
constexpr int kChunk = 4096;        // frame pixels per work item at level 0
// Coarser levels use smaller items so that their (4x, 16x fewer) pixels still
// spread over enough blocks: 4096, 2048, 1024, 1024.
__host__ __device__ constexpr int level_chunk(int level) {
  return (kChunk >> level) > 1024 ? (kChunk >> level) : 1024;
}
constexpr int kMaxBins = 4096;
// Default band-edge windows of the association pass (KParams::win_*): the
// next iteration at a level expects its edge within [g - 5, g + 3] of this
// one's, a finer level's first iteration within [g - 8, g + 2] of the
// coarser level's last edge.
#ifndef KF_WIN_SAME_BELOW
#define KF_WIN_SAME_BELOW 5
#endif
#ifndef KF_WIN_SAME_ABOVE
#define KF_WIN_SAME_ABOVE 3
#endif
#ifndef KF_WIN_NEXT_BELOW
#define KF_WIN_NEXT_BELOW 8
#endif
#ifndef KF_WIN_NEXT_ABOVE
#define KF_WIN_NEXT_ABOVE 2
#endif
constexpr int kMaxWindow = 8;
constexpr int kDescListMax = 64;    // pairs per front-end launch

// Maps of one pyramid level. Every map is stored as planes: x plane, then y,
// then z. Model planes hold (mw * mh) elements each; frame planes are fps
// elements apart, fw * fh rounded up to a multiple of kPlaneAlign, so that
// every plane and every item of a plane starts on a 128-byte boundary (bulk
// copies need 16) and a copy rounded up past the last pixel stays inside.
constexpr int kPlaneAlign = 64;
__host__ __device__ constexpr int frame_plane_stride(int w, int h) {
  return (w * h + kPlaneAlign - 1) / kPlaneAlign * kPlaneAlign;
}
struct LevelMaps {
  int fw, fh;                 // frame level size
  int fps;                    // frame plane stride (elements)
  int mw, mh;                 // model level size
  float ffx, ffy, fcx, fcy;   // frame level intrinsics (vertex map)
  float mfx, mfy, mcx, mcy;   // model level intrinsics (projection)
  float* fdepth;              // filtered depth, fw * fh
  void* fV;                   // frame vertices, camera frame; NaN where the
                              // vertex or its normal is invalid
  void* fN;                   // frame normals, camera frame; NaN invalid
  void* mV;                   // model vertices, world frame; NaN at holes
  void* mN;                   // model normals, world frame
};

struct PairState {
  double T[12];               // current estimate, 3x4 row-major camera->world
  float xf[24];               // float32 Rw[9] tw[3] (camera->world) Rr[9] tr[3]
                              // (camera->model camera) used by the decisions
  double lambda_c;
  int cur_level;              // level being iterated, -1 when finished
  int stopped;                // 1 after an error stop
  int status;
  int iters[KF_MAX_LEVELS];
  int median_bin[KF_MAX_LEVELS];
  int total_iters;
  int hist_len;
  int kmed_hist[kMaxWindow];
  int N, kmed, klo, khi;      // current iteration (written by the histogram stage)
  int w0, w1;                 // band-edge window of the current iteration: the
                              // association pass sums bins < w0 and records bins
                              // in [w0, w1); w0 = -1: no window (histogram only)
  int hit;                    // 1: the band edge fell in the window, the
                              // reduction pass adds the recorded pixels only
  int valid_pairs, inliers;   // last completed iteration
  double rms;
  double dbg_sums[kSums];     // filled by the reduction stage in inspection mode
  double prior_R[9];          // IMU prior rotation (valid when has_prior)
  int has_prior;
  int pad2_;
  int trace_len;
  int pad_;
  kf_iter_record trace[KF_TRACE_MAX];
};

struct PairDesc {
  LevelMaps lv[KF_MAX_LEVELS];
  int levels;
  int iw, ih;                 // level-0 frame size
  const float* depth_raw;     // level-0 raw depth (tracker buffer)
  double Tm[12];              // model pose 3x4 camera->world
  PairState* st;
  unsigned* hist;             // [bins]
  float* partials;            // [items][kPartialStride]
  unsigned* counters;         // [2]: histogram stage, reduction stage
  float4* recs;               // [2 * (px + kChunk)] records of the window pixels:
                              // row a[0..5], b and bin (int bits), written by the
                              // association pass, read by the reduction pass;
                              // warp w of item li packs its records from place
                              // li * chunk + w * chunk / kBlockWarps
  unsigned* wcount;           // [items * kBlockWarps] records per item and warp
  int* dbg_index;             // [iw*ih] inspection outputs (may be null)
  int* dbg_bin;
  int partial_cap;            // work-item partials the buffer holds
  int px_cap;                 // frame pixels recs (+ kChunk) / dbg_* hold
};

// Active work list of one launch, built on the device (int buffer):
//   [0] items in the list  [1] pairs in the list  [2] level  [3] unused
//   [4 .. 4+cap)            pair index (into the descriptor list) per entry
//   [4+cap .. 4+2cap+1)     item prefix: entry s owns items [prefix[s], prefix[s+1])
// Item j of a pair at level l covers frame pixels [j c, min(w h, (j+1) c)),
// c = level_chunk(l).
__host__ __device__ constexpr int list_ints(int cap) { return 4 + 2 * cap + 1; }

// Queue of the scheduled ICP launch: header words (each on its own 128-byte
// line), then a ring of 64-bit task slots. Zeroed before each launch.
constexpr int kQHead = 0;    // next ticket to claim
constexpr int kQTail = 32;   // next ticket to reserve
constexpr int kQDone = 64;   // pairs finished
constexpr int kQErr = 96;    // 1: a bounded wait ran out
constexpr int kQSeed = 128;  // next pair to seed
constexpr int kQHeaderWords = 256;
constexpr int kMaxItemsPerLevel = 131071;  // 17-bit item field of a task
constexpr int kMaxSchedPairs = 65535;      // 16-bit pair field

struct DescList {
  const PairDesc* d[kDescListMax];
  const float* depth[kDescListMax];  // level-0 raw depth of each pair (device)
  int n;
};

// Parameters shared by every kernel, passed by value.
struct KParams {
  int levels;
  int caps[KF_MAX_LEVELS];
  int bins;
  float d_max32;
  float scale32;              // (float)(bins / d_max)
  double kappa;
  float cos_min32;
  int use_angle;
  int conv_window;
  int lambda_mode;
  int n_min;
  unsigned flags;
  int precision;
  // band-edge windows of the association pass: the next iteration at the
  // same level expects its band edge in [g - below, g + above] around this
  // iteration's edge g; the first iteration of a finer level around the
  // coarser level's last edge
  int split_ok;               // a window can hit (the band always starts at bin 0)
  int win_same_below, win_same_above, win_next_below, win_next_above;
  // front end
  int bil_radius;
  float bil_inv2sr2;          // 1 / (2 sigma_r^2)
  float bil_sw[81];           // -(dx^2 + dy^2) / (2 sigma_s^2), (2r+1)^2 entries
  float bil_sw2[81];          // the same times log2(e) (exponent for exp2)
  float bil_c2;               // log2(e) / (2 sigma_r^2)
  float bil_k;                // sqrt(bil_c2): the range term is (k zn - k z)^2
  float thr3sr32;             // (float)(3 sigma_r)
  // normals and association variants
  int normal_mode;            // KF_NORMALS_CROSS | KF_NORMALS_INTEGRAL
  float ii_a, ii_b;           // window half-size a + b z at level 0
  float ii_delta;             // relative depth change of an edge
  int ii_rmax;                // cap on the half-size
  int shoot_w;                // normal-shooting window half-size (0: projective)
};

struct PairInput {
  double prior_R[9];
  double init[16];
  double lambda;
  int has_prior;
  int pad_;
};

struct PairOutput {
  double pose[16];
  kf_result res;
};

// ---- checked builds (-DKF_CHECKED): guarded accesses record the first
// violation (code and two values) in a device fault word and are skipped;
// the host reports it as KF_ERR_INTERNAL. Unchecked builds compile the guard
// away and the access runs unconditionally.
#ifdef KF_CHECKED
__device__ void kf_fault(int code, long long a, long long b);
#define KF_GUARD(cond, code, a, b) \
  if (!(cond)) {                   \
    kf_fault((code), (a), (b));    \
  } else
#else
#define KF_GUARD(cond, code, a, b)
#endif
// host side of checked builds: copies and clears the fault word (0 = none)
void checked_fault(long long out[3]);

// ---- storage-type helpers -------------------------------------------------
template <class T> struct Store;
template <> struct Store<float> {
  static __device__ __forceinline__ float ld(const float* p, int i) { return __ldg(p + i); }
  static __device__ __forceinline__ void st(float* p, int i, float v) { p[i] = v; }
};
template <> struct Store<__half> {
  static __device__ __forceinline__ float ld(const __half* p, int i) { return __half2float(p[i]); }
  static __device__ __forceinline__ void st(__half* p, int i, float v) { p[i] = __float2half_rn(v); }
};

}  // namespace kf

// ---- launchers implemented in the .cu files ---------------------------------
namespace kf {
// Frames of a batch pulled from page-locked host memory into device buffers
// by one kernel (16-byte loads, several in flight per thread), instead of
// one copy per frame issued by the host.
struct FrameCopyList {
  const float* src[kDescListMax];
  float* dst[kDescListMax];
  int count[kDescListMax];  // floats
  int n;
};
cudaError_t launch_copy_frames(const FrameCopyList& list, int max_count, cudaStream_t s);
cudaError_t launch_frontend(const DescList& list, int max_w, int max_h, int levels,
                            const KParams& P, cudaStream_t s);
// integral-image normals of every level of the listed frames (after the
// front end): replaces the frame normals and drops vertices without one
cudaError_t launch_integral_normals(const DescList& list, int max_w, int max_h, int levels,
                                    const KParams& P, cudaStream_t s);
cudaError_t launch_model_prep(const PairDesc* d_desc, const float* V, const float* N, int w,
                              int h, int levels, const int* mw, const int* mh, int precision,
                              const LevelMaps* host_levels, cudaStream_t s);
// grid sizes (one wave) of the per-stage and the scheduled ICP kernels
void icp_grids(const KParams& P, int* g_assoc, int* g_reduce, int* g_sched);
cudaError_t launch_icp_init(const PairDesc* const* descs, const PairInput* in, int n, int* list,
                            const KParams& P, cudaStream_t s);
// mode 0: an iteration; 1: inspection (per-pixel outputs, no window);
// 2: inspection of the sums (the band and window set by launch_debug_setup)
cudaError_t launch_assoc_hist(const PairDesc* const* descs, const int* list, int cap, int grid,
                              int level, int mode, const KParams& P, cudaStream_t s);
// in_list: the pairs to reduce; out_list: where the launch's last block writes
// the next launch's active list (level next_level; -1: none)
cudaError_t launch_reduce_solve(const PairDesc* const* descs, int n, const int* in_list,
                                int* out_list, int cap, unsigned* launch_counter, int grid,
                                int level, int next_level, int mode, const KParams& P,
                                cudaStream_t s);
// the whole ICP of a batch in one persistent launch; queue: kQHeaderWords
// header words then (qmask + 1) slots, zeroed; a block whose wait for its
// next task exceeds wait_limit_ns sets queue[kQErr] and returns
constexpr unsigned long long kSchedWaitLimitNs = 2000000000ull;  // 2 s
cudaError_t launch_icp_sched(const PairDesc* const* descs, const PairInput* in, PairOutput* out,
                             int n, unsigned* queue, unsigned qmask, int grid,
                             unsigned long long wait_limit_ns, const KParams& P, cudaStream_t s);
cudaError_t launch_icp_finish(const PairDesc* const* descs, PairOutput* out, int n,
                              const KParams& P, cudaStream_t s);
// inspection set-up of one pair: pose, level, band [klo, khi] and window
// [w0, w1) (w0 = -1: none) with its hit flag
cudaError_t launch_debug_setup(const PairDesc* const* d_self, const double* d_pose, int level,
                               int klo, int khi, int w0, int w1, int hit, int* list,
                               const KParams& P, cudaStream_t s);
}  // namespace kf
