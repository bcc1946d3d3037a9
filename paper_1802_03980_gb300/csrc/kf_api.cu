// C ABI and tracker runtime: device buffers, per-pair descriptors, launch
// plans and the CUDA graph of the alignment loop.
#include <cuda_fp16.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "kf_internal.cuh"

using namespace kf;

namespace {

struct Plan {
  std::vector<kf_tracker*> list;
  std::vector<unsigned long long> uids;
  std::vector<unsigned> versions;
  int n = 0;
  const PairDesc** d_descs = nullptr;
  int* d_list = nullptr;                 // active work list (list_ints(n) ints)
  unsigned* d_launch_counter = nullptr;  // arrival counter of the reduction launches
  PairInput* d_in = nullptr;
  PairOutput* d_out = nullptr;           // outputs, then (at out_pad) the queue
  PairInput* h_in = nullptr;
  PairOutput* h_out = nullptr;           // outputs and the queue header's first words
  size_t out_pad = 0;                    // output bytes rounded up to 256
  size_t queue_bytes = 0;                // queue header + slots
  unsigned qmask = 0;                    // slots - 1 (a power of two)
  int grid = 0;                          // blocks of the scheduled launch
  bool sched = false;                    // one persistent launch (else per-iteration launches)
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  bool profiled = false;
  std::vector<cudaEvent_t> ev;   // profiled plans: start, then one per launch
  std::vector<int> ev_kind;      // 0 association, 1 reduction (for ev[i] -> ev[i+1])
  std::vector<long long> pair_px;  // [n * levels] frame pixels per device pair and level
  // device pair k is the caller's pair order[k]: the largest level-0 frames
  // first (ties in the caller's order), so the pairs with the longest stages
  // are seeded, and start their chains of stages, first
  std::vector<int> order;
};

void plan_free(Plan* pl) {
  if (!pl) return;
  for (cudaEvent_t e : pl->ev) cudaEventDestroy(e);
  if (pl->exec) cudaGraphExecDestroy(pl->exec);
  if (pl->graph) cudaGraphDestroy(pl->graph);
  cudaFree(pl->d_descs);
  cudaFree(pl->d_list);
  cudaFree(pl->d_launch_counter);
  cudaFree(pl->d_in);
  cudaFree(pl->d_out);
  cudaFreeHost(pl->h_in);
  cudaFreeHost(pl->h_out);
  delete pl;
}

}  // namespace

struct kf_tracker {
  unsigned long long uid = 0;     // unique per tracker; cached plans check it
  kf_params p;
  KParams kp;
  int max_w = 0, max_h = 0, device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  size_t elem = 4;
  std::vector<void*> allocs;
  float* d_depth_raw = nullptr;
  float* d_model_stage = nullptr;   // 2 x max_w x max_h x 3 floats, host model uploads
  float* d_frame_stage = nullptr;   // frames of a batch moved by the copy engine
  size_t frame_stage_bytes = 0;
  PairDesc h_desc;
  PairDesc* d_desc = nullptr;
  const PairDesc** d_self = nullptr;
  PairState* d_state = nullptr;
  int* d_dbg_list = nullptr;
  unsigned* d_dbg_counter = nullptr;
  double* d_dbg_pose = nullptr;
  int max_items = 0;
  int grid_assoc = 0, grid_reduce = 0, grid_sched = 0;
  bool has_frame = false, has_model = false;
  unsigned geom_version = 0;
  Plan* plan1 = nullptr;
  Plan* planN = nullptr;
  bool profiling = false;
  kf_profile prof = {};
  cudaEvent_t fe_ev[2] = {nullptr, nullptr};
  std::string err;
};

namespace {

kf_status fail(kf_tracker* t, kf_status s, const char* msg) {
  if (t) t->err = msg;
  return s;
}

kf_status cuda_fail(kf_tracker* t, cudaError_t e, const char* where) {
  if (t) t->err = std::string(where) + ": " + cudaGetErrorString(e);
  return e == cudaErrorMemoryAllocation ? KF_ERR_OOM : KF_ERR_CUDA;
}

#define KF_CK(t, expr)                                  \
  do {                                                  \
    cudaError_t e_ = (expr);                            \
    if (e_ != cudaSuccess) return cuda_fail(t, e_, #expr); \
  } while (0)

bool params_valid(const kf_params* p, std::string& why) {
  if (p->levels < 1 || p->levels > KF_MAX_LEVELS) { why = "levels must be 1..4"; return false; }
  for (int l = 0; l < p->levels; ++l)
    if (p->max_iters[l] < 1 || p->max_iters[l] > 1000) { why = "max_iters must be 1..1000"; return false; }
  if (p->hist_bins < 1 || p->hist_bins > kMaxBins) { why = "hist_bins must be 1..4096"; return false; }
  if (!(p->d_max > 0) || !std::isfinite(p->d_max)) { why = "d_max must be > 0"; return false; }
  if (!(p->band_kappa >= 0) || !std::isfinite(p->band_kappa)) { why = "band_kappa must be >= 0"; return false; }
  if (p->conv_window < 1 || p->conv_window > kMaxWindow) { why = "conv_window must be 1..8"; return false; }
  if (p->lambda_mode < 0 || p->lambda_mode > 4) { why = "lambda_mode must be 0..4"; return false; }
  if (p->n_min < 1) { why = "n_min must be >= 1"; return false; }
  if (p->precision != KF_FP32 && p->precision != KF_FP16) { why = "precision must be KF_FP32 or KF_FP16"; return false; }
  if (p->bilateral_radius < 0 || p->bilateral_radius > 4) { why = "bilateral_radius must be 0..4"; return false; }
  if (!(p->bilateral_sigma_s > 0) || !(p->bilateral_sigma_r > 0)) { why = "bilateral sigmas must be > 0"; return false; }
  if (std::isnan(p->cos_angle_min)) { why = "cos_angle_min is NaN"; return false; }
  if (p->normal_mode != KF_NORMALS_CROSS && p->normal_mode != KF_NORMALS_INTEGRAL) {
    why = "normal_mode must be KF_NORMALS_CROSS or KF_NORMALS_INTEGRAL";
    return false;
  }
  if (p->normal_mode == KF_NORMALS_INTEGRAL) {
    if (!(p->ii_radius_a >= 0) || !(p->ii_radius_b >= 0) || !std::isfinite(p->ii_radius_a) ||
        !std::isfinite(p->ii_radius_b)) { why = "ii_radius_a and ii_radius_b must be >= 0"; return false; }
    if (!(p->ii_depth_change > 0) || !std::isfinite(p->ii_depth_change)) { why = "ii_depth_change must be > 0"; return false; }
    if (p->ii_radius_max < 1 || p->ii_radius_max > 15) { why = "ii_radius_max must be 1..15"; return false; }
  }
  if (p->shoot_radius < 0 || p->shoot_radius > 4) { why = "shoot_radius must be 0..4"; return false; }
  return true;
}

KParams make_kparams(const kf_params* p) {
  KParams k;
  memset(&k, 0, sizeof(k));
  k.levels = p->levels;
  for (int l = 0; l < KF_MAX_LEVELS; ++l) k.caps[l] = l < p->levels ? p->max_iters[l] : 0;
  k.bins = p->hist_bins;
  k.d_max32 = (float)p->d_max;
  k.scale32 = (float)((double)p->hist_bins / p->d_max);
  k.kappa = p->band_kappa;
  k.cos_min32 = (float)p->cos_angle_min;
  k.use_angle = p->cos_angle_min > -1.0;
  k.conv_window = p->conv_window;
  k.lambda_mode = p->lambda_mode;
  k.n_min = p->n_min;
  k.flags = p->flags;
  k.precision = p->precision;
  // a band-edge window can only hit when the band starts at bin 0
  k.split_ok = !(p->flags & KF_USE_FILTER) || p->band_kappa >= 1.0;
  k.win_same_below = KF_WIN_SAME_BELOW;
  k.win_same_above = KF_WIN_SAME_ABOVE;
  k.win_next_below = KF_WIN_NEXT_BELOW;
  k.win_next_above = KF_WIN_NEXT_ABOVE;
  k.bil_radius = p->bilateral_radius;
  k.bil_inv2sr2 = (float)(1.0 / (2.0 * p->bilateral_sigma_r * p->bilateral_sigma_r));
  const int r = p->bilateral_radius, wd = 2 * r + 1;
  for (int dy = -r; dy <= r; ++dy)
    for (int dx = -r; dx <= r; ++dx)
      k.bil_sw[(dy + r) * wd + (dx + r)] =
          (float)(-(double)(dx * dx + dy * dy) / (2.0 * p->bilateral_sigma_s * p->bilateral_sigma_s));
  const double log2e = 1.4426950408889634;
  for (int i = 0; i < wd * wd; ++i) {
    const int dy = i / wd - r, dx = i % wd - r;
    k.bil_sw2[i] = (float)(-(double)(dx * dx + dy * dy) * log2e /
                           (2.0 * p->bilateral_sigma_s * p->bilateral_sigma_s));
  }
  k.bil_c2 = (float)(log2e / (2.0 * p->bilateral_sigma_r * p->bilateral_sigma_r));
  k.bil_k = (float)std::sqrt(log2e / (2.0 * p->bilateral_sigma_r * p->bilateral_sigma_r));
  k.thr3sr32 = (float)(3.0 * p->bilateral_sigma_r);
  k.normal_mode = p->normal_mode;
  k.ii_a = (float)p->ii_radius_a;
  k.ii_b = (float)p->ii_radius_b;
  k.ii_delta = (float)p->ii_depth_change;
  k.ii_rmax = p->ii_radius_max;
  k.shoot_w = p->shoot_radius;
  return k;
}

bool same_params(const kf_params& a, const kf_params& b) {
  if (a.levels != b.levels || a.hist_bins != b.hist_bins || a.d_max != b.d_max ||
      a.band_kappa != b.band_kappa || a.cos_angle_min != b.cos_angle_min ||
      a.conv_window != b.conv_window || a.lambda_mode != b.lambda_mode ||
      a.lambda_c != b.lambda_c || a.n_min != b.n_min || a.precision != b.precision ||
      a.flags != b.flags || a.bilateral_sigma_s != b.bilateral_sigma_s ||
      a.bilateral_sigma_r != b.bilateral_sigma_r || a.bilateral_radius != b.bilateral_radius ||
      a.normal_mode != b.normal_mode || a.shoot_radius != b.shoot_radius)
    return false;
  if (a.normal_mode == KF_NORMALS_INTEGRAL &&
      (a.ii_radius_a != b.ii_radius_a || a.ii_radius_b != b.ii_radius_b ||
       a.ii_depth_change != b.ii_depth_change || a.ii_radius_max != b.ii_radius_max))
    return false;
  for (int l = 0; l < a.levels; ++l)
    if (a.max_iters[l] != b.max_iters[l]) return false;
  return true;
}

template <class T>
cudaError_t tmalloc(kf_tracker* t, T** p, size_t bytes) {
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, bytes);
  if (e == cudaSuccess) {
    t->allocs.push_back(q);
    *p = static_cast<T*>(q);
  }
  return e;
}

bool intr_valid(const kf_intrinsics* K, int levels, int max_w, int max_h, std::string& why) {
  if (!K) { why = "null intrinsics"; return false; }
  if (K->width < 1 || K->height < 1 || K->width > max_w || K->height > max_h) {
    why = "image size outside 1..max size of the tracker";
    return false;
  }
  if ((K->width >> (levels - 1)) < 2 || (K->height >> (levels - 1)) < 2) {
    why = "image too small for the number of pyramid levels";
    return false;
  }
  if (!(K->fx > 0) || !(K->fy > 0) || !std::isfinite(K->cx) || !std::isfinite(K->cy) ||
      !std::isfinite(K->fx) || !std::isfinite(K->fy)) {
    why = "intrinsics must be finite with fx, fy > 0";
    return false;
  }
  return true;
}

// Frame level l: f / 2^l, c_{l+1} = (c_l - 0.5) / 2 (2x2 block averaging);
// returns true if the level geometry changed.
bool set_frame_levels(kf_tracker* t, const kf_intrinsics* K) {
  bool dims_changed = false;
  double fx = K->fx, fy = K->fy, cx = K->cx, cy = K->cy;
  int w = K->width, h = K->height;
  if (t->h_desc.iw != w || t->h_desc.ih != h) dims_changed = true;
  t->h_desc.iw = w;
  t->h_desc.ih = h;
  for (int l = 0; l < t->p.levels; ++l) {
    if (l > 0) {
      w /= 2;
      h /= 2;
      fx /= 2;
      fy /= 2;
      cx = (cx - 0.5) / 2;
      cy = (cy - 0.5) / 2;
    }
    LevelMaps& L = t->h_desc.lv[l];
    L.fw = w;
    L.fh = h;
    L.fps = frame_plane_stride(w, h);
    L.ffx = (float)fx;
    L.ffy = (float)fy;
    L.fcx = (float)cx;
    L.fcy = (float)cy;
  }
  return dims_changed;
}

kf_status upload_desc(kf_tracker* t, cudaStream_t s) {
  KF_CK(t, cudaMemcpyAsync(t->d_desc, &t->h_desc, sizeof(PairDesc), cudaMemcpyHostToDevice, s));
  return KF_OK;
}

kf_status copy_in(kf_tracker* t, void* dst, const void* src, size_t bytes, int is_dev,
                  cudaStream_t s) {
  KF_CK(t, cudaMemcpyAsync(dst, src, bytes, is_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
  return KF_OK;
}

// The tracker's staging buffer for frames the copy engine moves, grown on
// demand (a grow first waits for the stream: a queued front end may still
// read the old buffer).
kf_status frame_stage(kf_tracker* t, size_t bytes) {
  if (t->frame_stage_bytes >= bytes) return KF_OK;
  if (t->d_frame_stage) {
    KF_CK(t, cudaStreamSynchronize(t->stream));
    auto it = std::find(t->allocs.begin(), t->allocs.end(), static_cast<void*>(t->d_frame_stage));
    if (it != t->allocs.end()) t->allocs.erase(it);
    cudaFree(t->d_frame_stage);
    t->d_frame_stage = nullptr;
    t->frame_stage_bytes = 0;
  }
  KF_CK(t, tmalloc(t, &t->d_frame_stage, bytes));
  t->frame_stage_bytes = bytes;
  return KF_OK;
}

kf_status build_plan(kf_tracker* const* trk, int n, Plan** slot) {
  kf_tracker* t0 = trk[0];
  plan_free(*slot);
  *slot = nullptr;
  Plan* pl = new Plan();
  pl->n = n;
  pl->list.assign(trk, trk + n);
  for (int i = 0; i < n; ++i) {
    pl->versions.push_back(trk[i]->geom_version);
    pl->uids.push_back(trk[i]->uid);
  }
  pl->order.resize(n);
  for (int i = 0; i < n; ++i) pl->order[i] = i;
  auto px0 = [&](int i) { return (long long)trk[i]->h_desc.lv[0].fw * trk[i]->h_desc.lv[0].fh; };
  std::stable_sort(pl->order.begin(), pl->order.end(), [&](int a, int b) { return px0(a) > px0(b); });
  std::vector<const PairDesc*> descs(n);
  for (int k = 0; k < n; ++k) descs[k] = trk[pl->order[k]]->d_desc;
  const int L = t0->p.levels;
  cudaStream_t s = t0->stream;
  cudaError_t e = cudaSuccess;
  auto ck = [&](cudaError_t x) { if (e == cudaSuccess) e = x; };
  ck(cudaMalloc(&pl->d_descs, sizeof(PairDesc*) * n));
  ck(cudaMalloc(&pl->d_list, sizeof(int) * list_ints(n)));
  ck(cudaMalloc(&pl->d_launch_counter, sizeof(unsigned)));
  // scheduled path: every pair has at most one stage queued, so the ring
  // holds each pair's largest level plus one exit word per block
  const KParams& P0 = t0->kp;
  long long ring = (long long)t0->grid_sched + 64;
  int max_items = 0;
  for (int i = 0; i < n; ++i) {
    int m = 0;
    for (int l = 0; l < L; ++l) {
      const long long px = (long long)trk[i]->h_desc.lv[l].fw * trk[i]->h_desc.lv[l].fh;
      m = std::max(m, (int)((px + level_chunk(l) - 1) / level_chunk(l)));
    }
    ring += m;
    max_items = std::max(max_items, m);
  }
  unsigned slots = 1024;
  while ((long long)slots < ring) slots <<= 1;
  // no stage has more tasks than the batch has items at its widest level, so
  // a small batch takes only that many blocks and leaves the other SMs to
  // kernels of other streams (the next frames' front end); results do not
  // depend on the grid
  long long widest = 0;
  for (int i = 0; i < n; ++i) {
    int m = 0;
    for (int l = 0; l < L; ++l) {
      const long long px = (long long)trk[i]->h_desc.lv[l].fw * trk[i]->h_desc.lv[l].fh;
      m = std::max(m, (int)((px + level_chunk(l) - 1) / level_chunk(l)));
    }
    widest += m;
  }
  pl->grid = (int)std::max(1LL, std::min((long long)t0->grid_sched, widest));
  pl->sched = !(P0.flags & KF_LAUNCH_PER_ITERATION) && n <= kMaxSchedPairs &&
              max_items <= kMaxItemsPerLevel;
  pl->qmask = slots - 1;
  pl->out_pad = (sizeof(PairOutput) * n + 255) / 256 * 256;
  pl->queue_bytes = sizeof(unsigned) * kQHeaderWords + sizeof(unsigned long long) * slots;
  ck(cudaMalloc(&pl->d_in, sizeof(PairInput) * n));
  ck(cudaMalloc(&pl->d_out, pl->out_pad + pl->queue_bytes));
  ck(cudaMallocHost(&pl->h_in, sizeof(PairInput) * n));
  ck(cudaMallocHost(&pl->h_out, pl->out_pad + 512));
  if (e == cudaSuccess) {
    ck(cudaMemcpyAsync(pl->d_descs, descs.data(), sizeof(PairDesc*) * n, cudaMemcpyHostToDevice, s));
    ck(cudaMemsetAsync(pl->d_launch_counter, 0, sizeof(unsigned), s));
    ck(cudaStreamSynchronize(s));
  }
  if (e == cudaSuccess) {
    pl->profiled = t0->profiling;
    if (pl->profiled) {
      int total = 0;
      for (int l = 0; l < L; ++l) total += t0->kp.caps[l];
      pl->ev.resize(pl->sched ? 3 : 2 * total + 3, nullptr);
      for (auto& ev : pl->ev) ck(cudaEventCreate(&ev));
    }
    for (int k = 0; k < n; ++k)
      for (int l = 0; l < L; ++l) {
        const kf_tracker* t = trk[pl->order[k]];
        pl->pair_px.push_back((long long)t->h_desc.lv[l].fw * t->h_desc.lv[l].fh);
      }
    if (e == cudaSuccess) ck(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    if (e == cudaSuccess) {
      const KParams& P = t0->kp;
      size_t evi = 0;
      auto mark = [&](int kind) -> cudaError_t {
        if (!pl->profiled) return cudaSuccess;
        pl->ev_kind.push_back(kind);
        return cudaEventRecordWithFlags(pl->ev[evi++], s, cudaEventRecordExternal);
      };
      cudaError_t le = mark(-1);
      unsigned* queue = reinterpret_cast<unsigned*>(reinterpret_cast<char*>(pl->d_out) + pl->out_pad);
      if (pl->sched) {
        // the whole loop in one persistent launch after zeroing its queue
        if (le == cudaSuccess) le = cudaMemsetAsync(queue, 0, pl->queue_bytes, s);
        if (le == cudaSuccess) le = mark(3);
        if (le == cudaSuccess)
          le = launch_icp_sched(pl->d_descs, pl->d_in, pl->d_out, n, queue, pl->qmask,
                                pl->grid, kSchedWaitLimitNs, P, s);
        if (le == cudaSuccess) le = mark(-1);
      }
      if (!pl->sched && le == cudaSuccess) le = launch_icp_init(pl->d_descs, pl->d_in, n, pl->d_list, P, s);
      for (int l = L - 1; l >= 0 && le == cudaSuccess && !pl->sched; --l)
        for (int it = 0; it < P.caps[l] && le == cudaSuccess; ++it) {
          // the level of the launch that follows this iteration's reduction
          const int next = it + 1 < P.caps[l] ? l : l - 1;
          // association pass, then the reduction pass for every active pair
          le = mark(0);
          if (le == cudaSuccess)
            le = launch_assoc_hist(pl->d_descs, pl->d_list, n, t0->grid_assoc, l, 0, P, s);
          if (le == cudaSuccess) le = mark(1);
          if (le == cudaSuccess)
            le = launch_reduce_solve(pl->d_descs, n, pl->d_list, pl->d_list, n,
                                     pl->d_launch_counter, t0->grid_reduce, l, next, 0, P, s);
        }
      if (!pl->sched) {
        if (le == cudaSuccess) le = mark(-1);
        if (le == cudaSuccess) le = launch_icp_finish(pl->d_descs, pl->d_out, n, P, s);
        if (le == cudaSuccess) le = mark(-1);
      }
      cudaGraph_t g = nullptr;
      cudaError_t ee = cudaStreamEndCapture(s, &g);
      ck(le);
      ck(ee);
      pl->graph = g;
      if (e == cudaSuccess) ck(cudaGraphInstantiate(&pl->exec, g, 0));
    }
  }
  if (e != cudaSuccess) {
    plan_free(pl);
    return cuda_fail(t0, e, "building the alignment plan");
  }
  *slot = pl;
  return KF_OK;
}

bool plan_current(const Plan* pl, kf_tracker* const* trk, int n) {
  if (!pl || pl->n != n || pl->profiled != trk[0]->profiling) return false;
  for (int i = 0; i < n; ++i)
    if (pl->list[i] != trk[i] || pl->uids[i] != trk[i]->uid ||
        pl->versions[i] != trk[i]->geom_version)
      return false;
  return true;
}

kf_status ensure_debug_buffers(kf_tracker* t) {
  if (t->h_desc.dbg_index) return KF_OK;
  const size_t px = (size_t)t->max_w * t->max_h;
  KF_CK(t, tmalloc(t, &t->h_desc.dbg_index, px * sizeof(int)));
  KF_CK(t, tmalloc(t, &t->h_desc.dbg_bin, px * sizeof(int)));
  return upload_desc(t, t->stream);
}

float half_bits_to_float(uint16_t b) {
  __half_raw r;
  r.x = b;
  return __half2float(__half(r));
}

// planes (x, y, z) of n elements of the map's storage type -> interleaved float
// planes of `stride` elements (x, y, z) -> n interleaved xyz floats
void planes_to_xyz(const std::vector<unsigned char>& buf, size_t n, size_t stride, size_t elem,
                   float* out) {
  for (size_t i = 0; i < n; ++i)
    for (int c = 0; c < 3; ++c) {
      const size_t k = c * stride + i;
      float v;
      if (elem == 4) {
        memcpy(&v, buf.data() + 4 * k, 4);
      } else {
        uint16_t b;
        memcpy(&b, buf.data() + 2 * k, 2);
        v = half_bits_to_float(b);
      }
      out[3 * i + c] = v;
    }
}

}  // namespace

extern "C" {

kf_status kf_default_params(kf_params* p) {
  if (!p) return KF_ERR_INVALID_ARG;
  memset(p, 0, sizeof(*p));
  p->levels = 3;
  p->max_iters[0] = 10;
  p->max_iters[1] = 5;
  p->max_iters[2] = 4;
  p->max_iters[3] = 4;
  p->hist_bins = 512;
  p->d_max = 0.16;
  p->band_kappa = 1.0;
  p->cos_angle_min = -2.0;
  p->conv_window = 3;
  p->lambda_mode = KF_LAMBDA_CONST;
  p->lambda_c = 5.0;
  p->n_min = 6;
  p->precision = KF_FP32;
  p->flags = KF_USE_PRIOR | KF_USE_FILTER | KF_USE_CONVERGENCE;
  p->bilateral_sigma_s = 4.0;
  p->bilateral_sigma_r = 0.03;
  p->bilateral_radius = 2;
  p->normal_mode = KF_NORMALS_CROSS;
  p->ii_radius_a = 2.0;
  p->ii_radius_b = 1.0;
  p->ii_depth_change = 0.02;
  p->ii_radius_max = 8;
  p->shoot_radius = 0;
  return KF_OK;
}

kf_status kf_track_create(const kf_params* p, int max_w, int max_h, void* cuda_stream,
                          kf_tracker** out) {
  if (!p || !out) return KF_ERR_INVALID_ARG;
  *out = nullptr;
  std::string why;
  if (!params_valid(p, why)) return KF_ERR_INVALID_ARG;
  if (max_w < 2 || max_h < 2 || max_w > 16384 || max_h > 16384) return KF_ERR_INVALID_ARG;
  if ((max_w >> (p->levels - 1)) < 2 || (max_h >> (p->levels - 1)) < 2) return KF_ERR_INVALID_ARG;
  kf_tracker* t = new (std::nothrow) kf_tracker();
  if (!t) return KF_ERR_OOM;
  static std::atomic<unsigned long long> next_uid{1};
  t->uid = next_uid.fetch_add(1);
  t->p = *p;
  t->kp = make_kparams(p);
  t->max_w = max_w;
  t->max_h = max_h;
  t->elem = p->precision == KF_FP16 ? 2 : 4;
  memset(&t->h_desc, 0, sizeof(PairDesc));
  cudaError_t e = cudaGetDevice(&t->device);
  auto bail = [&](cudaError_t err) {
    kf_status s = err == cudaErrorMemoryAllocation ? KF_ERR_OOM : KF_ERR_CUDA;
    kf_track_destroy(t);
    return s;
  };
  if (e != cudaSuccess) return bail(e);
  if (cuda_stream) {
    t->stream = static_cast<cudaStream_t>(cuda_stream);
  } else {
    e = cudaStreamCreateWithFlags(&t->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) return bail(e);
    t->own_stream = true;
  }
  // pixel buffers hold the largest level-0 plane rounded up, plus one
  // alignment unit: bulk copies round a range's end up to 16 bytes
  const size_t px0 = (size_t)frame_plane_stride(max_w, max_h) + kPlaneAlign;
  PairDesc& D = t->h_desc;
  D.levels = p->levels;
  if ((e = tmalloc(t, &t->d_depth_raw, px0 * sizeof(float))) != cudaSuccess) return bail(e);
  D.depth_raw = t->d_depth_raw;
  for (int l = 0; l < p->levels; ++l) {
    const size_t pl = (size_t)(max_w >> l) * (max_h >> l);
    const size_t fpl = (size_t)frame_plane_stride(max_w >> l, max_h >> l) + kPlaneAlign;
    LevelMaps& L = D.lv[l];
    if ((e = tmalloc(t, &L.fdepth, pl * sizeof(float))) != cudaSuccess) return bail(e);
    if ((e = tmalloc(t, &L.fV, 3 * fpl * t->elem)) != cudaSuccess) return bail(e);
    if ((e = tmalloc(t, &L.fN, 3 * fpl * t->elem)) != cudaSuccess) return bail(e);
    if ((e = tmalloc(t, &L.mV, 3 * pl * t->elem)) != cudaSuccess) return bail(e);
    if ((e = tmalloc(t, &L.mN, 3 * pl * t->elem)) != cudaSuccess) return bail(e);
  }
  t->max_items = (int)(((size_t)max_w * max_h + kChunk - 1) / kChunk);
  if ((e = tmalloc(t, &t->d_state, sizeof(PairState))) != cudaSuccess) return bail(e);
  if ((e = tmalloc(t, &D.hist, sizeof(unsigned) * p->hist_bins)) != cudaSuccess) return bail(e);
  if ((e = tmalloc(t, &D.partials, sizeof(float) * kPartialStride * t->max_items)) != cudaSuccess) return bail(e);
  D.partial_cap = t->max_items;
  D.px_cap = (int)px0;
  if ((e = tmalloc(t, &D.counters, sizeof(unsigned) * 2)) != cudaSuccess) return bail(e);
  if ((e = tmalloc(t, &D.recs, 2 * sizeof(float4) * (px0 + kChunk))) != cudaSuccess) return bail(e);
  if ((e = tmalloc(t, &D.wcount, sizeof(unsigned) * kBlockWarps * t->max_items)) != cudaSuccess)
    return bail(e);
  if ((e = tmalloc(t, &t->d_desc, sizeof(PairDesc))) != cudaSuccess) return bail(e);
  if ((e = tmalloc(t, &t->d_self, sizeof(PairDesc*))) != cudaSuccess) return bail(e);
  if ((e = tmalloc(t, &t->d_dbg_list, sizeof(int) * list_ints(1))) != cudaSuccess) return bail(e);
  if ((e = tmalloc(t, &t->d_dbg_counter, sizeof(unsigned))) != cudaSuccess) return bail(e);
  if ((e = cudaMemsetAsync(t->d_dbg_counter, 0, sizeof(unsigned), t->stream)) != cudaSuccess) return bail(e);
  icp_grids(t->kp, &t->grid_assoc, &t->grid_reduce, &t->grid_sched);
  if ((e = tmalloc(t, &t->d_dbg_pose, sizeof(double) * 16)) != cudaSuccess) return bail(e);
  D.st = t->d_state;
  if ((e = cudaMemsetAsync(t->d_state, 0, sizeof(PairState), t->stream)) != cudaSuccess) return bail(e);
  if ((e = cudaMemsetAsync(D.counters, 0, sizeof(unsigned) * 2, t->stream)) != cudaSuccess) return bail(e);
  if ((e = cudaMemcpyAsync(t->d_desc, &D, sizeof(PairDesc), cudaMemcpyHostToDevice, t->stream)) != cudaSuccess) return bail(e);
  const PairDesc* self = t->d_desc;
  if ((e = cudaMemcpyAsync(t->d_self, &self, sizeof(self), cudaMemcpyHostToDevice, t->stream)) != cudaSuccess) return bail(e);
  if ((e = cudaStreamSynchronize(t->stream)) != cudaSuccess) return bail(e);
  *out = t;
  return KF_OK;
}

void kf_track_destroy(kf_tracker* t) {
  if (!t) return;
  if (t->stream) cudaStreamSynchronize(t->stream);
  plan_free(t->plan1);
  plan_free(t->planN);
  for (cudaEvent_t e : t->fe_ev)
    if (e) cudaEventDestroy(e);
  for (void* q : t->allocs) cudaFree(q);
  if (t->own_stream && t->stream) cudaStreamDestroy(t->stream);
  delete t;
}

const char* kf_last_error(const kf_tracker* t) { return t ? t->err.c_str() : "null tracker"; }

kf_status kf_set_frame_batch(kf_tracker* const* trk, int n, const float* const* depth,
                             const kf_intrinsics* K, int is_device_ptr) {
  if (!trk || n < 1 || !depth || !K) return KF_ERR_INVALID_ARG;
  if (is_device_ptr != KF_FRAME_HOST && is_device_ptr != KF_FRAME_DEVICE &&
      is_device_ptr != KF_FRAME_HOST_COPY_ENGINE)
    return fail(trk[0], KF_ERR_INVALID_ARG, "is_device_ptr must be KF_FRAME_HOST, _DEVICE or _HOST_COPY_ENGINE");
  try {
    kf_tracker* t0 = trk[0];
    if (!t0) return KF_ERR_INVALID_ARG;
    cudaStream_t s = t0->stream;
    std::string why;
    for (int i = 0; i < n; ++i) {
      kf_tracker* t = trk[i];
      if (!t || !depth[i]) return fail(t0, KF_ERR_INVALID_ARG, "null tracker or depth");
      if (t->device != t0->device || !same_params(t->p, t0->p))
        return fail(t0, KF_ERR_INVALID_ARG, "batched trackers need one device and equal params");
      if (!intr_valid(&K[i], t->p.levels, t->max_w, t->max_h, why))
        return fail(t, KF_ERR_INVALID_ARG, why.c_str());
    }
    // where the front end reads each frame: device frames in place; with
    // KF_FRAME_HOST, host frames from the tracker's buffer, filled by one
    // gather kernel for the page-locked ones (the GPU pulls them over the
    // host link, no copy for the host to issue per frame) and by a copy each
    // for pageable ones; with KF_FRAME_HOST_COPY_ENGINE, from trk[0]'s
    // staging buffer
    std::vector<const float*> src(n);
    bool copied = false;  // a pageable host frame went through a copy
    FrameCopyList pull;
    pull.n = 0;
    int pull_max = 0;
    if (is_device_ptr == KF_FRAME_HOST_COPY_ENGINE) {
      // copies on the batch's stream into trk[0]'s staging buffer: the copy
      // engine moves page-locked frames without taking SMs, so the upload can
      // overlap kernels of other streams; frames that follow one another in
      // host memory move as one copy (a copy costs the host microseconds to
      // issue however small it is); a copy from pageable memory returns only
      // once the frame has been staged, so the caller may reuse it at once
      // either way (no query of the memory kind, no wait)
      size_t total = 0;
      for (int i = 0; i < n; ++i) total += (size_t)K[i].width * K[i].height;
      kf_status st = frame_stage(t0, total * sizeof(float));
      if (st != KF_OK) return st;
      size_t off = 0, run0 = 0;  // staging offset of frame i, of the current run
      int i0 = 0;                // first frame of the current run
      for (int i = 0; i < n; ++i) {
        const size_t cnt = (size_t)K[i].width * K[i].height;
        src[i] = t0->d_frame_stage + off;
        off += cnt;
        if (i + 1 == n || depth[i + 1] != depth[i] + cnt) {
          st = copy_in(t0, t0->d_frame_stage + run0, depth[i0], (off - run0) * sizeof(float), 0, s);
          if (st != KF_OK) return st;
          i0 = i + 1;
          run0 = off;
        }
      }
    }
    for (int i = 0; i < n; ++i) {
      kf_tracker* t = trk[i];
      if (is_device_ptr == KF_FRAME_HOST_COPY_ENGINE) {
        // src[i] set above
      } else if (is_device_ptr == KF_FRAME_HOST) {
        src[i] = depth[i];
        cudaPointerAttributes a;
        if (cudaPointerGetAttributes(&a, depth[i]) == cudaSuccess && a.type == cudaMemoryTypeHost &&
            a.devicePointer) {
          if (pull.n == kDescListMax) {
            KF_CK(t0, launch_copy_frames(pull, pull_max, s));
            pull.n = 0;
            pull_max = 0;
          }
          const int cnt = K[i].width * K[i].height;
          pull.src[pull.n] = static_cast<const float*>(a.devicePointer);
          pull.dst[pull.n] = t->d_depth_raw;
          pull.count[pull.n++] = cnt;
          pull_max = std::max(pull_max, cnt);
          src[i] = t->d_depth_raw;
        } else {
          (void)cudaGetLastError();  // clear a failed query: the frame is copied instead
          const size_t bytes = (size_t)K[i].width * K[i].height * sizeof(float);
          kf_status st = copy_in(t, t->d_depth_raw, depth[i], bytes, 0, s);
          if (st != KF_OK) return st;
          src[i] = t->d_depth_raw;
          copied = true;
        }
      } else {
        src[i] = depth[i];  // a device frame, read in place
      }
      PairDesc before = t->h_desc;
      if (set_frame_levels(t, &K[i])) ++t->geom_version;
      if (memcmp(&before, &t->h_desc, sizeof(PairDesc)) != 0 || !t->has_frame) {
        kf_status st = upload_desc(t, s);
        if (st != KF_OK) return st;
      }
    }
    KF_CK(t0, launch_copy_frames(pull, pull_max, s));
    const bool prof = t0->profiling;
    if (prof) KF_CK(t0, cudaEventRecord(t0->fe_ev[0], s));
    for (int c0 = 0; c0 < n; c0 += kDescListMax) {
      DescList list;
      list.n = std::min(kDescListMax, n - c0);
      int mw = 0, mh = 0;
      for (int i = 0; i < list.n; ++i) {
        list.d[i] = trk[c0 + i]->d_desc;
        list.depth[i] = src[c0 + i];
        mw = std::max(mw, K[c0 + i].width);
        mh = std::max(mh, K[c0 + i].height);
      }
      KF_CK(t0, launch_frontend(list, mw, mh, t0->p.levels, t0->kp, s));
      if (t0->kp.normal_mode == KF_NORMALS_INTEGRAL)
        KF_CK(t0, launch_integral_normals(list, mw, mh, t0->p.levels, t0->kp, s));
    }
    for (int i = 0; i < n; ++i) trk[i]->has_frame = true;
    if (prof) {
      KF_CK(t0, cudaEventRecord(t0->fe_ev[1], s));
      KF_CK(t0, cudaEventSynchronize(t0->fe_ev[1]));
      float ms = 0.f;
      KF_CK(t0, cudaEventElapsedTime(&ms, t0->fe_ev[0], t0->fe_ev[1]));
      t0->prof.frontend_ms += ms;
      t0->prof.frontend_calls += 1;
    }
    // pageable host frames may be reused as soon as the call returns
    if (copied) KF_CK(t0, cudaStreamSynchronize(s));
    return KF_OK;
  } catch (...) {
    return KF_ERR_INTERNAL;
  }
}

kf_status kf_set_frame(kf_tracker* t, const float* depth, const kf_intrinsics* K,
                       int is_device_ptr) {
  if (!t) return KF_ERR_INVALID_ARG;
  return kf_set_frame_batch(&t, 1, &depth, K, is_device_ptr);
}

kf_status kf_set_model(kf_tracker* t, const float* vertex, const float* normal,
                       const double model_pose[16], const kf_intrinsics* K, int is_device_ptr) {
  if (!t) return KF_ERR_INVALID_ARG;
  if (!vertex || !normal || !model_pose) return fail(t, KF_ERR_INVALID_ARG, "null model input");
  std::string why;
  if (!intr_valid(K, t->p.levels, t->max_w, t->max_h, why)) return fail(t, KF_ERR_INVALID_ARG, why.c_str());
  for (int i = 0; i < 16; ++i)
    if (!std::isfinite(model_pose[i])) return fail(t, KF_ERR_INVALID_ARG, "non-finite model pose");
  try {
    cudaStream_t s = t->stream;
    const size_t n3 = (size_t)K->width * K->height * 3;
    const float* V = vertex;
    const float* N = normal;
    if (!is_device_ptr) {
      if (!t->d_model_stage)
        KF_CK(t, tmalloc(t, &t->d_model_stage, 2 * sizeof(float) * 3 * (size_t)t->max_w * t->max_h));
      KF_CK(t, cudaMemcpyAsync(t->d_model_stage, vertex, n3 * sizeof(float), cudaMemcpyHostToDevice, s));
      KF_CK(t, cudaMemcpyAsync(t->d_model_stage + n3, normal, n3 * sizeof(float), cudaMemcpyHostToDevice, s));
      V = t->d_model_stage;
      N = t->d_model_stage + n3;
    }
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 4; ++j) t->h_desc.Tm[i * 4 + j] = model_pose[i * 4 + j];
    double fx = K->fx, fy = K->fy, cx = K->cx, cy = K->cy;
    int w = K->width, h = K->height;
    int mw[KF_MAX_LEVELS], mh[KF_MAX_LEVELS];
    for (int l = 0; l < t->p.levels; ++l) {
      if (l > 0) {  // model level l+1 = level l at even pixels: f / 2, c / 2
        w /= 2;
        h /= 2;
        fx /= 2;
        fy /= 2;
        cx /= 2;
        cy /= 2;
      }
      LevelMaps& L = t->h_desc.lv[l];
      L.mw = mw[l] = w;
      L.mh = mh[l] = h;
      L.mfx = (float)fx;
      L.mfy = (float)fy;
      L.mcx = (float)cx;
      L.mcy = (float)cy;
    }
    kf_status st = upload_desc(t, s);
    if (st != KF_OK) return st;
    KF_CK(t, launch_model_prep(t->d_desc, V, N, K->width, K->height, t->p.levels, mw, mh,
                               t->p.precision, nullptr, s));
    if (!is_device_ptr) KF_CK(t, cudaStreamSynchronize(s));
    t->has_model = true;
    return KF_OK;
  } catch (...) {
    return KF_ERR_INTERNAL;
  }
}

kf_status kf_align_batch(kf_tracker* const* trk, int n, const double* prior_R,
                         const double* init_pose, const double* lambda, double* out_pose,
                         kf_result* out) {
  if (!trk || n < 1 || !init_pose || !lambda || !out_pose) return KF_ERR_INVALID_ARG;
  try {
    kf_tracker* t0 = trk[0];
    if (!t0) return KF_ERR_INVALID_ARG;
    for (int i = 0; i < n; ++i) {
      kf_tracker* t = trk[i];
      if (!t) return fail(t0, KF_ERR_INVALID_ARG, "null tracker");
      if (t->device != t0->device || !same_params(t->p, t0->p))
        return fail(t0, KF_ERR_INVALID_ARG, "batched trackers need one device and equal params");
      if (!t->has_frame) return fail(t, KF_ERR_NO_FRAME, "kf_set_frame has not been called");
      if (!t->has_model) return fail(t, KF_ERR_NO_MODEL, "kf_set_model has not been called");
      for (int k = 0; k < 16; ++k)
        if (!std::isfinite(init_pose[16 * i + k])) return fail(t, KF_ERR_INVALID_ARG, "non-finite init pose");
      if (prior_R)
        for (int k = 0; k < 9; ++k)
          if (!std::isfinite(prior_R[9 * i + k])) return fail(t, KF_ERR_INVALID_ARG, "non-finite prior");
      if (std::isnan(lambda[i])) return fail(t, KF_ERR_INVALID_ARG, "NaN lambda");
    }
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < i; ++j)
        if (trk[i] == trk[j]) return fail(t0, KF_ERR_INVALID_ARG, "a tracker appears twice in the batch");
    Plan** slot = n == 1 ? &t0->plan1 : &t0->planN;
    if (!plan_current(*slot, trk, n)) {
      kf_status st = build_plan(trk, n, slot);
      if (st != KF_OK) return st;
    }
    Plan* pl = *slot;
    cudaStream_t s = t0->stream;
    for (int k = 0; k < n; ++k) {  // device pair k: the caller's pair i
      const int i = pl->order[k];
      PairInput& in = pl->h_in[k];
      memset(&in, 0, sizeof(in));
      if (prior_R) memcpy(in.prior_R, prior_R + 9 * i, sizeof(double) * 9);
      memcpy(in.init, init_pose + 16 * i, sizeof(double) * 16);
      in.lambda = lambda[i] < 0 ? t0->p.lambda_c : lambda[i];
      in.has_prior = prior_R ? 1 : 0;
    }
    KF_CK(t0, cudaMemcpyAsync(pl->d_in, pl->h_in, sizeof(PairInput) * n, cudaMemcpyHostToDevice, s));
    KF_CK(t0, cudaGraphLaunch(pl->exec, s));
    // outputs and, after them, the scheduled launch's queue header (error word)
    KF_CK(t0, cudaMemcpyAsync(pl->h_out, pl->d_out, pl->out_pad + 512, cudaMemcpyDeviceToHost, s));
    KF_CK(t0, cudaStreamSynchronize(s));
    if (pl->sched) {
      const unsigned* qh = reinterpret_cast<const unsigned*>(reinterpret_cast<const char*>(pl->h_out) + pl->out_pad);
      if (qh[kQErr] != 0u)
        return fail(t0, KF_ERR_TIMEOUT, "a bounded device wait of the scheduled ICP launch ran out");
    }
#ifdef KF_CHECKED
    {
      long long f[3];
      checked_fault(f);
      if (f[0] != 0) {
        char msg[160];
        snprintf(msg, sizeof msg, "checked build: guard %lld failed (%lld, %lld)", f[0], f[1], f[2]);
        return fail(t0, KF_ERR_INTERNAL, msg);
      }
    }
#endif
    if (pl->profiled) {
      kf_profile& pr = t0->prof;
      // per-iteration plans: ev[0] start, then (mark0, mark1) per iteration, then
      // two finish marks; scheduled plans: start, the launch, end;
      // ev_kind[i] says what runs between ev[i] and ev[i+1]
      for (size_t i = 0; i + 1 < pl->ev.size(); ++i) {
        float ms = 0.f;
        KF_CK(t0, cudaEventElapsedTime(&ms, pl->ev[i], pl->ev[i + 1]));
        if (pl->ev_kind[i] == 0) {
          pr.assoc_ms += ms;
          pr.assoc_launches += 1;
        } else if (pl->ev_kind[i] == 1) {
          pr.reduce_ms += ms;
          pr.reduce_launches += 1;
        } else if (pl->ev_kind[i] == 2) {
          pr.fused_ms += ms;
          pr.fused_launches += 1;
        } else if (pl->ev_kind[i] == 3) {
          pr.sched_ms += ms;
          pr.sched_launches += 1;
        }
      }
      float all = 0.f;
      KF_CK(t0, cudaEventElapsedTime(&all, pl->ev.front(), pl->ev.back()));
      pr.align_ms += all;
      pr.graph_launches += 1;
      pr.alignments += n;
      const int L = t0->p.levels;
      for (int i = 0; i < n; ++i)
        for (int l = 0; l < L; ++l) pr.pixel_iters += pl->pair_px[i * L + l] * pl->h_out[i].res.iters[l];
    }
    // most severe status: the lowest error if any, else the warning, else OK
    int worst = KF_OK;
    for (int k = 0; k < n; ++k) {
      const int i = pl->order[k];
      memcpy(out_pose + 16 * i, pl->h_out[k].pose, sizeof(double) * 16);
      if (out) out[i] = pl->h_out[k].res;
      const int st = pl->h_out[k].res.status;
      if (st < 0 && (worst >= 0 || st < worst)) worst = st;
      else if (st == KF_NOT_CONVERGED && worst == KF_OK) worst = st;
    }
    return (kf_status)worst;
  } catch (...) {
    return KF_ERR_INTERNAL;
  }
}

kf_status kf_align(kf_tracker* t, const double prior_R[9], const double init_pose[16],
                   double lambda, double out_pose[16], kf_result* out) {
  if (!t) return KF_ERR_INVALID_ARG;
  return kf_align_batch(&t, 1, prior_R, init_pose, &lambda, out_pose, out);
}

kf_status kf_debug_frame_level(kf_tracker* t, int level, float* depth, float* vertex,
                               float* normal, int dims[2]) {
  if (!t || level < 0 || level >= t->p.levels) return KF_ERR_INVALID_ARG;
  if (!t->has_frame) return fail(t, KF_ERR_NO_FRAME, "no frame");
  try {
    const LevelMaps& L = t->h_desc.lv[level];
    const size_t n = (size_t)L.fw * L.fh;
    KF_CK(t, cudaStreamSynchronize(t->stream));
    if (dims) {
      dims[0] = L.fw;
      dims[1] = L.fh;
    }
    if (depth) KF_CK(t, cudaMemcpy(depth, L.fdepth, n * sizeof(float), cudaMemcpyDeviceToHost));
    std::vector<unsigned char> buf(3 * (size_t)L.fps * t->elem);
    if (vertex) {
      KF_CK(t, cudaMemcpy(buf.data(), L.fV, buf.size(), cudaMemcpyDeviceToHost));
      planes_to_xyz(buf, n, L.fps, t->elem, vertex);
    }
    if (normal) {
      KF_CK(t, cudaMemcpy(buf.data(), L.fN, buf.size(), cudaMemcpyDeviceToHost));
      planes_to_xyz(buf, n, L.fps, t->elem, normal);
    }
    return KF_OK;
  } catch (...) {
    return KF_ERR_INTERNAL;
  }
}

kf_status kf_debug_model_level(kf_tracker* t, int level, float* vertex, float* normal, int dims[2]) {
  if (!t || level < 0 || level >= t->p.levels) return KF_ERR_INVALID_ARG;
  if (!t->has_model) return fail(t, KF_ERR_NO_MODEL, "no model");
  try {
    const LevelMaps& L = t->h_desc.lv[level];
    const size_t n = (size_t)L.mw * L.mh;
    KF_CK(t, cudaStreamSynchronize(t->stream));
    if (dims) {
      dims[0] = L.mw;
      dims[1] = L.mh;
    }
    std::vector<unsigned char> buf(3 * n * t->elem);
    if (vertex) {
      KF_CK(t, cudaMemcpy(buf.data(), L.mV, buf.size(), cudaMemcpyDeviceToHost));
      planes_to_xyz(buf, n, n, t->elem, vertex);
    }
    if (normal) {
      KF_CK(t, cudaMemcpy(buf.data(), L.mN, buf.size(), cudaMemcpyDeviceToHost));
      planes_to_xyz(buf, n, n, t->elem, normal);
    }
    return KF_OK;
  } catch (...) {
    return KF_ERR_INTERNAL;
  }
}

static kf_status debug_prepare(kf_tracker* t, int level, const double pose[16], int klo, int khi,
                               int w0, int w1, int hit) {
  if (!t || level < 0 || level >= t->p.levels || !pose) return KF_ERR_INVALID_ARG;
  if (!t->has_frame) return fail(t, KF_ERR_NO_FRAME, "no frame");
  if (!t->has_model) return fail(t, KF_ERR_NO_MODEL, "no model");
  kf_status st = ensure_debug_buffers(t);
  if (st != KF_OK) return st;
  double p12[12];
  for (int i = 0; i < 12; ++i) p12[i] = pose[i];
  cudaStream_t s = t->stream;
  KF_CK(t, cudaMemcpyAsync(t->d_dbg_pose, p12, sizeof(p12), cudaMemcpyHostToDevice, s));
  KF_CK(t, launch_debug_setup(t->d_self, t->d_dbg_pose, level, klo, khi, w0, w1, hit,
                              t->d_dbg_list, t->kp, s));
  return KF_OK;
}

kf_status kf_debug_associate(kf_tracker* t, int level, const double pose[16], int* model_index,
                             int* bin, unsigned* hist) {
  try {
    kf_status st = debug_prepare(t, level, pose, 0, 0, -1, -1, 0);
    if (st != KF_OK) return st;
    cudaStream_t s = t->stream;
    KF_CK(t, launch_assoc_hist(t->d_self, t->d_dbg_list, 1, t->grid_assoc, level, 1, t->kp, s));
    KF_CK(t, cudaStreamSynchronize(s));
    const LevelMaps& L = t->h_desc.lv[level];
    const size_t px = (size_t)L.fw * L.fh;
    if (model_index) KF_CK(t, cudaMemcpy(model_index, t->h_desc.dbg_index, px * sizeof(int), cudaMemcpyDeviceToHost));
    if (bin) KF_CK(t, cudaMemcpy(bin, t->h_desc.dbg_bin, px * sizeof(int), cudaMemcpyDeviceToHost));
    if (hist) KF_CK(t, cudaMemcpy(hist, t->h_desc.hist, sizeof(unsigned) * t->p.hist_bins, cudaMemcpyDeviceToHost));
    return KF_OK;
  } catch (...) {
    return KF_ERR_INTERNAL;
  }
}

kf_status kf_debug_reduce(kf_tracker* t, int level, const double pose[16], int klo, int khi,
                          double sums[29]) {
  if (!sums) return KF_ERR_INVALID_ARG;
  if (!t || klo < 0 || khi < klo) return KF_ERR_INVALID_ARG;
  try {
    // a band from bin 0 goes the way of an iteration whose band edge fell in
    // the window: the association pass with a window around khi, then the
    // recorded pixels; any other band is one re-association with the band
    // known (the way of a window that missed)
    const bool split = klo == 0;
    const int w0 = split ? std::max(0, khi - 3) : -1, w1 = split ? khi + 4 : -1;
    kf_status st = debug_prepare(t, level, pose, klo, khi, w0, w1, split ? 1 : 0);
    if (st != KF_OK) return st;
    cudaStream_t s = t->stream;
    if (split)
      KF_CK(t, launch_assoc_hist(t->d_self, t->d_dbg_list, 1, t->grid_assoc, level, 2, t->kp, s));
    KF_CK(t, launch_reduce_solve(t->d_self, 1, t->d_dbg_list, t->d_dbg_list, 1, t->d_dbg_counter,
                                 t->grid_reduce, level, -1, 2, t->kp, s));
    KF_CK(t, cudaStreamSynchronize(s));
    KF_CK(t, cudaMemcpy(sums, reinterpret_cast<const char*>(t->d_state) + offsetof(PairState, dbg_sums),
                        sizeof(double) * kSums, cudaMemcpyDeviceToHost));
    return KF_OK;
  } catch (...) {
    return KF_ERR_INTERNAL;
  }
}

kf_status kf_debug_trace(kf_tracker* t, kf_iter_record* rec, int max, int* count) {
  if (!t || !count || max < 0 || (max > 0 && !rec)) return KF_ERR_INVALID_ARG;
  KF_CK(t, cudaStreamSynchronize(t->stream));
  int len = 0;
  KF_CK(t, cudaMemcpy(&len, reinterpret_cast<const char*>(t->d_state) + offsetof(PairState, trace_len),
                      sizeof(int), cudaMemcpyDeviceToHost));
  len = std::min(len, std::min(max, KF_TRACE_MAX));
  if (len > 0)
    KF_CK(t, cudaMemcpy(rec, reinterpret_cast<const char*>(t->d_state) + offsetof(PairState, trace),
                        sizeof(kf_iter_record) * len, cudaMemcpyDeviceToHost));
  *count = len;
  return KF_OK;
}

kf_status kf_debug_wait_timeout(kf_tracker* t, double wait_ms) {
  if (!t || !(wait_ms == wait_ms)) return KF_ERR_INVALID_ARG;
  try {
    const double ms = std::min(2000.0, std::max(1.0, wait_ms));
    const unsigned slots = 1024;  // more than the blocks of one wave claim
    const size_t bytes = sizeof(unsigned) * kQHeaderWords + sizeof(unsigned long long) * slots;
    unsigned* queue = nullptr;
    KF_CK(t, cudaMalloc(&queue, bytes));
    cudaStream_t s = t->stream;
    cudaError_t e = cudaMemsetAsync(queue, 0, bytes, s);
    if (e == cudaSuccess)
      e = launch_icp_sched(t->d_self, nullptr, nullptr, 0, queue, slots - 1,
                           (unsigned)std::min(t->grid_sched, (int)slots - 1),
                           (unsigned long long)(ms * 1e6), t->kp, s);
    unsigned err = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&err, queue + kQErr, sizeof(err), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(queue);
    if (e != cudaSuccess) return cuda_fail(t, e, "kf_debug_wait_timeout");
    if (err == 0u) return fail(t, KF_ERR_INTERNAL, "the empty scheduled launch ended without a wait running out");
    return fail(t, KF_ERR_TIMEOUT, "a bounded device wait ran out (expected: nothing was queued)");
  } catch (...) {
    return KF_ERR_INTERNAL;
  }
}

kf_status kf_profile_enable(kf_tracker* t, int on) {
  if (!t) return KF_ERR_INVALID_ARG;
  if (on) {
    for (int i = 0; i < 2; ++i)
      if (!t->fe_ev[i]) KF_CK(t, cudaEventCreate(&t->fe_ev[i]));
    memset(&t->prof, 0, sizeof(t->prof));
  }
  t->profiling = on != 0;
  return KF_OK;
}

kf_status kf_profile_read(kf_tracker* t, kf_profile* out) {
  if (!t || !out) return KF_ERR_INVALID_ARG;
  *out = t->prof;
  return KF_OK;
}

}  // extern "C"
