/*
 * kf_track.h - C ABI of the GB300 camera-tracking library.
 *
 * Tracking hot path of "Integration of Absolute Orientation Measurements in
 * the KinectFusion Reconstruction pipeline" (Giancola, Schneider, Wonka,
 * Ghanem; arXiv 1802.03980): coarse-to-fine projective point-to-plane ICP
 * (Eq. 1-3) seeded by an absolute orientation measured by an IMU (Sec. 3),
 * solved with the orientation-regularised normal equations (Eq. 4, 5), with
 * the closest-point distance histogram (Sec. 3.2), the median-based pair
 * filter (Sec. 3.3) and median-driven convergence control (Sec. 3.4).
 * Options cover the paper's own normal estimation and association (Sec. 3.3:
 * integral-image normals, normal shooting) and its regulariser schedules;
 * kf_volume_* is the model producer (TSDF integration and raycast of the
 * model maps the frames are aligned to).
 *
 * Conventions shared by every entry point
 *  - A pose is a row-major 4x4 double matrix mapping camera coordinates to
 *    world coordinates (last row 0 0 0 1).
 *  - Depth is float32 metres, row-major W x H; 0, negative or non-finite
 *    values mean "no measurement".
 *  - Model maps are float32, row-major W x H x 3 (x, y, z interleaved), world
 *    coordinates; a model pixel is a hole when any vertex or normal component
 *    is non-finite or the normal is all zero.
 *  - Camera frame: x right, y down, z forward; pixel (u, v) has its centre at
 *    integer coordinates.
 *  - A tracker is bound to one CUDA stream (the one given at creation) and is
 *    not thread-safe. Entry points given pageable host pointers return once
 *    the host memory is no longer needed; page-locked depth frames given to
 *    kf_set_frame(_batch) are read after the call returns (see KF_FRAME_*).
 *    No exception crosses this ABI.
 *  - Every entry point returns a kf_status; KF_OK (0) and KF_NOT_CONVERGED
 *    (1, a warning) are success. On an error, kf_last_error() describes it.
 *  - Device pointers (is_device_ptr != 0) must point to memory of the
 *    tracker's device. The copy into tracker-owned buffers is queued on the
 *    tracker's stream; the caller may reuse the buffer once that stream has
 *    passed the call.
 */
#ifndef KF_TRACK_H
#define KF_TRACK_H

#ifdef __cplusplus
extern "C" {
#endif

#define KF_MAX_LEVELS 4
#define KF_TRACE_MAX 64

typedef struct kf_tracker kf_tracker; /* opaque; owns its device buffers */

typedef enum {
  KF_OK = 0,
  KF_NOT_CONVERGED = 1,       /* warning: the finest level hit its iteration cap
                                 without meeting the convergence rule (Sec. 3.4) */
  KF_ERR_INVALID_ARG = -1,
  KF_ERR_CUDA = -2,
  KF_ERR_OOM = -3,
  KF_ERR_NO_FRAME = -4,
  KF_ERR_NO_MODEL = -5,
  KF_ERR_TOO_FEW_INLIERS = -6, /* fewer than n_min matched pairs or inliers */
  KF_ERR_DEGENERATE = -7,      /* Cholesky pivot <= 1e-12 of its diagonal entry */
  KF_ERR_TIMEOUT = -8,
  KF_ERR_INTERNAL = -9,
  KF_ERR_SCRATCH_LIMIT = -10   /* input larger than kf_reduce_noalloc's fixed scratch */
} kf_status;

/* Flags of kf_params.flags. All three off is the original KinectFusion loop
 * (no IMU seed, every match within d_max used, fixed iteration counts). */
#define KF_USE_PRIOR 1u       /* seed T0 = [R_prior | t_init] (Sec. 3) */
#define KF_USE_FILTER 2u      /* median band filter (Sec. 3.3) */
#define KF_USE_CONVERGENCE 4u /* stop a level after 3 equal medians (Sec. 3.4) */
/* Accepted and ignored (kept for source compatibility): the association pass
 * always reads each frame vertex and its model match once, summing the rows
 * it can before the band is known (see kf_iter_record.passes). */
#define KF_SINGLE_PASS 8u
/* Opt-in execution variant (same results, bit for bit): one launch per stage
 * and iteration, every pair of the batch in step, instead of the default
 * single persistent launch in which each pair advances on its own. */
#define KF_LAUNCH_PER_ITERATION 16u
/* Regulariser variant (not in the paper): hold the rotation of the UPDATED
 * pose toward the IMU prior instead of penalising the increment's rotation:
 * lambda |log(Exp(w) R R_prior^T)|^2, linearised as lambda |w + r|^2 with
 * r = log(R R_prior^T); the matrix of Eq. 5 is unchanged and its right-hand
 * side becomes A^T b - 2 lambda n P^T r. Needs prior_R (ignored without it). */
#define KF_PRIOR_ANCHORED 32u

/* kf_params.normal_mode. Integral-image normals (Sec. 3.3; Holzer et al.):
 * per pixel the average 3D gradient over a square window, g_h = sum of the
 * vertices right of the pixel minus the sum left of it (rows y-r..y+r) and
 * g_v likewise below minus above, n = g_h x g_v normalised and facing the
 * camera. The half-size r = min(floor((a + b z) / 2^l), dist - 1, distance to
 * the image border, r_max), dist the chessboard distance to the nearest depth
 * edge (no depth, or a 4-neighbour without depth or differing by more than
 * ii_depth_change z); no normal unless r >= 1. Vertices enter in fixed
 * point (units of 2^-20 m), so the window sums are exact; the normal is
 * float32. A frame pixel without a normal takes no part in the alignment. */
#define KF_NORMALS_CROSS 0
#define KF_NORMALS_INTEGRAL 1

/* Storage precision of the vertex / normal maps read by the ICP loop. */
#define KF_FP32 0
#define KF_FP16 1

/* lambda(n) schedules of the regularisation weight (Sec. 3.1 and the lambda
 * table of Sec. 5.2): c, c/sqrt(n), c/n, c/n^2, c*ln(n). The table prints the
 * last one as -c ln(n), which is negative for n > 1; it is read as c ln(n). */
#define KF_LAMBDA_CONST 0
#define KF_LAMBDA_C_SQRT_N 1
#define KF_LAMBDA_C_N 2
#define KF_LAMBDA_C_N2 3
#define KF_LAMBDA_C_LOG_N 4

typedef struct {
  int width, height;
  double fx, fy, cx, cy; /* pixels; level-0 values */
} kf_intrinsics;

typedef struct {
  int levels;                     /* pyramid levels, 1..KF_MAX_LEVELS (default 3) */
  int max_iters[KF_MAX_LEVELS];   /* iteration caps, FINEST level first: 10, 5, 4
                                     (the paper's (4,5,10) cadence run coarse to fine) */
  int hist_bins;                  /* B distance-histogram bins, 1..4096 (512) */
  double d_max;                   /* histogram range and distance gate, metres (0.16) */
  double band_kappa;              /* filter band |d - m| <= kappa m (1.0) */
  double cos_angle_min;           /* normal-angle gate; <= -1 disables it (-2) */
  int conv_window;                /* equal medians that end a level, 1..8 (3) */
  int lambda_mode;                /* KF_LAMBDA_* (KF_LAMBDA_CONST) */
  double lambda_c;                /* c of the schedule when kf_align's lambda < 0 (5) */
  int n_min;                      /* minimum matched pairs and inliers (6) */
  int precision;                  /* KF_FP32 | KF_FP16 */
  unsigned flags;                 /* KF_USE_* (all three) */
  double bilateral_sigma_s;       /* pixels (4) */
  double bilateral_sigma_r;       /* metres (0.03); also sets the 3 sigma_r
                                     depth-similarity test of the pyramid */
  int bilateral_radius;           /* window half-size, 0..4; 0 disables the filter (2) */
  /* Frame normals and association: the paper's own choices (Sec. 3.3) as
   * options; the defaults are KinectFusion's cross-product normals and
   * projective association. */
  int normal_mode;                /* KF_NORMALS_CROSS (default) | KF_NORMALS_INTEGRAL */
  double ii_radius_a;             /* integral-image window half-size a + b z pixels
                                     at level 0, halved per level (a = 2) */
  double ii_radius_b;             /* (b = 1 pixel per metre) */
  double ii_depth_change;         /* a 4-neighbour whose depth differs by more than
                                     this fraction of z marks a depth edge (0.02) */
  int ii_radius_max;              /* cap on the half-size, 1..15 (8) */
  int shoot_radius;               /* 0: projective association (default); w in 1..4:
                                     normal shooting over the (2w+1)^2 model pixels
                                     around the projection */
} kf_params;

typedef struct {
  int status;                     /* kf_status of the alignment */
  int iters[KF_MAX_LEVELS];       /* iterations run per level (finest first) */
  int total_iters;
  int inliers;                    /* n of the last iteration (post-filter) */
  int valid_pairs;                /* N of the last iteration (matched within d_max) */
  int median_bin[KF_MAX_LEVELS];  /* last median bin per level, -1 if not run */
  double rms_residual;            /* sqrt(sum b^2 / n) of the last iteration, metres */
} kf_result;

/* One iteration of the alignment loop, recorded on the device. */
typedef struct {
  int level, iter;                /* level (0 finest) and iteration within it */
  int N;                          /* matched pairs (histogram total) */
  int kmed, klo, khi;             /* median bin and inlier band */
  int n;                          /* inliers */
  int solve_ns;                   /* device time of the FP64 solve and update, ns */
  int passes;                     /* 1: the band edge fell in the window the association
                                     pass expected from the previous band edge: the
                                     frame was read once and only the pixels recorded
                                     near the edge were added afterwards; 2: the
                                     frame was associated again with the band known */
  int w0, w1;                     /* the window: bins below w0 were summed and bins in
                                     [w0, w1) recorded by the association pass
                                     (w0 = -1: none, the alignment's first iteration) */
  int pad;
  double lambda;                  /* lambda(n) used */
  double x[6];                    /* solved increment (alpha, beta, gamma, tx, ty, tz) */
} kf_iter_record;

/* Fill *p with the defaults listed above. Returns KF_ERR_INVALID_ARG on NULL. */
kf_status kf_default_params(kf_params* p);

/* Create a tracker for frames and models up to max_w x max_h on the current
 * CUDA device. cuda_stream is a cudaStream_t; NULL makes the tracker create
 * and own a non-blocking stream (the legacy default stream cannot be captured
 * into the alignment graph).
 * Allocates every device buffer the tracker needs; *out owns them until
 * kf_track_destroy. Errors: INVALID_ARG (bad params or sizes), OOM, CUDA. */
kf_status kf_track_create(const kf_params* p, int max_w, int max_h, void* cuda_stream,
                          kf_tracker** out);

/* Release a tracker and its device memory (synchronises its stream). NULL is a no-op. */
void kf_track_destroy(kf_tracker* t);

/* Where kf_set_frame / kf_set_frame_batch find the depth (is_device_ptr). */
#define KF_FRAME_HOST 0              /* host memory: pageable frames are copied and
                                        the call returns when the copy is done;
                                        page-locked frames are pulled by one queued
                                        kernel per batch over the host link */
#define KF_FRAME_DEVICE 1            /* device memory of this device, read in place */
#define KF_FRAME_HOST_COPY_ENGINE 2  /* host memory, moved by cudaMemcpyAsync on the
                                        batch's stream into a staging buffer of the
                                        batch's first tracker (grown on demand): one
                                        copy per run of frames that follow one another
                                        in host memory (a batch stored contiguously
                                        moves as one copy). Page-locked frames move by
                                        the copy engine, which needs no SMs, so the
                                        upload overlaps kernels of other streams (a
                                        second set of trackers aligning the previous
                                        batch); a pageable frame is staged before the
                                        call returns */

/* Queue the front end for a new depth frame: bilateral filter at level 0,
 * 2x2 downsampling with the 3 sigma_r similarity test, vertex and normal maps
 * per level (KinectFusion preprocessing that the paper's coarse-to-fine ICP
 * runs on). depth: W x H float32 metres, found as is_device_ptr says
 * (KF_FRAME_*). Page-locked and device frames must stay unchanged until the
 * tracker's stream has passed the call (kf_align on the same stream
 * returning is enough). K: level-0 intrinsics, width/height <= the tracker's
 * maximum. Errors: INVALID_ARG (sizes, an unknown is_device_ptr), CUDA. */
kf_status kf_set_frame(kf_tracker* t, const float* depth, const kf_intrinsics* K,
                       int is_device_ptr);

/* Same for n trackers in one batch of launches (one launch per front-end stage
 * for all n frames). depth[i] / K[i] belong to trackers[i]; all trackers must
 * share one device; the work runs on trackers[0]'s stream. */
kf_status kf_set_frame_batch(kf_tracker* const* trackers, int n, const float* const* depth,
                             const kf_intrinsics* K, int is_device_ptr);

/* Set the model the frame is aligned to (Sec. 3, "the model reconstructed so
 * far"): world vertex and normal maps of size K->width x K->height (x, y, z
 * interleaved), the model camera's pose (camera->world) and intrinsics. Holes
 * are marked as in the conventions above. Coarser model levels take every
 * second pixel of the level above. */
kf_status kf_set_model(kf_tracker* t, const float* vertex, const float* normal,
                       const double model_pose[16], const kf_intrinsics* K, int is_device_ptr);

/* Align the current frame to the current model (the hot path).
 * prior_R: 3x3 row-major IMU orientation (camera->world rotation), or NULL for
 * no prior; with KF_USE_PRIOR the seed is T0 = [prior_R | init_pose's t]
 * (Sec. 3), else T0 = init_pose. lambda: the constant c of the lambda(n)
 * schedule (Eq. 4, 5); a negative value selects params.lambda_c.
 * Writes the final pose (the last good iterate) to out_pose and, if out is not
 * NULL, the statistics. Both are written for every status except INVALID_ARG,
 * NO_FRAME, NO_MODEL and CUDA. Returns the alignment's status. */
kf_status kf_align(kf_tracker* t, const double prior_R[9], const double init_pose[16],
                   double lambda, double out_pose[16], kf_result* out);

/* Batched form: align n trackers' frames in one CUDA graph launch on
 * trackers[0]'s stream. prior_R: n x 9 (or NULL: no prior for any pair),
 * init_pose: n x 16, lambda: n (per pair), out_pose: n x 16, out: n (may be
 * NULL). All trackers need equal params except their frames and models. The
 * first call with a given tracker list (or after a set_frame size change)
 * builds and caches a launch plan and graph; later calls reuse it. Returns the
 * lowest (most severe) status over the pairs, or an error of the call itself. */
kf_status kf_align_batch(kf_tracker* const* trackers, int n, const double* prior_R,
                         const double* init_pose, const double* lambda, double* out_pose,
                         kf_result* out);

/* Message of the last error on this tracker (never NULL; "" if none). */
const char* kf_last_error(const kf_tracker* t);

/* ---- inspection hooks: copy intermediate results to HOST memory. They
 * synchronise the tracker's stream and exist for parity tests and tooling. ---- */

/* Frame level maps: depth W_l x H_l, vertex / normal W_l x H_l x 3 (camera
 * frame, NaN = invalid), dequantised to float32 for the FP16 form. Any output
 * pointer may be NULL. dims (optional): W_l, H_l. */
kf_status kf_debug_frame_level(kf_tracker* t, int level, float* depth, float* vertex,
                               float* normal, int dims[2]);

/* Model level maps as stored (dequantised to float32), world frame, holes NaN. */
kf_status kf_debug_model_level(kf_tracker* t, int level, float* vertex, float* normal,
                               int dims[2]);

/* Run the association + histogram stage (Sec. 3.2) once at `level` for the
 * given pose: per frame pixel the model pixel index v*W_m + u (or -1) and the
 * histogram bin (or -1), plus the B-bin histogram. Any output may be NULL. */
kf_status kf_debug_associate(kf_tracker* t, int level, const double pose[16], int* model_index,
                             int* bin, unsigned* hist);

/* Run the filter + reduction stage once at `level` for the given pose and
 * inlier band [klo, khi]: sums[0..20] = upper triangle of A^T A (row-major),
 * sums[21..26] = A^T b, sums[27] = n, sums[28] = sum b^2. A band from bin 0
 * takes the way of an iteration whose band edge fell in the expected window
 * (association pass with a window around khi, then the recorded pixels);
 * any other band the way of a window that missed (one re-association with
 * the band known). Errors: INVALID_ARG (klo < 0 or khi < klo), NO_FRAME,
 * NO_MODEL, CUDA. */
kf_status kf_debug_reduce(kf_tracker* t, int level, const double pose[16], int klo, int khi,
                          double sums[29]);

/* Per-iteration records of the last kf_align / kf_align_batch on this
 * tracker, at most KF_TRACE_MAX; *count receives the number written. */
kf_status kf_debug_trace(kf_tracker* t, kf_iter_record* rec, int max, int* count);

/* Failure-detection check of the device scheduler's bounded waits (the paper
 * has no counterpart). Launches the persistent ICP kernel of kf_align_batch
 * over an empty batch with every wait limited to wait_ms (clamped to 1..2000):
 * no task is ever queued, so each block's wait for its next task runs out,
 * sets the launch's error word and returns, and the call reports that as a
 * normal status. Returns KF_ERR_TIMEOUT when the error word was set (the
 * expected outcome), KF_ERR_INTERNAL if the launch ended without it, or a CUDA
 * error. The tracker stays usable; its frame, model and plans are untouched. */
kf_status kf_debug_wait_timeout(kf_tracker* t, double wait_ms);

/* ---- stage timing (tracing). With profiling on, CUDA events recorded on the
 * tracker's stream (inside the alignment graph, around every launch) time
 * each stage on the device; kf_profile_read sums them since the last enable.
 * For a batch the counters of trackers[0] are used. ---- */
typedef struct {
  double frontend_ms;        /* kf_set_frame(_batch): filter, pyramid, maps */
  double assoc_ms;           /* association-pass launches (KF_LAUNCH_PER_ITERATION) */
  double reduce_ms;          /* reduction + solve launches (KF_LAUNCH_PER_ITERATION) */
  double fused_ms;           /* unused (0) */
  double align_ms;           /* whole alignment graphs */
  long long frontend_calls;  /* set-frame calls (one front-end launch each) */
  long long assoc_launches, reduce_launches, fused_launches /* unused (0) */, graph_launches;
  long long pixel_iters;     /* frame pixels associated, summed over the
                                iterations each pair actually ran */
  long long alignments;      /* frame pairs aligned */
  double sched_ms;           /* persistent scheduled ICP launches (the default) */
  long long sched_launches;
} kf_profile;

/* on != 0 resets the counters and turns timing on (cached launch plans are
 * rebuilt with event nodes); on == 0 turns it off. */
kf_status kf_profile_enable(kf_tracker* t, int on);
kf_status kf_profile_read(kf_tracker* t, kf_profile* out);

/* ---- model producer: TSDF volume and raycast (KinectFusion's mapping half;
 * the paper keeps a 512^3 cube of at most 6 m side, Sec. 4.4, and aligns each
 * frame to the model reconstructed so far, Sec. 3). The raycast's maps are
 * what kf_set_model takes (world vertices and normals, x, y, z interleaved,
 * NaN where the ray finds no surface), so a tracker can follow its own map.
 *
 * Field F in [-1, 1] and weight W per voxel, float32, [z][y][x]; voxel i of an
 * axis is centred at origin + (i + 1/2) side / res. Integration (per voxel):
 * camera point p = R^T (x - t); pixel (rint(fx p.x / p.z + cx),
 * rint(fy p.y / p.z + cy)); raw depth D there (finite, > 0); eta = D - p.z;
 * where eta >= -mu: F <- (W F + min(1, eta / mu)) / (W + 1),
 * W <- min(W + 1, w_max). Raycast (per pixel): samples every dz of camera
 * depth from z_near to z_far, trilinear F of cells whose 8 corners were
 * observed; the first sign change from + to 0 or - is the surface (linear
 * refinement), a change from - to + ends the ray; the normal is the
 * normalised central-difference gradient of F (facing the camera). ---- */
typedef struct kf_volume kf_volume;

typedef struct {
  int res;          /* voxels per axis, 2..1024 (512: 1 GB of device memory) */
  float side;       /* cube side, metres */
  float origin[3];  /* world position of the cube's lower corner */
  float mu;         /* truncation distance, metres */
  float w_max;      /* weight cap (>= 1) */
} kf_volume_params;

/* 512^3 voxels, 6 m side centred on the world origin, mu 5 cm (about 4
 * voxels: choose mu of 3 voxels or more, and a raycast step dz of mu / 2 or
 * less, or rays step over the observed band behind a surface), w_max 64. */
kf_status kf_volume_default_params(kf_volume_params* p);
/* Allocates the field (F = 1, W = 0). cuda_stream as for kf_track_create.
 * Errors: INVALID_ARG, OOM, CUDA. */
kf_status kf_volume_create(const kf_volume_params* p, void* cuda_stream, kf_volume** out);
void kf_volume_destroy(kf_volume* v);
const char* kf_volume_last_error(const kf_volume* v);
/* F = 1, W = 0 everywhere. */
kf_status kf_volume_reset(kf_volume* v);
/* Fuse a raw depth frame (W x H float32 metres, host memory copied before
 * return, or device memory read by the queued kernel) seen from the
 * camera->world pose (row-major 4x4 FP64) with intrinsics K. */
kf_status kf_volume_integrate(kf_volume* v, const float* depth, const kf_intrinsics* K,
                              const double pose[16], int is_device_ptr);
/* Vertex and normal maps (K->width x K->height x 3 float32 each) of the field
 * seen from the pose: host memory (filled before return) or device memory
 * (written by the queued kernel). dz > 0; at most 1e6 samples per ray. */
kf_status kf_volume_raycast(kf_volume* v, const kf_intrinsics* K, const double pose[16],
                            float z_near, float z_far, float dz, float* vertex, float* normal,
                            int is_device_ptr);
/* Copies of F and W (res^3 floats each, either may be NULL; inspection). */
kf_status kf_volume_read(kf_volume* v, float* F, float* W);

/* ---- allocation-free reduction. The paper has no counterpart: this entry
 * point exists for callers that cannot allocate device memory themselves -
 * a plug-in running inside a host application whose CUDA allocator belongs
 * to another runtime, or a caller that must not insert cudaMalloc/cudaFree
 * (and the device synchronisation they imply) while its other work is in
 * flight. It needs no tracker and allocates nothing.
 *
 * It computes the filtered point-to-plane normal-equation sums of one frame
 * against one model: for every frame pixel with a finite vertex, the
 * projective match and float32 distance bin (as kf_align computes them,
 * without the normal-angle gate), kept when the matched model pixel is not a
 * hole (header conventions: a non-finite vertex or normal component, or an
 * all-zero normal) and the bin lies in [klo, khi]; sums[0..20] = upper
 * triangle of A^T A (row-major), sums[21..26] = A^T b, sums[27] = n,
 * sums[28] = sum b^2. Frame normals are not read: a frame pixel whose normal
 * is invalid must already have a NaN vertex (the tracker's own frame maps
 * do). With such maps the sums are those of kf_debug_reduce at the same pose
 * and band.
 *
 * Inputs and outputs belong to the caller and are DEVICE memory of the
 * current device: frame_vertex width x height x 3 floats (camera frame,
 * interleaved xyz, a pixel takes part when all three are finite);
 * model_vertex / model_normal model_K->width x model_K->height x 3 floats
 * (world frame; 3 x width x height must stay below 2^31); sums: 29 doubles,
 * written when the stream gets there. pose / model_pose (host,
 * camera->world 4x4 row-major), d_max, hist_bins, klo, khi as in kf_params /
 * the band of kf_iter_record. cuda_stream: a cudaStream_t (NULL = legacy
 * default stream). The interleaved loads are not coalesced; the entry point
 * is a side path, not the tracker's hot path.
 *
 * Scratch: a fixed 131,584-byte array in the library's device image (every
 * GPU that loads the library holds it until the process exits). It bounds the
 * frame to width * height <= 4,194,304 pixels; larger inputs return
 * KF_ERR_SCRATCH_LIMIT and queue nothing. The first call on each device looks
 * up the array's device address (with that device current); make that first
 * call before any stream capture. Every call on a device shares the array,
 * which keeps the previous call's contents (the call resets what must start
 * at zero), so calls whose work overlaps on the GPU - on different streams
 * or threads - race: order them on one stream.
 * Errors: INVALID_ARG (null pointer, bad size or band), SCRATCH_LIMIT, CUDA. */
kf_status kf_reduce_noalloc(const float* frame_vertex, int width, int height,
                            const float* model_vertex, const float* model_normal,
                            const kf_intrinsics* model_K, const double pose[16],
                            const double model_pose[16], double d_max, int hist_bins, int klo,
                            int khi, double sums[29], void* cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* KF_TRACK_H */
