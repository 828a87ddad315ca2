/*
 * far.h - C ABI of the GB300 (sm_103a) scan-to-map registration library.
 *
 * The library implements the data-parallel hot path of FAR-LIO (Sec. III-A):
 * the voxel hashmap with batched insert, adaptive-density cap and eviction
 * (Sec. III-A.2 "cuVoxelMap", Sec. III-A.3), the 27-voxel neighbour search,
 * per-point covariances (Eq. 1), and the sparsity-aware GICP Gauss-Newton
 * loop (Eq. 2-6). All arithmetic runs in the library's own CUDA kernels.
 *
 * Conventions shared by every entry point
 *  - Status: every function returns far_status and never aborts. On error the
 *    outputs are left untouched and far_last_error() describes the cause
 *    (a thread-local string).
 *  - Points: `xyz` is an array of n records of `stride_bytes` bytes whose first
 *    12 bytes are float x, y, z (stride_bytes >= 12, a multiple of 4). The
 *    pointer may be host memory (pageable or pinned) or device memory; the
 *    library detects which and copies host data on the map's stream. The caller
 *    keeps ownership of every input and output buffer.
 *  - Poses: row-major 4x4 double, sensor-to-map. Only the top 3x4 is read.
 *  - Covariances: 6x6 row-major double, ordered [rotation; translation].
 *  - Streams: each map is bound to the CUDA stream given at creation; all work
 *    of that map is ordered on it. Calls on one map must not overlap in time
 *    from several host threads. Functions that return host results synchronise
 *    that stream before returning.
 *  - Point ids: every point admitted to a map gets a 32-bit id, assigned
 *    consecutively in (call, input index) order; ids break distance ties.
 */
#ifndef FAR_H
#define FAR_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum far_status {
    FAR_OK = 0,
    FAR_ERR_INVALID = 1,     /* bad argument (null pointer, size, parameter) */
    FAR_ERR_OOM = 2,         /* device allocation failed or HBM budget exceeded */
    FAR_ERR_CAPACITY = 3,    /* table, bucket pool or id space full; excess points dropped */
    FAR_ERR_CUDA = 4,        /* a CUDA runtime call failed */
    FAR_ERR_DEGENERATE = 5,  /* fewer than 6 correspondences or H not positive definite */
    FAR_ERR_TIMEOUT = 6      /* registration exceeded its time budget */
} far_status;

/* Opaque map: owns all device memory of one voxel map and its scratch. */
typedef struct far_map far_map;

/*
 * Map parameters (Sec. III-A.2: voxel size v, at most N points per voxel,
 * "regularly spaced"; Eq. 1: k nearest neighbours for covariances).
 */
typedef struct far_map_params {
    float voxel_size;           /* v in metres, > 0 */
    uint32_t max_pts_per_voxel; /* N_max, 1..64 */
    uint32_t k_cov;             /* k for Eq. 1, 1..16 */
    float min_spacing;          /* d_min between points of a voxel; < 0 => v / sqrt(N_max); 0 => off */
    uint64_t max_voxels;        /* size of the bucket pool (live voxels) */
    float load_factor;          /* hash slots = next_pow2(max_voxels / load_factor), 0.05..0.95 */
    uint32_t max_scan_points;   /* largest scan accepted by insert / register */
    uint32_t precision_mode;    /* 0: FP32 world coordinates, FP32 covariances.
                                 * 1: mixed-precision storage: points FP32 relative to the origin of
                                 *    their 50 m tile (tile T = floor(x / 50), key = T * 50/v +
                                 *    clamp(floor(fp32(x - 50 T) * fp32(1/v)), 0, 50/v - 1), with the
                                 *    world point in FP64), covariances FP16 with one power-of-two
                                 *    exponent per voxel, Gauss-Newton linearised about the corner of
                                 *    the tile holding the initial position (same iterates; the FP32
                                 *    arithmetic runs on small numbers). v must divide 50 m, else
                                 *    FAR_ERR_INVALID. */
} far_map_params;

/* Adaptive Submap Density cap of an insert (Sec. III-A.3). */
typedef struct far_insert_params {
    int32_t asmd;     /* 0: cap = N_max for every voxel; 1: adaptive cap */
    double r_near;    /* close-range radius r_c (m) over which the mean occupancy is taken */
    double r_max;     /* range (m) at which the cap has decayed to k */
} far_insert_params;

/* Registration parameters (Sec. III-A.2, Eq. 4-6 and the termination rule). */
typedef struct far_reg_params {
    uint32_t max_iters;         /* Gauss-Newton iterations at most */
    double conv_eps;            /* stop when the increment measured at the initial sensor position c,
                                 * ||[phi; rho + phi x c]||_2 with xi = [phi; rho] about the world
                                 * origin, is <= conv_eps (paper: 5e-3); 0 => run max_iters */
    float tau;                  /* correspondence distance threshold (m) */
    float kappa;                /* Cauchy kernel scale (Eq. 5) */
    double time_budget_s;       /* wall-clock cap of one registration; <= 0 => none */
    uint32_t threads_per_point; /* lanes that search one source point together: 1, 4, 8 or 32; 0 = default */
} far_reg_params;

typedef struct far_reg_stats {
    uint32_t iters;      /* Gauss-Newton updates applied */
    uint32_t n_src;      /* source points after scan-local downsampling */
    uint32_t n_corr;     /* correspondences of the last linearisation */
    uint32_t n_p2p;      /* of which point-to-point (SA GICP special case) */
    int32_t converged;   /* 1 if ||xi|| <= conv_eps was reached */
    int32_t status;      /* far_status of the registration */
    double chi2;         /* sum of the Cauchy cost of the last linearisation */
} far_reg_stats;

/* Human-readable name of a status code (static string). */
const char* far_status_string(far_status s);
/* Description of the last error raised on the calling thread (static per thread). */
const char* far_last_error(void);
/* Library version string. */
const char* far_version(void);

/* Device bytes a map with these parameters preallocates (for HBM budgeting). */
far_status far_map_bytes(const far_map_params* params, uint64_t* out_bytes);

/*
 * Create a map and preallocate all its device memory (the paper preallocates
 * its VRAM, Sec. IV-B). `cuda_stream` is a cudaStream_t (NULL = legacy default).
 */
far_status far_map_create(const far_map_params* params, void* cuda_stream, far_map** out);
far_status far_map_destroy(far_map* map);
/* Remove every voxel; ids restart at 0. */
far_status far_map_clear(far_map* map);

/*
 * Insert a scan (Sec. III-A.3): points are transformed by `pose`
 * (x_w = fp32(R p + t), evaluated in FP64), keyed by voxel, and admitted in input
 * order while their voxel holds fewer than its cap and every point already in it
 * is at least d_min away. The cap is N_max, or with ASMD
 *   N_ASMD(r) = clamp(round(N_near + (k - N_near) * min(r / r_max, 1)), k, N_max),
 * N_near = mean point count of this scan's voxels within r_near of the sensor,
 * r = distance from the voxel centre to the sensor. Then the Eq. 1 covariance of
 * every added point is computed against the updated map. `params` may be NULL
 * (cap = N_max). `n_inserted` (may be NULL) receives the number of added points.
 * Points with non-finite coordinates or keys beyond +-2^20 voxels are skipped.
 */
far_status far_map_insert(far_map* map, const float* xyz, uint64_t n, uint32_t stride_bytes,
                          const double pose[16], const far_insert_params* params, uint64_t* n_inserted);

/*
 * Evict (Sec. III-A.3): remove every voxel whose centre ((key + 0.5) v) is
 * farther than `radius` from `center` (distance computed in FP64).
 */
far_status far_map_evict(far_map* map, const double center[3], double radius, uint64_t* n_removed);

/* Live voxels and points of the map. */
far_status far_map_size(const far_map* map, uint64_t* n_voxels, uint64_t* n_points);

/*
 * Sorted dump of the map (parity checks): voxels in ascending (x, y, z) key
 * order, points of a voxel in insertion order. Host output arrays:
 * keys[3 * voxels], counts[voxels], ids[points], xyz[3 * points],
 * cov[6 * points] (xx xy xz yy yz zz), valid[points]. Capacities are checked
 * against far_map_size(); any pointer except keys/counts may be NULL.
 * precision_mode 1: xyz = fp32(50 T + tile-relative value) and the FP16
 * covariances decoded to FP32.
 */
far_status far_map_export(const far_map* map, int32_t* keys, uint32_t* counts, uint32_t* ids, float* xyz,
                          float* cov, uint8_t* valid, uint64_t cap_voxels, uint64_t cap_points);

/*
 * 1-NN over the 27 voxels around each query point's voxel (Sec. III-A.2):
 * smallest FP32 d^2 = ((dx*dx + dy*dy) + dz*dz), ties to the smaller id.
 * precision_mode 1: the distance is taken in the frame of the query's tile
 * (query fp32(q - 50 T_q), map point fp32(p_tile + 50 (T_p - T_q))).
 * out_ids[i] = id, or -1 when there is no candidate or d^2 > fp32(tau)^2.
 * out_d2 (may be NULL) receives d^2 (+inf without a candidate).
 * Outputs may be host or device pointers.
 */
far_status far_map_nearest(far_map* map, const float* q, uint64_t n, uint32_t stride_bytes, float tau,
                           int64_t* out_ids, float* out_d2);

/*
 * k nearest map points (k <= 16) over the 27 voxels, ordered by (d^2, id).
 * out_ids[n * k] (0xFFFFFFFF padding), out_found[n]. Host or device outputs.
 */
far_status far_map_knn(far_map* map, const float* q, uint64_t n, uint32_t stride_bytes, uint32_t k,
                       uint32_t* out_ids, int32_t* out_found);

/*
 * Source side of a registration (Sec. III-A.2 Cov-Calc): build a scan-local
 * voxel map with the map's v, N_max and d_min (no ASMD), keep the admitted
 * points (the downsampling), and compute their Eq. 1 covariances from k
 * neighbours in that local map. Outputs (host or device, room for n entries):
 * index[n_src] (input index of each admitted point, ascending), cov[6 n_src],
 * valid[n_src], knn_ids[k n_src] (local admission ranks; may be NULL).
 */
far_status far_scan_sources(far_map* map, const float* xyz, uint64_t n, uint32_t stride_bytes, int64_t* out_index,
                            float* out_cov, uint8_t* out_valid, uint32_t* out_knn_ids, uint64_t* n_src);

/*
 * One Gauss-Newton linearisation of Eq. 4 at `pose` without the update:
 * H (36, row-major) and g (6) as defined by J = [[q - A]x, -I] with the anchor A
 * (the origin; precision_mode 1: 50 floor(t / 50) of the pose's translation), IRLS Cauchy weights
 * w = 1 / (1 + e^2 / kappa^2), e^2 = d^T M d, M = (Sigma_r + R Sigma_s R^T)^-1
 * or I when either covariance is invalid. out_corr[n_src] (may be NULL) receives
 * the map id matched by each source point or -1. The search query of a source
 * point s is the FP32 chain fma(R_i0, s_0, fma(R_i1, s_1, fma(R_i2, s_2, t_i)))
 * of the pose rounded once to FP32 (translation taken relative to A), so the
 * matches of a pose are one exact answer. threads_per_point as in far_reg_params
 * (the lanes that search one point; the matches do not depend on it). Host outputs.
 */
far_status far_linearize(far_map* map, const float* xyz, uint64_t n, uint32_t stride_bytes, const double pose[16],
                         float tau, float kappa, uint32_t threads_per_point, double out_H[36], double out_g[6],
                         int32_t* out_corr, far_reg_stats* stats);

/*
 * Register a scan against the map (Sec. III-A.2): scan-local downsampling and
 * covariances, then Gauss-Newton iterations from `init_pose`, each solving
 * H xi = -g by FP64 Cholesky and applying T <- exp(xi) T (Eq. 6), until
 * the increment at the initial sensor position is <= conv_eps (see
 * far_reg_params) or max_iters. out_cov (may be NULL) receives H^-1 of the
 * last linearisation. Returns FAR_ERR_DEGENERATE (pose = last good estimate)
 * when fewer than 6 correspondences remain or H is not positive definite.
 */
far_status far_register_scan(far_map* map, const float* xyz, uint64_t n, uint32_t stride_bytes,
                             const double init_pose[16], const far_reg_params* params, double out_pose[16],
                             double out_cov[36], far_reg_stats* stats);

typedef struct far_step_result {
    far_reg_stats reg;    /* registration of the scan */
    uint64_t n_inserted;  /* points added to the map */
    uint64_t n_removed;   /* points evicted */
    uint64_t n_voxels;    /* map size after the step */
    uint64_t n_points;
} far_step_result;

/*
 * Start copying a host scan to the device ahead of the call that will use it: the copy runs on
 * the map's own copy stream into one of two staging buffers (set up on the first call), so it
 * overlaps the map's kernels of the scan in progress (for pinned host memory). Up to two
 * prefetched scans are kept; a third replaces the older one. A later call on this map that
 * ingests points (far_process_scan, far_register_scan, far_map_insert, ...) with exactly a kept
 * xyz, n and stride_bytes uses that copy instead of making its own; any other call copies as
 * usual. The caller must not change the host array in between. Device pointers and n = 0 are
 * accepted and do nothing. Records wider than 32 bytes are staged as their first 32 bytes.
 */
far_status far_prefetch_points(far_map* map, const float* xyz, uint64_t n, uint32_t stride_bytes);

/*
 * One scan of the LiDAR pipeline on the device (Sec. III-A.2 then III-A.3):
 * far_register_scan from `init_pose`, then - when the registration succeeded -
 * the insert of the same scan at the registered pose with the cap of `ins`
 * (NULL: N_max), then eviction of the voxels farther than `evict_radius` from the
 * registered position (0 or +inf: no eviction). The registered pose never leaves
 * the device between the stages; the call synchronises once at the end.
 * Returns the registration status (a degenerate or timed-out scan is discarded,
 * the map is left unchanged except for eviction), or FAR_ERR_CAPACITY.
 */
far_status far_process_scan(far_map* map, const float* xyz, uint64_t n, uint32_t stride_bytes,
                            const double init_pose[16], const far_reg_params* reg, const far_insert_params* ins,
                            double evict_radius, double out_pose[16], double out_cov[36], far_step_result* result);

/*
 * Motion undistortion (Sec. III-A.1). A spinning LiDAR fires its points over a sweep while
 * it moves; each record carries its firing time tau (FP32 seconds, relative to the sweep's
 * reference time, the last point's time stamp, so tau <= 0) at byte `time_offset_bytes`. The
 * LiDAR's angular and linear velocity in its own frame are modelled as lines in tau,
 * w(tau) = w0 + w1 tau and v(tau) = v0 + v1 tau (from a regression over the velocity history:
 * far_motion_fit). A point fired at tau is moved to the reference frame by the SE(3)
 * exponential of the twist integrated from 0 to tau:
 *   p_ref = R p + V rho,  [phi; rho] = [w0 tau + w1 tau^2 / 2; v0 tau + v1 tau^2 / 2],
 *   R = exp([phi]x) (Rodrigues), V the matching left Jacobian (exact for a constant twist).
 * The kernel computes in FP32 (Taylor series of R and V below |phi| = 0.25 rad).
 */
typedef struct far_motion {
    double w0[3], w1[3];          /* rad/s, rad/s^2 */
    double v0[3], v1[3];          /* m/s, m/s^2 */
    uint32_t time_offset_bytes;   /* offset of tau in each record: a multiple of 4, 12..stride_bytes - 4 */
} far_motion;
/*
 * Least-squares lines through n samples (times t[i] in seconds, rates w[3 i..], velocities
 * v[3 i..], LiDAR frame) as functions of t - t_ref; one distinct time stamp gives constants.
 * Host code; fills every field of `out` (time_offset_bytes as given).
 */
far_status far_motion_fit(const double* t, const double* w, const double* v, uint32_t n, double t_ref,
                          uint32_t time_offset_bytes, far_motion* out);
/*
 * The de-skew alone (parity): n records of stride_bytes (>= 16) on the device -> out_xyz
 * (device, 3 n floats, the points at the reference time). Runs on cuda_stream, synchronises it.
 */
far_status far_undistort(const float* xyz, uint64_t n, uint32_t stride_bytes, const far_motion* motion,
                         float* out_xyz, void* cuda_stream);
/*
 * far_process_scan with the de-skew fused into the ingest of the scan (motion NULL: none).
 * Host records wider than 32 bytes need time_offset_bytes <= 28. The registered pose is
 * the pose at the sweep's reference time.
 */
far_status far_process_scan_motion(far_map* map, const float* xyz, uint64_t n, uint32_t stride_bytes,
                                   const far_motion* motion, const double init_pose[16], const far_reg_params* reg,
                                   const far_insert_params* ins, double evict_radius, double out_pose[16],
                                   double out_cov[36], far_step_result* result);
/*
 * far_process_scan_motion in two halves, so that the caller's host work that does not depend on
 * this scan's result (e.g. far_prefetch_points of the next scan) overlaps the device work.
 * far_process_scan_async checks its arguments and enqueues the whole step on the map's stream
 * (the pose covariance too when want_cov is non-zero), then returns without waiting;
 * far_process_scan_wait waits for it and fills the outputs exactly as far_process_scan_motion
 * does (which is async followed by wait). One step may be pending per map: a second async call
 * before the wait, or a wait without a pending step, is FAR_ERR_INVALID (a wait whose outputs
 * are invalid leaves the step pending). Between the two calls the map must not be used
 * otherwise, and host points that were not prefetched must stay valid and unchanged (their copy
 * may still be in flight). The wait returns the step's status as far_process_scan_motion would.
 */
far_status far_process_scan_async(far_map* map, const float* xyz, uint64_t n, uint32_t stride_bytes,
                                  const far_motion* motion, const double init_pose[16], const far_reg_params* reg,
                                  const far_insert_params* ins, double evict_radius, int32_t want_cov);
far_status far_process_scan_wait(far_map* map, double out_pose[16], double out_cov[36], far_step_result* result);

/*
 * Batched registration: many independent problems (each scan against its own map) run
 * together. Per problem the scan-local sources are built on worker streams; then every
 * Gauss-Newton iteration is ONE linearisation launch whose resident grid is shared by all
 * problems (blocks in proportion to the point counts) and ONE solve launch with a block per
 * problem; each problem stops on its own convergence flag. The whole batch is captured in
 * a CUDA graph on the first call and replayed while the input pointers, sizes, strides,
 * max_iters and threads_per_point stay the same (init poses, tau, kappa, conv_eps and the
 * time budget may change between calls). Inputs must be device or pinned host memory.
 * The batch runs on its own stream after the work already queued on `cuda_stream`, and
 * returns when it is done. The maps are used exclusively by the batch during a call.
 */
typedef struct far_batch far_batch;
far_status far_batch_create(far_map* const* maps, uint32_t count, void* cuda_stream, far_batch** out);
far_status far_batch_destroy(far_batch* batch);
/* xyz[i], n[i], stride_bytes[i]: problem i; init_poses / out_poses: 16 doubles per problem;
 * params: one set for all (params_count = 1) or one per problem (params_count = count; their
 * max_iters and threads_per_point must agree); stats (may be NULL): one per problem.
 * Returns FAR_OK, or the first problem's failure. */
far_status far_batch_register(far_batch* batch, const float* const* xyz, const uint64_t* n,
                              const uint32_t* stride_bytes, const double* init_poses, const far_reg_params* params,
                              uint32_t params_count, double* out_poses, far_reg_stats* stats);
/*
 * The whole per-scan step (far_process_scan) for every problem of the batch at once:
 * batched registration, then each scan inserted into its map at its registered pose (kept on
 * the device) and eviction around it, on worker streams. Issued directly (no graph), so the
 * sizes and inputs may change on every call (a serving loop). results: one per problem.
 */
far_status far_batch_process(far_batch* batch, const float* const* xyz, const uint64_t* n,
                             const uint32_t* stride_bytes, const double* init_poses, const far_reg_params* params,
                             uint32_t params_count, const far_insert_params* ins, double evict_radius,
                             double* out_poses, far_step_result* results);

/*
 * far_scan_sources_static - far_scan_sources without any device allocation.
 * The paper has no counterpart: this entry point exists for callers that cannot
 * call cudaMalloc - a process whose device memory is fixed before it starts (an
 * embedded or safety partition, a memory-capped client of a shared GPU server),
 * or a thread that must not allocate while other threads capture CUDA graphs -
 * and therefore cannot create a far_map. It runs the same kernels (scan-local
 * downsampling with the spacing rule, then the covariance of every kept point
 * from its k nearest kept neighbours, regularised as far_scan_sources does) on
 * one ~8 MB file-scope device array that every GPU loading the library keeps
 * until the process exits. Limits: n <= 16384 points, max_pts_per_voxel <= 20,
 * k_cov <= 16; larger sizes return FAR_ERR_INVALID with a message.
 * Inputs and outputs are DEVICE pointers of the current device (or managed
 * memory) owned by the caller; memory of another GPU returns FAR_ERR_INVALID.
 * Outputs have room for n entries: index[n], cov[6 n], valid[n], knn_ids[k n]
 * or NULL; n_src is host memory. Work runs on `cuda_stream`; the call
 * synchronises it.
 * The first call on a device resolves the array's address (cudaGetSymbolAddress)
 * for that device with it current, and the address is kept for the life of the
 * process: make that first call before any stream capture, and do not reset the
 * device (cudaDeviceReset) after it. Every call reuses the same array and first
 * clears what must start at zero (also after a call that failed half-way), so
 * calls whose GPU work overlaps (other streams, other host threads, one device)
 * race and must be serialised by the caller.
 */
far_status far_scan_sources_static(const float* xyz, uint64_t n, uint32_t stride_bytes, float voxel_size,
                                   uint32_t max_pts_per_voxel, uint32_t k_cov, float min_spacing, void* cuda_stream,
                                   int64_t* out_index, float* out_cov, uint8_t* out_valid, uint32_t* out_knn_ids,
                                   uint64_t* n_src);

/* ---------------------------------------------------------------- instrumentation */

/* Kernel launches issued by the library since it was loaded (all maps). */
unsigned long long far_launch_count(void);

/*
 * Per-stage device timeline of the last far_process_scan / far_register_scan
 * (CUDA events on the map's stream; the paper reports the same split per frame,
 * Sec. IV-B, Fig. 4a). Stages: ingest (a copy of host points and packing),
 * sources (scan-local map and Eq. 1 covariances), Gauss-Newton (all launches),
 * insert (ASMD cap, admission, added-point covariances), evict.
 * Each Gauss-Newton iteration is a linearisation launch (search, Eq. 3-5, block
 * sums) and a one-block solve launch (reduction, Cholesky, SE(3) update);
 * gn_launch_ms / gn_solve_ms are their mean durations over the iterations that did work.
 */
typedef struct far_stage_times {
    double ingest_ms, sources_ms, gauss_newton_ms, gn_launch_ms;
    uint32_t gn_launches;
    double insert_ms, evict_ms, total_ms, gn_solve_ms;
} far_stage_times;
far_status far_set_profiling(far_map* map, int enable);
far_status far_get_stage_times(const far_map* map, far_stage_times* out);

/*
 * Parts of the two inserts of the last profiled scan (milliseconds, CUDA events on the
 * map's stream): out[0] the scan-local map that yields the sources (cov_ms: their Eq. 1
 * covariances), out[1] the insert into the map (cov_ms: covariances of the added points).
 * keys: transform, keys and hash slots; sort: grouping by slot; group: group bounds, ASMD
 * and voxel order; admit: capped spaced admission; ids: ids and the grouped order.
 */
typedef struct far_insert_times {
    double keys_ms, sort_ms, group_ms, admit_ms, ids_ms, cov_ms;
} far_insert_times;
far_status far_get_insert_times(const far_map* map, far_insert_times out[2]);

/*
 * Footprint of one Gauss-Newton launch at the last registration's final pose:
 * out[0] = source points, out[1] = distinct map voxels probed by their
 * 27-neighbourhoods, out[2] = points held by those voxels. Diagnostic only.
 */
far_status far_gn_footprint(far_map* map, uint64_t out[3]);

/*
 * Adaptive correspondence threshold (the scheme the paper adopts from
 * Vizzo et al., Sec. III-A.2), pure host code: sigma = sqrt(mean delta^2) over
 * recorded frames (sigma0 before any), tau = 3 sigma, kappa = sigma / 3. A frame
 * is recorded when the translation of init^-1 * result exceeds min_motion;
 * delta = 2 r_max sin(theta / 2) + ||dt||.
 */
typedef struct far_threshold {
    double sigma0, min_motion, r_max, sse;
    int64_t n;
} far_threshold;
far_status far_threshold_init(far_threshold* t, double sigma0, double min_motion, double r_max);
far_status far_threshold_get(const far_threshold* t, double* tau, double* kappa);
far_status far_threshold_update(far_threshold* t, const double init_pose[16], const double result_pose[16]);

/* ---------------------------------------------------------------- sensor fusion (host, FP64)
 *
 * The thin consumer of the registration (Sec. III-B): it turns registered poses into the
 * odometry the scan pipeline feeds back as its next initial guess. Pure host code: no GPU
 * is needed, nothing here touches a far_map.
 */

/*
 * Eq. 7: the LiDAR's 3D velocity in its own frame from the registered poses of two scans
 * dt seconds apart, v = R_cur^-1 (t_cur - t_prev) / dt (row-major 4x4 poses; dt > 0).
 */
far_status far_lidar_velocity(const double T_prev[16], const double T_cur[16], double dt, double v[3]);

/*
 * Kinematic EKF (Sec. III-B). State (Eq. 8) x = [t (map position), theta (roll, pitch, yaw
 * with R(theta) = Rz(yaw) Ry(pitch) Rx(roll)), v (velocity in the body frame)], input
 * u = [a_m (specific force), omega_m (rate)] of the IMU, body frame = LiDAR frame.
 * far_ekf_predict applies Eq. 9 as one explicit Euler step from the filter's time to t:
 *   t += dt R v,  theta += dt E(theta) (omega_m - omega_b),
 *   v += dt (-[omega_m]x v + (a_m - a_b) + R^T (0, 0, -g)),
 * with the analytic Jacobian and Q = diag(q) dt; the state is kept in a history of
 * `history` entries, each with the IMU input of the prediction that produced it.
 * far_ekf_update takes a registration that refers to time t_meas (the scan's time stamp,
 * possibly in the past): z_s = [t_L, theta_L, v_L] and, when r_ref is set, the reference roll
 * and pitch theta_ref (Eq. 10), projected to the current time by Eq. 11,
 * z_k = z_s + h(x) - h(x_s), with x_s the stored state at or just before t_meas (the oldest one
 * if t_meas precedes the history) and h selecting the measured states (theta_ref measures the
 * state's roll and pitch); then a Kalman update with R = diag(r, r_ref) (Joseph form), angle
 * innovations wrapped to (-pi, pi]. theta_ref comes from x_s's velocity and the IMU input that
 * produced x_s: gravity in the body frame from Eq. 9's velocity equation taken as steady,
 * g = [omega_m]x v - (a_m - a_b), solved for roll = atan2(-g_y, -g_z) and
 * pitch = atan2(g_x, sqrt(g_y^2 + g_z^2)) (an entry with no IMU input yet, e.g. the initial
 * state, gives no theta_ref rows). Biases are fixed parameters (calibrated at standstill, as
 * the paper does). FAR_ERR_INVALID on bad arguments or time going backwards;
 * FAR_ERR_DEGENERATE when H P H^T + R is not positive definite.
 */
typedef struct far_ekf far_ekf;
typedef struct far_ekf_params {
    double gravity;       /* g in m/s^2 */
    double acc_bias[3];   /* a_b */
    double gyro_bias[3];  /* omega_b */
    double q[9];          /* process noise density per state: Q = diag(q) dt */
    double r[9];          /* measurement noise variances of [t_L, theta_L, v_L] */
    uint32_t history;     /* stored states for the delay compensation, 2..2^20 */
    double r_ref[2];      /* variances of the reference roll and pitch; both 0: no theta_ref rows */
} far_ekf_params;
far_status far_ekf_create(const far_ekf_params* params, double t0, const double x0[9], const double P0[81],
                          far_ekf** out);
far_status far_ekf_destroy(far_ekf* ekf);
far_status far_ekf_predict(far_ekf* ekf, double t, const double acc[3], const double gyro[3]);
far_status far_ekf_update(far_ekf* ekf, double t_meas, const double pose[16], const double v_L[3]);
/*
 * The upsampled update of Sec. III-B (end): the measurement is projected by Eq. 11 and its
 * Kalman gain and covariance update are those of far_ekf_update, but the state correction
 * K y is spread in `cycles` equal shares over as many update cycles: one share now, one
 * after each of the next cycles - 1 far_ekf_predict calls (added after that call's
 * propagation, before its state enters the history), so the odometry moves smoothly
 * instead of jumping at each LiDAR measurement. cycles = 1 is far_ekf_update. A new update
 * first adds the shares still pending at once. Choose cycles so that the shares are added
 * before the next measurement's time stamp: Eq. 11 compares that measurement with the
 * stored state at its time, which holds only the shares added by then.
 * FAR_ERR_INVALID when cycles is outside 1..1000.
 */
far_status far_ekf_update_spread(far_ekf* ekf, double t_meas, const double pose[16], const double v_L[3],
                                 uint32_t cycles);
/* Current time, state, covariance (row-major 9x9) and pose (row-major 4x4); any may be NULL. */
far_status far_ekf_get(const far_ekf* ekf, double* t, double x[9], double P[81], double pose[16]);

#ifdef __cplusplus
}
#endif
#endif /* FAR_H */
