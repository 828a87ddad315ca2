#pragma once
#include "far_internal.cuh"

namespace far {

// One voxel map on the device (the registration map, or the scan-local map
// used for the source covariances, FAR-LIO Sec. III-A.2 "Cov-Calc").
struct DeviceMap {
    Slot* slots = nullptr;
    Slot* slots_alt = nullptr;   // rebuild target (registration map only)
    u32 cap = 0, mask = 0;
    int key_bits = 0;            // bits of a slot index plus one (sort key incl. sentinel)
    float4* pts = nullptr;
    float4* cov = nullptr;       // null for the scan-local map
    u32* ring = nullptr;
    u32 max_buckets = 0;
    MapCounters* ctr = nullptr;
    u32 nmax = 0, k = 0;
    float v = 0, inv_v = 0, dmin2 = 0;
    // precision variant (registration map only): tv > 0, FP16 covariances, cov == null
    int tv = 0;
    uint2* cov_h4 = nullptr;
    u32* cov_h2 = nullptr;
    int* cexp = nullptr;

    MapView view() const {
        MapView mv;
        mv.slots = slots;
        mv.pts = pts;
        mv.cov = cov;
        mv.ctr = ctr;
        mv.mask = mask;
        mv.nmax = nmax;
        mv.inv_v = inv_v;
        mv.v = v;
        mv.tv = tv;
        mv.cov_h4 = cov_h4;
        mv.cov_h2 = cov_h2;
        mv.cexp = cexp;
        return mv;
    }
};

// Per-scan scratch, sized once for the largest accepted scan.
struct Scratch {
    u32 max_n = 0;
    void* staging = nullptr;
    size_t staging_bytes = 0;
    float4* in4 = nullptr;     // packed input points, w = input index
    float4* world = nullptr;   // keyed points (map frame), by input index
    u64* keys = nullptr;
    u32 *sk = nullptr, *sv = nullptr, *sk_alt = nullptr, *sv_alt = nullptr;
    u32 *flags = nullptr, *gstart = nullptr;
    u32 *gsize = nullptr, *gslot = nullptr;       // by group: size and hash slot
    u32 *slot_cnt = nullptr, *slot_base = nullptr;  // by hash slot (both maps): batch counts, group bases
    u32 *admitted = nullptr, *rank = nullptr, *pos = nullptr, *added = nullptr;
    // voxel-grouped order of the admitted points: voxels ordered by their first input index,
    // points of a voxel in input order (deterministic, and follows the scan's spatial order)
    u32 *head_ord = nullptr;   // by input index: ordinal of the voxel whose first candidate it is
    u32 *grp_cnt = nullptr;    // by voxel ordinal: points admitted by this batch -> exclusive prefix
    u32 *a_ord = nullptr;      // by input index: voxel ordinal of an admitted point
    u32 *a_j = nullptr;        // by input index: position among the voxel's points admitted by this batch
    u32 *dest = nullptr;       // by input index: position of an admitted point in the grouped order
    u32* partials = nullptr;
    u32* scal = nullptr;       // device scalars, see SCAL_*
    // registration sources
    float4 *src = nullptr, *src_cov = nullptr;
    u32* src_index = nullptr;
    // stage outputs
    u32* knn_ids = nullptr;
    int32_t* i32_out = nullptr;
    float* f32_out = nullptr;
    int64_t* i64_out = nullptr;
    // Gauss-Newton
    double* gn_partials = nullptr;
    u32 max_gn_blocks = 0;
    RegState* st = nullptr;
    // diagnostics
    u32* touched = nullptr;              // one flag per registration-map slot
    unsigned long long* foot = nullptr;  // footprint counters
    // precision variant only (null otherwise)
    float4* cov_tmp = nullptr;           // FP32 covariances of added points, 2 per point (grouped order)
    u64* added_key = nullptr;            // voxel key of each added point (grouped order)
    u32* grp_bucket = nullptr;           // by voxel ordinal: bucket, count before the insert, old exponent
    u32* grp_cnt0 = nullptr;
    int* grp_exp0 = nullptr;
    uint2* src_h4 = nullptr;             // FP16 source covariances (see far_internal.cuh)
    u32* src_h2 = nullptr;
    signed char* src_exp = nullptr;      // exponent of each source's scan-local voxel
};

// SCAL_IDBASE: the map's next point id when the insert began (the first id it assigns)
// SCAL_NBIG: groups above ADMIT_BIG members (listed by k_group_sort, admitted by whole blocks);
// SCAL_BIGNEXT: the next of them a block of k_admit claims
// SCAL_NHUGE: groups above GS_BLOCK_MIN members (listed by k_group_alloc, sorted by whole blocks
// of k_group_sort); SCAL_HUGENEXT: the next of them a block claims
enum { SCAL_NGROUPS = 0, SCAL_NADMIT = 1, SCAL_NVALID = 2, SCAL_IDBASE = 3, SCAL_NBIG = 4, SCAL_BIGNEXT = 5,
       SCAL_NHUGE = 6, SCAL_HUGENEXT = 7, SCAL_COUNT = 8 };

struct InsertCfg {
    int asmd = 0;
    double sx = 0, sy = 0, sz = 0;  // sensor position (ignored when a device pose is given)
    double rc2 = 0;                 // r_near^2
    double r_max = 1;
};

// Pose of an insert kept on the device (the result of a registration): the map
// transform and the sensor position are read from T, and nothing is inserted
// unless *status == 0.
struct DevicePose {
    const double* T = nullptr;      // row-major 4x4
    const u32* status = nullptr;
};

struct Pose12 {
    double m[12];
};

// Motion of the LiDAR during a sweep (Sec. III-A.1): angular and linear velocity in the LiDAR
// frame as lines in the time tau relative to the reference time, w(tau) = w0 + w1 tau,
// v(tau) = v0 + v1 tau (FP32 copies of the caller's values), and the byte offset of each
// record's FP32 tau.
struct SweepMotion {
    float w0[3], w1[3], v0[3], v1[3];
    u32 time_offset;
};

// Pack `n` records of `stride` bytes (first 12 bytes xyz) into s.in4 (w = index), each point
// first moved to the reference time of the sweep: p_ref = exp(integral of the twist from 0 to
// tau) p, the exponential of [phi; rho] = [w0 tau + w1 tau^2 / 2; v0 tau + v1 tau^2 / 2].
cudaError_t pack_points_deskew(const void* src, u32 n, u32 stride, const SweepMotion& mo, float4* out,
                               cudaStream_t st);
// The same de-skew into a dense (n, 3) FP32 array (the stage entry point).
cudaError_t deskew_points(const void* src, u32 n, u32 stride, const SweepMotion& mo, float* out, cudaStream_t st);

// Pack `n` records of `stride` bytes (first 12 bytes xyz) into s.in4 (w = index).
cudaError_t pack_points(const void* src, u32 n, u32 stride, float4* out, cudaStream_t st);

// Events recorded between the parts of an insert (profiling): [0] after keys and slots,
// [1] after the sort, [2] after grouping (and ASMD), [3] after admission, [4] after ids and
// the grouped order, [5] after the covariances of added points.
struct InsertMarks {
    cudaEvent_t ev[6];
};

// Insert the packed points s.in4[0..n) into m (Sec. III-A.3). pose == nullptr keys the
// raw points (scan-local map). Ids start at m.ctr->next_id. With `covariances`, Eq. 1
// covariances of the added points are computed against the updated map. With `emit_sources`
// (scan-local map), the admitted points are also written to s.src / s.src_index in
// voxel-grouped order (s.src[j].w = admission rank).
cudaError_t map_insert_batch(DeviceMap& m, Scratch& s, u32 n, const Pose12* pose, const InsertCfg& cfg,
                             bool covariances, cudaStream_t st, DevicePose dpose = DevicePose(),
                             const InsertMarks* marks = nullptr, bool emit_sources = false);

// Empty the scan-local map m after an insert of n points through scratch s (only the slots that
// insert used), so that it can serve the next scan without a full clear.
cudaError_t map_local_reset(DeviceMap& m, const Scratch& s, u32 n, cudaStream_t st);

// Covariances of the scan-local sources (s.src, written by map_insert_batch on the local map
// with emit_sources) from the local map; knn_ids_out rows are indexed by rank.
cudaError_t make_sources(DeviceMap& local, Scratch& s, u32 n, u32* knn_ids_out, cudaStream_t st);

// Reset a map to empty (keys, counters, free ring).
cudaError_t map_clear(DeviceMap& m, cudaStream_t st);

// Evict voxels whose centre is farther than radius from center (tombstones the slots).
cudaError_t map_evict(DeviceMap& m, const double center[3], double radius, cudaStream_t st,
                      const double* dev_pose = nullptr);
// Re-insert the live slots into the spare slot array and swap (drops tombstones).
cudaError_t map_rebuild(DeviceMap& m, cudaStream_t st);

// Compact live slots into (key, bucket, count) triples (at most cap_out written); *n_out
// receives the number of live slots found.
cudaError_t map_list_slots(const DeviceMap& m, u64* keys, u32* buckets, u32* counts, u32* n_out, u32 cap_out,
                           cudaStream_t st);

// Gather points of the listed buckets into contiguous arrays (offsets = exclusive prefix of counts).
// keys[g] is the voxel key of buckets[g] (precision variant: world coordinates and FP32
// covariances are restored from the tile-relative / FP16 records).
cudaError_t map_gather(const DeviceMap& m, const u32* buckets, const u32* counts, const u32* offsets,
                       const u64* keys, u32 nvox, float4* pts_out, float4* cov_out, cudaStream_t st);

// k-NN and 1-NN of packed queries (stage entry points).
cudaError_t map_knn(const DeviceMap& m, const float4* q, u32 n, u32 k, u32* ids, int32_t* found, cudaStream_t st);
cudaError_t map_nearest(const DeviceMap& m, const float4* q, u32 n, float tau2, int64_t* ids, float* d2,
                        cudaStream_t st);

}  // namespace far
