// C ABI of the registration library (declarations and contracts in include/far.h).
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "far.h"
#include "gicp.cuh"
#include "map.cuh"
#include "primitives.cuh"

using namespace far;

namespace {
std::atomic<unsigned long long> g_launches{0};
}

void far::note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

namespace {

thread_local std::string g_last_error;

// Events of the per-stage timeline (Sec. IV-B reports per-stage runtimes per frame).
enum { EV_INGEST = 0, EV_SOURCES, EV_INSERT, EV_EVICT, EV_END, EV_GN0, EV_COUNT_FIXED = EV_GN0 };
constexpr int MAX_ITERS = 1000;

}  // namespace

void far::set_last_error(const char* msg) { g_last_error = msg ? msg : ""; }

namespace {

far_status fail(far_status s, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return s;
}

#define CK(call)                                                                                     \
    do {                                                                                             \
        cudaError_t e__ = (call);                                                                    \
        if (e__ != cudaSuccess)                                                                      \
            return fail(FAR_ERR_CUDA, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e__), __FILE__, \
                        __LINE__);                                                                   \
    } while (0)

u32 next_pow2(uint64_t x) {
    uint64_t p = 64;
    while (p < x) p <<= 1;
    return (u32)p;
}

int log2_u32(u32 x) {
    int b = 0;
    while ((1u << b) < x) ++b;
    return b;
}

// Planned device allocations of one map (sizes in bytes), shared by create and far_map_bytes.
struct Plan {
    u32 cap, local_cap, max_buckets, local_buckets, max_n, nmax;
    std::vector<std::pair<void**, size_t>> items;
    size_t total = 0;
};

}  // namespace

struct far_map {
    far_map_params p{};
    cudaStream_t stream = nullptr;
    DeviceMap map;
    DeviceMap local;
    Scratch s;
    double* d_cov36 = nullptr;
    MapCounters* h_ctr = nullptr;  // pinned mirrors
    RegState* h_st = nullptr;
    u32* h_scal = nullptr;
    double* h_cov36 = nullptr;
    std::vector<void*> allocs;
    // profiling
    bool profiling = false;
    std::vector<cudaEvent_t> ev;     // EV_COUNT_FIXED + MAX_ITERS + 1
    bool ev_used[EV_COUNT_FIXED] = {};
    u32 gn_launched = 0;
    far_stage_times last{};
    GnArgs last_gn{};                // arguments of the last registration (footprint diagnostics)
    GnArgs* d_args = nullptr;        // device copy of the registration arguments (graph loop)
    GnArgs* h_args = nullptr;        // pinned staging of d_args
    std::vector<GnGraph> gn_graphs;  // instantiated Gauss-Newton loops (grid, lanes, precision)
    bool gn_graph_used = false;      // the last registration ran the graph loop
    // profiling of the two inserts of a scan: [0] the scan-local map (sources), [1] the map
    InsertMarks ins_marks[2] = {};
    cudaEvent_t ins_start[2] = {nullptr, nullptr};
    cudaEvent_t src_end = nullptr;
    bool ins_used[2] = {false, false};
    far_insert_times ins_last[2] = {};
    bool local_dirty = false;        // the scan-local map may hold a scan (see build_sources)
    bool step_pending = false;       // far_process_scan_async launched a step that no wait has collected
    bool step_want_cov = false;      // ... and computed the pose covariance
    // prefetch of the next host scan (far_prefetch_points): two staging buffers filled on a copy
    // stream; a buffer is reused only after the map's stream has packed what it held
    cudaStream_t copy_stream = nullptr;
    void* pre_buf[2] = {nullptr, nullptr};
    cudaEvent_t pre_ready[2] = {nullptr, nullptr};
    cudaEvent_t pre_used[2] = {nullptr, nullptr};
    bool pre_used_recorded[2] = {false, false};
    const void* pre_ptr[2] = {nullptr, nullptr};   // the host array each buffer holds (null: none pending)
    uint64_t pre_n[2] = {0, 0};
    uint32_t pre_stride[2] = {0, 0}, pre_width[2] = {0, 0};
    int pre_last = 1;                              // the buffer filled last
};

namespace {

far_status validate_params(const far_map_params* p) {
    if (!p) return fail(FAR_ERR_INVALID, "params is NULL");
    if (!(p->voxel_size > 0.0f) || !std::isfinite(p->voxel_size))
        return fail(FAR_ERR_INVALID, "voxel_size must be finite and > 0");
    if (p->max_pts_per_voxel < 1 || p->max_pts_per_voxel > (u32)NMAX_LIMIT)
        return fail(FAR_ERR_INVALID, "max_pts_per_voxel must be in 1..%d", NMAX_LIMIT);
    if (p->k_cov < 1 || p->k_cov > (u32)KMAX) return fail(FAR_ERR_INVALID, "k_cov must be in 1..%d", KMAX);
    if (p->max_voxels < 1) return fail(FAR_ERR_INVALID, "max_voxels must be >= 1");
    if (!(p->load_factor >= 0.05f && p->load_factor <= 0.95f))
        return fail(FAR_ERR_INVALID, "load_factor must be in [0.05, 0.95]");
    if (p->max_scan_points < 1 || p->max_scan_points > (1u << 26))
        return fail(FAR_ERR_INVALID, "max_scan_points must be in 1..2^26");
    if (p->precision_mode > 1) return fail(FAR_ERR_INVALID, "precision_mode %u is not supported", p->precision_mode);
    if (p->precision_mode == 1) {
        // 50 m tiles: the voxel size must divide the tile
        const double r = 50.0 / (double)p->voxel_size;
        const long tv = std::lround(r);
        if (tv < 1 || std::fabs(r - (double)tv) > 1e-9 * r || tv > (1 << 20))
            return fail(FAR_ERR_INVALID, "precision_mode 1 needs a voxel size that divides 50 m (got %g)",
                        (double)p->voxel_size);
    }
    if ((double)p->max_voxels * p->max_pts_per_voxel >= 4294967295.0)
        return fail(FAR_ERR_INVALID, "max_voxels * max_pts_per_voxel must stay below 2^32");
    if ((double)p->max_voxels / p->load_factor > 2147483648.0)
        return fail(FAR_ERR_INVALID, "hash table would exceed 2^31 slots");
    if (!std::isfinite(p->min_spacing)) return fail(FAR_ERR_INVALID, "min_spacing must be finite");
    return FAR_OK;
}

Plan make_plan(const far_map_params& p, far_map* m) {
    Plan pl;
    pl.max_n = p.max_scan_points;
    pl.nmax = p.max_pts_per_voxel;
    pl.max_buckets = (u32)p.max_voxels;
    pl.cap = next_pow2((uint64_t)std::ceil((double)p.max_voxels / p.load_factor));
    pl.local_buckets = pl.max_n;
    pl.local_cap = next_pow2((uint64_t)pl.max_n * 2);
    const size_t n = pl.max_n;
    const size_t partials = 2 * scan_blocks(pl.max_n) + 2;   // scan_exclusive2: two jobs
    const size_t slots_max = std::max<size_t>(pl.cap, pl.local_cap) + 1;
    static far_map dummy;
    far_map* t = m ? m : &dummy;
    auto add = [&](void** ptr, size_t bytes) {
        bytes = (bytes + 255) & ~(size_t)255;
        pl.items.push_back({ptr, bytes});
        pl.total += bytes;
    };
    // registration map
    add((void**)&t->map.slots, (size_t)pl.cap * sizeof(Slot));
    add((void**)&t->map.slots_alt, (size_t)pl.cap * sizeof(Slot));
    add((void**)&t->map.pts, (size_t)pl.max_buckets * pl.nmax * sizeof(float4));
    const bool prec = p.precision_mode == 1;
    if (prec) {
        // FP16 covariances (12 B per point) and one exponent per voxel
        add((void**)&t->map.cov_h4, (size_t)pl.max_buckets * pl.nmax * sizeof(uint2));
        add((void**)&t->map.cov_h2, (size_t)pl.max_buckets * pl.nmax * sizeof(u32));
        add((void**)&t->map.cexp, (size_t)pl.max_buckets * sizeof(int));
    } else {
        add((void**)&t->map.cov, (size_t)pl.max_buckets * pl.nmax * 2 * sizeof(float4));
    }
    add((void**)&t->map.ring, (size_t)pl.max_buckets * sizeof(u32));
    add((void**)&t->map.ctr, sizeof(MapCounters));
    // scan-local map
    add((void**)&t->local.slots, (size_t)pl.local_cap * sizeof(Slot));
    add((void**)&t->local.pts, (size_t)pl.local_buckets * pl.nmax * sizeof(float4));
    add((void**)&t->local.ring, (size_t)pl.local_buckets * sizeof(u32));
    add((void**)&t->local.ctr, sizeof(MapCounters));
    // scratch
    add(&t->s.staging, n * 32);
    add((void**)&t->s.in4, n * sizeof(float4));
    add((void**)&t->s.world, n * sizeof(float4));
    add((void**)&t->s.keys, n * sizeof(u64));
    for (u32** a : {&t->s.sk, &t->s.sv, &t->s.sk_alt, &t->s.sv_alt, &t->s.flags, &t->s.gsize, &t->s.gslot, &t->s.admitted,
                    &t->s.rank, &t->s.pos, &t->s.added, &t->s.src_index, &t->s.head_ord, &t->s.grp_cnt,
                    &t->s.a_ord, &t->s.a_j, &t->s.dest})
        add((void**)a, (n + 1) * sizeof(u32));
    add((void**)&t->s.gstart, (n + 2) * sizeof(u32));
    add((void**)&t->s.slot_cnt, slots_max * sizeof(u32));
    add((void**)&t->s.slot_base, slots_max * sizeof(u32));
    add((void**)&t->s.partials, partials * sizeof(u32));
    add((void**)&t->s.scal, SCAL_COUNT * sizeof(u32));
    add((void**)&t->s.src, n * sizeof(float4));
    add((void**)&t->s.src_cov, n * 2 * sizeof(float4));
    add((void**)&t->s.knn_ids, n * KMAX * sizeof(u32));
    add((void**)&t->s.i32_out, n * sizeof(int32_t));
    add((void**)&t->s.f32_out, n * 6 * sizeof(float));
    add((void**)&t->s.i64_out, n * sizeof(int64_t));
    add((void**)&t->s.gn_partials, gn_partials_doubles(pl.max_n) * sizeof(double));
    add((void**)&t->s.st, sizeof(RegState));
    add((void**)&t->d_args, sizeof(GnArgs));
    add((void**)&t->d_cov36, 36 * sizeof(double));
    add((void**)&t->s.touched, (size_t)pl.cap * sizeof(u32));
    add((void**)&t->s.foot, 2 * sizeof(unsigned long long));
    if (prec) {
        add((void**)&t->s.cov_tmp, n * 2 * sizeof(float4));
        add((void**)&t->s.added_key, n * sizeof(u64));
        add((void**)&t->s.grp_bucket, (n + 1) * sizeof(u32));
        add((void**)&t->s.grp_cnt0, (n + 1) * sizeof(u32));
        add((void**)&t->s.grp_exp0, (n + 1) * sizeof(int));
        add((void**)&t->s.src_h4, n * sizeof(uint2));
        add((void**)&t->s.src_h2, n * sizeof(u32));
        add((void**)&t->s.src_exp, n);
    }
    return pl;
}

void release(far_map* m) {
    if (!m) return;
    if (m->stream) cudaStreamSynchronize(m->stream);
    if (m->copy_stream) {
        cudaStreamSynchronize(m->copy_stream);
        cudaStreamDestroy(m->copy_stream);
        m->copy_stream = nullptr;
    }
    for (int b = 0; b < 2; ++b) {
        if (m->pre_buf[b]) cudaFree(m->pre_buf[b]);
        if (m->pre_ready[b]) cudaEventDestroy(m->pre_ready[b]);
        if (m->pre_used[b]) cudaEventDestroy(m->pre_used[b]);
        m->pre_buf[b] = nullptr;
        m->pre_ready[b] = m->pre_used[b] = nullptr;
    }
    for (cudaEvent_t e : m->ev) cudaEventDestroy(e);
    m->ev.clear();
    for (int w = 0; w < 2; ++w) {
        if (m->ins_start[w]) cudaEventDestroy(m->ins_start[w]);
        for (cudaEvent_t e : m->ins_marks[w].ev)
            if (e) cudaEventDestroy(e);
    }
    if (m->src_end) cudaEventDestroy(m->src_end);
    for (void* p : m->allocs) cudaFree(p);
    m->allocs.clear();
    for (GnGraph& g : m->gn_graphs) gn_graph_destroy(&g);
    m->gn_graphs.clear();
    if (m->h_args) cudaFreeHost(m->h_args);
    m->h_args = nullptr;
    if (m->h_ctr) cudaFreeHost(m->h_ctr);
    if (m->h_st) cudaFreeHost(m->h_st);
    if (m->h_scal) cudaFreeHost(m->h_scal);
    if (m->h_cov36) cudaFreeHost(m->h_cov36);
    m->h_ctr = nullptr;
    m->h_st = nullptr;
    m->h_scal = nullptr;
    m->h_cov36 = nullptr;
}

bool finite_pose(const double* T) {
    for (int i = 0; i < 12; ++i)
        if (!std::isfinite(T[i])) return false;
    return true;
}

far_status check_points(const far_map* m, const float* xyz, uint64_t n, uint32_t stride) {
    if (!m) return fail(FAR_ERR_INVALID, "map is NULL");
    if (n > 0 && !xyz) return fail(FAR_ERR_INVALID, "xyz is NULL");
    if (n > 0 && (stride < 12 || stride % 4 != 0))
        return fail(FAR_ERR_INVALID, "stride_bytes must be >= 12 and a multiple of 4");
    if (n > m->p.max_scan_points)
        return fail(FAR_ERR_INVALID, "n = %llu exceeds max_scan_points = %u", (unsigned long long)n,
                    m->p.max_scan_points);
    return FAR_OK;
}

bool is_device_pointer(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// The FP32 copy of a sweep's motion model, checked: finite, and a time offset that lies inside
// the record after x, y, z, 4-byte aligned.
far_status sweep_motion(const far_motion* mo, uint32_t stride, SweepMotion* out) {
    for (int a = 0; a < 3; ++a) {
        const double v[4] = {mo->w0[a], mo->w1[a], mo->v0[a], mo->v1[a]};
        for (double x : v)
            if (!std::isfinite(x)) return fail(FAR_ERR_INVALID, "motion: velocities must be finite");
        out->w0[a] = (float)mo->w0[a];
        out->w1[a] = (float)mo->w1[a];
        out->v0[a] = (float)mo->v0[a];
        out->v1[a] = (float)mo->v1[a];
    }
    if (mo->time_offset_bytes < 12 || mo->time_offset_bytes % 4 != 0 || mo->time_offset_bytes + 4 > stride)
        return fail(FAR_ERR_INVALID, "motion: time_offset_bytes must be a multiple of 4 in [12, stride_bytes - 4]");
    out->time_offset = mo->time_offset_bytes;
    return FAR_OK;
}

// a1: bring the caller's points (host or device, AoS with stride) into s.in4; with a motion
// model, each point is first moved to the sweep's reference time (Sec. III-A.1).
far_status ingest(far_map* m, const float* xyz, u32 n, u32 stride, const far_motion* motion = nullptr) {
    if (n == 0) return FAR_OK;
    SweepMotion mo;
    if (motion) {
        far_status st = sweep_motion(motion, stride, &mo);
        if (st != FAR_OK) return st;
    }
    const void* src = xyz;
    u32 eff = stride;
    const u32 need_width = motion ? mo.time_offset + 4 : 12;
    int used_slot = -1;
    for (int b = 0; b < 2; ++b)
        if (m->pre_ptr[b] == (const void*)xyz && m->pre_n[b] == n && m->pre_stride[b] == stride &&
            m->pre_width[b] >= need_width)
            used_slot = b;
    if (used_slot >= 0) {
        // prefetched on the copy stream (far_prefetch_points): wait for that copy, not for a new one
        CK(cudaStreamWaitEvent(m->stream, m->pre_ready[used_slot], 0));
        src = m->pre_buf[used_slot];
        eff = stride <= 32 ? stride : 32;
        m->pre_ptr[used_slot] = nullptr;
    } else if (!is_device_pointer(xyz)) {
        if (stride <= 32) {
            CK(cudaMemcpyAsync(m->s.staging, xyz, (size_t)n * stride, cudaMemcpyHostToDevice, m->stream));
        } else {
            // copy x, y, z (and the time stamp) of each record into 32-byte staging records
            const u32 width = motion ? mo.time_offset + 4 : 12;
            if (width > 32)
                return fail(FAR_ERR_INVALID, "host records wider than 32 bytes need time_offset_bytes <= 28");
            CK(cudaMemcpy2DAsync(m->s.staging, 32, xyz, stride, width, n, cudaMemcpyHostToDevice, m->stream));
            eff = 32;
        }
        src = m->s.staging;
    }
    if (motion) CK(pack_points_deskew(src, n, eff, mo, m->s.in4, m->stream));
    else CK(pack_points(src, n, eff, m->s.in4, m->stream));
    if (used_slot >= 0) {
        CK(cudaEventRecord(m->pre_used[used_slot], m->stream));
        m->pre_used_recorded[used_slot] = true;
    }
    return FAR_OK;
}

far_status copy_out(void* dst, const void* src, size_t bytes, cudaStream_t st) {
    if (!dst || bytes == 0) return FAR_OK;
    CK(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, st));
    return FAR_OK;
}

far_status check_device_errors(far_map* m, const char* what) {
    const u32 err = m->h_ctr->err;
    if (!err) return FAR_OK;
    CK(cudaMemsetAsync(&m->map.ctr->err, 0, sizeof(u32), m->stream));
    CK(cudaMemsetAsync(&m->map.ctr->n_dropped, 0, sizeof(u32), m->stream));
    return fail(FAR_ERR_CAPACITY, "%s: %s%s%s(%u points dropped)", what, (err & ERR_TABLE_FULL) ? "hash table full; " : "",
                (err & ERR_BUCKETS_FULL) ? "bucket pool exhausted; " : "",
                (err & ERR_ID_OVERFLOW) ? "point ids exhausted; " : "", m->h_ctr->n_dropped);
}

void mark(far_map* m, int e) {
    if (!m->profiling) return;
    cudaEventRecord(m->ev[e], m->stream);
    if (e < EV_COUNT_FIXED) m->ev_used[e] = true;
}

void reset_marks(far_map* m) {
    for (bool& u : m->ev_used) u = false;
    m->gn_launched = 0;
    m->ins_used[0] = m->ins_used[1] = false;
}

// Events around one insert (profiling only); which = 0 scan-local map, 1 registration map.
const InsertMarks* insert_marks(far_map* m, int which) {
    if (!m->profiling) return nullptr;
    cudaEventRecord(m->ins_start[which], m->stream);
    m->ins_used[which] = true;
    return &m->ins_marks[which];
}

void collect_insert_times(far_map* m) {
    for (int w = 0; w < 2; ++w) {
        if (!m->ins_used[w]) continue;
        const InsertMarks& k = m->ins_marks[w];
        float t[6] = {0, 0, 0, 0, 0, 0};
        cudaEventElapsedTime(&t[0], m->ins_start[w], k.ev[0]);
        for (int i = 1; i < 5; ++i) cudaEventElapsedTime(&t[i], k.ev[i - 1], k.ev[i]);
        // the sources' covariances are computed after the local insert (make_sources)
        cudaEventElapsedTime(&t[5], k.ev[4], w == 0 ? m->src_end : k.ev[5]);
        far_insert_times& o = m->ins_last[w];
        o.keys_ms = t[0];
        o.sort_ms = t[1];
        o.group_ms = t[2];
        o.admit_ms = t[3];
        o.ids_ms = t[4];
        o.cov_ms = t[5];
    }
}

float span_ms(far_map* m, int a, int b) {
    float t = 0.f;
    if (cudaEventElapsedTime(&t, m->ev[a], m->ev[b]) != cudaSuccess) {
        cudaGetLastError();
        return 0.f;
    }
    return t;
}

// Fill m->last from the recorded events (after the stream has been synchronised).
void collect_times(far_map* m, u32 iters_done, u32 status) {
    if (!m->profiling) return;
    far_stage_times t{};
    if (m->ev_used[EV_INGEST] && m->ev_used[EV_SOURCES]) t.ingest_ms = span_ms(m, EV_INGEST, EV_SOURCES);
    if (m->ev_used[EV_SOURCES] && m->gn_launched) t.sources_ms = span_ms(m, EV_SOURCES, EV_GN0);
    if (m->gn_launched) {
        t.gauss_newton_ms = span_ms(m, EV_GN0, EV_GN0 + 2 * (int)m->gn_launched);
        u32 working = std::min(m->gn_launched, iters_done + (status != 0 ? 1u : 0u));
        t.gn_launches = working;
        double lin = 0.0, sol = 0.0;
        for (u32 i = 0; i < working; ++i) {
            lin += span_ms(m, EV_GN0 + 2 * (int)i, EV_GN0 + 1 + 2 * (int)i);
            sol += span_ms(m, EV_GN0 + 1 + 2 * (int)i, EV_GN0 + 2 + 2 * (int)i);
        }
        if (working) {
            t.gn_launch_ms = lin / working;
            t.gn_solve_ms = sol / working;
        }
    }
    if (m->ev_used[EV_INSERT] && m->ev_used[EV_EVICT]) t.insert_ms = span_ms(m, EV_INSERT, EV_EVICT);
    if (m->ev_used[EV_EVICT] && m->ev_used[EV_END]) t.evict_ms = span_ms(m, EV_EVICT, EV_END);
    if (m->ev_used[EV_END]) {
        const int first = m->ev_used[EV_INGEST] ? EV_INGEST : (m->gn_launched ? EV_GN0 : EV_INSERT);
        t.total_ms = span_ms(m, first, EV_END);
    }
    m->last = t;
}

// Launch the Gauss-Newton chain (max_iters iterations of linearise + solve). When the loop
// can stop early (conv_eps > 0, or a time budget) and nothing is profiled, it is one launch
// of an instantiated graph whose device-side loop ends at convergence, so no launch follows
// it; a fixed iteration count runs as explicit launches, whose programmatic dependent
// launches overlap better than graph nodes; with profiling, explicit launches marked by
// events (start, the end of each linearisation, the end of each solve).
far_status run_gn(far_map* m, const GnArgs& a, u32 n_upper, u32 iters) {
    m->last_gn = a;
    if (!m->profiling && iters > 0 && (a.conv_eps > 0.0 || a.budget_ns > 0)) {
        const bool prec = a.map.tv > 0;
        const u32 grid = gn_grid(n_upper, a.tpp);
        GnGraph* g = nullptr;
        for (GnGraph& c : m->gn_graphs)
            if (c.grid == grid && c.tpp == gn_tpp(a.tpp) && c.prec == prec) g = &c;
        if (!g) {
            if (m->gn_graphs.size() >= 8) {
                gn_graph_destroy(&m->gn_graphs.front());
                m->gn_graphs.erase(m->gn_graphs.begin());
            }
            GnGraph ng;
            CK(gn_graph_build(m->d_args, n_upper, a.tpp, prec, &ng));
            m->gn_graphs.push_back(ng);
            g = &m->gn_graphs.back();
        }
        // the previous registration's copy has completed: every call ends with a stream sync
        *m->h_args = a;
        m->h_args->max_iters = iters;
        CK(cudaMemcpyAsync(m->d_args, m->h_args, sizeof(GnArgs), cudaMemcpyHostToDevice, m->stream));
        CK(cudaGraphLaunch(g->exec, m->stream));
        m->gn_graph_used = true;
        m->gn_launched = 0;
        return FAR_OK;
    }
    m->gn_graph_used = false;
    mark(m, EV_GN0);
    for (u32 it = 0; it < iters; ++it) {
        u32 nb = 0;
        CK(gn_linearise(a, n_upper, m->stream, &nb));
        mark(m, EV_GN0 + 1 + 2 * (int)it);
        CK(gn_solve(a, nb, m->stream));
        mark(m, EV_GN0 + 2 + 2 * (int)it);
    }
    m->gn_launched = iters;
    return FAR_OK;
}

// Count the kernels the graph loop ran (one linearisation and one solve per trip: every
// trip applies an update, except a final degenerate one).
void account_gn_graph(far_map* m, const RegState& r) {
    if (!m->gn_graph_used) return;
    const u32 trips = r.iters + (r.status == 5 ? 1u : 0u);
    for (u32 i = 0; i < 2 * trips; ++i) note_launch();
    m->gn_graph_used = false;
}

Pose12 pose12(const double* T) {
    Pose12 p;
    for (int i = 0; i < 12; ++i) p.m[i] = T[i];
    return p;
}

// Scan-local map + Eq. 1 source covariances (a2, a3) from s.in4[0..n).
// The scan-local map starts empty (cleared at creation) and is emptied again after each use
// by resetting only the slots the insert used; a build that stopped half-way leaves it dirty,
// and the next one clears it in full.
far_status build_sources(far_map* m, u32 n, u32* knn_ids) {
    if (m->local_dirty) CK(map_clear(m->local, m->stream));
    m->local_dirty = true;
    InsertCfg cfg;
    CK(map_insert_batch(m->local, m->s, n, nullptr, cfg, false, m->stream, DevicePose(), insert_marks(m, 0), true));
    CK(make_sources(m->local, m->s, n, knn_ids, m->stream));
    if (m->profiling) cudaEventRecord(m->src_end, m->stream);
    CK(map_local_reset(m->local, m->s, n, m->stream));
    m->local_dirty = false;
    return FAR_OK;
}

// pose: the initial pose; for the precision variant it fixes the linearisation anchor, the
// corner A = 50 floor(t / 50) of the tile holding the initial position.
GnArgs gn_args(far_map* m, const double* pose, u32 n, float tau, float kappa, double conv_eps, int update,
               int32_t* corr, double budget_s, int tpp = 0) {
    GnArgs a;
    a.tpp = tpp;
    a.max_iters = 0;
    for (int j = 0; j < 3; ++j) {
        a.anchor[j] = 0.0;
        a.ftile[j] = 0;
        if (m->map.tv > 0) {
            // floor(t / 50) exactly (the rounded quotient's floor, corrected by the exact 50 T)
            double T = std::floor(pose[4 * j + 3] / 50.0);
            if (50.0 * T > pose[4 * j + 3]) T -= 1.0;
            else if (50.0 * (T + 1.0) <= pose[4 * j + 3]) T += 1.0;
            a.ftile[j] = (int)T;
            a.anchor[j] = 50.0 * T;
        }
        a.conv_center[j] = pose[4 * j + 3] - a.anchor[j];
    }
    a.src_h4 = m->s.src_h4;
    a.src_h2 = m->s.src_h2;
    a.src_exp = m->s.src_exp;
    a.map = m->map.view();
    a.src = m->s.src;
    a.src_cov = m->s.src_cov;
    a.n_src = m->s.scal + SCAL_NADMIT;
    a.n_max = n;
    a.st = m->s.st;
    a.partials = m->s.gn_partials;
    a.tau2 = tau * tau;
    a.kappa2 = kappa * kappa;
    a.conv_eps = conv_eps;
    a.update = update;
    a.corr_out = corr;
    a.budget_ns = budget_s > 0 ? (unsigned long long)(budget_s * 1e9) : 0ull;
    return a;
}

}  // namespace

extern "C" {

const char* far_status_string(far_status s) {
    switch (s) {
        case FAR_OK: return "FAR_OK";
        case FAR_ERR_INVALID: return "FAR_ERR_INVALID";
        case FAR_ERR_OOM: return "FAR_ERR_OOM";
        case FAR_ERR_CAPACITY: return "FAR_ERR_CAPACITY";
        case FAR_ERR_CUDA: return "FAR_ERR_CUDA";
        case FAR_ERR_DEGENERATE: return "FAR_ERR_DEGENERATE";
        case FAR_ERR_TIMEOUT: return "FAR_ERR_TIMEOUT";
    }
    return "FAR_ERR_UNKNOWN";
}

const char* far_last_error(void) { return g_last_error.c_str(); }

const char* far_version(void) { return "far-gb300 0.1 (sm_103a)"; }

far_status far_map_bytes(const far_map_params* params, uint64_t* out_bytes) {
    far_status st = validate_params(params);
    if (st != FAR_OK) return st;
    if (!out_bytes) return fail(FAR_ERR_INVALID, "out_bytes is NULL");
    Plan pl = make_plan(*params, nullptr);
    *out_bytes = pl.total;
    return FAR_OK;
}

far_status far_map_create(const far_map_params* params, void* cuda_stream, far_map** out) {
    far_status st = validate_params(params);
    if (st != FAR_OK) return st;
    if (!out) return fail(FAR_ERR_INVALID, "out is NULL");
    int ndev = 0;
    cudaError_t de = cudaGetDeviceCount(&ndev);
    if (de != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return fail(FAR_ERR_CUDA, "no usable CUDA device: %s", cudaGetErrorString(de));
    }
    far_map* m = new far_map();
    m->p = *params;
    m->stream = static_cast<cudaStream_t>(cuda_stream);
    Plan pl = make_plan(*params, m);
    for (auto& it : pl.items) {
        void* p = nullptr;
        cudaError_t e = cudaMalloc(&p, it.second);
        if (e != cudaSuccess) {
            cudaGetLastError();
            release(m);
            delete m;
            return fail(FAR_ERR_OOM, "cudaMalloc of %zu bytes failed: %s", it.second, cudaGetErrorString(e));
        }
        *it.first = p;
        m->allocs.push_back(p);
    }
    if (cudaMallocHost((void**)&m->h_ctr, sizeof(MapCounters)) != cudaSuccess ||
        cudaMallocHost((void**)&m->h_st, sizeof(RegState)) != cudaSuccess ||
        cudaMallocHost((void**)&m->h_scal, SCAL_COUNT * sizeof(u32)) != cudaSuccess ||
        cudaMallocHost((void**)&m->h_cov36, 36 * sizeof(double)) != cudaSuccess ||
        cudaMallocHost((void**)&m->h_args, sizeof(GnArgs)) != cudaSuccess) {
        cudaGetLastError();
        release(m);
        delete m;
        return fail(FAR_ERR_OOM, "pinned host allocation failed");
    }
    const float v = params->voxel_size;
    const u32 nmax = params->max_pts_per_voxel;
    float dmin = params->min_spacing < 0.0f ? (float)((double)v / std::sqrt((double)nmax)) : params->min_spacing;
    for (DeviceMap* d : {&m->map, &m->local}) {
        d->nmax = nmax;
        d->k = params->k_cov;
        d->v = v;
        d->inv_v = 1.0f / v;
        d->dmin2 = dmin * dmin;
    }
    if (params->precision_mode == 1) m->map.tv = (int)std::lround(50.0 / (double)v);
    m->map.cap = pl.cap;
    m->map.mask = pl.cap - 1;
    m->map.key_bits = log2_u32(pl.cap) + 1;
    m->map.max_buckets = pl.max_buckets;
    m->local.cap = pl.local_cap;
    m->local.mask = pl.local_cap - 1;
    m->local.key_bits = log2_u32(pl.local_cap) + 1;
    m->local.max_buckets = pl.local_buckets;
    m->local.cov = nullptr;
    m->local.slots_alt = nullptr;
    m->s.max_n = pl.max_n;
    m->s.staging_bytes = (size_t)pl.max_n * 32;
    m->s.max_gn_blocks = (u32)(gn_partials_doubles(pl.max_n) / 32);
    cudaError_t e = map_clear(m->map, m->stream);
    if (e == cudaSuccess) e = map_clear(m->local, m->stream);
    // per-slot batch counters start at zero (every insert leaves them zero)
    if (e == cudaSuccess)
        e = cudaMemsetAsync(m->s.slot_cnt, 0, (std::max<size_t>(pl.cap, pl.local_cap) + 1) * sizeof(u32), m->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
    if (e != cudaSuccess) {
        release(m);
        delete m;
        return fail(FAR_ERR_CUDA, "map initialisation failed: %s", cudaGetErrorString(e));
    }
    *out = m;
    return FAR_OK;
}

far_status far_map_destroy(far_map* map) {
    if (!map) return fail(FAR_ERR_INVALID, "map is NULL");
    release(map);
    delete map;
    return FAR_OK;
}

far_status far_map_clear(far_map* map) {
    if (!map) return fail(FAR_ERR_INVALID, "map is NULL");
    CK(map_clear(map->map, map->stream));
    CK(cudaStreamSynchronize(map->stream));
    return FAR_OK;
}

far_status far_map_insert(far_map* map, const float* xyz, uint64_t n, uint32_t stride_bytes, const double pose[16],
                          const far_insert_params* params, uint64_t* n_inserted) {
    far_status st = check_points(map, xyz, n, stride_bytes);
    if (st != FAR_OK) return st;
    if (!pose || !finite_pose(pose)) return fail(FAR_ERR_INVALID, "pose is NULL or not finite");
    InsertCfg cfg;
    if (params && params->asmd) {
        if (!(params->r_max > 0.0) || !(params->r_near >= 0.0) || !std::isfinite(params->r_max))
            return fail(FAR_ERR_INVALID, "ASMD needs r_near >= 0 and finite r_max > 0");
        cfg.asmd = 1;
        cfg.rc2 = params->r_near * params->r_near;
        cfg.r_max = params->r_max;
    }
    cfg.sx = pose[3];
    cfg.sy = pose[7];
    cfg.sz = pose[11];
    if ((st = ingest(map, xyz, (u32)n, stride_bytes)) != FAR_OK) return st;
    Pose12 T = pose12(pose);
    CK(map_insert_batch(map->map, map->s, (u32)n, &T, cfg, true, map->stream));
    CK(cudaMemcpyAsync(map->h_ctr, map->map.ctr, sizeof(MapCounters), cudaMemcpyDeviceToHost, map->stream));
    CK(cudaStreamSynchronize(map->stream));
    if (n_inserted) *n_inserted = map->h_ctr->n_added;
    return check_device_errors(map, "far_map_insert");
}

far_status far_map_evict(far_map* map, const double center[3], double radius, uint64_t* n_removed) {
    if (!map || !center) return fail(FAR_ERR_INVALID, "map or center is NULL");
    if (!(radius >= 0.0) || !std::isfinite(center[0]) || !std::isfinite(center[1]) || !std::isfinite(center[2]))
        return fail(FAR_ERR_INVALID, "radius must be >= 0 and center finite");
    CK(map_evict(map->map, center, radius, map->stream));
    CK(cudaMemcpyAsync(map->h_ctr, map->map.ctr, sizeof(MapCounters), cudaMemcpyDeviceToHost, map->stream));
    CK(cudaStreamSynchronize(map->stream));
    if (n_removed) *n_removed = map->h_ctr->removed;
    if (map->h_ctr->n_tomb > map->map.cap / 4) {
        CK(map_rebuild(map->map, map->stream));
        CK(cudaStreamSynchronize(map->stream));
    }
    return FAR_OK;
}

far_status far_map_size(const far_map* map, uint64_t* n_voxels, uint64_t* n_points) {
    if (!map) return fail(FAR_ERR_INVALID, "map is NULL");
    CK(cudaMemcpyAsync(map->h_ctr, map->map.ctr, sizeof(MapCounters), cudaMemcpyDeviceToHost, map->stream));
    CK(cudaStreamSynchronize(map->stream));
    if (n_voxels) *n_voxels = map->h_ctr->n_voxels;
    if (n_points) *n_points = map->h_ctr->n_points;
    return FAR_OK;
}

far_status far_map_export(const far_map* cmap, int32_t* keys, uint32_t* counts, uint32_t* ids, float* xyz,
                          float* cov, uint8_t* valid, uint64_t cap_voxels, uint64_t cap_points) {
    far_map* map = const_cast<far_map*>(cmap);
    if (!map || !keys || !counts) return fail(FAR_ERR_INVALID, "map, keys or counts is NULL");
    uint64_t nv = 0, np = 0;
    far_status st = far_map_size(map, &nv, &np);
    if (st != FAR_OK) return st;
    if (nv > cap_voxels || np > cap_points) return fail(FAR_ERR_INVALID, "export buffers too small");
    if (nv == 0) return FAR_OK;
    u64* d_keys = nullptr;
    u32 *d_buckets = nullptr, *d_counts = nullptr, *d_n = nullptr, *d_off = nullptr;
    float4 *d_pts = nullptr, *d_cov = nullptr;
    auto cleanup = [&]() {
        cudaFree(d_keys); cudaFree(d_buckets); cudaFree(d_counts); cudaFree(d_n); cudaFree(d_off);
        cudaFree(d_pts); cudaFree(d_cov);
    };
    if (cudaMalloc(&d_keys, nv * sizeof(u64)) != cudaSuccess || cudaMalloc(&d_buckets, nv * sizeof(u32)) != cudaSuccess ||
        cudaMalloc(&d_counts, nv * sizeof(u32)) != cudaSuccess || cudaMalloc(&d_n, sizeof(u32)) != cudaSuccess ||
        cudaMalloc(&d_off, nv * sizeof(u32)) != cudaSuccess ||
        cudaMalloc(&d_pts, std::max<uint64_t>(np, 1) * sizeof(float4)) != cudaSuccess ||
        cudaMalloc(&d_cov, std::max<uint64_t>(np, 1) * 2 * sizeof(float4)) != cudaSuccess) {
        cudaGetLastError();
        cleanup();
        return fail(FAR_ERR_OOM, "export scratch allocation failed");
    }
    std::vector<u64> hk(nv);
    std::vector<u32> hb(nv), hc(nv);
    u32 hn = 0;
    cudaError_t e = map_list_slots(map->map, d_keys, d_buckets, d_counts, d_n, (u32)nv, map->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hn, d_n, sizeof(u32), cudaMemcpyDeviceToHost, map->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(map->stream);
    if (e == cudaSuccess && hn > nv) e = cudaErrorInvalidValue;
    if (e == cudaSuccess) e = cudaMemcpy(hk.data(), d_keys, hn * sizeof(u64), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(hb.data(), d_buckets, hn * sizeof(u32), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(hc.data(), d_counts, hn * sizeof(u32), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) {
        cleanup();
        return fail(FAR_ERR_CUDA, "export listing failed: %s", cudaGetErrorString(e));
    }
    auto unpack = [](u64 k, int32_t* o) {
        o[0] = (int32_t)((k >> 42) & 0x1FFFFF) - (1 << 20);
        o[1] = (int32_t)((k >> 21) & 0x1FFFFF) - (1 << 20);
        o[2] = (int32_t)(k & 0x1FFFFF) - (1 << 20);
    };
    std::vector<u32> order(hn);
    for (u32 i = 0; i < hn; ++i) order[i] = i;
    std::vector<int32_t> kk(3 * (size_t)hn);
    for (u32 i = 0; i < hn; ++i) unpack(hk[i], &kk[3 * (size_t)i]);
    std::sort(order.begin(), order.end(), [&](u32 a, u32 b) {
        const int32_t* x = &kk[3 * (size_t)a];
        const int32_t* y = &kk[3 * (size_t)b];
        if (x[0] != y[0]) return x[0] < y[0];
        if (x[1] != y[1]) return x[1] < y[1];
        return x[2] < y[2];
    });
    std::vector<u32> sb(hn), sc(hn), so(hn);
    std::vector<u64> sk(hn);
    u32 total = 0;
    for (u32 i = 0; i < hn; ++i) {
        sb[i] = hb[order[i]];
        sc[i] = hc[order[i]];
        sk[i] = hk[order[i]];
        so[i] = total;
        total += sc[i];
        std::memcpy(keys + 3 * (size_t)i, &kk[3 * (size_t)order[i]], 3 * sizeof(int32_t));
        counts[i] = sc[i];
    }
    if (total > np) {
        cleanup();
        return fail(FAR_ERR_CUDA, "export: listed %u points but the map counts %llu", total, (unsigned long long)np);
    }
    std::vector<float4> hp(total), hcv(2 * (size_t)total);
    e = cudaMemcpy(d_buckets, sb.data(), hn * sizeof(u32), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(d_counts, sc.data(), hn * sizeof(u32), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(d_off, so.data(), hn * sizeof(u32), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(d_keys, sk.data(), hn * sizeof(u64), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = map_gather(map->map, d_buckets, d_counts, d_off, d_keys, hn, d_pts, d_cov, map->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(map->stream);
    if (e == cudaSuccess && total) e = cudaMemcpy(hp.data(), d_pts, total * sizeof(float4), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && total)
        e = cudaMemcpy(hcv.data(), d_cov, total * 2 * sizeof(float4), cudaMemcpyDeviceToHost);
    cleanup();
    if (e != cudaSuccess) return fail(FAR_ERR_CUDA, "export gather failed: %s", cudaGetErrorString(e));
    for (u32 i = 0; i < total; ++i) {
        const float4 p = hp[i];
        u32 id;
        std::memcpy(&id, &p.w, 4);
        if (ids) ids[i] = id;
        if (xyz) {
            xyz[3 * (size_t)i] = p.x;
            xyz[3 * (size_t)i + 1] = p.y;
            xyz[3 * (size_t)i + 2] = p.z;
        }
        const float4 c0 = hcv[2 * (size_t)i], c1 = hcv[2 * (size_t)i + 1];
        if (cov) {
            float* o = cov + 6 * (size_t)i;
            o[0] = c0.x; o[1] = c0.y; o[2] = c0.z; o[3] = c0.w; o[4] = c1.x; o[5] = c1.y;
        }
        if (valid) valid[i] = c1.z > 0.5f ? 1 : 0;
    }
    return FAR_OK;
}

far_status far_map_nearest(far_map* map, const float* q, uint64_t n, uint32_t stride_bytes, float tau,
                           int64_t* out_ids, float* out_d2) {
    far_status st = check_points(map, q, n, stride_bytes);
    if (st != FAR_OK) return st;
    if (n > 0 && !out_ids) return fail(FAR_ERR_INVALID, "out_ids is NULL");
    if (n == 0) return FAR_OK;
    if ((st = ingest(map, q, (u32)n, stride_bytes)) != FAR_OK) return st;
    const float tau2 = tau * tau;
    CK(map_nearest(map->map, map->s.in4, (u32)n, tau2, map->s.i64_out, map->s.f32_out, map->stream));
    if ((st = copy_out(out_ids, map->s.i64_out, n * sizeof(int64_t), map->stream)) != FAR_OK) return st;
    if ((st = copy_out(out_d2, map->s.f32_out, n * sizeof(float), map->stream)) != FAR_OK) return st;
    CK(cudaStreamSynchronize(map->stream));
    return FAR_OK;
}

far_status far_map_knn(far_map* map, const float* q, uint64_t n, uint32_t stride_bytes, uint32_t k,
                       uint32_t* out_ids, int32_t* out_found) {
    far_status st = check_points(map, q, n, stride_bytes);
    if (st != FAR_OK) return st;
    if (k < 1 || k > (u32)KMAX) return fail(FAR_ERR_INVALID, "k must be in 1..%d", KMAX);
    if (n > 0 && (!out_ids || !out_found)) return fail(FAR_ERR_INVALID, "outputs are NULL");
    if (n == 0) return FAR_OK;
    if ((st = ingest(map, q, (u32)n, stride_bytes)) != FAR_OK) return st;
    CK(map_knn(map->map, map->s.in4, (u32)n, k, map->s.knn_ids, map->s.i32_out, map->stream));
    if ((st = copy_out(out_ids, map->s.knn_ids, n * k * sizeof(u32), map->stream)) != FAR_OK) return st;
    if ((st = copy_out(out_found, map->s.i32_out, n * sizeof(int32_t), map->stream)) != FAR_OK) return st;
    CK(cudaStreamSynchronize(map->stream));
    return FAR_OK;
}

}  // extern "C"

namespace far {
cudaError_t export_sources(const Scratch& s, u32 n, int64_t* index, float* cov6, uint8_t* valid, cudaStream_t st);
}

extern "C" {

far_status far_scan_sources(far_map* map, const float* xyz, uint64_t n, uint32_t stride_bytes, int64_t* out_index,
                            float* out_cov, uint8_t* out_valid, uint32_t* out_knn_ids, uint64_t* n_src) {
    far_status st = check_points(map, xyz, n, stride_bytes);
    if (st != FAR_OK) return st;
    if (n == 0) {
        if (n_src) *n_src = 0;
        return FAR_OK;
    }
    if ((st = ingest(map, xyz, (u32)n, stride_bytes)) != FAR_OK) return st;
    if ((st = build_sources(map, (u32)n, map->s.knn_ids)) != FAR_OK) return st;
    uint8_t* vbuf = reinterpret_cast<uint8_t*>(map->s.i32_out);
    CK(export_sources(map->s, (u32)n, map->s.i64_out, map->s.f32_out, vbuf, map->stream));
    CK(cudaMemcpyAsync(map->h_scal, map->s.scal, SCAL_COUNT * sizeof(u32), cudaMemcpyDeviceToHost, map->stream));
    CK(cudaStreamSynchronize(map->stream));
    const uint64_t m = map->h_scal[SCAL_NADMIT];
    if ((st = copy_out(out_index, map->s.i64_out, m * sizeof(int64_t), map->stream)) != FAR_OK) return st;
    if ((st = copy_out(out_cov, map->s.f32_out, m * 6 * sizeof(float), map->stream)) != FAR_OK) return st;
    if ((st = copy_out(out_valid, vbuf, m, map->stream)) != FAR_OK) return st;
    if ((st = copy_out(out_knn_ids, map->s.knn_ids, m * map->p.k_cov * sizeof(u32), map->stream)) != FAR_OK) return st;
    CK(cudaStreamSynchronize(map->stream));
    if (n_src) *n_src = m;
    return FAR_OK;
}

far_status far_linearize(far_map* map, const float* xyz, uint64_t n, uint32_t stride_bytes, const double pose[16],
                         float tau, float kappa, uint32_t threads_per_point, double out_H[36], double out_g[6],
                         int32_t* out_corr, far_reg_stats* stats) {
    far_status st = check_points(map, xyz, n, stride_bytes);
    if (st != FAR_OK) return st;
    if (!pose || !finite_pose(pose) || !out_H || !out_g) return fail(FAR_ERR_INVALID, "pose/H/g invalid");
    if (!(kappa > 0.0f) || !(tau >= 0.0f)) return fail(FAR_ERR_INVALID, "kappa must be > 0 and tau >= 0");
    const u32 nn = (u32)n;
    if ((st = ingest(map, xyz, nn, stride_bytes)) != FAR_OK) return st;
    if (nn) {
        if ((st = build_sources(map, nn, nullptr)) != FAR_OK) return st;
    } else {
        CK(cudaMemsetAsync(map->s.scal, 0, SCAL_COUNT * sizeof(u32), map->stream));
    }
    CK(gn_begin(map->s.st, pose, map->s.scal + SCAL_NADMIT, map->stream));
    GnArgs a = gn_args(map, pose, std::max(nn, 1u), tau, kappa, 0.0, 0, map->s.i32_out, 0.0, (int)threads_per_point);
    reset_marks(map);
    if ((st = run_gn(map, a, std::max(nn, 1u), 1)) != FAR_OK) return st;
    mark(map, EV_END);
    CK(cudaMemcpyAsync(map->h_st, map->s.st, sizeof(RegState), cudaMemcpyDeviceToHost, map->stream));
    CK(cudaMemcpyAsync(map->h_scal, map->s.scal, SCAL_COUNT * sizeof(u32), cudaMemcpyDeviceToHost, map->stream));
    CK(cudaStreamSynchronize(map->stream));
    collect_times(map, 0, 1);
    const uint64_t m = map->h_st->n_src;
    if ((st = copy_out(out_corr, map->s.i32_out, m * sizeof(int32_t), map->stream)) != FAR_OK) return st;
    CK(cudaStreamSynchronize(map->stream));
    std::memcpy(out_H, map->h_st->H, 36 * sizeof(double));
    std::memcpy(out_g, map->h_st->g, 6 * sizeof(double));
    if (stats) {
        stats->iters = 0;
        stats->n_src = (uint32_t)m;
        stats->n_corr = map->h_st->n_corr;
        stats->n_p2p = map->h_st->n_p2p;
        stats->converged = 0;
        stats->status = FAR_OK;
        stats->chi2 = map->h_st->chi2;
    }
    return FAR_OK;
}

far_status far_register_scan(far_map* map, const float* xyz, uint64_t n, uint32_t stride_bytes,
                             const double init_pose[16], const far_reg_params* params, double out_pose[16],
                             double out_cov[36], far_reg_stats* stats) {
    far_status st = check_points(map, xyz, n, stride_bytes);
    if (st != FAR_OK) return st;
    if (!params || !init_pose || !finite_pose(init_pose) || !out_pose)
        return fail(FAR_ERR_INVALID, "params, init_pose or out_pose invalid");
    if (!(params->kappa > 0.0f) || !(params->tau >= 0.0f) || params->max_iters > 1000)
        return fail(FAR_ERR_INVALID, "kappa must be > 0, tau >= 0, max_iters <= 1000");
    const u32 nn = (u32)n;
    reset_marks(map);
    mark(map, EV_INGEST);
    if ((st = ingest(map, xyz, nn, stride_bytes)) != FAR_OK) return st;
    mark(map, EV_SOURCES);
    if (nn) {
        if ((st = build_sources(map, nn, nullptr)) != FAR_OK) return st;
    } else {
        CK(cudaMemsetAsync(map->s.scal, 0, SCAL_COUNT * sizeof(u32), map->stream));
    }
    CK(gn_begin(map->s.st, init_pose, map->s.scal + SCAL_NADMIT, map->stream));
    GnArgs a = gn_args(map, init_pose, std::max(nn, 1u), params->tau, params->kappa, params->conv_eps, 1, nullptr,
                       params->time_budget_s, (int)params->threads_per_point);
    if ((st = run_gn(map, a, std::max(nn, 1u), params->max_iters)) != FAR_OK) return st;
    mark(map, EV_END);
    if (out_cov) CK(gn_covariance(map->s.st, map->d_cov36, map->stream));
    CK(cudaMemcpyAsync(map->h_st, map->s.st, sizeof(RegState), cudaMemcpyDeviceToHost, map->stream));
    CK(cudaMemcpyAsync(map->h_scal, map->s.scal, SCAL_COUNT * sizeof(u32), cudaMemcpyDeviceToHost, map->stream));
    if (out_cov) CK(cudaMemcpyAsync(map->h_cov36, map->d_cov36, 36 * sizeof(double), cudaMemcpyDeviceToHost, map->stream));
    CK(cudaStreamSynchronize(map->stream));
    const RegState& r = *map->h_st;
    account_gn_graph(map, r);
    collect_times(map, r.iters, r.status);
    if (map->profiling) collect_insert_times(map);
    std::memcpy(out_pose, r.T, 16 * sizeof(double));
    if (out_cov) std::memcpy(out_cov, map->h_cov36, 36 * sizeof(double));
    far_status result = FAR_OK;
    if (r.status == 5) result = fail(FAR_ERR_DEGENERATE, "registration degenerate (%u correspondences)", r.n_corr);
    if (r.status == 6) result = fail(FAR_ERR_TIMEOUT, "registration exceeded its time budget after %u iterations", r.iters);
    if (r.status == 7) result = fail(FAR_ERR_CUDA, "internal: the Gauss-Newton loop ran past its iteration limit");
    if (stats) {
        stats->iters = r.iters;
        stats->n_src = r.n_src;
        stats->n_corr = r.n_corr;
        stats->n_p2p = r.n_p2p;
        stats->converged = (int32_t)r.converged;
        stats->status = result;
        stats->chi2 = r.chi2;
    }
    return result;
}

far_status far_prefetch_points(far_map* map, const float* xyz, uint64_t n, uint32_t stride_bytes) {
    far_status st = check_points(map, xyz, n, stride_bytes);
    if (st != FAR_OK) return st;
    if (n == 0 || is_device_pointer(xyz)) return FAR_OK;   // nothing to copy ahead
    if (!map->copy_stream) {
        // set up once: a copy stream, two staging buffers of the map's largest scan, four events
        const size_t bytes = (size_t)map->p.max_scan_points * 32;
        CK(cudaStreamCreateWithFlags(&map->copy_stream, cudaStreamNonBlocking));
        for (int b = 0; b < 2; ++b) {
            cudaError_t e = cudaMalloc(&map->pre_buf[b], bytes);
            if (e != cudaSuccess) {
                cudaGetLastError();
                return fail(FAR_ERR_OOM, "far_prefetch_points: staging allocation failed: %s", cudaGetErrorString(e));
            }
            CK(cudaEventCreateWithFlags(&map->pre_ready[b], cudaEventDisableTiming));
            CK(cudaEventCreateWithFlags(&map->pre_used[b], cudaEventDisableTiming));
        }
    }
    // a free buffer, else the one filled earlier (its pending copy is dropped)
    const int slot = !map->pre_ptr[0] ? 0 : (!map->pre_ptr[1] ? 1 : 1 - map->pre_last);
    // the buffer's previous contents must have been packed by the map's stream
    if (map->pre_used_recorded[slot]) CK(cudaStreamWaitEvent(map->copy_stream, map->pre_used[slot], 0));
    const uint32_t width = stride_bytes <= 32 ? stride_bytes : 32;
    if (stride_bytes <= 32)
        CK(cudaMemcpyAsync(map->pre_buf[slot], xyz, (size_t)n * stride_bytes, cudaMemcpyHostToDevice,
                           map->copy_stream));
    else
        CK(cudaMemcpy2DAsync(map->pre_buf[slot], 32, xyz, stride_bytes, 32, n, cudaMemcpyHostToDevice,
                             map->copy_stream));
    CK(cudaEventRecord(map->pre_ready[slot], map->copy_stream));
    map->pre_ptr[slot] = xyz;
    map->pre_n[slot] = n;
    map->pre_stride[slot] = stride_bytes;
    map->pre_width[slot] = width;
    map->pre_last = slot;
    return FAR_OK;
}

far_status far_process_scan(far_map* map, const float* xyz, uint64_t n, uint32_t stride_bytes,
                            const double init_pose[16], const far_reg_params* reg, const far_insert_params* ins,
                            double evict_radius, double out_pose[16], double out_cov[36], far_step_result* result) {
    return far_process_scan_motion(map, xyz, n, stride_bytes, nullptr, init_pose, reg, ins, evict_radius, out_pose,
                                   out_cov, result);
}

far_status far_process_scan_async(far_map* map, const float* xyz, uint64_t n, uint32_t stride_bytes,
                                  const far_motion* motion, const double init_pose[16], const far_reg_params* reg,
                                  const far_insert_params* ins, double evict_radius, int32_t want_cov) {
    far_status st = check_points(map, xyz, n, stride_bytes);
    if (st != FAR_OK) return st;
    if (map->step_pending) return fail(FAR_ERR_INVALID, "a step is pending: call far_process_scan_wait first");
    if (!reg || !init_pose || !finite_pose(init_pose))
        return fail(FAR_ERR_INVALID, "reg params or init_pose invalid");
    if (!(reg->kappa > 0.0f) || !(reg->tau >= 0.0f) || reg->max_iters > 1000)
        return fail(FAR_ERR_INVALID, "kappa must be > 0, tau >= 0, max_iters <= 1000");
    if (!(evict_radius >= 0.0) || std::isnan(evict_radius)) return fail(FAR_ERR_INVALID, "evict_radius must be >= 0");
    InsertCfg cfg;
    if (ins && ins->asmd) {
        if (!(ins->r_max > 0.0) || !(ins->r_near >= 0.0) || !std::isfinite(ins->r_max))
            return fail(FAR_ERR_INVALID, "ASMD needs r_near >= 0 and finite r_max > 0");
        cfg.asmd = 1;
        cfg.rc2 = ins->r_near * ins->r_near;
        cfg.r_max = ins->r_max;
    }
    const u32 nn = (u32)n;
    reset_marks(map);
    mark(map, EV_INGEST);
    if ((st = ingest(map, xyz, nn, stride_bytes, motion)) != FAR_OK) return st;
    mark(map, EV_SOURCES);
    if (nn) {
        if ((st = build_sources(map, nn, nullptr)) != FAR_OK) return st;
    } else {
        CK(cudaMemsetAsync(map->s.scal, 0, SCAL_COUNT * sizeof(u32), map->stream));
    }
    CK(gn_begin(map->s.st, init_pose, map->s.scal + SCAL_NADMIT, map->stream));
    GnArgs a = gn_args(map, init_pose, std::max(nn, 1u), reg->tau, reg->kappa, reg->conv_eps, 1, nullptr,
                       reg->time_budget_s, (int)reg->threads_per_point);
    if ((st = run_gn(map, a, std::max(nn, 1u), reg->max_iters)) != FAR_OK) return st;
    if (want_cov) CK(gn_covariance(map->s.st, map->d_cov36, map->stream));
    mark(map, EV_INSERT);
    // Sec. III-A.3 submap update at the registered pose, read from the device (skipped unless status == 0)
    DevicePose dp;
    dp.T = map->s.st->T;
    dp.status = &map->s.st->status;
    CK(map_insert_batch(map->map, map->s, nn, nullptr, cfg, true, map->stream, dp, insert_marks(map, 1)));
    mark(map, EV_EVICT);
    if (evict_radius > 0.0 && std::isfinite(evict_radius))
        CK(map_evict(map->map, nullptr, evict_radius, map->stream, map->s.st->T));
    else
        CK(cudaMemsetAsync(&map->map.ctr->removed, 0, sizeof(unsigned long long), map->stream));
    mark(map, EV_END);
    CK(cudaMemcpyAsync(map->h_st, map->s.st, sizeof(RegState), cudaMemcpyDeviceToHost, map->stream));
    CK(cudaMemcpyAsync(map->h_ctr, map->map.ctr, sizeof(MapCounters), cudaMemcpyDeviceToHost, map->stream));
    if (want_cov) CK(cudaMemcpyAsync(map->h_cov36, map->d_cov36, 36 * sizeof(double), cudaMemcpyDeviceToHost, map->stream));
    map->step_pending = true;
    map->step_want_cov = want_cov != 0;
    return FAR_OK;
}

far_status far_process_scan_wait(far_map* map, double out_pose[16], double out_cov[36], far_step_result* result) {
    if (!map) return fail(FAR_ERR_INVALID, "map is NULL");
    if (!map->step_pending) return fail(FAR_ERR_INVALID, "no step is pending (far_process_scan_async first)");
    if (!out_pose) return fail(FAR_ERR_INVALID, "out_pose is NULL");
    if (out_cov && !map->step_want_cov) return fail(FAR_ERR_INVALID, "out_cov given but the step did not ask for it");
    map->step_pending = false;
    CK(cudaStreamSynchronize(map->stream));
    if (map->h_ctr->n_tomb > map->map.cap / 4) {
        CK(map_rebuild(map->map, map->stream));
        CK(cudaStreamSynchronize(map->stream));
    }
    const RegState& r = *map->h_st;
    account_gn_graph(map, r);
    collect_times(map, r.iters, r.status);
    if (map->profiling) collect_insert_times(map);
    std::memcpy(out_pose, r.T, 16 * sizeof(double));
    if (out_cov) std::memcpy(out_cov, map->h_cov36, 36 * sizeof(double));
    far_status res = FAR_OK;
    if (r.status == 5) res = fail(FAR_ERR_DEGENERATE, "registration degenerate (%u correspondences); scan not inserted",
                                  r.n_corr);
    if (r.status == 6) res = fail(FAR_ERR_TIMEOUT, "registration exceeded its time budget; scan not inserted");
    if (r.status == 7) res = fail(FAR_ERR_CUDA, "internal: the Gauss-Newton loop ran past its iteration limit");
    if (result) {
        result->reg.iters = r.iters;
        result->reg.n_src = r.n_src;
        result->reg.n_corr = r.n_corr;
        result->reg.n_p2p = r.n_p2p;
        result->reg.converged = (int32_t)r.converged;
        result->reg.status = res;
        result->reg.chi2 = r.chi2;
        result->n_inserted = map->h_ctr->n_added;
        result->n_removed = map->h_ctr->removed;
        result->n_voxels = map->h_ctr->n_voxels;
        result->n_points = map->h_ctr->n_points;
    }
    if (res == FAR_OK) return check_device_errors(map, "far_process_scan");
    return res;
}


far_status far_process_scan_motion(far_map* map, const float* xyz, uint64_t n, uint32_t stride_bytes,
                                   const far_motion* motion, const double init_pose[16], const far_reg_params* reg,
                                   const far_insert_params* ins, double evict_radius, double out_pose[16],
                                   double out_cov[36], far_step_result* result) {
    if (map && !out_pose) return fail(FAR_ERR_INVALID, "reg params, init_pose or out_pose invalid");
    const far_status st = far_process_scan_async(map, xyz, n, stride_bytes, motion, init_pose, reg, ins, evict_radius,
                                                 out_cov != nullptr);
    if (st != FAR_OK) return st;
    return far_process_scan_wait(map, out_pose, out_cov, result);
}

// ---------------------------------------------------------------- motion undistortion (Sec. III-A.1)
far_status far_motion_fit(const double* t, const double* w, const double* v, uint32_t n, double t_ref,
                          uint32_t time_offset_bytes, far_motion* out) {
    if (!t || !w || !v || !out) return fail(FAR_ERR_INVALID, "far_motion_fit: NULL argument");
    if (n < 1) return fail(FAR_ERR_INVALID, "far_motion_fit: no samples");
    if (!std::isfinite(t_ref)) return fail(FAR_ERR_INVALID, "far_motion_fit: t_ref not finite");
    for (uint32_t i = 0; i < n; ++i)
        if (!std::isfinite(t[i]) || !std::isfinite(w[3 * i]) || !std::isfinite(w[3 * i + 1]) ||
            !std::isfinite(w[3 * i + 2]) || !std::isfinite(v[3 * i]) || !std::isfinite(v[3 * i + 1]) ||
            !std::isfinite(v[3 * i + 2]))
            return fail(FAR_ERR_INVALID, "far_motion_fit: non-finite sample");
    // least-squares line y = a + b (t - t_ref) per component, about the mean time for accuracy
    double tm = 0.0;
    for (uint32_t i = 0; i < n; ++i) tm += t[i] - t_ref;
    tm /= n;
    double stt = 0.0;
    for (uint32_t i = 0; i < n; ++i) stt += (t[i] - t_ref - tm) * (t[i] - t_ref - tm);
    far_motion m{};
    for (int a = 0; a < 6; ++a) {
        const double* y = a < 3 ? w : v;
        const int c = a % 3;
        double ym = 0.0;
        for (uint32_t i = 0; i < n; ++i) ym += y[3 * i + c];
        ym /= n;
        double sty = 0.0;
        for (uint32_t i = 0; i < n; ++i) sty += (t[i] - t_ref - tm) * (y[3 * i + c] - ym);
        const double slope = stt > 0.0 ? sty / stt : 0.0;   // one time stamp: a constant
        const double icpt = ym - slope * tm;
        if (a < 3) {
            m.w0[c] = icpt;
            m.w1[c] = slope;
        } else {
            m.v0[c] = icpt;
            m.v1[c] = slope;
        }
    }
    m.time_offset_bytes = time_offset_bytes;
    *out = m;
    return FAR_OK;
}

far_status far_undistort(const float* xyz, uint64_t n, uint32_t stride_bytes, const far_motion* motion,
                         float* out_xyz, void* cuda_stream) {
    if (!motion) return fail(FAR_ERR_INVALID, "far_undistort: motion is NULL");
    if (n == 0) return FAR_OK;
    if (!xyz || !out_xyz || !is_device_pointer(xyz) || !is_device_pointer(out_xyz))
        return fail(FAR_ERR_INVALID, "far_undistort: xyz and out_xyz must be device pointers");
    if (n > 0xFFFFFFFFull) return fail(FAR_ERR_INVALID, "far_undistort: n exceeds 2^32 - 1");
    if (stride_bytes < 16 || stride_bytes % 4 != 0)
        return fail(FAR_ERR_INVALID, "far_undistort: stride_bytes must be >= 16 and a multiple of 4");
    SweepMotion mo;
    far_status st = sweep_motion(motion, stride_bytes, &mo);
    if (st != FAR_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    CK(deskew_points(xyz, (u32)n, stride_bytes, mo, out_xyz, s));
    CK(cudaStreamSynchronize(s));
    return FAR_OK;
}

// ---------------------------------------------------------------- batched registration
}  // extern "C"

struct far_batch {
    std::vector<far_map*> maps;
    cudaStream_t user_stream = nullptr;   // the caller's stream: the batch starts after its prior work
    cudaEvent_t ev_user = nullptr;
    cudaStream_t stream = nullptr;        // own stream: graphs cannot be captured on the legacy default stream
    std::vector<cudaStream_t> side;
    cudaEvent_t ev_fork = nullptr, ev_fork2 = nullptr;
    std::vector<cudaEvent_t> ev_join, ev_join2;
    BatchProblem* d_probs = nullptr;
    BatchProblem* h_probs = nullptr;       // pinned mirror, copied in stream order each launch
    u32* d_block_prob = nullptr;
    u32* h_block_prob = nullptr;           // pinned mirror
    u32 max_blocks = 0;                    // capacity of the block -> problem table
    double* d_init = nullptr;
    double* h_init = nullptr;              // pinned
    RegState* d_states = nullptr;
    RegState* h_states = nullptr;          // pinned
    MapCounters* h_ctr = nullptr;          // pinned, one per problem (process mode)
    u32 total_blocks = 0;
    cudaGraphExec_t exec = nullptr;
    // what the captured graph was built for
    std::vector<const void*> key_ptr;
    std::vector<uint64_t> key_n;
    std::vector<uint32_t> key_stride;
    uint32_t key_iters = 0;
    int key_tpp = -1;
};

namespace {

void batch_release(far_batch* b) {
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    for (cudaStream_t s : b->side) cudaStreamDestroy(s);
    for (cudaEvent_t e : b->ev_join) cudaEventDestroy(e);
    for (cudaEvent_t e : b->ev_join2) cudaEventDestroy(e);
    if (b->ev_fork) cudaEventDestroy(b->ev_fork);
    if (b->ev_fork2) cudaEventDestroy(b->ev_fork2);
    if (b->ev_user) cudaEventDestroy(b->ev_user);
    if (b->stream) cudaStreamDestroy(b->stream);
    cudaFree(b->d_probs);
    cudaFree(b->d_block_prob);
    cudaFree(b->d_init);
    cudaFree(b->d_states);
    cudaFreeHost(b->h_probs);
    cudaFreeHost(b->h_block_prob);
    cudaFreeHost(b->h_init);
    cudaFreeHost(b->h_states);
    cudaFreeHost(b->h_ctr);
}

bool is_registered_or_device(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged || a.type == cudaMemoryTypeHost;
}

// Each problem gets exactly the linearisation grid that the single-problem path launches
// for it (gn_grid of its point count), so its block partials, their reduction order and its
// result are bit-identical alone and in any mix; the blocks of all problems share one launch.
far_status batch_assign_blocks(far_batch* b, const uint64_t* n, int tpp) {
    const u32 np = (u32)b->maps.size();
    u32 total = 0;
    for (u32 p = 0; p < np; ++p) {
        const u32 n_up = (u32)std::max<uint64_t>(n[p], 1);
        const u32 share = gn_grid(n_up, tpp);
        if ((u64)total + share > b->max_blocks) return fail(FAR_ERR_INVALID, "batch grid larger than its table");
        BatchProblem& bp = b->h_probs[p];
        bp.block_begin = total;
        bp.nblocks = share;
        for (u32 j = 0; j < share; ++j) b->h_block_prob[total + j] = p;
        total += share;
    }
    b->total_blocks = total;
    return FAR_OK;
}

// Issue a batch on the batch's streams: sources of every problem on worker streams, the
// batched Gauss-Newton chain on the main stream, optionally (ins != null) the insert of each
// scan at its registered pose and the eviction on worker streams, then the state gather.
far_status batch_enqueue(far_batch* b, const float* const* xyz, const uint64_t* n, const uint32_t* stride,
                         uint32_t iters, int tpp, const InsertCfg* ins, double evict_radius) {
    const u32 np = (u32)b->maps.size();
    std::vector<cudaStream_t> saved(np);
    for (u32 p = 0; p < np; ++p) saved[p] = b->maps[p]->stream;
    struct Restore {
        far_batch* b;
        std::vector<cudaStream_t>& saved;
        ~Restore() {
            for (size_t p = 0; p < saved.size(); ++p) b->maps[p]->stream = saved[p];
        }
    } restore{b, saved};
    // larger problems first, each to the worker stream with the least work so far
    std::vector<u32> order(np);
    for (u32 p = 0; p < np; ++p) order[p] = p;
    std::sort(order.begin(), order.end(), [&](u32 a, u32 c) { return n[a] > n[c]; });
    std::vector<double> load(b->side.size(), 0.0);
    std::vector<u32> lane(np, 0);
    for (u32 p : order) {
        const size_t w = std::min_element(load.begin(), load.end()) - load.begin();
        lane[p] = (u32)w;
        load[w] += (double)n[p] + 1000.0;
    }
    CK(cudaMemcpyAsync(b->d_probs, b->h_probs, np * sizeof(BatchProblem), cudaMemcpyHostToDevice, b->stream));
    CK(cudaMemcpyAsync(b->d_block_prob, b->h_block_prob, b->total_blocks * sizeof(u32),
                       cudaMemcpyHostToDevice, b->stream));
    CK(cudaMemcpyAsync(b->d_init, b->h_init, np * 16 * sizeof(double), cudaMemcpyHostToDevice, b->stream));
    CK(cudaEventRecord(b->ev_fork, b->stream));
    for (cudaStream_t s : b->side) CK(cudaStreamWaitEvent(s, b->ev_fork, 0));
    for (u32 p : order) {
        far_map* m = b->maps[p];
        m->stream = b->side[lane[p]];
        const u32 nn = (u32)n[p];
        far_status st = ingest(m, xyz[p], nn, stride[p]);
        if (st != FAR_OK) return st;
        if (nn) {
            if ((st = build_sources(m, nn, nullptr)) != FAR_OK) return st;
        } else {
            CK(cudaMemsetAsync(m->s.scal, 0, SCAL_COUNT * sizeof(u32), m->stream));
        }
    }
    for (size_t i = 0; i < b->side.size(); ++i) {
        CK(cudaEventRecord(b->ev_join[i], b->side[i]));
        CK(cudaStreamWaitEvent(b->stream, b->ev_join[i], 0));
    }
    CK(gn_batch_begin(b->d_probs, np, b->d_init, b->stream));
    for (u32 it = 0; it < iters; ++it)
        CK(gn_batch_iteration(b->d_probs, b->d_block_prob, b->total_blocks, np, tpp, b->maps[0]->map.tv > 0,
                              b->stream));
    if (ins) {
        CK(cudaEventRecord(b->ev_fork2, b->stream));
        for (cudaStream_t s : b->side) CK(cudaStreamWaitEvent(s, b->ev_fork2, 0));
        for (u32 p : order) {
            far_map* m = b->maps[p];
            m->stream = b->side[lane[p]];
            DevicePose dp;
            dp.T = m->s.st->T;
            dp.status = &m->s.st->status;
            CK(map_insert_batch(m->map, m->s, (u32)n[p], nullptr, *ins, true, m->stream, dp));
            if (evict_radius > 0.0 && std::isfinite(evict_radius))
                CK(map_evict(m->map, nullptr, evict_radius, m->stream, m->s.st->T));
            else
                CK(cudaMemsetAsync(&m->map.ctr->removed, 0, sizeof(unsigned long long), m->stream));
            CK(cudaMemcpyAsync(b->h_ctr + p, m->map.ctr, sizeof(MapCounters), cudaMemcpyDeviceToHost, m->stream));
        }
        for (size_t i = 0; i < b->side.size(); ++i) {
            CK(cudaEventRecord(b->ev_join2[i], b->side[i]));
            CK(cudaStreamWaitEvent(b->stream, b->ev_join2[i], 0));
        }
    }
    CK(gn_batch_gather(b->d_probs, np, b->d_states, b->stream));
    CK(cudaMemcpyAsync(b->h_states, b->d_states, np * sizeof(RegState), cudaMemcpyDeviceToHost, b->stream));
    return FAR_OK;
}

// Record a registration batch into a CUDA graph.
far_status batch_capture(far_batch* b, const float* const* xyz, const uint64_t* n, const uint32_t* stride,
                         uint32_t iters, int tpp) {
    const u32 np = (u32)b->maps.size();
    if (b->exec) {
        cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
    }
    cudaGraph_t graph = nullptr;
    CK(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
    far_status st = batch_enqueue(b, xyz, n, stride, iters, tpp, nullptr, 0.0);
    cudaError_t e = cudaStreamEndCapture(b->stream, &graph);
    if (st != FAR_OK) {
        if (graph) cudaGraphDestroy(graph);
        return st;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(FAR_ERR_CUDA, "batch graph capture failed: %s", cudaGetErrorString(e));
    }
    b->key_ptr.assign(xyz, xyz + np);
    b->key_n.assign(n, n + np);
    b->key_stride.assign(stride, stride + np);
    b->key_iters = iters;
    b->key_tpp = tpp;
    return FAR_OK;
}

far_status batch_check(far_batch* b, const float* const* xyz, const uint64_t* n, const uint32_t* stride,
                       const double* init_poses, const far_reg_params* params, uint32_t params_count,
                       const double* out_poses) {
    if (!b || !xyz || !n || !stride || !init_poses || !params || !out_poses)
        return fail(FAR_ERR_INVALID, "NULL argument");
    const u32 np = (u32)b->maps.size();
    if (params_count != 1 && params_count != np) return fail(FAR_ERR_INVALID, "params_count must be 1 or the batch size");
    for (u32 i = 0; i < params_count; ++i) {
        const far_reg_params& q = params[i];
        if (!(q.kappa > 0.0f) || !(q.tau >= 0.0f) || q.max_iters > 1000)
            return fail(FAR_ERR_INVALID, "kappa must be > 0, tau >= 0, max_iters <= 1000 (params %u)", i);
        if (q.max_iters != params[0].max_iters || gn_tpp((int)q.threads_per_point) != gn_tpp((int)params[0].threads_per_point))
            return fail(FAR_ERR_INVALID, "max_iters and threads_per_point must be the same for every problem");
    }
    for (u32 p = 0; p < np; ++p) {
        far_status st = check_points(b->maps[p], xyz[p], n[p], stride[p]);
        if (st != FAR_OK) return st;
        if (n[p] && !is_registered_or_device(xyz[p]))
            return fail(FAR_ERR_INVALID, "batch inputs must be device or pinned host memory (problem %u)", p);
        if (!finite_pose(init_poses + 16 * (size_t)p)) return fail(FAR_ERR_INVALID, "init pose %u not finite", p);
    }
    return FAR_OK;
}

void batch_set_args(far_batch* b, const uint64_t* n, const double* init_poses, const far_reg_params* params,
                    uint32_t params_count, int tpp) {
    const u32 np = (u32)b->maps.size();
    for (u32 p = 0; p < np; ++p) {
        const u32 n_up = (u32)std::max<uint64_t>(n[p], 1);
        const far_reg_params& q = params[params_count == 1 ? 0 : p];
        b->h_probs[p].args = gn_args(b->maps[p], init_poses + 16 * (size_t)p, n_up, q.tau, q.kappa, q.conv_eps, 1,
                                     nullptr, q.time_budget_s, tpp);
    }
    std::memcpy(b->h_init, init_poses, np * 16 * sizeof(double));
}

far_status batch_results(far_batch* b, double* out_poses, far_reg_stats* stats, far_step_result* steps) {
    const u32 np = (u32)b->maps.size();
    far_status worst = FAR_OK;
    for (u32 p = 0; p < np; ++p) {
        const RegState& r = b->h_states[p];
        std::memcpy(out_poses + 16 * (size_t)p, r.T, 16 * sizeof(double));
        far_status sp = r.status == 5 ? FAR_ERR_DEGENERATE : (r.status == 6 ? FAR_ERR_TIMEOUT : FAR_OK);
        if (sp != FAR_OK && worst == FAR_OK) worst = sp;
        far_reg_stats rs;
        rs.iters = r.iters;
        rs.n_src = r.n_src;
        rs.n_corr = r.n_corr;
        rs.n_p2p = r.n_p2p;
        rs.converged = (int32_t)r.converged;
        rs.status = sp;
        rs.chi2 = r.chi2;
        if (stats) stats[p] = rs;
        if (steps) {
            steps[p].reg = rs;
            steps[p].n_inserted = b->h_ctr[p].n_added;
            steps[p].n_removed = b->h_ctr[p].removed;
            steps[p].n_voxels = b->h_ctr[p].n_voxels;
            steps[p].n_points = b->h_ctr[p].n_points;
        }
    }
    if (worst != FAR_OK) return fail(worst, "at least one problem of the batch did not register (see stats)");
    return FAR_OK;
}

}  // namespace

extern "C" {

far_status far_batch_create(far_map* const* maps, uint32_t count, void* cuda_stream, far_batch** out) {
    if (!maps || !out || count == 0 || count > 4096) return fail(FAR_ERR_INVALID, "maps/out NULL or count not in 1..4096");
    for (uint32_t i = 0; i < count; ++i) {
        if (!maps[i]) return fail(FAR_ERR_INVALID, "maps[%u] is NULL", i);
        for (uint32_t j = 0; j < i; ++j)
            if (maps[j] == maps[i]) return fail(FAR_ERR_INVALID, "a map appears twice in the batch");
        if (maps[i]->p.precision_mode != maps[0]->p.precision_mode)
            return fail(FAR_ERR_INVALID, "all maps of a batch must use the same precision_mode");
    }
    far_batch* b = new far_batch();
    b->maps.assign(maps, maps + count);
    b->user_stream = static_cast<cudaStream_t>(cuda_stream);
    const u32 nside = std::min<u32>(count, 16);
    cudaError_t e = cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_fork2, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_user, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
    for (u32 i = 0; e == cudaSuccess && i < nside; ++i) {
        cudaStream_t s = nullptr;
        cudaEvent_t ev = nullptr, ev2 = nullptr;
        e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
        if (e == cudaSuccess) b->side.push_back(s);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        if (e == cudaSuccess) b->ev_join.push_back(ev);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev2, cudaEventDisableTiming);
        if (e == cudaSuccess) b->ev_join2.push_back(ev2);
    }
    for (uint32_t i = 0; i < count; ++i) b->max_blocks += gn_max_blocks(maps[i]->p.max_scan_points);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_probs, count * sizeof(BatchProblem));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_block_prob, (size_t)b->max_blocks * sizeof(u32));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_init, count * 16 * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_states, count * sizeof(RegState));
    if (e == cudaSuccess) e = cudaMallocHost(&b->h_probs, count * sizeof(BatchProblem));
    if (e == cudaSuccess) e = cudaMallocHost(&b->h_block_prob, (size_t)b->max_blocks * sizeof(u32));
    if (e == cudaSuccess) e = cudaMallocHost(&b->h_init, count * 16 * sizeof(double));
    if (e == cudaSuccess) e = cudaMallocHost(&b->h_states, count * sizeof(RegState));
    if (e == cudaSuccess) e = cudaMallocHost(&b->h_ctr, count * sizeof(MapCounters));
    if (e != cudaSuccess) {
        cudaGetLastError();
        batch_release(b);
        delete b;
        return fail(FAR_ERR_OOM, "batch allocation failed: %s", cudaGetErrorString(e));
    }
    *out = b;
    return FAR_OK;
}

far_status far_batch_destroy(far_batch* batch) {
    if (!batch) return fail(FAR_ERR_INVALID, "batch is NULL");
    batch_release(batch);
    delete batch;
    return FAR_OK;
}

far_status far_batch_register(far_batch* b, const float* const* xyz, const uint64_t* n, const uint32_t* stride,
                              const double* init_poses, const far_reg_params* params, uint32_t params_count,
                              double* out_poses, far_reg_stats* stats) {
    far_status st = batch_check(b, xyz, n, stride, init_poses, params, params_count, out_poses);
    if (st != FAR_OK) return st;
    const u32 np = (u32)b->maps.size();
    const int tpp = gn_tpp((int)params->threads_per_point);
    batch_set_args(b, n, init_poses, params, params_count, tpp);
    bool same = b->exec && b->key_iters == params->max_iters && b->key_tpp == tpp;
    for (u32 p = 0; same && p < np; ++p)
        same = b->key_ptr[p] == (const void*)xyz[p] && b->key_n[p] == n[p] && b->key_stride[p] == stride[p];
    // the graph copies the block table and descriptors from the pinned mirrors at launch; the
    // assignment is a function of (n, tpp), so recomputing it restores what the graph was built for
    if ((st = batch_assign_blocks(b, n, tpp)) != FAR_OK) return st;
    if (!same && (st = batch_capture(b, xyz, n, stride, params->max_iters, tpp)) != FAR_OK) return st;
    CK(cudaEventRecord(b->ev_user, b->user_stream));
    CK(cudaStreamWaitEvent(b->stream, b->ev_user, 0));
    CK(cudaGraphLaunch(b->exec, b->stream));
    CK(cudaStreamSynchronize(b->stream));
    return batch_results(b, out_poses, stats, nullptr);
}

far_status far_batch_process(far_batch* b, const float* const* xyz, const uint64_t* n, const uint32_t* stride,
                             const double* init_poses, const far_reg_params* params, uint32_t params_count,
                             const far_insert_params* ins, double evict_radius, double* out_poses,
                             far_step_result* results) {
    far_status st = batch_check(b, xyz, n, stride, init_poses, params, params_count, out_poses);
    if (st != FAR_OK) return st;
    if (!(evict_radius >= 0.0) || std::isnan(evict_radius)) return fail(FAR_ERR_INVALID, "evict_radius must be >= 0");
    InsertCfg cfg;
    if (ins && ins->asmd) {
        if (!(ins->r_max > 0.0) || !(ins->r_near >= 0.0) || !std::isfinite(ins->r_max))
            return fail(FAR_ERR_INVALID, "ASMD needs r_near >= 0 and finite r_max > 0");
        cfg.asmd = 1;
        cfg.rc2 = ins->r_near * ins->r_near;
        cfg.r_max = ins->r_max;
    }
    const u32 np = (u32)b->maps.size();
    const int tpp = gn_tpp((int)params->threads_per_point);
    batch_set_args(b, n, init_poses, params, params_count, tpp);
    if ((st = batch_assign_blocks(b, n, tpp)) != FAR_OK) return st;
    CK(cudaEventRecord(b->ev_user, b->user_stream));
    CK(cudaStreamWaitEvent(b->stream, b->ev_user, 0));
    if ((st = batch_enqueue(b, xyz, n, stride, params->max_iters, tpp, &cfg, evict_radius)) != FAR_OK) return st;
    CK(cudaStreamSynchronize(b->stream));
    for (u32 p = 0; p < np; ++p) {
        far_map* m = b->maps[p];
        if (b->h_ctr[p].n_tomb > m->map.cap / 4) {
            CK(map_rebuild(m->map, m->stream));
            CK(cudaStreamSynchronize(m->stream));
        }
    }
    st = batch_results(b, out_poses, nullptr, results);
    if (st == FAR_OK) {
        for (u32 p = 0; p < np; ++p) {
            if (b->h_ctr[p].err) {
                *b->maps[p]->h_ctr = b->h_ctr[p];
                far_status e2 = check_device_errors(b->maps[p], "far_batch_process");
                if (e2 != FAR_OK) return e2;
            }
        }
    }
    return st;
}

unsigned long long far_launch_count(void) { return g_launches.load(); }

far_status far_set_profiling(far_map* map, int enable) {
    if (!map) return fail(FAR_ERR_INVALID, "map is NULL");
    if (enable && map->ev.empty()) {
        map->ev.resize(EV_COUNT_FIXED + 2 * MAX_ITERS + 1, nullptr);
        for (cudaEvent_t& e : map->ev) CK(cudaEventCreate(&e));
        for (int w = 0; w < 2; ++w) {
            CK(cudaEventCreate(&map->ins_start[w]));
            for (cudaEvent_t& e : map->ins_marks[w].ev) CK(cudaEventCreate(&e));
        }
        CK(cudaEventCreate(&map->src_end));
    }
    map->profiling = enable != 0;
    return FAR_OK;
}

far_status far_get_insert_times(const far_map* map, far_insert_times out[2]) {
    if (!map || !out) return fail(FAR_ERR_INVALID, "NULL argument");
    if (!map->profiling) return fail(FAR_ERR_INVALID, "profiling is off (far_set_profiling)");
    out[0] = map->ins_last[0];
    out[1] = map->ins_last[1];
    return FAR_OK;
}

far_status far_get_stage_times(const far_map* map, far_stage_times* out) {
    if (!map || !out) return fail(FAR_ERR_INVALID, "NULL argument");
    if (!map->profiling) return fail(FAR_ERR_INVALID, "profiling is off (far_set_profiling)");
    *out = map->last;
    return FAR_OK;
}

far_status far_gn_footprint(far_map* map, uint64_t out[3]) {
    if (!map || !out) return fail(FAR_ERR_INVALID, "NULL argument");
    GnArgs a = map->last_gn;
    a.map = map->map.view();
    a.src = map->s.src;
    a.st = map->s.st;
    CK(gn_footprint(a, map->s.touched, map->map.cap, map->s.foot, map->p.max_scan_points, map->stream));
    unsigned long long f[2];
    CK(cudaMemcpyAsync(map->h_st, map->s.st, sizeof(RegState), cudaMemcpyDeviceToHost, map->stream));
    CK(cudaMemcpyAsync(f, map->s.foot, sizeof(f), cudaMemcpyDeviceToHost, map->stream));
    CK(cudaStreamSynchronize(map->stream));
    out[0] = map->h_st->n_src;
    out[1] = f[0];
    out[2] = f[1];
    return FAR_OK;
}

// ---- adaptive threshold (host) ----
far_status far_threshold_init(far_threshold* t, double sigma0, double min_motion, double r_max) {
    if (!t || !(sigma0 > 0) || !(r_max > 0) || !(min_motion >= 0)) return fail(FAR_ERR_INVALID, "bad threshold params");
    t->sigma0 = sigma0;
    t->min_motion = min_motion;
    t->r_max = r_max;
    t->sse = 0.0;
    t->n = 0;
    return FAR_OK;
}

far_status far_threshold_get(const far_threshold* t, double* tau, double* kappa) {
    if (!t || !tau || !kappa) return fail(FAR_ERR_INVALID, "NULL argument");
    const double sigma = t->n > 0 ? std::sqrt(t->sse / (double)t->n) : t->sigma0;
    *tau = 3.0 * sigma;
    *kappa = sigma / 3.0;
    return FAR_OK;
}

far_status far_threshold_update(far_threshold* t, const double a[16], const double b[16]) {
    if (!t || !a || !b) return fail(FAR_ERR_INVALID, "NULL argument");
    // D = a^-1 b for rigid a: R_D = R_a^T R_b, t_D = R_a^T (t_b - t_a)
    double RD[3][3], tD[3];
    for (int i = 0; i < 3; ++i) {
        for (int j = 0; j < 3; ++j) {
            double s = 0;
            for (int l = 0; l < 3; ++l) s += a[4 * l + i] * b[4 * l + j];
            RD[i][j] = s;
        }
        double s = 0;
        for (int l = 0; l < 3; ++l) s += a[4 * l + i] * (b[4 * l + 3] - a[4 * l + 3]);
        tD[i] = s;
    }
    const double c = std::max(-1.0, std::min(1.0, 0.5 * (RD[0][0] + RD[1][1] + RD[2][2] - 1.0)));
    const double theta = std::acos(c);
    const double dt = std::sqrt(tD[0] * tD[0] + tD[1] * tD[1] + tD[2] * tD[2]);
    const double delta = 2.0 * t->r_max * std::sin(0.5 * theta) + dt;
    if (dt > t->min_motion) {
        t->sse += delta * delta;
        t->n += 1;
    }
    return FAR_OK;
}

}  // extern "C"
