// far_scan_sources_static: the scan-local downsampling and the per-point
// covariances of each kept point from its k nearest kept neighbours (the same
// kernels as far_scan_sources) for callers that cannot allocate
// device memory, e.g. a process whose memory is fixed before it starts (an
// embedded or safety partition, a memory-capped multi-process server client),
// or code that must not call cudaMalloc while other work may be capturing CUDA
// graphs. All scratch lives in one file-scope __device__ array below, sized for
// at most kStaticMaxPoints input points and kStaticMaxPerVoxel points per voxel.
// The array exists once per GPU that loads this library and stays until exit.
#include <cmath>
#include <cstdio>
#include <mutex>

#include "far.h"
#include "map.cuh"
#include "primitives.cuh"

using namespace far;

namespace far {
cudaError_t export_sources(const Scratch& s, u32 n, int64_t* index, float* cov6, uint8_t* valid, cudaStream_t st);
void set_last_error(const char* msg);
}  // namespace far

namespace {

constexpr u32 kStaticMaxPoints = 16384;
constexpr u32 kStaticMaxPerVoxel = 20;
constexpr u32 kLocalCap = 2 * kStaticMaxPoints;           // power of two >= 2 n, as the map plan uses
constexpr u32 kPartialWords = 1024;

constexpr size_t up256(size_t b) { return (b + 255) & ~(size_t)255; }

// Byte offsets of every sub-buffer inside the static array.
struct Layout {
    size_t slots, pts, ring, ctr, in4, world, keys, u32s[17], gstart, slot_cnt, slot_base, partials, scal, src, src_cov,
        total;
};

constexpr Layout make_layout() {
    Layout L{};
    size_t o = 0;
    auto take = [&o](size_t bytes) {
        size_t at = o;
        o += up256(bytes);
        return at;
    };
    L.slots = take((size_t)kLocalCap * sizeof(Slot));
    L.pts = take((size_t)kStaticMaxPoints * kStaticMaxPerVoxel * sizeof(float4));
    L.ring = take((size_t)kStaticMaxPoints * sizeof(u32));
    L.ctr = take(sizeof(MapCounters));
    L.in4 = take((size_t)kStaticMaxPoints * sizeof(float4));
    L.world = take((size_t)kStaticMaxPoints * sizeof(float4));
    L.keys = take((size_t)kStaticMaxPoints * sizeof(u64));
    for (int i = 0; i < 17; ++i) L.u32s[i] = take((size_t)(kStaticMaxPoints + 1) * sizeof(u32));
    L.gstart = take((size_t)(kStaticMaxPoints + 2) * sizeof(u32));
    L.slot_cnt = take((size_t)(kLocalCap + 1) * sizeof(u32));   // zeroed at the start of every call
    L.slot_base = take((size_t)(kLocalCap + 1) * sizeof(u32));
    L.partials = take((size_t)kPartialWords * sizeof(u32));
    L.scal = take((size_t)SCAL_COUNT * sizeof(u32));
    L.src = take((size_t)kStaticMaxPoints * sizeof(float4));
    L.src_cov = take((size_t)kStaticMaxPoints * 2 * sizeof(float4));
    L.total = o;
    return L;
}

constexpr Layout kLayout = make_layout();

// The scratch of far_scan_sources_static (about 8 MB). Host code must not use
// this name as an address: it is resolved per device with cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_static_scratch[kLayout.total];

std::mutex g_mu;
constexpr int kMaxDevices = 64;
unsigned char* g_dev_base[kMaxDevices] = {};

far_status reject(far_status s, const char* msg) {
    set_last_error(msg);
    return s;
}

// Device memory of the current device `dev` (or managed memory): the kernels read and
// write these pointers directly, so memory of another GPU is rejected.
bool on_device(const void* p, int dev) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (a.type == cudaMemoryTypeManaged) return true;
    return a.type == cudaMemoryTypeDevice && a.device == dev;
}

}  // namespace

extern "C" far_status far_scan_sources_static(const float* xyz, uint64_t n, uint32_t stride_bytes, float voxel_size,
                                              uint32_t max_pts_per_voxel, uint32_t k_cov, float min_spacing,
                                              void* cuda_stream, int64_t* out_index, float* out_cov,
                                              uint8_t* out_valid, uint32_t* out_knn_ids, uint64_t* n_src) {
    if (!n_src) return reject(FAR_ERR_INVALID, "n_src is NULL");
    if (n > kStaticMaxPoints) {
        char msg[160];
        snprintf(msg, sizeof(msg), "n = %llu exceeds the static-scratch limit of %u points", (unsigned long long)n,
                 kStaticMaxPoints);
        return reject(FAR_ERR_INVALID, msg);
    }
    if (!(voxel_size > 0.0f) || !std::isfinite(voxel_size)) return reject(FAR_ERR_INVALID, "voxel_size must be > 0");
    if (max_pts_per_voxel < 1 || max_pts_per_voxel > kStaticMaxPerVoxel)
        return reject(FAR_ERR_INVALID, "max_pts_per_voxel must be in 1..20 for the static-scratch entry point");
    if (k_cov < 1 || k_cov > (u32)KMAX) return reject(FAR_ERR_INVALID, "k_cov must be in 1..16");
    if (!std::isfinite(min_spacing)) return reject(FAR_ERR_INVALID, "min_spacing must be finite");
    if (n == 0) {
        *n_src = 0;
        return FAR_OK;
    }
    if (stride_bytes < 12 || stride_bytes % 4 != 0)
        return reject(FAR_ERR_INVALID, "stride_bytes must be >= 12 and a multiple of 4");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return reject(FAR_ERR_CUDA, "no current CUDA device");
    }
    if (!xyz || !on_device(xyz, dev)) return reject(FAR_ERR_INVALID, "xyz must be memory of the current device");
    if (!out_index || !out_cov || !out_valid || !on_device(out_index, dev) || !on_device(out_cov, dev) ||
        !on_device(out_valid, dev) || (out_knn_ids && !on_device(out_knn_ids, dev)))
        return reject(FAR_ERR_INVALID,
                      "outputs must be memory of the current device (out_knn_ids may be NULL)");
    if (2 * scan_blocks((u32)n) + 2 > kPartialWords)
        return reject(FAR_ERR_INVALID, "internal: static scratch layout too small");
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);

    // Set-up, once per device with that device current: resolve the array's device address.
    // The address is cached for the life of the process; a device reset after the first call
    // reloads the module elsewhere and is not supported.
    unsigned char* base = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_dev_base[dev]) {
            void* p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
            if (e != cudaSuccess || !p) {
                cudaGetLastError();
                char msg[200];
                snprintf(msg, sizeof(msg), "cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
                return reject(FAR_ERR_CUDA, msg);
            }
            g_dev_base[dev] = static_cast<unsigned char*>(p);
        }
        base = g_dev_base[dev];
    }

    DeviceMap local;
    local.slots = reinterpret_cast<Slot*>(base + kLayout.slots);
    local.cap = kLocalCap;
    local.mask = kLocalCap - 1;
    int bits = 0;
    while ((1u << bits) < kLocalCap) ++bits;
    local.key_bits = bits + 1;
    local.pts = reinterpret_cast<float4*>(base + kLayout.pts);
    local.ring = reinterpret_cast<u32*>(base + kLayout.ring);
    local.max_buckets = kStaticMaxPoints;
    local.ctr = reinterpret_cast<MapCounters*>(base + kLayout.ctr);
    local.nmax = max_pts_per_voxel;
    local.k = k_cov;
    local.v = voxel_size;
    local.inv_v = 1.0f / voxel_size;
    const float dmin =
        min_spacing < 0.0f ? (float)((double)voxel_size / std::sqrt((double)max_pts_per_voxel)) : min_spacing;
    local.dmin2 = dmin * dmin;

    Scratch s;
    s.max_n = kStaticMaxPoints;
    s.in4 = reinterpret_cast<float4*>(base + kLayout.in4);
    s.world = reinterpret_cast<float4*>(base + kLayout.world);
    s.keys = reinterpret_cast<u64*>(base + kLayout.keys);
    u32** u32s[17] = {&s.sk,   &s.sv,    &s.sk_alt,    &s.sv_alt,   &s.flags,   &s.gsize, &s.admitted, &s.rank, &s.pos,
                      &s.added, &s.src_index, &s.head_ord, &s.grp_cnt, &s.a_ord, &s.a_j,   &s.dest,     &s.gslot};
    for (int i = 0; i < 17; ++i) *u32s[i] = reinterpret_cast<u32*>(base + kLayout.u32s[i]);
    s.gstart = reinterpret_cast<u32*>(base + kLayout.gstart);
    s.slot_cnt = reinterpret_cast<u32*>(base + kLayout.slot_cnt);
    s.slot_base = reinterpret_cast<u32*>(base + kLayout.slot_base);
    s.partials = reinterpret_cast<u32*>(base + kLayout.partials);
    s.scal = reinterpret_cast<u32*>(base + kLayout.scal);
    s.src = reinterpret_cast<float4*>(base + kLayout.src);
    s.src_cov = reinterpret_cast<float4*>(base + kLayout.src_cov);

    // The array keeps the previous call's contents, possibly of a call that stopped half-way:
    // the per-slot counters are zeroed here, map_clear resets the table, the bucket ring and the
    // map counters, and the insert resets every other counter and flag it reads.
    cudaError_t e = cudaMemsetAsync(s.slot_cnt, 0, (size_t)(kLocalCap + 1) * sizeof(u32), st);
    if (e == cudaSuccess) e = pack_points(xyz, (u32)n, stride_bytes, s.in4, st);
    if (e == cudaSuccess) e = map_clear(local, st);
    InsertCfg cfg;
    if (e == cudaSuccess) e = map_insert_batch(local, s, (u32)n, nullptr, cfg, false, st, DevicePose(), nullptr, true);
    if (e == cudaSuccess) e = make_sources(local, s, (u32)n, out_knn_ids, st);
    if (e == cudaSuccess) e = export_sources(s, (u32)n, out_index, out_cov, out_valid, st);
    u32 h_n = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h_n, s.scal + SCAL_NADMIT, sizeof(u32), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        char msg[200];
        snprintf(msg, sizeof(msg), "far_scan_sources_static: CUDA error: %s", cudaGetErrorString(e));
        return reject(FAR_ERR_CUDA, msg);
    }
    *n_src = h_n;
    return FAR_OK;
}
