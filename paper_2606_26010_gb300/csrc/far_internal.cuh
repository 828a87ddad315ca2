// Internal device structures and helpers of the FAR registration library (sm_103a).
//
// Voxel map layout in HBM (cuVoxelMap analogue, FAR-LIO Sec. III-A.2):
//   slots[cap]    16 B open-addressing slots {u64 key, u32 bucket, u32 count};
//                 eight slots per 128 B line, linear probing with step 1, so a
//                 lookup normally touches one line. Keys pack the 3 voxel
//                 indices (21 bits each).
//   pts[B * N]    float4 {x, y, z, id bits} per point, N = max points per voxel,
//                 bucket b occupies pts[b * N, b * N + N).
//   cov[2 B N]    two float4 per point {c00 c01 c02 c11} {c12 c22 valid 0}.
//   ring[B]       free-bucket ring (allocation at head, eviction returns at tail).
//
// Precision variant (precision_mode = 1, 50 m tiles):
//   pts           {x, y, z} relative to the origin of the voxel's 50 m tile, id bits.
//   cov_h4[B N]   FP16 {c00 c01 c02 c11} per point,
//   cov_h2[B N]   FP16 {c12 c22} per point: the values are Sigma / 2^E with E the
//                 voxel's exponent; a zero c00 marks an invalid covariance.
//   cexp[B]       per-voxel exponent E (the largest entry of any point of the voxel
//                 is below 2^E), raised as points arrive (older entries rescaled).
#pragma once

#include <cstdint>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

namespace far {

// Host-side count of kernel launches issued by the library (all maps, all threads).
void note_launch();
// Set the message far_last_error() returns on the calling thread.
void set_last_error(const char* msg);
// Launch a kernel and count it. Every kernel of the library begins with pdl_wait() and is
// launched with programmatic dependent launch (FAR_LAUNCH_PDL below).
#define FAR_LAUNCH(kernel_, grid_, block_, smem_, stream_, ...) \
    FAR_LAUNCH_PDL(kernel_, grid_, block_, smem_, stream_, __VA_ARGS__)

// Programmatic dependent launch: the kernel may start while the previous kernel of its stream
// still runs (hiding the launch latency); it must call pdl_wait() before it touches anything
// that kernel wrote, and pdl_wait() returns once that kernel has completed and its writes are
// visible. Kernels launched this way call pdl_wait() first.
#define FAR_LAUNCH_PDL(kernel_, grid_, block_, smem_, stream_, ...)                     \
    do {                                                                                 \
        cudaLaunchConfig_t cfg__ = {};                                                   \
        cfg__.gridDim = dim3(grid_);                                                     \
        cfg__.blockDim = dim3(block_);                                                   \
        cfg__.dynamicSmemBytes = (smem_);                                                \
        cfg__.stream = (stream_);                                                        \
        cudaLaunchAttribute at__[1];                                                     \
        at__[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;                 \
        at__[0].val.programmaticStreamSerializationAllowed = 1;                          \
        cfg__.attrs = at__;                                                              \
        cfg__.numAttrs = 1;                                                              \
        (void)cudaLaunchKernelEx(&cfg__, kernel_, __VA_ARGS__);                          \
        ::far::note_launch();                                                            \
    } while (0)

typedef unsigned long long u64;
typedef uint32_t u32;

constexpr u64 KEY_EMPTY = ~0ull;          // memset(0xFF) state of a slot
constexpr u64 KEY_TOMB = ~0ull - 1ull;    // evicted voxel
constexpr u64 KEY_INVALID = ~0ull - 2ull; // point without a key (never stored)
constexpr u32 NO_BUCKET = 0xFFFFFFFFu;
constexpr u32 NO_ID = 0xFFFFFFFFu;
constexpr int KEY_BIAS = 1 << 20;         // keys lie in [-2^20, 2^20)
constexpr float KEY_LIMIT = 1048576.0f;
constexpr int KMAX = 16;                  // largest k of the kNN kernels
constexpr int NMAX_LIMIT = 64;            // largest N_max
constexpr float TILE_M = 50.0f;           // tile side of the precision variant
constexpr double TILE_D = 50.0;
constexpr int EXP_NONE = -1000;           // voxel without a valid FP16 covariance yet

enum ErrFlag : u32 {
    ERR_TABLE_FULL = 1u,
    ERR_BUCKETS_FULL = 2u,
    ERR_ID_OVERFLOW = 4u,
    ERR_TIMEOUT = 8u,
};

struct __align__(16) Slot {
    u64 key;
    u32 bucket;
    u32 count;
};

// Device-resident counters of one map.
struct MapCounters {
    u32 ring_head;       // next free-ring position to allocate from
    u32 ring_tail;       // next free-ring position to return to
    u32 n_voxels;        // live voxels (slots holding a key)
    u32 n_tomb;          // tombstones
    u32 next_id;         // next point id
    u32 max_probe;       // longest probe distance of any stored key
    u32 err;             // ErrFlag bits
    u32 n_dropped;       // points dropped by capacity errors
    unsigned long long n_points;      // live points
    unsigned long long removed;       // points removed by the last eviction
    unsigned long long near_sum;      // ASMD: sum of near-voxel candidate counts
    unsigned long long near_cnt;      // ASMD: number of near voxels
    u32 n_added;         // points admitted by the last insert
    u32 pad[3];
};

// Read-only view of a map handed to search kernels.
struct MapView {
    const Slot* slots;
    const float4* pts;
    const float4* cov;   // may be null (scan-local map, precision variant)
    const MapCounters* ctr;
    u32 mask;
    u32 nmax;
    float inv_v;
    float v;
    int tv;              // voxels per tile side (precision variant), else 0
    const uint2* cov_h4; // precision variant covariances (see above)
    const u32* cov_h2;
    const int* cexp;
};

// Registration state kept on the device between Gauss-Newton launches.
struct RegState {
    double T[16];        // current pose
    double H[36];        // last linearisation
    double g[6];
    double xi[6];
    double chi2;
    double xi_norm2;     // squared norm of the last increment
    u32 n_corr, n_p2p;
    u32 iters;           // updates applied
    u32 converged;
    u32 status;          // 0 ok, 5 degenerate, 6 time budget, 7 graph loop overran (internal)
    u32 done;            // stop flag read at kernel entry
    u32 block_counter;   // last-block detection
    u32 trips;           // executions of the graph loop's body (bounds the loop)
    double red[32];      // the reduced values of the last linearisation (one per solve block)
    u32 n_src;           // source points of this registration
    unsigned long long t_start_ns;  // %globaltimer at the start of the registration
};

// Wait for the previous kernel of the stream (programmatic dependent launch); a no-op for a
// kernel launched without the attribute.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
// Allow the next programmatically dependent kernel of the stream to begin launching.
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// ----------------------------------------------------------------------------- keys
__device__ __forceinline__ bool voxel_key3(float x, float y, float z, float inv_v, int& kx, int& ky, int& kz) {
    // Key reading: floor(x * fp32(1/v)) with one FP32 rounding of the product.
    float sx = __fmul_rn(x, inv_v), sy = __fmul_rn(y, inv_v), sz = __fmul_rn(z, inv_v);
    if (!(sx >= -KEY_LIMIT && sx < KEY_LIMIT && sy >= -KEY_LIMIT && sy < KEY_LIMIT && sz >= -KEY_LIMIT &&
          sz < KEY_LIMIT))
        return false;
    kx = (int)floorf(sx);
    ky = (int)floorf(sy);
    kz = (int)floorf(sz);
    return true;
}

__device__ __forceinline__ bool key_in_range(int k) { return k >= -KEY_BIAS && k < KEY_BIAS; }

__device__ __forceinline__ u64 pack_key(int kx, int ky, int kz) {
    return ((u64)(u32)(kx + KEY_BIAS) << 42) | ((u64)(u32)(ky + KEY_BIAS) << 21) | (u64)(u32)(kz + KEY_BIAS);
}

__device__ __forceinline__ void unpack_key(u64 k, int& kx, int& ky, int& kz) {
    kx = (int)((k >> 42) & 0x1FFFFF) - KEY_BIAS;
    ky = (int)((k >> 21) & 0x1FFFFF) - KEY_BIAS;
    kz = (int)(k & 0x1FFFFF) - KEY_BIAS;
}

// Spatial hash of Teschner/Niessner (primes 73856093, 19349669, 83492791) on the voxel
// indices, followed by the MurmurHash3 32-bit finalizer: the XOR of products alone leaves
// neighbouring voxels in clusters of the low bits, which lengthens linear-probing runs in a
// power-of-two table. The finalizer is a bijection, so distinct hashes stay distinct; only
// slot placement changes, never a result.
__device__ __forceinline__ u32 hash_key(int kx, int ky, int kz) {
    u32 h = ((u32)kx * 73856093u) ^ ((u32)ky * 19349669u) ^ ((u32)kz * 83492791u);
    h ^= h >> 16;
    h *= 0x85ebca6bu;
    h ^= h >> 13;
    h *= 0xc2b2ae35u;
    h ^= h >> 16;
    return h;
}

// Candidate distance reading: ((dx*dx + dy*dy) + dz*dz), FP32 round-to-nearest, no contraction.
__device__ __forceinline__ float dist2_rn(float ax, float ay, float az, float bx, float by, float bz) {
    float dx = __fsub_rn(ax, bx), dy = __fsub_rn(ay, by), dz = __fsub_rn(az, bz);
    return __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
}

// Find the slot of a key; returns its contents in `out` (bucket/count) or false.
__device__ __forceinline__ bool find_slot(const Slot* __restrict__ slots, u32 mask, u32 max_probe, int kx, int ky,
                                          int kz, u32& bucket, u32& count) {
    const u64 key = pack_key(kx, ky, kz);
    u32 h = hash_key(kx, ky, kz) & mask;
    for (u32 p = 0; p <= max_probe; ++p) {
        uint4 raw = __ldg(reinterpret_cast<const uint4*>(slots + h));
        u64 k = ((u64)raw.y << 32) | raw.x;
        if (k == key) {
            bucket = raw.z;
            count = raw.w;
            return raw.z != NO_BUCKET;
        }
        if (k == KEY_EMPTY) return false;
        h = (h + 1) & mask;
    }
    return false;
}

// (d2, id) lexicographic "better than"
__device__ __forceinline__ bool better(float d2, u32 id, float bd2, u32 bid) {
    return d2 < bd2 || (d2 == bd2 && id < bid);
}

// ----------------------------------------------------------------------------- precision variant
__device__ __forceinline__ int floor_div(int k, int tv) { return k >= 0 ? k / tv : -((-k + tv - 1) / tv); }

// floor(x / 50) in exact arithmetic, without an FP64 division: the floor of x * 0.02 is
// off by at most one, which the exact products 50 T and 50 (T + 1) settle.
__device__ __forceinline__ double tile_floor(double x) {
    double T = floor(__dmul_rn(x, 0.02));
    if (__dmul_rn(TILE_D, T) > x) T -= 1.0;
    else if (__dmul_rn(TILE_D, T + 1.0) <= x) T += 1.0;
    return T;
}

// Tile reading: T = floor(x / 50) (exact), x_t = fp32(x - 50 T), key = T tv + clamp(floor(fp32(x_t * inv_v)),
// 0, tv - 1). Returns false when x is not finite or the key leaves [-2^20, 2^20).
__device__ __forceinline__ bool tile_key_axis(double x, float inv_v, int tv, int& key, float& local) {
    if (!isfinite(x)) return false;
    const double T = tile_floor(x);
    if (!(fabs(T) * (double)tv < (double)KEY_BIAS)) return false;
    const float xt = __double2float_rn(__dsub_rn(x, __dmul_rn(TILE_D, T)));
    int kin = (int)floorf(__fmul_rn(xt, inv_v));
    kin = kin < 0 ? 0 : (kin > tv - 1 ? tv - 1 : kin);
    const long long k = (long long)T * tv + kin;
    if (k < -(long long)KEY_BIAS || k >= (long long)KEY_BIAS) return false;
    key = (int)k;
    local = xt;
    return true;
}

// 2^e as a float for |e| <= 126 (exact power of two).
__device__ __forceinline__ float pow2f(int e) { return __int_as_float((127 + e) << 23); }

// Exponent E with every |c_j| < 2^E (frexp of the largest magnitude); EXP_NONE for all zeros.
__device__ __forceinline__ int cov_exponent(const float (&c)[6]) {
    float m = 0.f;
#pragma unroll
    for (int j = 0; j < 6; ++j) m = fmaxf(m, fabsf(c[j]));
    if (!(m > 0.f) || !isfinite(m)) return EXP_NONE;
    int e;
    frexpf(m, &e);
    return e < -100 ? -100 : (e > 100 ? 100 : e);
}

// FP16 record of c / 2^E (round to nearest).
__device__ __forceinline__ void cov16_encode(const float (&c)[6], int E, uint2& h4, u32& h2) {
    const float s = pow2f(-E);
    const __half h[6] = {__float2half_rn(c[0] * s), __float2half_rn(c[1] * s), __float2half_rn(c[2] * s),
                         __float2half_rn(c[3] * s), __float2half_rn(c[4] * s), __float2half_rn(c[5] * s)};
    h4.x = (u32)__half_as_ushort(h[0]) | ((u32)__half_as_ushort(h[1]) << 16);
    h4.y = (u32)__half_as_ushort(h[2]) | ((u32)__half_as_ushort(h[3]) << 16);
    h2 = (u32)__half_as_ushort(h[4]) | ((u32)__half_as_ushort(h[5]) << 16);
}

// Decode; returns false for an invalid record (c00 == 0).
__device__ __forceinline__ bool cov16_decode(uint2 h4, u32 h2, int E, float (&c)[6]) {
    const float s = pow2f(E < -100 ? -100 : E);
    c[0] = __half2float(__ushort_as_half((unsigned short)(h4.x & 0xFFFFu))) * s;
    c[1] = __half2float(__ushort_as_half((unsigned short)(h4.x >> 16))) * s;
    c[2] = __half2float(__ushort_as_half((unsigned short)(h4.y & 0xFFFFu))) * s;
    c[3] = __half2float(__ushort_as_half((unsigned short)(h4.y >> 16))) * s;
    c[4] = __half2float(__ushort_as_half((unsigned short)(h2 & 0xFFFFu))) * s;
    c[5] = __half2float(__ushort_as_half((unsigned short)(h2 >> 16))) * s;
    return (h4.x & 0xFFFFu) != 0u;
}

}  // namespace far
