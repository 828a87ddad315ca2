// Device-wide exclusive scan (u32). Used for voxel ordinals, point ids (admission flags in
// input order) and the grouped order of admitted points.
#include "primitives.cuh"

namespace far {

namespace {

constexpr int SCAN_THREADS = 256;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

__device__ __forceinline__ u32 warp_incl_scan(u32 v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        u32 t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

// Exclusive scan of one value per thread over the block; returns the block total via `total`.
__device__ __forceinline__ u32 block_excl_scan(u32 v, u32* smem_warp, u32& total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    u32 incl = warp_incl_scan(v);
    if (lane == 31) smem_warp[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        u32 w = (lane < nwarps) ? smem_warp[lane] : 0u;
        u32 wi = warp_incl_scan(w);
        if (lane < nwarps) smem_warp[lane] = wi - w;
        if (lane == nwarps - 1) smem_warp[32] = wi;
    }
    __syncthreads();
    u32 res = incl - v + smem_warp[warp];
    total = smem_warp[32];
    __syncthreads();
    return res;
}

// One array of a launch: blockIdx.y selects the job; each job has nb partial sums.
struct ScanJob {
    const u32* in;
    u32* out;
    u32 n;
    const u32* n_dev;   // may be null
    u32* total;         // may be null
};
struct ScanJobs {
    ScanJob j[2];
    u32 nb;             // blocks per job
};

__global__ void k_scan_reduce(ScanJobs J, u32* partials) {
    pdl_wait();
    pdl_trigger();
    __shared__ u32 sw[33];
    const ScanJob jb = J.j[blockIdx.y];
    u32 n = jb.n;
    if (jb.n_dev) n = min(n, *jb.n_dev);
    const u32 base = blockIdx.x * SCAN_TILE;
    u32 s = 0;
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i) {
        u32 idx = base + i * SCAN_THREADS + threadIdx.x;
        if (idx < n) s += jb.in[idx];
    }
    u32 total;
    block_excl_scan(s, sw, total);
    if (threadIdx.x == 0) partials[blockIdx.y * J.nb + blockIdx.x] = total;
}

// Downsweep: every block adds up the sums of the blocks before it (a short strided
// sum over at most a few hundred partials) and scans its own tile; the last block also
// writes the total. Two launches per scan, no waiting between blocks.
__global__ void k_scan_down(ScanJobs J, const u32* __restrict__ partials) {
    pdl_wait();
    pdl_trigger();
    __shared__ u32 sw[33];
    __shared__ u32 s_off;
    const ScanJob jb = J.j[blockIdx.y];
    const u32* part = partials + blockIdx.y * J.nb;
    u32 n = jb.n;
    if (jb.n_dev) n = min(n, *jb.n_dev);
    u32 pre = 0;
    for (u32 b = threadIdx.x; b < blockIdx.x; b += blockDim.x) pre += part[b];
    u32 ptot;
    block_excl_scan(pre, sw, ptot);
    if (threadIdx.x == 0) s_off = ptot;
    __syncthreads();
    const u32 off = s_off;
    const u32 base = blockIdx.x * SCAN_TILE + threadIdx.x * SCAN_ITEMS;
    u32 v[SCAN_ITEMS];
    u32 s = 0;
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i) {
        v[i] = (base + i < n) ? jb.in[base + i] : 0u;
        s += v[i];
    }
    u32 total;
    u32 run = block_excl_scan(s, sw, total) + off;
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i)
        if (base + i < n) {
            jb.out[base + i] = run;
            run += v[i];
        }
    if (jb.total && blockIdx.x == J.nb - 1 && threadIdx.x == 0) *jb.total = off + total;
}

cudaError_t scan_jobs(const ScanJobs& J, u32 njobs, u32* partials, cudaStream_t s) {
    if (J.nb > 1024u * 64u) return cudaErrorInvalidValue;
    const dim3 grid(J.nb, njobs);
    FAR_LAUNCH(k_scan_reduce, grid, SCAN_THREADS, 0, s, J, partials);
    FAR_LAUNCH(k_scan_down, grid, SCAN_THREADS, 0, s, J, partials);
    return cudaGetLastError();
}

}  // namespace

u32 scan_blocks(u32 n) { return (n + SCAN_TILE - 1) / SCAN_TILE; }

cudaError_t scan_exclusive(const u32* in, u32* out, u32 n, const u32* n_dev, u32* total_dev, u32* partials,
                           cudaStream_t s) {
    ScanJobs J{};
    J.j[0] = ScanJob{in, out, n, n_dev, total_dev};
    J.nb = max(1u, scan_blocks(n));
    return scan_jobs(J, 1, partials, s);
}

cudaError_t scan_exclusive2(const u32* in0, u32* out0, const u32* n_dev0, u32* total0, const u32* in1, u32* out1,
                            const u32* n_dev1, u32* total1, u32 n, u32* partials, cudaStream_t s) {
    ScanJobs J{};
    J.j[0] = ScanJob{in0, out0, n, n_dev0, total0};
    J.j[1] = ScanJob{in1, out1, n, n_dev1, total1};
    J.nb = max(1u, scan_blocks(n));
    return scan_jobs(J, 2, partials, s);
}

}  // namespace far
