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

__global__ void k_scan_reduce(const u32* __restrict__ in, u32 n, const u32* __restrict__ n_dev, u32* partials) {
    pdl_wait();
    pdl_trigger();
    __shared__ u32 sw[33];
    if (n_dev) n = min(n, *n_dev);
    const u32 base = blockIdx.x * SCAN_TILE;
    u32 s = 0;
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i) {
        u32 idx = base + i * SCAN_THREADS + threadIdx.x;
        if (idx < n) s += in[idx];
    }
    u32 total;
    block_excl_scan(s, sw, total);
    if (threadIdx.x == 0) partials[blockIdx.x] = total;
}

// Downsweep: every block adds up the sums of the blocks before it (a short strided
// sum over at most a few hundred partials) and scans its own tile; the last block also
// writes the total. Two launches per scan, no waiting between blocks.
__global__ void k_scan_down(const u32* __restrict__ in, u32* __restrict__ out, u32 n, const u32* __restrict__ n_dev,
                            const u32* __restrict__ partials, u32 nb, u32* __restrict__ total_out) {
    pdl_wait();
    pdl_trigger();
    __shared__ u32 sw[33];
    __shared__ u32 s_off;
    if (n_dev) n = min(n, *n_dev);
    u32 pre = 0;
    for (u32 b = threadIdx.x; b < blockIdx.x; b += blockDim.x) pre += partials[b];
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
        v[i] = (base + i < n) ? in[base + i] : 0u;
        s += v[i];
    }
    u32 total;
    u32 run = block_excl_scan(s, sw, total) + off;
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i)
        if (base + i < n) {
            out[base + i] = run;
            run += v[i];
        }
    if (total_out && blockIdx.x == nb - 1 && threadIdx.x == 0) *total_out = off + total;
}

}  // namespace

u32 scan_blocks(u32 n) { return (n + SCAN_TILE - 1) / SCAN_TILE; }

cudaError_t scan_exclusive(const u32* in, u32* out, u32 n, const u32* n_dev, u32* total_dev, u32* partials,
                           cudaStream_t s) {
    u32 nb = scan_blocks(n);
    if (nb == 0) nb = 1;
    if (nb > 1024u * 64u) return cudaErrorInvalidValue;
    FAR_LAUNCH(k_scan_reduce, nb, SCAN_THREADS, 0, s, in, n, n_dev, partials);
    FAR_LAUNCH(k_scan_down, nb, SCAN_THREADS, 0, s, in, out, n, n_dev, partials, nb, total_dev);
    return cudaGetLastError();
}

}  // namespace far
