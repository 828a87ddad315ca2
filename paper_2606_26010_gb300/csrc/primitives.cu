// Device-wide exclusive scan and stable LSD radix sort (u32 key, u32 value).
// Used to group scan points by voxel in input order (deterministic admission)
// and to assign point ids in input order.
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

// ------------------------------------------------------------------ radix sort
constexpr int RS_THREADS = 256;
constexpr int RS_ROUNDS = 8;
constexpr int RS_TILE = RS_THREADS * RS_ROUNDS;
constexpr int RS_BINS = 256;

__global__ void k_radix_hist(const u32* __restrict__ keys, u32 n, int shift, u32* __restrict__ hist, u32 nblk) {
    pdl_wait();
    pdl_trigger();
    __shared__ u32 h[RS_BINS];
    h[threadIdx.x] = 0;
    __syncthreads();
    const u32 base = blockIdx.x * RS_TILE;
#pragma unroll
    for (int r = 0; r < RS_ROUNDS; ++r) {
        u32 idx = base + r * RS_THREADS + threadIdx.x;
        if (idx < n) atomicAdd(&h[(keys[idx] >> shift) & 0xFFu], 1u);
    }
    __syncthreads();
    hist[threadIdx.x * nblk + blockIdx.x] = h[threadIdx.x];
}

// Stable scatter: items of a tile are ranked in index order (round-major, then
// thread order), using warp match_any for the rank among equal digits.
__global__ void k_radix_scatter(const u32* __restrict__ keys, const u32* __restrict__ vals, u32 n, int shift,
                                const u32* __restrict__ offs, u32 nblk, u32* __restrict__ keys_out,
                                u32* __restrict__ vals_out) {
    pdl_wait();
    pdl_trigger();
    __shared__ u32 wcnt[RS_THREADS / 32][RS_BINS];
    __shared__ u32 running[RS_BINS];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const u32 lt_mask = (1u << lane) - 1u;
    running[threadIdx.x] = offs[threadIdx.x * nblk + blockIdx.x];
    const u32 base = blockIdx.x * RS_TILE;
    for (int r = 0; r < RS_ROUNDS; ++r) {
        const u32 idx = base + r * RS_THREADS + threadIdx.x;
        const bool ok = idx < n;
        const u32 k = ok ? keys[idx] : 0u;
        const u32 v = ok ? vals[idx] : 0u;
        const u32 d = ok ? ((k >> shift) & 0xFFu) : 0x100u;
#pragma unroll
        for (int w = 0; w < RS_THREADS / 32; ++w) wcnt[w][threadIdx.x] = 0;
        __syncthreads();
        const u32 peers = __match_any_sync(0xffffffffu, d);
        const u32 rank = __popc(peers & lt_mask);
        if (ok && lane == __ffs(peers) - 1) wcnt[warp][d] = __popc(peers);
        __syncthreads();
        {
            u32 b = running[threadIdx.x];
#pragma unroll
            for (int w = 0; w < RS_THREADS / 32; ++w) {
                u32 c = wcnt[w][threadIdx.x];
                wcnt[w][threadIdx.x] = b;
                b += c;
            }
            running[threadIdx.x] = b;
        }
        __syncthreads();
        if (ok) {
            const u32 pos = wcnt[warp][d] + rank;
            keys_out[pos] = k;
            vals_out[pos] = v;
        }
        __syncthreads();
    }
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

u32 radix_blocks(u32 n) { return (n + RS_TILE - 1) / RS_TILE; }

cudaError_t radix_sort_pairs(u32* keys, u32* vals, u32* keys_alt, u32* vals_alt, u32 n, int bits, u32* hist,
                             u32* scan_partials, cudaStream_t s, bool* result_in_alt) {
    *result_in_alt = false;
    if (n == 0) return cudaSuccess;
    const u32 nblk = radix_blocks(n);
    u32 *kin = keys, *vin = vals, *kout = keys_alt, *vout = vals_alt;
    for (int shift = 0; shift < bits; shift += 8) {
        FAR_LAUNCH(k_radix_hist, nblk, RS_THREADS, 0, s, kin, n, shift, hist, nblk);
        cudaError_t e = scan_exclusive(hist, hist, RS_BINS * nblk, nullptr, nullptr, scan_partials, s);
        if (e != cudaSuccess) return e;
        FAR_LAUNCH(k_radix_scatter, nblk, RS_THREADS, 0, s, kin, vin, n, shift, hist, nblk, kout, vout);
        u32* t = kin; kin = kout; kout = t;
        t = vin; vin = vout; vout = t;
        *result_in_alt = !*result_in_alt;
    }
    return cudaGetLastError();
}

}  // namespace far
