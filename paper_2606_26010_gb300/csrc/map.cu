// Voxel map kernels: batched insert with the spacing rule and the Adaptive
// Submap Density cap, eviction, rebuild, export helpers and stage searches.
// FAR-LIO Sec. III-A.2 (cuVoxelMap) and Sec. III-A.3 (submap update).
//
// Determinism: the points of a batch are grouped by hash slot (a per-slot counter gives
// each point its rank in its group and each group a contiguous range, placed in whatever
// order the atomics happen to run); each group is then sorted by input index, so admission
// inside a voxel follows the input order; point ids are an exclusive scan of the admission
// flags in input order. Slot, bucket and group placement depend on thread timing, but
// nothing visible does.
#include "map.cuh"
#include "primitives.cuh"
#include "search.cuh"

namespace far {

namespace {

constexpr int TPB = 256;

inline u32 blocks_for(u32 n, u32 tpb = TPB) {
    u32 b = (n + tpb - 1) / tpb;
    return b ? b : 1;
}

__global__ void k_pack(const char* __restrict__ src, u32 n, u32 stride, float4* __restrict__ out) {
    pdl_wait();
    pdl_trigger();
    const u32 i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float* p = reinterpret_cast<const float*>(src + (size_t)i * stride);
    out[i] = make_float4(p[0], p[1], p[2], __uint_as_float(i));
}

// Sec. III-A.1 motion undistortion of one point (FP32): the LiDAR pose at its firing time tau,
// relative to the reference time, is the SE(3) exponential of the twist integrated from 0 to
// tau, [phi; rho] = [w0 tau + w1 tau^2 / 2; v0 tau + v1 tau^2 / 2]; the point moves to
// p_ref = R(phi) p + V(phi) rho with R = I + A [phi]x + B [phi]x^2, V = I + B [phi]x + C [phi]x^2,
// A = sin(t)/t, B = (1 - cos t)/t^2, C = (t - sin t)/t^3, t = |phi| (Taylor series below t = 0.25,
// terms to t^6; the first omitted term is below 1e-8 of the leading one).
__device__ __forceinline__ float3 deskew_point(float x, float y, float z, float tau, const SweepMotion& mo) {
    const float h = 0.5f * tau * tau;
    float ph[3], ro[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        ph[a] = fmaf(mo.w1[a], h, mo.w0[a] * tau);
        ro[a] = fmaf(mo.v1[a], h, mo.v0[a] * tau);
    }
    const float t2 = ph[0] * ph[0] + ph[1] * ph[1] + ph[2] * ph[2];
    float A, B, C;
    if (t2 < 0.0625f) {
        A = 1.0f - t2 * (1.0f / 6.0f) * (1.0f - t2 * (1.0f / 20.0f) * (1.0f - t2 * (1.0f / 42.0f)));
        B = 0.5f * (1.0f - t2 * (1.0f / 12.0f) * (1.0f - t2 * (1.0f / 30.0f) * (1.0f - t2 * (1.0f / 56.0f))));
        C = (1.0f / 6.0f) * (1.0f - t2 * (1.0f / 20.0f) * (1.0f - t2 * (1.0f / 42.0f) * (1.0f - t2 * (1.0f / 72.0f))));
    } else {
        const float t = sqrtf(t2);
        float sn, cs;
        sincosf(t, &sn, &cs);
        A = sn / t;
        B = (1.0f - cs) / t2;
        C = (t - sn) / (t2 * t);
    }
    // [phi]x p and [phi]x^2 p = phi x (phi x p)
    const float c1x = ph[1] * z - ph[2] * y, c1y = ph[2] * x - ph[0] * z, c1z = ph[0] * y - ph[1] * x;
    const float c2x = ph[1] * c1z - ph[2] * c1y, c2y = ph[2] * c1x - ph[0] * c1z, c2z = ph[0] * c1y - ph[1] * c1x;
    const float r1x = ph[1] * ro[2] - ph[2] * ro[1], r1y = ph[2] * ro[0] - ph[0] * ro[2], r1z = ph[0] * ro[1] - ph[1] * ro[0];
    const float r2x = ph[1] * r1z - ph[2] * r1y, r2y = ph[2] * r1x - ph[0] * r1z, r2z = ph[0] * r1y - ph[1] * r1x;
    const float tx = ro[0] + B * r1x + C * r2x, ty = ro[1] + B * r1y + C * r2y, tz = ro[2] + B * r1z + C * r2z;
    return make_float3(x + A * c1x + B * c2x + tx, y + A * c1y + B * c2y + ty, z + A * c1z + B * c2z + tz);
}

__global__ void k_pack_deskew(const char* __restrict__ src, u32 n, u32 stride, SweepMotion mo,
                              float4* __restrict__ out4, float* __restrict__ out3) {
    pdl_wait();
    pdl_trigger();
    const u32 i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const char* rec = src + (size_t)i * stride;
    const float* p = reinterpret_cast<const float*>(rec);
    const float tau = *reinterpret_cast<const float*>(rec + mo.time_offset);
    const float3 q = deskew_point(p[0], p[1], p[2], tau, mo);
    if (out4) out4[i] = make_float4(q.x, q.y, q.z, __uint_as_float(i));
    if (out3) {
        out3[3 * (size_t)i] = q.x;
        out3[3 * (size_t)i + 1] = q.y;
        out3[3 * (size_t)i + 2] = q.z;
    }
}

// Slot of a point's voxel (inserting new keys), and the point's arrival rank among the points of
// this batch in that slot (out_rank, from the per-slot counter slot_cnt). The lanes of a warp that
// found the same slot take their ranks with one atomic (points of a voxel arrive together in scan
// order). Every lane of the warp calls this (key KEY_INVALID and i >= n for lanes without a point).
__device__ __forceinline__ void find_or_insert_slot(u64 key, u32 i, u32 n, Slot* slots, u32 mask,
                                                    u32* __restrict__ out_slot, u32* __restrict__ out_rank,
                                                    MapCounters* ctr, u32* __restrict__ slot_cnt) {
    const int lane = threadIdx.x & 31;
    const u32 sentinel = mask + 1u;
    u32 found = sentinel, probes = 0;
    if (key != KEY_INVALID) {
        int kx, ky, kz;
        unpack_key(key, kx, ky, kz);
        u32 h = hash_key(kx, ky, kz) & mask;
        for (u32 p = 0; p <= mask; ++p) {
            const u64 k = *reinterpret_cast<volatile u64*>(&slots[h].key);
            if (k == key) {
                found = h;
                probes = p;
                break;
            }
            if (k == KEY_EMPTY) {
                const u64 old = atomicCAS(&slots[h].key, KEY_EMPTY, key);
                if (old == KEY_EMPTY || old == key) {
                    found = h;
                    probes = p;
                    break;
                }
            }
            h = (h + 1u) & mask;
        }
        if (found == sentinel) {
            atomicOr(&ctr->err, (u32)ERR_TABLE_FULL);
            atomicAdd(&ctr->n_dropped, 1u);
        }
    }
    const u32 peers = __match_any_sync(0xffffffffu, found);
    const int leader = __ffs(peers) - 1;
    u32 base = 0;
    if (lane == leader && found != sentinel) base = atomicAdd(&slot_cnt[found], (u32)__popc(peers));
    base = __shfl_sync(0xffffffffu, base, leader);
    const u32 pmax = __reduce_max_sync(0xffffffffu, probes);
    if (lane == 0 && pmax > 0) atomicMax(&ctr->max_probe, pmax);
    if (i >= n) return;
    out_slot[i] = found;
    if (found != sentinel) out_rank[i] = base + (u32)__popc(peers & ((1u << lane) - 1u));
}

// a11: x_w = fp32(((R0 x + R1 y) + R2 z) + t) in FP64 without contraction; then the key, and the
// slot of the key in the map with the point's rank in it (find_or_insert_slot).
// Precision variant (tv > 0): x_w stays FP64, the key follows the tile reading and `world`
// receives the coordinates relative to the tile origin.
__global__ void k_world_keys(const float4* __restrict__ in, u32 n, Pose12 T, int has_pose, DevicePose dp,
                             float inv_v, int tv, float4* __restrict__ world, u64* __restrict__ keys,
                             u32* __restrict__ scal, MapCounters* ctr, u32* __restrict__ admitted,
                             u32* __restrict__ flags, Slot* slots, u32 mask, u32* __restrict__ out_slot,
                             u32* __restrict__ out_rank, u32* __restrict__ slot_cnt) {
    pdl_wait();
    pdl_trigger();
    const u32 i = blockIdx.x * blockDim.x + threadIdx.x;
    // the insert's first kernel clears its per-insert state (scalars, ASMD sums, admitted flags)
    // and records the first id it will assign
    if (i < SCAL_COUNT) scal[i] = (i == SCAL_IDBASE) ? ctr->next_id : 0u;
    if (i == 0) {
        ctr->near_sum = 0ull;
        ctr->near_cnt = 0ull;
        ctr->n_added = 0u;
    }
    u64 key = KEY_INVALID;
    if (i < n) {
        admitted[i] = 0u;
        flags[i] = 0u;
        if (dp.T) {
#pragma unroll
            for (int j = 0; j < 12; ++j) T.m[j] = dp.T[j];
        }
        const float4 p = in[i];
        float w[3] = {p.x, p.y, p.z};
        const bool finite = isfinite(p.x) && isfinite(p.y) && isfinite(p.z) && !(dp.status && *dp.status != 0);
        if (tv > 0) {
            int k[3];
            bool ok = finite;
            for (int r = 0; r < 3 && ok; ++r) {
                double x = (&p.x)[r];
                if (has_pose) {
                    const double px = p.x, py = p.y, pz = p.z;
                    double s = __dadd_rn(__dmul_rn(T.m[4 * r + 0], px), __dmul_rn(T.m[4 * r + 1], py));
                    s = __dadd_rn(s, __dmul_rn(T.m[4 * r + 2], pz));
                    x = __dadd_rn(s, T.m[4 * r + 3]);
                }
                ok = tile_key_axis(x, inv_v, tv, k[r], w[r]);
            }
            if (ok) key = pack_key(k[0], k[1], k[2]);
        } else {
            if (has_pose && finite) {
                const double x = p.x, y = p.y, z = p.z;
#pragma unroll
                for (int r = 0; r < 3; ++r) {
                    double s = __dadd_rn(__dmul_rn(T.m[4 * r + 0], x), __dmul_rn(T.m[4 * r + 1], y));
                    s = __dadd_rn(s, __dmul_rn(T.m[4 * r + 2], z));
                    s = __dadd_rn(s, T.m[4 * r + 3]);
                    w[r] = __double2float_rn(s);
                }
            }
            int kx, ky, kz;
            if (finite && voxel_key3(w[0], w[1], w[2], inv_v, kx, ky, kz)) key = pack_key(kx, ky, kz);
        }
        world[i] = make_float4(w[0], w[1], w[2], p.w);
        keys[i] = key;
    }
    find_or_insert_slot(key, i, n, slots, mask, out_slot, out_rank, ctr, slot_cnt);
}

// Groups of more members than this are sorted by a whole block of k_group_sort (one pass over
// a bitmap of up to 262144 input indices in the block's shared memory) instead of one warp.
#ifndef FAR_GS_BLOCK_MIN
#define FAR_GS_BLOCK_MIN 1024
#endif
constexpr u32 GS_BLOCK_MIN = FAR_GS_BLOCK_MIN;

// Groups: the first point of each slot (rank 0) opens the slot's group, a contiguous range
// of its size taken from the running total, and records it under a group index. The heads of
// a warp take their group indices and ranges with one atomic each.
__global__ void k_group_alloc(const u32* __restrict__ slot_of, const u32* __restrict__ rank, u32 n, u32 sentinel,
                              const u32* __restrict__ slot_cnt, u32* __restrict__ slot_base, u32* __restrict__ scal,
                              u32* __restrict__ gstart, u32* __restrict__ gsize, u32* __restrict__ gslot,
                              u32* __restrict__ huge_list) {
    pdl_wait();
    pdl_trigger();
    const u32 i = blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    u32 h = sentinel;
    bool head = false;
    if (i < n) {
        h = slot_of[i];
        head = h != sentinel && rank[i] == 0u;
    }
    const u32 size = head ? slot_cnt[h] : 0u;
    const u32 heads = __ballot_sync(0xffffffffu, head);
    if (heads == 0u) return;
    u32 incl = size;   // inclusive prefix of the sizes over the warp
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const u32 t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    const u32 total = __shfl_sync(0xffffffffu, incl, 31);
    u32 g0 = 0, b0 = 0;
    if (lane == 0) {
        g0 = atomicAdd(&scal[SCAL_NGROUPS], (u32)__popc(heads));
        b0 = atomicAdd(&scal[SCAL_NVALID], total);
    }
    g0 = __shfl_sync(0xffffffffu, g0, 0);
    b0 = __shfl_sync(0xffffffffu, b0, 0);
    if (!head) return;
    const u32 g = g0 + (u32)__popc(heads & ((1u << lane) - 1u));
    const u32 base = b0 + incl - size;
    slot_base[h] = base;
    gstart[g] = base;
    gsize[g] = size;
    gslot[g] = h;
    if (size > GS_BLOCK_MIN) huge_list[atomicAdd(&scal[SCAL_NHUGE], 1u)] = g;
}

// Every point to its place in its group (arrival order for now).
__global__ void k_group_scatter(const u32* __restrict__ slot_of, const u32* __restrict__ rank, u32 n, u32 sentinel,
                                const u32* __restrict__ slot_base, u32* __restrict__ members) {
    pdl_wait();
    pdl_trigger();
    const u32 i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const u32 h = slot_of[i];
    if (h != sentinel) members[slot_base[h] + rank[i]] = i;
}

__device__ __forceinline__ double centre_dist2(int kx, int ky, int kz, double v, double sx, double sy,
                                               double sz) {
    const double dx = __dsub_rn(__dmul_rn(__dadd_rn((double)kx, 0.5), v), sx);
    const double dy = __dsub_rn(__dmul_rn(__dadd_rn((double)ky, 0.5), v), sy);
    const double dz = __dsub_rn(__dmul_rn(__dadd_rn((double)kz, 0.5), v), sz);
    return __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
}

// Sort of one group's input indices by one warp (values are distinct; at most GS_BLOCK_MIN of
// them, larger groups go to whole blocks). Groups of up to 128 are sorted in registers (bitonic
// network over 32 lanes x R values). Larger ones take the cheaper of a bitmap of their index
// range (sort_group_bitmap; its cost grows with the range) and a bitonic network over compare
// pairs in the warp's shared buffer of GS_SMEM values.
constexpr int GS_SMEM = 1024;
constexpr int GS_WARPS = TPB / 32;

// Bitonic sort of 32 * R values held R per lane (element e = lane * R + r), registers only.
template <int R>
__device__ __forceinline__ void bitonic_regs(u32 (&v)[R], int lane) {
    constexpr int N = 32 * R;
#pragma unroll
    for (int k = 2; k <= N; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            if (j < R) {
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const int p = r ^ j;
                    if (p > r) {
                        const bool up = (((lane * R + r) & k) == 0);
                        const u32 a = v[r], b = v[p];
                        v[r] = up ? min(a, b) : max(a, b);
                        v[p] = up ? max(a, b) : min(a, b);
                    }
                }
            } else {
                const int lm = j / R;
                const bool lower = (lane & lm) == 0;
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const u32 o = __shfl_xor_sync(0xffffffffu, v[r], lm);
                    const bool up = (((lane * R + r) & k) == 0);
                    v[r] = (lower == up) ? min(v[r], o) : max(v[r], o);
                }
            }
        }
    }
}

template <int R>
__device__ __forceinline__ void sort_group_regs(u32* a, u32 size, int lane) {
    u32 v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const u32 e = (u32)(lane * R + r);
        v[r] = e < size ? a[e] : 0xFFFFFFFFu;
    }
    bitonic_regs<R>(v, lane);
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const u32 e = (u32)(lane * R + r);
        if (e < size) a[e] = v[r];
    }
}

// Bitonic sort of 1024 values in shared memory by one warp: every stage's 512 compare pairs
// (i, i + j) are split over the lanes, 16 each, and loaded 8 at a time so that the loads of a
// batch are in flight together.
__device__ __forceinline__ void bitonic_smem_pairs(u32* buf, int lane) {
#pragma unroll 1
    for (int k = 2; k <= 1024; k <<= 1) {
#pragma unroll 1
        for (int j = k >> 1; j > 0; j >>= 1) {
#pragma unroll
            for (int bt = 0; bt < 2; ++bt) {
                u32 va[8], vb[8];
                int ia[8];
#pragma unroll
                for (int t = 0; t < 8; ++t) {
                    const int q = lane + 32 * (8 * bt + t);          // pair 0..511
                    const int i = ((q & ~(j - 1)) << 1) | (q & (j - 1));
                    ia[t] = i;
                    va[t] = buf[i];
                    vb[t] = buf[i + j];
                }
#pragma unroll
                for (int t = 0; t < 8; ++t) {
                    const bool up = (ia[t] & k) == 0;
                    const u32 lo = min(va[t], vb[t]), hi = max(va[t], vb[t]);
                    buf[ia[t]] = up ? lo : hi;
                    buf[ia[t] + j] = up ? hi : lo;
                }
            }
            __syncwarp();
        }
    }
}

// Sort of distinct values through a bitmap of their range [lo, hi]: each pass marks the members
// that fall in a window of 32768 values in the warp's shared buffer (1024 words), then reads
// the marks back in order, one row of 32 consecutive words (one per lane) at a time; a warp
// scan of the row's popcounts gives each lane its output position. With one pass the output
// goes to `a` in place (every member is marked before any is written), else through `tmp`.
__device__ __forceinline__ void sort_group_bitmap(u32* a, u32 size, u32 lo, u32 hi, u32* tmp, u32* buf,
                                                  int lane) {
    const u32 passes = ((hi - lo) >> 15) + 1u;
    u32* out = passes == 1u ? a : tmp;
    u32 pos = 0;   // outputs of the rows done so far (the same on every lane)
    for (u32 p = 0; p < passes; ++p) {
        const u32 w0 = lo + (p << 15);
        const u32 span = min(hi - w0, 32767u);   // the window's last offset that can hold a member
        const u32 rows = (span >> 10) + 1u;
        for (u32 r = 0; r < rows; ++r) buf[r * 32u + lane] = 0u;
        __syncwarp();
        for (u32 i = lane; i < size; i += 32) {
            const u32 d = a[i] - w0;
            if (d <= span) atomicOr(&buf[d >> 5], 1u << (d & 31u));
        }
        __syncwarp();
        for (u32 r = 0; r < rows; ++r) {
            u32 word = buf[r * 32u + lane];
            if (__ballot_sync(0xffffffffu, word != 0u) == 0u) continue;
            const u32 c = __popc(word);
            u32 incl = c;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const u32 t = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += t;
            }
            u32 q = pos + incl - c;
            const u32 base = w0 + ((r * 32u + (u32)lane) << 5);
            while (word) {
                out[q++] = base + (u32)(__ffs(word) - 1);
                word &= word - 1u;
            }
            pos += __shfl_sync(0xffffffffu, incl, 31);
        }
        __syncwarp();
    }
    if (passes > 1u) {
        for (u32 i = lane; i < size; i += 32) a[i] = tmp[i];
        __syncwarp();
    }
}

// Sort of one group's distinct input indices by the whole block, through a bitmap of their range
// [lo, hi] in windows of 262144 values (8192 words of shared memory, `buf`): all members are
// marked, then the words are read back in rows of 32 consecutive words (one per lane, the
// block's warps taking the rows in turn). A first read gives each row's count, one warp turns
// the counts into row offsets, and a second read writes every member at its row offset plus its
// lane prefix. With one window the output goes to `a` in place (every member is marked before
// any is written), else through `tmp`. Every thread of the block must call this; it ends with a
// barrier. s_rows holds 256 words, s_red 2 * GS_WARPS.
constexpr u32 GSB_WORDS = GS_WARPS * GS_SMEM;        // 8192
constexpr u32 GSB_SPAN = GSB_WORDS * 32u;             // 262144 values per window
__device__ __forceinline__ void sort_group_block(u32* a, u32 size, u32* tmp, u32* buf, u32* s_rows, u32* s_red) {
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    u32 lo = 0xFFFFFFFFu, hi = 0u;
    for (u32 i = t; i < size; i += TPB) {
        const u32 x = a[i];
        lo = min(lo, x);
        hi = max(hi, x);
    }
    lo = __reduce_min_sync(0xffffffffu, lo);
    hi = __reduce_max_sync(0xffffffffu, hi);
    if (lane == 0) {
        s_red[warp] = lo;
        s_red[GS_WARPS + warp] = hi;
    }
    __syncthreads();
#pragma unroll
    for (int w2 = 0; w2 < GS_WARPS; ++w2) {
        lo = min(lo, s_red[w2]);
        hi = max(hi, s_red[GS_WARPS + w2]);
    }
    const u32 passes = ((hi - lo) / GSB_SPAN) + 1u;
    u32* out = passes == 1u ? a : tmp;
    u32 pos = 0;   // members written by the windows before (the same in every thread)
    for (u32 p = 0; p < passes; ++p) {
        const u32 w0 = lo + p * GSB_SPAN;
        const u32 span = min(hi - w0, GSB_SPAN - 1u);   // the window's last offset that can hold a member
        const u32 rows = (span >> 10) + 1u;             // rows of 32 words (1024 values)
        __syncthreads();   // the previous window's readers (and s_red's) are done
        for (u32 i = t; i < rows * 32u; i += TPB) buf[i] = 0u;
        __syncthreads();
        for (u32 i = t; i < size; i += TPB) {
            const u32 d = a[i] - w0;
            if (d <= span) atomicOr(&buf[d >> 5], 1u << (d & 31u));
        }
        __syncthreads();
        for (u32 r = warp; r < rows; r += GS_WARPS) {
            const u32 c = __reduce_add_sync(0xffffffffu, (u32)__popc(buf[r * 32u + lane]));
            if (lane == 0) s_rows[r] = c;
        }
        __syncthreads();
        if (warp == 0) {
            // exclusive offsets of the rows (at most 256: 8 per lane), the window's total last
            u32 v[8];
            u32 sum = 0;
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const u32 r = (u32)lane * 8u + (u32)k;
                v[k] = r < rows ? s_rows[r] : 0u;
                sum += v[k];
            }
            u32 incl = sum;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const u32 y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            u32 run = incl - sum;
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const u32 r = (u32)lane * 8u + (u32)k;
                if (r < rows) s_rows[r] = run;
                run += v[k];
            }
            if (lane == 31) s_red[0] = incl;
        }
        __syncthreads();
        for (u32 r = warp; r < rows; r += GS_WARPS) {
            u32 word = buf[r * 32u + lane];
            const u32 c = __popc(word);
            u32 incl = c;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const u32 y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            u32 q = pos + s_rows[r] + incl - c;
            const u32 base = w0 + ((r * 32u + (u32)lane) << 5);
            while (word) {
                out[q++] = base + (u32)(__ffs(word) - 1);
                word &= word - 1u;
            }
        }
        pos += s_red[0];
    }
    __syncthreads();
    if (passes > 1u) {
        for (u32 i = t; i < size; i += TPB) a[i] = tmp[i];
        __syncthreads();
    }
}

__device__ __forceinline__ void sort_group(u32* a, u32 size, u32* tmp, u32* buf, int lane) {
    if (size <= 1) return;
    if (size <= 32) {
        sort_group_regs<1>(a, size, lane);
        return;
    }
    if (size <= 128) {
        sort_group_regs<4>(a, size, lane);
        return;
    }
    u32 lo = 0xFFFFFFFFu, hi = 0u;
    for (u32 i = lane; i < size; i += 32) {
        const u32 x = a[i];
        lo = min(lo, x);
        hi = max(hi, x);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    // estimated instructions per lane of each way: the bitmap ~512 per 32768 values of range
    // plus ~8 per 32 members and pass; the shared-memory network ~3300 (up to 1024 values;
    // larger groups are sorted by whole blocks, see sort_group_block)
    const unsigned long long bitmap_cost = (unsigned long long)(((hi - lo) >> 15) + 1u) * (512ull + size / 4u);
    if (bitmap_cost <= 3300ull) {
        sort_group_bitmap(a, size, lo, hi, tmp, buf, lane);
        return;
    }
    // in the warp's shared buffer, padded to 1024: a bitonic network over compare pairs, each
    // lane taking 16 of a stage's 512 pairs, their loads issued in batches of 8
    for (u32 i = lane; i < 1024; i += 32) buf[i] = i < size ? a[i] : 0xFFFFFFFFu;
    __syncwarp();
    bitonic_smem_pairs(buf, lane);
    for (u32 i = lane; i < size; i += 32) a[i] = buf[i];
    __syncwarp();
}

// Groups of more candidates than this are admitted by a whole block of k_admit rather than one
// warp (their serial walk would outlast the rest of the launch).
#ifndef FAR_ADMIT_BIG
#define FAR_ADMIT_BIG 192
#endif
constexpr u32 ADMIT_BIG = FAR_ADMIT_BIG;

// Warp w of W takes the groups w, w + W, w + 2W, ... (32 per pass, one per lane), so that the
// large groups, which lie close together in group order, spread over the warps.
// Groups of at most GS_LANE_MAX members are sorted by one lane each (insertion network in
// registers); larger ones by the whole warp (sort_group).
constexpr u32 GS_LANE_MAX = 8;

__device__ __forceinline__ void sort_lane(u32* a, u32 size, u32& head) {
    u32 v[GS_LANE_MAX];
#pragma unroll
    for (u32 r = 0; r < GS_LANE_MAX; ++r) v[r] = r < size ? a[r] : 0xFFFFFFFFu;
#pragma unroll
    for (u32 i = 1; i < GS_LANE_MAX; ++i)
#pragma unroll
        for (u32 j = i; j > 0; --j) {
            const u32 lo = min(v[j - 1], v[j]), hi = max(v[j - 1], v[j]);
            v[j - 1] = lo;
            v[j] = hi;
        }
#pragma unroll
    for (u32 r = 0; r < GS_LANE_MAX; ++r)
        if (r < size) a[r] = v[r];
    head = v[0];
}

// Each lane of a warp takes one group of a batch of 32 (strided over the group range): sort its members by input index,
// flag the group's first input index (its voxel ordinal follows from a scan of the flags),
// clear the slot's counter for the next insert and, with ASMD (a10), add the group to the
// near-voxel sums when its voxel centre lies within r_c of the sensor. Groups larger than
// GS_LANE_MAX are sorted afterwards by the whole warp, one at a time; groups larger than
// GS_BLOCK_MIN (listed by k_group_alloc in huge_list) by whole blocks once their warps are
// done; groups larger than ADMIT_BIG are listed in big_list for the admission.
__global__ void __launch_bounds__(TPB) k_group_sort(u32* __restrict__ members, u32* __restrict__ tmp,
                                                    u32* __restrict__ scal, u32* __restrict__ big_list,
                                                    const u32* __restrict__ gstart,
                                                    const u32* __restrict__ gsize, const u32* __restrict__ gslot,
                                                    u32* __restrict__ slot_cnt, u32* __restrict__ flags,
                                                    const Slot* __restrict__ slots, double v, InsertCfg cfg,
                                                    const double* __restrict__ dev_T, MapCounters* ctr,
                                                    const u32* __restrict__ huge_list) {
    pdl_wait();
    pdl_trigger();
    __shared__ u32 sbuf[GS_WARPS][GS_SMEM];
    if (cfg.asmd && dev_T) {
        cfg.sx = dev_T[3];
        cfg.sy = dev_T[7];
        cfg.sz = dev_T[11];
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const u32 ng = scal[SCAL_NGROUPS];
    const u32 warps_total = (gridDim.x * blockDim.x) >> 5;
    const u32 w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    unsigned long long near_sum = 0, near_cnt = 0;
    for (u32 j0 = 0; w + j0 * warps_total < ng; j0 += 32) {
        const u32 g = w + (j0 + lane) * warps_total;
        const bool gv = g < ng;
        u32 base = 0, size = 0, h = 0, head = 0;
        bool mine = false;   // sorted here (groups above GS_BLOCK_MIN go to whole blocks below)
        if (gv) {
            base = gstart[g];
            size = gsize[g];
            h = gslot[g];
            mine = size <= GS_BLOCK_MIN;
            if (size <= GS_LANE_MAX) sort_lane(members + base, size, head);
        }
        u32 big = __ballot_sync(0xffffffffu, mine && size > GS_LANE_MAX);
        while (big) {
            const int f = __ffs(big) - 1;
            big &= big - 1u;
            const u32 fb = __shfl_sync(0xffffffffu, base, f), fs = __shfl_sync(0xffffffffu, size, f);
            sort_group(members + fb, fs, tmp + fb, sbuf[warp], lane);
            __syncwarp();
            if (lane == f) head = members[fb];
        }
        if (mine) {
            flags[head] = 1u;
            slot_cnt[h] = 0u;
            if (size > ADMIT_BIG) big_list[atomicAdd(&scal[SCAL_NBIG], 1u)] = g;
            if (cfg.asmd) {
                int kx, ky, kz;
                unpack_key(slots[h].key, kx, ky, kz);
                if (centre_dist2(kx, ky, kz, v, cfg.sx, cfg.sy, cfg.sz) <= cfg.rc2) {
                    near_sum += size;
                    near_cnt += 1;
                }
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        near_sum += __shfl_xor_sync(0xffffffffu, near_sum, o);
        near_cnt += __shfl_xor_sync(0xffffffffu, near_cnt, o);
    }
    if (lane == 0 && near_cnt) {
        atomicAdd(&ctr->near_sum, near_sum);
        atomicAdd(&ctr->near_cnt, near_cnt);
    }
    // groups above GS_BLOCK_MIN, each sorted by a whole block, claimed after the block's warp
    // work; the same bookkeeping as a lane's
    const u32 nhuge = scal[SCAL_NHUGE];
    if (nhuge) {
        __shared__ u32 s_claim, s_rows[256], s_red[2 * GS_WARPS];
        for (;;) {
            __syncthreads();   // sbuf, s_claim and s_red are free
            if (threadIdx.x == 0) s_claim = atomicAdd(&scal[SCAL_HUGENEXT], 1u);
            __syncthreads();
            const u32 b = s_claim;
            if (b >= nhuge) break;
            const u32 g = huge_list[b];
            const u32 base = gstart[g], size = gsize[g], h = gslot[g];
            sort_group_block(members + base, size, tmp + base, &sbuf[0][0], s_rows, s_red);
            if (threadIdx.x == 0) {
                flags[members[base]] = 1u;
                slot_cnt[h] = 0u;
                if (size > ADMIT_BIG) big_list[atomicAdd(&scal[SCAL_NBIG], 1u)] = g;
                if (cfg.asmd) {
                    int kx, ky, kz;
                    unpack_key(slots[h].key, kx, ky, kz);
                    if (centre_dist2(kx, ky, kz, v, cfg.sx, cfg.sy, cfg.sz) <= cfg.rc2) {
                        atomicAdd(&ctr->near_sum, (unsigned long long)size);
                        atomicAdd(&ctr->near_cnt, 1ull);
                    }
                }
            }
        }
    }
}

// N_ASMD(r) = clamp(round(N_near + (k - N_near) min(r / r_max, 1)), k, N_max), FP64.
__device__ __forceinline__ u32 asmd_cap(int kx, int ky, int kz, double v, const InsertCfg& cfg, double n_near,
                                        u32 k, u32 nmax) {
    const double r = __dsqrt_rn(centre_dist2(kx, ky, kz, v, cfg.sx, cfg.sy, cfg.sz));
    double f = __ddiv_rn(r, cfg.r_max);
    if (f > 1.0) f = 1.0;
    const double val = __dadd_rn(n_near, __dmul_rn(__dsub_rn((double)k, n_near), f));
    const double c = floor(__dadd_rn(val, 0.5));
    if (c > (double)nmax) return nmax;
    if (c < (double)k) return k;
    return (u32)c;
}

struct AdmitArgs {
    const u32* gslot;     // slot of each group
    const u32* sv;        // group members (input indices), each group sorted ascending
    const u32* gstart;
    const u32* gsize;
    const u32* scal;
    const float4* world;
    Slot* slots;
    float4* pts;
    const u32* ring;
    u32 max_buckets;
    MapCounters* ctr;
    u32 nmax, k;
    float dmin2;
    double v;
    InsertCfg cfg;
    const double* dev_T;
    u32* admitted;
    const u32* head_ord;
    u32* grp_cnt;
    u32* a_ord;
    u32* a_j;
    u32* pos;
    // precision variant: per-voxel FP16 exponents and the state of each touched voxel
    int* cexp;          // null for plain maps
    u32* grp_bucket;
    u32* grp_cnt0;
    int* grp_exp0;
    const u32* big_list;  // groups above ADMIT_BIG members (SCAL_NBIG of them)
    u32* big_next;        // the claim counter over big_list
    // the map was emptied just before this insert (the scan-local map): its bucket ring is the
    // identity with head 0, every group opens a new voxel, and the group of ordinal o takes
    // bucket o with no atomic on the ring head (every warp's atomic on that one address
    // serialised the header phase)
    int fresh;
};

// a11 admission. A warp takes 32 voxel groups at a time (strided over the group range): each
// lane reads the header of one group (members, slot, bucket, fill, ASMD cap) and opens a bucket for a new voxel. The warp
// then walks the groups that can still take points. Candidates are walked in input order; a
// candidate enters while the voxel holds fewer than its cap and no point of the voxel is
// closer than d_min (FP32 d^2 >= d_min^2). The voxel's points sit in the warp's shared buffer;
// each lane holds one candidate of a window of 32 (in input order) and tests it against them
// (broadcast reads), then the passing candidates are admitted in input order.
// Candidate windows of 32 a warp tests at once in the admission (see k_admit).
#ifndef FAR_ADMIT_U
#define FAR_ADMIT_U 2
#endif
constexpr int ADMIT_U = FAR_ADMIT_U;

// Admission of one large group by the whole block, the same decisions as the warp's walk in
// k_admit: a candidate enters while the voxel holds fewer than its cap and every point in it is
// at least d_min away, in input order. The candidates go in tiles of TPB * BIG_PER_THREAD
// (candidate tile + r TPB + t on thread t). Each is tested once against the voxel's points so
// far; then, round after round, the first candidate of the tile that still passes (a block
// minimum of r TPB + t) is admitted, the ones before it are settled, and the later ones are
// re-tested against it only. Thread 0 does the header steps of a lane of the warp path.
constexpr int BIG_PER_THREAD = 4;

__device__ __forceinline__ void admit_big_group(const AdmitArgs& a, u32 g, double n_near, u32 ring_tail,
                                                float4* s_pts, u32* s_red, u32* s_hdr) {
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    if (t == 0) {
        const u32 start = a.gstart[g], size = a.gsize[g], slot = a.gslot[g];
        const u32 ord = a.head_ord[a.sv[start]];
        Slot* sp = a.slots + slot;
        u32 bucket = sp->bucket;
        const u32 cnt = (bucket == NO_BUCKET) ? 0u : sp->count;
        u32 cap = 0;
        if (bucket == NO_BUCKET) {
            const u32 h = a.fresh ? ord : atomicAdd(&a.ctr->ring_head, 1u);
            if (h < ring_tail) {
                bucket = a.ring[h % a.max_buckets];
                sp->bucket = bucket;
                sp->count = 0;
                if (a.cexp) a.cexp[bucket] = EXP_NONE;
                if (!a.fresh) atomicAdd(&a.ctr->n_voxels, 1u);
            } else {
                atomicOr(&a.ctr->err, (u32)ERR_BUCKETS_FULL);
                atomicAdd(&a.ctr->n_dropped, size);
            }
        }
        if (bucket != NO_BUCKET) {
            cap = a.nmax;
            if (a.cfg.asmd) {
                int kx, ky, kz;
                unpack_key(sp->key, kx, ky, kz);
                cap = asmd_cap(kx, ky, kz, a.v, a.cfg, n_near, a.k, a.nmax);
            }
            if (a.cexp) {
                a.grp_bucket[ord] = bucket;
                a.grp_cnt0[ord] = cnt;
                a.grp_exp0[ord] = a.cexp[bucket];
            }
        }
        if (cnt >= cap) a.grp_cnt[ord] = 0;
        s_hdr[0] = start;
        s_hdr[1] = start + size;
        s_hdr[2] = slot;
        s_hdr[3] = ord;
        s_hdr[4] = bucket;
        s_hdr[5] = cnt;
        s_hdr[6] = cap;
    }
    __syncthreads();
    const u32 start = s_hdr[0], end = s_hdr[1], slot = s_hdr[2], ord = s_hdr[3], bucket = s_hdr[4];
    const u32 cnt0 = s_hdr[5], cap = s_hdr[6];
    if (cnt0 >= cap) {
        __syncthreads();   // s_hdr is read by every thread before the next group's header
        return;
    }
    float4* bp = a.pts + (size_t)bucket * a.nmax;
    for (u32 i = t; i < cnt0; i += TPB) s_pts[i] = bp[i];
    __syncthreads();
    u32 c_n = cnt0;
    constexpr u32 TILE = TPB * BIG_PER_THREAD;
    for (u32 tile = start; tile < end && c_n < cap; tile += TILE) {
        float cx[BIG_PER_THREAD], cy[BIG_PER_THREAD], cz[BIG_PER_THREAD];
        u32 pass = 0;
#pragma unroll
        for (int r = 0; r < BIG_PER_THREAD; ++r) {
            const u32 i = tile + (u32)r * TPB + (u32)t;
            cx[r] = cy[r] = cz[r] = 0.f;
            if (i < end) {
                const float4 p = a.world[a.sv[i]];
                cx[r] = p.x;
                cy[r] = p.y;
                cz[r] = p.z;
                pass |= 1u << r;
            }
        }
        for (u32 j = 0; j < c_n && pass; ++j) {
            const float4 e = s_pts[j];
#pragma unroll
            for (int r = 0; r < BIG_PER_THREAD; ++r)
                if (((pass >> r) & 1u) && !(dist2_rn(cx[r], cy[r], cz[r], e.x, e.y, e.z) >= a.dmin2))
                    pass &= ~(1u << r);
        }
        while (c_n < cap) {
            // the tile's first passing candidate, as its tile order r TPB + t
            u32 key = pass ? (u32)(__ffs(pass) - 1) * TPB + (u32)t : 0xFFFFFFFFu;
            key = __reduce_min_sync(0xffffffffu, key);
            if (lane == 0) s_red[warp] = key;
            __syncthreads();
            u32 best = s_red[0];
#pragma unroll
            for (int w = 1; w < TPB / 32; ++w) best = min(best, s_red[w]);
            if (best == 0xFFFFFFFFu) break;
            if ((u32)t == best % TPB) {
                const u32 rb = best / TPB, i = tile + best, idx = a.sv[i];
                float x = 0.f, y = 0.f, z = 0.f;
#pragma unroll
                for (int r = 0; r < BIG_PER_THREAD; ++r)
                    if ((u32)r == rb) {
                        x = cx[r];
                        y = cy[r];
                        z = cz[r];
                    }
                const float4 c = make_float4(x, y, z, __uint_as_float(NO_ID));
                bp[c_n] = c;
                s_pts[c_n] = c;
                a.pos[idx] = bucket * a.nmax + c_n;
                a.admitted[idx] = 1u;
                a.a_ord[idx] = ord;
                a.a_j[idx] = c_n - cnt0;
            }
            __syncthreads();   // the admitted point is in s_pts; every thread has read s_red
            const float4 e = s_pts[c_n];
            ++c_n;
#pragma unroll
            for (int r = 0; r < BIG_PER_THREAD; ++r) {
                if (!((pass >> r) & 1u)) continue;
                if ((u32)r * TPB + (u32)t <= best || !(dist2_rn(cx[r], cy[r], cz[r], e.x, e.y, e.z) >= a.dmin2))
                    pass &= ~(1u << r);
            }
        }
        __syncthreads();   // the last round's reads of s_red come before the next tile's writes
    }
    if (t == 0) {
        if (c_n != cnt0) a.slots[slot].count = c_n;
        a.grp_cnt[ord] = c_n - cnt0;
    }
    __syncthreads();   // s_pts and s_hdr are free for the next group
}

__global__ void __launch_bounds__(TPB) k_admit(AdmitArgs a) {
    pdl_wait();
    pdl_trigger();
    if (a.dev_T) {
        a.cfg.sx = a.dev_T[3];
        a.cfg.sy = a.dev_T[7];
        a.cfg.sz = a.dev_T[11];
    }
    const int lane = threadIdx.x & 31;
    const u32 warps_total = (gridDim.x * blockDim.x) >> 5;
    const u32 ng = a.scal[SCAL_NGROUPS];
    // N_near once per block (FP64 divisions and square roots are slow on this GPU: each is
    // evaluated by one thread and shared)
    __shared__ double s_near;
    __shared__ float4 s_vox[TPB / 32][NMAX_LIMIT];   // per warp: the points of the voxel it admits into
    if (threadIdx.x == 0) {
        double nn = (double)a.nmax;
        if (a.cfg.asmd && a.ctr->near_cnt > 0) nn = __ddiv_rn((double)a.ctr->near_sum, (double)a.ctr->near_cnt);
        s_near = nn;
    }
    __syncthreads();
    const double n_near = s_near;
    const u32 ring_tail = a.ctr->ring_tail;
    if (a.fresh && blockIdx.x == 0 && threadIdx.x == 0) {
        // every group of a fresh map opens a voxel (those beyond the pool are dropped in their headers)
        const u32 opened = min(ng, ring_tail);
        a.ctr->ring_head = opened;
        a.ctr->n_voxels = opened;
    }
    const float4 far4 = make_float4(F_INF, F_INF, F_INF, 0.f);
    const u32 w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    for (u32 j0 = 0; w + j0 * warps_total < ng; j0 += 32) {
        // --- lane-parallel headers (large groups are left to whole blocks, below)
        const u32 g = w + (j0 + lane) * warps_total;
        const bool gv = g < ng && a.gsize[g] <= ADMIT_BIG;
        u32 start = 0, end = 0, slot = 0, ord = 0, bucket = NO_BUCKET, cnt = 0, cap = 0;
        Slot* sp = nullptr;
        if (gv) {
            start = a.gstart[g];
            end = start + a.gsize[g];
            slot = a.gslot[g];
            ord = a.head_ord[a.sv[start]];
            sp = a.slots + slot;
            bucket = sp->bucket;
            cnt = (bucket == NO_BUCKET) ? 0u : sp->count;
        }
        // new voxels take buckets from the ring: by ordinal on a fresh map, else one atomic per warp
        const bool need = gv && bucket == NO_BUCKET;
        const u32 need_mask = __ballot_sync(0xffffffffu, need);
        if (a.fresh) {
            if (need) {
                if (ord < ring_tail) {
                    bucket = a.ring[ord];
                    sp->bucket = bucket;
                    sp->count = 0;
                    if (a.cexp) a.cexp[bucket] = EXP_NONE;
                } else {
                    atomicOr(&a.ctr->err, (u32)ERR_BUCKETS_FULL);
                    atomicAdd(&a.ctr->n_dropped, end - start);
                }
            }
        } else if (need_mask) {
            u32 h0 = 0;
            if (lane == __ffs(need_mask) - 1) h0 = atomicAdd(&a.ctr->ring_head, (u32)__popc(need_mask));
            h0 = __shfl_sync(0xffffffffu, h0, __ffs(need_mask) - 1);
            const u32 h = h0 + __popc(need_mask & ((1u << lane) - 1u));
            bool got = false;
            if (need) {
                if (h < ring_tail) {
                    bucket = a.ring[h % a.max_buckets];
                    sp->bucket = bucket;
                    sp->count = 0;
                    if (a.cexp) a.cexp[bucket] = EXP_NONE;  // a recycled bucket starts without an exponent
                    got = true;
                } else {
                    atomicOr(&a.ctr->err, (u32)ERR_BUCKETS_FULL);
                    atomicAdd(&a.ctr->n_dropped, end - start);
                }
            }
            const u32 got_mask = __ballot_sync(0xffffffffu, got);
            if (lane == 0 && got_mask) atomicAdd(&a.ctr->n_voxels, (u32)__popc(got_mask));
        }
        if (gv) {
            if (bucket != NO_BUCKET) {
                cap = a.nmax;
                if (a.cfg.asmd) {
                    int kx, ky, kz;
                    unpack_key(sp->key, kx, ky, kz);
                    cap = asmd_cap(kx, ky, kz, a.v, a.cfg, n_near, a.k, a.nmax);
                }
                if (a.cexp) {
                    a.grp_bucket[ord] = bucket;
                    a.grp_cnt0[ord] = cnt;
                    a.grp_exp0[ord] = a.cexp[bucket];
                }
            }
            if (cnt >= cap) a.grp_cnt[ord] = 0;
        }
        // --- groups that can take points, one at a time by the whole warp
        u32 work = __ballot_sync(0xffffffffu, cnt < cap);
        while (work) {
            const int f = __ffs(work) - 1;
            work &= work - 1u;
            const u32 w_start = __shfl_sync(0xffffffffu, start, f);
            const u32 w_end = __shfl_sync(0xffffffffu, end, f);
            const u32 w_ord = __shfl_sync(0xffffffffu, ord, f);
            const u32 w_bucket = __shfl_sync(0xffffffffu, bucket, f);
            const u32 w_cap = __shfl_sync(0xffffffffu, cap, f);
            const u32 w_slot = __shfl_sync(0xffffffffu, slot, f);
            const u32 cnt0 = __shfl_sync(0xffffffffu, cnt, f);
            u32 c_n = cnt0;
            float4* bp = a.pts + (size_t)w_bucket * a.nmax;
            // the voxel's points in the warp's shared buffer (the previous group's readers are done)
            float4* vp = s_vox[threadIdx.x >> 5];
            __syncwarp();
            if (lane < (int)c_n) vp[lane] = bp[lane];
            if (lane + 32 < (int)c_n) vp[lane + 32] = bp[lane + 32];
            __syncwarp();
            for (u32 w0 = w_start; w0 < w_end && c_n < w_cap; w0 += 32u * ADMIT_U) {
                // ADMIT_U windows of 32 candidates at once, candidate w0 + 32 u + l on lane l: their
                // loads are in flight together, and each broadcast read of a voxel point is tested
                // against all of them
                u32 my_idx[ADMIT_U];
                float4 my_c[ADMIT_U];
                bool pass[ADMIT_U];
#pragma unroll
                for (int u = 0; u < ADMIT_U; ++u) {
                    const u32 i = w0 + 32u * u + lane;
                    pass[u] = i < w_end;
                    my_idx[u] = pass[u] ? a.sv[i] : 0u;
                }
#pragma unroll
                for (int u = 0; u < ADMIT_U; ++u) my_c[u] = pass[u] ? a.world[my_idx[u]] : far4;
                for (u32 j = 0; j < c_n; ++j) {
                    const float4 e = vp[j];   // the same address for every lane: one broadcast read
#pragma unroll
                    for (int u = 0; u < ADMIT_U; ++u)
                        pass[u] = pass[u] && (dist2_rn(my_c[u].x, my_c[u].y, my_c[u].z, e.x, e.y, e.z) >= a.dmin2);
                }
                // resolve in input order (window u before u + 1, lanes in order): the first passing
                // candidate is admitted, the later ones are re-tested against it only (the earlier
                // ones already failed against a subset)
#pragma unroll
                for (int u = 0; u < ADMIT_U; ++u) {
                    while (c_n < w_cap) {
                        const u32 ballot = __ballot_sync(0xffffffffu, pass[u]);
                        if (ballot == 0u) break;
                        const int fl = __ffs(ballot) - 1;
                        const float cx = __shfl_sync(0xffffffffu, my_c[u].x, fl);
                        const float cy = __shfl_sync(0xffffffffu, my_c[u].y, fl);
                        const float cz = __shfl_sync(0xffffffffu, my_c[u].z, fl);
                        const float4 c = make_float4(cx, cy, cz, __uint_as_float(NO_ID));
                        if (lane == fl) {
                            bp[c_n] = c;
                            vp[c_n] = c;
                            a.pos[my_idx[u]] = w_bucket * a.nmax + c_n;
                            a.admitted[my_idx[u]] = 1u;
                            a.a_ord[my_idx[u]] = w_ord;
                            a.a_j[my_idx[u]] = c_n - cnt0;
                        }
                        ++c_n;
                        if (lane <= fl) pass[u] = false;
                        else if (pass[u]) pass[u] = dist2_rn(my_c[u].x, my_c[u].y, my_c[u].z, cx, cy, cz) >= a.dmin2;
#pragma unroll
                        for (int v2 = u + 1; v2 < ADMIT_U; ++v2)
                            if (pass[v2])
                                pass[v2] = dist2_rn(my_c[v2].x, my_c[v2].y, my_c[v2].z, cx, cy, cz) >= a.dmin2;
                    }
                }
                __syncwarp();   // this window's admitted points are visible to the next window
            }
            if (lane == 0) {
                if (c_n != cnt0) a.slots[w_slot].count = c_n;
                a.grp_cnt[w_ord] = c_n - cnt0;
            }
        }
    }
    // large groups, each by a whole block, claimed after the block's small groups (blocks
    // without small groups start with them)
    const u32 nbig = a.scal[SCAL_NBIG];
    if (nbig) {
        __shared__ u32 s_claim, s_red[TPB / 32], s_hdr[8];
        __syncthreads();   // the warps' use of s_vox is over
        for (;;) {
            if (threadIdx.x == 0) s_claim = atomicAdd(a.big_next, 1u);
            __syncthreads();
            const u32 b = s_claim;
            __syncthreads();   // read by every thread before thread 0 claims again
            if (b >= nbig) break;
            admit_big_group(a, a.big_list[b], n_near, ring_tail, s_vox[0], s_red, s_hdr);
        }
    }
}

// Admitted points after the two scans: the id (first id + rank in input order), the position
// in the grouped order (the voxel's ordinal base + its index among the voxel's admitted
// points) and the list of added positions (and keys); thread 0 advances the map's counters
// (no thread of this launch reads them).
__global__ void k_place_admitted(const u32* __restrict__ admitted, const u32* __restrict__ rank,
                                 const u32* __restrict__ a_ord, const u32* __restrict__ a_j,
                                 const u32* __restrict__ grp_base, const u32* __restrict__ pos, u32 n,
                                 float4* pts, u32* __restrict__ dest, u32* __restrict__ added,
                                 const u64* __restrict__ keys, u64* __restrict__ added_key,
                                 const u32* __restrict__ scal, MapCounters* ctr, const float4* __restrict__ in4,
                                 float4* __restrict__ src, u32* __restrict__ src_index) {
    pdl_wait();
    pdl_trigger();
    const u32 i = blockIdx.x * blockDim.x + threadIdx.x;
    const u32 id0 = scal[SCAL_IDBASE], n_add = scal[SCAL_NADMIT];
    if (i == 0) {
        ctr->next_id = id0 + n_add;
        ctr->n_points += n_add;
        ctr->n_added = n_add;
        if ((unsigned long long)id0 + n_add > 0xFFFFFFFFull) atomicOr(&ctr->err, (u32)ERR_ID_OVERFLOW);
    }
    if (i >= n || !admitted[i]) return;
    const u32 p = pos[i];
    pts[p].w = __uint_as_float(id0 + rank[i]);
    const u32 d = grp_base[a_ord[i]] + a_j[i];
    dest[i] = d;
    if (added) added[d] = p;
    if (added_key) added_key[d] = keys[i];
    if (src) {
        // scan-local insert: the registration sources in the same grouped order (consecutive
        // threads of the registration kernels then share their 27-neighbourhoods), w = the
        // admission rank (the local id)
        const float4 v = in4[i];
        src[d] = make_float4(v.x, v.y, v.z, __uint_as_float(rank[i]));
        src_index[d] = i;
    }
}

// Lanes cooperating on one k-NN query (group_knn); every grid-stride step is warp-uniform.
constexpr int KNN_TPP = 4;

// Eq. 1 covariances of query points against map m. Queries are either q[r]
// (q != null) or m.pts[qpos[r]]; output index is out_pos[r] (map points) or r.
// With knn_ids, the output row of a query is its rank, taken from q[r].w.
template <int K>
__global__ void __launch_bounds__(TPB, K <= 6 ? 3 : 2) k_knn_cov(MapView m, const float4* __restrict__ q,
                                                 const u32* __restrict__ qpos, u32 n, const u32* __restrict__ n_dev,
                                                 float4* __restrict__ cov_out, const u32* __restrict__ out_pos,
                                                 u32* __restrict__ knn_ids) {
    pdl_wait();
    pdl_trigger();
    const u32 nn = n_dev ? min(n, *n_dev) : n;
    const u32 max_probe = m.ctr->max_probe;
    const u32 t = blockIdx.x * blockDim.x + threadIdx.x;
    const int sl = threadIdx.x % KNN_TPP;
    __shared__ unsigned char vlist[TPB / KNN_TPP][28];   // surviving neighbour voxels per query
    const u32 stride = gridDim.x * blockDim.x / KNN_TPP;
    const int zero[3] = {0, 0, 0};
    for (u32 base = (t & ~31u) / KNN_TPP; base < nn; base += stride) {   // warp-uniform trip count
        const u32 r = base + (threadIdx.x & 31u) / KNN_TPP;
        const bool active = r < nn;
        const float4 p = active ? (q ? q[r] : m.pts[qpos[r]]) : make_float4(0.f, 0.f, 0.f, 0.f);
        QFrame<false> f;
        const bool keyed = active && make_qframe<false>(m, p.x, p.y, p.z, zero, f);
        unsigned long long bk[K];
        u32 bpos[K];
        const int found =
            group_knn<K, KNN_TPP, false>(m, max_probe, f, keyed, sl, vlist[threadIdx.x / KNN_TPP], bk, bpos);
        if (!active || sl != 0) continue;
        float4 c0 = make_float4(0.f, 0.f, 0.f, 0.f), c1 = make_float4(0.f, 0.f, 0.f, 0.f);
        if (found >= K) covariance_from_neighbours<K>(m.pts, bpos, p.x, p.y, p.z, c0, c1);
        const u32 o = out_pos ? out_pos[r] : r;
        cov_out[2 * (size_t)o] = c0;
        cov_out[2 * (size_t)o + 1] = c1;
        if (knn_ids) {
            const size_t row = __float_as_uint(p.w);
#pragma unroll
            for (int j = 0; j < K; ++j) knn_ids[row * K + j] = (j < found) ? (u32)bk[j] : NO_ID;
        }
    }
}

// Precision variant, a12: Eq. 1 covariances of the added map points (grouped order r,
// map position qpos[r], voxel key qkey[r]) in the frame of each point's tile, kept in FP32
// in cov_tmp; each valid covariance raises its voxel's exponent.
template <int K>
__global__ void __launch_bounds__(TPB, K <= 6 ? 3 : 2) k_knn_cov_tile(MapView m, const u32* __restrict__ qpos,
                                                      const u64* __restrict__ qkey, u32 n,
                                                      const u32* __restrict__ n_dev, float4* __restrict__ cov_tmp,
                                                      int* __restrict__ cexp) {
    pdl_wait();
    pdl_trigger();
    const u32 nn = min(n, *n_dev);
    const u32 max_probe = m.ctr->max_probe;
    const u32 t = blockIdx.x * blockDim.x + threadIdx.x;
    const int sl = threadIdx.x % KNN_TPP;
    __shared__ unsigned char vlist[TPB / KNN_TPP][28];   // surviving neighbour voxels per query
    const u32 stride = gridDim.x * blockDim.x / KNN_TPP;
    for (u32 base = (t & ~31u) / KNN_TPP; base < nn; base += stride) {   // warp-uniform trip count
        const u32 r = base + (threadIdx.x & 31u) / KNN_TPP;
        const bool active = r < nn;
        const u32 pos = active ? qpos[r] : 0u;
        const float4 p = active ? m.pts[pos] : make_float4(0.f, 0.f, 0.f, 0.f);
        int kx = 0, ky = 0, kz = 0;
        if (active) unpack_key(qkey[r], kx, ky, kz);
        QFrame<true> f;
        own_qframe(m, p.x, p.y, p.z, kx, ky, kz, f);
        unsigned long long bk[K];
        u32 bpos[K];
        const int found =
            group_knn<K, KNN_TPP, true>(m, max_probe, f, active, sl, vlist[threadIdx.x / KNN_TPP], bk, bpos);
        if (!active || sl != 0) continue;
        float c[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        bool valid = false;
        if (found >= K) {
            valid = true;
            covariance_from_neighbours_f<K>(m.pts, bpos, p.x, p.y, p.z, TileOffset(), c);
        }
        cov_tmp[2 * (size_t)r] = make_float4(c[0], c[1], c[2], c[3]);
        cov_tmp[2 * (size_t)r + 1] = make_float4(c[4], c[5], valid ? 1.0f : 0.0f, 0.0f);
        if (valid) atomicMax(cexp + pos / m.nmax, cov_exponent(c));
    }
}

// Precision variant: one warp per touched voxel (ordinal g). If the voxel's exponent rose,
// the FP16 entries of its older points are rescaled by the power of two (exact unless they
// become subnormal); then the added points of the voxel (grouped positions base[g] ..) are
// written as FP16 at the final exponent. The result does not depend on thread timing.
__global__ void k_cov_encode(const u32* __restrict__ grp_base, const u32* __restrict__ scal,
                             const u32* __restrict__ grp_bucket, const u32* __restrict__ grp_cnt0,
                             const int* __restrict__ grp_exp0, const int* __restrict__ cexp,
                             const u32* __restrict__ added, const float4* __restrict__ cov_tmp, u32 nmax,
                             uint2* __restrict__ cov_h4, u32* __restrict__ cov_h2) {
    pdl_wait();
    pdl_trigger();
    const int lane = threadIdx.x & 31;
    const u32 ng = scal[SCAL_NGROUPS];
    const u32 n_add = scal[SCAL_NADMIT];
    for (u32 g = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; g < ng; g += (gridDim.x * blockDim.x) >> 5) {
        const u32 b0 = grp_base[g];
        const u32 b1 = (g + 1 < ng) ? grp_base[g + 1] : n_add;
        if (b1 == b0) continue;
        const u32 bucket = grp_bucket[g];
        const int E = cexp[bucket], E0 = grp_exp0[g];
        if (E0 != EXP_NONE && E > E0) {
            const float s = pow2f(E0 - E);
            for (u32 j = lane; j < grp_cnt0[g]; j += 32) {
                const size_t o = (size_t)bucket * nmax + j;
                float c[6];
                if (!cov16_decode(cov_h4[o], cov_h2[o], 0, c)) continue;
#pragma unroll
                for (int t = 0; t < 6; ++t) c[t] *= s;
                cov16_encode(c, 0, cov_h4[o], cov_h2[o]);
            }
        }
        for (u32 r = b0 + lane; r < b1; r += 32) {
            const float4 c0 = cov_tmp[2 * (size_t)r], c1 = cov_tmp[2 * (size_t)r + 1];
            const u32 o = added[r];
            if (c1.z > 0.5f) {
                const float c[6] = {c0.x, c0.y, c0.z, c0.w, c1.x, c1.y};
                cov16_encode(c, E, cov_h4[o], cov_h2[o]);
            } else {
                cov_h4[o] = make_uint2(0u, 0u);
                cov_h2[o] = 0u;
            }
        }
    }
}

// Precision variant sources: the FP32 covariances of each scan-local voxel (grouped
// positions base[g] ..) are stored as FP16 with the voxel's exponent, kept per point.
__global__ void k_src_encode(const u32* __restrict__ grp_base, const u32* __restrict__ scal,
                             const float4* __restrict__ src_cov, uint2* __restrict__ h4, u32* __restrict__ h2,
                             signed char* __restrict__ e_out) {
    pdl_wait();
    pdl_trigger();
    const int lane = threadIdx.x & 31;
    const u32 ng = scal[SCAL_NGROUPS];
    const u32 n_add = scal[SCAL_NADMIT];
    for (u32 g = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; g < ng; g += (gridDim.x * blockDim.x) >> 5) {
        const u32 b0 = grp_base[g];
        const u32 b1 = (g + 1 < ng) ? grp_base[g + 1] : n_add;
        if (b1 == b0) continue;
        int E = EXP_NONE;
        for (u32 r = b0 + lane; r < b1; r += 32) {
            const float4 c0 = src_cov[2 * (size_t)r], c1 = src_cov[2 * (size_t)r + 1];
            if (c1.z > 0.5f) {
                const float c[6] = {c0.x, c0.y, c0.z, c0.w, c1.x, c1.y};
                E = max(E, cov_exponent(c));
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) E = max(E, __shfl_xor_sync(0xffffffffu, E, o));
        for (u32 r = b0 + lane; r < b1; r += 32) {
            const float4 c0 = src_cov[2 * (size_t)r], c1 = src_cov[2 * (size_t)r + 1];
            if (c1.z > 0.5f) {
                const float c[6] = {c0.x, c0.y, c0.z, c0.w, c1.x, c1.y};
                cov16_encode(c, E, h4[r], h2[r]);
            } else {
                h4[r] = make_uint2(0u, 0u);
                h2[r] = 0u;
            }
            e_out[r] = (signed char)(E == EXP_NONE ? 0 : E);
        }
    }
}

__global__ void k_iota(u32* a, u32 n) {
    pdl_wait();
    pdl_trigger();
    for (u32 i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) a[i] = i;
}

// Slots per thread of the eviction scan: all of a thread's slot loads are issued before any is
// tested (the table is mostly empty slots, so the scan is bound by the loads' latency).
constexpr u32 EVICT_PER_THREAD = 4;

__global__ void k_evict(Slot* slots, u32 cap, double v, double cx, double cy, double cz, double r2, u32* ring,
                        u32 max_buckets, MapCounters* ctr, const double* __restrict__ dev_T) {
    pdl_wait();
    pdl_trigger();
    // thread t takes slots t, t + T, t + 2 T, t + 3 T (T = threads in the grid): the whole slot
    // (key, bucket, count) in one 16 B load each
    const u32 nthreads = gridDim.x * blockDim.x;
    const u32 t = blockIdx.x * blockDim.x + threadIdx.x;
    uint4 raw[EVICT_PER_THREAD];
#pragma unroll
    for (u32 k = 0; k < EVICT_PER_THREAD; ++k) {
        const u32 h = t + k * nthreads;
        raw[k] = h < cap ? *reinterpret_cast<const uint4*>(slots + h) : make_uint4(0xFFFFFFFFu, 0xFFFFFFFFu, 0u, 0u);
    }
    if (dev_T) {
        cx = dev_T[3];
        cy = dev_T[7];
        cz = dev_T[11];
    }
    const float fv = (float)v, fcx = (float)cx, fcy = (float)cy, fcz = (float)cz, fr2 = (float)r2;
    // Each FP32 centre difference is off by at most a few ulps of the largest coordinate M,
    // so e2 is within about 8 * 2^-23 * M / r of d^2 in relative terms near the radius r;
    // the band below is twice that (plus 2e-5), and everything inside it takes the FP64
    // test. The band is FP32 arithmetic: FP64 square roots and divisions in every thread
    // would cost more than the whole table scan on this GPU.
    const float fr = sqrtf(fr2);
    const float Mf = fabsf(fcx) + fabsf(fcy) + fabsf(fcz) + fr + fv;
    const float band = 2e-5f + 2e-6f * Mf / fmaxf(fr, 1e-3f);
    const float lo2 = fr2 * (1.0f - band), hi2 = fr2 * (1.0f + band);
#pragma unroll
    for (u32 k = 0; k < EVICT_PER_THREAD; ++k) {
        const u64 key = ((u64)raw[k].y << 32) | raw[k].x;
        if (key >> 63) continue;  // empty, tombstone or beyond the table
        const u32 h = t + k * nthreads;
        int kx, ky, kz;
        unpack_key(key, kx, ky, kz);
        // FP32 estimate first; only distances near the radius take the exact FP64 test
        const float ex = ((float)kx + 0.5f) * fv - fcx, ey = ((float)ky + 0.5f) * fv - fcy,
                    ez = ((float)kz + 0.5f) * fv - fcz;
        const float e2 = ex * ex + ey * ey + ez * ez;
        bool far_away;
        if (e2 < lo2) far_away = false;
        else if (e2 > hi2) far_away = true;
        else far_away = centre_dist2(kx, ky, kz, v, cx, cy, cz) > r2;
        if (!far_away) continue;
        const u32 b = raw[k].z;
        const u32 c = raw[k].w;
        slots[h].key = KEY_TOMB;
        slots[h].bucket = NO_BUCKET;
        slots[h].count = 0;
        atomicAdd(&ctr->n_tomb, 1u);
        if (b != NO_BUCKET) {
            const u32 tt = atomicAdd(&ctr->ring_tail, 1u);
            ring[tt % max_buckets] = b;
            atomicSub(&ctr->n_voxels, 1u);
            atomicAdd(&ctr->removed, (unsigned long long)c);
            atomicAdd(&ctr->n_points, (unsigned long long)(0ull - (unsigned long long)c));
        }
    }
}

__global__ void k_rebuild(const Slot* __restrict__ old_slots, u32 old_cap, Slot* new_slots, u32 mask,
                          MapCounters* ctr) {
    pdl_wait();
    pdl_trigger();
    for (u32 h = blockIdx.x * blockDim.x + threadIdx.x; h < old_cap; h += gridDim.x * blockDim.x) {
        const Slot s = old_slots[h];
        if (s.key >> 63) continue;
        int kx, ky, kz;
        unpack_key(s.key, kx, ky, kz);
        u32 j = hash_key(kx, ky, kz) & mask;
        for (u32 p = 0; p <= mask; ++p) {
            if (atomicCAS(&new_slots[j].key, KEY_EMPTY, s.key) == KEY_EMPTY) {
                new_slots[j].bucket = s.bucket;
                new_slots[j].count = s.count;
                atomicMax(&ctr->max_probe, p);
                break;
            }
            j = (j + 1u) & mask;
        }
    }
}

__global__ void k_list_slots(const Slot* __restrict__ slots, u32 cap, u64* keys, u32* buckets, u32* counts,
                             u32* n_out, u32 cap_out) {
    pdl_wait();
    pdl_trigger();
    for (u32 h = blockIdx.x * blockDim.x + threadIdx.x; h < cap; h += gridDim.x * blockDim.x) {
        const Slot s = slots[h];
        if ((s.key >> 63) || s.bucket == NO_BUCKET || s.count == 0) continue;
        const u32 o = atomicAdd(n_out, 1u);
        if (o >= cap_out) continue;  // counted, not written: the caller sees n_out > cap_out
        keys[o] = s.key;
        buckets[o] = s.bucket;
        counts[o] = s.count;
    }
}

__global__ void k_gather(MapView m, const u32* __restrict__ buckets, const u32* __restrict__ counts,
                         const u32* __restrict__ offsets, const u64* __restrict__ keys, u32 nvox,
                         float4* __restrict__ pts_out, float4* __restrict__ cov_out) {
    pdl_wait();
    pdl_trigger();
    const int lane = threadIdx.x & 31;
    const u32 nmax = m.nmax;
    for (u32 g = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; g < nvox; g += (gridDim.x * blockDim.x) >> 5) {
        const u32 b = buckets[g], c = counts[g], o = offsets[g];
        int tile[3] = {0, 0, 0};
        if (m.tv > 0) {
            int k[3];
            unpack_key(keys[g], k[0], k[1], k[2]);
#pragma unroll
            for (int a = 0; a < 3; ++a) tile[a] = floor_div(k[a], m.tv);
        }
        for (u32 j = lane; j < c; j += 32) {
            const size_t src = (size_t)b * nmax + j;
            float4 p = m.pts[src];
            if (m.tv > 0) {
                // world FP32 = fp32(50 T + tile-relative value), exact in FP64 before the rounding
                p.x = __double2float_rn(__dadd_rn(TILE_D * (double)tile[0], (double)p.x));
                p.y = __double2float_rn(__dadd_rn(TILE_D * (double)tile[1], (double)p.y));
                p.z = __double2float_rn(__dadd_rn(TILE_D * (double)tile[2], (double)p.z));
            }
            pts_out[o + j] = p;
            if (!cov_out) continue;
            if (m.tv > 0) {
                float cv[6];
                const bool ok = cov16_decode(m.cov_h4[src], m.cov_h2[src], m.cexp[b], cv);
                cov_out[2 * (size_t)(o + j)] = ok ? make_float4(cv[0], cv[1], cv[2], cv[3]) : make_float4(0, 0, 0, 0);
                cov_out[2 * (size_t)(o + j) + 1] = ok ? make_float4(cv[4], cv[5], 1.0f, 0.0f) : make_float4(0, 0, 0, 0);
            } else {
                cov_out[2 * (size_t)(o + j)] = m.cov[2 * src];
                cov_out[2 * (size_t)(o + j) + 1] = m.cov[2 * src + 1];
            }
        }
    }
}

// Precision variant: frame of a world query = its own tile, T = floor(q / 50), q_F = fp32(q - 50 T).
__device__ __forceinline__ bool world_query_frame(const MapView& m, float qx, float qy, float qz, QFrame<true>& f) {
    const float q[3] = {qx, qy, qz};
    int ft[3];
    float qf[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const double x = (double)q[a];
        if (!isfinite(x)) return false;
        const double T = tile_floor(x);
        if (!(fabs(T) * (double)m.tv < (double)KEY_BIAS)) return false;
        ft[a] = (int)T;
        qf[a] = __double2float_rn(__dsub_rn(x, __dmul_rn(TILE_D, T)));
    }
    return make_qframe<true>(m, qf[0], qf[1], qf[2], ft, f);
}

template <int K>
__global__ void __launch_bounds__(TPB) k_knn_stage(MapView m, const float4* __restrict__ q, u32 n,
                                                   u32* __restrict__ ids, int32_t* __restrict__ found_out) {
    pdl_wait();
    pdl_trigger();
    const u32 max_probe = m.ctr->max_probe;
    const u32 t = blockIdx.x * blockDim.x + threadIdx.x;
    const int sl = threadIdx.x % KNN_TPP;
    __shared__ unsigned char vlist[TPB / KNN_TPP][28];   // surviving neighbour voxels per query
    const u32 stride = gridDim.x * blockDim.x / KNN_TPP;
    const int zero[3] = {0, 0, 0};
    for (u32 base = (t & ~31u) / KNN_TPP; base < n; base += stride) {   // warp-uniform trip count
        const u32 r = base + (threadIdx.x & 31u) / KNN_TPP;
        const bool active = r < n;
        const float4 p = active ? q[r] : make_float4(0.f, 0.f, 0.f, 0.f);
        unsigned long long bk[K];
        u32 bpos[K];
        int found;
        if (m.tv > 0) {
            QFrame<true> f;
            const bool keyed = active && world_query_frame(m, p.x, p.y, p.z, f);
            found = group_knn<K, KNN_TPP, true>(m, max_probe, f, keyed, sl, vlist[threadIdx.x / KNN_TPP], bk,
                                                bpos);
        } else {
            QFrame<false> f;
            const bool keyed = active && make_qframe<false>(m, p.x, p.y, p.z, zero, f);
            found = group_knn<K, KNN_TPP, false>(m, max_probe, f, keyed, sl, vlist[threadIdx.x / KNN_TPP], bk,
                                                 bpos);
        }
        if (!active || sl != 0) continue;
        found_out[r] = found;
#pragma unroll
        for (int j = 0; j < K; ++j) ids[(size_t)r * K + j] = (j < found) ? (u32)bk[j] : NO_ID;
    }
}

__global__ void __launch_bounds__(TPB) k_nearest_stage(MapView m, const float4* __restrict__ q, u32 n, float tau2,
                                                       int64_t* __restrict__ ids, float* __restrict__ d2_out) {
    pdl_wait();
    pdl_trigger();
    const u32 max_probe = m.ctr->max_probe;
    for (u32 r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
        const float4 p = q[r];
        float bd2 = F_INF;
        u32 bid = NO_ID, bpos = 0;
        bool any = false;
        if (m.tv > 0) {
            QFrame<true> f;
            int bv;
            if (world_query_frame(m, p.x, p.y, p.z, f)) any = nearest27q<true>(m, max_probe, f, F_INF, bd2, bid, bpos, bv);
        } else {
            any = nearest27(m, max_probe, p.x, p.y, p.z, F_INF, bd2, bid, bpos);
        }
        d2_out[r] = bd2;
        ids[r] = (any && !(bd2 > tau2)) ? (int64_t)bid : (int64_t)-1;
    }
}

// Grid of the k-NN kernels: KNN_TPP lanes per query, at most 16 blocks per SM (grid-stride).
inline u32 knn_blocks(u32 n) { return min(blocks_for(n * KNN_TPP), 152u * 16u); }

template <int K>
cudaError_t launch_knn_cov(const DeviceMap& m, const float4* q, const u32* qpos, u32 n, const u32* n_dev,
                           float4* cov_out, const u32* out_pos, u32* knn_ids, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    FAR_LAUNCH(k_knn_cov<K>, knn_blocks(n), TPB, 0, st, m.view(), q, qpos, n, n_dev, cov_out, out_pos, knn_ids);
    return cudaGetLastError();
}

template <int K>
cudaError_t launch_knn_stage(const DeviceMap& m, const float4* q, u32 n, u32* ids, int32_t* found, cudaStream_t st) {
    FAR_LAUNCH(k_knn_stage<K>, knn_blocks(n), TPB, 0, st, m.view(), q, n, ids, found);
    return cudaGetLastError();
}

// One instantiation per exact k (1..16).
#define FAR_K_CASES(F, ...)                    \
    switch (k) {                               \
        case 1: return F<1>(__VA_ARGS__);      \
        case 2: return F<2>(__VA_ARGS__);      \
        case 3: return F<3>(__VA_ARGS__);      \
        case 4: return F<4>(__VA_ARGS__);      \
        case 5: return F<5>(__VA_ARGS__);      \
        case 6: return F<6>(__VA_ARGS__);      \
        case 7: return F<7>(__VA_ARGS__);      \
        case 8: return F<8>(__VA_ARGS__);      \
        case 9: return F<9>(__VA_ARGS__);      \
        case 10: return F<10>(__VA_ARGS__);    \
        case 11: return F<11>(__VA_ARGS__);    \
        case 12: return F<12>(__VA_ARGS__);    \
        case 13: return F<13>(__VA_ARGS__);    \
        case 14: return F<14>(__VA_ARGS__);    \
        case 15: return F<15>(__VA_ARGS__);    \
        case 16: return F<16>(__VA_ARGS__);    \
        default: return cudaErrorInvalidValue; \
    }

cudaError_t knn_cov(const DeviceMap& m, const float4* q, const u32* qpos, u32 n, const u32* n_dev,
                    float4* cov_out, const u32* out_pos, u32* knn_ids, cudaStream_t st) {
    const u32 k = m.k;
    FAR_K_CASES(launch_knn_cov, m, q, qpos, n, n_dev, cov_out, out_pos, knn_ids, st)
}

template <int K>
cudaError_t launch_knn_cov_tile(const DeviceMap& m, const u32* qpos, const u64* qkey, u32 n, const u32* n_dev,
                                float4* cov_tmp, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    FAR_LAUNCH(k_knn_cov_tile<K>, knn_blocks(n), TPB, 0, st, m.view(), qpos, qkey, n, n_dev, cov_tmp, m.cexp);
    return cudaGetLastError();
}

cudaError_t knn_cov_tile(const DeviceMap& m, const u32* qpos, const u64* qkey, u32 n, const u32* n_dev,
                         float4* cov_tmp, cudaStream_t st) {
    const u32 k = m.k;
    FAR_K_CASES(launch_knn_cov_tile, m, qpos, qkey, n, n_dev, cov_tmp, st)
}

}  // namespace

#define FAR_TRY(x)                                  \
    do {                                            \
        cudaError_t e__ = (x);                      \
        if (e__ != cudaSuccess) return e__;         \
    } while (0)

cudaError_t pack_points_deskew(const void* src, u32 n, u32 stride, const SweepMotion& mo, float4* out,
                               cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    FAR_LAUNCH(k_pack_deskew, blocks_for(n), TPB, 0, st, static_cast<const char*>(src), n, stride, mo, out,
               (float*)nullptr);
    return cudaGetLastError();
}

cudaError_t deskew_points(const void* src, u32 n, u32 stride, const SweepMotion& mo, float* out, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    FAR_LAUNCH(k_pack_deskew, blocks_for(n), TPB, 0, st, static_cast<const char*>(src), n, stride, mo,
               (float4*)nullptr, out);
    return cudaGetLastError();
}

cudaError_t pack_points(const void* src, u32 n, u32 stride, float4* out, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    FAR_LAUNCH(k_pack, blocks_for(n), TPB, 0, st, static_cast<const char*>(src), n, stride, out);
    return cudaGetLastError();
}

cudaError_t map_insert_batch(DeviceMap& m, Scratch& s, u32 n, const Pose12* pose, const InsertCfg& cfg,
                             bool covariances, cudaStream_t st, DevicePose dpose, const InsertMarks* marks,
                             bool emit_sources) {
    auto mark = [&](int i) {
        if (marks) cudaEventRecord(marks->ev[i], st);
    };
    if (n == 0) {
        // zero the per-insert scalars and counters (near_sum, near_cnt, n_added)
        FAR_TRY(cudaMemsetAsync(s.scal, 0, SCAL_COUNT * sizeof(u32), st));
        FAR_TRY(cudaMemsetAsync(&m.ctr->near_sum, 0, 2 * sizeof(unsigned long long), st));
        FAR_TRY(cudaMemsetAsync(&m.ctr->n_added, 0, sizeof(u32), st));
        return cudaSuccess;
    }
    const u32 sentinel = m.mask + 1u;
    Pose12 T{};
    if (pose) T = *pose;
    FAR_LAUNCH(k_world_keys, blocks_for(n), TPB, 0, st, s.in4, n, T, pose != nullptr || dpose.T != nullptr, dpose,
               m.inv_v, m.tv, s.world, s.keys, s.scal, m.ctr, s.admitted, s.flags, m.slots, m.mask, s.sk, s.sv,
               s.slot_cnt);
    mark(0);
    // groups by slot: contiguous ranges of s.sv_alt, each sorted by input index
    // groups above GS_BLOCK_MIN members are listed in s.pos (free until the admission)
    FAR_LAUNCH(k_group_alloc, blocks_for(n), TPB, 0, st, s.sk, s.sv, n, sentinel, s.slot_cnt, s.slot_base, s.scal,
               s.gstart, s.gsize, s.gslot, s.pos);
    FAR_LAUNCH(k_group_scatter, blocks_for(n), TPB, 0, st, s.sk, s.sv, n, sentinel, s.slot_base, s.sv_alt);
    mark(1);
    {
        // one resident wave (3 blocks of 8 warps per SM at 77 registers)
        const u32 warps = min(n, 152u * 24u);
        FAR_LAUNCH(k_group_sort, blocks_for(warps * 32u), TPB, 0, st, s.sv_alt, s.sk_alt, s.scal, s.rank, s.gstart,
                   s.gsize,
                   s.gslot, s.slot_cnt, s.flags, m.slots, (double)m.v, cfg, dpose.T, m.ctr, s.pos);
    }
    // voxel ordinals in first-input-index order (k_world_keys cleared the flags)
    FAR_TRY(scan_exclusive(s.flags, s.head_ord, n, nullptr, nullptr, s.partials, st));
    mark(2);
    AdmitArgs a;
    a.gslot = s.gslot;
    a.sv = s.sv_alt;
    a.gstart = s.gstart;
    a.gsize = s.gsize;
    a.scal = s.scal;
    a.world = s.world;
    a.slots = m.slots;
    a.pts = m.pts;
    a.ring = m.ring;
    a.max_buckets = m.max_buckets;
    a.ctr = m.ctr;
    a.nmax = m.nmax;
    a.k = m.k;
    a.dmin2 = m.dmin2;
    a.v = (double)m.v;
    a.cfg = cfg;
    a.dev_T = dpose.T;
    a.admitted = s.admitted;
    a.head_ord = s.head_ord;
    a.grp_cnt = s.grp_cnt;
    a.a_ord = s.a_ord;
    a.a_j = s.a_j;
    a.pos = s.pos;
    a.cexp = m.tv > 0 ? m.cexp : nullptr;
    a.grp_bucket = s.grp_bucket;
    a.grp_cnt0 = s.grp_cnt0;
    a.grp_exp0 = s.grp_exp0;
    a.big_list = s.rank;   // listed by k_group_sort; the ranks are written after the admission
    a.big_next = s.scal + SCAL_BIGNEXT;
    // the scan-local insert (the one that emits the sources) always runs on a map emptied just
    // before (map_clear, or k_local_reset after the previous scan)
    a.fresh = emit_sources ? 1 : 0;
    // groups <= n, up to 32 per warp and pass; one resident wave (4 blocks of 8 warps per SM at
    // 64 registers)
    const u32 warps = min(n, 152u * 32u);
    FAR_LAUNCH(k_admit, blocks_for(warps * 32u), TPB, 0, st, a);
    mark(3);
    // ranks of the admitted points (input order) and the voxels' bases in the grouped order
    FAR_TRY(scan_exclusive2(s.admitted, s.rank, nullptr, s.scal + SCAL_NADMIT, s.grp_cnt, s.grp_cnt,
                            s.scal + SCAL_NGROUPS, nullptr, n, s.partials, st));
    const bool prec = m.tv > 0;
    const bool covs = covariances && (m.cov || prec);
    FAR_LAUNCH(k_place_admitted, blocks_for(n), TPB, 0, st, s.admitted, s.rank, s.a_ord, s.a_j, s.grp_cnt, s.pos, n,
               m.pts, s.dest, covs ? s.added : nullptr, s.keys, (covs && prec) ? s.added_key : nullptr, s.scal,
               m.ctr, s.in4, emit_sources ? s.src : nullptr, s.src_index);
    mark(4);
    if (covs && !prec)
        FAR_TRY(knn_cov(m, nullptr, s.added, n, s.scal + SCAL_NADMIT, m.cov, s.added, nullptr, st));
    if (covs && prec) {
        FAR_TRY(knn_cov_tile(m, s.added, s.added_key, n, s.scal + SCAL_NADMIT, s.cov_tmp, st));
        const u32 warps = min(n, 152u * 64u);
        FAR_LAUNCH(k_cov_encode, blocks_for(warps * 32u), TPB, 0, st, s.grp_cnt, s.scal, s.grp_bucket, s.grp_cnt0,
                   s.grp_exp0, m.cexp, s.added, s.cov_tmp, m.nmax, m.cov_h4, m.cov_h2);
    }
    mark(5);
    return cudaGetLastError();
}

cudaError_t make_sources(DeviceMap& local, Scratch& s, u32 n, u32* knn_ids_out, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    FAR_TRY(knn_cov(local, s.src, nullptr, n, s.scal + SCAL_NADMIT, s.src_cov, nullptr, knn_ids_out, st));
    if (s.src_h4) {
        // precision variant: FP16 copies with one exponent per scan-local voxel
        const u32 warps = min(n, 152u * 64u);
        FAR_LAUNCH(k_src_encode, blocks_for(warps * 32u), TPB, 0, st, s.grp_cnt, s.scal, s.src_cov, s.src_h4,
                   s.src_h2, s.src_exp);
    }
    return cudaGetLastError();
}

__global__ void k_clear_counters(MapCounters* ctr, u32 ring_tail) {
    pdl_wait();
    pdl_trigger();
    MapCounters c{};
    c.ring_tail = ring_tail;
    *ctr = c;
}

cudaError_t map_clear(DeviceMap& m, cudaStream_t st) {
    FAR_TRY(cudaMemsetAsync(m.slots, 0xFF, (size_t)m.cap * sizeof(Slot), st));
    // every bucket free: ring = identity, head = 0, tail = number of buckets
    FAR_LAUNCH(k_iota, min(blocks_for(m.max_buckets), 152u * 8u), TPB, 0, st, m.ring, m.max_buckets);
    FAR_LAUNCH(k_clear_counters, 1, 1, 0, st, m.ctr, m.max_buckets);
    return cudaGetLastError();
}

// Empty again the slots a scan-local insert used (its group slots: every slot that received a
// key) and reset the counters. The scan-local map never evicts, so its bucket ring is still the
// identity and only the head and tail need resetting.
__global__ void k_local_reset(Slot* slots, const u32* __restrict__ gslot, const u32* __restrict__ scal,
                              MapCounters* ctr, u32 max_buckets) {
    pdl_wait();
    pdl_trigger();
    const u32 ng = scal[SCAL_NGROUPS];
    const u32 t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t == 0) {
        MapCounters c{};
        c.ring_tail = max_buckets;
        *ctr = c;
    }
    for (u32 g = t; g < ng; g += gridDim.x * blockDim.x) {
        Slot* sp = slots + gslot[g];
        sp->key = KEY_EMPTY;
        sp->bucket = NO_BUCKET;
        sp->count = 0xFFFFFFFFu;   // as the cleared table holds
    }
}

cudaError_t map_local_reset(DeviceMap& m, const Scratch& s, u32 n, cudaStream_t st) {
    FAR_LAUNCH(k_local_reset, max(1u, min(blocks_for(n), 152u * 8u)), TPB, 0, st, m.slots, s.gslot, s.scal, m.ctr,
               m.max_buckets);
    return cudaGetLastError();
}

cudaError_t map_evict(DeviceMap& m, const double center[3], double radius, cudaStream_t st, const double* dev_pose) {
    FAR_TRY(cudaMemsetAsync(&m.ctr->removed, 0, sizeof(unsigned long long), st));
    const u32 blocks = max(1u, (u32)(((u64)m.cap + (u64)TPB * EVICT_PER_THREAD - 1) / ((u64)TPB * EVICT_PER_THREAD)));
    const double c0 = center ? center[0] : 0.0, c1 = center ? center[1] : 0.0, c2 = center ? center[2] : 0.0;
    FAR_LAUNCH(k_evict, blocks, TPB, 0, st, m.slots, m.cap, (double)m.v, c0, c1, c2, radius * radius, m.ring, m.max_buckets,
                                    m.ctr, dev_pose);
    return cudaGetLastError();
}

cudaError_t map_rebuild(DeviceMap& m, cudaStream_t st) {
    FAR_TRY(cudaMemsetAsync(m.slots_alt, 0xFF, (size_t)m.cap * sizeof(Slot), st));
    FAR_TRY(cudaMemsetAsync(&m.ctr->max_probe, 0, sizeof(u32), st));
    FAR_TRY(cudaMemsetAsync(&m.ctr->n_tomb, 0, sizeof(u32), st));
    const u32 blocks = min(blocks_for(m.cap), 152u * 16u);
    FAR_LAUNCH(k_rebuild, blocks, TPB, 0, st, m.slots, m.cap, m.slots_alt, m.mask, m.ctr);
    Slot* t = m.slots;
    m.slots = m.slots_alt;
    m.slots_alt = t;
    return cudaGetLastError();
}

cudaError_t map_list_slots(const DeviceMap& m, u64* keys, u32* buckets, u32* counts, u32* n_out, u32 cap_out,
                           cudaStream_t st) {
    FAR_TRY(cudaMemsetAsync(n_out, 0, sizeof(u32), st));
    const u32 blocks = min(blocks_for(m.cap), 152u * 16u);
    FAR_LAUNCH(k_list_slots, blocks, TPB, 0, st, m.slots, m.cap, keys, buckets, counts, n_out, cap_out);
    return cudaGetLastError();
}

cudaError_t map_gather(const DeviceMap& m, const u32* buckets, const u32* counts, const u32* offsets,
                       const u64* keys, u32 nvox, float4* pts_out, float4* cov_out, cudaStream_t st) {
    if (nvox == 0) return cudaSuccess;
    FAR_LAUNCH(k_gather, blocks_for(nvox * 32u), TPB, 0, st, m.view(), buckets, counts, offsets, keys, nvox, pts_out,
               (m.cov || m.tv > 0) ? cov_out : nullptr);
    return cudaGetLastError();
}

cudaError_t map_knn(const DeviceMap& m, const float4* q, u32 n, u32 k, u32* ids, int32_t* found, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    FAR_K_CASES(launch_knn_stage, m, q, n, ids, found, st)
}

cudaError_t map_nearest(const DeviceMap& m, const float4* q, u32 n, float tau2, int64_t* ids, float* d2,
                        cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    FAR_LAUNCH(k_nearest_stage, blocks_for(n), TPB, 0, st, m.view(), q, n, tau2, ids, d2);
    return cudaGetLastError();
}

}  // namespace far

namespace far {

namespace {
// Outputs in admission-rank order (ascending input index); sources are stored voxel-grouped.
__global__ void k_export_sources(const float4* __restrict__ src, const u32* __restrict__ src_index,
                                 const float4* __restrict__ src_cov, const u32* __restrict__ n_dev, u32 n,
                                 int64_t* __restrict__ index, float* __restrict__ cov6, uint8_t* __restrict__ valid) {
    pdl_wait();
    pdl_trigger();
    const u32 nn = min(n, *n_dev);
    for (u32 j = blockIdx.x * blockDim.x + threadIdx.x; j < nn; j += gridDim.x * blockDim.x) {
        const u32 r = __float_as_uint(src[j].w);
        index[r] = (int64_t)src_index[j];
        const float4 c0 = src_cov[2 * (size_t)j], c1 = src_cov[2 * (size_t)j + 1];
        float* o = cov6 + 6 * (size_t)r;
        o[0] = c0.x; o[1] = c0.y; o[2] = c0.z; o[3] = c0.w; o[4] = c1.x; o[5] = c1.y;
        valid[r] = c1.z > 0.5f ? 1 : 0;
    }
}
}  // namespace

cudaError_t export_sources(const Scratch& s, u32 n, int64_t* index, float* cov6, uint8_t* valid, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    FAR_LAUNCH(k_export_sources, blocks_for(n), TPB, 0, st, s.src, s.src_index, s.src_cov, s.scal + SCAL_NADMIT, n,
               index, cov6, valid);
    return cudaGetLastError();
}

}  // namespace far
