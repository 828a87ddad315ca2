// Sparsity-aware GICP Gauss-Newton iteration (FAR-LIO Sec. III-A.2, Eq. 2-6).
//
// One launch = one iteration, fully on the device:
//   per source point (one thread): q = R s + t (FP32), 1-NN over the 27 voxels,
//   rejection by tau, M = (Sigma_r + R Sigma_s R^T)^-1 or I (SA GICP),
//   d = r - q, Cauchy IRLS weight w = 1 / (1 + e^2/kappa^2), e^2 = d^T M d,
//   accumulate w J^T M J (21 values) and w J^T M d (6) with J = [[q]x, -I];
//   FP32 per thread and per warp (shuffles), FP64 across warps and blocks;
//   the last block to finish reduces the block partials in a fixed order,
//   solves H xi = -g by FP64 Cholesky and applies T <- exp(xi) T (Eq. 6).
// The iteration checks a stop flag at entry, so a fixed-size chain of launches
// (or a CUDA graph of them) stops doing work once converged.
#include "gicp.cuh"
#include "search.cuh"

namespace far {

namespace {

// Threads per block and minimum resident blocks per SM of the linearisation kernel
// (compile-time tuning knobs; 128 x 5 keeps the kernel free of register spills).
#ifndef FAR_GN_THREADS
#define FAR_GN_THREADS 128
#endif
#ifndef FAR_GN_MIN_BLOCKS
#define FAR_GN_MIN_BLOCKS 5
#endif
constexpr int GN_THREADS = FAR_GN_THREADS;
constexpr int NACC = 28;   // 21 H + 6 g + chi2
constexpr int NPART = 32;  // doubles per block partial: 28 + n_corr + n_p2p + pad
constexpr int kDefaultTpp = 4;  // measured fastest on the 128 x 2048 workload

__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// ---- FP64 6x6 Cholesky solve and SE(3) exponential (single thread, registers only) ----
// Every loop has constant bounds and is unrolled, so the matrices stay in registers.
// Cholesky H = L L^T with one reciprocal square root per column (no divisions):
// r_j = 1 / sqrt(s_j), L_jj = s_j r_j, L_ij = t_ij r_j, and the substitutions multiply by r_j.
__device__ __forceinline__ bool chol6_solve(const double (&H)[6][6], const double (&b)[6], double (&x)[6]) {
    double L[6][6], r[6];
#pragma unroll
    for (int j = 0; j < 6; ++j) {
        double sj = H[j][j];
#pragma unroll
        for (int k = 0; k < j; ++k) sj -= L[j][k] * L[j][k];
        if (!(sj > 0.0)) return false;
        r[j] = rsqrt(sj);
        L[j][j] = sj * r[j];
#pragma unroll
        for (int i = j + 1; i < 6; ++i) {
            double t = H[i][j];
#pragma unroll
            for (int k = 0; k < j; ++k) t -= L[i][k] * L[j][k];
            L[i][j] = t * r[j];
        }
    }
    double y[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        double t = b[i];
#pragma unroll
        for (int k = 0; k < i; ++k) t -= L[i][k] * y[k];
        y[i] = t * r[i];
    }
#pragma unroll
    for (int i = 5; i >= 0; --i) {
        double t = y[i];
#pragma unroll
        for (int k = i + 1; k < 6; ++k) t -= L[k][i] * x[k];
        x[i] = t * r[i];
    }
    return true;
}

__device__ __forceinline__ u32 warp_sum_u(u32 v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Scan voxel c_nb_order[v] around the query for its nearest candidate, unless its box
// distance exceeds `bound`. Candidates are loaded four at a time.
template <bool PREC>
__device__ __forceinline__ void nn_try_voxel(const MapView& m, u32 max_probe, const QFrame<PREC>& f,
                                             const FaceDist& fd, int v, float bound, unsigned long long& best_key,
                                             u32& best_pos, int& best_v) {
    const int dx = c_nb_order[v][0], dy = c_nb_order[v][1], dz = c_nb_order[v][2];
    const int nx = f.k[0] + dx, ny = f.k[1] + dy, nz = f.k[2] + dz;
    u32 bucket, count;
    if (box_lb2(fd, dx, dy, dz) > bound || !key_in_range(nx) || !key_in_range(ny) || !key_in_range(nz) ||
        !find_slot(m.slots, m.mask, max_probe, nx, ny, nz, bucket, count))
        return;
    const float qx = f.q[0], qy = f.q[1], qz = f.q[2];
    const u32 base = bucket * m.nmax;
    const float ox = f.off(0, dx), oy = f.off(1, dy), oz = f.off(2, dz);
    for (u32 j0 = 0; j0 < count; j0 += 4) {
        float4 c[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            c[u] = (j0 + u < count) ? __ldg(m.pts + base + j0 + u) : make_float4(0.f, 0.f, 0.f, 0.f);
            if constexpr (PREC) {
                c[u].x = __fadd_rn(c[u].x, ox);
                c[u].y = __fadd_rn(c[u].y, oy);
                c[u].z = __fadd_rn(c[u].z, oz);
            }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            if (j0 + u < count) {
                const float d2 = dist2_rn(qx, qy, qz, c[u].x, c[u].y, c[u].z);
                const unsigned long long key = ((unsigned long long)__float_as_uint(d2) << 32) | __float_as_uint(c[u].w);
                if (key < best_key) {
                    best_key = key;
                    best_pos = base + j0 + u;
                    if constexpr (PREC) best_v = v;
                }
            }
        }
    }
}

// Share the group's best (packed key d2 bits << 32 | id, ordered like (d2, id) since d2 >= 0).
template <int TPP, bool PREC>
__device__ __forceinline__ void group_best(unsigned long long& best_key, u32& best_pos, int& best_v) {
#pragma unroll
    for (int o = TPP / 2; o > 0; o >>= 1) {
        const unsigned long long ok = __shfl_xor_sync(0xffffffffu, best_key, o);
        const u32 op = __shfl_xor_sync(0xffffffffu, best_pos, o);
        int ov = 0;
        if constexpr (PREC) ov = __shfl_xor_sync(0xffffffffu, best_v, o);
        if (ok < best_key) {
            best_key = ok;
            best_pos = op;
            if constexpr (PREC) best_v = ov;
        }
    }
}

__device__ __forceinline__ float nn_group_bound(unsigned long long best_key, float limit2) {
    return best_key == ~0ull ? limit2 : fminf(__uint_as_float((u32)(best_key >> 32)), limit2);
}

// Nearest map point of q (smallest (d^2, id)) searched by a group of TPP consecutive
// lanes. A first round scans TPP voxels at once: the own voxel and the TPP - 1 faces nearest
// to the query (TPP <= 6), else entries 0 .. TPP - 1 of the order own, faces, edges, corners
// (lane sl takes entry sl); the group then keeps only the other voxels whose box distance
// does not exceed min(best, tau^2), lists them in shared memory (`list`, 27 entries per
// group) and scans them TPP at a time, sharing the best after each round. A voxel whose box
// distance exceeds the bound cannot hold a point with a smaller (d^2, id), so the result is
// the exact minimum over the 27 voxels. best_v is the c_nb_order index of the winner's voxel
// (its frame offset in the precision variant). Every lane of the warp must call this.
template <int TPP, bool PREC>
__device__ __forceinline__ void group_nearest(const MapView& m, u32 max_probe, const QFrame<PREC>& f, bool keyed,
                                              float limit2, int sl, unsigned long long& best_key, u32& best_pos,
                                              int& best_v, unsigned char* list) {
    best_key = ~0ull;
    best_pos = 0;
    best_v = 0;
    const FaceDist fd = face_distances(f.q[0], f.q[1], f.q[2], f.lk[0], f.lk[1], f.lk[2], m.v);
    // first round: entries 0 .. TPP - 1 of the order; with fewer than 7 lanes, lane 0 takes the own
    // voxel and lanes 1 .. TPP - 1 the faces nearest to the query (face j = entry 1 + j, ties to
    // the lower entry), so that the first bound is as tight as the round allows
    u32 chosen = 0;   // bit v: entry v scanned in the first round (TPP <= 6)
    int my_first = sl;
    if constexpr (TPP <= 6) {
        const float fdist[6] = {fd.lo[0], fd.hi[0], fd.lo[1], fd.hi[1], fd.lo[2], fd.hi[2]};
        my_first = 0;
#pragma unroll
        for (int j = 0; j < 6; ++j) {
            int rank = 0;
#pragma unroll
            for (int i = 0; i < 6; ++i) rank += (fdist[i] < fdist[j] || (fdist[i] == fdist[j] && i < j)) ? 1 : 0;
            if (rank < TPP - 1) chosen |= 1u << (1 + j);
            if (rank == sl - 1) my_first = 1 + j;
        }
    }
    if (keyed && my_first < 27) nn_try_voxel<PREC>(m, max_probe, f, fd, my_first, limit2, best_key, best_pos, best_v);
    group_best<TPP, PREC>(best_key, best_pos, best_v);
    // survivors of the other voxels under the group's bound, compacted in input order
    const float bound0 = nn_group_bound(best_key, limit2);
    constexpr int kRest0 = TPP <= 6 ? 1 : TPP;   // first entry of the survivor scan
    u32 mine = 0;
    int k = 0;
    for (int v = kRest0 + sl; v < 27; v += TPP, ++k)
        if (keyed && !((chosen >> v) & 1u) &&
            !(box_lb2(fd, c_nb_order[v][0], c_nb_order[v][1], c_nb_order[v][2]) > bound0))
            mine |= 1u << k;
    const int cnt = __popc(mine);
    int pre = cnt;   // inclusive prefix over the group's lanes
#pragma unroll
    for (int o = 1; o < TPP; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, pre, o, TPP);
        if (sl >= o) pre += t;
    }
    const int total = __shfl_sync(0xffffffffu, pre, TPP - 1, TPP);
    pre -= cnt;
    k = 0;
    for (int v = kRest0 + sl; v < 27; v += TPP, ++k)
        if (mine & (1u << k)) list[pre++] = (unsigned char)v;
    __syncwarp();
    const int rounds = (__reduce_max_sync(0xffffffffu, (u32)total) + TPP - 1) / TPP;   // warp-uniform
    for (int r = 0; r < rounds; ++r) {
        const int s2 = r * TPP + sl;
        if (s2 < total)
            nn_try_voxel<PREC>(m, max_probe, f, fd, list[s2], nn_group_bound(best_key, limit2), best_key, best_pos,
                               best_v);
        group_best<TPP, PREC>(best_key, best_pos, best_v);
    }
    __syncwarp();
}

// Linearisation half of a Gauss-Newton iteration: TPP lanes cooperate on each source
// point's search, the group's first lane linearises it, and every block writes its
// partial sums (FP32 within warps, FP64 across the block's warps).
template <int TPP, bool PREC>
__device__ __forceinline__ void gn_lin_block(const GnArgs& a, u32 vblock, u32 vgrid) {
    // Each group of TPP lanes accumulates its 28 values in shared memory (its first lane
    // adds; an odd row stride keeps the adding lanes of a warp on distinct banks), which
    // keeps the accumulators out of the registers of every lane.
    constexpr int kGroups = GN_THREADS / TPP;
    constexpr int ACC_STRIDE = NACC + 3;
    constexpr int kParts = GN_THREADS / 32;
    __shared__ float gacc[kGroups * ACC_STRIDE];
    __shared__ unsigned char vlist[kGroups][28];   // surviving neighbour voxels of each group's query
    __shared__ float red[kParts][NACC + 2];
    __shared__ float pose_f[12];
    __shared__ u32 s_flag;
    RegState* st = a.st;
    if (threadIdx.x == 0) s_flag = *reinterpret_cast<volatile u32*>(&st->done);
    if (threadIdx.x < 12) {
        // the pose relative to the anchor (translation column minus A, in FP64, then rounded)
        const int j = threadIdx.x;
        double t = st->T[j];
        if ((j & 3) == 3) t = __dsub_rn(t, a.anchor[j >> 2]);
        pose_f[j] = (float)t;
    }
    for (int j = threadIdx.x; j < kGroups * ACC_STRIDE; j += GN_THREADS) gacc[j] = 0.f;
    __syncthreads();
    if (s_flag) return;

    const float R00 = pose_f[0], R01 = pose_f[1], R02 = pose_f[2], tx = pose_f[3];
    const float R10 = pose_f[4], R11 = pose_f[5], R12 = pose_f[6], ty = pose_f[7];
    const float R20 = pose_f[8], R21 = pose_f[9], R22 = pose_f[10], tz = pose_f[11];
    const MapView m = a.map;
    const u32 max_probe = m.ctr->max_probe;
    const u32 n = min(a.n_max, *a.n_src);
    const int sl = threadIdx.x % TPP;
    constexpr u32 kGroupsPerBlock = GN_THREADS / TPP;
    const u32 group = vblock * kGroupsPerBlock + threadIdx.x / TPP;
    const u32 warp_first = vblock * kGroupsPerBlock + (threadIdx.x & ~31u) / TPP;
    const u32 stride = vgrid * kGroupsPerBlock;

    u32 n_corr = 0, n_p2p = 0;

    for (u32 off = 0; warp_first + off < n; off += stride) {   // warp-uniform trip count
        const u32 i = group + off;
        const bool active = i < n;
        const float4 s = active ? a.src[i] : make_float4(0.f, 0.f, 0.f, 0.f);
        // Eq. 2 / Eq. 6: current estimate applied to the source point
        const float qx = fmaf(R00, s.x, fmaf(R01, s.y, fmaf(R02, s.z, tx)));
        const float qy = fmaf(R10, s.x, fmaf(R11, s.y, fmaf(R12, s.z, ty)));
        const float qz = fmaf(R20, s.x, fmaf(R21, s.y, fmaf(R22, s.z, tz)));
        unsigned long long bkey = ~0ull;
        u32 bpos = 0;
        int bv = 0;
        QFrame<PREC> f;
        const bool keyed = active && make_qframe<PREC>(m, qx, qy, qz, a.ftile, f);
        if constexpr (TPP == 1) {
            float d2b;
            u32 idb;
            if (keyed && nearest27q<PREC>(m, max_probe, f, a.tau2, d2b, idb, bpos, bv))
                bkey = ((unsigned long long)__float_as_uint(d2b) << 32) | idb;
        } else {
            group_nearest<TPP, PREC>(m, max_probe, f, keyed, a.tau2, sl, bkey, bpos, bv, vlist[threadIdx.x / TPP]);
        }
        if (!active || sl != 0) continue;
        const float bd2 = __uint_as_float((u32)(bkey >> 32));
        const bool ok = bkey != ~0ull && !(bd2 > a.tau2);
        if (a.corr_out) a.corr_out[__float_as_uint(s.w)] = ok ? (int32_t)(u32)bkey : -1;
        if (!ok) continue;
        float4 r = __ldg(m.pts + bpos);
        float rc[6], sc[6];
        bool r_ok, s_ok;
        if constexpr (PREC) {
            // the winner's frame offset; TPP == 1 reports its voxel as (dx+1)*9+(dy+1)*3+(dz+1)
            int dx, dy, dz;
            if constexpr (TPP == 1) {
                dx = bv / 9 - 1;
                dy = (bv / 3) % 3 - 1;
                dz = bv % 3 - 1;
            } else {
                dx = c_nb_order[bv][0];
                dy = c_nb_order[bv][1];
                dz = c_nb_order[bv][2];
            }
            r.x = __fadd_rn(r.x, f.off(0, dx));
            r.y = __fadd_rn(r.y, f.off(1, dy));
            r.z = __fadd_rn(r.z, f.off(2, dz));
            r_ok = cov16_decode(__ldg(m.cov_h4 + bpos), __ldg(m.cov_h2 + bpos), __ldg(m.cexp + bpos / m.nmax), rc);
            s_ok = cov16_decode(a.src_h4[i], a.src_h2[i], (int)a.src_exp[i], sc);
        } else {
            const float4 rc0 = __ldg(m.cov + 2 * (size_t)bpos);
            const float4 rc1 = __ldg(m.cov + 2 * (size_t)bpos + 1);
            const float4 sc0 = a.src_cov[2 * (size_t)i];
            const float4 sc1 = a.src_cov[2 * (size_t)i + 1];
            rc[0] = rc0.x; rc[1] = rc0.y; rc[2] = rc0.z; rc[3] = rc0.w; rc[4] = rc1.x; rc[5] = rc1.y;
            sc[0] = sc0.x; sc[1] = sc0.y; sc[2] = sc0.z; sc[3] = sc0.w; sc[4] = sc1.x; sc[5] = sc1.y;
            r_ok = rc1.z > 0.5f;
            s_ok = sc1.z > 0.5f;
        }
        // M: (Sigma_r + R Sigma_s R^T)^-1, or I when a covariance is invalid (SA GICP)
        float M00 = 1.f, M01 = 0.f, M02 = 0.f, M11 = 1.f, M12 = 0.f, M22 = 1.f;
        const bool p2p = !(r_ok && s_ok);
        if (!p2p) {
            const float S00 = sc[0], S01 = sc[1], S02 = sc[2], S11 = sc[3], S12 = sc[4], S22 = sc[5];
            // A = R S
            const float A00 = R00 * S00 + R01 * S01 + R02 * S02, A01 = R00 * S01 + R01 * S11 + R02 * S12,
                        A02 = R00 * S02 + R01 * S12 + R02 * S22;
            const float A10 = R10 * S00 + R11 * S01 + R12 * S02, A11 = R10 * S01 + R11 * S11 + R12 * S12,
                        A12 = R10 * S02 + R11 * S12 + R12 * S22;
            const float A20 = R20 * S00 + R21 * S01 + R22 * S02, A21 = R20 * S01 + R21 * S11 + R22 * S12,
                        A22 = R20 * S02 + R21 * S12 + R22 * S22;
            // C = Sigma_r + A R^T (symmetric)
            const float a_ = rc[0] + A00 * R00 + A01 * R01 + A02 * R02;
            const float b_ = rc[1] + A00 * R10 + A01 * R11 + A02 * R12;
            const float c_ = rc[2] + A00 * R20 + A01 * R21 + A02 * R22;
            const float d_ = rc[3] + A10 * R10 + A11 * R11 + A12 * R12;
            const float e_ = rc[4] + A10 * R20 + A11 * R21 + A12 * R22;
            const float f_ = rc[5] + A20 * R20 + A21 * R21 + A22 * R22;
            const float C00 = d_ * f_ - e_ * e_, C01 = c_ * e_ - b_ * f_, C02 = b_ * e_ - c_ * d_;
            const float C11 = a_ * f_ - c_ * c_, C12 = b_ * c_ - a_ * e_, C22 = a_ * d_ - b_ * b_;
            const float idet = 1.0f / (a_ * C00 + b_ * C01 + c_ * C02);
            M00 = C00 * idet; M01 = C01 * idet; M02 = C02 * idet;
            M11 = C11 * idet; M12 = C12 * idet; M22 = C22 * idet;
        }
        // Eq. 3 residual and Eq. 4/5 weight
        const float dx = r.x - qx, dy = r.y - qy, dz = r.z - qz;
        const float Mdx = M00 * dx + M01 * dy + M02 * dz;
        const float Mdy = M01 * dx + M11 * dy + M12 * dz;
        const float Mdz = M02 * dx + M12 * dy + M22 * dz;
        const float e2 = dx * Mdx + dy * Mdy + dz * Mdz;
        const float w = a.kappa2 / (a.kappa2 + e2);
        // MQ = M [q]x
        const float MQ00 = M01 * qz - M02 * qy, MQ01 = M02 * qx - M00 * qz, MQ02 = M00 * qy - M01 * qx;
        const float MQ10 = M11 * qz - M12 * qy, MQ11 = M12 * qx - M01 * qz, MQ12 = M01 * qy - M11 * qx;
        const float MQ20 = M12 * qz - M22 * qy, MQ21 = M22 * qx - M02 * qz, MQ22 = M02 * qy - M12 * qx;
        // [q]x^T MQ: row a of [q]x^T is column a of [q]x
        // [q]x = [[0,-qz,qy],[qz,0,-qx],[-qy,qx,0]]
        const float T00 = qz * MQ10 - qy * MQ20, T01 = qz * MQ11 - qy * MQ21, T02 = qz * MQ12 - qy * MQ22;
        const float T11 = -qz * MQ01 + qx * MQ21, T12 = -qz * MQ02 + qx * MQ22;
        const float T22 = qy * MQ02 - qx * MQ12;
        float* h = gacc + (threadIdx.x / TPP) * ACC_STRIDE;
        // row 0..2 rotational block, cross block -MQ^T, translational block M
        h[0] = fmaf(w, T00, h[0]);   h[1] = fmaf(w, T01, h[1]);   h[2] = fmaf(w, T02, h[2]);
        h[3] = fmaf(w, -MQ00, h[3]); h[4] = fmaf(w, -MQ10, h[4]); h[5] = fmaf(w, -MQ20, h[5]);
        h[6] = fmaf(w, T11, h[6]);   h[7] = fmaf(w, T12, h[7]);
        h[8] = fmaf(w, -MQ01, h[8]); h[9] = fmaf(w, -MQ11, h[9]); h[10] = fmaf(w, -MQ21, h[10]);
        h[11] = fmaf(w, T22, h[11]);
        h[12] = fmaf(w, -MQ02, h[12]); h[13] = fmaf(w, -MQ12, h[13]); h[14] = fmaf(w, -MQ22, h[14]);
        h[15] = fmaf(w, M00, h[15]); h[16] = fmaf(w, M01, h[16]); h[17] = fmaf(w, M02, h[17]);
        h[18] = fmaf(w, M11, h[18]); h[19] = fmaf(w, M12, h[19]);
        h[20] = fmaf(w, M22, h[20]);
        // g = w [Md x q; -Md]
        h[21] = fmaf(w, Mdy * qz - Mdz * qy, h[21]);
        h[22] = fmaf(w, Mdz * qx - Mdx * qz, h[22]);
        h[23] = fmaf(w, Mdx * qy - Mdy * qx, h[23]);
        h[24] = fmaf(w, -Mdx, h[24]);
        h[25] = fmaf(w, -Mdy, h[25]);
        h[26] = fmaf(w, -Mdz, h[26]);
        h[27] += 0.5f * a.kappa2 * log1pf(e2 / a.kappa2);
        ++n_corr;
        if (p2p) ++n_p2p;
    }

    // ---- reduction: FP32 over the groups of each part, FP64 across parts and blocks ----
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    n_corr = warp_sum_u(n_corr);
    n_p2p = warp_sum_u(n_p2p);
    __syncthreads();
    {
        // thread (part, j): FP32 sum of value j over groups part * G/P .. in order
        constexpr int kPer = kGroups / kParts;
        if (lane < NACC) {
            float v = 0.f;
#pragma unroll 4
            for (int g = 0; g < kPer; ++g) v += gacc[(warp * kPer + g) * ACC_STRIDE + lane];
            red[warp][lane] = v;
        } else if (lane == NACC) {
            red[warp][NACC] = __uint_as_float(n_corr);
            red[warp][NACC + 1] = __uint_as_float(n_p2p);
        }
    }
    __syncthreads();
    if (threadIdx.x < NPART) {
        double s = 0.0;
        if (threadIdx.x < NACC) {
            for (int w = 0; w < kParts; ++w) s += (double)red[w][threadIdx.x];
        } else if (threadIdx.x < NACC + 2) {
            for (int w = 0; w < kParts; ++w) s += (double)__float_as_uint(red[w][threadIdx.x]);
        }
        // value-major: partials[v * blocks + block], read coalesced by the solve kernel
        a.partials[(size_t)threadIdx.x * vgrid + vblock] = s;
    }
}

// The Gauss-Newton chain (lin, solve, lin, ...) is launched with programmatic dependent launch:
// each kernel waits for its predecessor first and immediately lets its successor launch.
template <int TPP, bool PREC>
__global__ void __launch_bounds__(GN_THREADS, FAR_GN_MIN_BLOCKS) k_gn_lin(GnArgs a) {
    pdl_wait();
    pdl_trigger();
    gn_lin_block<TPP, PREC>(a, blockIdx.x, gridDim.x);
}

// Batched linearisation: the grid is shared by all problems; block b works for problem
// block_prob[b] as its (b - block_begin)-th block of nblocks.
template <int TPP, bool PREC>
__global__ void __launch_bounds__(GN_THREADS, FAR_GN_MIN_BLOCKS) k_gn_lin_batch(const BatchProblem* __restrict__ probs,
                                                                                const u32* __restrict__ block_prob) {
    pdl_wait();
    pdl_trigger();
    const BatchProblem& p = probs[block_prob[blockIdx.x]];
    gn_lin_block<TPP, PREC>(p.args, blockIdx.x - p.block_begin, p.nblocks);
}

// Upper-triangle index of H[r][c] (r <= c) in the reduced values: row-major, 21 entries.
__device__ __forceinline__ int tri_upper(int r, int c) { return r * 6 - (r * (r - 1)) / 2 + (c - r); }

// The solving warp: H and g from the reduced values, FP64 Cholesky, SE(3) update (Eq. 6),
// convergence and time checks, bookkeeping. The FP64 work is spread over the lanes (this GPU's
// FP64 rate, about 2 fma per cycle per SM, makes an FP64 instruction cost the warp about as much
// with one active lane as with 32; one lane doing it all took 9.3 us, the lanes together 5.6): lane
// l < 21 holds the lower-triangle entry (i, j) with l = i (i + 1) / 2 + j and the Cholesky is
// right-looking (each column scaled by its r_k = 1 / sqrt(pivot), then the trailing entries
// updated, one fma per entry and column, in the same order as a row-by-row factorisation);
// the substitutions run on lanes 0-5, the exponential's 12 entries and the pose update on
// lanes 0-11. Every lane of the warp must call this.
__device__ __forceinline__ void gn_solve_warp(const GnArgs& a, const double* tot, int lane) {
    constexpr unsigned FULL = 0xffffffffu;
    RegState* st = a.st;
    const u32 n_corr_tot = (u32)tot[28];
    // lane -> (i, j), i >= j, for the 21 entries of the lower triangle
    int li = 0, lj = lane;
    while (li < 6 && lj > li) {
        lj -= li + 1;
        ++li;
    }
    const bool tri = lane < 21;
    if (!tri) li = lj = 0;
    if (a.update) {
        const double Tl = lane < 12 ? st->T[lane] : 0.0;     // the pose (loaded while the solve runs)
        double e = tri ? tot[tri_upper(lj, li)] : 0.0;      // H[i][j], becomes L[i][j]
        double bv = lane < 6 ? -tot[21 + lane] : 0.0;        // -g, becomes y, then xi
        bool ok = n_corr_tot >= 6;
        double rk[6];
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            const double d = __shfl_sync(FULL, e, k * (k + 1) / 2 + k);   // the pivot after k updates
            if (!(d > 0.0)) ok = false;
            const double r = ok ? rsqrt(d) : 0.0;
            rk[k] = r;
            if (tri && lj == k) e = (li == k) ? d * r : e * r;
            const double lik = __shfl_sync(FULL, e, li >= k ? li * (li + 1) / 2 + k : 0);
            const double ljk = __shfl_sync(FULL, e, lj >= k ? lj * (lj + 1) / 2 + k : 0);
            if (tri && lj > k) e = fma(-lik, ljk, e);
        }
        // L y = -g, then L^T xi = y
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            const double yk = __shfl_sync(FULL, bv, k) * rk[k];
            const double lik = __shfl_sync(FULL, e, (lane > k && lane < 6) ? lane * (lane + 1) / 2 + k : 0);
            if (lane == k) bv = yk;
            else if (lane > k && lane < 6) bv = fma(-lik, yk, bv);
        }
#pragma unroll
        for (int k = 5; k >= 0; --k) {
            const double xk = __shfl_sync(FULL, bv, k) * rk[k];
            const double lki = __shfl_sync(FULL, e, lane < k ? k * (k + 1) / 2 + lane : 0);
            if (lane == k) bv = xk;
            else if (lane < k) bv = fma(-lki, xk, bv);
        }
        double xi[6];
#pragma unroll
        for (int j = 0; j < 6; ++j) xi[j] = __shfl_sync(FULL, bv, j);
        if (ok) {
            // SE(3) exponential, xi = [phi; rho]: R = I + A K + B K^2, V = I + B K + C K^2 with
            // A = sin t / t, B = (1 - cos t) / t^2, C = (t - sin t) / t^3. Below t = 0.1 the three
            // are evaluated from their Taylor series in t^2 (terms through t^10; the first omitted
            // term is below 1e-21), which needs neither sqrt nor sincos; above, from sincos.
            const double px = xi[0], py = xi[1], pz = xi[2];
            const double t2 = px * px + py * py + pz * pz;
            double A, B, C;
            if (t2 < 1e-2) {
                // the three series are one nested form s0 (1 - t2 d1 (1 - t2 d2 (... (1 - t2 d5)))),
                // lane 0 evaluating A, lane 1 B and lane 2 C (one FP64 sequence for all three)
                const int f = lane < 3 ? lane : 0;
                const double s0 = f == 0 ? 1.0 : (f == 1 ? 0.5 : 1.0 / 6.0);
                const double d1 = f == 0 ? 1.0 / 6.0 : (f == 1 ? 1.0 / 12.0 : 1.0 / 20.0);
                const double d2 = f == 0 ? 1.0 / 20.0 : (f == 1 ? 1.0 / 30.0 : 1.0 / 42.0);
                const double d3 = f == 0 ? 1.0 / 42.0 : (f == 1 ? 1.0 / 56.0 : 1.0 / 72.0);
                const double d4 = f == 0 ? 1.0 / 72.0 : (f == 1 ? 1.0 / 90.0 : 1.0 / 110.0);
                const double d5 = f == 0 ? 1.0 / 110.0 : (f == 1 ? 1.0 / 132.0 : 1.0 / 156.0);
                const double v = s0 * (1.0 - t2 * d1 * (1.0 - t2 * d2 * (1.0 - t2 * d3 * (1.0 - t2 * d4 *
                                                                                     (1.0 - t2 * d5)))));
                A = __shfl_sync(FULL, v, 0);
                B = __shfl_sync(FULL, v, 1);
                C = __shfl_sync(FULL, v, 2);
            } else {
                const double th = sqrt(t2);
                double sn, cs;
                sincos(th, &sn, &cs);
                A = sn / th;
                B = (1.0 - cs) / t2;
                C = (th - sn) / (t2 * th);
            }
            // entry (row, col) of [R | V rho] on lane 4 row + col, lanes 0-11; K^2 = phi phi^T - t2 I
            const int row = (lane >> 2) % 3, col = lane & 3;
            const double phr = row == 0 ? px : (row == 1 ? py : pz);
            auto kmat = [&](int i, int j) {   // K = [phi]x
                if (i == j) return 0.0;
                const int o = 3 - i - j;       // the third axis
                const double ph = o == 0 ? px : (o == 1 ? py : pz);
                return ((j - i + 3) % 3 == 1) ? -ph : ph;
            };
            // R and V entry (row, c) on lanes with col = c < 3; the translation V rho of a row on its
            // lane with col = 3, summed over the row's V entries in column order
            const int cc = col < 3 ? col : 0;
            const double phc = cc == 0 ? px : (cc == 1 ? py : pz);
            const double k2 = phr * phc - ((row == cc) ? t2 : 0.0);
            const double id = (row == cc) ? 1.0 : 0.0;
            const double kk = kmat(row, cc);
            const double Rv = id + A * kk + B * k2;
            const double Vv = id + B * kk + C * k2;
            const double v0 = __shfl_sync(FULL, Vv, 4 * row), v1 = __shfl_sync(FULL, Vv, 4 * row + 1);
            const double v2 = __shfl_sync(FULL, Vv, 4 * row + 2);
            double Ev = Rv;
            if (col == 3) {
                double t = 0.0;
                t += v0 * xi[3];
                t += v1 * xi[4];
                t += v2 * xi[5];
                Ev = t;
            }
            // Eq. 6: T <- exp(xi) T about the anchor A (t - A is updated, then A is added back),
            // written before the bookkeeping (the next launch waits on it)
            const double e0 = __shfl_sync(FULL, Ev, 4 * row), e1 = __shfl_sync(FULL, Ev, 4 * row + 1);
            const double e2 = __shfl_sync(FULL, Ev, 4 * row + 2), e3 = __shfl_sync(FULL, Ev, 4 * row + 3);
            const double ta = __shfl_sync(FULL, Tl, col), tb = __shfl_sync(FULL, Tl, 4 + col);
            const double tc = __shfl_sync(FULL, Tl, 8 + col);
            if (lane < 12) {
                if (col < 3) {
                    st->T[lane] = e0 * ta + e1 * tb + e2 * tc;
                } else {
                    const double tr0 = ta - a.anchor[0], tr1 = tb - a.anchor[1], tr2 = tc - a.anchor[2];
                    const double ar = row == 0 ? a.anchor[0] : (row == 1 ? a.anchor[1] : a.anchor[2]);
                    st->T[lane] = (e0 * tr0 + e1 * tr1 + e2 * tr2 + e3) + ar;
                }
            }
            if (lane < 6) st->xi[lane] = bv;   // lane j holds xi[j]
            if (lane == 0) {
                // termination: the increment expressed at the initial sensor position c (relative to
                // the anchor), [phi; rho + phi x c], so the test does not depend on where the world
                // origin lies
                const double* c = a.conv_center;
                const double r0 = xi[3] + (xi[1] * c[2] - xi[2] * c[1]);
                const double r1 = xi[4] + (xi[2] * c[0] - xi[0] * c[2]);
                const double r2 = xi[5] + (xi[0] * c[1] - xi[1] * c[0]);
                const double nx = xi[0] * xi[0] + xi[1] * xi[1] + xi[2] * xi[2] + r0 * r0 + r1 * r1 + r2 * r2;
                st->xi_norm2 = nx;
                st->iters += 1;
                if (nx <= a.conv_eps * a.conv_eps) {
                    st->converged = 1;
                    st->done = 1;
                }
                if (a.budget_ns > 0 && globaltimer_ns() - st->t_start_ns > a.budget_ns) {
                    st->status = 6;
                    st->done = 1;
                }
            }
        } else if (lane == 0) {
            st->status = 5;
            st->done = 1;
        }
    } else if (lane == 0) {
        st->done = 1;
    }
    // the linearisation's H (full), g, chi2 and counts
    {
        const int r = lane / 6, c = lane % 6;
        st->H[lane] = tot[r <= c ? tri_upper(r, c) : tri_upper(c, r)];
        if (lane < 4) {
            const int r2 = (32 + lane) / 6, c2 = (32 + lane) % 6;
            st->H[32 + lane] = tot[r2 <= c2 ? tri_upper(r2, c2) : tri_upper(c2, r2)];
        }
        if (lane < 6) st->g[lane] = tot[21 + lane];
        if (lane == 0) {
            st->chi2 = tot[27];
            st->n_corr = n_corr_tot;
            st->n_p2p = (u32)tot[29];
        }
    }
}

// Solve half of a Gauss-Newton iteration. Value v of the block partials (col = partials +
// v * nblocks) is summed in FP64 by one warp in a fixed order: lane l adds blocks l, l + 64, ...
// and l + 32, l + 96, ... in two chains, then the two chains, then a fixed shuffle tree (every
// lane ends with the same sum). The order depends neither on timing nor on the kernel that runs
// it, so a problem's result is the same alone and in a batch.
__device__ __forceinline__ double warp_reduce_value(const double* __restrict__ col, u32 nblocks, int lane) {
    double c0 = 0.0, c1 = 0.0;
    u32 b = lane;
#pragma unroll 4
    for (; b + 32 < nblocks; b += 64) {
        c0 += __ldcg(col + b);
        c1 += __ldcg(col + b + 32);
    }
    if (b < nblocks) c0 += __ldcg(col + b);
    double s = c0 + c1;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    return s;
}

// Solve half of one registration over NPART one-warp blocks (the FP64 rate of a single SM
// would otherwise bound the reduction): block v reduces value v into st->red[v]; every block
// then takes a ticket, and the block that takes the last one (all values written and fenced
// before their tickets) solves. Returns true in that block.
__device__ __forceinline__ bool gn_solve_wide(const GnArgs& a, u32 nblocks) {
    static_assert(NPART == 32, "one lane per reduced value in the solving block");
    RegState* st = a.st;
    const int lane = threadIdx.x & 31;
    // once the stop flag is set a launch only keeps the ticket count (no reduction, no solve)
    const bool stopped = *reinterpret_cast<volatile u32*>(&st->done) != 0u;
    const double v = stopped ? 0.0 : warp_reduce_value(a.partials + (size_t)blockIdx.x * nblocks, nblocks, lane);
    __shared__ u32 s_last;
    __shared__ double tot[NPART];
    if (lane == 0) {
        st->red[blockIdx.x] = v;
        __threadfence();
        const u32 t = atomicAdd(&st->block_counter, 1u);
        s_last = t + 1u == gridDim.x;
        if (s_last) st->block_counter = 0u;   // ready for the next launch
    }
    __syncwarp();
    if (!s_last) return false;
    __threadfence();
    tot[lane] = __ldcg(&st->red[lane]);
    __syncwarp();
    if (__shfl_sync(0xffffffffu, *reinterpret_cast<volatile u32*>(&st->done), 0) == 0u) gn_solve_warp(a, tot, lane);
    return true;
}

__global__ void __launch_bounds__(32) k_gn_solve(GnArgs a, u32 nblocks) {
    pdl_wait();
    pdl_trigger();
    gn_solve_wide(a, nblocks);
}

// Batched solve: blocks (v, p) reduce value v of problem p; the last of problem p's blocks
// solves it (the same arithmetic as the single-problem solve).
__global__ void __launch_bounds__(32) k_gn_solve_batch(const BatchProblem* __restrict__ probs) {
    pdl_wait();
    pdl_trigger();
    const BatchProblem& p = probs[blockIdx.y];
    gn_solve_wide(p.args, p.nblocks);
}

// Kernels of the graph loop: the arguments come from device memory.
template <int TPP, bool PREC>
__global__ void __launch_bounds__(GN_THREADS, FAR_GN_MIN_BLOCKS) k_gn_lin_dev(const GnArgs* __restrict__ ap) {
    pdl_wait();
    pdl_trigger();
    gn_lin_block<TPP, PREC>(*ap, blockIdx.x, gridDim.x);
}

__global__ void __launch_bounds__(32) k_gn_solve_dev(const GnArgs* __restrict__ ap, u32 nblocks,
                                                    cudaGraphConditionalHandle loop) {
    pdl_wait();
    pdl_trigger();
    const GnArgs& a = *ap;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        // the body runs at most max_iters times (every run but a final one applies an update);
        // past that bound the loop ends with an internal error instead of running on
        RegState* st = a.st;
        if (st->trips++ > a.max_iters) {
            st->status = 7;
            st->done = 1;
            cudaGraphSetConditional(loop, 0u);
        }
    }
    if (gn_solve_wide(a, nblocks) && threadIdx.x == 0) {
        const RegState* st = a.st;
        const bool stop = *reinterpret_cast<const volatile u32*>(&st->done) != 0u ||
                          *reinterpret_cast<const volatile u32*>(&st->iters) >= a.max_iters;
        cudaGraphSetConditional(loop, stop ? 0u : 1u);
    }
}

// Reset every problem's state to its initial pose (init: 16 doubles per problem).
__global__ void k_gn_begin_batch(const BatchProblem* __restrict__ probs, u32 nprob, const double* __restrict__ init) {
    pdl_wait();
    pdl_trigger();
    const u32 p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= nprob) return;
    RegState* st = probs[p].args.st;
    for (int j = 0; j < 16; ++j) st->T[j] = init[16 * (size_t)p + j];
    for (int j = 0; j < 36; ++j) st->H[j] = 0.0;
    for (int j = 0; j < 6; ++j) {
        st->g[j] = 0.0;
        st->xi[j] = 0.0;
    }
    st->chi2 = 0.0;
    st->xi_norm2 = 0.0;
    st->n_corr = st->n_p2p = st->iters = st->converged = st->status = st->done = 0;
    st->block_counter = 0;
    st->trips = 0;
    st->n_src = *probs[p].args.n_src;
    st->t_start_ns = globaltimer_ns();
}

// Copy every problem's state into one array (one device-to-host copy afterwards).
__global__ void k_gather_states(const BatchProblem* __restrict__ probs, u32 nprob, RegState* __restrict__ out) {
    pdl_wait();
    pdl_trigger();
    const u32 p = blockIdx.x;
    if (p >= nprob) return;
    const u32* src = reinterpret_cast<const u32*>(probs[p].args.st);
    u32* dst = reinterpret_cast<u32*>(out + p);
    for (u32 j = threadIdx.x; j < sizeof(RegState) / 4; j += blockDim.x) dst[j] = src[j];
}

__global__ void k_gn_begin(RegState* st, Pose16 init, const u32* n_src) {
    pdl_wait();
    pdl_trigger();
    st->n_src = n_src ? *n_src : 0u;
    for (int j = 0; j < 16; ++j) st->T[j] = init.m[j];
    for (int j = 0; j < 36; ++j) st->H[j] = 0.0;
    for (int j = 0; j < 6; ++j) {
        st->g[j] = 0.0;
        st->xi[j] = 0.0;
    }
    st->chi2 = 0.0;
    st->xi_norm2 = 0.0;
    st->n_corr = st->n_p2p = st->iters = st->converged = st->status = st->done = 0;
    st->block_counter = 0;
    st->trips = 0;
    st->t_start_ns = globaltimer_ns();
}

// Output covariance: H^-1 of the last linearisation (FP64, single thread).
__global__ void k_gn_cov(RegState* st, double* cov) {
    pdl_wait();
    pdl_trigger();
    double H[6][6], e[6], x[6];
#pragma unroll
    for (int r = 0; r < 6; ++r)
#pragma unroll
        for (int c = 0; c < 6; ++c) H[r][c] = st->H[6 * r + c];
    for (int c = 0; c < 6; ++c) {
#pragma unroll
        for (int r = 0; r < 6; ++r) e[r] = (r == c) ? 1.0 : 0.0;
        if (!chol6_solve(H, e, x)) {
            for (int j = 0; j < 36; ++j) cov[j] = 0.0;
            return;
        }
#pragma unroll
        for (int r = 0; r < 6; ++r) cov[6 * r + c] = x[r];
    }
}

// Map footprint of one Gauss-Newton launch at the current pose: the distinct
// voxels probed by the 27-neighbourhoods of all source points and the points
// they hold (the unique data a launch must read at least once).
__global__ void k_footprint(GnArgs a, u32* __restrict__ touched, unsigned long long* __restrict__ out) {
    pdl_wait();
    pdl_trigger();
    const MapView m = a.map;
    const RegState* st = a.st;
    const u32 n = st->n_src;
    const u32 max_probe = m.ctr->max_probe;
    float T[12];
    for (int j = 0; j < 12; ++j) T[j] = (float)((j & 3) == 3 ? st->T[j] - a.anchor[j >> 2] : st->T[j]);
    for (u32 i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float4 s = a.src[i];
        const float qx = fmaf(T[0], s.x, fmaf(T[1], s.y, fmaf(T[2], s.z, T[3])));
        const float qy = fmaf(T[4], s.x, fmaf(T[5], s.y, fmaf(T[6], s.z, T[7])));
        const float qz = fmaf(T[8], s.x, fmaf(T[9], s.y, fmaf(T[10], s.z, T[11])));
        int kx, ky, kz;
        if (!voxel_key3(qx, qy, qz, m.inv_v, kx, ky, kz)) continue;
        if (m.tv > 0) {
            kx += a.ftile[0] * m.tv;
            ky += a.ftile[1] * m.tv;
            kz += a.ftile[2] * m.tv;
        }
        for (int dx = -1; dx <= 1; ++dx)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dz = -1; dz <= 1; ++dz) {
                    const int nx = kx + dx, ny = ky + dy, nz = kz + dz;
                    if (!key_in_range(nx) || !key_in_range(ny) || !key_in_range(nz)) continue;
                    const u64 key = pack_key(nx, ny, nz);
                    u32 h = hash_key(nx, ny, nz) & m.mask;
                    for (u32 p = 0; p <= max_probe; ++p) {
                        const Slot sl = m.slots[h];
                        if (sl.key == key) {
                            if (sl.bucket != NO_BUCKET && atomicExch(&touched[h], 1u) == 0u) {
                                atomicAdd(&out[0], 1ull);
                                atomicAdd(&out[1], (unsigned long long)sl.count);
                            }
                            break;
                        }
                        if (sl.key == KEY_EMPTY) break;
                        h = (h + 1) & m.mask;
                    }
                }
    }
}

}  // namespace

cudaError_t gn_footprint(const GnArgs& a, u32* touched, u32 cap, unsigned long long* out2, u32 n_upper,
                         cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(touched, 0, (size_t)cap * sizeof(u32), s);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(out2, 0, 2 * sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    FAR_LAUNCH(k_footprint, gn_grid(n_upper, 1), GN_THREADS, 0, s, a, touched, out2);
    return cudaGetLastError();
}

cudaError_t gn_covariance(RegState* st, double* cov36, cudaStream_t s) {
    FAR_LAUNCH(k_gn_cov, 1, 1, 0, s, st, cov36);
    return cudaGetLastError();
}

namespace {
constexpr u32 kMaxGnBlocks = 152u * 8u;

// Blocks of k_gn_lin<TPP> that fit on the device at once (one wave), at most kMaxGnBlocks.
template <int TPP>
u32 resident_gn_blocks() {
    // the grid must not depend on the map's precision mode (a batch may mix modes); both
    // kernels are compiled for FAR_GN_MIN_BLOCKS resident blocks, the plain one is measured
    static u32 cached = 0;
    if (cached) return cached;
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_gn_lin<TPP, false>, GN_THREADS, 0) != cudaSuccess ||
        sms <= 0 || per_sm <= 0) {
        cudaGetLastError();
        return kMaxGnBlocks;
    }
    const u32 r = (u32)sms * (u32)per_sm;
    cached = r < kMaxGnBlocks ? r : kMaxGnBlocks;
    return cached;
}

template <int TPP>
u32 grid_for(u32 n_upper) {
    const u64 groups = (u64)n_upper;
    u64 b = (groups * TPP + GN_THREADS - 1) / GN_THREADS;
    if (b == 0) b = 1;
    const u32 r = resident_gn_blocks<TPP>();
    return b < r ? (u32)b : r;
}
}  // namespace

int gn_tpp(int requested) {
    switch (requested) {
        case 1: case 4: case 8: case 32: return requested;
        default: return kDefaultTpp;
    }
}

// One wave of resident blocks; each group of lanes strides over the source points.
u32 gn_grid(u32 n_upper, int tpp) {
    switch (gn_tpp(tpp)) {
        case 4: return grid_for<4>(n_upper);
        case 8: return grid_for<8>(n_upper);
        case 32: return grid_for<32>(n_upper);
        default: return grid_for<1>(n_upper);
    }
}

// Partials for the largest grid any lanes-per-point setting can launch (32 lanes per point).
u32 gn_max_blocks(u32 n_upper) { return (u32)(gn_partials_doubles(n_upper) / NPART); }

size_t gn_partials_doubles(u32 n_upper) {
    u64 b = ((u64)n_upper * 32 + GN_THREADS - 1) / GN_THREADS;
    if (b == 0) b = 1;
    return (size_t)(b < kMaxGnBlocks ? b : kMaxGnBlocks) * NPART;
}

cudaError_t gn_begin(RegState* st, const double init[16], const u32* n_src, cudaStream_t s) {
    Pose16 p;
    for (int j = 0; j < 16; ++j) p.m[j] = init[j];
    FAR_LAUNCH(k_gn_begin, 1, 1, 0, s, st, p, n_src);
    return cudaGetLastError();
}

cudaError_t gn_linearise(const GnArgs& a, u32 n_upper, cudaStream_t s, u32* nblocks) {
    const u32 g = gn_grid(n_upper, a.tpp);
    const bool prec = a.map.tv > 0;
    switch (gn_tpp(a.tpp)) {
        case 4: if (prec) FAR_LAUNCH_PDL((k_gn_lin<4, true>), g, GN_THREADS, 0, s, a);
                else FAR_LAUNCH_PDL((k_gn_lin<4, false>), g, GN_THREADS, 0, s, a);
                break;
        case 8: if (prec) FAR_LAUNCH_PDL((k_gn_lin<8, true>), g, GN_THREADS, 0, s, a);
                else FAR_LAUNCH_PDL((k_gn_lin<8, false>), g, GN_THREADS, 0, s, a);
                break;
        case 32: if (prec) FAR_LAUNCH_PDL((k_gn_lin<32, true>), g, GN_THREADS, 0, s, a);
                 else FAR_LAUNCH_PDL((k_gn_lin<32, false>), g, GN_THREADS, 0, s, a);
                 break;
        default: if (prec) FAR_LAUNCH_PDL((k_gn_lin<1, true>), g, GN_THREADS, 0, s, a);
                 else FAR_LAUNCH_PDL((k_gn_lin<1, false>), g, GN_THREADS, 0, s, a);
                 break;
    }
    *nblocks = g;
    return cudaGetLastError();
}

cudaError_t gn_solve(const GnArgs& a, u32 nblocks, cudaStream_t s) {
    FAR_LAUNCH_PDL(k_gn_solve, NPART, 32, 0, s, a, nblocks);
    return cudaGetLastError();
}


cudaError_t gn_batch_begin(const BatchProblem* probs, u32 nprob, const double* init, cudaStream_t s) {
    FAR_LAUNCH(k_gn_begin_batch, (nprob + 127) / 128, 128, 0, s, probs, nprob, init);
    return cudaGetLastError();
}

cudaError_t gn_batch_iteration(const BatchProblem* probs, const u32* block_prob, u32 total_blocks, u32 nprob,
                               int tpp, bool prec, cudaStream_t s) {
    switch (gn_tpp(tpp)) {
        case 4: if (prec) FAR_LAUNCH_PDL((k_gn_lin_batch<4, true>), total_blocks, GN_THREADS, 0, s, probs, block_prob);
                else FAR_LAUNCH_PDL((k_gn_lin_batch<4, false>), total_blocks, GN_THREADS, 0, s, probs, block_prob);
                break;
        case 8: if (prec) FAR_LAUNCH_PDL((k_gn_lin_batch<8, true>), total_blocks, GN_THREADS, 0, s, probs, block_prob);
                else FAR_LAUNCH_PDL((k_gn_lin_batch<8, false>), total_blocks, GN_THREADS, 0, s, probs, block_prob);
                break;
        case 32: if (prec) FAR_LAUNCH_PDL((k_gn_lin_batch<32, true>), total_blocks, GN_THREADS, 0, s, probs, block_prob);
                 else FAR_LAUNCH_PDL((k_gn_lin_batch<32, false>), total_blocks, GN_THREADS, 0, s, probs, block_prob);
                 break;
        default: if (prec) FAR_LAUNCH_PDL((k_gn_lin_batch<1, true>), total_blocks, GN_THREADS, 0, s, probs, block_prob);
                 else FAR_LAUNCH_PDL((k_gn_lin_batch<1, false>), total_blocks, GN_THREADS, 0, s, probs, block_prob);
                 break;
    }
    FAR_LAUNCH_PDL(k_gn_solve_batch, dim3(NPART, nprob), 32, 0, s, probs);
    return cudaGetLastError();
}

cudaError_t gn_batch_gather(const BatchProblem* probs, u32 nprob, RegState* out, cudaStream_t s) {
    FAR_LAUNCH(k_gather_states, nprob, 128, 0, s, probs, nprob, out);
    return cudaGetLastError();
}

u32 gn_threads_per_block() { return GN_THREADS; }

cudaError_t gn_iteration(const GnArgs& a, u32 n_upper, cudaStream_t s) {
    u32 nb = 0;
    cudaError_t e = gn_linearise(a, n_upper, s, &nb);
    if (e != cudaSuccess) return e;
    return gn_solve(a, nb, s);
}

namespace {
void* lin_dev_fn(int tpp, bool prec) {
    switch (gn_tpp(tpp)) {
        case 4: return prec ? (void*)k_gn_lin_dev<4, true> : (void*)k_gn_lin_dev<4, false>;
        case 8: return prec ? (void*)k_gn_lin_dev<8, true> : (void*)k_gn_lin_dev<8, false>;
        case 32: return prec ? (void*)k_gn_lin_dev<32, true> : (void*)k_gn_lin_dev<32, false>;
        default: return prec ? (void*)k_gn_lin_dev<1, true> : (void*)k_gn_lin_dev<1, false>;
    }
}
}  // namespace

cudaError_t gn_graph_build(const GnArgs* d_args, u32 n_upper, int tpp, bool prec, GnGraph* out) {
    u32 grid = gn_grid(n_upper, tpp);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaGraphCreate(&graph, 0);
    if (e != cudaSuccess) return e;
    cudaGraphConditionalHandle loop;
    e = cudaGraphConditionalHandleCreate(&loop, graph, 1u, cudaGraphCondAssignDefault);
    cudaGraphNodeParams cp = {};
    cudaGraphNode_t cnode = nullptr;
    if (e == cudaSuccess) {
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = loop;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        e = cudaGraphAddNode(&cnode, graph, nullptr, nullptr, 0, &cp);
    }
    cudaGraphNode_t lin = nullptr, solve = nullptr;
    if (e == cudaSuccess) {
        cudaGraph_t body = cp.conditional.phGraph_out[0];
        const GnArgs* ap = d_args;
        void* largs[] = {(void*)&ap};
        cudaKernelNodeParams lp = {};
        lp.func = lin_dev_fn(tpp, prec);
        lp.gridDim = dim3(grid);
        lp.blockDim = dim3(GN_THREADS);
        lp.kernelParams = largs;
        e = cudaGraphAddKernelNode(&lin, body, nullptr, 0, &lp);
        void* sargs[] = {(void*)&ap, (void*)&grid, (void*)&loop};
        // programmatic edge: the solve launches while the linearisation runs and waits for it
        // in pdl_wait(), as the explicit chain does
        cudaGraphNodeParams sp = {};
        sp.type = cudaGraphNodeTypeKernel;
        sp.kernel.func = (void*)k_gn_solve_dev;
        sp.kernel.gridDim = dim3(NPART);
        sp.kernel.blockDim = dim3(32);
        sp.kernel.kernelParams = sargs;
        cudaGraphEdgeData ed = {};
        ed.from_port = cudaGraphKernelNodePortProgrammatic;
        ed.type = cudaGraphDependencyTypeProgrammatic;
        if (e == cudaSuccess) e = cudaGraphAddNode(&solve, body, &lin, &ed, 1, &sp);
    }
    cudaGraphExec_t exec = nullptr;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return e;
    out->exec = exec;
    out->grid = grid;
    out->tpp = gn_tpp(tpp);
    out->prec = prec;
    return cudaSuccess;
}

void gn_graph_destroy(GnGraph* g) {
    if (g->exec) cudaGraphExecDestroy(g->exec);
    g->exec = nullptr;
}

}  // namespace far
