// 27-voxel neighbour search and Eq. 1 covariance (device functions).
//
// FAR-LIO Sec. III-A.2: a query searches the voxel containing it and the 26
// around it. Candidates are ordered by FP32 d^2 (defined expression) and then
// by point id, so the k-NN and 1-NN sets have one exact answer.
#pragma once
#include <math_constants.h>
#include "far_internal.cuh"

namespace far {

#define F_INF CUDART_INF_F

// The 27 neighbour offsets ordered own voxel, 6 faces, 12 edges, 8 corners, so that a
// close candidate is usually found first and farther voxels can be skipped.
__constant__ signed char c_nb_order[27][3] = {
    {0, 0, 0},
    {-1, 0, 0}, {1, 0, 0}, {0, -1, 0}, {0, 1, 0}, {0, 0, -1}, {0, 0, 1},
    {-1, -1, 0}, {-1, 1, 0}, {1, -1, 0}, {1, 1, 0}, {-1, 0, -1}, {-1, 0, 1},
    {1, 0, -1}, {1, 0, 1}, {0, -1, -1}, {0, -1, 1}, {0, 1, -1}, {0, 1, 1},
    {-1, -1, -1}, {-1, -1, 1}, {-1, 1, -1}, {-1, 1, 1}, {1, -1, -1}, {1, -1, 1}, {1, 1, -1}, {1, 1, 1}};

// Distances from q to the lower and upper faces of its voxel along each axis, reduced
// by a margin that covers the rounding of the key (a point of voxel k + 1 satisfies
// x >= (k + 1) v (1 - 3 eps)) and of the FP32 distance expression, clamped at 0.
// A neighbour voxel whose squared box distance exceeds the current best d^2 cannot
// hold a point with a d^2 at or below it, so skipping it leaves the (d^2, id) minimum unchanged.
struct FaceDist {
    float lo[3], hi[3];
};

__device__ __forceinline__ FaceDist face_distances(float qx, float qy, float qz, int kx, int ky, int kz, float v) {
    const float margin = 1e-6f * (fabsf(qx) + fabsf(qy) + fabsf(qz)) + 1e-5f;
    FaceDist f;
    const float q[3] = {qx, qy, qz};
    const int k[3] = {kx, ky, kz};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        f.lo[a] = fmaxf(q[a] - (float)k[a] * v - margin, 0.0f);
        f.hi[a] = fmaxf((float)(k[a] + 1) * v - q[a] - margin, 0.0f);
    }
    return f;
}

__device__ __forceinline__ float box_lb2(const FaceDist& f, int dx, int dy, int dz) {
    const float ax = dx < 0 ? f.lo[0] : (dx > 0 ? f.hi[0] : 0.0f);
    const float ay = dy < 0 ? f.lo[1] : (dy > 0 ? f.hi[1] : 0.0f);
    const float az = dz < 0 ? f.lo[2] : (dz > 0 ? f.hi[2] : 0.0f);
    return ax * ax + ay * ay + az * az;
}

// A query in search coordinates. Plain maps search in world coordinates. In the precision
// variant the search runs in the frame of a tile F (coordinates relative to its origin): a
// map point of tile T_p enters as fp32(p + 50 (T_p - F)), one FP32 addition of an exact
// multiple of 50. k is the centre voxel (global key), lk the centre relative to the frame
// origin (face distances), ct / cin its tile relative to F and its index inside that tile.
template <bool PREC>
struct QFrame {
    float q[3];
    int k[3], lk[3];
    int ct[3], cin[3];
    int tv;
    // offset of neighbour voxel lk + d along axis a (0 for plain maps)
    __device__ __forceinline__ float off(int a, int d) const {
        if constexpr (!PREC) {
            return 0.0f;
        } else {
            const int c = cin[a] + d;
            const int t = ct[a] + (c < 0 ? -1 : (c >= tv ? 1 : 0));
            return TILE_M * (float)t;
        }
    }
};

// Query given in frame coordinates (world for plain maps; frame tile ftile otherwise):
// centre = K_F + floor(fp32(q * inv_v)).
template <bool PREC>
__device__ __forceinline__ bool make_qframe(const MapView& m, float qx, float qy, float qz, const int (&ftile)[3],
                                            QFrame<PREC>& f) {
    f.q[0] = qx;
    f.q[1] = qy;
    f.q[2] = qz;
    f.tv = m.tv;
#pragma unroll
    for (int a = 0; a < 3; ++a) f.k[a] = f.lk[a] = f.ct[a] = f.cin[a] = 0;
    if (!voxel_key3(qx, qy, qz, m.inv_v, f.lk[0], f.lk[1], f.lk[2])) return false;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if constexpr (PREC) {
            const long long k = (long long)f.lk[a] + (long long)ftile[a] * m.tv;
            if (k < -(long long)KEY_BIAS || k >= (long long)KEY_BIAS) return false;
            f.k[a] = (int)k;
            f.ct[a] = floor_div(f.lk[a], m.tv);
            f.cin[a] = f.lk[a] - f.ct[a] * m.tv;
        } else {
            f.k[a] = f.lk[a];
            f.ct[a] = 0;
            f.cin[a] = 0;
        }
    }
    return true;
}

// Query that is a map point: centre = its own voxel key, frame = that voxel's tile,
// coordinates = its stored (tile-relative) coordinates.
__device__ __forceinline__ void own_qframe(const MapView& m, float qx, float qy, float qz, int kx, int ky, int kz,
                                           QFrame<true>& f) {
    f.q[0] = qx;
    f.q[1] = qy;
    f.q[2] = qz;
    f.tv = m.tv;
    const int k[3] = {kx, ky, kz};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        f.k[a] = k[a];
        f.lk[a] = k[a] - floor_div(k[a], m.tv) * m.tv;
        f.ct[a] = 0;
        f.cin[a] = f.lk[a];
    }
}

// A k-NN list entry: the packed key (d2 bits << 32 | id), whose integer order is the (d2, id)
// order for d2 >= 0, and the candidate's position in the map's point array. An empty entry
// holds KNN_EMPTY (+inf, no id), which every candidate precedes.
constexpr unsigned long long KNN_EMPTY = (0x7F800000ull << 32) | 0xFFFFFFFFull;

__device__ __forceinline__ float knn_d2(unsigned long long key) { return __uint_as_float((u32)(key >> 32)); }

// Merge the points of voxel (nx, ny, nz) into the sorted K best of q.
template <int K, bool PREC = false>
__device__ __forceinline__ void knn_scan_voxel(const MapView& m, u32 max_probe, int nx, int ny, int nz, float qx,
                                               float qy, float qz, int& found, unsigned long long (&bk)[K],
                                               u32 (&bpos)[K], float ox = 0.f, float oy = 0.f, float oz = 0.f) {
    u32 bucket, count;
    if (!find_slot(m.slots, m.mask, max_probe, nx, ny, nz, bucket, count)) return;
    const u32 base = bucket * m.nmax;
    found += (int)count;
    // points are loaded four at a time so that several loads are in flight
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
            if (j0 + u >= count) continue;
            const float d2 = dist2_rn(qx, qy, qz, c[u].x, c[u].y, c[u].z);
            unsigned long long ck = ((unsigned long long)__float_as_uint(d2) << 32) | __float_as_uint(c[u].w);
            if (!(ck < bk[K - 1])) continue;
            // sorted insert: the candidate bubbles up past every worse entry
            u32 cp = base + j0 + u;
#pragma unroll
            for (int s2 = 0; s2 < K; ++s2) {
                const bool sw = ck < bk[s2];
                const unsigned long long tk = bk[s2];
                const u32 tp = bpos[s2];
                bk[s2] = sw ? ck : tk;
                bpos[s2] = sw ? cp : tp;
                ck = sw ? tk : ck;
                cp = sw ? tp : cp;
            }
        }
    }
}

// Merge the points of voxel (nx, ny, nz) into the nearest of q, kept as the packed key
// (d2 bits << 32 | id): for d2 >= 0 the integer order is the (d2, id) order. Points are
// loaded four at a time so that several loads are in flight.
template <bool PREC = false>
__device__ __forceinline__ bool nn_scan_voxel(const MapView& m, u32 max_probe, int nx, int ny, int nz, float qx,
                                              float qy, float qz, unsigned long long& best_key, u32& best_pos,
                                              float ox = 0.f, float oy = 0.f, float oz = 0.f) {
    u32 bucket, count;
    if (!find_slot(m.slots, m.mask, max_probe, nx, ny, nz, bucket, count)) return false;
    const u32 base = bucket * m.nmax;
    const unsigned long long before = best_key;
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
                }
            }
        }
    }
    return best_key != before;
}

__device__ __forceinline__ float nn_bound(unsigned long long best_key, float limit2) {
    const float b = best_key == ~0ull ? F_INF : __uint_as_float((u32)(best_key >> 32));
    return fminf(b, limit2);
}

template <int K>
__device__ __forceinline__ void knn_init(unsigned long long (&bk)[K], u32 (&bpos)[K]) {
#pragma unroll
    for (int j = 0; j < K; ++j) {
        bk[j] = KNN_EMPTY;
        bpos[j] = 0;
    }
}

// The K best of two sorted lists (ascending keys, disjoint candidates) into the second: the K
// smallest of the union are min(a_i, b_{K-1-i}) (a bitonic sequence), which an odd-even
// transposition sort puts back in order. Registers only.
template <int K>
__device__ __forceinline__ void knn_merge(const unsigned long long (&ok)[K], const u32 (&op)[K],
                                          unsigned long long (&bk)[K], u32 (&bpos)[K]) {
#pragma unroll
    for (int i = 0; i < K; ++i) {
        const int j = K - 1 - i;
        if (ok[j] < bk[i]) {
            bk[i] = ok[j];
            bpos[i] = op[j];
        }
    }
#pragma unroll
    for (int pass = 0; pass < K; ++pass)
#pragma unroll
        for (int i = pass & 1; i + 1 < K; i += 2) {
            const bool sw = bk[i + 1] < bk[i];
            const unsigned long long k0 = bk[i], k1 = bk[i + 1];
            const u32 p0 = bpos[i], p1 = bpos[i + 1];
            bk[i] = sw ? k1 : k0;
            bk[i + 1] = sw ? k0 : k1;
            bpos[i] = sw ? p1 : p0;
            bpos[i + 1] = sw ? p0 : p1;
        }
}

// K-th smallest distance of the union of the group's TPP sorted lists (distances only, every
// lane of the group ends with it): a butterfly over the lanes keeps the K smallest of each pair,
// min(a_i, b_{K-1-i}), sorted again by an odd-even transposition sort.
template <int K, int TPP>
__device__ __forceinline__ float group_union_kth(const unsigned long long (&bk)[K]) {
    float c[K];
#pragma unroll
    for (int i = 0; i < K; ++i) c[i] = knn_d2(bk[i]);
#pragma unroll
    for (int o = 1; o < TPP; o <<= 1) {
        float p[K];
#pragma unroll
        for (int i = 0; i < K; ++i) p[i] = __shfl_xor_sync(0xffffffffu, c[i], o);
#pragma unroll
        for (int i = 0; i < K; ++i) c[i] = fminf(c[i], p[K - 1 - i]);
#pragma unroll
        for (int pass = 0; pass < K; ++pass)
#pragma unroll
            for (int i = pass & 1; i + 1 < K; i += 2) {
                const float lo = fminf(c[i], c[i + 1]), hi = fmaxf(c[i], c[i + 1]);
                c[i] = lo;
                c[i + 1] = hi;
            }
    }
    return c[K - 1];
}

// K nearest of the query searched by a group of TPP consecutive lanes. Lane 0 first scans the
// query's own voxel and lanes 1 .. TPP - 1 the faces nearest to the query, each into its own
// sorted K best; the group then
// takes the K-th distance of the union of the lanes' lists as its bound (group_union_kth; the K
// best of all 27 voxels are at least that close), lists the remaining voxels whose box distance
// does not exceed it
// (compacted into `list`, at least 27 - TPP bytes of the group's own memory) and scans them
// TPP at a time, re-testing each against the bound of the round before. The lanes' lists are
// then merged pairwise (knn_merge), so every lane of the group ends with the K best of the union in
// (d2, id) order (the lanes saw disjoint voxels). Returns the number of candidates the group
// saw, capped at K. Every lane of the warp must call this.
template <int K, int TPP, bool PREC>
__device__ __forceinline__ int group_knn(const MapView& m, u32 max_probe, const QFrame<PREC>& f, bool keyed,
                                         int sl, unsigned char* list, unsigned long long (&bk)[K],
                                         u32 (&bpos)[K]) {
    knn_init<K>(bk, bpos);
    int found = 0;
    const FaceDist fd = face_distances(f.q[0], f.q[1], f.q[2], f.lk[0], f.lk[1], f.lk[2], m.v);
    auto scan = [&](int v) {
        const int dx = c_nb_order[v][0], dy = c_nb_order[v][1], dz = c_nb_order[v][2];
        const int nx = f.k[0] + dx, ny = f.k[1] + dy, nz = f.k[2] + dz;
        if (key_in_range(nx) && key_in_range(ny) && key_in_range(nz))
            knn_scan_voxel<K, PREC>(m, max_probe, nx, ny, nz, f.q[0], f.q[1], f.q[2], found, bk, bpos,
                                    f.off(0, dx), f.off(1, dy), f.off(2, dz));
    };
    auto group_bound = [&]() {
        float kth = knn_d2(bk[K - 1]);
#pragma unroll
        for (int o = TPP / 2; o > 0; o >>= 1) kth = fminf(kth, __shfl_xor_sync(0xffffffffu, kth, o));
        return kth;
    };
    static_assert(TPP >= 2 && TPP <= 7, "the first round takes the own voxel and TPP - 1 faces");
    // first round: lane 0 the own voxel, lanes 1 .. TPP - 1 the faces nearest to the query (face
    // j = c_nb_order entry 1 + j, at distance lo/hi of its axis; ties to the lower entry), so that
    // the first bound is as tight as the first round allows
    const float fdist[6] = {fd.lo[0], fd.hi[0], fd.lo[1], fd.hi[1], fd.lo[2], fd.hi[2]};
    u32 chosen = 0;   // bit v: entry v scanned in the first round
    int my_first = 0;
#pragma unroll
    for (int j = 0; j < 6; ++j) {
        int rank = 0;
#pragma unroll
        for (int i = 0; i < 6; ++i) rank += (fdist[i] < fdist[j] || (fdist[i] == fdist[j] && i < j)) ? 1 : 0;
        if (rank < TPP - 1) chosen |= 1u << (1 + j);
        if (rank == sl - 1) my_first = 1 + j;
    }
    if (keyed) scan(my_first);
    // the K best of the union are at least as close as the union's K-th distance, which is finite
    // once the first round's voxels hold K points together (sparse regions)
    float bound = group_union_kth<K, TPP>(bk);
    // survivors of the other voxels under the group's bound, compacted in voxel order
    u32 mine = 0;
    int k = 0;
    for (int v = 1 + sl; v < 27; v += TPP, ++k)
        if (keyed && !((chosen >> v) & 1u) &&
            !(box_lb2(fd, c_nb_order[v][0], c_nb_order[v][1], c_nb_order[v][2]) > bound))
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
    for (int v = 1 + sl; v < 27; v += TPP, ++k)
        if (mine & (1u << k)) list[pre++] = (unsigned char)v;
    __syncwarp();
    const int rounds = (__reduce_max_sync(0xffffffffu, (u32)total) + TPP - 1) / TPP;   // warp-uniform
    for (int r = 0; r < rounds; ++r) {
        const int s2 = r * TPP + sl;
        if (s2 < total) {
            const int v = list[s2];
            if (!(box_lb2(fd, c_nb_order[v][0], c_nb_order[v][1], c_nb_order[v][2]) > bound)) scan(v);
        }
        bound = fminf(bound, group_bound());
    }
    __syncwarp();
#pragma unroll
    for (int o = TPP / 2; o > 0; o >>= 1) {
        found += __shfl_xor_sync(0xffffffffu, found, o);
        unsigned long long ok[K];
        u32 op[K];
#pragma unroll
        for (int j = 0; j < K; ++j) {
            ok[j] = __shfl_xor_sync(0xffffffffu, bk[j], o);
            op[j] = __shfl_xor_sync(0xffffffffu, bpos[j], o);
        }
        knn_merge<K>(ok, op, bk, bpos);
    }
    return found < K ? found : K;
}

// Nearest map point of the query over the 27 voxels (smallest (d^2, id)). Voxels whose box
// distance exceeds the best so far, or limit2, are skipped: with limit2 = tau^2 a nearest
// point beyond tau is not reported, which is the rejection rule anyway. best_v is the
// index (dx + 1) * 9 + (dy + 1) * 3 + (dz + 1) of the voxel holding the winner.
// Returns false when no candidate was found.
template <bool PREC>
__device__ __forceinline__ bool nearest27q(const MapView& m, u32 max_probe, const QFrame<PREC>& f, float limit2,
                                           float& best_d2, u32& best_id, u32& best_pos, int& best_v) {
    best_d2 = F_INF;
    best_id = NO_ID;
    best_pos = 0;
    best_v = 13;
    const float qx = f.q[0], qy = f.q[1], qz = f.q[2];
    const int kx = f.k[0], ky = f.k[1], kz = f.k[2];
    const FaceDist fd = face_distances(qx, qy, qz, f.lk[0], f.lk[1], f.lk[2], m.v);
    unsigned long long best_key = ~0ull;
    // own voxel first, then only the neighbours on the sides within reach of the bound
    nn_scan_voxel<PREC>(m, max_probe, kx, ky, kz, qx, qy, qz, best_key, best_pos, f.off(0, 0), f.off(1, 0),
                        f.off(2, 0));
    const float b0 = nn_bound(best_key, limit2);
    bool reach[3][2];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        reach[a][0] = fd.lo[a] * fd.lo[a] <= b0;
        reach[a][1] = fd.hi[a] * fd.hi[a] <= b0;
    }
    for (int dx = -1; dx <= 1; ++dx) {
        if ((dx < 0 && !reach[0][0]) || (dx > 0 && !reach[0][1]) || !key_in_range(kx + dx)) continue;
        for (int dy = -1; dy <= 1; ++dy) {
            if ((dy < 0 && !reach[1][0]) || (dy > 0 && !reach[1][1]) || !key_in_range(ky + dy)) continue;
            for (int dz = -1; dz <= 1; ++dz) {
                if ((dz < 0 && !reach[2][0]) || (dz > 0 && !reach[2][1]) || !key_in_range(kz + dz)) continue;
                if (dx == 0 && dy == 0 && dz == 0) continue;
                if (box_lb2(fd, dx, dy, dz) > nn_bound(best_key, limit2)) continue;
                if (nn_scan_voxel<PREC>(m, max_probe, kx + dx, ky + dy, kz + dz, qx, qy, qz, best_key, best_pos,
                                        f.off(0, dx), f.off(1, dy), f.off(2, dz)))
                    best_v = (dx + 1) * 9 + (dy + 1) * 3 + (dz + 1);
            }
        }
    }
    if (best_key == ~0ull) {
        best_d2 = F_INF;
        return false;
    }
    best_d2 = __uint_as_float((u32)(best_key >> 32));
    best_id = (u32)best_key;
    return true;
}

// Nearest map point of a world-coordinate query of a plain map.
__device__ __forceinline__ bool nearest27(const MapView& m, u32 max_probe, float qx, float qy, float qz,
                                          float limit2, float& best_d2, u32& best_id, u32& best_pos) {
    best_d2 = F_INF;
    best_id = NO_ID;
    best_pos = 0;
    QFrame<false> f;
    const int zero[3] = {0, 0, 0};
    if (!make_qframe<false>(m, qx, qy, qz, zero, f)) return false;
    int bv;
    return nearest27q<false>(m, max_probe, f, limit2, best_d2, best_id, best_pos, bv);
}

// Eq. 1 from the K neighbours' offsets r_j = p_j - q from the query point (FP32 accuracy):
// Sigma-hat (1/K, about the neighbour mean), C = Sigma-hat + 1e-3 I, Sigma = ||C^-1||_F C
// (equal to (C^-1 / ||C^-1||_F)^-1).
template <int K>
__device__ __forceinline__ void covariance_eq1_rel(const float (&rx)[K], const float (&ry)[K], const float (&rz)[K],
                                                   float (&c)[6]) {
    float mx = 0.f, my = 0.f, mz = 0.f;
#pragma unroll
    for (int j = 0; j < K; ++j) {
        mx += rx[j];
        my += ry[j];
        mz += rz[j];
    }
    const float ik = 1.0f / (float)K;
    mx *= ik;
    my *= ik;
    mz *= ik;
    float sxx = 0, sxy = 0, sxz = 0, syy = 0, syz = 0, szz = 0;
#pragma unroll
    for (int j = 0; j < K; ++j) {
        const float dx = rx[j] - mx, dy = ry[j] - my, dz = rz[j] - mz;
        sxx = fmaf(dx, dx, sxx);
        sxy = fmaf(dx, dy, sxy);
        sxz = fmaf(dx, dz, sxz);
        syy = fmaf(dy, dy, syy);
        syz = fmaf(dy, dz, syz);
        szz = fmaf(dz, dz, szz);
    }
    const float a = fmaf(sxx, ik, 1e-3f), b = sxy * ik, c_ = sxz * ik;
    const float d = fmaf(syy, ik, 1e-3f), e = syz * ik, f = fmaf(szz, ik, 1e-3f);
    // adjugate of the symmetric C
    const float A00 = d * f - e * e, A01 = c_ * e - b * f, A02 = b * e - c_ * d;
    const float A11 = a * f - c_ * c_, A12 = b * c_ - a * e, A22 = a * d - b * b;
    const float det = a * A00 + b * A01 + c_ * A02;
    const float fro2 = A00 * A00 + A11 * A11 + A22 * A22 + 2.f * (A01 * A01 + A02 * A02 + A12 * A12);
    const float s = sqrtf(fro2) / fabsf(det);  // ||C^-1||_F
    c[0] = a * s;
    c[1] = b * s;
    c[2] = c_ * s;
    c[3] = d * s;
    c[4] = e * s;
    c[5] = f * s;
}

// Eq. 1 from k neighbour positions read from the map: pts are the neighbours' stored
// coordinates; off_of(p, ...) gives the frame offset of a neighbour (zero for plain maps;
// see TileOffset).
template <int K, class Off>
__device__ __forceinline__ void covariance_from_neighbours_f(const float4* __restrict__ pts, const u32 (&bpos)[K],
                                                             float qx, float qy, float qz, const Off& off_of,
                                                             float (&c)[6]) {
    float rx[K], ry[K], rz[K];
#pragma unroll
    for (int j = 0; j < K; ++j) {
        const float4 p = __ldg(pts + bpos[j]);
        float ox, oy, oz;
        off_of(p, qx, qy, qz, ox, oy, oz);
        rx[j] = __fadd_rn(p.x, ox) - qx;
        ry[j] = __fadd_rn(p.y, oy) - qy;
        rz[j] = __fadd_rn(p.z, oz) - qz;
    }
    covariance_eq1_rel<K>(rx, ry, rz, c);
}

struct NoOffset {
    __device__ __forceinline__ void operator()(const float4&, float, float, float, float& x, float& y,
                                               float& z) const {
        x = y = z = 0.f;
    }
};

// Frame offset of a neighbour of the precision variant: the neighbour lies within two voxels
// of the query, while the candidate offsets differ by 50 m, so the multiple of 50 nearest to
// q - p is the one the search added.
struct TileOffset {
    __device__ __forceinline__ void operator()(const float4& p, float qx, float qy, float qz, float& x, float& y,
                                               float& z) const {
        x = TILE_M * rintf((qx - p.x) * (1.0f / TILE_M));
        y = TILE_M * rintf((qy - p.y) * (1.0f / TILE_M));
        z = TILE_M * rintf((qz - p.z) * (1.0f / TILE_M));
    }
};

template <int K>
__device__ __forceinline__ void covariance_from_neighbours(const float4* __restrict__ pts, const u32 (&bpos)[K],
                                                           float qx, float qy, float qz, float4& c0, float4& c1) {
    float c[6];
    covariance_from_neighbours_f<K>(pts, bpos, qx, qy, qz, NoOffset(), c);
    c0 = make_float4(c[0], c[1], c[2], c[3]);
    c1 = make_float4(c[4], c[5], 1.0f, 0.0f);
}

}  // namespace far
