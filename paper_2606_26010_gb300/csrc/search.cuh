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

// Merge the points of voxel (nx, ny, nz) into the sorted K best of q.
template <int K>
__device__ __forceinline__ void knn_scan_voxel(const MapView& m, u32 max_probe, int nx, int ny, int nz, float qx,
                                               float qy, float qz, int& found, float (&bd)[K], u32 (&bid)[K],
                                               u32 (&bpos)[K]) {
    u32 bucket, count;
    if (!find_slot(m.slots, m.mask, max_probe, nx, ny, nz, bucket, count)) return;
    const u32 base = bucket * m.nmax;
    for (u32 j = 0; j < count; ++j) {
        const float4 p = __ldg(m.pts + base + j);
        const float d2 = dist2_rn(qx, qy, qz, p.x, p.y, p.z);
        const u32 id = __float_as_uint(p.w);
        ++found;
        if (!better(d2, id, bd[K - 1], bid[K - 1])) continue;
        // sorted insert: the candidate bubbles up past every worse entry
        float cd = d2;
        u32 ci = id, cp = base + j;
#pragma unroll
        for (int s = 0; s < K; ++s) {
            const bool sw = better(cd, ci, bd[s], bid[s]);
            const float td = bd[s];
            const u32 ti = bid[s], tp = bpos[s];
            bd[s] = sw ? cd : td;
            bid[s] = sw ? ci : ti;
            bpos[s] = sw ? cp : tp;
            cd = sw ? td : cd;
            ci = sw ? ti : ci;
            cp = sw ? tp : cp;
        }
    }
}

// Merge the points of voxel (nx, ny, nz) into the nearest of q, kept as the packed key
// (d2 bits << 32 | id): for d2 >= 0 the integer order is the (d2, id) order. Points are
// loaded four at a time so that several loads are in flight.
__device__ __forceinline__ void nn_scan_voxel(const MapView& m, u32 max_probe, int nx, int ny, int nz, float qx,
                                              float qy, float qz, unsigned long long& best_key, u32& best_pos) {
    u32 bucket, count;
    if (!find_slot(m.slots, m.mask, max_probe, nx, ny, nz, bucket, count)) return;
    const u32 base = bucket * m.nmax;
    for (u32 j0 = 0; j0 < count; j0 += 4) {
        float4 c[4];
#pragma unroll
        for (int u = 0; u < 4; ++u)
            c[u] = (j0 + u < count) ? __ldg(m.pts + base + j0 + u) : make_float4(0.f, 0.f, 0.f, 0.f);
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
}

__device__ __forceinline__ float nn_bound(unsigned long long best_key, float limit2) {
    const float b = best_key == ~0ull ? F_INF : __uint_as_float((u32)(best_key >> 32));
    return fminf(b, limit2);
}

// K nearest of q (K is the exact k: a run-time k would push the arrays to local
// memory); arrays sorted ascending by (d2, id). Returns the number found (<= K).
template <int K>
__device__ __forceinline__ int knn27(const MapView& m, u32 max_probe, float qx, float qy, float qz,
                                     float (&bd)[K], u32 (&bid)[K], u32 (&bpos)[K]) {
#pragma unroll
    for (int j = 0; j < K; ++j) {
        bd[j] = F_INF;
        bid[j] = NO_ID;
        bpos[j] = 0;
    }
    int kx, ky, kz;
    if (!voxel_key3(qx, qy, qz, m.inv_v, kx, ky, kz)) return 0;
    int found = 0;
    const FaceDist fd = face_distances(qx, qy, qz, kx, ky, kz, m.v);
    // own voxel first, then only the neighbours on the sides within reach of the k-th distance
    knn_scan_voxel<K>(m, max_probe, kx, ky, kz, qx, qy, qz, found, bd, bid, bpos);
    const float b0 = (found >= K) ? bd[K - 1] : F_INF;
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
                if (found >= K && box_lb2(fd, dx, dy, dz) > bd[K - 1]) continue;
                knn_scan_voxel<K>(m, max_probe, kx + dx, ky + dy, kz + dz, qx, qy, qz, found, bd, bid, bpos);
            }
        }
    }
    return found < K ? found : K;
}

// Nearest map point of q over the 27 voxels (smallest (d^2, id)). Voxels whose box
// distance exceeds the best so far, or limit2, are skipped: with limit2 = tau^2 a
// nearest point beyond tau is not reported, which is the rejection rule anyway.
// Returns false when no candidate was found.
__device__ __forceinline__ bool nearest27(const MapView& m, u32 max_probe, float qx, float qy, float qz,
                                          float limit2, float& best_d2, u32& best_id, u32& best_pos) {
    best_d2 = F_INF;
    best_id = NO_ID;
    best_pos = 0;
    int kx, ky, kz;
    if (!voxel_key3(qx, qy, qz, m.inv_v, kx, ky, kz)) return false;
    const FaceDist fd = face_distances(qx, qy, qz, kx, ky, kz, m.v);
    unsigned long long best_key = ~0ull;
    // own voxel first, then only the neighbours on the sides within reach of the bound
    nn_scan_voxel(m, max_probe, kx, ky, kz, qx, qy, qz, best_key, best_pos);
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
                nn_scan_voxel(m, max_probe, kx + dx, ky + dy, kz + dz, qx, qy, qz, best_key, best_pos);
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

// Eq. 1 from k neighbour positions: Sigma-hat (1/k, about the neighbour mean),
// C = Sigma-hat + 1e-3 I, Sigma = ||C^-1||_F C (equal to (C^-1 / ||C^-1||_F)^-1).
// Coordinates are taken relative to the query point for FP32 accuracy.
template <int K>
__device__ __forceinline__ void covariance_from_neighbours(const float4* __restrict__ pts, const u32 (&bpos)[K],
                                                           float qx, float qy, float qz, float4& c0, float4& c1) {
    float mx = 0.f, my = 0.f, mz = 0.f;
    float rx[K], ry[K], rz[K];
#pragma unroll
    for (int j = 0; j < K; ++j) {
        const float4 p = __ldg(pts + bpos[j]);
        rx[j] = p.x - qx;
        ry[j] = p.y - qy;
        rz[j] = p.z - qz;
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
    const float a = fmaf(sxx, ik, 1e-3f), b = sxy * ik, c = sxz * ik;
    const float d = fmaf(syy, ik, 1e-3f), e = syz * ik, f = fmaf(szz, ik, 1e-3f);
    // adjugate of the symmetric C
    const float A00 = d * f - e * e, A01 = c * e - b * f, A02 = b * e - c * d;
    const float A11 = a * f - c * c, A12 = b * c - a * e, A22 = a * d - b * b;
    const float det = a * A00 + b * A01 + c * A02;
    const float fro2 = A00 * A00 + A11 * A11 + A22 * A22 + 2.f * (A01 * A01 + A02 * A02 + A12 * A12);
    const float s = sqrtf(fro2) / fabsf(det);  // ||C^-1||_F
    c0 = make_float4(a * s, b * s, c * s, d * s);
    c1 = make_float4(e * s, f * s, 1.0f, 0.0f);
}

}  // namespace far
