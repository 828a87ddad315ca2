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

// k nearest (k <= K) of q; arrays sorted ascending by (d2, id). Returns found (<= k).
template <int K>
__device__ __forceinline__ int knn27(const MapView& m, u32 max_probe, float qx, float qy, float qz, int k,
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
    for (int dx = -1; dx <= 1; ++dx) {
        const int nx = kx + dx;
        if (!key_in_range(nx)) continue;
        for (int dy = -1; dy <= 1; ++dy) {
            const int ny = ky + dy;
            if (!key_in_range(ny)) continue;
            for (int dz = -1; dz <= 1; ++dz) {
                const int nz = kz + dz;
                if (!key_in_range(nz)) continue;
                u32 bucket, count;
                if (!find_slot(m.slots, m.mask, max_probe, nx, ny, nz, bucket, count)) continue;
                const u32 base = bucket * m.nmax;
                for (u32 j = 0; j < count; ++j) {
                    const float4 p = __ldg(m.pts + base + j);
                    const float d2 = dist2_rn(qx, qy, qz, p.x, p.y, p.z);
                    const u32 id = __float_as_uint(p.w);
                    ++found;
                    if (!better(d2, id, bd[k - 1], bid[k - 1])) continue;
                    bool placed = false;
#pragma unroll
                    for (int s = K - 1; s >= 1; --s) {
                        if (s < k && !placed) {
                            if (better(d2, id, bd[s - 1], bid[s - 1])) {
                                bd[s] = bd[s - 1];
                                bid[s] = bid[s - 1];
                                bpos[s] = bpos[s - 1];
                            } else {
                                bd[s] = d2;
                                bid[s] = id;
                                bpos[s] = base + j;
                                placed = true;
                            }
                        }
                    }
                    if (!placed) {
                        bd[0] = d2;
                        bid[0] = id;
                        bpos[0] = base + j;
                    }
                }
            }
        }
    }
    return found < k ? found : k;
}

// Nearest map point of q over the 27 voxels. Returns false when there is none.
__device__ __forceinline__ bool nearest27(const MapView& m, u32 max_probe, float qx, float qy, float qz,
                                          float& best_d2, u32& best_id, u32& best_pos) {
    best_d2 = F_INF;
    best_id = NO_ID;
    best_pos = 0;
    int kx, ky, kz;
    if (!voxel_key3(qx, qy, qz, m.inv_v, kx, ky, kz)) return false;
    bool any = false;
    for (int dx = -1; dx <= 1; ++dx) {
        const int nx = kx + dx;
        if (!key_in_range(nx)) continue;
        for (int dy = -1; dy <= 1; ++dy) {
            const int ny = ky + dy;
            if (!key_in_range(ny)) continue;
            for (int dz = -1; dz <= 1; ++dz) {
                const int nz = kz + dz;
                if (!key_in_range(nz)) continue;
                u32 bucket, count;
                if (!find_slot(m.slots, m.mask, max_probe, nx, ny, nz, bucket, count)) continue;
                const u32 base = bucket * m.nmax;
                for (u32 j = 0; j < count; ++j) {
                    const float4 p = __ldg(m.pts + base + j);
                    const float d2 = dist2_rn(qx, qy, qz, p.x, p.y, p.z);
                    const u32 id = __float_as_uint(p.w);
                    if (!any || better(d2, id, best_d2, best_id)) {
                        best_d2 = d2;
                        best_id = id;
                        best_pos = base + j;
                        any = true;
                    }
                }
            }
        }
    }
    return any;
}

// Eq. 1 from k neighbour positions: Sigma-hat (1/k, about the neighbour mean),
// C = Sigma-hat + 1e-3 I, Sigma = ||C^-1||_F C (equal to (C^-1 / ||C^-1||_F)^-1).
// Coordinates are taken relative to the query point for FP32 accuracy.
template <int K>
__device__ __forceinline__ void covariance_from_neighbours(const float4* __restrict__ pts, const u32 (&bpos)[K],
                                                           int k, float qx, float qy, float qz, float4& c0,
                                                           float4& c1) {
    float mx = 0.f, my = 0.f, mz = 0.f;
    float rx[K], ry[K], rz[K];
#pragma unroll
    for (int j = 0; j < K; ++j) {
        if (j < k) {
            const float4 p = __ldg(pts + bpos[j]);
            rx[j] = p.x - qx;
            ry[j] = p.y - qy;
            rz[j] = p.z - qz;
            mx += rx[j];
            my += ry[j];
            mz += rz[j];
        }
    }
    const float ik = 1.0f / (float)k;
    mx *= ik;
    my *= ik;
    mz *= ik;
    float sxx = 0, sxy = 0, sxz = 0, syy = 0, syz = 0, szz = 0;
#pragma unroll
    for (int j = 0; j < K; ++j) {
        if (j < k) {
            const float dx = rx[j] - mx, dy = ry[j] - my, dz = rz[j] - mz;
            sxx = fmaf(dx, dx, sxx);
            sxy = fmaf(dx, dy, sxy);
            sxz = fmaf(dx, dz, sxz);
            syy = fmaf(dy, dy, syy);
            syz = fmaf(dy, dz, syz);
            szz = fmaf(dz, dz, szz);
        }
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
