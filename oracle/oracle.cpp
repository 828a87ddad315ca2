// Plain CPU oracle of the FAR-LIO scan-to-map registration loop (TEST INFRASTRUCTURE).
//
// This file is the slow, obviously correct reference that the CUDA library is
// checked against. Only the tests, the smoke check and the CPU-baseline leg of
// the benchmark may load it; the product path never does.
//
// It shares no code with the CUDA path. Arithmetic is FP64 except the voxel key
// and the candidate-distance expressions, which are defined in FP32 (round to
// nearest, no contraction: build with -ffp-contract=off) so that voxel keys,
// map contents and neighbour sets have one exact answer on both sides.
//
// Passages followed (FAR-LIO, Sec. III-A):
//   voxel hashmap, 27-voxel search ............ Sec. III-A.2 (cuVoxelMap)
//   v, N points per voxel, regular spacing .... Sec. III-A.2 (parameters)
//   covariance regularisation ................ Eq. 1
//   initial transform ......................... Eq. 2
//   residual / GICP objective / Cauchy ........ Eq. 3, Eq. 4, Eq. 5
//   sparsity-aware special case ............... Sec. III-A.2 (SA GICP)
//   iterative update, termination ............. Eq. 6 and the text after it
//   adaptive submap density, insert, eviction . Sec. III-A.3
// Readings where the paper is silent (key rounding, spacing rule, tie-break,
// Cauchy argument, linearisation, exp map, adaptive threshold, ASMD constants)
// are the ones listed in the design notes; each is restated where it is used.
//
// Precision variant (precision_mode = 1, the mixed-precision storage scheme):
// the method is the same; what changes is where rounding to FP32 happens. Map
// points keep their unrounded FP64 world position for all arithmetic; keys use
// the tile rule (50 m tiles, see tile_key); the FP32 decision expressions
// (spacing, candidate order) are evaluated on coordinates relative to a tile
// origin instead of the world origin; Gauss-Newton is linearised about an
// anchor (the tile corner of the initial position) instead of the world origin.
//
// Threads (CPU-baseline timing only): om_set_threads(n) splits the per-point loops
// (scan-local covariances, added-point covariances, linearisation) into n fixed
// contiguous chunks run on std::threads; the linearisation sums each chunk in order and
// adds the chunk sums in chunk order, so a run is deterministic for a given n, and n = 1
// is exactly the sequential code. Map inserts stay sequential (admission is ordered).
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <limits>
#include <thread>
#include <unordered_map>
#include <vector>

namespace {

int g_threads = 1;

// Run fn(chunk, begin, end) over [0, n) in g_threads fixed contiguous chunks (chunk c covers
// [c n / T, (c + 1) n / T)); one thread runs everything on the caller's thread.
template <class F>
void parallel_chunks(size_t n, int chunks, F fn) {
    if (chunks <= 1 || n < 2) {
        fn(0, (size_t)0, n);
        return;
    }
    std::vector<std::thread> pool;
    for (int c = 0; c < chunks; ++c) {
        const size_t b = n * (size_t)c / (size_t)chunks, e = n * (size_t)(c + 1) / (size_t)chunks;
        pool.emplace_back([&fn, c, b, e]() { fn(c, b, e); });
    }
    for (std::thread& t : pool) t.join();
}

// ------------------------------------------------------------------ voxel keys
// Key reading: k = floor(x * (1/v)) per axis, the product rounded to FP32, with
// 1/v rounded to FP32 once. Keys must lie in [-2^20, 2^20) per axis.
constexpr float kKeyLimit = 1048576.0f;

struct Key {
    int32_t x, y, z;
    bool operator==(const Key& o) const { return x == o.x && y == o.y && z == o.z; }
    bool operator<(const Key& o) const {
        if (x != o.x) return x < o.x;
        if (y != o.y) return y < o.y;
        return z < o.z;
    }
};
struct KeyHash {
    size_t operator()(const Key& k) const {
        uint64_t h = (uint64_t)(uint32_t)k.x * 0x9E3779B97F4A7C15ull;
        h ^= (uint64_t)(uint32_t)k.y * 0xC2B2AE3D27D4EB4Full + (h << 6) + (h >> 2);
        h ^= (uint64_t)(uint32_t)k.z * 0x165667B19E3779F9ull + (h << 6) + (h >> 2);
        return (size_t)h;
    }
};

bool voxel_key(const float p[3], float inv_v, Key* out) {
    int32_t k[3];
    for (int a = 0; a < 3; ++a) {
        float s = p[a] * inv_v;                   // one FP32 rounding
        if (!(s >= -kKeyLimit && s < kKeyLimit)) return false;  // also rejects NaN
        k[a] = (int32_t)std::floor(s);
    }
    *out = Key{k[0], k[1], k[2]};
    return true;
}

// Candidate distance reading: d^2 = ((dx*dx + dy*dy) + dz*dz), dx = qx - px, FP32.
float dist2_f32(const float a[3], const float b[3]) {
    float dx = a[0] - b[0];
    float dy = a[1] - b[1];
    float dz = a[2] - b[2];
    float sx = dx * dx;
    float sy = dy * dy;
    float sz = dz * dz;
    float s = sx + sy;
    return s + sz;
}

// ------------------------------------------------------------------ precision variant: 50 m tiles
// Tile reading (precision_mode = 1): the tile of a world coordinate x is
// T = floor(x / 50) (exact, see tile_floor), the tile-relative coordinate is
// x_t = fp32(x - 50 T), and the voxel key is T tv + clamp(floor(fp32(x_t * inv_v)), 0, tv - 1)
// with tv = 50 / v voxels per tile side (v must divide 50 m). The clamp keeps every key
// inside the tile of its point when x_t rounds to 50 or to a tiny negative value.
constexpr double kTile = 50.0;

// floor(x / 50) in exact arithmetic: the rounded quotient's floor, moved by one when 50 T
// (exact in FP64) shows it is off.
double tile_floor(double x) {
    double T = std::floor(x / kTile);
    if (kTile * T > x) T -= 1.0;
    else if (kTile * (T + 1.0) <= x) T += 1.0;
    return T;
}

bool tile_key(const double x[3], float inv_v, int tv, Key* out, float local[3], int32_t tile[3]) {
    int32_t k[3];
    for (int a = 0; a < 3; ++a) {
        if (!std::isfinite(x[a])) return false;
        double T = tile_floor(x[a]);
        if (!(std::fabs(T) * tv < (double)kKeyLimit)) return false;
        float xt = (float)(x[a] - kTile * T);
        float s = xt * inv_v;
        int32_t kin = (int32_t)std::floor(s);
        if (kin < 0) kin = 0;
        if (kin > tv - 1) kin = tv - 1;
        int64_t key = (int64_t)T * tv + kin;
        if (key < -(int64_t)kKeyLimit || key >= (int64_t)kKeyLimit) return false;
        k[a] = (int32_t)key;
        local[a] = xt;
        tile[a] = (int32_t)T;
    }
    *out = Key{k[0], k[1], k[2]};
    return true;
}

// Tile of a key (floor division by tv).
int32_t tile_of(int32_t k, int tv) { return (int32_t)std::floor((double)k / (double)tv); }

// A search frame: the origin of tile (fx, fy, fz); fx = fy = fz = 0 with tv = 0 is the
// world frame of the plain map. Frame coordinates of a map point: fp32(p + 50 (T_p - F)),
// one FP32 addition of an exact multiple of 50.
struct Frame {
    int32_t f[3] = {0, 0, 0};
    int tv = 0;
};

// ------------------------------------------------------------------ small linear algebra (FP64)

void mat3_inverse(const double a[3][3], double out[3][3], double* det_out) {
    double c00 = a[1][1] * a[2][2] - a[1][2] * a[2][1];
    double c01 = a[1][2] * a[2][0] - a[1][0] * a[2][2];
    double c02 = a[1][0] * a[2][1] - a[1][1] * a[2][0];
    double det = a[0][0] * c00 + a[0][1] * c01 + a[0][2] * c02;
    double inv = 1.0 / det;
    out[0][0] = c00 * inv;
    out[0][1] = (a[0][2] * a[2][1] - a[0][1] * a[2][2]) * inv;
    out[0][2] = (a[0][1] * a[1][2] - a[0][2] * a[1][1]) * inv;
    out[1][0] = c01 * inv;
    out[1][1] = (a[0][0] * a[2][2] - a[0][2] * a[2][0]) * inv;
    out[1][2] = (a[0][2] * a[1][0] - a[0][0] * a[1][2]) * inv;
    out[2][0] = c02 * inv;
    out[2][1] = (a[0][1] * a[2][0] - a[0][0] * a[2][1]) * inv;
    out[2][2] = (a[0][0] * a[1][1] - a[0][1] * a[1][0]) * inv;
    if (det_out) *det_out = det;
}

void skew(const double v[3], double s[3][3]) {
    s[0][0] = 0; s[0][1] = -v[2]; s[0][2] = v[1];
    s[1][0] = v[2]; s[1][1] = 0; s[1][2] = -v[0];
    s[2][0] = -v[1]; s[2][1] = v[0]; s[2][2] = 0;
}

// SE(3) exponential (reading: closed-form Rodrigues rotation and V matrix,
// second-order Taylor terms for theta < 1e-8). xi = [phi; rho].
void se3_exp(const double xi[6], double T[16]) {
    const double* phi = xi;
    const double* rho = xi + 3;
    double th2 = phi[0] * phi[0] + phi[1] * phi[1] + phi[2] * phi[2];
    double th = std::sqrt(th2);
    double A, B, C;  // R = I + A K + B K^2,  V = I + B K + C K^2
    if (th < 1e-8) {
        A = 1.0 - th2 / 6.0;
        B = 0.5 - th2 / 24.0;
        C = 1.0 / 6.0 - th2 / 120.0;
    } else {
        A = std::sin(th) / th;
        B = (1.0 - std::cos(th)) / th2;
        C = (th - std::sin(th)) / (th2 * th);
    }
    double K[3][3], K2[3][3];
    skew(phi, K);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            K2[i][j] = 0;
            for (int l = 0; l < 3; ++l) K2[i][j] += K[i][l] * K[l][j];
        }
    double R[3][3], V[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double id = (i == j) ? 1.0 : 0.0;
            R[i][j] = id + A * K[i][j] + B * K2[i][j];
            V[i][j] = id + B * K[i][j] + C * K2[i][j];
        }
    std::memset(T, 0, 16 * sizeof(double));
    for (int i = 0; i < 3; ++i) {
        for (int j = 0; j < 3; ++j) T[4 * i + j] = R[i][j];
        T[4 * i + 3] = V[i][0] * rho[0] + V[i][1] * rho[1] + V[i][2] * rho[2];
    }
    T[15] = 1.0;
}

// SE(3) logarithm for rotation angles below pi (used by the round-trip check).
void se3_log(const double T[16], double xi[6]) {
    double tr = T[0] + T[5] + T[10];
    double c = std::max(-1.0, std::min(1.0, 0.5 * (tr - 1.0)));
    double th = std::acos(c);
    double w[3] = {T[9] - T[6], T[2] - T[8], T[4] - T[1]};  // R - R^T, vee
    double f = (th < 1e-8) ? 0.5 + th * th / 12.0 : th / (2.0 * std::sin(th));
    double phi[3] = {f * w[0], f * w[1], f * w[2]};
    double th2 = th * th;
    double K[3][3], K2[3][3];
    skew(phi, K);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            K2[i][j] = 0;
            for (int l = 0; l < 3; ++l) K2[i][j] += K[i][l] * K[l][j];
        }
    // V^-1 = I - K/2 + (1/th^2)(1 - (th sin th)/(2(1 - cos th))) K^2
    double D = (th < 1e-8) ? 1.0 / 12.0 : (1.0 - th * std::sin(th) / (2.0 * (1.0 - std::cos(th)))) / th2;
    double t[3] = {T[3], T[7], T[11]};
    for (int i = 0; i < 3; ++i) {
        double acc = 0;
        for (int j = 0; j < 3; ++j) {
            double vij = ((i == j) ? 1.0 : 0.0) - 0.5 * K[i][j] + D * K2[i][j];
            acc += vij * t[j];
        }
        xi[3 + i] = acc;
        xi[i] = phi[i];
    }
}

void mat4_mul(const double a[16], const double b[16], double out[16]) {
    double r[16];
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) {
            double s = 0;
            for (int l = 0; l < 4; ++l) s += a[4 * i + l] * b[4 * l + j];
            r[4 * i + j] = s;
        }
    std::memcpy(out, r, sizeof(r));
}

void rigid_inverse(const double T[16], double out[16]) {
    double r[16] = {0};
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) r[4 * i + j] = T[4 * j + i];
    for (int i = 0; i < 3; ++i) r[4 * i + 3] = -(r[4 * i + 0] * T[3] + r[4 * i + 1] * T[7] + r[4 * i + 2] * T[11]);
    r[15] = 1.0;
    std::memcpy(out, r, sizeof(r));
}

// Cholesky of a 6x6 SPD matrix (textbook, lower factor). false if not PD.
bool cholesky6(const double H[36], double L[36]) {
    std::memset(L, 0, 36 * sizeof(double));
    for (int j = 0; j < 6; ++j) {
        double s = H[6 * j + j];
        for (int k = 0; k < j; ++k) s -= L[6 * j + k] * L[6 * j + k];
        if (!(s > 0.0)) return false;
        double d = std::sqrt(s);
        L[6 * j + j] = d;
        for (int i = j + 1; i < 6; ++i) {
            double t = H[6 * i + j];
            for (int k = 0; k < j; ++k) t -= L[6 * i + k] * L[6 * j + k];
            L[6 * i + j] = t / d;
        }
    }
    return true;
}

void cholesky6_solve(const double L[36], const double b[6], double x[6]) {
    double y[6];
    for (int i = 0; i < 6; ++i) {
        double s = b[i];
        for (int k = 0; k < i; ++k) s -= L[6 * i + k] * y[k];
        y[i] = s / L[6 * i + i];
    }
    for (int i = 5; i >= 0; --i) {
        double s = y[i];
        for (int k = i + 1; k < 6; ++k) s -= L[6 * k + i] * x[k];
        x[i] = s / L[6 * i + i];
    }
}

// ------------------------------------------------------------------ voxel map (cuVoxelMap analogue)
struct MapPoint {
    float p[3];        // FP32 world point (plain) or tile-relative coordinates (precision variant)
    double w[3];       // world point used by all arithmetic: (double)p (plain) or the unrounded transform
    int32_t tile[3];   // tile of the point's voxel (precision variant; 0 otherwise)
    uint32_t id;
    double cov[6];  // xx xy xz yy yz zz
    int valid;
};
struct Voxel {
    std::vector<MapPoint> pts;
};

}  // namespace

struct OracleMap {
    float v;
    float inv_v;
    int nmax;
    int k;
    float dmin2;
    int prec = 0;   // precision variant (tile keys, FP64 world points)
    int tv = 0;     // voxels per tile side (precision variant)
    std::unordered_map<Key, Voxel, KeyHash> vox;
    uint32_t next_id = 0;
    uint64_t npoints = 0;
};

namespace {

// Frame coordinates of a map point (see Frame).
void frame_coords(const MapPoint& p, const Frame& fr, float out[3]) {
    for (int a = 0; a < 3; ++a) {
        float off = (fr.tv > 0) ? (float)(kTile * (double)(p.tile[a] - fr.f[a])) : 0.0f;
        out[a] = p.p[a] + off;
    }
}

// Centre key of a query given in frame coordinates: K_F + floor(fp32(q_F * inv_v)).
bool frame_key(const OracleMap& m, const float qf[3], const Frame& fr, Key* out) {
    Key c;
    if (!voxel_key(qf, m.inv_v, &c)) return false;
    if (fr.tv > 0) {
        int64_t k[3] = {(int64_t)c.x + (int64_t)fr.f[0] * fr.tv, (int64_t)c.y + (int64_t)fr.f[1] * fr.tv,
                        (int64_t)c.z + (int64_t)fr.f[2] * fr.tv};
        for (int a = 0; a < 3; ++a)
            if (k[a] < -(int64_t)kKeyLimit || k[a] >= (int64_t)kKeyLimit) return false;
        c = Key{(int32_t)k[0], (int32_t)k[1], (int32_t)k[2]};
    }
    *out = c;
    return true;
}

// kNN over the 27 voxels around centre key c, ordered by (d^2, id) with the FP32
// distance between the query and the points, both in frame coordinates.
// Returns the number found (<= k); ids/points of the k best in order.
int knn27_at(const OracleMap& m, const Key& c, const float qf[3], const Frame& fr, int k,
             std::vector<const MapPoint*>* best) {
    best->clear();
    std::vector<std::pair<std::pair<float, uint32_t>, const MapPoint*>> cand;
    for (int dx = -1; dx <= 1; ++dx)
        for (int dy = -1; dy <= 1; ++dy)
            for (int dz = -1; dz <= 1; ++dz) {
                Key n{c.x + dx, c.y + dy, c.z + dz};
                auto it = m.vox.find(n);
                if (it == m.vox.end()) continue;
                for (const MapPoint& p : it->second.pts) {
                    float pf[3];
                    frame_coords(p, fr, pf);
                    cand.push_back({{dist2_f32(qf, pf), p.id}, &p});
                }
            }
    std::sort(cand.begin(), cand.end(),
              [](const auto& a, const auto& b) { return a.first < b.first; });
    int found = (int)std::min<size_t>(cand.size(), (size_t)k);
    for (int i = 0; i < found; ++i) best->push_back(cand[i].second);
    return found;
}

// kNN of a query in world FP32 coordinates (plain map: the world frame; precision
// variant: the frame of the query's own tile).
int knn27(const OracleMap& m, const float q[3], int k, std::vector<const MapPoint*>* best) {
    best->clear();
    Frame fr;
    float qf[3] = {q[0], q[1], q[2]};
    if (m.prec) {
        fr.tv = m.tv;
        for (int a = 0; a < 3; ++a) {
            double T = tile_floor((double)q[a]);
            fr.f[a] = (int32_t)T;
            qf[a] = (float)((double)q[a] - kTile * T);
        }
    }
    Key c;
    if (!frame_key(m, qf, fr, &c)) return 0;
    return knn27_at(m, c, qf, fr, k, best);
}

// Eq. 1: Sigma-hat from the k nearest neighbours (population form, 1/k, around
// the neighbour mean), C = Sigma-hat + 1e-3 I, Sigma = (C^-1 / ||C^-1||_F)^-1.
void covariance_eq1(const std::vector<const MapPoint*>& nb, double out[6]) {
    double k = (double)nb.size();
    double mu[3] = {0, 0, 0};
    for (const MapPoint* p : nb)
        for (int a = 0; a < 3; ++a) mu[a] += p->w[a];
    for (int a = 0; a < 3; ++a) mu[a] /= k;
    double S[3][3] = {{0}};
    for (const MapPoint* p : nb) {
        double d[3] = {p->w[0] - mu[0], p->w[1] - mu[1], p->w[2] - mu[2]};
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) S[i][j] += d[i] * d[j];
    }
    double C[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) C[i][j] = S[i][j] / k + ((i == j) ? 1e-3 : 0.0);
    double Ci[3][3];
    mat3_inverse(C, Ci, nullptr);
    double fro = 0;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) fro += Ci[i][j] * Ci[i][j];
    fro = std::sqrt(fro);
    double P[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) P[i][j] = Ci[i][j] / fro;
    double Sig[3][3];
    mat3_inverse(P, Sig, nullptr);
    out[0] = Sig[0][0]; out[1] = Sig[0][1]; out[2] = Sig[0][2];
    out[3] = Sig[1][1]; out[4] = Sig[1][2]; out[5] = Sig[2][2];
}

// World point of an insert: x_w = fp32(R p + t), evaluated in FP64 in a fixed
// order ((R0 px + R1 py) + R2 pz) + t and rounded once.
void transform_point_f32(const double T[16], const float p[3], float out[3]) {
    double x = p[0], y = p[1], z = p[2];
    for (int r = 0; r < 3; ++r) {
        double a = T[4 * r + 0] * x;
        double b = T[4 * r + 1] * y;
        double c = T[4 * r + 2] * z;
        double s = a + b;
        s = s + c;
        s = s + T[4 * r + 3];
        out[r] = (float)s;
    }
}

// World point of an insert in FP64 (precision variant): the same expression, not rounded.
void transform_point_f64(const double T[16], const float p[3], double out[3]) {
    double x = p[0], y = p[1], z = p[2];
    for (int r = 0; r < 3; ++r) {
        double a = T[4 * r + 0] * x;
        double b = T[4 * r + 1] * y;
        double c = T[4 * r + 2] * z;
        double s = a + b;
        s = s + c;
        out[r] = s + T[4 * r + 3];
    }
}

bool finite3(const float p[3]) { return std::isfinite(p[0]) && std::isfinite(p[1]) && std::isfinite(p[2]); }

struct InsertResult {
    uint64_t n_added = 0;
    double n_near = 0;
    std::vector<std::pair<Key, MapPoint*>> added;  // in id order
    std::vector<int64_t> admitted_index;           // input index of each added point, id order
};

// Sec. III-A.3 insert with the Adaptive Submap Density cap.
//   ASMD reading: N_near = mean (uncapped) count of this scan's voxels whose
//   centre lies within r_c of the sensor; per voxel
//   N_ASMD(r) = clamp(round(N_near + (k - N_near) min(r / r_max, 1)), k, N_max),
//   r = distance from the voxel centre to the sensor, all in FP64. With no voxel
//   within r_c, N_near = N_max. asmd = 0 uses N_max everywhere.
//   Admission reading: points are taken in input order; a point enters its voxel
//   while the voxel holds fewer than its cap and every point already there is at
//   least d_min away (FP32 d^2 >= d_min^2). Admitted points get consecutive ids.
InsertResult map_insert(OracleMap& m, const float* xyz, int64_t n, const double* T, int asmd,
                        double r_c, double r_max) {
    InsertResult res;
    const double sensor[3] = {T ? T[3] : 0.0, T ? T[7] : 0.0, T ? T[11] : 0.0};
    std::vector<float> w(3 * (size_t)n);      // FP32 decision coordinates (world or tile-relative)
    std::vector<double> w64(3 * (size_t)n);   // world point for arithmetic
    std::vector<int32_t> tiles(3 * (size_t)n, 0);
    std::vector<Key> keys((size_t)n);
    std::vector<char> ok((size_t)n, 0);
    std::unordered_map<Key, int64_t, KeyHash> scan_count;
    for (int64_t i = 0; i < n; ++i) {
        const float* p = xyz + 3 * i;
        if (!finite3(p)) continue;
        float* x = &w[3 * i];
        double* x64 = &w64[3 * i];
        if (m.prec) {
            // precision variant: FP64 world point, tile key, tile-relative FP32 coordinates
            if (T) transform_point_f64(T, p, x64);
            else for (int a = 0; a < 3; ++a) x64[a] = (double)p[a];
            if (!tile_key(x64, m.inv_v, m.tv, &keys[i], x, &tiles[3 * i])) continue;
        } else {
            if (T) transform_point_f32(T, p, x);
            else std::memcpy(x, p, 3 * sizeof(float));
            if (!voxel_key(x, m.inv_v, &keys[i])) continue;
            for (int a = 0; a < 3; ++a) x64[a] = (double)x[a];
        }
        ok[i] = 1;
        scan_count[keys[i]] += 1;
    }
    const double vd = (double)m.v;
    auto centre_dist2 = [&](const Key& key) {
        double cx = ((double)key.x + 0.5) * vd;
        double cy = ((double)key.y + 0.5) * vd;
        double cz = ((double)key.z + 0.5) * vd;
        double dx = cx - sensor[0], dy = cy - sensor[1], dz = cz - sensor[2];
        double s = dx * dx + dy * dy;
        return s + dz * dz;
    };
    double n_near = (double)m.nmax;
    if (asmd) {
        int64_t sum = 0, cnt = 0;
        double rc2 = r_c * r_c;
        for (const auto& kv : scan_count)
            if (centre_dist2(kv.first) <= rc2) { sum += kv.second; cnt += 1; }
        if (cnt > 0) n_near = (double)sum / (double)cnt;
    }
    res.n_near = n_near;
    auto cap_of = [&](const Key& key) -> int {
        if (!asmd) return m.nmax;
        double r = std::sqrt(centre_dist2(key));
        double f = r / r_max;
        if (f > 1.0) f = 1.0;
        double val = n_near + ((double)m.k - n_near) * f;
        double c = std::floor(val + 0.5);
        int cap = (int)c;
        if (c > (double)m.nmax) cap = m.nmax;
        if (c < (double)m.k) cap = m.k;
        return cap;
    };
    std::unordered_map<Key, int, KeyHash> caps;
    for (const auto& kv : scan_count) caps[kv.first] = cap_of(kv.first);

    std::vector<std::pair<Key, size_t>> added_pos;
    for (int64_t i = 0; i < n; ++i) {
        if (!ok[i]) continue;
        const float* x = &w[3 * i];
        Voxel& vx = m.vox[keys[i]];
        if ((int)vx.pts.size() >= caps[keys[i]]) continue;
        bool spaced = true;
        for (const MapPoint& q : vx.pts)
            if (!(dist2_f32(x, q.p) >= m.dmin2)) { spaced = false; break; }
        if (!spaced) continue;
        MapPoint mp;
        std::memcpy(mp.p, x, sizeof(mp.p));
        std::memcpy(mp.w, &w64[3 * i], sizeof(mp.w));
        std::memcpy(mp.tile, &tiles[3 * i], sizeof(mp.tile));
        mp.id = m.next_id++;
        std::memset(mp.cov, 0, sizeof(mp.cov));
        mp.valid = 0;
        vx.pts.push_back(mp);
        added_pos.push_back({keys[i], vx.pts.size() - 1});
        res.admitted_index.push_back(i);
        res.n_added += 1;
    }
    m.npoints += res.n_added;
    for (const auto& kp : added_pos) res.added.push_back({kp.first, &m.vox[kp.first].pts[kp.second]});
    return res;
}

// Sec. III-A.3: covariances are computed for the added points only, against the
// whole updated map; existing points keep theirs.
void added_covariances(OracleMap& m, InsertResult& res) {
    std::vector<double> covs(6 * res.added.size());
    std::vector<int> valid(res.added.size());
    parallel_chunks(res.added.size(), g_threads, [&](int, size_t b, size_t e) {
        std::vector<const MapPoint*> nb;
        for (size_t i = b; i < e; ++i) {
            const MapPoint* p = res.added[i].second;
            Frame fr;
            if (m.prec) {
                fr.tv = m.tv;
                std::memcpy(fr.f, p->tile, sizeof(fr.f));
            }
            // the query is the point itself, centred on its own voxel, in the frame of its tile
            int found = knn27_at(m, res.added[i].first, p->p, fr, m.k, &nb);
            valid[i] = (found >= m.k) ? 1 : 0;
            if (valid[i]) covariance_eq1(nb, &covs[6 * i]);
            else std::fill(&covs[6 * i], &covs[6 * i] + 6, 0.0);
        }
    });
    for (size_t i = 0; i < res.added.size(); ++i) {
        std::memcpy(res.added[i].second->cov, &covs[6 * i], 6 * sizeof(double));
        res.added[i].second->valid = valid[i];
    }
}

// Source point of a registration problem (Sec. III-A.2, Cov-Calc on a scan-local map).
struct SourcePoint {
    double s[3];
    float sf[3];
    double cov[6];
    int valid;
    int64_t index;  // input index
};

// The scan-local map: same v, N_max, spacing, no ASMD; only admitted points are
// registered (this is also the downsampling).
std::vector<SourcePoint> scan_local_sources(const float* xyz, int64_t n, float v, int nmax, int k, float dmin2,
                                            std::vector<uint32_t>* knn_ids) {
    OracleMap local;
    local.v = v;
    local.inv_v = 1.0f / v;
    local.nmax = nmax;
    local.k = k;
    local.dmin2 = dmin2;
    InsertResult ins = map_insert(local, xyz, n, nullptr, 0, 0.0, 1.0);
    // ids are the admission rank, which increases with the input index
    std::vector<SourcePoint> src(local.next_id);
    std::vector<const MapPoint*> by_id(local.next_id, nullptr);
    for (const auto& kv : local.vox)
        for (const MapPoint& p : kv.second.pts) by_id[p.id] = &p;
    if (knn_ids) knn_ids->assign((size_t)local.next_id * (size_t)k, 0xFFFFFFFFu);
    parallel_chunks(local.next_id, g_threads, [&](int, size_t b, size_t e) {
        std::vector<const MapPoint*> nb;
        for (size_t id = b; id < e; ++id) {
            SourcePoint& sp = src[id];
            const MapPoint* p = by_id[id];
            for (int a = 0; a < 3; ++a) { sp.sf[a] = p->p[a]; sp.s[a] = (double)p->p[a]; }
            sp.index = ins.admitted_index[id];
            int found = knn27(local, p->p, k, &nb);
            if (knn_ids)
                for (int j = 0; j < found; ++j) (*knn_ids)[id * k + j] = nb[j]->id;
            sp.valid = (found >= k) ? 1 : 0;
            if (sp.valid) covariance_eq1(nb, sp.cov);
            else std::fill(sp.cov, sp.cov + 6, 0.0);
        }
    });
    return src;
}

// 1-NN over the 27 voxels around the centre key of qf (frame coordinates), smallest
// (FP32 d^2, id) in frame coordinates.
const MapPoint* nearest27_frame(const OracleMap& m, const float qf[3], const Frame& fr, float* d2_out) {
    Key c;
    *d2_out = std::numeric_limits<float>::infinity();
    if (!frame_key(m, qf, fr, &c)) return nullptr;
    const MapPoint* best = nullptr;
    float bd = std::numeric_limits<float>::infinity();
    for (int dx = -1; dx <= 1; ++dx)
        for (int dy = -1; dy <= 1; ++dy)
            for (int dz = -1; dz <= 1; ++dz) {
                auto it = m.vox.find(Key{c.x + dx, c.y + dy, c.z + dz});
                if (it == m.vox.end()) continue;
                for (const MapPoint& p : it->second.pts) {
                    float pf[3];
                    frame_coords(p, fr, pf);
                    float d2 = dist2_f32(qf, pf);
                    if (best == nullptr || d2 < bd || (d2 == bd && p.id < best->id)) {
                        best = &p;
                        bd = d2;
                    }
                }
            }
    *d2_out = bd;
    return best;
}

// 1-NN of a query in world FP32 coordinates (frame as in knn27).
const MapPoint* nearest27(const OracleMap& m, const float q[3], float* d2_out) {
    Frame fr;
    float qf[3] = {q[0], q[1], q[2]};
    if (m.prec) {
        fr.tv = m.tv;
        for (int a = 0; a < 3; ++a) {
            double T = tile_floor((double)q[a]);
            fr.f[a] = (int32_t)T;
            qf[a] = (float)((double)q[a] - kTile * T);
        }
    }
    return nearest27_frame(m, qf, fr, d2_out);
}

// Gauss-Newton anchor: the world origin for the plain map; for the precision variant the
// corner of the tile holding the initial position, A = 50 floor(t / 50). The linearisation
// and the update are expressed about A (J = [[q - A]x, -I], T <- exp(xi) applied to the pose
// relative to A); the GN iterates are the same as about the origin, since exp(Ad_A xi) =
// A exp(xi) A^-1 and the linear model changes by the same invertible map.
Frame anchor_frame(const OracleMap& m, const double T[16], double A[3]) {
    Frame fr;
    A[0] = A[1] = A[2] = 0.0;
    if (m.prec) {
        fr.tv = m.tv;
        for (int a = 0; a < 3; ++a) {
            double t = tile_floor(T[4 * a + 3]);
            fr.f[a] = (int32_t)t;
            A[a] = kTile * t;
        }
    }
    return fr;
}

// T <- exp(xi) T about the anchor A (Eq. 6).
void apply_update(const double xi[6], const double A[3], double T[16]) {
    double E[16], Tr[16];
    se3_exp(xi, E);
    std::memcpy(Tr, T, sizeof(Tr));
    for (int a = 0; a < 3; ++a) Tr[4 * a + 3] = T[4 * a + 3] - A[a];
    mat4_mul(E, Tr, T);
    for (int a = 0; a < 3; ++a) T[4 * a + 3] = T[4 * a + 3] + A[a];
}

struct LinResult {
    double H[36];
    double g[6];
    int64_t n_corr = 0, n_p2p = 0;
    double chi2 = 0;
};

// One Gauss-Newton linearisation of Eq. 4 at pose T.
//   Correspondence: 1-NN of fp32(T s) over the 27 voxels (ties to the smaller
//   id), rejected when d^2 > tau^2 (FP32).
//   Eq. 3 residual d = r - T s; Mahalanobis matrix M = (Sigma_r + R Sigma_s R^T)^-1,
//   or M = I when either covariance is invalid (SA GICP).
//   Cauchy (Eq. 5) is applied to e = sqrt(d^T M d): IRLS weight w = 1 / (1 + e^2/kappa^2).
//   Left perturbation T <- exp(xi) T, xi = [phi; rho]: J = [[q]x, -I], with q taken
//   relative to the anchor A (the origin for the plain map, see anchor_frame).
//   H = sum w J^T M J, g = sum w J^T M d.
LinResult linearize_range(const OracleMap& m, const std::vector<SourcePoint>& src, size_t n_begin, size_t n_end,
                          const double T[16], const Frame& fr, const double A[3], float tau2, double kappa,
                          int32_t* corr_out) {
    LinResult L;
    std::memset(L.H, 0, sizeof(L.H));
    std::memset(L.g, 0, sizeof(L.g));
    double R[3][3], t[3];
    for (int i = 0; i < 3; ++i) {
        for (int j = 0; j < 3; ++j) R[i][j] = T[4 * i + j];
        t[i] = T[4 * i + 3];
    }
    double k2 = kappa * kappa;
    // The search query is an FP32 quantity (the paper registers in float32, Sec. III-A.2): the
    // pose rounded once to FP32 (rotation entries, and the translation relative to the anchor
    // A), applied to the FP32 source point as the chain fma(R_i0, s0, fma(R_i1, s1,
    // fma(R_i2, s2, t_i))) with one rounding per fused multiply-add. The residual and the
    // Jacobian below use the FP64 transform.
    float Rf[3][3], tf[3];
    for (int i = 0; i < 3; ++i) {
        for (int j = 0; j < 3; ++j) Rf[i][j] = (float)R[i][j];
        tf[i] = (float)(t[i] - A[i]);
    }
    for (size_t n = n_begin; n < n_end; ++n) {
        const SourcePoint& sp = src[n];
        double q[3];
        for (int i = 0; i < 3; ++i) q[i] = R[i][0] * sp.s[0] + R[i][1] * sp.s[1] + R[i][2] * sp.s[2] + t[i];  // Eq. 2 / Eq. 6
        // FP32 query in the frame of the anchor (the world frame for the plain map)
        float qf[3];
        for (int i = 0; i < 3; ++i)
            qf[i] = std::fmaf(Rf[i][0], sp.sf[0], std::fmaf(Rf[i][1], sp.sf[1], std::fmaf(Rf[i][2], sp.sf[2], tf[i])));
        float d2;
        const MapPoint* nn = nearest27_frame(m, qf, fr, &d2);
        if (corr_out) corr_out[n] = -1;
        if (!nn || d2 > tau2) continue;
        if (corr_out) corr_out[n] = (int32_t)nn->id;
        double M[3][3];
        bool p2p = !(sp.valid && nn->valid);
        if (p2p) {
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) M[i][j] = (i == j) ? 1.0 : 0.0;
        } else {
            double Ss[3][3] = {{sp.cov[0], sp.cov[1], sp.cov[2]},
                               {sp.cov[1], sp.cov[3], sp.cov[4]},
                               {sp.cov[2], sp.cov[4], sp.cov[5]}};
            double RS[3][3], C[3][3];
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) {
                    RS[i][j] = 0;
                    for (int l = 0; l < 3; ++l) RS[i][j] += R[i][l] * Ss[l][j];
                }
            const double* c = nn->cov;
            double Sr[3][3] = {{c[0], c[1], c[2]}, {c[1], c[3], c[4]}, {c[2], c[4], c[5]}};
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) {
                    double s = 0;
                    for (int l = 0; l < 3; ++l) s += RS[i][l] * R[j][l];
                    C[i][j] = Sr[i][j] + s;
                }
            mat3_inverse(C, M, nullptr);
        }
        double d[3] = {nn->w[0] - q[0], nn->w[1] - q[1], nn->w[2] - q[2]};  // Eq. 3
        double Md[3];
        for (int i = 0; i < 3; ++i) Md[i] = M[i][0] * d[0] + M[i][1] * d[1] + M[i][2] * d[2];
        double e2 = d[0] * Md[0] + d[1] * Md[1] + d[2] * Md[2];
        double w = 1.0 / (1.0 + e2 / k2);
        double J[3][6];
        double Q[3][3];
        const double qa[3] = {q[0] - A[0], q[1] - A[1], q[2] - A[2]};  // about the anchor
        skew(qa, Q);
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                J[i][j] = Q[i][j];
                J[i][3 + j] = (i == j) ? -1.0 : 0.0;
            }
        double MJ[3][6];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 6; ++j) MJ[i][j] = M[i][0] * J[0][j] + M[i][1] * J[1][j] + M[i][2] * J[2][j];
        for (int a = 0; a < 6; ++a) {
            for (int b = 0; b < 6; ++b)
                L.H[6 * a + b] += w * (J[0][a] * MJ[0][b] + J[1][a] * MJ[1][b] + J[2][a] * MJ[2][b]);
            L.g[a] += w * (J[0][a] * Md[0] + J[1][a] * Md[1] + J[2][a] * Md[2]);
        }
        L.chi2 += 0.5 * k2 * std::log(1.0 + e2 / k2);  // Eq. 5 with e^2 = d^T M d
        L.n_corr += 1;
        if (p2p) L.n_p2p += 1;
    }
    return L;
}

// The linearisation over all sources: per-chunk sums (one chunk with one thread), added in
// chunk order.
LinResult linearize(const OracleMap& m, const std::vector<SourcePoint>& src, const double T[16], const Frame& fr,
                    const double A[3], float tau2, double kappa, int32_t* corr_out) {
    if (g_threads <= 1) return linearize_range(m, src, 0, src.size(), T, fr, A, tau2, kappa, corr_out);
    std::vector<LinResult> part(g_threads);
    parallel_chunks(src.size(), g_threads, [&](int c, size_t b, size_t e) {
        part[c] = linearize_range(m, src, b, e, T, fr, A, tau2, kappa, corr_out);
    });
    LinResult L = part[0];
    for (int c = 1; c < g_threads; ++c) {
        for (int i = 0; i < 36; ++i) L.H[i] += part[c].H[i];
        for (int i = 0; i < 6; ++i) L.g[i] += part[c].g[i];
        L.n_corr += part[c].n_corr;
        L.n_p2p += part[c].n_p2p;
        L.chi2 += part[c].chi2;
    }
    return L;
}

}  // namespace

// ====================================================================== C API
extern "C" {

struct om_reg_params {
    uint32_t max_iters;
    double conv_eps;
    float tau;
    double kappa;
};

struct om_reg_stats {
    uint32_t iters, n_src, n_corr, n_p2p;
    int converged;
    int status;  // 0 ok, 5 degenerate
    double chi2;
};

OracleMap* om_create_prec(float voxel_size, int nmax, int k, float min_spacing, int precision_mode) {
    int tv = 0;
    if (precision_mode) {
        // tiles of 50 m: v must divide 50 m
        double r = 50.0 / (double)voxel_size;
        tv = (int)std::lround(r);
        if (tv < 1 || std::fabs(r - (double)tv) > 1e-9 * r) return nullptr;
    }
    OracleMap* m = new OracleMap();
    m->prec = precision_mode ? 1 : 0;
    m->tv = tv;
    m->v = voxel_size;
    m->inv_v = 1.0f / voxel_size;
    m->nmax = nmax;
    m->k = k;
    // spacing reading: d_min = v / sqrt(N_max) when min_spacing < 0
    float dmin = (min_spacing < 0.0f) ? (float)((double)voxel_size / std::sqrt((double)nmax)) : min_spacing;
    m->dmin2 = dmin * dmin;
    return m;
}

OracleMap* om_create(float voxel_size, int nmax, int k, float min_spacing) {
    return om_create_prec(voxel_size, nmax, k, min_spacing, 0);
}

void om_destroy(OracleMap* m) { delete m; }

float om_dmin2(const OracleMap* m) { return m->dmin2; }

uint64_t om_insert(OracleMap* m, const float* xyz, int64_t n, const double* pose, int asmd, double r_c,
                   double r_max, double* n_near_out) {
    InsertResult r = map_insert(*m, xyz, n, pose, asmd, r_c, r_max);
    added_covariances(*m, r);
    if (n_near_out) *n_near_out = r.n_near;
    return r.n_added;
}

// Sec. III-A.3 eviction reading: remove voxels whose centre ((key + 0.5) v, FP64)
// is strictly farther than `radius` from `center`.
uint64_t om_evict(OracleMap* m, const double* center, double radius) {
    uint64_t removed = 0;
    double r2 = radius * radius;
    const double vd = (double)m->v;
    for (auto it = m->vox.begin(); it != m->vox.end();) {
        double cx = ((double)it->first.x + 0.5) * vd - center[0];
        double cy = ((double)it->first.y + 0.5) * vd - center[1];
        double cz = ((double)it->first.z + 0.5) * vd - center[2];
        double s = cx * cx + cy * cy;
        s = s + cz * cz;
        if (s > r2) {
            removed += it->second.pts.size();
            it = m->vox.erase(it);
        } else {
            ++it;
        }
    }
    m->npoints -= removed;
    return removed;
}

uint64_t om_num_voxels(const OracleMap* m) { return m->vox.size(); }
uint64_t om_num_points(const OracleMap* m) { return m->npoints; }

// Export sorted by key (x, y, z); points within a voxel in insertion order.
void om_export(const OracleMap* m, int32_t* keys, uint32_t* counts, uint32_t* ids, float* xyz, double* cov,
               int32_t* valid) {
    std::vector<Key> ks;
    ks.reserve(m->vox.size());
    for (const auto& kv : m->vox) ks.push_back(kv.first);
    std::sort(ks.begin(), ks.end());
    size_t pi = 0;
    for (size_t i = 0; i < ks.size(); ++i) {
        const Voxel& vx = m->vox.at(ks[i]);
        keys[3 * i + 0] = ks[i].x;
        keys[3 * i + 1] = ks[i].y;
        keys[3 * i + 2] = ks[i].z;
        counts[i] = (uint32_t)vx.pts.size();
        for (const MapPoint& p : vx.pts) {
            ids[pi] = p.id;
            if (m->prec) {
                // world FP32: fp32(50 T + x_t), the tile-relative value restored exactly in FP64
                for (int a = 0; a < 3; ++a) xyz[3 * pi + a] = (float)(kTile * (double)p.tile[a] + (double)p.p[a]);
            } else {
                std::memcpy(xyz + 3 * pi, p.p, 3 * sizeof(float));
            }
            std::memcpy(cov + 6 * pi, p.cov, 6 * sizeof(double));
            valid[pi] = p.valid;
            ++pi;
        }
    }
}

// kNN (k <= 64) of query points against the map: ids (k per query, 0xFFFFFFFF pad), found count.
void om_knn(const OracleMap* m, const float* q, int64_t n, int k, uint32_t* ids, int32_t* found) {
    std::vector<const MapPoint*> nb;
    for (int64_t i = 0; i < n; ++i) {
        int f = knn27(*m, q + 3 * i, k, &nb);
        found[i] = f;
        for (int j = 0; j < k; ++j) ids[i * k + j] = (j < f) ? nb[j]->id : 0xFFFFFFFFu;
    }
}

// 1-NN of query points; ids[i] = -1 when there is no candidate or d^2 > tau2.
void om_nearest(const OracleMap* m, const float* q, int64_t n, float tau2, int64_t* ids, float* d2) {
    for (int64_t i = 0; i < n; ++i) {
        float dd;
        const MapPoint* p = nearest27(*m, q + 3 * i, &dd);
        d2[i] = dd;
        ids[i] = (p && !(dd > tau2)) ? (int64_t)p->id : -1;
    }
}

// Scan-local map + source covariances. Writes admitted input indices (index
// order), covariances (6 per admitted point), validity and kNN ids (k each).
// Returns the number of admitted points. Output arrays must hold n entries.
int64_t om_scan_sources(const float* xyz, int64_t n, float v, int nmax, int k, float min_spacing, int64_t* index,
                        double* cov, int32_t* valid, uint32_t* knn_ids) {
    float dmin = (min_spacing < 0.0f) ? (float)((double)v / std::sqrt((double)nmax)) : min_spacing;
    std::vector<uint32_t> kid;
    std::vector<SourcePoint> src = scan_local_sources(xyz, n, v, nmax, k, dmin * dmin, &kid);
    for (size_t i = 0; i < src.size(); ++i) {
        index[i] = src[i].index;
        std::memcpy(cov + 6 * i, src[i].cov, 6 * sizeof(double));
        valid[i] = src[i].valid;
        if (knn_ids) std::memcpy(knn_ids + i * (size_t)k, &kid[i * (size_t)k], (size_t)k * sizeof(uint32_t));
    }
    return (int64_t)src.size();
}

// One linearisation at `pose` for already-computed source points (input points,
// covariances, validity): H (36), g (6), correspondence ids (n), counts, chi2.
void om_linearize(const OracleMap* m, const float* src_xyz, const double* src_cov, const int32_t* src_valid,
                  int64_t n, const double* pose, float tau, double kappa, double* H, double* g, int32_t* corr,
                  int64_t* n_corr, int64_t* n_p2p, double* chi2) {
    std::vector<SourcePoint> src((size_t)n);
    for (int64_t i = 0; i < n; ++i) {
        for (int a = 0; a < 3; ++a) { src[i].sf[a] = src_xyz[3 * i + a]; src[i].s[a] = src_xyz[3 * i + a]; }
        std::memcpy(src[i].cov, src_cov + 6 * i, 6 * sizeof(double));
        src[i].valid = src_valid[i];
        src[i].index = i;
    }
    float tau2 = tau * tau;
    double A[3];
    Frame fr = anchor_frame(*m, pose, A);
    LinResult L = linearize(*m, src, pose, fr, A, tau2, kappa, corr);
    std::memcpy(H, L.H, sizeof(L.H));
    std::memcpy(g, L.g, sizeof(L.g));
    *n_corr = L.n_corr;
    *n_p2p = L.n_p2p;
    *chi2 = L.chi2;
}

// Threads of the per-point loops (1 = sequential); returns the value in effect.
int om_set_threads(int n) {
    g_threads = n < 1 ? 1 : (n > 256 ? 256 : n);
    return g_threads;
}

void om_se3_exp(const double* xi, double* T) { se3_exp(xi, T); }
void om_se3_log(const double* T, double* xi) { se3_log(T, xi); }

// Gauss-Newton step (solve H xi = -g by Cholesky, T <- exp(xi) T). Returns 0, or 5 if H is not PD.
int om_gn_step(const double* H, const double* g, const double* T, double* xi_out, double* T_out) {
    double Lc[36];
    if (!cholesky6(H, Lc)) return 5;
    double mg[6];
    for (int i = 0; i < 6; ++i) mg[i] = -g[i];
    cholesky6_solve(Lc, mg, xi_out);
    double E[16];
    se3_exp(xi_out, E);
    mat4_mul(E, T, T_out);
    return 0;
}

// Full registration (Sec. III-A.2): scan-local map, source covariances, then
// Gauss-Newton iterations until ||xi|| <= conv_eps or max_iters.
// out_cov = H^-1 of the last linearisation, ordered [rotation; translation], about the anchor.
int om_register(const OracleMap* m, const float* xyz, int64_t n, const double* init, const om_reg_params* prm,
                double* out_pose, double* out_cov, om_reg_stats* st) {
    std::vector<SourcePoint> src = scan_local_sources(xyz, n, m->v, m->nmax, m->k, m->dmin2, nullptr);
    double T[16];
    std::memcpy(T, init, sizeof(T));
    float tau2 = prm->tau * prm->tau;
    st->iters = 0;
    st->n_src = (uint32_t)src.size();
    st->n_corr = 0;
    st->n_p2p = 0;
    st->converged = 0;
    st->status = 0;
    st->chi2 = 0;
    double Hlast[36] = {0};
    bool have_h = false;
    double A[3];
    const Frame fr = anchor_frame(*m, init, A);
    for (uint32_t it = 0; it < prm->max_iters; ++it) {
        LinResult L = linearize(*m, src, T, fr, A, tau2, prm->kappa, nullptr);
        st->n_corr = (uint32_t)L.n_corr;
        st->n_p2p = (uint32_t)L.n_p2p;
        st->chi2 = L.chi2;
        if (L.n_corr < 6) { st->status = 5; break; }
        double Lc[36];
        if (!cholesky6(L.H, Lc)) { st->status = 5; break; }
        std::memcpy(Hlast, L.H, sizeof(Hlast));
        have_h = true;
        double mg[6], xi[6];
        for (int i = 0; i < 6; ++i) mg[i] = -L.g[i];
        cholesky6_solve(Lc, mg, xi);
        apply_update(xi, A, T);  // Eq. 6: the increment is applied on the left, about the anchor
        st->iters = it + 1;
        // termination reading: ||[phi; rho + phi x c]|| <= conv_eps, the increment expressed at the
        // initial sensor position c (relative to the anchor), i.e. in the frame of the LiDAR whose
        // transform the test is about, not at the world origin
        double c[3] = {init[3] - A[0], init[7] - A[1], init[11] - A[2]};
        double r[3] = {xi[3] + (xi[1] * c[2] - xi[2] * c[1]), xi[4] + (xi[2] * c[0] - xi[0] * c[2]),
                       xi[5] + (xi[0] * c[1] - xi[1] * c[0])};
        double nx = xi[0] * xi[0] + xi[1] * xi[1] + xi[2] * xi[2] + r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
        if (std::sqrt(nx) <= prm->conv_eps) { st->converged = 1; break; }
    }
    std::memcpy(out_pose, T, sizeof(T));
    if (out_cov) {
        std::memset(out_cov, 0, 36 * sizeof(double));
        double Lc[36];
        if (have_h && cholesky6(Hlast, Lc)) {
            for (int c = 0; c < 6; ++c) {
                double e[6] = {0}, x[6];
                e[c] = 1.0;
                cholesky6_solve(Lc, e, x);
                for (int r = 0; r < 6; ++r) out_cov[6 * r + c] = x[r];
            }
        }
    }
    return st->status;
}

// Adaptive correspondence threshold (reading of the scheme the paper adopts from
// KISS-ICP): sigma = sqrt(mean of delta^2 over recorded frames) or sigma0 with no
// record; tau = 3 sigma, kappa = sigma / 3. A frame is recorded when the
// translation of the model deviation init^-1 * result exceeds min_motion;
// delta = 2 r_max sin(theta / 2) + ||dt||.
struct OracleThreshold {
    double sigma0, min_motion, r_max, sse;
    int64_t n;
};
OracleThreshold* om_thr_create(double sigma0, double min_motion, double r_max) {
    return new OracleThreshold{sigma0, min_motion, r_max, 0.0, 0};
}
void om_thr_destroy(OracleThreshold* t) { delete t; }
void om_thr_get(const OracleThreshold* t, double* tau, double* kappa) {
    double sigma = (t->n > 0) ? std::sqrt(t->sse / (double)t->n) : t->sigma0;
    *tau = 3.0 * sigma;
    *kappa = sigma / 3.0;
}
void om_thr_update(OracleThreshold* t, const double* init, const double* result) {
    double Ii[16], D[16];
    rigid_inverse(init, Ii);
    mat4_mul(Ii, result, D);
    double tr = D[0] + D[5] + D[10];
    double c = std::max(-1.0, std::min(1.0, 0.5 * (tr - 1.0)));
    double th = std::acos(c);
    double dt = std::sqrt(D[3] * D[3] + D[7] * D[7] + D[11] * D[11]);
    double delta = 2.0 * t->r_max * std::sin(0.5 * th) + dt;
    if (dt > t->min_motion) {
        t->sse += delta * delta;
        t->n += 1;
    }
}

}  // extern "C"
