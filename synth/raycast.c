/*
 * Seeded synthetic spinning-LiDAR ray caster (input generator only).
 *
 * This file produces the synthetic scans that stand in for the paper's
 * datasets (KITTI, MulRan, the racing recordings), which are not available.
 * It holds none of the registration method's arithmetic: it intersects rays
 * with a few analytic primitives and adds Gaussian range noise.
 *
 * Scene primitives are packed 10 doubles each: [kind, p0 .. p8].
 *   kind 1  vertical wall segment   x0 y0 x1 y1 zlo zhi
 *   kind 2  vertical wall arc       cx cy radius a0 a1 zlo zhi   (a0 <= a1, radians, CCW)
 *   kind 3  vertical pole           cx cy radius zlo zhi
 *   kind 4  box with yaw            cx cy cz hx hy hz yaw
 * The ground plane z = 0 is always present.
 *
 * Noise is counter based (splitmix64 of seed, scan id and ray index, then
 * Box-Muller), so the output does not depend on the thread count.
 * Points are returned in the sensor frame, in azimuth-major ray order
 * (ray index = azimuth_bin * beams + beam), misses removed.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define PRIM_STRIDE 10
enum { PRIM_SEG = 1, PRIM_ARC = 2, PRIM_CYL = 3, PRIM_BOX = 4 };

static uint64_t mix64(uint64_t x) {
    /* splitmix64 finaliser (Steele, Lea, Flood 2014) */
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}

static double unit_open(uint64_t bits) {
    /* 53 random bits -> (0, 1] */
    return ((double)(bits >> 11) + 1.0) * (1.0 / 9007199254740992.0);
}

static double gauss(uint64_t seed, uint64_t scan_id, uint64_t ray) {
    uint64_t h = mix64(seed ^ mix64(scan_id ^ mix64(ray)));
    double u1 = unit_open(h);
    double u2 = unit_open(mix64(h));
    return sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
}

static double cross2(double ax, double ay, double bx, double by) { return ax * by - ay * bx; }

static int angle_in(double a, double a0, double a1) {
    const double two_pi = 6.283185307179586;
    while (a < a0) a += two_pi;
    while (a > a0 + two_pi) a -= two_pi;
    return a <= a1;
}

/* nearest hit distance along the unit ray o + t d, or INFINITY */
static double hit_prim(const double* p, const double o[3], const double d[3]) {
    int kind = (int)p[0];
    double best = INFINITY;
    if (kind == PRIM_SEG) {
        double ex = p[3] - p[1], ey = p[4] - p[2];
        double den = cross2(d[0], d[1], ex, ey);
        if (fabs(den) < 1e-12) return best;
        double wx = p[1] - o[0], wy = p[2] - o[1];
        double t = cross2(wx, wy, ex, ey) / den;
        double u = cross2(wx, wy, d[0], d[1]) / den;
        if (t > 0.0 && u >= 0.0 && u <= 1.0) {
            double z = o[2] + t * d[2];
            if (z >= p[5] && z <= p[6]) best = t;
        }
    } else if (kind == PRIM_ARC || kind == PRIM_CYL) {
        double fx = o[0] - p[1], fy = o[1] - p[2], r = p[3];
        double a = d[0] * d[0] + d[1] * d[1];
        if (a < 1e-18) return best;
        double b = 2.0 * (fx * d[0] + fy * d[1]);
        double c = fx * fx + fy * fy - r * r;
        double disc = b * b - 4.0 * a * c;
        if (disc < 0.0) return best;
        double sq = sqrt(disc);
        double ts[2] = {(-b - sq) / (2.0 * a), (-b + sq) / (2.0 * a)};
        double zlo = (kind == PRIM_ARC) ? p[6] : p[4];
        double zhi = (kind == PRIM_ARC) ? p[7] : p[5];
        int nroots = (kind == PRIM_CYL) ? 1 : 2; /* a pole is only hit from outside */
        for (int i = 0; i < nroots; ++i) {
            double t = ts[i];
            if (t <= 0.0) continue;
            double z = o[2] + t * d[2];
            if (z < zlo || z > zhi) continue;
            if (kind == PRIM_ARC) {
                double ang = atan2(o[1] + t * d[1] - p[2], o[0] + t * d[0] - p[1]);
                if (!angle_in(ang, p[4], p[5])) continue;
            }
            best = t;
            break;
        }
    } else if (kind == PRIM_BOX) {
        double cy = cos(p[7]), sy = sin(p[7]);
        double rx = o[0] - p[1], ry = o[1] - p[2], rz = o[2] - p[3];
        double lo[3] = {cy * rx + sy * ry, -sy * rx + cy * ry, rz};
        double ld[3] = {cy * d[0] + sy * d[1], -sy * d[0] + cy * d[1], d[2]};
        double h[3] = {p[4], p[5], p[6]};
        double tmin = -INFINITY, tmax = INFINITY;
        for (int k = 0; k < 3; ++k) {
            if (fabs(ld[k]) < 1e-15) {
                if (lo[k] < -h[k] || lo[k] > h[k]) return best;
            } else {
                double t1 = (-h[k] - lo[k]) / ld[k], t2 = (h[k] - lo[k]) / ld[k];
                if (t1 > t2) { double tt = t1; t1 = t2; t2 = tt; }
                if (t1 > tmin) tmin = t1;
                if (t2 < tmax) tmax = t2;
            }
        }
        if (tmax >= tmin && tmin > 0.0) best = tmin;
    }
    return best;
}

static void prim_bound(const double* p, double* cx, double* cy, double* rad) {
    int kind = (int)p[0];
    if (kind == PRIM_SEG) {
        *cx = 0.5 * (p[1] + p[3]); *cy = 0.5 * (p[2] + p[4]);
        *rad = 0.5 * hypot(p[3] - p[1], p[4] - p[2]);
    } else if (kind == PRIM_ARC || kind == PRIM_CYL) {
        *cx = p[1]; *cy = p[2]; *rad = p[3];
    } else {
        *cx = p[1]; *cy = p[2]; *rad = hypot(p[4], p[5]);
    }
}

/*
 * Cast beams x az_bins rays from the sensor at `pose` (row-major 4x4, sensor
 * to world) and write hits as sensor-frame float xyz into out_xyz (room for
 * beams*az_bins points). Returns the number of points written.
 */
int64_t synth_raycast(const double* prims, int64_t nprims, const double* pose,
                      int32_t beams, int32_t az_bins, double el_min_deg, double el_max_deg,
                      double r_min, double r_max, double sigma, uint64_t seed, uint64_t scan_id,
                      float* out_xyz, int32_t nthreads) {
    const double deg = 3.14159265358979323846 / 180.0;
    int64_t nrays = (int64_t)beams * az_bins;
    double o[3] = {pose[3], pose[7], pose[11]};

    /* cull primitives out of reach of this sensor position */
    int64_t* keep = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nprims > 0 ? nprims : 1));
    int64_t nkeep = 0;
    for (int64_t i = 0; i < nprims; ++i) {
        double cx, cy, rad;
        prim_bound(prims + i * PRIM_STRIDE, &cx, &cy, &rad);
        if (hypot(cx - o[0], cy - o[1]) - rad <= r_max) keep[nkeep++] = i;
    }

    float* tmp = (float*)malloc(sizeof(float) * 3 * (size_t)nrays);
    unsigned char* hit = (unsigned char*)malloc((size_t)nrays);

#pragma omp parallel for num_threads(nthreads > 0 ? nthreads : 1) schedule(static)
    for (int32_t a = 0; a < az_bins; ++a) {
        double az = 2.0 * 3.14159265358979323846 * (double)a / (double)az_bins;
        for (int32_t b = 0; b < beams; ++b) {
            int64_t ray = (int64_t)a * beams + b;
            double el = (beams > 1) ? (el_min_deg + (el_max_deg - el_min_deg) * (double)b / (double)(beams - 1)) * deg
                                    : el_min_deg * deg;
            double ds[3] = {cos(el) * cos(az), cos(el) * sin(az), sin(el)};
            double dw[3];
            for (int k = 0; k < 3; ++k)
                dw[k] = pose[4 * k + 0] * ds[0] + pose[4 * k + 1] * ds[1] + pose[4 * k + 2] * ds[2];
            double best = INFINITY;
            if (dw[2] < -1e-12) best = -o[2] / dw[2];
            for (int64_t j = 0; j < nkeep; ++j) {
                double t = hit_prim(prims + keep[j] * PRIM_STRIDE, o, dw);
                if (t < best) best = t;
            }
            hit[ray] = 0;
            if (best >= r_min && best <= r_max) {
                double rng = best + sigma * gauss(seed, scan_id, (uint64_t)ray);
                if (rng > 0.0) {
                    tmp[3 * ray + 0] = (float)(ds[0] * rng);
                    tmp[3 * ray + 1] = (float)(ds[1] * rng);
                    tmp[3 * ray + 2] = (float)(ds[2] * rng);
                    hit[ray] = 1;
                }
            }
        }
    }
    int64_t n = 0;
    for (int64_t r = 0; r < nrays; ++r) {
        if (!hit[r]) continue;
        memcpy(out_xyz + 3 * n, tmp + 3 * r, 3 * sizeof(float));
        ++n;
    }
    free(tmp);
    free(hit);
    free(keep);
    return n;
}


/*
 * A spinning sweep with motion: azimuth column a is fired from the sensor pose
 * poses[16 a .. 16 a + 15] (row-major 4x4, sensor to world) and its hits are written
 * in that pose's sensor frame, with the column index in out_col. Primitives are culled
 * around the first and last poses with r_max + reach. Same noise stream as
 * synth_raycast (seed, scan id, ray index).
 */
int64_t synth_raycast_columns(const double* prims, int64_t nprims, const double* poses, double reach,
                              int32_t beams, int32_t az_bins, double el_min_deg, double el_max_deg,
                              double r_min, double r_max, double sigma, uint64_t seed, uint64_t scan_id,
                              float* out_xyz, int32_t* out_col, int32_t nthreads) {
    const double deg = 3.14159265358979323846 / 180.0;
    int64_t nrays = (int64_t)beams * az_bins;
    const double* last = poses + 16 * (int64_t)(az_bins - 1);
    int64_t* keep = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nprims > 0 ? nprims : 1));
    int64_t nkeep = 0;
    for (int64_t i = 0; i < nprims; ++i) {
        double cx, cy, rad;
        prim_bound(prims + i * PRIM_STRIDE, &cx, &cy, &rad);
        if (hypot(cx - last[3], cy - last[7]) - rad <= r_max + reach ||
            hypot(cx - poses[3], cy - poses[7]) - rad <= r_max + reach)
            keep[nkeep++] = i;
    }
    float* tmp = (float*)malloc(sizeof(float) * 3 * (size_t)nrays);
    unsigned char* hit = (unsigned char*)malloc((size_t)nrays);

#pragma omp parallel for num_threads(nthreads > 0 ? nthreads : 1) schedule(static)
    for (int32_t a = 0; a < az_bins; ++a) {
        const double* pose = poses + 16 * (int64_t)a;
        double o[3] = {pose[3], pose[7], pose[11]};
        double az = 2.0 * 3.14159265358979323846 * (double)a / (double)az_bins;
        for (int32_t b = 0; b < beams; ++b) {
            int64_t ray = (int64_t)a * beams + b;
            double el = (beams > 1) ? (el_min_deg + (el_max_deg - el_min_deg) * (double)b / (double)(beams - 1)) * deg
                                    : el_min_deg * deg;
            double ds[3] = {cos(el) * cos(az), cos(el) * sin(az), sin(el)};
            double dw[3];
            for (int k = 0; k < 3; ++k)
                dw[k] = pose[4 * k + 0] * ds[0] + pose[4 * k + 1] * ds[1] + pose[4 * k + 2] * ds[2];
            double best = INFINITY;
            if (dw[2] < -1e-12) best = -o[2] / dw[2];
            for (int64_t j = 0; j < nkeep; ++j) {
                double t = hit_prim(prims + keep[j] * PRIM_STRIDE, o, dw);
                if (t < best) best = t;
            }
            hit[ray] = 0;
            if (best >= r_min && best <= r_max) {
                double rng = best + sigma * gauss(seed, scan_id, (uint64_t)ray);
                if (rng > 0.0) {
                    tmp[3 * ray + 0] = (float)(ds[0] * rng);
                    tmp[3 * ray + 1] = (float)(ds[1] * rng);
                    tmp[3 * ray + 2] = (float)(ds[2] * rng);
                    hit[ray] = 1;
                }
            }
        }
    }
    int64_t n = 0;
    for (int64_t r = 0; r < nrays; ++r) {
        if (!hit[r]) continue;
        memcpy(out_xyz + 3 * n, tmp + 3 * r, 3 * sizeof(float));
        out_col[n] = (int32_t)(r / beams);
        ++n;
    }
    free(tmp);
    free(hit);
    free(keep);
    return n;
}
