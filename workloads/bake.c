/*
 * bake.c -- scene construction for the seeded synthetic workloads.
 *
 * Evaluates the exact Euclidean signed distance of a union of analytic
 * primitives (sphere, axis-aligned box, capsule, ground half-space) at the
 * voxel centres of a volume, and the index of the primitive that attains the
 * minimum (ties go to the lowest index). This is input generation only: it
 * holds no step of the probe update, and both the CUDA path and the oracle
 * consume its output arrays as data.
 *
 * Bricks of 8^3 voxels cull primitives that cannot attain the minimum: with
 * every primitive inside a ball (c_k, R_k), sdf_k(x) >= |x - c_k| - R_k, so a
 * primitive whose lower bound over the brick exceeds the smallest upper bound
 * sdf_j(centre) + half-diagonal is skipped. The culled result is exactly the
 * brute-force minimum.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

enum { P_SPHERE = 0, P_BOX = 1, P_CAPSULE = 2, P_PLANE_Y = 3, P_INV_SPHERE = 4 };

static double prim_sdf(int type, const double* q, const double p[3]) {
    switch (type) {
        case P_SPHERE: {
            double dx = p[0] - q[0], dy = p[1] - q[1], dz = p[2] - q[2];
            return sqrt(dx * dx + dy * dy + dz * dz) - q[3];
        }
        case P_BOX: {
            double d[3], outside = 0.0, inside = -1e300;
            for (int a = 0; a < 3; ++a) {
                d[a] = fabs(p[a] - q[a]) - q[3 + a];
                double m = d[a] > 0.0 ? d[a] : 0.0;
                outside += m * m;
                if (d[a] > inside) inside = d[a];
            }
            return sqrt(outside) + (inside < 0.0 ? inside : 0.0);
        }
        case P_CAPSULE: {
            double pa[3], ba[3], dot_pb = 0.0, dot_bb = 0.0;
            for (int a = 0; a < 3; ++a) {
                pa[a] = p[a] - q[a];
                ba[a] = q[3 + a] - q[a];
                dot_pb += pa[a] * ba[a];
                dot_bb += ba[a] * ba[a];
            }
            double s = dot_bb > 0.0 ? dot_pb / dot_bb : 0.0;
            s = s < 0.0 ? 0.0 : (s > 1.0 ? 1.0 : s);
            double e = 0.0;
            for (int a = 0; a < 3; ++a) {
                double v = pa[a] - s * ba[a];
                e += v * v;
            }
            return sqrt(e) - q[6];
        }
        case P_INV_SPHERE: { /* solid everywhere outside the ball: a hollow spherical room */
            double dx = p[0] - q[0], dy = p[1] - q[1], dz = p[2] - q[2];
            return q[3] - sqrt(dx * dx + dy * dy + dz * dz);
        }
        case P_PLANE_Y:
        default:
            return p[1] - q[0];
    }
}

/* Bounding ball of a primitive; returns 0 for the unbounded half-space. */
static int prim_ball(int type, const double* q, double c[3], double* R) {
    switch (type) {
        case P_SPHERE:
            c[0] = q[0]; c[1] = q[1]; c[2] = q[2];
            *R = q[3];
            return 1;
        case P_BOX:
            c[0] = q[0]; c[1] = q[1]; c[2] = q[2];
            *R = sqrt(q[3] * q[3] + q[4] * q[4] + q[5] * q[5]);
            return 1;
        case P_CAPSULE: {
            double l = 0.0;
            for (int a = 0; a < 3; ++a) {
                c[a] = 0.5 * (q[a] + q[3 + a]);
                l += (q[3 + a] - q[a]) * (q[3 + a] - q[a]);
            }
            *R = 0.5 * sqrt(l) + q[6];
            return 1;
        }
        default:
            return 0;
    }
}

/* Exact union SDF (and owner) at n arbitrary world points, brute force. */
void wl_eval(int n_prim, const int32_t* types, const double* params, int64_t n, const double* pts,
             double* sdf, int32_t* owner) {
    for (int64_t i = 0; i < n; ++i) {
        double best = 1e300;
        int32_t arg = -1;
        for (int k = 0; k < n_prim; ++k) {
            double v = prim_sdf(types[k], params + 8 * k, pts + 3 * i);
            if (v < best) {
                best = v;
                arg = k;
            }
        }
        sdf[i] = best;
        if (owner) owner[i] = arg;
    }
}

static uint16_t double_to_half_rtz(double x) {
    uint16_t s = x < 0.0 ? 0x8000 : 0;
    double a = fabs(x);
    if (a >= 65504.0) return s | 0x7bff;
    if (a < ldexp(1.0, -14)) return s | (uint16_t)floor(a * 16777216.0); /* subnormal: units of 2^-24 */
    int E;
    double f = frexp(a, &E); /* a = f 2^E, f in [0.5, 1) */
    int e = E - 1;
    double m = floor((2.0 * f - 1.0) * 1024.0);
    return s | (uint16_t)(((e + 15) << 10) | (int)m);
}

/* Bake: voxel (x,y,z) centre = origin + (x+1/2, y+1/2, z+1/2) h, arrays [z][y][x].
 * Any of sdf64 / sdf32 / sdf16_rtz / owner may be NULL. float32 is rounded to
 * nearest; binary16 is rounded toward zero so that it never overstates a distance. */
void wl_bake(int nx, int ny, int nz, double h, const double origin[3], int n_prim, const int32_t* types,
             const double* params, double* sdf64, float* sdf32, uint16_t* sdf16_rtz, int32_t* owner,
             int n_threads) {
    const int B = 8;
    const int bx = (nx + B - 1) / B, by = (ny + B - 1) / B, bz = (nz + B - 1) / B;
    double* ball = (double*)malloc(sizeof(double) * 4 * (n_prim > 0 ? n_prim : 1));
    int* bounded = (int*)malloc(sizeof(int) * (n_prim > 0 ? n_prim : 1));
    for (int k = 0; k < n_prim; ++k) bounded[k] = prim_ball(types[k], params + 8 * k, ball + 4 * k, ball + 4 * k + 3);
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#pragma omp parallel
#endif
    {
        int* list = (int*)malloc(sizeof(int) * (n_prim > 0 ? n_prim : 1));
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 4)
#endif
        for (long b = 0; b < (long)bx * by * bz; ++b) {
            int ix = (int)(b % bx), iy = (int)((b / bx) % by), iz = (int)(b / ((long)bx * by));
            int x0 = ix * B, y0 = iy * B, z0 = iz * B;
            int x1 = x0 + B < nx ? x0 + B : nx, y1 = y0 + B < ny ? y0 + B : ny, z1 = z0 + B < nz ? z0 + B : nz;
            double lo[3] = {origin[0] + (x0 + 0.5) * h, origin[1] + (y0 + 0.5) * h, origin[2] + (z0 + 0.5) * h};
            double hi[3] = {origin[0] + (x1 - 0.5) * h, origin[1] + (y1 - 0.5) * h, origin[2] + (z1 - 0.5) * h};
            double c[3], half = 0.0;
            for (int a = 0; a < 3; ++a) {
                c[a] = 0.5 * (lo[a] + hi[a]);
                half += 0.25 * (hi[a] - lo[a]) * (hi[a] - lo[a]);
            }
            half = sqrt(half) * (1.0 + 1e-12) + 1e-12;
            double ub = 1e300;
            for (int k = 0; k < n_prim; ++k) {
                double v = prim_sdf(types[k], params + 8 * k, c) + half;
                if (v < ub) ub = v;
            }
            int nl = 0;
            for (int k = 0; k < n_prim; ++k) {
                if (bounded[k]) {
                    double dx = c[0] - ball[4 * k], dy = c[1] - ball[4 * k + 1], dz = c[2] - ball[4 * k + 2];
                    double lb = sqrt(dx * dx + dy * dy + dz * dz) - half - ball[4 * k + 3];
                    if (lb > ub) continue;
                }
                list[nl++] = k;
            }
            for (int z = z0; z < z1; ++z)
                for (int y = y0; y < y1; ++y)
                    for (int x = x0; x < x1; ++x) {
                        double p[3] = {origin[0] + (x + 0.5) * h, origin[1] + (y + 0.5) * h, origin[2] + (z + 0.5) * h};
                        double best = 1e300;
                        int32_t arg = -1;
                        for (int j = 0; j < nl; ++j) {
                            double v = prim_sdf(types[list[j]], params + 8 * list[j], p);
                            if (v < best) {
                                best = v;
                                arg = list[j];
                            }
                        }
                        size_t i = ((size_t)z * ny + y) * nx + x;
                        if (sdf64) sdf64[i] = best;
                        if (sdf32) sdf32[i] = (float)best;
                        if (sdf16_rtz) sdf16_rtz[i] = double_to_half_rtz(best);
                        if (owner) owner[i] = arg;
                    }
        }
        free(list);
    }
    free(ball);
    free(bounded);
}
