/*
 * oracle.c -- FP64 CPU oracle of the SDFDDGI per-frame probe update.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing on the product path loads this file: the
 * tests, the smoke check and the bench's CPU-baseline leg do. It is the plain
 * definition of what the CUDA library must compute, written from the paper
 * (Hu et al., "Signed Distance Fields Dynamic Diffuse Global Illumination",
 * arXiv 2007.14394) in double precision, probe by probe, ray by ray, texel by
 * texel, in the order of Sec. 3.3: trace the probe's rays, shade the hits,
 * then let every octahedral texel gather its cosine-weighted irradiance from
 * all of the probe's samples (Eq. 3) and mix it temporally with the last frame.
 *
 * Where the paper is silent, each function states the reading it takes (ray
 * set, trace termination, octahedral map and border, shading terms, temporal
 * mixing). Parity pins: every function here is checked in
 * tests/test_oracle_pins.py against closed forms, invariants or brute force
 * (no pin retypes a formula from this file).
 *
 * Independence from the implementation under test: the oracle may be told the
 * other side's DISCRETE outcomes of a ray (exit event, step count, light
 * visibility, owning primitive) and follows one only where its own FP64
 * decision lies within a stated rounding band of the threshold. It never takes
 * a continuous value (a distance, a radiance) from the other side.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define IRR_N 6   /* interior texels per side of an irradiance map (8x8 with border) */
#define DEP_N 14  /* interior texels per side of a depth-moment map (16x16 with border) */
#define IRR_T (IRR_N + 2)
#define DEP_T (DEP_N + 2)
#define HUGE_MARGIN 1e300

static const double kPi = 3.14159265358979323846;

/* ---------------------------------------------------------------- helpers */

static double half_to_double(uint16_t b) {
    int s = (b >> 15) & 1, e = (b >> 10) & 31, m = b & 1023;
    double v;
    if (e == 0)
        v = ldexp((double)m, -24);
    else if (e == 31)
        v = m ? NAN : INFINITY;
    else
        v = ldexp((double)(1024 + m), e - 25);
    return s ? -v : v;
}

static double dot3(const double a[3], const double b[3]) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

static double sign_nz(double x) { return x >= 0.0 ? 1.0 : -1.0; }

static double clampd(double x, double lo, double hi) { return x < lo ? lo : (x > hi ? hi : x); }

/* ------------------------------------------- ray directions (Sec. 3.3, O2) */

/* Spherical Fibonacci point i of n: z = 1 - (2i+1)/n, azimuth = 2 pi frac(i * phi^-1)
 * with the golden fraction taken in 32-bit fixed point, (i * 2654435769) mod 2^32 / 2^32,
 * so that both implementations start from the same exact phase. */
void oracle_sf_dir(int32_t i, int32_t n, double out[3]) {
    double z = 1.0 - (2.0 * i + 1.0) / n;
    uint32_t phase = (uint32_t)((uint64_t)(uint32_t)i * 2654435769ull);
    double phi = 2.0 * kPi * ((double)phase / 4294967296.0);
    double r = sqrt(fmax(0.0, 1.0 - z * z));
    out[0] = r * cos(phi);
    out[1] = r * sin(phi);
    out[2] = z;
}

/* ------------------------------------------------ octahedral map (O7, Sec. 3.3) */

void oracle_oct_encode(const double v[3], double uv[2]) {
    double l1 = fabs(v[0]) + fabs(v[1]) + fabs(v[2]);
    double qx = v[0] / l1, qy = v[1] / l1;
    if (v[2] < 0.0) {
        double ox = (1.0 - fabs(qy)) * sign_nz(qx);
        double oy = (1.0 - fabs(qx)) * sign_nz(qy);
        qx = ox;
        qy = oy;
    }
    uv[0] = 0.5 * (qx + 1.0);
    uv[1] = 0.5 * (qy + 1.0);
}

void oracle_oct_decode(const double uv[2], double v[3]) {
    double qx = 2.0 * uv[0] - 1.0, qy = 2.0 * uv[1] - 1.0;
    double z = 1.0 - fabs(qx) - fabs(qy);
    double x = qx, y = qy;
    if (z < 0.0) {
        x = (1.0 - fabs(qy)) * sign_nz(qx);
        y = (1.0 - fabs(qx)) * sign_nz(qy);
    }
    double len = sqrt(x * x + y * y + z * z);
    v[0] = x / len;
    v[1] = y / len;
    v[2] = z / len;
}

/* ------------------------------------------------ volume sampling (O1, O4) */

static double voxel_sdf(const or_volume* vol, int x, int y, int z) {
    size_t i = ((size_t)z * vol->ny + y) * vol->nx + x;
    if (vol->sdf_dtype == 1) return half_to_double(((const uint16_t*)vol->sdf)[i]);
    return (double)((const float*)vol->sdf)[i];
}

/* Trilinear cell and weights of world point p: voxel centres sit at integer
 * coordinates g = (p - origin)/h - 1/2; the cell is clamped to the volume
 * (clamp-to-edge) and the fractions to [0, 1]. */
static void trilinear_cell(const or_volume* vol, const double p[3], int i0[3], double f[3]) {
    const int n[3] = {vol->nx, vol->ny, vol->nz};
    for (int a = 0; a < 3; ++a) {
        double g = (p[a] - vol->origin[a]) / vol->h - 0.5;
        int i = (int)floor(g);
        if (i < 0) i = 0;
        if (i > n[a] - 2) i = n[a] - 2;
        i0[a] = i;
        f[a] = clampd(g - i, 0.0, 1.0);
    }
}

/* Exact Euclidean distance to one primitive (negative inside). */
static double prim_distance(const or_prim* q, const double x[3]) {
    const double* a = q->p;
    switch (q->type) {
        case 0: { /* sphere */
            double v[3] = {x[0] - a[0], x[1] - a[1], x[2] - a[2]};
            return sqrt(dot3(v, v)) - a[3];
        }
        case 1: { /* box: distance outside, largest (negative) face distance inside */
            double e[3], out2 = 0.0, in = -HUGE_VAL;
            for (int k = 0; k < 3; ++k) {
                e[k] = fabs(x[k] - a[k]) - a[3 + k];
                if (e[k] > 0.0) out2 += e[k] * e[k];
                in = fmax(in, e[k]);
            }
            return sqrt(out2) + fmin(in, 0.0);
        }
        case 2: { /* capsule: distance to the segment minus the radius */
            double ab[3] = {a[3] - a[0], a[4] - a[1], a[5] - a[2]};
            double ax[3] = {x[0] - a[0], x[1] - a[1], x[2] - a[2]};
            double L2 = dot3(ab, ab);
            double s = L2 > 0.0 ? clampd(dot3(ax, ab) / L2, 0.0, 1.0) : 0.0;
            double r[3] = {ax[0] - s * ab[0], ax[1] - s * ab[1], ax[2] - s * ab[2]};
            return sqrt(dot3(r, r)) - a[6];
        }
        case 3: /* solid below y = a[0] */
            return x[1] - a[0];
        case 4: { /* solid outside the ball */
            double v[3] = {x[0] - a[0], x[1] - a[1], x[2] - a[2]};
            return a[3] - sqrt(dot3(v, v));
        }
        default:
            return HUGE_VAL;
    }
}

double oracle_analytic_sdf(const or_volume* vol, const double p[3], int32_t* owner, double* second) {
    double best = HUGE_VAL, next = HUGE_VAL;
    int32_t arg = -1;
    for (int32_t k = 0; k < vol->n_prims; ++k) {
        const double d = prim_distance(&vol->prims[k], p);
        if (d < best) {
            next = best;
            best = d;
            arg = k;
        } else if (d < next) {
            next = d;
        }
    }
    if (owner) *owner = arg;
    if (second) *second = next;
    return best;
}

double oracle_sample_sdf(const or_volume* vol, const double p[3]) {
    if (vol->n_prims > 0) return oracle_analytic_sdf(vol, p, NULL, NULL);
    int i0[3];
    double f[3];
    trilinear_cell(vol, p, i0, f);
    double acc = 0.0;
    for (int c = 0; c < 8; ++c) {
        int dx = c & 1, dy = (c >> 1) & 1, dz = (c >> 2) & 1;
        double w = (dx ? f[0] : 1.0 - f[0]) * (dy ? f[1] : 1.0 - f[1]) * (dz ? f[2] : 1.0 - f[2]);
        acc += w * voxel_sdf(vol, i0[0] + dx, i0[1] + dy, i0[2] + dz);
    }
    return acc;
}

/* Albedo and emission at p: the material volume sampled with the same trilinear rule
 * (analytic scenes take the nearest primitive's material, in shade_at). */
static void sample_material(const or_volume* vol, const double p[3], double albedo[3], double emission[3]) {
    for (int k = 0; k < 3; ++k) albedo[k] = emission[k] = 0.0;
    if (!vol->material) return;
    int i0[3];
    double f[3];
    trilinear_cell(vol, p, i0, f);
    for (int c = 0; c < 8; ++c) {
        int dx = c & 1, dy = (c >> 1) & 1, dz = (c >> 2) & 1;
        double w = (dx ? f[0] : 1.0 - f[0]) * (dy ? f[1] : 1.0 - f[1]) * (dz ? f[2] : 1.0 - f[2]);
        size_t v = ((size_t)(i0[2] + dz) * vol->ny + (i0[1] + dy)) * vol->nx + (i0[0] + dx);
        const uint16_t* m = vol->material + 8 * v;
        for (int k = 0; k < 3; ++k) {
            albedo[k] += w * half_to_double(m[k]);
            emission[k] += w * half_to_double(m[4 + k]);
        }
    }
}

/* ------------------------------------------------ sphere trace (Sec. 3.3, O6) */

static double g_delta_vox = 2e-4; /* rounding band of distance decisions, voxels */
static double g_delta_cos = 1e-4; /* rounding band of light-gating decisions */

void oracle_set_delta(double delta_vox, double delta_cos) {
    g_delta_vox = delta_vox;
    g_delta_cos = delta_cos;
}

/* Derivative of the trilinear field along d at p (world units); zero across clamped axes. */
static double sdf_slope(const or_volume* vol, const double p[3], const double d[3]) {
    if (vol->n_prims > 0) { /* analytic: central difference of the exact field along d */
        const double e = 1e-6 * vol->h;
        double pp[3], pm[3];
        for (int a = 0; a < 3; ++a) {
            pp[a] = p[a] + e * d[a];
            pm[a] = p[a] - e * d[a];
        }
        return (oracle_analytic_sdf(vol, pp, NULL, NULL) - oracle_analytic_sdf(vol, pm, NULL, NULL)) / (2.0 * e);
    }
    int i0[3];
    double f[3], grad[3] = {0.0, 0.0, 0.0};
    trilinear_cell(vol, p, i0, f);
    for (int c = 0; c < 8; ++c) {
        int e[3] = {c & 1, (c >> 1) & 1, (c >> 2) & 1};
        double v = voxel_sdf(vol, i0[0] + e[0], i0[1] + e[1], i0[2] + e[2]);
        for (int a = 0; a < 3; ++a) {
            double w = e[a] ? 1.0 : -1.0;
            for (int b = 0; b < 3; ++b)
                if (b != a) w *= e[b] ? f[b] : 1.0 - f[b];
            grad[a] += w * v;
        }
    }
    return (grad[0] * d[0] + grad[1] * d[1] + grad[2] * d[2]) / vol->h;
}

/* Sphere tracing (Hart 1996) as the probe update uses it: step by the sampled
 * distance until it falls below eps (HIT), the point leaves the volume box
 * (LEFT_VOLUME) or t passes the limit (PAST_LIMIT), or the step budget runs out
 * (EXHAUSTED). `margin` is the closest any of these tests came to the other
 * outcome. With fe >= 0 the path follows the given event (fe) and step count (fs)
 * instead of its own tests; every test so overridden increments *forced, and
 * *hard as well when its margin was at least delta. *cond receives the first-order
 * float32 rounding bound of the returned t (voxels): see or_ray.t_cond.
 *
 * With omega > 1 the steps are over-relaxed (the accelerated sphere tracing of Sec. 3.3,
 * after enhanced sphere tracing): a step is omega times the sampled distance, and a sample
 * whose sphere does not overlap the previous sample's (sdf + previous sdf < step), or a step
 * that left the volume box, is discarded: the trace returns to the previous point plus its
 * sampled distance (the plain step) and stays plain (omega = 1) from there. The discarded
 * sample counts as a step.
 * Every such overlap test that lies within delta of the other outcome is "in band"; bit j of
 * `flip` reverses the j-th in-band test on the path (counted in *forced), and *n_inband
 * receives the number of in-band tests met. */
static int32_t trace_relaxed(const or_volume* vol, const double o[3], const double d[3], double eps_vox,
                             double tlimit, int32_t max_steps, double omega, int32_t fe, int32_t fs, uint32_t flip,
                             int32_t* n_inband, double* t_out, int32_t* steps_out, double* margin_vox,
                             int32_t* forced, int32_t* hard, double* cond) {
    const double h = vol->h, eps = eps_vox * h, band = g_delta_vox * h, u32 = ldexp(1.0, -24);
    const double lo[3] = {vol->origin[0], vol->origin[1], vol->origin[2]};
    const double hi[3] = {vol->origin[0] + vol->nx * h, vol->origin[1] + vol->ny * h,
                          vol->origin[2] + vol->nz * h};
    double t = 0.0, margin = HUGE_MARGIN, dt = 0.0;
    double w = omega > 1.0 ? omega : 1.0;  /* the current relaxation factor */
    double prev_r = 0.0, step = 0.0;        /* the previous sample's distance and the last step */
    double dt_prev = 0.0, slope_prev = 0.0; /* t's rounding bound and the slope at the previous point */
    int32_t inband = 0;
#define DECIDE(natural, wanted_if_forced, m)                      \
    ((fe < 0) ? (natural) : ((wanted_if_forced) != (natural)      \
                                 ? (++*forced, *hard += (m) >= band, (wanted_if_forced)) \
                                 : (natural)))
    *cond = 0.0;
    if (n_inband) *n_inband = 0;
    for (int32_t s = 0; s < max_steps; ++s) {
        double p[3] = {o[0] + t * d[0], o[1] + t * d[1], o[2] + t * d[2]};
        int outside = 0;
        double m_out = HUGE_MARGIN, pmax = 0.0;
        for (int a = 0; a < 3; ++a) {
            if (p[a] < lo[a] || p[a] > hi[a]) outside = 1;
            m_out = fmin(m_out, fmin(fabs(p[a] - lo[a]), fabs(p[a] - hi[a])));
            pmax = fmax(pmax, fmax(fabs(p[a]), fabs(p[a] - lo[a])));
        }
        margin = fmin(margin, m_out);
        if (w > 1.0) { /* over-relaxed: a step that left the box failed (in band: either way) */
            if (m_out < band) {
                if ((flip >> inband) & 1u) {
                    outside = !outside;
                    ++*forced;
                }
                ++inband;
            }
        } else if (DECIDE(outside, fe == OR_LEFT_VOLUME && s == fs, m_out)) {
            *t_out = tlimit;
            *steps_out = s;
            *margin_vox = margin / h;
            if (n_inband) *n_inband = inband;
            return OR_LEFT_VOLUME;
        }
        double sd = outside ? 0.0 : oracle_sample_sdf(vol, p);
        if (w > 1.0) { /* over-relaxed: does this sample's sphere overlap the previous one's? */
            const double m_sor = outside ? HUGE_MARGIN : fabs(sd + prev_r - step);
            int back = outside || sd + prev_r < step;
            margin = fmin(margin, m_sor);
            if (m_sor < band) {
                if ((flip >> inband) & 1u) {
                    back = !back;
                    ++*forced;
                }
                ++inband;
            }
            if (back) { /* discard the sample: the previous point's plain step instead */
                dt = dt_prev * fabs(1.0 + slope_prev) + u32 * (2.0 * pmax + 2.0 * fabs(step) + 2.0 * h + t);
                t = t - step + prev_r;
                step = prev_r;
                w = 1.0;
                continue; /* the budget test of this step is the loop's own */
            }
        }
        double m_hit = fabs(sd - eps);
        margin = fmin(margin, m_hit);
        if (DECIDE(sd < eps, fe == OR_HIT && s == fs - 1, m_hit)) {
            *t_out = t;
            *steps_out = s + 1;
            *margin_vox = margin / h;
            *cond = dt / h;
            if (n_inband) *n_inband = inband;
            return OR_HIT;
        }
        /* first-order propagation of a perturbation of t through this step, plus the
         * float32 rounding of this step's point, sample and sum */
        const double slope = sdf_slope(vol, p, d);
        dt_prev = dt;
        slope_prev = slope;
        dt = dt * fabs(1.0 + w * slope) + u32 * (2.0 * pmax + 2.0 * fabs(w * sd) + 2.0 * h + t);
        prev_r = sd;
        step = w * sd;
        t += step;
        double m_lim = fabs(t - tlimit);
        margin = fmin(margin, m_lim);
        if (DECIDE(t > tlimit, fe == OR_PAST_LIMIT && s == fs - 1, m_lim)) {
            *t_out = tlimit;
            *steps_out = s + 1;
            *margin_vox = margin / h;
            if (n_inband) *n_inband = inband;
            return OR_PAST_LIMIT;
        }
    }
#undef DECIDE
    if (fe >= 0 && fe != OR_EXHAUSTED) { /* the followed path ends on an event this path never reached */
        ++*forced;
        ++*hard;
    }
    *t_out = t;
    *steps_out = max_steps;
    *margin_vox = margin / h;
    *cond = dt / h;
    if (n_inband) *n_inband = inband;
    return OR_EXHAUSTED;
}

static int32_t trace_path(const or_volume* vol, const double o[3], const double d[3], double eps_vox,
                          double tlimit, int32_t max_steps, int32_t fe, int32_t fs, double* t_out,
                          int32_t* steps_out, double* margin_vox, int32_t* forced, int32_t* hard, double* cond) {
    return trace_relaxed(vol, o, d, eps_vox, tlimit, max_steps, 1.0, fe, fs, 0u, NULL, t_out, steps_out, margin_vox,
                         forced, hard, cond);
}

/* A path that follows the other side's event (fe) and step count (fs). Over-relaxed traces
 * also try reversing their in-band overlap tests (those within delta of the other outcome),
 * fewest reversals first, and take the first path whose forced tests are all in band. */
static int32_t trace_follow(const or_volume* vol, const double o[3], const double d[3], double eps_vox,
                            double tlimit, int32_t max_steps, double omega, int32_t fe, int32_t fs, int32_t n_inband,
                            double* t_out, int32_t* steps_out, double* margin_vox, int32_t* forced, int32_t* hard,
                            double* cond) {
    int32_t f0 = 0, h0 = 0, nb;
    int32_t ev = trace_relaxed(vol, o, d, eps_vox, tlimit, max_steps, omega, fe, fs, 0u, &nb, t_out, steps_out,
                               margin_vox, &f0, &h0, cond);
    const int32_t bits = n_inband < 6 ? n_inband : 6;
    if (h0 > 0 && omega > 1.0 && bits > 0) {
        for (int32_t k = 1; k <= bits; ++k)
            for (uint32_t mask = 1; mask < (1u << bits); ++mask) {
                if (__builtin_popcount(mask) != k) continue;
                int32_t f1 = 0, h1 = 0;
                double t1, m1, c1;
                int32_t s1;
                const int32_t e1 = trace_relaxed(vol, o, d, eps_vox, tlimit, max_steps, omega, fe, fs, mask, NULL, &t1,
                                                 &s1, &m1, &f1, &h1, &c1);
                if (h1 == 0) {
                    *t_out = t1;
                    *steps_out = s1;
                    *margin_vox = m1;
                    *cond = c1;
                    *forced += f1;
                    return e1;
                }
            }
    }
    *forced += f0;
    *hard += h0;
    return ev;
}

int32_t oracle_trace(const or_volume* vol, const double o[3], const double d[3],
                     double eps_vox, double tlimit, int32_t max_steps,
                     double* t_out, int32_t* steps_out, double* margin_vox) {
    int32_t forced = 0, hard = 0;
    double cond;
    return trace_path(vol, o, d, eps_vox, tlimit, max_steps, -1, 0, t_out, steps_out, margin_vox, &forced,
                      &hard, &cond);
}

int32_t oracle_trace_relaxed(const or_volume* vol, const double o[3], const double d[3], double eps_vox,
                             double tlimit, int32_t max_steps, double omega, double* t_out, int32_t* steps_out,
                             double* margin_vox) {
    int32_t forced = 0, hard = 0;
    double cond;
    return trace_relaxed(vol, o, d, eps_vox, tlimit, max_steps, omega, -1, 0, 0u, NULL, t_out, steps_out, margin_vox,
                         &forced, &hard, &cond);
}

int32_t oracle_record_sizes(int32_t which) { return which == 0 ? (int32_t)sizeof(or_ray) : (int32_t)sizeof(or_force); }

static int is_miss(int32_t event) { return event == OR_LEFT_VOLUME || event == OR_PAST_LIMIT; }

/* ------------------------------------------------ border fixup (O8) */

/* Copies into the one-texel border of an (n+2)^2 octahedral map the interior texel
 * that is its neighbour across the octahedron's fold: each edge is its own mirror
 * image about its midpoint, and each corner takes the diagonally opposite interior
 * corner. Map index (row y, column x), channels innermost. */
void oracle_border(double* map, int32_t n, int32_t C) {
    const int T = n + 2;
#define AT(y, x) (map + ((size_t)(y) * T + (x)) * C)
    for (int x = 1; x <= n; ++x) {
        memcpy(AT(0, x), AT(1, n + 1 - x), sizeof(double) * C);
        memcpy(AT(n + 1, x), AT(n, n + 1 - x), sizeof(double) * C);
    }
    for (int y = 1; y <= n; ++y) {
        memcpy(AT(y, 0), AT(n + 1 - y, 1), sizeof(double) * C);
        memcpy(AT(y, n + 1), AT(n + 1 - y, n), sizeof(double) * C);
    }
    memcpy(AT(0, 0), AT(n, n), sizeof(double) * C);
    memcpy(AT(0, n + 1), AT(n, 1), sizeof(double) * C);
    memcpy(AT(n + 1, 0), AT(1, n), sizeof(double) * C);
    memcpy(AT(n + 1, n + 1), AT(1, 1), sizeof(double) * C);
#undef AT
}

/* ------------------------------------------------ interpolation rule (O13) */

/* Bilinear fetch of the RGB of an irradiance map at direction v: texel centre of
 * interior texel a is uv = (a + 1/2)/n and sits at index a + 1 of the bordered map. */
static void fetch_oct_bilinear(const double* map, const double v[3], double out[3]) {
    double uv[2];
    oracle_oct_encode(v, uv);
    double cx = 1.0 + uv[0] * IRR_N - 0.5, cy = 1.0 + uv[1] * IRR_N - 0.5;
    int x0 = (int)floor(cx), y0 = (int)floor(cy);
    if (x0 > IRR_N) x0 = IRR_N;
    if (y0 > IRR_N) y0 = IRR_N;
    double fx = cx - x0, fy = cy - y0;
    for (int k = 0; k < 3; ++k) out[k] = 0.0;
    for (int c = 0; c < 4; ++c) {
        int dx = c & 1, dy = c >> 1;
        double w = (dx ? fx : 1.0 - fx) * (dy ? fy : 1.0 - fy);
        const double* texel = map + ((size_t)(y0 + dy) * IRR_T + (x0 + dx)) * 4;
        for (int k = 0; k < 3; ++k) out[k] += w * texel[k];
    }
}

/* Normalised irradiance at x for normal nrm: trilinear over the 8 probes of the grid
 * cell containing x (clamped to the grid), each probe weighted by its trilinear weight
 * times its history-valid flag, each contributing its map's bilinear value at nrm;
 * weights are renormalised, and an all-zero weight gives 0. */
void oracle_sample_irradiance(const or_grid* g, const double* irr, const uint8_t* valid,
                              const double x[3], const double nrm[3], double out[3]) {
    int base[3];
    double f[3];
    for (int a = 0; a < 3; ++a) {
        double c = clampd((x[a] - g->origin[a]) / g->spacing[a], 0.0, (double)(g->dims[a] - 1));
        int b = (int)floor(c);
        if (b > g->dims[a] - 2) b = g->dims[a] - 2;
        if (b < 0) b = 0;
        base[a] = b;
        f[a] = g->dims[a] > 1 ? c - b : 0.0;
    }
    double sw = 0.0, acc[3] = {0.0, 0.0, 0.0};
    for (int c = 0; c < 8; ++c) {
        int d[3] = {c & 1, (c >> 1) & 1, (c >> 2) & 1};
        double w = 1.0;
        int idx[3];
        for (int a = 0; a < 3; ++a) {
            w *= d[a] ? f[a] : 1.0 - f[a];
            idx[a] = base[a] + d[a];
            if (idx[a] > g->dims[a] - 1) idx[a] = g->dims[a] - 1;
        }
        size_t p = ((size_t)idx[2] * g->dims[1] + idx[1]) * g->dims[0] + idx[0];
        w *= valid[p] ? 1.0 : 0.0;
        if (w <= 0.0) continue;
        double v[3];
        fetch_oct_bilinear(irr + p * IRR_T * IRR_T * 4, nrm, v);
        for (int k = 0; k < 3; ++k) acc[k] += w * v[k];
        sw += w;
    }
    for (int k = 0; k < 3; ++k) out[k] = sw > 0.0 ? acc[k] / sw : 0.0;
}

/* The march of the soft SDF shadow trace of oracle_sample_irradiance_visible from state
 * (t, vis, step s0). *m_hit receives how far the hit tests whose other outcome would
 * change the result lie from flipping (voxels); with branch set, a hit within the
 * rounding band (g_delta_vox) is also followed the other way to see whether it matters. */
static double march_visibility(const or_volume* vol, const or_grid* g, const double xs[3], const double dir[3],
                               double L, double t, double vis, int s0, double softness, int branch,
                               double* m_hit, double* m_end) {
    const double h = vol->h, eps = g->eps_vox * h;
    double near_miss = HUGE_MARGIN;  /* samples just above eps: a flip would give 0 */
    for (int s = s0; s < g->max_steps; ++s) {
        if (t >= L) break;
        double p[3];
        for (int a = 0; a < 3; ++a) p[a] = xs[a] + t * dir[a];
        const double d = oracle_sample_sdf(vol, p);
        if (d < eps) {
            if (branch && (eps - d) / h < g_delta_vox) {
                const double vis2 = t > 0.0 ? fmin(vis, softness * d / t) : vis;
                double mh = HUGE_MARGIN, me = HUGE_MARGIN;
                if (march_visibility(vol, g, xs, dir, L, t + d, vis2, s + 1, softness, 0, &mh, &me) > 0.0)
                    *m_hit = fmin(*m_hit, (eps - d) / h);
            }
            return 0.0;
        }
        near_miss = fmin(near_miss, (d - eps) / h);
        if (t > 0.0) vis = fmin(vis, softness * d / t);
        t += d;
        *m_end = fmin(*m_end, fabs(t - L) / h);
    }
    vis = clampd(vis, 0.0, 1.0);
    if (vis > 0.0) *m_hit = fmin(*m_hit, near_miss);
    return vis;
}

/* Visibility of probe position q from x (normal nrm). */
static double probe_visibility(const or_volume* vol, const or_grid* g, const double x[3], const double nrm[3],
                               const double q[3], double softness, double* m_hit, double* m_end) {
    const double h = vol->h;
    double xs[3], v[3];
    for (int a = 0; a < 3; ++a) {
        xs[a] = x[a] + g->bias_vox * h * nrm[a];
        v[a] = q[a] - xs[a];
    }
    const double L = sqrt(dot3(v, v));
    *m_hit = HUGE_MARGIN;
    *m_end = HUGE_MARGIN;
    if (!(L > 0.0)) return 1.0;
    const double dir[3] = {v[0] / L, v[1] / L, v[2] / L};
    return march_visibility(vol, g, xs, dir, L, 0.0, 1.0, 0, softness, 1, m_hit, m_end);
}

void oracle_sample_irradiance_visible(const or_volume* vol, const or_grid* g, const double* irr,
                                      const uint8_t* valid, const float* probe_pos, double softness,
                                      const double x[3], const double nrm[3], double out[3], double vis[8],
                                      double margins[16]) {
    int base[3];
    double f[3];
    for (int a = 0; a < 3; ++a) {
        double c = clampd((x[a] - g->origin[a]) / g->spacing[a], 0.0, (double)(g->dims[a] - 1));
        int b = (int)floor(c);
        if (b > g->dims[a] - 2) b = g->dims[a] - 2;
        if (b < 0) b = 0;
        base[a] = b;
        f[a] = g->dims[a] > 1 ? c - b : 0.0;
    }
    double sw = 0.0, acc[3] = {0.0, 0.0, 0.0};
    for (int c = 0; c < 8; ++c) {
        int d[3] = {c & 1, (c >> 1) & 1, (c >> 2) & 1};
        double w = 1.0;
        int idx[3];
        for (int a = 0; a < 3; ++a) {
            w *= d[a] ? f[a] : 1.0 - f[a];
            idx[a] = base[a] + d[a];
            if (idx[a] > g->dims[a] - 1) idx[a] = g->dims[a] - 1;
        }
        size_t p = ((size_t)idx[2] * g->dims[1] + idx[1]) * g->dims[0] + idx[0];
        w *= valid[p] ? 1.0 : 0.0;
        vis[c] = -1.0;
        margins[2 * c] = margins[2 * c + 1] = HUGE_MARGIN;
        if (w <= 0.0) continue;
        double q[3];
        for (int a = 0; a < 3; ++a)
            q[a] = probe_pos ? (double)probe_pos[3 * p + a] : g->origin[a] + idx[a] * g->spacing[a];
        vis[c] = probe_visibility(vol, g, x, nrm, q, softness, &margins[2 * c], &margins[2 * c + 1]);
        w *= vis[c];
        if (w <= 0.0) continue;
        double val[3];
        fetch_oct_bilinear(irr + p * IRR_T * IRR_T * 4, nrm, val);
        for (int k = 0; k < 3; ++k) acc[k] += w * val[k];
        sw += w;
    }
    for (int k = 0; k < 3; ++k) out[k] = sw > 0.0 ? acc[k] / sw : 0.0;
}

/* ------------------------------------------------ shading (Sec. 3.3, O12) */

/* Radiance leaving hit point x back along the ray: emission stored with the scene,
 * plus Lambertian direct light (each light gated by a binary SDF shadow ray, the
 * stand-in for the paper's reflective-shadow-map flux), plus the multi-bounce term
 * albedo * k * (last frame's normalised irradiance at x for normal n). With a force
 * record, a light's visibility follows the record where this side's own decision
 * (gating or shadow trace) lay within the rounding band. */
static void shade_at(const or_volume* vol, const or_grid* g, const or_light* lights, int32_t n_lights,
                     const double* prev_irr, const uint8_t* prev_valid, const double x[3], const double d[3],
                     const or_force* force, or_ray* rec, int visibility_given, double L_out[3]);

void oracle_shade(const or_volume* vol, const or_grid* g, const or_light* lights, int32_t n_lights,
                  const double* prev_irr, const uint8_t* prev_valid,
                  const double x[3], const double d[3], const or_force* force, or_ray* rec) {
    shade_at(vol, g, lights, n_lights, prev_irr, prev_valid, x, d, force, rec, 0, rec->L);
    /* sensitivity of the radiance to the hit distance, visibility held fixed */
    const double step = 1e-3 * vol->h;
    double xp[3] = {x[0] + step * d[0], x[1] + step * d[1], x[2] + step * d[2]}, Lp[3];
    shade_at(vol, g, lights, n_lights, prev_irr, prev_valid, xp, d, NULL, rec, 1, Lp);
    for (int k = 0; k < 3; ++k) rec->dLdt[k] = (Lp[k] - rec->L[k]) / step;
}

/* The shading of one hit point. visibility_given: take each light's visibility from
 * rec->lit_mask (no shadow ray, no bookkeeping) instead of tracing it. */
static void shade_at(const or_volume* vol, const or_grid* g, const or_light* lights, int32_t n_lights,
                     const double* prev_irr, const uint8_t* prev_valid, const double x[3], const double d[3],
                     const or_force* force, or_ray* rec, int visibility_given, double L_out[3]) {
    const double h = vol->h;
    double grad[3];
    for (int a = 0; a < 3; ++a) {
        double pp[3] = {x[0], x[1], x[2]}, pm[3] = {x[0], x[1], x[2]};
        pp[a] += 0.5 * h;
        pm[a] -= 0.5 * h;
        grad[a] = oracle_sample_sdf(vol, pp) - oracle_sample_sdf(vol, pm);
    }
    double glen = sqrt(dot3(grad, grad));
    double n[3];
    for (int a = 0; a < 3; ++a) n[a] = glen > 0.0 ? grad[a] / glen : -d[a];

    double albedo[3], emission[3];
    if (vol->n_prims > 0) {
        /* the material of the primitive attaining the distance at the hit; a choice between
         * primitives within the rounding band follows the other side's record */
        int32_t own;
        double second;
        oracle_analytic_sdf(vol, x, &own, &second);
        const double best = prim_distance(&vol->prims[own], x);
        if (!visibility_given) {
            rec->natural_owner = own + 1;
            rec->margin_owner = (second - best) / h;
            if (force && force->owner > 0 && force->owner - 1 != own && force->owner - 1 < vol->n_prims) {
                rec->forced++;
                if (!(rec->margin_owner < g_delta_vox)) rec->hard++;
                own = force->owner - 1;
            }
            rec->owner = own + 1;
        } else if (rec->owner > 0) {
            own = rec->owner - 1;
        }
        for (int k = 0; k < 3; ++k) {
            albedo[k] = vol->prims[own].albedo[k];
            emission[k] = vol->prims[own].emission[k];
        }
    } else {
        sample_material(vol, x, albedo, emission);
    }

    double xs[3];
    for (int a = 0; a < 3; ++a) xs[a] = x[a] + g->bias_vox * h * n[a];
    const double tmax = g->tmax_vox * h;

    double direct[3] = {0.0, 0.0, 0.0}, dcos[3] = {0.0, 0.0, 0.0};
    for (int l = 0; l < n_lights; ++l) {
        const or_light* li = &lights[l];
        double ldir[3], scale = 0.0, tlimit = tmax, m_gate, per_cos = 1.0;
        int gate;
        if (li->type == 0) {
            for (int a = 0; a < 3; ++a) ldir[a] = li->v[a];
            double cosv = dot3(n, ldir);
            m_gate = fabs(cosv);
            gate = cosv > 0.0;
            scale = fmax(cosv, 0.0);
        } else {
            double Lv[3] = {li->v[0] - x[0], li->v[1] - x[1], li->v[2] - x[2]};
            double dist = sqrt(dot3(Lv, Lv));
            if (!(dist > 0.0)) continue;
            double cosv = (n[0] * Lv[0] + n[1] * Lv[1] + n[2] * Lv[2]) / dist;
            double q = dist / li->range;
            double q4 = (q * q) * (q * q);
            double win = clampd(1.0 - q4, 0.0, 1.0);
            win = win * win;
            m_gate = fmin(fabs(cosv), fabs(1.0 - q4));
            gate = cosv > 0.0 && win > 0.0;
            scale = fmax(cosv, 0.0) * win / (dist * dist);
            per_cos = win / (dist * dist);
            double Ls[3] = {li->v[0] - xs[0], li->v[1] - xs[1], li->v[2] - xs[2]};
            double ds = sqrt(dot3(Ls, Ls));
            for (int a = 0; a < 3; ++a) ldir[a] = Ls[a] / ds;
            tlimit = ds;
        }
        if (visibility_given) {
            if ((rec->lit_mask >> l) & 1u)
                for (int k = 0; k < 3; ++k) direct[k] += li->rgb[k] * scale;
            continue;
        }
        rec->margin_decision = fmin(rec->margin_decision, m_gate);
        int lit = 0;
        double m_sh = HUGE_MARGIN;
        if (gate) {
            double ts;
            int32_t st, f0 = 0, h0 = 0;
            double c0;
            int32_t ev = trace_relaxed(vol, xs, ldir, g->eps_vox, tlimit, g->max_steps, g->omega_shadow, -1, 0, 0u, NULL,
                                       &ts, &st, &m_sh, &f0, &h0, &c0);
            rec->traced_mask |= 1u << l;
            rec->shadow_steps += st;
            rec->margin_shadow = fmin(rec->margin_shadow, m_sh);
            lit = is_miss(ev); /* occluded by a hit or by a budget-exhausted graze */
        }
        if (lit) rec->natural_lit_mask |= 1u << l;
        if (force) {
            int want = (force->lit_mask >> l) & 1u;
            if (want != lit) {
                rec->forced++;
                if (!(m_gate < g_delta_cos || m_sh < g_delta_vox)) rec->hard++;
                lit = want;
            }
        }
        if (!lit) continue;
        rec->lit_mask |= 1u << l;
        for (int k = 0; k < 3; ++k) {
            direct[k] += li->rgb[k] * scale;
            dcos[k] += li->rgb[k] * per_cos;
        }
    }
    if (!visibility_given)
        for (int k = 0; k < 3; ++k) rec->dLdcos[k] = albedo[k] / kPi * dcos[k];

    double indirect[3] = {0.0, 0.0, 0.0};
    if (g->k_bounce != 0.0) oracle_sample_irradiance(g, prev_irr, prev_valid, x, n, indirect);
    for (int k = 0; k < 3; ++k)
        L_out[k] = emission[k] + albedo[k] / kPi * direct[k] + g->k_bounce * albedo[k] * indirect[k];
}

/* ------------------------------------------------ probe update (Sec. 3.3, Eq. 3) */

/* Cosine-lobe gather of Eq. 3 into one octahedral map, then temporal mixing:
 * for interior texel j with direction u_j, new_j = sum_i w_ij v_i / sum_i w_ij with
 * w_ij = max(0, u_j . d_i)^e (e = 1 for irradiance, e = p for depth moments);
 * out_j = h old_j + (1 - h) new_j; a texel that no ray reaches keeps its old value. */
static void gather_map(double* map, const double* old, int n, int C, int exponent,
                       const double* dirs, const double* vals, int nv, int R, double hyst) {
    const int T = n + 2;
    for (int b = 0; b < n; ++b) {
        for (int a = 0; a < n; ++a) {
            double uv[2] = {(a + 0.5) / n, (b + 0.5) / n}, u[3];
            oracle_oct_decode(uv, u);
            double sw = 0.0, acc[4] = {0.0, 0.0, 0.0, 0.0};
            for (int i = 0; i < R; ++i) {
                double c = dot3(u, dirs + 3 * i);
                if (!(c > 0.0)) continue;
                double w = exponent == 1 ? c : pow(c, (double)exponent);
                sw += w;
                for (int k = 0; k < nv; ++k) acc[k] += w * vals[(size_t)i * nv + k];
            }
            double* out = map + ((size_t)(b + 1) * T + (a + 1)) * C;
            const double* prev = old + ((size_t)(b + 1) * T + (a + 1)) * C;
            for (int k = 0; k < C; ++k) out[k] = prev[k];
            if (sw > 0.0) {
                for (int k = 0; k < nv; ++k) out[k] = hyst * prev[k] + (1.0 - hyst) * (acc[k] / sw);
                if (C > nv) out[nv] = 1.0; /* irradiance alpha: texel has received rays */
            }
        }
    }
    oracle_border(map, n, C);
}

static void update_one_probe(const or_volume* vol, const or_grid* g, const or_light* lights, int32_t n_lights,
                             const float rot[9], const or_probe* pr, size_t p,
                             const double* prev_irr, const double* prev_depth, const uint8_t* prev_valid,
                             double* cur_irr, double* cur_depth, uint8_t* cur_valid, const or_force* force,
                             or_ray* rays) {
    const size_t irr_sz = IRR_T * IRR_T * 4, dep_sz = DEP_T * DEP_T * 2;
    const int R = g->rays;
    if (!(pr->flags & 1u)) { /* inactive: keeps its maps and history, casts no ray */
        if (rays) {
            memset(rays, 0, sizeof(or_ray) * (size_t)R);
            for (int i = 0; i < R; ++i) rays[i].event = rays[i].natural_event = -1;
        }
        memcpy(cur_irr + p * irr_sz, prev_irr + p * irr_sz, sizeof(double) * irr_sz);
        memcpy(cur_depth + p * dep_sz, prev_depth + p * dep_sz, sizeof(double) * dep_sz);
        cur_valid[p] = prev_valid[p];
        return;
    }
    double hyst = (prev_valid[p] && !(pr->flags & 2u)) ? g->hysteresis : 0.0;
    const double h = vol->h, tmax = g->tmax_vox * h;
    const double o[3] = {pr->pos[0], pr->pos[1], pr->pos[2]};

    double* dirs = (double*)malloc(sizeof(double) * 3 * R);
    double* rad = (double*)malloc(sizeof(double) * 3 * R);
    double* mom = (double*)malloc(sizeof(double) * 2 * R);

    for (int i = 0; i < R; ++i) {
        double s[3], d[3];
        oracle_sf_dir(i, R, s);
        for (int r = 0; r < 3; ++r)
            d[r] = (double)rot[3 * r] * s[0] + (double)rot[3 * r + 1] * s[1] + (double)rot[3 * r + 2] * s[2];
        memcpy(dirs + 3 * i, d, sizeof d);

        or_ray rec;
        memset(&rec, 0, sizeof rec);
        rec.margin_shadow = HUGE_MARGIN;
        rec.margin_decision = HUGE_MARGIN;
        const or_force* fi = force ? &force[i] : NULL;
        double t;
        int32_t n_inband = 0;
        rec.natural_event = trace_relaxed(vol, o, d, g->eps_vox, tmax, g->max_steps, g->omega_primary, -1, 0, 0u, &n_inband,
                                          &t, &rec.natural_steps, &rec.margin_primary, &rec.forced, &rec.hard,
                                          &rec.t_cond);
        rec.event = rec.natural_event;
        rec.steps = rec.natural_steps;
        if (fi && (fi->event != rec.natural_event || fi->steps != rec.natural_steps)) {
            double m_unused;
            rec.event = trace_follow(vol, o, d, g->eps_vox, tmax, g->max_steps, g->omega_primary, fi->event, fi->steps,
                                     n_inband, &t, &rec.steps, &m_unused, &rec.forced, &rec.hard, &rec.t_cond);
        }
        rec.t = t;
        if (is_miss(rec.event)) {
            for (int k = 0; k < 3; ++k) rec.L[k] = g->sky[k];
            if (fi && fi->lit_mask) { /* the other side shaded a ray this path misses */
                rec.forced++;
                rec.hard++;
            }
        } else {
            double x[3] = {o[0] + t * d[0], o[1] + t * d[1], o[2] + t * d[2]};
            oracle_shade(vol, g, lights, n_lights, prev_irr, prev_valid, x, d, fi, &rec);
        }
        double td = is_miss(rec.event) ? tmax : fmin(t, tmax);
        for (int k = 0; k < 3; ++k) rad[3 * i + k] = rec.L[k];
        mom[2 * i] = td;
        mom[2 * i + 1] = td * td;
        if (rays) rays[i] = rec;
    }

    gather_map(cur_irr + p * irr_sz, prev_irr + p * irr_sz, IRR_N, 4, 1, dirs, rad, 3, R, hyst);
    gather_map(cur_depth + p * dep_sz, prev_depth + p * dep_sz, DEP_N, 2, g->depth_exponent, dirs, mom, 2, R, hyst);
    cur_valid[p] = 1;
    free(dirs);
    free(rad);
    free(mom);
}

int32_t oracle_update(const or_volume* vol, const or_grid* g, const or_light* lights, int32_t n_lights,
                      const float rot[9], const or_probe* probes,
                      const double* prev_irr, const double* prev_depth, const uint8_t* prev_valid,
                      double* cur_irr, double* cur_depth, uint8_t* cur_valid,
                      const int32_t* subset, int32_t n_subset, const or_force* force, or_ray* rays,
                      int32_t n_threads) {
    if (!vol || !g || !rot || !probes || !prev_irr || !prev_depth || !prev_valid || !cur_irr || !cur_depth ||
        !cur_valid || g->rays < 1 || g->max_steps < 1 || n_lights < 0 || n_lights > 32 || vol->nx < 2 ||
        vol->ny < 2 || vol->nz < 2 || (subset && n_subset < 0))
        return -1;
    const size_t P = (size_t)g->dims[0] * g->dims[1] * g->dims[2];
    const int32_t n = subset ? n_subset : (int32_t)P;
    const int R = g->rays;
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int32_t j = 0; j < n; ++j) {
        size_t p = subset ? (size_t)subset[j] : (size_t)j;
        update_one_probe(vol, g, lights, n_lights, rot, &probes[p], p, prev_irr, prev_depth, prev_valid,
                         cur_irr, cur_depth, cur_valid, force ? force + (size_t)j * R : NULL,
                         rays ? rays + (size_t)j * R : NULL);
    }
    (void)n_threads;
    return 0;
}

/* ------------------------------------------------ probe relocation (Sec. 3.2) */

/* Gradient of the trilinear field by central differences at +-h/2, per unit length. */
static void sdf_gradient(const or_volume* vol, const double p[3], double grad[3]) {
    const double h = vol->h;
    for (int a = 0; a < 3; ++a) {
        double pp[3] = {p[0], p[1], p[2]}, pm[3] = {p[0], p[1], p[2]};
        pp[a] += 0.5 * h;
        pm[a] -= 0.5 * h;
        grad[a] = (oracle_sample_sdf(vol, pp) - oracle_sample_sdf(vol, pm)) / h;
    }
}

void oracle_relocate(const or_volume* vol, const or_grid* g, const or_relocation* rp, const float* last_pos,
                     double* out_pos, uint32_t* out_flags, int32_t* out_iters, double* out_margin) {
    const int32_t P = g->dims[0] * g->dims[1] * g->dims[2];
    const double h = vol->h, c = rp->clearance_vox * h;
    for (int32_t p = 0; p < P; ++p) {
        const int idx[3] = {p % g->dims[0], (p / g->dims[0]) % g->dims[1], p / (g->dims[0] * g->dims[1])};
        double home[3], pos[3], last[3];
        for (int a = 0; a < 3; ++a) {
            home[a] = g->origin[a] + idx[a] * g->spacing[a];
            pos[a] = home[a];
            last[a] = last_pos ? (double)last_pos[3 * p + a] : home[a];
        }
        int32_t it = 0;
        if (rp->clearance_vox > 0.0) {
            while (it < rp->max_iters) {
                const double s = oracle_sample_sdf(vol, pos);
                if (s >= c) break;
                double grad[3];
                sdf_gradient(vol, pos, grad);
                const double g2 = dot3(grad, grad);
                if (!(g2 > 0.0)) break;
                for (int a = 0; a < 3; ++a) {
                    const double lim = rp->max_offset * g->spacing[a];
                    pos[a] = clampd(pos[a] + (c - s) * grad[a] / g2, home[a] - lim, home[a] + lim);
                }
                ++it;
            }
        }
        const double s_end = oracle_sample_sdf(vol, pos);
        const double dist = sqrt((pos[0] - last[0]) * (pos[0] - last[0]) + (pos[1] - last[1]) * (pos[1] - last[1]) +
                                 (pos[2] - last[2]) * (pos[2] - last[2]));
        uint32_t flags = s_end > rp->min_clearance_vox * h ? 1u : 0u;
        if (rp->reject_dist > 0.0 && dist > rp->reject_dist) flags |= 2u;
        for (int a = 0; a < 3; ++a) out_pos[3 * p + a] = pos[a];
        out_flags[p] = flags;
        if (out_iters) out_iters[p] = it;
        if (out_margin) {
            out_margin[2 * p] = s_end / h - rp->min_clearance_vox;
            out_margin[2 * p + 1] = dist - rp->reject_dist;
        }
    }
}

/* ------------------------------------------------ cascade blending (Sec. 3.5) */

/* Evaluated in long double (a 64-bit significand on x86-64): in FP64 the closed form loses
 * up to 1e-5 at points within 1e-7 spacings of a face's plane, where the per-triangle term is
 * a difference of nearly equal quantities. The angles come from atan2(|a x b|, a . b), which
 * keeps its accuracy near 0 and near pi, unlike the chord's arcsine, and the sines of the
 * spherical triangle's corner angles from the triple product (spherical law of sines). */
int32_t oracle_mvc(const double* verts, int32_t nv, const int32_t* tris, int32_t nt, const double x[3],
                   double* lambda) {
    typedef long double ld;
    const ld tiny = 1e-15L, pi = 3.141592653589793238462643383279502884L;
    ld* d = (ld*)malloc(sizeof(ld) * (size_t)nv);
    ld* u = (ld*)malloc(sizeof(ld) * 3 * (size_t)nv);
    ld* lam = (ld*)malloc(sizeof(ld) * (size_t)nv);
    int32_t on = 0;
    for (int32_t j = 0; j < nv; ++j) {
        lambda[j] = 0.0;
        lam[j] = 0.0L;
    }
    for (int32_t j = 0; j < nv && !on; ++j) {
        ld v[3] = {(ld)verts[3 * j] - x[0], (ld)verts[3 * j + 1] - x[1], (ld)verts[3 * j + 2] - x[2]};
        d[j] = sqrtl(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
        if (d[j] < tiny) { /* x at a vertex */
            lambda[j] = 1.0;
            on = 1;
            break;
        }
        for (int a = 0; a < 3; ++a) u[3 * j + a] = v[a] / d[j];
    }
    for (int32_t t = 0; t < nt && !on; ++t) {
        const int32_t id[3] = {tris[3 * t], tris[3 * t + 1], tris[3 * t + 2]};
        ld th[3], c[3], sn[3];
        for (int i = 0; i < 3; ++i) { /* angle at x between the two other corners */
            const ld* a = &u[3 * id[(i + 1) % 3]];
            const ld* b = &u[3 * id[(i + 2) % 3]];
            const ld cr[3] = {a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]};
            th[i] = atan2l(sqrtl(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]), a[0] * b[0] + a[1] * b[1] + a[2] * b[2]);
        }
        const ld hh = 0.5L * (th[0] + th[1] + th[2]);
        const ld* p0 = &u[3 * id[0]];
        const ld* p1 = &u[3 * id[1]];
        const ld* p2 = &u[3 * id[2]];
        const ld det = (p0[1] * p1[2] - p0[2] * p1[1]) * p2[0] + (p0[2] * p1[0] - p0[0] * p1[2]) * p2[1] +
                       (p0[0] * p1[1] - p0[1] * p1[0]) * p2[2];
        /* x in the triangle's plane: the triple product vanishes (to first order in the distance
         * to the plane; the angle sum's gap to 2 pi only to second order) */
        if (fabsl(det) <= tiny) {
            if (pi - hh < 1e-9L) { /* inside the triangle: barycentric coordinates */
                ld w[3], sw = 0.0L;
                for (int i = 0; i < 3; ++i) {
                    w[i] = sinl(th[i]) * d[id[(i + 2) % 3]] * d[id[(i + 1) % 3]];
                    sw += w[i];
                }
                for (int32_t j = 0; j < nv; ++j) lambda[j] = 0.0;
                for (int i = 0; i < 3; ++i) lambda[id[i]] += (double)(w[i] / sw);
                on = 1;
                break;
            }
            continue; /* outside it: no contribution */
        }
        for (int i = 0; i < 3; ++i) {
            const ld s1 = sinl(th[(i + 1) % 3]), s2 = sinl(th[(i + 2) % 3]);
            c[i] = 2.0L * sinl(hh) * sinl(hh - th[i]) / (s1 * s2) - 1.0L;
            /* sign(det) sqrt(1 - c^2) by the spherical law of sines, without its cancellation
             * where c is near -1 or 1 (x next to a face, or in a face's plane) */
            sn[i] = det / (s1 * s2);
        }
        for (int i = 0; i < 3; ++i) {
            const int i1 = (i + 1) % 3, i2 = (i + 2) % 3;
            lam[id[i]] += (th[i] - c[i1] * th[i2] - c[i2] * th[i1]) / (d[id[i]] * sinl(th[i1]) * sn[i2]);
        }
    }
    if (!on) {
        ld sw = 0.0L;
        for (int32_t j = 0; j < nv; ++j) sw += lam[j];
        for (int32_t j = 0; j < nv; ++j) lambda[j] = (double)(lam[j] / sw);
    }
    free(d);
    free(u);
    free(lam);
    return on;
}

/* The 12 triangles of an axis-aligned box, counter-clockwise seen from outside (corner c has
 * coordinates lo/hi by the bits x = c&1, y = c&2, z = c&4), or reversed. */
static void box_triangles(int base, int reversed, int32_t* tris) {
    static const int32_t faces[6][4] = {{0, 4, 6, 2}, {1, 3, 7, 5}, {0, 1, 5, 4},
                                        {2, 6, 7, 3}, {0, 2, 3, 1}, {4, 5, 7, 6}};
    for (int f = 0; f < 6; ++f) {
        const int32_t* q = faces[f];
        int32_t t0[3] = {q[0], q[1], q[2]}, t1[3] = {q[0], q[2], q[3]};
        for (int k = 0; k < 3; ++k) {
            tris[6 * f + k] = base + (reversed ? t0[2 - k] : t0[k]);
            tris[6 * f + 3 + k] = base + (reversed ? t1[2 - k] : t1[k]);
        }
    }
}

static void box_corners(const double lo[3], const double hi[3], double* v) {
    for (int c = 0; c < 8; ++c) {
        v[3 * c] = (c & 1) ? hi[0] : lo[0];
        v[3 * c + 1] = (c & 2) ? hi[1] : lo[1];
        v[3 * c + 2] = (c & 4) ? hi[2] : lo[2];
    }
}

static void probe_box(const or_grid* g, double lo[3], double hi[3]) {
    for (int a = 0; a < 3; ++a) {
        lo[a] = g->origin[a];
        hi[a] = g->origin[a] + (g->dims[a] - 1) * g->spacing[a];
    }
}

double oracle_cascade_weight(const or_grid* g, const double x[3]) {
    double lo[3], hi[3], ilo[3], ihi[3];
    probe_box(g, lo, hi);
    for (int a = 0; a < 3; ++a) {
        /* with fewer than 4 probes along an axis the inner box is empty or flat; a flat one
         * would make the shell a slit box whose weight is 0 off the plate: no transition */
        if (g->dims[a] < 4) return 1.0;
        ilo[a] = lo[a] + g->spacing[a];
        ihi[a] = hi[a] - g->spacing[a];
    }
    int inside_inner = 1;
    for (int a = 0; a < 3; ++a)
        if (x[a] < ilo[a] || x[a] > ihi[a]) inside_inner = 0;
    if (inside_inner) return 1.0;
    double v[48];
    int32_t tris[72];
    box_corners(lo, hi, v);
    box_corners(ilo, ihi, v + 24);
    box_triangles(0, 0, tris);
    box_triangles(8, 1, tris + 36);
    double lam[16];
    oracle_mvc(v, 16, tris, 24, x, lam);
    double w = 0.0;
    for (int j = 8; j < 16; ++j) w += lam[j];
    return clampd(w, 0.0, 1.0);
}

/* E_i of one cascade level: the plain rule, or (vols given, softness > 0, not the farthest
 * level) the rule with probe visibility, whose 16 margins go to m (HUGE_MARGIN otherwise). */
static void cascade_level_value(const or_volume* const* vols, const or_grid* const* grids,
                                const double* const* irr, const uint8_t* const* valid,
                                const float* const* probe_pos, int32_t n, double softness, int32_t i,
                                const double x[3], const double nrm[3], double e[3], double m[16]) {
    if (vols && softness > 0.0 && i < n - 1) {
        double vis[8];
        oracle_sample_irradiance_visible(vols[i], grids[i], irr[i], valid[i], probe_pos ? probe_pos[i] : NULL,
                                         softness, x, nrm, e, vis, m);
        return;
    }
    oracle_sample_irradiance(grids[i], irr[i], valid[i], x, nrm, e);
    for (int k = 0; k < 16; ++k) m[k] = HUGE_MARGIN;
}

void oracle_sample_irradiance_cascade_visible(const or_volume* const* vols, const or_grid* const* grids,
                                              const double* const* irr, const uint8_t* const* valid,
                                              const float* const* probe_pos, int32_t n, double softness,
                                              const double x[3], const double nrm[3], double out[3], double* w_out,
                                              int32_t* level_out, double margins[32]) {
    int32_t k = n - 1;
    for (int32_t i = 0; i < n; ++i) {
        double lo[3], hi[3];
        probe_box(grids[i], lo, hi);
        if (x[0] >= lo[0] && x[0] <= hi[0] && x[1] >= lo[1] && x[1] <= hi[1] && x[2] >= lo[2] && x[2] <= hi[2]) {
            k = i;
            break;
        }
    }
    double w = k < n - 1 ? oracle_cascade_weight(grids[k], x) : 1.0;
    double ek[3];
    cascade_level_value(vols, grids, irr, valid, probe_pos, n, softness, k, x, nrm, ek, margins);
    for (int a = 0; a < 3; ++a) out[a] = ek[a];
    for (int j = 16; j < 32; ++j) margins[j] = HUGE_MARGIN;
    if (w < 1.0) {
        double ec[3];
        cascade_level_value(vols, grids, irr, valid, probe_pos, n, softness, k + 1, x, nrm, ec, margins + 16);
        for (int a = 0; a < 3; ++a) out[a] = w * ek[a] + (1.0 - w) * ec[a];
    }
    *w_out = w;
    *level_out = k;
}

void oracle_sample_irradiance_cascade(const or_grid* const* grids, const double* const* irr,
                                      const uint8_t* const* valid, int32_t n, const double x[3],
                                      const double nrm[3], double out[3], double* w_out, int32_t* level_out) {
    double m[32];
    oracle_sample_irradiance_cascade_visible(NULL, grids, irr, valid, NULL, n, 0.0, x, nrm, out, w_out, level_out, m);
}
