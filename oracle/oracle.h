/*
 * oracle.h -- FP64 CPU oracle of the SDFDDGI per-frame probe update.
 *
 * TEST INFRASTRUCTURE. Only the tests, the smoke check and the bench's CPU
 * baseline leg may load this library. It is a plain, slow, obviously correct
 * restatement of the probe update of "Signed Distance Fields Dynamic Diffuse
 * Global Illumination" (Hu et al., arXiv 2007.14394), Sec. 3.3 "Probe update"
 * with Eq. 3, computed in double precision, probe by probe and ray by ray.
 * It shares no code, header, table or constant with the CUDA library.
 *
 * Units: every position and distance is in world units; parameters given
 * "in voxels" are multiplied by the voxel size h before use.
 */
#ifndef SDFDDGI_ORACLE_H
#define SDFDDGI_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Voxel signed-distance volume plus material volume.
 * Voxel (x, y, z) holds the field at world point origin + (x+1/2, y+1/2, z+1/2) h,
 * stored [z][y][x]. sdf_dtype 0 = float32, 1 = IEEE binary16 (raw bits).
 * material: [z][y][x][8] binary16 raw bits = albedo r,g,b, unused, emission r,g,b, unused;
 * NULL means albedo 0 and emission 0 everywhere. */
/* An analytic SDF primitive (the paper's scene representation, Sec. 3.1): type 0 sphere
 * (centre, radius), 1 axis-aligned box (centre, half-extents), 2 capsule (end a, end b,
 * radius), 3 half-space below the plane y = p[0], 4 hollow ball (solid outside the sphere
 * of centre p[0..2] and radius p[3]); albedo and emission per primitive. */
typedef struct {
    int32_t type, pad;
    double p[7];
    double albedo[3];
    double emission[3];
} or_prim;

/* The scene: a voxel SDF (sdf, dtype, trilinear with clamp-to-edge; material volume
 * optional), or, when n_prims > 0, the union of analytic primitives (the SDF is the
 * minimum of their distances; the material of a point is that of the primitive attaining
 * it, ties to the lowest index). Either way the box origin + [0, n*h] bounds the traces,
 * and h is the unit of the voxel-unit parameters. */
typedef struct {
    int32_t nx, ny, nz, sdf_dtype;
    double h;
    double origin[3];
    const void* sdf;
    const uint16_t* material;
    const or_prim* prims;
    int32_t n_prims, pad;
} or_volume;

/* Light: type 0 = directional (v = unit direction TOWARD the light, rgb = irradiance E),
 *        type 1 = point (v = position, rgb = intensity I, range r > 0). */
typedef struct {
    int32_t type, pad;
    double v[3];
    double rgb[3];
    double range;
} or_light;

/* Probe volume parameters (the same meaning as the library's volume description). */
typedef struct {
    int32_t dims[3];
    int32_t rays;              /* R, rays per probe */
    double origin[3];          /* world position of probe (0,0,0) */
    double spacing[3];         /* world spacing of the probe grid */
    int32_t max_steps;         /* S_max of every sphere trace */
    int32_t depth_exponent;    /* p: depth weight max(0, cos)^p */
    double eps_vox;            /* hit threshold, voxels */
    double tmax_vox;           /* trace length limit, voxels */
    double hysteresis;         /* h in out = h old + (1-h) new */
    double k_bounce;           /* gain of the previous-frame (multi-bounce) term */
    double bias_vox;           /* shadow-ray origin offset along the normal, voxels */
    double sky[3];             /* radiance of rays that miss */
    double omega_primary;      /* relaxation of the primary traces (1: plain sphere tracing) */
    double omega_shadow;       /* relaxation of the shadow traces */
} or_grid;

/* Probe state: world position and flags (bit 0 active, bit 1 reject history). */
typedef struct {
    float pos[3];
    uint32_t flags;
} or_probe;

/* Exit events of a sphere trace. A ray is a MISS when it ends by LEFT_VOLUME or
 * PAST_LIMIT; HIT and EXHAUSTED (budget spent, taken as a hit at the final t) shade. */
#define OR_LEFT_VOLUME 0
#define OR_HIT 1
#define OR_PAST_LIMIT 2
#define OR_EXHAUSTED 3

/* Discrete outcome of one ray as another implementation took it: the event and
 * step count of the primary trace and the visibility bit of every light. When
 * given, the oracle follows these decisions wherever its own double-precision
 * decision lies within delta of the threshold (a rounding-sensitive decision),
 * counts every such override, and counts as "hard" any override whose margin
 * was wider than delta. Everything continuous stays double precision. */
typedef struct {
    int32_t event;
    int32_t steps;
    uint32_t lit_mask;
    int32_t owner;           /* analytic scenes: index + 1 of the primitive whose material the hit
                                took (0: not given) */
} or_force;

/* Per-ray record of one update (one per (probe, ray)). */
typedef struct {
    double t;                /* hit distance (world) along the path taken; MISS records the trace limit */
    double L[3];             /* radiance carried back to the probe */
    double margin_primary;   /* voxels: closest approach of a natural termination test to flipping */
    double margin_shadow;    /* voxels: the same over all natural shadow traces (1e300 if none) */
    double margin_decision;  /* min over lights of |n.l| and, for point lights, |1-(d/r)^4| */
    int32_t event;           /* path taken */
    int32_t steps;           /* SDF samples of the primary trace, path taken */
    int32_t natural_event;   /* the oracle's own decisions */
    int32_t natural_steps;
    uint32_t lit_mask;       /* bit l: light l contributed with visibility 1 (path taken) */
    uint32_t natural_lit_mask;
    uint32_t traced_mask;    /* bit l: a natural shadow ray toward light l was traced */
    int32_t shadow_steps;    /* SDF samples over all natural shadow traces */
    int32_t forced;          /* decisions taken from the force record */
    int32_t hard;            /* of those, decisions whose margin exceeded delta */
    double t_cond;           /* voxels: first-order bound of the float32 rounding error of t, see
                                oracle_update */
    double dLdt[3];          /* derivative of L with respect to the hit distance, visibility held fixed */
    double dLdcos[3];        /* derivative of L with respect to each visible light's cosine n.l, summed
                                over those lights (sensitivity to the rounding of the shading normal) */
    int32_t owner;           /* analytic scenes: index + 1 of the primitive whose material was used */
    int32_t natural_owner;   /* the oracle's own choice */
    double margin_owner;     /* voxels: second-smallest minus smallest primitive distance at the hit */
} or_ray;

/* sizeof(or_ray) (which = 0) or sizeof(or_force) (which = 1), for bindings to check their layouts. */
int32_t oracle_record_sizes(int32_t which);

/* Spherical-Fibonacci direction i of n (unrotated). */
void oracle_sf_dir(int32_t i, int32_t n, double out[3]);
/* Octahedral map (pole +z). */
void oracle_oct_encode(const double v[3], double uv[2]);
void oracle_oct_decode(const double uv[2], double v[3]);
/* Distance of the union of analytic primitives at p; *owner receives the index of the
 * primitive attaining it (lowest index on ties) and *second the next smallest distance. */
double oracle_analytic_sdf(const or_volume* vol, const double p[3], int32_t* owner, double* second);
/* Trilinear sample of the signed-distance volume at world point p (or the analytic SDF). */
double oracle_sample_sdf(const or_volume* vol, const double p[3]);
/* One sphere trace; returns the exit event, writes t (world), steps and margin (voxels). */
int32_t oracle_trace(const or_volume* vol, const double o[3], const double d[3],
                     double eps_vox, double tlimit, int32_t max_steps,
                     double* t, int32_t* steps, double* margin_vox);

/* The same trace over-relaxed by omega > 1 (Sec. 3.3 accelerated sphere tracing): steps of
 * omega * sdf; a sample whose sphere misses the previous sample's (sdf + previous sdf < step)
 * is discarded for the previous point's plain step, and the rest of the ray is plain. */
int32_t oracle_trace_relaxed(const or_volume* vol, const double o[3], const double d[3], double eps_vox,
                             double tlimit, int32_t max_steps, double omega, double* t_out, int32_t* steps_out,
                             double* margin_vox);
/* Border fixup of one (n+2)x(n+2)xC map in place. */
void oracle_border(double* map, int32_t n, int32_t channels);
/* Interpolated normalised irradiance at world point x with unit normal nrm. */
void oracle_sample_irradiance(const or_grid* g, const double* irr, const uint8_t* valid,
                              const double x[3], const double nrm[3], double out[3]);
/* Radiance leaving hit point x toward a ray of direction d (shading step). */
void oracle_shade(const or_volume* vol, const or_grid* g, const or_light* lights, int32_t n_lights,
                  const double* prev_irr, const uint8_t* prev_valid,
                  const double x[3], const double d[3], const or_force* force, or_ray* rec);

/* Widths of the rounding-sensitive band: distances in voxels, cosines unitless. */
void oracle_set_delta(double delta_vox, double delta_cos);

/* One probe update over the probes listed in `subset` (all probes if subset is NULL).
 * Hit distances are always this side's own. Sphere tracing can amplify rounding: a
 * perturbation of t grows by (1 + dsdf/dt) per step, which exceeds 1 while a ray moves
 * away from a surface it grazed. Each record's t_cond propagates that first-order bound,
 * with a float32 rounding of the step's coordinates, distance and t as the per-step
 * perturbation, so that a test can tell an ill-conditioned ray from a wrong one.
 * prev_irr [P][8][8][4], prev_depth [P][16][16][2], prev_valid [P]: the previous maps.
 * cur_*: written for the listed probes only. rays: NULL or [n_subset][R] records.
 * force: NULL or [n_subset][R] outcomes to follow within the rounding band.
 * rot: row-major 3x3 frame rotation (float32 values, promoted exactly).
 * Returns 0, or -1 on invalid arguments. */
int32_t oracle_update(const or_volume* vol, const or_grid* g, const or_light* lights, int32_t n_lights,
                      const float rot[9], const or_probe* probes,
                      const double* prev_irr, const double* prev_depth, const uint8_t* prev_valid,
                      double* cur_irr, double* cur_depth, uint8_t* cur_valid,
                      const int32_t* subset, int32_t n_subset, const or_force* force, or_ray* rays,
                      int32_t n_threads);

/* Per-point interpolation with probe visibility (Sec. 3.4, per-pixel GI shading): each of
 * the 8 probes of the cell is weighted by trilinear weight x history flag x visibility,
 * the visibility an SDF shadow trace from the point (offset bias_vox * h along the
 * normal) toward the probe, soft in the manner of SDF soft shadows: vis = clamp(min over
 * the march (t > 0) of softness * sdf / t, 0, 1), 0 on a hit (sdf < eps), the march
 * ending when t reaches the probe's distance or after max_steps. No cosine or other
 * extra weight. probe_pos: NULL (grid positions) or [P][3] float probe positions.
 * Outputs the rgb, each corner's visibility (-1 for a corner of weight 0) and, per
 * corner, how far the decisions that could change the visibility lie from flipping: the
 * hit tests whose other outcome changes the result (|sdf - eps|, voxels; a hit within
 * the rounding band of oracle_set_delta is followed the other way to find out) and the
 * end test (|t - distance|, voxels). */
void oracle_sample_irradiance_visible(const or_volume* vol, const or_grid* g, const double* irr,
                                      const uint8_t* valid, const float* probe_pos, double softness,
                                      const double x[3], const double nrm[3], double out[3], double vis[8],
                                      double margins[16]);

/* Mean value coordinates (Floater, Kos and Reimers 2005; Ju, Schaefer and Warren 2005)
 * of x with respect to a closed, consistently oriented triangle mesh (nv vertices [nv][3],
 * nt triangles [nt][3] of vertex indices, counter-clockwise seen from outside the domain):
 * lambda [nv] with sum 1 and sum lambda_j p_j = x. Returns 0, or 1 when x lies on the mesh
 * (lambda then holds the barycentric coordinates of its triangle or the vertex delta). */
int32_t oracle_mvc(const double* verts, int32_t nv, const int32_t* tris, int32_t nt, const double x[3],
                   double* lambda);

/* Cascade blending (Sec. 3.5): the transition weight of volume k at x. The shell between its
 * probe box (outer) and that box shrunk by one probe spacing (inner) is a closed surface
 * (inner faces reversed); w = the sum of the mean value coordinates of the 8 inner corners,
 * 1 on and inside the inner box, 0 on the outer box, clamped to [0, 1]; 1 everywhere when an
 * axis has fewer than 4 probes (no inner box of positive volume). */
double oracle_cascade_weight(const or_grid* g, const double x[3]);

/* Irradiance at x (normal nrm) from volumes grids[0] (finest) .. grids[n-1] (coarsest), each
 * with its maps: the finest volume k whose probe box holds x (the coarsest if none),
 * E = w E_k + (1 - w) E_{k+1} with w = oracle_cascade_weight(grids[k], x) (w = 1 for the
 * coarsest), E_i the plain interpolation rule of volume i. Writes *w_out and *level_out. */
void oracle_sample_irradiance_cascade(const or_grid* const* grids, const double* const* irr,
                                      const uint8_t* const* valid, int32_t n, const double x[3],
                                      const double nrm[3], double out[3], double* w_out, int32_t* level_out);

/* The same with the paper's probe visibility (Sec. 3.4) in every level but the farthest
 * (Sec. 3.5): with vols != NULL and softness > 0, level i < n - 1 takes
 * oracle_sample_irradiance_visible on vols[i] (probe positions probe_pos[i], or the grid
 * positions where probe_pos or probe_pos[i] is NULL). margins[0..15] are that call's margins
 * for level k, margins[16..31] for level k + 1 (HUGE where no visibility test ran). */
void oracle_sample_irradiance_cascade_visible(const or_volume* const* vols, const or_grid* const* grids,
                                              const double* const* irr, const uint8_t* const* valid,
                                              const float* const* probe_pos, int32_t n, double softness,
                                              const double x[3], const double nrm[3], double out[3], double* w_out,
                                              int32_t* level_out, double margins[32]);

/* Probe relocation (Sec. 3.2, the procedure UpdateProbePos). The paper gives the steps
 * (query the SDF at the grid position; if below threshold1, move the probe by gradient
 * descent on the SDF; if it then lies farther than threshold2 from last frame's
 * position, reject its history) but not the descent itself. Reading taken: Gauss-Newton
 * steps on E(p) = (c - sdf(p))^2 / 2 toward the level set sdf = c = clearance_vox * h,
 *     p <- p + (c - sdf(p)) * g / |g|^2,   g = the central-difference gradient of the
 *     trilinear field at +-h/2 (the shading normal's rule) divided by h,
 * while sdf(p) < c and |g| > 0, at most max_iters steps, each followed by a clamp of
 * every coordinate to within max_offset * spacing of the grid position. The probe ends
 * active iff sdf(p) > min_clearance_vox * h. */
typedef struct {
    double clearance_vox;      /* threshold1, voxels; <= 0: no probe moves */
    double reject_dist;        /* threshold2, world units; <= 0: no rejection */
    double max_offset;         /* per-axis displacement limit, as a fraction of the spacing */
    double min_clearance_vox;  /* active iff the final SDF exceeds this (voxels) */
    int32_t max_iters;
    int32_t pad;
} or_relocation;

/* Relocates every probe of grid g. last_pos: NULL (the grid positions) or [P][3] float
 * positions of the last frame. Outputs [P][3] positions, [P] flags (bit 0 active, bit 1
 * reject history), [P] steps taken, and [P][2] decision margins: final SDF minus the
 * active threshold (voxels), and displacement minus threshold2 (world). */
void oracle_relocate(const or_volume* vol, const or_grid* g, const or_relocation* rp, const float* last_pos,
                     double* out_pos, uint32_t* out_flags, int32_t* out_iters, double* out_margin);

#ifdef __cplusplus
}
#endif
#endif
