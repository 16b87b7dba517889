/*
 * FP64 CPU oracle for the field-line advection hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links, loads or
 * calls this file; only the tests, the smoke check and the benchmark's CPU
 * baseline leg do.  It shares no code, header, table or constant generator
 * with the CUDA library: the status numbering below is an interface value that
 * both sides spell out on their own.
 *
 * What it computes (Zellmann et al., "Streami", Sec. 3.1.1, Sec. 3.1.2 and
 * Listing 1, Sec. 3.2 and Listing 2, Sec. 3.3):
 *
 *  - sample(): the field reconstructed at a position.  The paper's structured
 *    field samples a uniform voxel grid "by computing offsets" (Sec. 3.3); the
 *    interpolant is trilinear, written here as its plain definition, the sum of
 *    the eight corner values times the products of the 1-D hat weights.
 *  - the advection step of Listing 1 (Sec. 3.1.2): classical fourth-order
 *    Runge-Kutta with stage points P0 + k1/2, P0 + k2/2, P0 + k3 and weights
 *    (1, 2, 2, 1)/6, each k_i = dt * v(stage point); a failed sample ends the
 *    particle at its last position (the early returns of Listing 1).
 *  - trace(): steps until the step cap is met or the particle stops (Sec. 3.2).
 *  - streaklines (Sec. 3.2, Listing 2): one new particle per release point per
 *    step, the field linear in time between stored slices.
 *  - the per-brick quantisation of the stored field (BF16 / FP16 codes, or
 *    21-bit fixed-point codes, and a per-brick power-of-two scale), which the
 *    paper does not have; it is the precision form of the field store,
 *    restated here from its definition.
 *
 * Readings where the paper is silent (each is also stated where it is used):
 *  - positions are in index space (cells); world = origin + spacing * index;
 *    the domain is the closed box [0, N-1] per axis.
 *  - k_i = dt * V, V = v / spacing (cells per unit time), the field not
 *    normalised; "1/6" of Listing 1 is read as the real number one sixth and
 *    the position handed to destinationID as the new position.
 *  - termination, tested in this order before each step: step cap (MAXSTEPS);
 *    v(P0) not finite (NANFIELD); |v(P0)| < eps in world units (STAGNANT).
 *    During the step: any stage sample not finite (NANFIELD); any stage point
 *    or the new position outside the domain (EXIT).  A stopped step adds no
 *    vertex.  A seed outside the domain gets status OUT and no vertex.
 *  - at the upper face the cell index is clamped to N-2 (fraction 1).
 *  - margin: for EXIT the distance in cells by which the offending point lies
 *    outside the domain; for STAGNANT (eps - |v0|) / eps; otherwise +inf.  A
 *    line whose margin is below a caller's threshold is a boundary tie.
 *
 * Build: gcc -O2 -fopenmp -ffp-contract=off -shared -fPIC oracle.c -lm
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* line status (same numbering as the library's public header) */
#define OR_ACTIVE 0
#define OR_MAXSTEPS 1
#define OR_EXIT 2
#define OR_STAGNANT 3
#define OR_NANFIELD 4
#define OR_OUT 5

/* field storage types of the quantised store */
#define OR_F32 0
#define OR_BF16 1
#define OR_F16 2
#define OR_FX21 3

int or_version(void) { return 1; }

/* ------------------------------------------------------------------------ */
/* samplers: a sampler fills v (world units) at index-space point p.          */

typedef void (*sampler_fn)(const void *ctx, const double p[3], double t, double v[3]);

typedef struct {
    const float *F;       /* AoS [nz][ny][nx][3] */
    int64_t dims[3];
} grid_ctx;

/* Trilinear interpolation as the weighted sum of the 8 corner samples.  The
 * lower corner index is floor(p) clamped to [0, N-2]; weights are the hat
 * functions (1-f, f) per axis. */
static void grid_sample_at(const float *F, const int64_t dims[3], const double p[3], double v[3])
{
    int64_t c[3];
    double f[3];
    for (int a = 0; a < 3; ++a) {
        double fl = floor(p[a]);
        int64_t ci = (int64_t)fl;
        if (ci > dims[a] - 2) ci = dims[a] - 2;
        if (ci < 0) ci = 0;
        c[a] = ci;
        f[a] = p[a] - (double)ci;
    }
    v[0] = v[1] = v[2] = 0.0;
    for (int dz = 0; dz < 2; ++dz)
        for (int dy = 0; dy < 2; ++dy)
            for (int dx = 0; dx < 2; ++dx) {
                double w = (dx ? f[0] : 1.0 - f[0]) * (dy ? f[1] : 1.0 - f[1]) * (dz ? f[2] : 1.0 - f[2]);
                int64_t idx = ((c[2] + dz) * dims[1] + (c[1] + dy)) * dims[0] + (c[0] + dx);
                const float *s = F + 3 * idx;
                v[0] += w * (double)s[0];
                v[1] += w * (double)s[1];
                v[2] += w * (double)s[2];
            }
}

static void grid_sampler(const void *ctx, const double p[3], double t, double v[3])
{
    (void)t;
    const grid_ctx *g = (const grid_ctx *)ctx;
    grid_sample_at(g->F, g->dims, p, v);
}

/* Time-dependent grid: slices at times s * slice_dt, linear in time between
 * consecutive slices.  Reading: a time t falls in the interval (s, s+1] in
 * slice units, s = ceil(t/slice_dt) - 1 clamped to [0, n_slices-2], and
 * alpha = t/slice_dt - s; so the end of a step uses the pair it started in. */
typedef struct {
    const float *F;       /* n_slices consecutive grids */
    int64_t dims[3];
    int64_t n_slices;
    double slice_dt;
} slices_ctx;

static void slice_pair(const slices_ctx *g, double t, int64_t *s_out, double *alpha_out)
{
    double u = t / g->slice_dt;
    int64_t s = (int64_t)ceil(u) - 1;
    if (s > g->n_slices - 2) s = g->n_slices - 2;
    if (s < 0) s = 0;
    *s_out = s;
    *alpha_out = u - (double)s;
}

static void slices_sampler(const void *ctx, const double p[3], double t, double v[3])
{
    const slices_ctx *g = (const slices_ctx *)ctx;
    int64_t s;
    double al;
    slice_pair(g, t, &s, &al);
    int64_t cells = g->dims[0] * g->dims[1] * g->dims[2];
    double a[3], b[3];
    grid_sample_at(g->F + 3 * cells * s, g->dims, p, a);
    grid_sample_at(g->F + 3 * cells * (s + 1), g->dims, p, b);
    for (int c = 0; c < 3; ++c) v[c] = (1.0 - al) * a[c] + al * b[c];
}

/* Analytic ABC flow (no grid), used to check the integrator's order.  Index
 * space equals world space scaled by spacing: x_world = origin + spacing * p. */
typedef struct {
    double A, B, C;
    double origin[3], spacing[3];
} abc_ctx;

static void abc_sampler(const void *ctx, const double p[3], double t, double v[3])
{
    (void)t;
    const abc_ctx *g = (const abc_ctx *)ctx;
    double x = g->origin[0] + g->spacing[0] * p[0];
    double y = g->origin[1] + g->spacing[1] * p[1];
    double z = g->origin[2] + g->spacing[2] * p[2];
    v[0] = g->A * sin(z) + g->C * cos(y);
    v[1] = g->B * sin(x) + g->A * cos(z);
    v[2] = g->C * sin(y) + g->B * cos(x);
}

/* ------------------------------------------------------------------------ */
/* domain tests                                                               */

static int in_domain(const double p[3], const double hi[3])
{
    for (int a = 0; a < 3; ++a)
        if (!(p[a] >= 0.0 && p[a] <= hi[a])) return 0;   /* NaN is outside */
    return 1;
}

static double outside_distance(const double p[3], const double hi[3])
{
    double d = 0.0;
    for (int a = 0; a < 3; ++a) {
        if (p[a] != p[a]) return 0.0;
        if (-p[a] > d) d = -p[a];
        if (p[a] - hi[a] > d) d = p[a] - hi[a];
    }
    return d;
}

static int all_finite(const double v[3])
{
    return isfinite(v[0]) && isfinite(v[1]) && isfinite(v[2]);
}

/* ------------------------------------------------------------------------ */
/* one RK4 step (Listing 1).  Returns OR_ACTIVE on success with pn filled,
 * else the status that stops the particle; *margin is set for EXIT/STAGNANT.
 * inv_sp converts world velocity to cells per unit time. */

static int rk4_step(sampler_fn S, const void *ctx, const double p[3], double t, double dt,
                    const double inv_sp[3], const double hi[3], double eps,
                    double pn[3], double *margin)
{
    double v[3], k1[3], k2[3], k3[3], k4[3], q[3];

    S(ctx, p, t, v);
    if (!all_finite(v)) return OR_NANFIELD;
    double speed = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    if (speed < eps) {
        *margin = (eps - speed) / eps;
        return OR_STAGNANT;
    }
    for (int a = 0; a < 3; ++a) k1[a] = dt * v[a] * inv_sp[a];

    for (int a = 0; a < 3; ++a) q[a] = p[a] + 0.5 * k1[a];
    if (!in_domain(q, hi)) { *margin = outside_distance(q, hi); return OR_EXIT; }
    S(ctx, q, t + 0.5 * dt, v);
    if (!all_finite(v)) return OR_NANFIELD;
    for (int a = 0; a < 3; ++a) k2[a] = dt * v[a] * inv_sp[a];

    for (int a = 0; a < 3; ++a) q[a] = p[a] + 0.5 * k2[a];
    if (!in_domain(q, hi)) { *margin = outside_distance(q, hi); return OR_EXIT; }
    S(ctx, q, t + 0.5 * dt, v);
    if (!all_finite(v)) return OR_NANFIELD;
    for (int a = 0; a < 3; ++a) k3[a] = dt * v[a] * inv_sp[a];

    for (int a = 0; a < 3; ++a) q[a] = p[a] + k3[a];
    if (!in_domain(q, hi)) { *margin = outside_distance(q, hi); return OR_EXIT; }
    S(ctx, q, t + dt, v);
    if (!all_finite(v)) return OR_NANFIELD;
    for (int a = 0; a < 3; ++a) k4[a] = dt * v[a] * inv_sp[a];

    for (int a = 0; a < 3; ++a) pn[a] = p[a] + (k1[a] + 2.0 * k2[a] + 2.0 * k3[a] + k4[a]) / 6.0;
    if (!in_domain(pn, hi)) { *margin = outside_distance(pn, hi); return OR_EXIT; }
    return OR_ACTIVE;
}

/* One streamline from seed index point p0; writes up to max_steps+1 vertices
 * (index space) into verts. */
static void trace_line(sampler_fn S, const void *ctx, const double p0[3], double t0, double dt,
                       int64_t max_steps, double eps, const double inv_sp[3], const double hi[3],
                       double *verts, int32_t *len, uint8_t *status, double *margin)
{
    double p[3] = {p0[0], p0[1], p0[2]};
    *margin = INFINITY;
    if (!in_domain(p, hi)) {
        *len = 0;
        *status = OR_OUT;
        return;
    }
    int64_t n = 0;
    memcpy(verts, p, sizeof p);
    n = 1;
    for (int64_t s = 0;; ++s) {
        if (s == max_steps) { *status = OR_MAXSTEPS; break; }
        double pn[3];
        int st = rk4_step(S, ctx, p, t0 + (double)s * dt, dt, inv_sp, hi, eps, pn, margin);
        if (st != OR_ACTIVE) { *status = (uint8_t)st; break; }
        memcpy(p, pn, sizeof p);
        memcpy(verts + 3 * n, p, sizeof p);
        ++n;
    }
    *len = (int32_t)n;
}

static void set_threads(int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
}

/* Steady streamlines on a grid.  seeds: n x 3 world (double).  verts: n x
 * (max_steps+1) x 3 index-space doubles.  Returns 0 or -1 on bad arguments. */
int or_trace_streamlines(const float *F, const int64_t dims[3], const double origin[3],
                         const double spacing[3], const double *seeds, int64_t n, double dt,
                         int64_t max_steps, double eps, double *verts, int32_t *len,
                         uint8_t *status, double *margin, int nthreads)
{
    for (int a = 0; a < 3; ++a)
        if (dims[a] < 2 || !(spacing[a] > 0.0)) return -1;
    if (max_steps < 0 || n < 0) return -1;
    grid_ctx g;
    g.F = F;
    memcpy(g.dims, dims, sizeof g.dims);
    double inv_sp[3], hi[3];
    for (int a = 0; a < 3; ++a) {
        inv_sp[a] = 1.0 / spacing[a];
        hi[a] = (double)(dims[a] - 1);
    }
    set_threads(nthreads);
    int64_t stride = 3 * (max_steps + 1);
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < n; ++i) {
        double p0[3];
        for (int a = 0; a < 3; ++a) p0[a] = (seeds[3 * i + a] - origin[a]) / spacing[a];
        trace_line(grid_sampler, &g, p0, 0.0, dt, max_steps, eps, inv_sp, hi, verts + stride * i,
                   len + i, status + i, margin + i);
    }
    return 0;
}

/* The same loop with the analytic ABC sampler (RK4 order checks). */
int or_trace_abc(double A, double B, double C, const int64_t dims[3], const double origin[3],
                 const double spacing[3], const double *seeds, int64_t n, double dt,
                 int64_t max_steps, double eps, double *verts, int32_t *len, uint8_t *status,
                 double *margin)
{
    abc_ctx g = {A, B, C, {origin[0], origin[1], origin[2]}, {spacing[0], spacing[1], spacing[2]}};
    double inv_sp[3], hi[3];
    for (int a = 0; a < 3; ++a) {
        inv_sp[a] = 1.0 / spacing[a];
        hi[a] = (double)(dims[a] - 1);
    }
    int64_t stride = 3 * (max_steps + 1);
    for (int64_t i = 0; i < n; ++i) {
        double p0[3];
        for (int a = 0; a < 3; ++a) p0[a] = (seeds[3 * i + a] - origin[a]) / spacing[a];
        trace_line(abc_sampler, &g, p0, 0.0, dt, max_steps, eps, inv_sp, hi, verts + stride * i,
                   len + i, status + i, margin + i);
    }
    return 0;
}

/* Trilinear sample at index points (n x 3) -> v (n x 3), world units. */
int or_sample(const float *F, const int64_t dims[3], const double *p, int64_t n, double *v)
{
    for (int64_t i = 0; i < n; ++i) grid_sample_at(F, dims, p + 3 * i, v + 3 * i);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Streaklines.  R release points (world), field slices at times s*slice_dt.
 * Particle (r, b) is released at release point r at time b*dt (b = 0 ..
 * n_inject-1).  Step j (j = 1 .. n_steps) first advances every live particle
 * from time (j-1)*dt to j*dt, then releases births j (if j < n_inject), so
 * after a step the newest particle of each release point sits on it
 * (Listing 2: update, then generate new particles).
 * Outputs, per (r, b) in r-major order: pos (index space, 3 doubles), status
 * (OR_ACTIVE while alive, else the stop status; 255 = not yet released), steps
 * taken, margin. */
int or_trace_streaklines(const float *slices, int64_t n_slices, const int64_t dims[3],
                         const double origin[3], const double spacing[3], double slice_dt,
                         const double *release, int64_t R, double dt, int64_t n_steps,
                         int64_t n_inject, double eps, double *pos, uint8_t *status,
                         int32_t *steps, double *margin, int nthreads)
{
    for (int a = 0; a < 3; ++a)
        if (dims[a] < 2 || !(spacing[a] > 0.0)) return -1;
    if (n_slices < 2 || R < 0 || n_inject < 1 || n_steps < 0) return -1;
    slices_ctx g;
    g.F = slices;
    memcpy(g.dims, dims, sizeof g.dims);
    g.n_slices = n_slices;
    g.slice_dt = slice_dt;
    double inv_sp[3], hi[3];
    for (int a = 0; a < 3; ++a) {
        inv_sp[a] = 1.0 / spacing[a];
        hi[a] = (double)(dims[a] - 1);
    }
    set_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t r = 0; r < R; ++r) {
        double p0[3];
        for (int a = 0; a < 3; ++a) p0[a] = (release[3 * r + a] - origin[a]) / spacing[a];
        for (int64_t b = 0; b < n_inject; ++b) {
            int64_t k = r * n_inject + b;
            double *p = pos + 3 * k;
            margin[k] = INFINITY;
            steps[k] = 0;
            if (b > n_steps) {          /* never released within n_steps steps */
                status[k] = 255;
                p[0] = p[1] = p[2] = 0.0;
                continue;
            }
            memcpy(p, p0, sizeof p0);
            if (!in_domain(p, hi)) { status[k] = OR_OUT; continue; }
            status[k] = OR_ACTIVE;
            for (int64_t j = b + 1; j <= n_steps; ++j) {
                double pn[3];
                int st = rk4_step(slices_sampler, &g, p, (double)(j - 1) * dt, dt, inv_sp, hi, eps,
                                  pn, margin + k);
                if (st != OR_ACTIVE) { status[k] = (uint8_t)st; break; }
                memcpy(p, pn, sizeof pn);
                steps[k] += 1;
            }
        }
    }
    return 0;
}

/* Path lines: every seed released once at time 0 and followed through the
 * time-dependent field (slices at times s*slice_dt, linear in time between
 * them); step j takes the particle from time (j-1)*dt to j*dt.  The same
 * per-line loop as a streamline with the time-dependent sampler.  Outputs as
 * or_trace_streamlines. */
int or_trace_pathlines(const float *slices, int64_t n_slices, const int64_t dims[3], const double origin[3],
                       const double spacing[3], double slice_dt, const double *seeds, int64_t n, double dt,
                       int64_t max_steps, double eps, double *verts, int32_t *len, uint8_t *status,
                       double *margin, int nthreads)
{
    for (int a = 0; a < 3; ++a)
        if (dims[a] < 2 || !(spacing[a] > 0.0)) return -1;
    if (n_slices < 2 || n < 0 || max_steps < 0 || !(slice_dt > 0.0)) return -1;
    slices_ctx g;
    g.F = slices;
    memcpy(g.dims, dims, sizeof g.dims);
    g.n_slices = n_slices;
    g.slice_dt = slice_dt;
    double inv_sp[3], hi[3];
    for (int a = 0; a < 3; ++a) {
        inv_sp[a] = 1.0 / spacing[a];
        hi[a] = (double)(dims[a] - 1);
    }
    set_threads(nthreads);
    int64_t stride = 3 * (max_steps + 1);
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < n; ++i) {
        double p0[3];
        for (int a = 0; a < 3; ++a) p0[a] = (seeds[3 * i + a] - origin[a]) / spacing[a];
        trace_line(slices_sampler, &g, p0, 0.0, dt, max_steps, eps, inv_sp, hi, verts + stride * i, len + i,
                   status + i, margin + i);
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Unstructured fields (the second field type of Sec. 3.3): cells are
 * tetrahedra (4 vertices), pyramids (5), prisms (6) and hexahedra (8), with
 * the VTK vertex orders; velocity is given at the vertices and interpolated
 * with the cell's isoparametric shape functions N_i(r):
 *   tet      1-r-s-t, r, s, t                       (r, s, t >= 0, r+s+t <= 1)
 *   pyramid  (1-r)(1-s)(1-t), r(1-s)(1-t), rs(1-t), (1-r)s(1-t), t
 *                                                      (r, s, t in [0, 1])
 *   prism    (1-r-s)(1-t), r(1-t), s(1-t), (1-r-s)t, rt, st
 *                                                      (r, s >= 0, r+s <= 1, t in [0, 1])
 *   hex      (1-r)(1-s)(1-t), r(1-s)(1-t), rs(1-t), (1-r)s(1-t),
 *            (1-r)(1-s)t, r(1-s)t, rst, (1-r)st        (r, s, t in [0, 1])
 * A point p lies in a cell if the parametric solution of sum N_i(r) x_i = p
 * (Newton's method from the cell's centre) satisfies the cell's inequalities
 * within tau.  Point location: the cell found for the particle's previous
 * sample is tried first, then every cell in index order (brute force).
 * Streamlines: the same RK4 steps as a grid field, in world coordinates; a
 * stage point or new position in no cell stops the line (EXIT) with margin =
 * how far outside (parametric) the particle's current cell it lies.        */

typedef struct {
    const double *X;      /* vertices, n_vertices x 3 world */
    const double *V;      /* velocity at the vertices */
    const int32_t *idx;   /* cell vertex lists */
    const int64_t *off;   /* cell c: idx[off[c] .. off[c+1]) */
    const uint8_t *type;  /* 4, 5, 6, 8 */
    int64_t n_cells;
    double tau;
    const int64_t *vc_off;   /* cells around each vertex (search order only) */
    const int64_t *vc;
} umesh;

static void shape_fn(int type, const double r[3], double N[8], double dN[8][3])
{
    const double a = r[0], b = r[1], c = r[2];
    switch (type) {
    case 4:
        N[0] = 1.0 - a - b - c; N[1] = a; N[2] = b; N[3] = c;
        for (int i = 0; i < 4; ++i) for (int k = 0; k < 3; ++k) dN[i][k] = 0.0;
        dN[0][0] = dN[0][1] = dN[0][2] = -1.0;
        dN[1][0] = 1.0; dN[2][1] = 1.0; dN[3][2] = 1.0;
        break;
    case 5:
        N[0] = (1 - a) * (1 - b) * (1 - c); N[1] = a * (1 - b) * (1 - c);
        N[2] = a * b * (1 - c); N[3] = (1 - a) * b * (1 - c); N[4] = c;
        dN[0][0] = -(1 - b) * (1 - c); dN[0][1] = -(1 - a) * (1 - c); dN[0][2] = -(1 - a) * (1 - b);
        dN[1][0] = (1 - b) * (1 - c);  dN[1][1] = -a * (1 - c);       dN[1][2] = -a * (1 - b);
        dN[2][0] = b * (1 - c);        dN[2][1] = a * (1 - c);        dN[2][2] = -a * b;
        dN[3][0] = -b * (1 - c);       dN[3][1] = (1 - a) * (1 - c);  dN[3][2] = -(1 - a) * b;
        dN[4][0] = 0.0;                dN[4][1] = 0.0;                dN[4][2] = 1.0;
        break;
    case 6:
        N[0] = (1 - a - b) * (1 - c); N[1] = a * (1 - c); N[2] = b * (1 - c);
        N[3] = (1 - a - b) * c;       N[4] = a * c;       N[5] = b * c;
        dN[0][0] = -(1 - c); dN[0][1] = -(1 - c); dN[0][2] = -(1 - a - b);
        dN[1][0] = (1 - c);  dN[1][1] = 0.0;      dN[1][2] = -a;
        dN[2][0] = 0.0;      dN[2][1] = (1 - c);  dN[2][2] = -b;
        dN[3][0] = -c;       dN[3][1] = -c;       dN[3][2] = (1 - a - b);
        dN[4][0] = c;        dN[4][1] = 0.0;      dN[4][2] = a;
        dN[5][0] = 0.0;      dN[5][1] = c;        dN[5][2] = b;
        break;
    default:
        N[0] = (1 - a) * (1 - b) * (1 - c); N[1] = a * (1 - b) * (1 - c);
        N[2] = a * b * (1 - c);             N[3] = (1 - a) * b * (1 - c);
        N[4] = (1 - a) * (1 - b) * c;       N[5] = a * (1 - b) * c;
        N[6] = a * b * c;                   N[7] = (1 - a) * b * c;
        dN[0][0] = -(1 - b) * (1 - c); dN[0][1] = -(1 - a) * (1 - c); dN[0][2] = -(1 - a) * (1 - b);
        dN[1][0] = (1 - b) * (1 - c);  dN[1][1] = -a * (1 - c);       dN[1][2] = -a * (1 - b);
        dN[2][0] = b * (1 - c);        dN[2][1] = a * (1 - c);        dN[2][2] = -a * b;
        dN[3][0] = -b * (1 - c);       dN[3][1] = (1 - a) * (1 - c);  dN[3][2] = -(1 - a) * b;
        dN[4][0] = -(1 - b) * c;       dN[4][1] = -(1 - a) * c;       dN[4][2] = (1 - a) * (1 - b);
        dN[5][0] = (1 - b) * c;        dN[5][1] = -a * c;             dN[5][2] = a * (1 - b);
        dN[6][0] = b * c;              dN[6][1] = a * c;              dN[6][2] = a * b;
        dN[7][0] = -b * c;             dN[7][1] = (1 - a) * c;        dN[7][2] = (1 - a) * b;
        break;
    }
}

/* How far (parametric) r lies outside the cell's reference domain; <= 0 inside. */
static double param_violation(int type, const double r[3])
{
    double v = -INFINITY;
    for (int k = 0; k < 3; ++k) v = fmax(v, -r[k]);
    if (type == 4) v = fmax(v, r[0] + r[1] + r[2] - 1.0);
    else if (type == 6) { v = fmax(v, r[0] + r[1] - 1.0); v = fmax(v, r[2] - 1.0); }
    else for (int k = 0; k < 3; ++k) v = fmax(v, r[k] - 1.0);
    return v;
}

/* Parametric coordinates of p in cell c (Newton's method); returns the
 * violation of the cell's inequalities (<= tau: inside). */
static double cell_param(const umesh *m, int64_t c, const double p[3], double r[3])
{
    const int type = m->type[c];
    const int32_t *vi = m->idx + m->off[c];
    const int nv = type;
    r[0] = r[1] = r[2] = (type == 4) ? 0.25 : (type == 6 ? 1.0 / 3.0 : 0.5);
    if (type == 6) r[2] = 0.5;
    if (type == 5) r[2] = 0.2;
    for (int it = 0; it < 60; ++it) {
        double N[8], dN[8][3], x[3] = {0, 0, 0}, J[3][3] = {{0}};
        shape_fn(type, r, N, dN);
        for (int i = 0; i < nv; ++i) {
            const double *X = m->X + 3 * (int64_t)vi[i];
            for (int k = 0; k < 3; ++k) {
                x[k] += N[i] * X[k];
                for (int l = 0; l < 3; ++l) J[k][l] += X[k] * dN[i][l];
            }
        }
        double F[3] = {x[0] - p[0], x[1] - p[1], x[2] - p[2]};
        double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
                     J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
                     J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
        if (!(fabs(det) > 0.0)) break;
        double d[3];
        for (int k = 0; k < 3; ++k) {
            double M[3][3];
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) M[a][b] = (b == k) ? F[a] : J[a][b];
            d[k] = (M[0][0] * (M[1][1] * M[2][2] - M[1][2] * M[2][1]) - M[0][1] * (M[1][0] * M[2][2] - M[1][2] * M[2][0]) +
                    M[0][2] * (M[1][0] * M[2][1] - M[1][1] * M[2][0])) / det;
        }
        for (int k = 0; k < 3; ++k) r[k] -= d[k];
        if (fabs(d[0]) + fabs(d[1]) + fabs(d[2]) < 1e-15) break;
        if (fabs(r[0]) + fabs(r[1]) + fabs(r[2]) > 1e6) break;   /* far outside: diverged */
    }
    /* a parametric point counts only if it maps back onto p (Newton converged) */
    double N[8], dN[8][3], x[3] = {0, 0, 0}, ext = 0.0;
    shape_fn(type, r, N, dN);
    for (int i = 0; i < nv; ++i) {
        const double *X = m->X + 3 * (int64_t)vi[i];
        for (int k = 0; k < 3; ++k) {
            x[k] += N[i] * X[k];
            ext = fmax(ext, fabs(X[k] - m->X[3 * (int64_t)vi[0] + k]));
        }
    }
    const double res = fabs(x[0] - p[0]) + fabs(x[1] - p[1]) + fabs(x[2] - p[2]);
    if (!(res <= 1e-9 * ext)) return INFINITY;
    return param_violation(type, r);
}

static void cell_value(const umesh *m, int64_t c, const double r[3], double v[3])
{
    const int type = m->type[c];
    const int32_t *vi = m->idx + m->off[c];
    double N[8], dN[8][3];
    shape_fn(type, r, N, dN);
    v[0] = v[1] = v[2] = 0.0;
    for (int i = 0; i < type; ++i)
        for (int k = 0; k < 3; ++k) v[k] += N[i] * m->V[3 * (int64_t)vi[i] + k];
}

/* Cell containing p, or -1; r receives its parametric coordinates.  Search
 * order: the hint, the cells sharing a vertex with it, then every cell (any
 * containing cell gives the same value on a conforming mesh). */
static int64_t umesh_locate(const umesh *m, const double p[3], int64_t hint, double r[3])
{
    if (hint >= 0) {
        if (cell_param(m, hint, p, r) <= m->tau) return hint;
        for (int64_t k = m->off[hint]; k < m->off[hint + 1]; ++k) {
            const int32_t v = m->idx[k];
            for (int64_t j = m->vc_off[v]; j < m->vc_off[v + 1]; ++j)
                if (cell_param(m, m->vc[j], p, r) <= m->tau) return m->vc[j];
        }
    }
    for (int64_t c = 0; c < m->n_cells; ++c)
        if (cell_param(m, c, p, r) <= m->tau) return c;
    return -1;
}

/* vertex -> cells adjacency (CSR); the caller frees both arrays */
static int build_adjacency(umesh *m, int64_t n_vertices)
{
    int64_t *cnt = (int64_t *)calloc((size_t)n_vertices + 1, sizeof(int64_t));
    if (!cnt) return -1;
    for (int64_t k = 0; k < m->off[m->n_cells]; ++k) cnt[m->idx[k] + 1] += 1;
    for (int64_t v = 0; v < n_vertices; ++v) cnt[v + 1] += cnt[v];
    int64_t *vc = (int64_t *)malloc(sizeof(int64_t) * (size_t)(cnt[n_vertices] + 1));
    int64_t *pos = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n_vertices + 1));
    if (!vc || !pos) { free(cnt); free(vc); free(pos); return -1; }
    memcpy(pos, cnt, sizeof(int64_t) * (size_t)(n_vertices + 1));
    for (int64_t c = 0; c < m->n_cells; ++c)
        for (int64_t k = m->off[c]; k < m->off[c + 1]; ++k) vc[pos[m->idx[k]]++] = c;
    free(pos);
    m->vc_off = cnt;
    m->vc = vc;
    return 0;
}

int or_umesh_sample(const double *X, const double *V, const int32_t *idx, const int64_t *off, const uint8_t *type,
                    int64_t n_cells, double tau, const double *points, int64_t n, double *v, int64_t *cell)
{
    umesh m = {X, V, idx, off, type, n_cells, tau, NULL, NULL};
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < n; ++i) {
        double r[3];
        int64_t c = umesh_locate(&m, points + 3 * i, -1, r);
        cell[i] = c;
        if (c >= 0) cell_value(&m, c, r, v + 3 * i);
        else v[3 * i] = v[3 * i + 1] = v[3 * i + 2] = NAN;
    }
    return 0;
}

/* One RK4 step in world coordinates (Listing 1) on the unstructured field. */
static int umesh_rk4(const umesh *m, const double p[3], double dt, double eps, int64_t *hint, double pn[3],
                     double *margin)
{
    double r[3], v[3], k[4][3], q[3];
    int64_t c = umesh_locate(m, p, *hint, r);
    const int64_t c0 = c;
    cell_value(m, c, r, v);
    if (!all_finite(v)) return OR_NANFIELD;
    double speed = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    if (speed < eps) { *margin = (eps - speed) / eps; return OR_STAGNANT; }
    const double w[3] = {0.5, 0.5, 1.0};
    for (int a = 0; a < 3; ++a) k[0][a] = dt * v[a];
    for (int s = 1; s < 4; ++s) {
        for (int a = 0; a < 3; ++a) q[a] = p[a] + w[s - 1] * k[s - 1][a];
        c = umesh_locate(m, q, c, r);
        if (c < 0) { double rr[3]; *margin = cell_param(m, c0, q, rr); return OR_EXIT; }
        cell_value(m, c, r, v);
        if (!all_finite(v)) return OR_NANFIELD;
        for (int a = 0; a < 3; ++a) k[s][a] = dt * v[a];
    }
    for (int a = 0; a < 3; ++a) pn[a] = p[a] + (k[0][a] + 2.0 * k[1][a] + 2.0 * k[2][a] + k[3][a]) / 6.0;
    c = umesh_locate(m, pn, c, r);
    if (c < 0) { double rr[3]; *margin = cell_param(m, c0, pn, rr); return OR_EXIT; }
    *hint = c;
    return OR_ACTIVE;
}

/* Streamlines on an unstructured field.  seeds and verts in world
 * coordinates (verts: n x (max_steps+1) x 3). */
int or_umesh_trace(const double *X, const double *V, const int32_t *idx, const int64_t *off, const uint8_t *type,
                   int64_t n_cells, int64_t n_vertices, double tau, const double *seeds, int64_t n, double dt,
                   int64_t max_steps, double eps, double *verts, int32_t *len, uint8_t *status, double *margin,
                   int nthreads)
{
    if (n < 0 || max_steps < 0 || n_cells < 0 || n_vertices < 0) return -1;
    umesh m = {X, V, idx, off, type, n_cells, tau, NULL, NULL};
    if (build_adjacency(&m, n_vertices)) return -1;
    set_threads(nthreads);
    int64_t stride = 3 * (max_steps + 1);
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t i = 0; i < n; ++i) {
        double p[3] = {seeds[3 * i], seeds[3 * i + 1], seeds[3 * i + 2]}, r[3];
        double *out = verts + stride * i;
        margin[i] = INFINITY;
        int64_t hint = umesh_locate(&m, p, -1, r);
        if (hint < 0) { len[i] = 0; status[i] = OR_OUT; continue; }
        memcpy(out, p, sizeof p);
        int64_t nv = 1;
        for (int64_t s = 0;; ++s) {
            if (s == max_steps) { status[i] = OR_MAXSTEPS; break; }
            double pn[3];
            int st = umesh_rk4(&m, p, dt, eps, &hint, pn, margin + i);
            if (st != OR_ACTIVE) { status[i] = (uint8_t)st; break; }
            memcpy(p, pn, sizeof p);
            memcpy(out + 3 * nv, p, sizeof p);
            ++nv;
        }
        len[i] = (int32_t)nv;
    }
    free((void *)m.vc_off);
    free((void *)m.vc);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Brick decomposition and the quantised field store.
 *
 * Reading (macrocells with a halo, Sec. 3.1.1): B bricks per axis; each owns
 * n = ceil((N-1)/B) cells per axis, brick b the index interval [b*n, b*n+n),
 * the last brick also its upper face; a point on an interior face belongs to
 * the upper brick.  A brick stores samples b*n-1 .. b*n+n+1 (n+3 per axis),
 * indices clamped to [0, N-1]: a one-cell ghost shell. */

int or_brick_cells(const int64_t dims[3], const int32_t bricks[3], int64_t n_out[3])
{
    for (int a = 0; a < 3; ++a) {
        if (dims[a] < 2 || bricks[a] < 1) return -1;
        int64_t n = (dims[a] - 1 + bricks[a] - 1) / bricks[a];
        if ((int64_t)(bricks[a] - 1) * n >= dims[a] - 1) return -1;  /* last brick would be empty */
        n_out[a] = n;
    }
    return 0;
}

/* Owning brick of an index point (destinationID for a uniform macrocell grid). */
int or_owner_brick(const int64_t dims[3], const int32_t bricks[3], const double p[3], int32_t b_out[3])
{
    int64_t n[3];
    if (or_brick_cells(dims, bricks, n)) return -1;
    for (int a = 0; a < 3; ++a) {
        int64_t b = (int64_t)floor(p[a] / (double)n[a]);
        if (b < 0) b = 0;
        if (b > bricks[a] - 1) b = bricks[a] - 1;
        b_out[a] = (int32_t)b;
    }
    return 0;
}

/* Round a finite double x (|x| <= 1 after scaling) to nearest-even with `bits`
 * significant bits and minimum normal exponent `emin` (values below 2^emin use
 * the fixed subnormal quantum 2^(emin - bits + 1)).  Returns the rounded value
 * as a double (exact).  Used for BF16 (bits 8, emin -126) and FP16 (bits 11,
 * emin -14). */
static double round_to_format(double x, int bits, int emin)
{
    if (x == 0.0 || !isfinite(x)) return x;
    int e;
    frexp(fabs(x), &e);              /* |x| = m * 2^e, m in [0.5, 1) -> exponent e-1 */
    int ex = e - 1;
    if (ex < emin) ex = emin;
    double quantum = ldexp(1.0, ex - (bits - 1));
    double q = nearbyint(x / quantum);  /* default rounding mode: to nearest, ties to even */
    return q * quantum;
}

/* Bit pattern of a value already representable in the format. */
static uint16_t encode_bits(double r, int dtype)
{
    if (r != r) return dtype == OR_BF16 ? 0x7FC0 : 0x7E00;
    uint16_t sign = signbit(r) ? 0x8000 : 0;
    double a = fabs(r);
    if (a == 0.0) return sign;
    int bits = dtype == OR_BF16 ? 8 : 11;
    int emin = dtype == OR_BF16 ? -126 : -14;
    int bias = dtype == OR_BF16 ? 127 : 15;
    int mant_bits = bits - 1;
    int e;
    double m = frexp(a, &e);
    int ex = e - 1;
    if (ex < emin) {                 /* subnormal: a = frac * 2^(emin - mant_bits) */
        uint32_t frac = (uint32_t)ldexp(a, -(emin - mant_bits));
        return (uint16_t)(sign | frac);
    }
    if (ex > bias) return (uint16_t)(sign | (dtype == OR_BF16 ? 0x7F80 : 0x7C00));  /* inf */
    uint32_t frac = (uint32_t)ldexp(m * 2.0 - 1.0, mant_bits);
    return (uint16_t)(sign | ((uint32_t)(ex + bias) << mant_bits) | frac);
}

/* Per-brick scale: the smallest power of two >= the largest finite |component|
 * over the brick's stored samples (owned and ghost); 1 if there is none or it
 * is zero.  Reading: a power-of-two form of the max-abs scale, so that a
 * sample stored in two bricks decodes to the same value in both. */
static float pow2_ceil(float m)
{
    if (!(m > 0.0f) || !isfinite(m)) return 1.0f;
    int e;
    float fr = frexpf(m, &e);        /* m = fr * 2^e, fr in [0.5, 1) */
    if (fr == 0.5f) return m;        /* already a power of two */
    return ldexpf(1.0f, e);
}

static int64_t clampi(int64_t v, int64_t lo, int64_t hi) { return v < lo ? lo : (v > hi ? hi : v); }

/* 21-bit fixed point: q = round-to-nearest-even(r * 2^20) with r = v / s_b,
 * clamped to +-(2^20 - 1).  Decodes as q * s_b * 2^-20. */
static int32_t fx21_q(float r)
{
    double q = nearbyint((double)r * 1048576.0);
    if (q > 1048575.0) q = 1048575.0;
    if (q < -1048575.0) q = -1048575.0;
    return (int32_t)q;
}

/* Quantise the global FP32 field into bricks.
 *   scales: nbricks floats (brick order x fastest), may be NULL; for OR_FX21
 *           the scale is the quantum s_b * 2^-20;
 *   codes:  nbricks * (n+3)^3 * 3 codes (brick-major, then z, y, x, comp), may
 *           be NULL: uint16 for BF16/FP16, int32 q for FX21 (INT32_MIN in all
 *           three components of a sample with a non-finite component);
 *   dequant: N^3 * 3 floats, each sample decoded with its owning brick's scale
 *            (exactly representable in float), may be NULL; for FX21 a sample
 *            with a non-finite component decodes as NaN in all components.
 * dtype OR_F32 gives scales of 1, no codes, dequant = input. */
int or_quantize_field(const float *F, const int64_t dims[3], const int32_t bricks[3], int dtype,
                      float *scales, void *codes_out, float *dequant)
{
    uint16_t *codes = (uint16_t *)codes_out;
    int32_t *qcodes = (int32_t *)codes_out;
    int64_t n[3];
    if (or_brick_cells(dims, bricks, n)) return -1;
    if (dtype != OR_F32 && dtype != OR_BF16 && dtype != OR_F16 && dtype != OR_FX21) return -1;
    int64_t nb = (int64_t)bricks[0] * bricks[1] * bricks[2];
    float *sc = (float *)malloc(sizeof(float) * (size_t)nb);
    if (!sc) return -2;
    int64_t S[3] = {n[0] + 3, n[1] + 3, n[2] + 3};
    for (int64_t b = 0; b < nb; ++b) {
        int64_t bx = b % bricks[0], by = (b / bricks[0]) % bricks[1], bz = b / ((int64_t)bricks[0] * bricks[1]);
        float m = 0.0f;
        for (int64_t sz = 0; sz < S[2]; ++sz)
            for (int64_t sy = 0; sy < S[1]; ++sy)
                for (int64_t sx = 0; sx < S[0]; ++sx) {
                    int64_t gx = clampi(bx * n[0] - 1 + sx, 0, dims[0] - 1);
                    int64_t gy = clampi(by * n[1] - 1 + sy, 0, dims[1] - 1);
                    int64_t gz = clampi(bz * n[2] - 1 + sz, 0, dims[2] - 1);
                    const float *s = F + 3 * ((gz * dims[1] + gy) * dims[0] + gx);
                    for (int c = 0; c < 3; ++c) {
                        float a = fabsf(s[c]);
                        if (isfinite(a) && a > m) m = a;
                    }
                }
        sc[b] = dtype == OR_F32 ? 1.0f : pow2_ceil(m);
        if (scales) scales[b] = dtype == OR_FX21 ? sc[b] / 1048576.0f : sc[b];
        if (codes_out && dtype == OR_FX21) {
            int32_t *cb = qcodes + b * S[0] * S[1] * S[2] * 3;
            for (int64_t sz = 0; sz < S[2]; ++sz)
                for (int64_t sy = 0; sy < S[1]; ++sy)
                    for (int64_t sx = 0; sx < S[0]; ++sx) {
                        int64_t gx = clampi(bx * n[0] - 1 + sx, 0, dims[0] - 1);
                        int64_t gy = clampi(by * n[1] - 1 + sy, 0, dims[1] - 1);
                        int64_t gz = clampi(bz * n[2] - 1 + sz, 0, dims[2] - 1);
                        const float *smp = F + 3 * ((gz * dims[1] + gy) * dims[0] + gx);
                        int32_t *o = cb + ((sz * S[1] + sy) * S[0] + sx) * 3;
                        int bad = !(isfinite(smp[0]) && isfinite(smp[1]) && isfinite(smp[2]));
                        for (int c = 0; c < 3; ++c) o[c] = bad ? INT32_MIN : fx21_q(smp[c] / sc[b]);
                    }
        } else if (codes_out && dtype != OR_F32) {
            uint16_t *cb = codes + b * S[0] * S[1] * S[2] * 3;
            for (int64_t sz = 0; sz < S[2]; ++sz)
                for (int64_t sy = 0; sy < S[1]; ++sy)
                    for (int64_t sx = 0; sx < S[0]; ++sx) {
                        int64_t gx = clampi(bx * n[0] - 1 + sx, 0, dims[0] - 1);
                        int64_t gy = clampi(by * n[1] - 1 + sy, 0, dims[1] - 1);
                        int64_t gz = clampi(bz * n[2] - 1 + sz, 0, dims[2] - 1);
                        const float *s = F + 3 * ((gz * dims[1] + gy) * dims[0] + gx);
                        for (int c = 0; c < 3; ++c) {
                            /* the quotient is taken in FP32, as the store does it */
                            float r = isfinite(s[c]) ? s[c] / sc[b] : NAN;
                            double q = round_to_format((double)r, dtype == OR_BF16 ? 8 : 11,
                                                       dtype == OR_BF16 ? -126 : -14);
                            cb[((sz * S[1] + sy) * S[0] + sx) * 3 + c] = encode_bits(q, dtype);
                        }
                    }
        }
    }
    if (dequant) {
        for (int64_t gz = 0; gz < dims[2]; ++gz)
            for (int64_t gy = 0; gy < dims[1]; ++gy)
                for (int64_t gx = 0; gx < dims[0]; ++gx) {
                    int64_t bx = clampi(gx / n[0], 0, bricks[0] - 1);
                    int64_t by = clampi(gy / n[1], 0, bricks[1] - 1);
                    int64_t bz = clampi(gz / n[2], 0, bricks[2] - 1);
                    float s_b = sc[(bz * bricks[1] + by) * bricks[0] + bx];
                    int64_t i = 3 * ((gz * dims[1] + gy) * dims[0] + gx);
                    if (dtype == OR_FX21) {
                        int bad = !(isfinite(F[i]) && isfinite(F[i + 1]) && isfinite(F[i + 2]));
                        for (int c = 0; c < 3; ++c)
                            dequant[i + c] = bad ? NAN : (float)((double)fx21_q(F[i + c] / s_b) * (double)s_b / 1048576.0);
                        continue;
                    }
                    for (int c = 0; c < 3; ++c) {
                        if (dtype == OR_F32) { dequant[i + c] = F[i + c]; continue; }
                        float r = isfinite(F[i + c]) ? F[i + c] / s_b : NAN;
                        double q = round_to_format((double)r, dtype == OR_BF16 ? 8 : 11,
                                                   dtype == OR_BF16 ? -126 : -14);
                        dequant[i + c] = (float)(q * (double)s_b);
                    }
                }
    }
    free(sc);
    return 0;
}

/* Decode one stored code with its brick's scale (exact in double). */
double or_decode(uint16_t code, float scale, int dtype)
{
    int bits = dtype == OR_BF16 ? 8 : 11;
    int mant_bits = bits - 1;
    int bias = dtype == OR_BF16 ? 127 : 15;
    int exp_bits = dtype == OR_BF16 ? 8 : 5;
    int sign = code >> 15;
    int ex = (code >> mant_bits) & ((1 << exp_bits) - 1);
    uint32_t frac = code & ((1u << mant_bits) - 1);
    double v;
    if (ex == (1 << exp_bits) - 1) v = frac ? NAN : INFINITY;
    else if (ex == 0) v = ldexp((double)frac, 1 - bias - mant_bits);
    else v = ldexp(1.0 + ldexp((double)frac, -mant_bits), ex - bias);
    v *= (double)scale;
    return sign ? -v : v;
}

/* max over samples of |v / spacing| (cells per unit time) */
double or_max_speed(const float *F, const int64_t dims[3], const double spacing[3])
{
    double m = 0.0;
    int64_t cells = dims[0] * dims[1] * dims[2];
    for (int64_t i = 0; i < cells; ++i) {
        double s = 0.0;
        for (int c = 0; c < 3; ++c) {
            double w = (double)F[3 * i + c] / spacing[c];
            s += w * w;
        }
        s = sqrt(s);
        if (s > m) m = s;
    }
    return m;
}
