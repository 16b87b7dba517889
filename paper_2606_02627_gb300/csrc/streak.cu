// Streaklines (Sec. 3.2, Listing 2): every step advances all released
// particles through the time-dependent field, then releases one new particle
// at every release point; a streakline joins the particles of one release
// point in birth order.
//
// The field is linear in time between stored slices (time s * slice_dt): a
// time t lies in the interval (s, s+1] in slice units, s = ceil(t/slice_dt)-1
// (at least 0), with weight alpha = t/slice_dt - s on slice s+1.  The slices a
// step needs are resident slots of the field, streamed in from page-locked
// host memory on a side stream; the step waits on the slots' events.
#include <math.h>
#include <string.h>

#include "rk4.cuh"

namespace sg {

struct StreakParams {
    DevField F;                 // geometry (data pointers below)
    const char *slot_data[6];   // per stage: slice a, slice b (3 stages)
    const float *slot_scale[6];
    float alpha[3];             // weight on slice b per stage time
    Particle *state;            // [R][inj]
    uint8_t *status;
    float *margin;
    const float *release;       // R x 3 world
    long long R;
    int inj;
    int births;                 // particles per release point released so far
    float dtc[3];
    float eps;
    double origin_d[3], spacing_d[3];
};

template <int DT>
__device__ __forceinline__ float3 sample_slot(const DevField &F, const char *data, const float *scales, int layout,
                                              const int q[3], const float g[3])
{
    using T = typename Elem<DT>::T;
    int b[3], lo[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        b[a] = min(q[a] / F.n[a], F.B[a] - 1);
        lo[a] = b[a] * F.n[a];
    }
    const int id = (b[2] * F.B[1] + b[1]) * F.B[0] + b[0];
    const T *brick = reinterpret_cast<const T *>(data) + (long long)id * F.brick_stride;
    const int sx = q[0] - lo[0] + 1, sy = q[1] - lo[1] + 1, sz = q[2] - lo[2] + 1;
    float3 v = layout == SG_LAYOUT_LINEAR  ? trilerp<DT, SG_LAYOUT_LINEAR>(brick, F, sx, sy, sz, g[0], g[1], g[2])
               : layout == SG_LAYOUT_CELL8 ? trilerp<DT, SG_LAYOUT_CELL8>(brick, F, sx, sy, sz, g[0], g[1], g[2])
                                           : trilerp<DT, SG_LAYOUT_TILED4>(brick, F, sx, sy, sz, g[0], g[1], g[2]);
    if (DT != SG_F32) {
        const float s = __ldg(scales + id);
        v.x *= s;
        v.y *= s;
        v.z *= s;
    }
    return v;
}

template <int DT>
__device__ __forceinline__ float3 sample_time(const StreakParams &P, int layout, int stage, const int q[3],
                                              const float g[3])
{
    const float3 a = sample_slot<DT>(P.F, P.slot_data[2 * stage], P.slot_scale[2 * stage], layout, q, g);
    const float3 b = sample_slot<DT>(P.F, P.slot_data[2 * stage + 1], P.slot_scale[2 * stage + 1], layout, q, g);
    const float al = P.alpha[stage];
    return make_float3(lerpf(a.x, b.x, al), lerpf(a.y, b.y, al), lerpf(a.z, b.z, al));
}

__device__ __forceinline__ bool dom(const DevField &F, const int q[3], const float g[3])
{
    return in_axis(q[0], g[0], F.nm1[0]) && in_axis(q[1], g[1], F.nm1[1]) && in_axis(q[2], g[2], F.nm1[2]);
}

__device__ __forceinline__ float dom_out(const DevField &F, const int q[3], const float g[3])
{
    return fmaxf(out_axis(q[0], g[0], F.nm1[0]), fmaxf(out_axis(q[1], g[1], F.nm1[1]), out_axis(q[2], g[2], F.nm1[2])));
}

// One RK4 step of a particle through the time-dependent field (stage times
// t, t+dt/2, t+dt/2, t+dt use stage slots 0, 1, 1, 2).  On success updates
// (c, f) and returns SG_LINE_ACTIVE; else the stop status (margin set for
// EXIT and STAGNANT), the particle left at P0.
template <int DT>
__device__ __forceinline__ int rk4_time(const StreakParams &P, int layout, int c[3], float f[3], float &margin)
{
    int q[3];
    float g[3];
    float k1[3], k2[3], k3[3], k4[3];
    float3 v = sample_time<DT>(P, layout, 0, c, f);
    if (bad3(v)) return SG_LINE_NANFIELD;
    const float sp = sqrtf(v.x * v.x + v.y * v.y + v.z * v.z);
    if (sp < P.eps) {
        margin = (P.eps - sp) / P.eps;
        return SG_LINE_STAGNANT;
    }
    k1[0] = v.x * P.dtc[0]; k1[1] = v.y * P.dtc[1]; k1[2] = v.z * P.dtc[2];
    for (int a = 0; a < 3; ++a) locate(f[a], 0.5f * k1[a], c[a], q[a], g[a]);
    if (!dom(P.F, q, g)) { margin = dom_out(P.F, q, g); return SG_LINE_EXIT; }
    v = sample_time<DT>(P, layout, 1, q, g);
    if (bad3(v)) return SG_LINE_NANFIELD;
    k2[0] = v.x * P.dtc[0]; k2[1] = v.y * P.dtc[1]; k2[2] = v.z * P.dtc[2];
    for (int a = 0; a < 3; ++a) locate(f[a], 0.5f * k2[a], c[a], q[a], g[a]);
    if (!dom(P.F, q, g)) { margin = dom_out(P.F, q, g); return SG_LINE_EXIT; }
    v = sample_time<DT>(P, layout, 1, q, g);
    if (bad3(v)) return SG_LINE_NANFIELD;
    k3[0] = v.x * P.dtc[0]; k3[1] = v.y * P.dtc[1]; k3[2] = v.z * P.dtc[2];
    for (int a = 0; a < 3; ++a) locate(f[a], k3[a], c[a], q[a], g[a]);
    if (!dom(P.F, q, g)) { margin = dom_out(P.F, q, g); return SG_LINE_EXIT; }
    v = sample_time<DT>(P, layout, 2, q, g);
    if (bad3(v)) return SG_LINE_NANFIELD;
    k4[0] = v.x * P.dtc[0]; k4[1] = v.y * P.dtc[1]; k4[2] = v.z * P.dtc[2];
    for (int a = 0; a < 3; ++a)
        locate(f[a], (k1[a] + k4[a] + 2.0f * (k2[a] + k3[a])) * (1.0f / 6.0f), c[a], q[a], g[a]);
    if (!dom(P.F, q, g)) { margin = dom_out(P.F, q, g); return SG_LINE_EXIT; }
    for (int a = 0; a < 3; ++a) {
        c[a] = q[a];
        f[a] = g[a];
    }
    return SG_LINE_ACTIVE;
}

// One RK4 step of every released, live particle.
template <int DT>
__global__ void streak_advect_kernel(const __grid_constant__ StreakParams P, int layout)
{
    const long long total = P.R * P.inj;
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < total; k += (long long)gridDim.x * blockDim.x) {
        const int b = (int)(k % P.inj);
        if (b >= P.births || P.status[k] != SG_LINE_ACTIVE) continue;
        Particle pr = P.state[k];
        int c[3] = {pr.cx, pr.cy, pr.cz};
        float f[3] = {pr.fx, pr.fy, pr.fz};
        float margin = INFINITY;
        const int st = rk4_time<DT>(P, layout, c, f, margin);
        if (st == SG_LINE_ACTIVE) {
            pr.cx = c[0]; pr.cy = c[1]; pr.cz = c[2];
            pr.fx = f[0]; pr.fy = f[1]; pr.fz = f[2];
            pr.step += 1;
            P.state[k] = pr;
        } else {
            P.status[k] = (uint8_t)st;
            P.margin[k] = margin;
        }
    }
}

// Path lines: every live particle takes step `step` (from time (step-1) dt)
// and writes its vertex; the line stops at its first failed step or when it
// reaches max_steps.  *active counts the lines still moving afterwards.
struct PathLines {
    Particle *state;
    float *slab;
    uint32_t *len;
    uint8_t *status;
    float *margin;
    long long W;
    long long n;
    uint32_t max_steps;
    float tie_cells, tie_eps_rel;
    unsigned long long *active;
};

template <int DT>
__global__ void path_advect_kernel(const __grid_constant__ StreakParams P, int layout, PathLines L, uint32_t step)
{
    unsigned long long moving = 0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < L.n; i += (long long)gridDim.x * blockDim.x) {
        if (L.status[i] != SG_LINE_ACTIVE) continue;
        if (step > L.max_steps) {
            L.status[i] = SG_LINE_MAXSTEPS;
            continue;
        }
        Particle pr = L.state[i];
        int c[3] = {pr.cx, pr.cy, pr.cz};
        float f[3] = {pr.fx, pr.fy, pr.fz};
        float margin = INFINITY;
        const int st = rk4_time<DT>(P, layout, c, f, margin);
        if (st == SG_LINE_ACTIVE) {
            pr.cx = c[0]; pr.cy = c[1]; pr.cz = c[2];
            pr.fx = f[0]; pr.fy = f[1]; pr.fz = f[2];
            pr.step = step;
            L.state[i] = pr;
            float *o = L.slab + (i * L.W + step) * 3;
            o[0] = fmaf(P.F.spacing[0], (float)c[0] + f[0], P.F.origin[0]);
            o[1] = fmaf(P.F.spacing[1], (float)c[1] + f[1], P.F.origin[1]);
            o[2] = fmaf(P.F.spacing[2], (float)c[2] + f[2], P.F.origin[2]);
            L.len[i] = step + 1;
            if (step >= L.max_steps) L.status[i] = SG_LINE_MAXSTEPS;
            else ++moving;
        } else {
            L.status[i] = stop_code_t(st, margin, L.tie_cells, L.tie_eps_rel);
            L.margin[i] = margin;
        }
    }
    for (int o = 16; o > 0; o >>= 1) moving += __shfl_xor_sync(SG_FULL_MASK, moving, o);
    if ((threadIdx.x & 31) == 0 && moving) atomicAdd(L.active, moving);
}

// Path-line start: particle state, first vertex (the seed), status.
__global__ void path_init_kernel(const float *seeds, long long n, DevField F, double ox, double oy, double oz,
                                 double hx, double hy, double hz, PathLines L)
{
    const double org[3] = {ox, oy, oz}, sp[3] = {hx, hy, hz};
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        double p[3];
        bool inside = true;
        for (int a = 0; a < 3; ++a) {
            p[a] = ((double)seeds[3 * i + a] - org[a]) / sp[a];
            inside = inside && p[a] >= 0.0 && p[a] <= (double)F.nm1[a];
        }
        L.margin[i] = INFINITY;
        if (!inside) {
            L.len[i] = 0;
            L.status[i] = SG_LINE_OUT;
            continue;
        }
        Particle pr;
        int c[3];
        float f[3];
        for (int a = 0; a < 3; ++a) {
            const double fl = floor(p[a]);
            c[a] = (int)fl;
            f[a] = (float)(p[a] - fl);
            if (f[a] >= 1.0f) { f[a] = 0.0f; c[a] += 1; }
        }
        pr.cx = c[0]; pr.cy = c[1]; pr.cz = c[2];
        pr.fx = f[0]; pr.fy = f[1]; pr.fz = f[2];
        pr.line = (uint32_t)i;
        pr.step = 0;
        L.state[i] = pr;
        float *o = L.slab + i * L.W * 3;
        o[0] = seeds[3 * i];
        o[1] = seeds[3 * i + 1];
        o[2] = seeds[3 * i + 2];
        L.len[i] = 1;
        L.status[i] = L.max_steps == 0 ? SG_LINE_MAXSTEPS : SG_LINE_ACTIVE;
    }
}

// Releases birth `birth` at every release point (birth 0 also resets the rest).
__global__ void streak_release_kernel(const __grid_constant__ StreakParams P, int birth, int reset)
{
    const long long total = P.R * P.inj;
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < total; k += (long long)gridDim.x * blockDim.x) {
        const int b = (int)(k % P.inj);
        const long long r = k / P.inj;
        if (b != birth) {
            if (reset) {
                P.status[k] = 255;       // not released yet
                P.margin[k] = INFINITY;
            }
            continue;
        }
        double p[3];
        bool inside = true;
        for (int a = 0; a < 3; ++a) {
            p[a] = ((double)P.release[3 * r + a] - P.origin_d[a]) / P.spacing_d[a];
            inside = inside && p[a] >= 0.0 && p[a] <= (double)P.F.nm1[a];
        }
        Particle pr;
        int c[3] = {0, 0, 0};
        float f[3] = {0.f, 0.f, 0.f};
        if (inside) {
            for (int a = 0; a < 3; ++a) {
                const double fl = floor(p[a]);
                c[a] = (int)fl;
                f[a] = (float)(p[a] - fl);
                if (f[a] >= 1.0f) { f[a] = 0.0f; c[a] += 1; }
            }
        }
        pr.cx = c[0]; pr.cy = c[1]; pr.cz = c[2];
        pr.fx = f[0]; pr.fy = f[1]; pr.fz = f[2];
        pr.line = (uint32_t)r;
        pr.step = 0;
        P.state[k] = pr;
        P.status[k] = inside ? SG_LINE_ACTIVE : SG_LINE_OUT;
        P.margin[k] = INFINITY;
    }
}

// Per release point: live particles (low 40 bits) and runs of consecutive live
// particles (high 24 bits), packed for one scan.
// Also adds every released particle's successful steps to *steps_total.
__global__ void streak_count_kernel(const uint8_t *status, const Particle *state, long long R, int inj, int births,
                                    unsigned long long *packed, unsigned long long *steps_total)
{
    for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < R; r += (long long)gridDim.x * blockDim.x) {
        unsigned long long live = 0, runs = 0, steps = 0;
        bool prev = false;
        for (int b = 0; b < births; ++b) {
            const uint8_t st = status[r * inj + b];
            const bool l = st == SG_LINE_ACTIVE;
            live += l;
            runs += (l && !prev);
            prev = l;
            if (st != 255 && st != SG_LINE_OUT) steps += state[r * inj + b].step;
        }
        packed[r] = live + (runs << 40);
        atomicAdd(steps_total, steps);
    }
}

// Exclusive scan of packed[0..n) into excl (n+1 entries); single pass per
// 1024-entry chunk with a carried prefix (n is the number of release points).
__global__ void scan_u64_kernel(const unsigned long long *in, long long n, unsigned long long *excl, int64_t *totals)
{
    __shared__ unsigned long long ws[32];
    __shared__ unsigned long long carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const unsigned lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (long long base = 0; base < n; base += blockDim.x) {
        const long long i = base + threadIdx.x;
        const unsigned long long v = i < n ? in[i] : 0ull;
        unsigned long long x = v;
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(SG_FULL_MASK, x, o);
            if ((int)lane >= o) x += y;
        }
        if (lane == 31) ws[warp] = x;
        __syncthreads();
        if (warp == 0) {
            unsigned long long w = lane < (blockDim.x >> 5) ? ws[lane] : 0ull;
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned long long y = __shfl_up_sync(SG_FULL_MASK, w, o);
                if ((int)lane >= o) w += y;
            }
            ws[lane] = w;
        }
        __syncthreads();
        const unsigned long long before = carry + (warp ? ws[warp - 1] : 0ull) + x - v;
        if (i < n) excl[i] = before;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry = before + v;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        excl[n] = carry;
        totals[0] = (int64_t)(carry & ((1ull << 40) - 1));   // vertices
        totals[1] = (int64_t)(carry >> 40);                  // lines
    }
}

// One thread per release point: its runs become lines.
__global__ void streak_gather_kernel(const Particle *state, const uint8_t *status, long long R, int inj, int births,
                                     const unsigned long long *excl, DevField F, int64_t *offsets, float *vertices,
                                     uint8_t *st_out, float *mg_out, int32_t *source)
{
    for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < R; r += (long long)gridDim.x * blockDim.x) {
        long long v = (long long)(excl[r] & ((1ull << 40) - 1));
        long long line = (long long)(excl[r] >> 40);
        bool prev = false;
        for (int b = 0; b < births; ++b) {
            const long long k = r * inj + b;
            const bool l = status[k] == SG_LINE_ACTIVE;
            if (l && !prev) {
                if (offsets) offsets[line] = v;
                if (st_out) st_out[line] = SG_LINE_ACTIVE;
                if (mg_out) mg_out[line] = INFINITY;
                if (source) source[line] = (int32_t)r;
                ++line;
            }
            if (l) {
                if (vertices) {
                    const Particle p = state[k];
                    vertices[3 * v] = fmaf(F.spacing[0], (float)p.cx + p.fx, F.origin[0]);
                    vertices[3 * v + 1] = fmaf(F.spacing[1], (float)p.cy + p.fy, F.origin[1]);
                    vertices[3 * v + 2] = fmaf(F.spacing[2], (float)p.cz + p.fz, F.origin[2]);
                }
                ++v;
            }
            prev = l;
        }
    }
    if (offsets && blockIdx.x == 0 && threadIdx.x == 0) offsets[excl[R] >> 40] = (int64_t)(excl[R] & ((1ull << 40) - 1));
}

static StreakParams streak_params(const sg_tracer *t)
{
    StreakParams P;
    memset(&P, 0, sizeof P);
    const sg_field *f = t->field;
    P.F = field_view(f, 0);
    for (int i = 0; i < 6; ++i) {
        P.slot_data[i] = f->slot_data[0];
        P.slot_scale[i] = f->slot_scales[0];
    }
    P.state = t->sk_state;
    P.status = t->sk_status;
    P.margin = t->sk_margin;
    P.release = t->seeds;
    P.R = t->n_seeds;
    P.inj = t->p.inject_steps;
    P.births = t->births;
    for (int a = 0; a < 3; ++a) {
        P.dtc[a] = (float)(t->p.dt / f->desc.spacing[a]);
        P.origin_d[a] = f->desc.origin[a];
        P.spacing_d[a] = f->desc.spacing[a];
    }
    P.eps = t->p.eps;
    return P;
}

static int grid_for(const sg_tracer *t, long long n)
{
    long long g = (n + 255) / 256;
    const long long cap = (long long)t->ctx->sm_count * 16;
    if (g > cap) g = cap;
    return g < 1 ? 1 : (int)g;
}

sg_status streak_upload(sg_tracer *t, cudaStream_t s)
{
    t->births = 1;
    t->steps_done = 0;
    StreakParams P = streak_params(t);
    const long long total = t->n_seeds * (long long)t->p.inject_steps;
    if (total == 0) return SG_OK;
    streak_release_kernel<<<grid_for(t, total), 256, 0, s>>>(P, 0, 1);
    SG_CUDA(cudaGetLastError());
    return SG_OK;
}

// Slice pair of time t: s = ceil(t/slice_dt) - 1 (>= 0), alpha = t/slice_dt - s.
// A time within a relative 1e-9 of a slice time is taken as that slice time,
// so that a step whose dt is a multiple or a fraction of slice_dt never asks
// for a slice whose weight is a rounding error.
static void slice_pair(double t, double sdt, int *s_out, double *alpha_out)
{
    double u = t / sdt;
    const double r = nearbyint(u);
    if (fabs(u - r) <= 1e-9 * fmax(1.0, fabs(u))) u = r;
    long long s = (long long)ceil(u) - 1;
    if (s < 0) s = 0;
    *s_out = (int)s;
    *alpha_out = u - (double)s;
}

// The resident slots that step j's three stage times sample (into P), after
// the stream has waited for each slot's copy; need[][] lists the slices.
static sg_status stage_slots(sg_tracer *t, int j, StreakParams &P, int need[3][2], cudaStream_t s)
{
    sg_field *f = t->field;
    const double dt = t->p.dt, sdt = f->desc.slice_dt;
    const double t0 = (double)(j - 1) * dt;
    const double times[3] = {t0, t0 + 0.5 * dt, t0 + dt};
    for (int st = 0; st < 3; ++st) {
        int sl;
        double al;
        slice_pair(times[st], sdt, &sl, &al);
        // a slice with weight zero is not needed: sample the other one twice
        need[st][0] = al == 1.0 ? sl + 1 : sl;
        need[st][1] = al == 0.0 ? sl : sl + 1;
        for (int h = 0; h < 2; ++h) {
            const int slice = need[st][h];
            const int slot = slice % f->desc.n_slots;
            SG_CHECK(f->slot_slice[slot] == slice, SG_ERR_STATE,
                     "step %d needs time slice %d, which is not resident (slot %d holds %d)", j, slice, slot,
                     f->slot_slice[slot]);
            SG_CUDA(cudaStreamWaitEvent(s, f->slot_ready[slot], 0));
            P.slot_data[2 * st + h] = f->slot_data[slot];
            P.slot_scale[2 * st + h] = f->slot_scales[slot];
        }
        P.alpha[st] = (float)al;
    }
    return SG_OK;
}

// Later streams into the slots a step sampled wait for the step.
static sg_status release_slots(sg_tracer *t, const int need[3][2], cudaStream_t s)
{
    sg_field *f = t->field;
    for (int st = 0; st < 3; ++st)
        for (int h = 0; h < 2; ++h) SG_CUDA(cudaEventRecord(f->slot_used[need[st][h] % f->desc.n_slots], s));
    return SG_OK;
}

sg_status streak_step(sg_tracer *t, int32_t n_steps, int32_t *any_active, cudaStream_t s)
{
    sg_field *f = t->field;
    for (int i = 0; i < n_steps; ++i) {
        const int j = t->steps_done + 1;
        StreakParams P = streak_params(t);
        int need[3][2];
        sg_status st = stage_slots(t, j, P, need, s);
        if (st) return st;
        const long long total = t->n_seeds * (long long)t->p.inject_steps;
        if (total > 0) {
            with_dtype(f->desc.dtype, [&](auto D) {
                streak_advect_kernel<decltype(D)::value><<<grid_for(t, total), 256, 0, s>>>(P, f->desc.layout);
            });
            SG_CUDA(cudaGetLastError());
            if (j < t->p.inject_steps) {
                streak_release_kernel<<<grid_for(t, total), 256, 0, s>>>(P, j, 0);
                SG_CUDA(cudaGetLastError());
            }
        }
        st = release_slots(t, need, s);
        if (st) return st;
        if (j < t->p.inject_steps) t->births = j + 1;
        t->steps_done = j;
    }
    t->scanned = false;
    if (any_active) {
        SG_CUDA(cudaStreamSynchronize(s));
        *any_active = t->n_seeds > 0 ? 1 : 0;
    }
    return SG_OK;
}

// ------------------------------------------------------------------ path lines

static PathLines path_lines(const sg_tracer *t)
{
    PathLines L;
    L.state = t->q;
    L.slab = t->slab;
    L.len = t->line_len;
    L.status = t->line_status;
    L.margin = t->line_margin;
    L.W = slab_stride(t->p.max_steps);
    L.n = t->n_lines;
    L.max_steps = (uint32_t)t->p.max_steps;
    L.tie_cells = t->p.tie_cells;
    L.tie_eps_rel = t->p.tie_eps_rel;
    L.active = reinterpret_cast<unsigned long long *>(t->totals + 3);
    return L;
}

sg_status path_upload(sg_tracer *t, cudaStream_t s)
{
    t->steps_done = 0;
    const long long n = t->n_lines;
    if (n == 0) return SG_OK;
    const sg_field *f = t->field;
    const sg_field_desc &d = f->desc;
    path_init_kernel<<<grid_for(t, n), 256, 0, s>>>(t->seeds, n, field_view(f, 0), d.origin[0], d.origin[1],
                                                    d.origin[2], d.spacing[0], d.spacing[1], d.spacing[2],
                                                    path_lines(t));
    SG_CUDA(cudaGetLastError());
    return SG_OK;
}

// Advances every moving path line by up to n_steps steps (time slices of
// each step must be resident); *any_active: lines still moving.
sg_status path_step(sg_tracer *t, int32_t n_steps, int32_t *any_active, cudaStream_t s)
{
    sg_field *f = t->field;
    const PathLines L = path_lines(t);
    bool ran = false;
    for (int i = 0; i < n_steps && t->steps_done < t->p.max_steps; ++i) {
        const int j = t->steps_done + 1;
        StreakParams P = streak_params(t);
        int need[3][2];
        sg_status st = stage_slots(t, j, P, need, s);
        if (st) return st;
        SG_CUDA(cudaMemsetAsync(L.active, 0, sizeof(unsigned long long), s));
        if (L.n > 0) {
            with_dtype(f->desc.dtype, [&](auto D) {
                path_advect_kernel<decltype(D)::value><<<grid_for(t, L.n), 256, 0, s>>>(P, f->desc.layout, L,
                                                                                      (uint32_t)j);
            });
            SG_CUDA(cudaGetLastError());
        }
        st = release_slots(t, need, s);
        if (st) return st;
        t->steps_done = j;
        ran = true;
    }
    t->scanned = false;
    if (any_active) {
        unsigned long long moving = 0;
        if (ran) SG_CUDA(cudaMemcpyAsync(&moving, L.active, sizeof moving, cudaMemcpyDeviceToHost, s));
        SG_CUDA(cudaStreamSynchronize(s));
        *any_active = (ran && moving > 0) ? 1 : 0;
    }
    return SG_OK;
}

sg_status launch_streak_scan(sg_tracer *t, cudaStream_t s)
{
    const long long R = t->n_seeds;
    unsigned long long *packed = t->block_sums;      // R + 2 entries are carved for this
    unsigned long long *excl = reinterpret_cast<unsigned long long *>(t->offsets);
    SG_CUDA(cudaMemsetAsync(t->totals + 2, 0, sizeof(int64_t), s));
    if (R > 0) {
        streak_count_kernel<<<grid_for(t, R), 256, 0, s>>>(t->sk_status, t->sk_state, R, t->p.inject_steps, t->births,
                                                           packed, reinterpret_cast<unsigned long long *>(t->totals + 2));
        SG_CUDA(cudaGetLastError());
    }
    scan_u64_kernel<<<1, 1024, 0, s>>>(packed, R, excl, t->totals);
    SG_CUDA(cudaGetLastError());
    return SG_OK;
}

sg_status launch_streak_gather(sg_tracer *t, int64_t *offsets, float *vertices, uint8_t *status, float *margin,
                               int32_t *source, cudaStream_t s)
{
    const long long R = t->n_seeds;
    const unsigned long long *excl = reinterpret_cast<const unsigned long long *>(t->offsets);
    streak_gather_kernel<<<grid_for(t, R > 0 ? R : 1), 256, 0, s>>>(t->sk_state, t->sk_status, R, t->p.inject_steps,
                                                                     t->births, excl, field_view(t->field, 0), offsets,
                                                                     vertices, status, margin, source);
    SG_CUDA(cudaGetLastError());
    return SG_OK;
}

sg_status launch_streak_release(sg_tracer *t, int birth, cudaStream_t s)
{
    StreakParams P = streak_params(t);
    const long long total = t->n_seeds * (long long)t->p.inject_steps;
    if (total == 0) return SG_OK;
    streak_release_kernel<<<grid_for(t, total), 256, 0, s>>>(P, birth, 0);
    SG_CUDA(cudaGetLastError());
    return SG_OK;
}

}  // namespace sg
