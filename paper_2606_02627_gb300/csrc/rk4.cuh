// Device building blocks of the streamline kernels: brick lookup
// (destinationID), sampling inside a brick, one RK4 step (Listing 1) and the
// particle-record / warp-aggregated queue helpers.  Shared by the tracer's
// kernels and the request batch's kernel.
#pragma once

#include "tracer.cuh"

namespace sg {

template <int DT>
struct BrickRef {
    const typename Elem<DT>::T *data;
    float scale;
    int lo[3];   // first owned cell per axis
    int hi[3];   // one past the last owned cell (dims for the last brick)
};

template <int DT>
__device__ __forceinline__ void brick_of(const DevField &F, const int c[3], BrickRef<DT> &br)
{
    int b[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        int bb = c[a] / F.n[a];
        if (bb > F.B[a] - 1) bb = F.B[a] - 1;
        b[a] = bb;
        br.lo[a] = bb * F.n[a];
        br.hi[a] = (bb == F.B[a] - 1) ? F.dims[a] : br.lo[a] + F.n[a];
    }
    const int id = (b[2] * F.B[1] + b[1]) * F.B[0] + b[0];
    br.data = reinterpret_cast<const typename Elem<DT>::T *>(F.data) + (long long)id * F.brick_stride;
    br.scale = (DT == SG_F32) ? 1.0f : __ldg(F.scales + id);
}

// Trilinear sample at global cell c, fraction f, from the particle's brick,
// before the brick scale.  Returns SG_LINE_HALO if the point is outside the
// brick's ghost shell and SG_LINE_NANFIELD if the sample is not finite.
template <int DT, int LAYOUT>
__device__ __forceinline__ int sample_brick(const DevField &F, const BrickRef<DT> &br, const int c[3], const float f[3],
                                            float3 &u)
{
    const int sx = c[0] - br.lo[0] + 1, sy = c[1] - br.lo[1] + 1, sz = c[2] - br.lo[2] + 1;
    if ((unsigned)sx > (unsigned)(F.S[0] - 2) || (unsigned)sy > (unsigned)(F.S[1] - 2) ||
        (unsigned)sz > (unsigned)(F.S[2] - 2))
        return SG_LINE_HALO;
    bool bad;
    u = trilerp<DT, LAYOUT>(br.data, F, sx, sy, sz, f[0], f[1], f[2], bad);
    return bad ? SG_LINE_NANFIELD : 0;
}

// The same at a cell the brick owns, which is always inside its ghost shell.
template <int DT, int LAYOUT>
__device__ __forceinline__ int sample_owned(const DevField &F, const BrickRef<DT> &br, const int c[3], const float f[3],
                                            float3 &u)
{
    bool bad;
    u = trilerp<DT, LAYOUT>(br.data, F, c[0] - br.lo[0] + 1, c[1] - br.lo[1] + 1, c[2] - br.lo[2] + 1, f[0], f[1], f[2],
                            bad);
    return bad ? SG_LINE_NANFIELD : 0;
}

__device__ __forceinline__ bool in_domain(const DevField &F, const int q[3], const float g[3])
{
    return in_axis(q[0], g[0], F.nm1[0]) && in_axis(q[1], g[1], F.nm1[1]) && in_axis(q[2], g[2], F.nm1[2]);
}

__device__ __forceinline__ float out_dist(const DevField &F, const int q[3], const float g[3])
{
    return fmaxf(out_axis(q[0], g[0], F.nm1[0]), fmaxf(out_axis(q[1], g[1], F.nm1[1]), out_axis(q[2], g[2], F.nm1[2])));
}

// The products and sums below are written as explicit round-to-nearest
// intrinsics so that no multiply is fused into a later add: every kernel that
// inlines this step (tracer, Listing-1 form, request batch) then produces the
// same bits for the same particle.
//
// The brick scale s of the compact formats is a power of two, so it moves
// from the samples into the step factor without changing a bit:
// (u s) (dt/h) = u (s dt/h) and |u s| = |u| s exactly (no overflow or
// underflow at the scales a brick can have).
//
// One RK4 step of a particle owned by brick br.  On success updates (c, f)
// and returns SG_LINE_ACTIVE; otherwise returns the stop status and leaves the
// particle at P0.  margin is set for EXIT and STAGNANT.
template <int DT, int LAYOUT>
__device__ __forceinline__ int rk4_bricked(const DevField &F, const float dtc[3], float eps, const BrickRef<DT> &br,
                                           int c[3], float f[3], float &margin)
{
    float ds[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) ds[a] = (DT == SG_F32) ? dtc[a] : __fmul_rn(dtc[a], br.scale);
    float3 v;
    if (sample_owned<DT, LAYOUT>(F, br, c, f, v)) return SG_LINE_NANFIELD;
    float sp = sqrtf(__fadd_rn(__fadd_rn(__fmul_rn(v.x, v.x), __fmul_rn(v.y, v.y)), __fmul_rn(v.z, v.z)));
    if (DT != SG_F32) sp = __fmul_rn(sp, br.scale);
    if (sp < eps) {
        margin = (eps - sp) / eps;
        return SG_LINE_STAGNANT;
    }
    float k1[3] = {__fmul_rn(v.x, ds[0]), __fmul_rn(v.y, ds[1]), __fmul_rn(v.z, ds[2])};
    int q[3];
    float g[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) locate(f[a], 0.5f * k1[a], c[a], q[a], g[a]);
    if (!in_domain(F, q, g)) {
        margin = out_dist(F, q, g);
        return SG_LINE_EXIT;
    }
    if (int r = sample_brick<DT, LAYOUT>(F, br, q, g, v)) return r;
    float k2[3] = {__fmul_rn(v.x, ds[0]), __fmul_rn(v.y, ds[1]), __fmul_rn(v.z, ds[2])};
#pragma unroll
    for (int a = 0; a < 3; ++a) locate(f[a], 0.5f * k2[a], c[a], q[a], g[a]);
    if (!in_domain(F, q, g)) {
        margin = out_dist(F, q, g);
        return SG_LINE_EXIT;
    }
    if (int r = sample_brick<DT, LAYOUT>(F, br, q, g, v)) return r;
    float k3[3] = {__fmul_rn(v.x, ds[0]), __fmul_rn(v.y, ds[1]), __fmul_rn(v.z, ds[2])};
#pragma unroll
    for (int a = 0; a < 3; ++a) locate(f[a], k3[a], c[a], q[a], g[a]);
    if (!in_domain(F, q, g)) {
        margin = out_dist(F, q, g);
        return SG_LINE_EXIT;
    }
    if (int r = sample_brick<DT, LAYOUT>(F, br, q, g, v)) return r;
    const float k4[3] = {__fmul_rn(v.x, ds[0]), __fmul_rn(v.y, ds[1]), __fmul_rn(v.z, ds[2])};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float d = __fmul_rn(__fadd_rn(__fadd_rn(k1[a], k4[a]), __fmul_rn(2.0f, __fadd_rn(k2[a], k3[a]))),
                                  1.0f / 6.0f);
        locate(f[a], d, c[a], q[a], g[a]);
    }
    if (!in_domain(F, q, g)) {
        margin = out_dist(F, q, g);
        return SG_LINE_EXIT;
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        c[a] = q[a];
        f[a] = g[a];
    }
    return SG_LINE_ACTIVE;
}

// Stores and loads of data that no lane of this SM reads again soon (line
// vertices, queue records) skip L1 allocation, which leaves L1 to the field's
// cell records.
__device__ __forceinline__ void st_na(float *p, float v)
{
    asm volatile("st.global.L1::no_allocate.f32 [%0], %1;" ::"l"(p), "f"(v));
}

__device__ __forceinline__ void st_na4(void *p, uint4 v)
{
    asm volatile("st.global.L1::no_allocate.v4.u32 [%0], {%1, %2, %3, %4};" ::"l"(p), "r"(v.x), "r"(v.y), "r"(v.z),
                 "r"(v.w));
}

__device__ __forceinline__ uint4 ld_na4(const void *p)
{
    uint4 v;
    asm("ld.global.nc.L1::no_allocate.v4.u32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "l"(p));
    return v;
}

__device__ __forceinline__ void store_particle(Particle *dst, const int c[3], const float f[3], uint32_t line,
                                               uint32_t step)
{
    st_na4(dst, make_uint4(__float_as_uint(f[0]), __float_as_uint(f[1]), __float_as_uint(f[2]), line));
    st_na4(reinterpret_cast<uint4 *>(dst) + 1, make_uint4((unsigned)c[0], (unsigned)c[1], (unsigned)c[2], step));
}

__device__ __forceinline__ void load_particle(const Particle *src, int c[3], float f[3], uint32_t &line, uint32_t &step)
{
    const uint4 a = ld_na4(src);
    const uint4 b = ld_na4(reinterpret_cast<const uint4 *>(src) + 1);
    f[0] = __uint_as_float(a.x);
    f[1] = __uint_as_float(a.y);
    f[2] = __uint_as_float(a.z);
    line = a.w;
    c[0] = (int)b.x;
    c[1] = (int)b.y;
    c[2] = (int)b.z;
    step = b.w;
}

// Warp-aggregated append: every lane of the warp calls it; lanes with `want`
// get consecutive slots of dst from one atomicAdd on *count.
__device__ __forceinline__ void warp_append(bool want, Particle *dst, uint32_t *count, const int c[3], const float f[3],
                                            uint32_t line, uint32_t step)
{
    const unsigned m = __ballot_sync(SG_FULL_MASK, want);
    if (!m) return;
    const unsigned lane = threadIdx.x & 31;
    const int leader = __ffs(m) - 1;
    uint32_t base = 0;
    if ((int)lane == leader) base = atomicAdd(count, (uint32_t)__popc(m));
    base = __shfl_sync(SG_FULL_MASK, base, leader);
    if (want) store_particle(dst + base + __popc(m & ((1u << lane) - 1u)), c, f, line, step);
}


__device__ __forceinline__ uint8_t stop_code_t(int st, float margin, float tie_cells, float tie_eps_rel)
{
    uint8_t s = (uint8_t)st;
    if ((st == SG_LINE_EXIT && margin < tie_cells) || (st == SG_LINE_STAGNANT && margin < tie_eps_rel))
        s |= SG_LINE_TIE;
    return s;
}

}  // namespace sg
