// Internal definitions shared by the translation units of libstreamgb.
//
// Method (Zellmann et al., "Streami", Sec. 3.1, Listing 1): particles are
// advected by classical RK4 with stage points P0 + k1/2, P0 + k2/2, P0 + k3,
// k_i = dt * v(stage point) / spacing (cells), through a structured field
// sampled by trilinear interpolation; a failed sample ends the particle; the
// destination macrocell (brick) is computed from the new position.
//
// Position representation: a particle keeps its global cell index (int) and
// its fraction inside the cell (float in [0,1)).  Stage points are formed as
// fraction + offset relative to the particle's cell, so the fraction used by
// the interpolation carries ~2^-24 cells of rounding wherever the particle is,
// and moving between bricks needs no change of coordinates.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>
#include <stddef.h>

#include <type_traits>

#include "streamgb.h"

#define SG_FULL_MASK 0xffffffffu

namespace sg {

// ------------------------------------------------------------------ errors
void set_error(const char *fmt, ...);
sg_status cuda_error(cudaError_t e, const char *what);
#define SG_CUDA(call)                                                   \
    do {                                                                \
        cudaError_t e_ = (call);                                        \
        if (e_ != cudaSuccess) return ::sg::cuda_error(e_, #call);      \
    } while (0)
#define SG_CHECK(cond, code, ...)                                       \
    do {                                                                \
        if (!(cond)) {                                                  \
            ::sg::set_error(__VA_ARGS__);                               \
            return (code);                                              \
        }                                                               \
    } while (0)

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Bump allocator over a caller-owned buffer.
struct Carve {
    char *base;
    size_t off;
    size_t cap;
    void *take(size_t bytes, size_t align = 256) {
        off = align_up(off, align);
        void *p = base ? base + off : nullptr;
        off += bytes;
        return p;
    }
};

// ------------------------------------------------------------------ field geometry

// Device view of one resident slot of a bricked field.
struct DevField {
    const char *data;        // slot storage: nb bricks of brick_bytes each
    const float *scales;     // per-brick decode scale (1 for FP32)
    int dims[3];             // samples per axis
    int nm1[3];              // dims - 1: upper face index
    int n[3];                // owned cells per brick per axis
    int B[3];                // bricks per axis
    int S[3];                // stored samples per brick per axis (n + 3)
    int T[3];                // tiles of 4 per axis (tiled layout)
    int C[3];                // cells per brick per axis (cell-record layout: n + 2)
    long long brick_elems;   // samples per brick (with tile padding)
    long long brick_stride;  // samples from one brick's start to the next
    float origin[3];
    float spacing[3];
};

}  // namespace sg

struct sg_context {
    int device;
    int sm_count;
    int max_threads_per_sm;
    int max_smem_optin;
    long long l2_bytes;
};

struct sg_field {
    sg_context *ctx;
    sg_field_desc desc;
    sg::DevField geom;       // data/scales of slot 0 (per-slot pointers below)
    char *storage;
    size_t bytes;
    int nb;
    size_t elem_bytes;       // 16 (FP32) or 8 (BF16/FP16); 12 for SG_FIELD_GLOBAL
    size_t brick_bytes;
    char *slot_data[64];
    float *slot_scales[64];
    unsigned *maxbits;       // nb scratch words for the per-brick max-abs reduction
    float *staging;          // one global FP32 slice (streamed slices)
    unsigned *speed_bits;    // 1 word: max speed reduction
    int slot_slice[64];      // slice held by each slot (-1 = none)
    cudaEvent_t slot_ready[64];  // recorded when a slot's contents are complete
    cudaEvent_t slot_used[64];   // recorded after the last queued step that reads a slot
};

namespace sg {

DevField field_view(const sg_field *f, int slot);

// ------------------------------------------------------------------ particles

// Queue record of one particle: 32 bytes, two 16-byte vectors.
struct __align__(16) Particle {
    float fx, fy, fz;        // fraction in the cell, [0,1)
    uint32_t line;           // line (seed) index
    int cx, cy, cz;          // global cell index
    uint32_t step;           // successful steps so far
};

// Counters of a tracer's round loop (device memory).
struct Ctrl {
    uint32_t q_count;        // particles in the brick-sorted queue of this round
    uint32_t q_head;         // pop cursor of that queue
    uint32_t o_count;        // records appended to the outgoing buffer this round
    uint32_t p_count;        // parked records (reached the step horizon)
    uint32_t round;          // rounds run by the current call
    uint32_t err;            // bit 0: round cap reached with particles left
    uint32_t max_rounds;
    uint32_t horizon;        // a particle advances while step < horizon
    uint32_t last_rounds;    // rounds of the last finished call
    // rounds policy: with window > 0 a round advances only the particles of
    // `window` consecutive bricks (round-robin from win_lo, skipping empty
    // ones); the queue then holds q_total records, of which [win_start,
    // q_count) are the round's and the rest are carried to the next round
    uint32_t window;
    uint32_t win_lo;
    uint32_t win_start;
    uint32_t q_total;
    uint32_t pad[3];
};

enum { CTRL_ERR_ROUND_LIMIT = 1u, CTRL_ERR_TIMEOUT = 2u };

// ------------------------------------------------------------------ sampling helpers

template <int DT> struct Elem;
template <> struct Elem<SG_F32> { using T = float4; };
template <> struct Elem<SG_BF16> { using T = uint2; };
template <> struct Elem<SG_F16> { using T = uint2; };
template <> struct Elem<SG_FX21> { using T = uint2; };

// Dispatch on the storage type: fn(std::integral_constant<int, DT>{}).
template <class Fn>
inline bool with_dtype(int dt, Fn &&fn)
{
    switch (dt) {
    case SG_F32: fn(std::integral_constant<int, SG_F32>{}); return true;
    case SG_BF16: fn(std::integral_constant<int, SG_BF16>{}); return true;
    case SG_F16: fn(std::integral_constant<int, SG_F16>{}); return true;
    case SG_FX21: fn(std::integral_constant<int, SG_FX21>{}); return true;
    default: return false;
    }
}

template <class Fn>
inline bool with_layout(int layout, Fn &&fn)
{
    switch (layout) {
    case SG_LAYOUT_LINEAR: fn(std::integral_constant<int, SG_LAYOUT_LINEAR>{}); return true;
    case SG_LAYOUT_TILED4: fn(std::integral_constant<int, SG_LAYOUT_TILED4>{}); return true;
    case SG_LAYOUT_CELL8: fn(std::integral_constant<int, SG_LAYOUT_CELL8>{}); return true;
    default: return false;
    }
}

template <int DT>
__device__ __forceinline__ float3 decode_elem(typename Elem<DT>::T v);

template <>
__device__ __forceinline__ float3 decode_elem<SG_F32>(float4 v) { return make_float3(v.x, v.y, v.z); }

template <>
__device__ __forceinline__ float3 decode_elem<SG_BF16>(uint2 v)
{
    return make_float3(__uint_as_float(v.x << 16), __uint_as_float(v.x & 0xffff0000u), __uint_as_float(v.y << 16));
}

template <>
__device__ __forceinline__ float3 decode_elem<SG_F16>(uint2 v)
{
    __half2 h = *reinterpret_cast<__half2 *>(&v.x);
    float2 a = __half22float2(h);
    float z = __half2float(__ushort_as_half((unsigned short)(v.y & 0xffffu)));
    return make_float3(a.x, a.y, z);
}

// FX21: each component is q + 2^20 in 21 bits; OR-ing the exponent of 2^23
// over the low 23 bits gives the float 2^23 + q + 2^20 exactly, and one
// subtraction of 2^23 + 2^20 leaves q (no integer-to-float conversion).
constexpr unsigned FX21_MASK = 0x1FFFFFu;
constexpr unsigned FX21_FLAG = 0x400u;     // bit 42 of the sample = bit 10 of the high word
__device__ __forceinline__ float fx21_value(unsigned u) { return __int_as_float(0x4B000000u | u) - 9437184.0f; }

template <>
__device__ __forceinline__ float3 decode_elem<SG_FX21>(uint2 v)
{
    return make_float3(fx21_value(v.x & FX21_MASK), fx21_value(__funnelshift_r(v.x, v.y, 21) & FX21_MASK),
                       fx21_value(v.y >> 11));
}

// Non-finite flag of a stored sample (only FX21 has one; the float formats
// carry NaN in the value itself).
template <int DT>
__device__ __forceinline__ unsigned elem_flag(typename Elem<DT>::T v)
{
    if constexpr (DT == SG_FX21) return v.y & FX21_FLAG;
    else return 0u;
}

template <int DT>
__device__ __forceinline__ typename Elem<DT>::T load_elem(const typename Elem<DT>::T *p)
{
    return __ldg(p);
}

__device__ __forceinline__ float lerpf(float a, float b, float t) { return fmaf(t, b - a, a); }

// Two FP32 values in one 64-bit register pair, with the packed FP32
// arithmetic of sm_100 and later: one instruction does the operation on both
// halves, each rounded as the scalar instruction (round to nearest, no flush
// of subnormals), so packed and scalar code give the same bits.
typedef unsigned long long f32x2;

__device__ __forceinline__ f32x2 pk2(float lo, float hi)
{
    f32x2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ float2 upk2(f32x2 v)
{
    float2 r;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(v));
    return r;
}
__device__ __forceinline__ f32x2 add2(f32x2 a, f32x2 b)
{
    f32x2 r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f32x2 sub2(f32x2 a, f32x2 b)
{
    f32x2 r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f32x2 mul2(f32x2 a, f32x2 b)
{
    f32x2 r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f32x2 fma2(f32x2 a, f32x2 b, f32x2 c)
{
    f32x2 r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}
// lerpf on both halves
__device__ __forceinline__ f32x2 lerp2(f32x2 a, f32x2 b, f32x2 t) { return fma2(t, sub2(b, a), a); }

// Storage offset of a sample inside a brick (fits in 32 bits: checked when the
// field is created), separable per axis: off = ox(x) + oy(y) + oz(z).
template <int LAYOUT>
struct Offsets {
    __device__ __forceinline__ static int ox(int x, const DevField &F)
    {
        if (LAYOUT == SG_LAYOUT_LINEAR) return x;
        return (x >> 2) * 64 + (x & 3);
    }
    __device__ __forceinline__ static int oy(int y, const DevField &F)
    {
        if (LAYOUT == SG_LAYOUT_LINEAR) return y * F.S[0];
        return (y >> 2) * F.T[0] * 64 + (y & 3) * 4;
    }
    __device__ __forceinline__ static int oz(int z, const DevField &F)
    {
        if (LAYOUT == SG_LAYOUT_LINEAR) return z * F.S[0] * F.S[1];
        return (z >> 2) * F.T[0] * F.T[1] * 64 + (z & 3) * 16;
    }
};

inline __host__ __device__ long long storage_index(int layout, int x, int y, int z, const DevField &F)
{
    if (layout == SG_LAYOUT_LINEAR) return ((long long)z * F.S[1] + y) * F.S[0] + x;
    if (layout == SG_LAYOUT_CELL8) {
        // the copy of sample (x,y,z) held by the cell whose lower corner it is
        // (the last cell for the upper layer); 8-byte samples only (FP32
        // records split the components: cell8_f32_index)
        const int cx = x < F.C[0] ? x : F.C[0] - 1, cy = y < F.C[1] ? y : F.C[1] - 1, cz = z < F.C[2] ? z : F.C[2] - 1;
        const int corner = (x - cx) | ((y - cy) << 1) | ((z - cz) << 2);
        return (((long long)cz * F.C[1] + cy) * F.C[0] + cx) * 8 + corner;
    }
    return (((long long)(z >> 2) * F.T[1] + (y >> 2)) * F.T[0] + (x >> 2)) * 64 + ((z & 3) * 4 + (y & 3)) * 4 + (x & 3);
}

__device__ __forceinline__ float3 lerp8(const float3 &c000, const float3 &c100, const float3 &c010, const float3 &c110,
                                        const float3 &c001, const float3 &c101, const float3 &c011, const float3 &c111,
                                        float fx, float fy, float fz)
{
    // x and y components as packed pairs, z alone: the same operations per
    // component as three scalar lerp trees
    const f32x2 tx = pk2(fx, fx), ty = pk2(fy, fy), tz = pk2(fz, fz);
    auto xy = [](const float3 &c) { return pk2(c.x, c.y); };
    const f32x2 rxy = lerp2(lerp2(lerp2(xy(c000), xy(c100), tx), lerp2(xy(c010), xy(c110), tx), ty),
                            lerp2(lerp2(xy(c001), xy(c101), tx), lerp2(xy(c011), xy(c111), tx), ty), tz);
    const float2 v = upk2(rxy);
    float3 r;
    r.x = v.x;
    r.y = v.y;
    r.z = lerpf(lerpf(lerpf(c000.z, c100.z, fx), lerpf(c010.z, c110.z, fx), fy),
                lerpf(lerpf(c001.z, c101.z, fx), lerpf(c011.z, c111.z, fx), fy), fz);
    return r;
}

// Not finite in any component (NaN or inf).  The sum of magnitudes is finite
// exactly when every component is finite, for |v| well below FLT_MAX.
__device__ __forceinline__ bool bad3(float3 v) { return !(fabsf(v.x) + fabsf(v.y) + fabsf(v.z) < INFINITY); }

// One 32-byte load through the read-only path (sm_100 and later): two
// 16-byte halves.  p must be 32-byte aligned.
__device__ __forceinline__ void ld_nc32(const void *p, uint4 &a, uint4 &b)
{
    asm("ld.global.nc.v8.u32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
        : "=r"(a.x), "=r"(a.y), "=r"(a.z), "=r"(a.w), "=r"(b.x), "=r"(b.y), "=r"(b.z), "=r"(b.w)
        : "l"(p));
}

// Asynchronous copies into shared memory and their completion on an
// mbarrier (sm_80 and later).  Addresses are shared-window byte offsets.
__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

// Non-blocking: has the phase of the given parity completed?
__device__ __forceinline__ bool mbar_done(uint32_t bar, unsigned parity)
{
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0u;
}

// One bulk copy by the TMA engine of `bytes` from global to shared memory,
// completing on the barrier: this thread's arrival on the barrier also adds
// `bytes` to the transaction count of the phase, which the copy counts down
// as it lands.  dst and src 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_copy_arrive(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}

// Makes mbarrier initialisation visible to the TMA engine (the async proxy).
__device__ __forceinline__ void mbar_init_fence()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// A cell record (CELL8 layout) as 16-byte chunks.  8-byte samples: 4 chunks,
// chunk j holding corners 2j and 2j+1 (corner k = (x, y, z) = (k & 1,
// k >> 1 & 1, k >> 2) from the cell's lower corner).  FP32: 6 chunks, one
// component after the other (x, y, z), each as two chunks: the four corners
// with x = 0, then the four with x = 1, each chunk in the order (y, z) =
// (0,0), (0,1), (1,0), (1,1).  That order puts the two z corners of one
// (x, y) edge side by side, so the x and y lerps run on packed pairs.
template <int DT>
struct Record {
    static constexpr int chunks = (DT == SG_F32) ? 6 : 4;
    uint4 r[chunks];
};

// Elements (Elem<DT>::T) from one record to the next.
template <int DT>
__host__ __device__ constexpr int record_elems() { return DT == SG_F32 ? 6 : 8; }

// Float index of component a of corner (dx, dy, dz) within an FP32 record.
inline __host__ __device__ int f32_record_index(int a, int dx, int dy, int dz)
{
    return a * 8 + dx * 4 + dy * 2 + dz;
}

// Float index of component a of sample (x, y, z) in an FP32 CELL8 brick: the
// copy held by the cell whose lower corner it is (the last cell for the upper
// layer), as storage_index.
inline __host__ __device__ long long cell8_f32_index(int x, int y, int z, int a, const DevField &F)
{
    const int cx = x < F.C[0] ? x : F.C[0] - 1, cy = y < F.C[1] ? y : F.C[1] - 1, cz = z < F.C[2] ? z : F.C[2] - 1;
    return (((long long)cz * F.C[1] + cy) * F.C[0] + cx) * 24 + f32_record_index(a, x - cx, y - cy, z - cz);
}

// Reads one record: 32-byte loads (records are 64-byte aligned).
template <int DT>
__device__ __forceinline__ void load_record(const typename Elem<DT>::T *__restrict__ rec, Record<DT> &R)
{
    const uint4 *p = reinterpret_cast<const uint4 *>(rec);
#pragma unroll
    for (int k = 0; k < Record<DT>::chunks; k += 2) ld_nc32(p + k, R.r[k], R.r[k + 1]);
}

// Trilinear interpolation of the eight corners of a record.  bad reports a
// sample that is not finite: for FX21 from the stored flags of the eight
// corners (the interpolated value itself stays finite), for the float formats
// from the interpolated value.
template <int DT>
__device__ __forceinline__ float3 interp_record(const Record<DT> &R, float fx, float fy, float fz, bool &bad)
{
    if constexpr (DT == SG_FX21) {
        // x pairs interpolate the biased floats 2^23 + u directly: their
        // difference is exact, and the bias leaves with the lower corner
        // (the same value as subtracting it from both corners first)
        const uint4 a = R.r[0], b = R.r[1], c = R.r[2], d = R.r[3];
        const float C = 9437184.0f;
        auto raw = [](unsigned lo, unsigned hi) {
            return make_float3(__int_as_float(0x4B000000u | (lo & FX21_MASK)),
                               __int_as_float(0x4B000000u | (__funnelshift_r(lo, hi, 21) & FX21_MASK)),
                               __int_as_float(0x4B000000u | (hi >> 11)));
        };
        // x and y components as packed pairs, z alone
        const f32x2 tx = pk2(fx, fx), ty = pk2(fy, fy), tz = pk2(fz, fz), C2 = pk2(C, C);
        struct X {
            f32x2 xy;
            float z;
        };
        auto xl = [&](float3 p, float3 q) {
            const f32x2 pxy = pk2(p.x, p.y);
            return X{fma2(tx, sub2(pk2(q.x, q.y), pxy), sub2(pxy, C2)), fmaf(fx, q.z - p.z, p.z - C)};
        };
        const X x00 = xl(raw(a.x, a.y), raw(a.z, a.w));   // (y0, z0)
        const X x10 = xl(raw(b.x, b.y), raw(b.z, b.w));   // (y1, z0)
        const X x01 = xl(raw(c.x, c.y), raw(c.z, c.w));   // (y0, z1)
        const X x11 = xl(raw(d.x, d.y), raw(d.z, d.w));   // (y1, z1)
        const float2 vxy = upk2(lerp2(lerp2(x00.xy, x10.xy, ty), lerp2(x01.xy, x11.xy, ty), tz));
        float3 v;
        v.x = vxy.x;
        v.y = vxy.y;
        v.z = lerpf(lerpf(x00.z, x10.z, fy), lerpf(x01.z, x11.z, fy), fz);
        bad = ((a.y | a.w | b.y | b.w | c.y | c.w | d.y | d.w) & FX21_FLAG) != 0u;
        return v;
    } else if constexpr (DT == SG_F32) {
        // per component: x lerps of the (z0, z1) pairs at y0 and at y1, one y
        // lerp of the two results, the z lerp of its halves; the same
        // operations as lerp8
        const f32x2 tx = pk2(fx, fx), ty = pk2(fy, fy);
        auto comp = [&](uint4 lo, uint4 hi) {
            const f32x2 y0 = lerp2(pk2(__uint_as_float(lo.x), __uint_as_float(lo.y)),
                                   pk2(__uint_as_float(hi.x), __uint_as_float(hi.y)), tx);
            const f32x2 y1 = lerp2(pk2(__uint_as_float(lo.z), __uint_as_float(lo.w)),
                                   pk2(__uint_as_float(hi.z), __uint_as_float(hi.w)), tx);
            const float2 z = upk2(lerp2(y0, y1, ty));
            return lerpf(z.x, z.y, fz);
        };
        const float3 v = make_float3(comp(R.r[0], R.r[1]), comp(R.r[2], R.r[3]), comp(R.r[4], R.r[5]));
        bad = bad3(v);
        return v;
    } else {
        const uint4 a = R.r[0], b = R.r[1], c = R.r[2], d = R.r[3];
        const float3 v =
            lerp8(decode_elem<DT>(make_uint2(a.x, a.y)), decode_elem<DT>(make_uint2(a.z, a.w)),
                  decode_elem<DT>(make_uint2(b.x, b.y)), decode_elem<DT>(make_uint2(b.z, b.w)),
                  decode_elem<DT>(make_uint2(c.x, c.y)), decode_elem<DT>(make_uint2(c.z, c.w)),
                  decode_elem<DT>(make_uint2(d.x, d.y)), decode_elem<DT>(make_uint2(d.z, d.w)), fx, fy, fz);
        bad = bad3(v);
        return v;
    }
}

template <int DT>
__device__ __forceinline__ float3 trilerp_record(const typename Elem<DT>::T *__restrict__ rec, float fx, float fy,
                                                 float fz, bool &bad)
{
    Record<DT> R;
    load_record<DT>(rec, R);
    return interp_record<DT>(R, fx, fy, fz, bad);
}

// Trilinear interpolation inside one brick: (sx, sy, sz) is the storage index
// of the lower corner (for CELL8: the cell index), (fx, fy, fz) the fractions.
// Returns the value before the brick scale (multiply by it for world units);
// bad as for trilerp_record.
template <int DT, int LAYOUT>
__device__ __forceinline__ float3 trilerp(const typename Elem<DT>::T *__restrict__ brick, const DevField &F,
                                          int sx, int sy, int sz, float fx, float fy, float fz, bool &bad)
{
    if constexpr (LAYOUT == SG_LAYOUT_CELL8) {
        const int cell = (sz * F.C[1] + sy) * F.C[0] + sx;
        return trilerp_record<DT>(brick + (long long)cell * record_elems<DT>(), fx, fy, fz, bad);
    } else {
        using O = Offsets<LAYOUT>;
        const int x0 = O::ox(sx, F), x1 = O::ox(sx + 1, F);
        const int y0 = O::oy(sy, F), y1 = O::oy(sy + 1, F);
        const int z0 = O::oz(sz, F), z1 = O::oz(sz + 1, F);
        const auto e000 = load_elem<DT>(brick + (z0 + y0 + x0));
        const auto e100 = load_elem<DT>(brick + (z0 + y0 + x1));
        const auto e010 = load_elem<DT>(brick + (z0 + y1 + x0));
        const auto e110 = load_elem<DT>(brick + (z0 + y1 + x1));
        const auto e001 = load_elem<DT>(brick + (z1 + y0 + x0));
        const auto e101 = load_elem<DT>(brick + (z1 + y0 + x1));
        const auto e011 = load_elem<DT>(brick + (z1 + y1 + x0));
        const auto e111 = load_elem<DT>(brick + (z1 + y1 + x1));
        const float3 v =
            lerp8(decode_elem<DT>(e000), decode_elem<DT>(e100), decode_elem<DT>(e010), decode_elem<DT>(e110),
                  decode_elem<DT>(e001), decode_elem<DT>(e101), decode_elem<DT>(e011), decode_elem<DT>(e111), fx, fy,
                  fz);
        if constexpr (DT == SG_FX21) {
            bad = (elem_flag<DT>(e000) | elem_flag<DT>(e100) | elem_flag<DT>(e010) | elem_flag<DT>(e110) |
                   elem_flag<DT>(e001) | elem_flag<DT>(e101) | elem_flag<DT>(e011) | elem_flag<DT>(e111)) != 0u;
        } else {
            bad = bad3(v);
        }
        return v;
    }
}

// The same with a non-finite sample reported as a NaN value (every format).
template <int DT, int LAYOUT>
__device__ __forceinline__ float3 trilerp(const typename Elem<DT>::T *__restrict__ brick, const DevField &F,
                                          int sx, int sy, int sz, float fx, float fy, float fz)
{
    bool bad;
    float3 v = trilerp<DT, LAYOUT>(brick, F, sx, sy, sz, fx, fy, fz, bad);
    if (DT == SG_FX21 && bad) v = make_float3(NAN, NAN, NAN);
    return v;
}


// Stage point relative to a particle's cell: q = frac + dk gives the cell
// offset floor(q) and the new fraction q - floor(q) (exact for |q| < 2^23);
// a fraction that rounds up to 1 moves to the next cell.
__device__ __forceinline__ void locate(float frac, float dk, int cell, int &cell_out, float &frac_out)
{
    const float q = frac + dk;
    const float d = floorf(q);
    float fr = q - d;
    int di = (int)d;
    if (fr >= 1.0f) {
        fr = 0.0f;
        di += 1;
    }
    cell_out = cell + di;
    frac_out = fr;
}

// Inside the closed domain [0, N-1] along one axis.
__device__ __forceinline__ bool in_axis(int cell, float frac, int nm1)
{
    return cell >= 0 && (cell < nm1 || (cell == nm1 && frac == 0.0f));
}

// Distance outside the domain along one axis (0 if inside).
__device__ __forceinline__ float out_axis(int cell, float frac, int nm1)
{
    if (cell < 0) return (float)(-cell) - frac;
    if (cell > nm1 || (cell == nm1 && frac > 0.0f)) return (float)(cell - nm1) + frac;
    return 0.0f;
}

// ------------------------------------------------------------------ host-side launchers (per file)

sg_status launch_brick_store(sg_field *f, int slot, const float *src, int src_mode, int brick_index,
                             cudaStream_t s);
sg_status launch_max_speed(sg_field *f, int slot, cudaStream_t s);

int pointer_kind(const void *p);   // 0 = device/managed, 1 = page-locked host, 2 = pageable host, -1 error
enum { PTR_DEVICE = 0, PTR_PINNED = 1, PTR_PAGEABLE = 2 };

}  // namespace sg
