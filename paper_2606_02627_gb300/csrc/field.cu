// Brick field store: cutting a global field (or one application brick) into
// bricks with a one-cell ghost shell, per-brick scale and BF16/FP16 encoding,
// and reductions over the stored samples.
//
// The field is the paper's structured VecField whose data is distributed over
// a uniform grid of macrocells, each with a halo (Sec. 3.1.1, Sec. 3.3).  On
// one GPU every macrocell is a brick of the same device buffer; the halo is
// the one-cell ghost shell that lets a particle owned by the brick finish a
// step of at most one cell without touching another brick.
#include <algorithm>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include "common.cuh"

namespace sg {

DevField field_view(const sg_field *f, int slot)
{
    DevField v = f->geom;
    v.data = f->slot_data[slot];
    v.scales = f->slot_scales[slot];
    return v;
}

// ------------------------------------------------------------------ kernels

// src_mode 0: src is the global AoS array [dims2][dims1][dims0][3].
// src_mode 1: src is one brick's own (n+3)^3 AoS samples (ghost shell included).
struct StoreArgs {
    const float *src;
    int src_mode;
    int brick0;               // first brick index handled by blockIdx.y == 0
    DevField F;
    char *data;
    float *scales;
    unsigned *maxbits;
    long long brick_bytes;
};

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

__device__ __forceinline__ const float *src_sample(const StoreArgs &A, int b, int sx, int sy, int sz)
{
    const DevField &F = A.F;
    if (A.src_mode == 1) return A.src + 3 * (((long long)sz * F.S[1] + sy) * F.S[0] + sx);
    const int bx = b % F.B[0], by = (b / F.B[0]) % F.B[1], bz = b / (F.B[0] * F.B[1]);
    const int gx = clampi(bx * F.n[0] - 1 + sx, 0, F.nm1[0]);
    const int gy = clampi(by * F.n[1] - 1 + sy, 0, F.nm1[1]);
    const int gz = clampi(bz * F.n[2] - 1 + sz, 0, F.nm1[2]);
    return A.src + 3 * (((long long)gz * F.dims[1] + gy) * F.dims[0] + gx);
}

// Largest finite |component| over each brick's stored samples (grid.y = brick).
__global__ void brick_maxabs_kernel(StoreArgs A)
{
    const DevField &F = A.F;
    const int b = A.brick0 + blockIdx.y;
    const long long total = (long long)F.S[0] * F.S[1] * F.S[2];
    float m = 0.0f;
    for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < total;
         r += (long long)gridDim.x * blockDim.x) {
        const int sx = (int)(r % F.S[0]);
        const int sy = (int)((r / F.S[0]) % F.S[1]);
        const int sz = (int)(r / ((long long)F.S[0] * F.S[1]));
        const float *s = src_sample(A, b, sx, sy, sz);
        for (int c = 0; c < 3; ++c) {
            const float a = fabsf(s[c]);
            if (a < INFINITY && a > m) m = a;
        }
    }
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(SG_FULL_MASK, m, o));
    if ((threadIdx.x & 31) == 0 && m > 0.0f) atomicMax(A.maxbits + b, __float_as_uint(m));
}

// Smallest power of two >= m; 1 when there is no positive finite magnitude.
__device__ __forceinline__ float pow2_ceil(float m)
{
    if (!(m > 0.0f) || !(m < INFINITY)) return 1.0f;
    int e;
    const float fr = frexpf(m, &e);
    return fr == 0.5f ? m : ldexpf(1.0f, e);
}

// mult: 1 for the float formats; 2^-20 for FX21, whose stored scale is the
// quantum s_b * 2^-20 (a power of two as well).
__global__ void brick_scale_kernel(unsigned *maxbits, float *scales, int b0, int nb, float mult)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nb) return;
    scales[b0 + i] = pow2_ceil(__uint_as_float(maxbits[b0 + i])) * mult;
    maxbits[b0 + i] = 0u;   // ready for the next store
}

// Encoding of one sample (x, y, z) with the brick's scale (FP32: as given).
template <int DT>
__device__ __forceinline__ typename Elem<DT>::T encode_elem(float x, float y, float z, float scale);

template <>
__device__ __forceinline__ float4 encode_elem<SG_F32>(float x, float y, float z, float)
{
    return make_float4(x, y, z, 0.0f);
}

// code = round-to-nearest-even(v / s) in the storage format; the quotient is an
// IEEE single-precision division; a non-finite sample stores NaN.
__device__ __forceinline__ float scaled(float v, float s) { return (fabsf(v) < INFINITY) ? v / s : __int_as_float(0x7fc00000); }

template <>
__device__ __forceinline__ uint2 encode_elem<SG_BF16>(float x, float y, float z, float s)
{
    const unsigned short bx = __bfloat16_as_ushort(__float2bfloat16_rn(scaled(x, s)));
    const unsigned short by = __bfloat16_as_ushort(__float2bfloat16_rn(scaled(y, s)));
    const unsigned short bz = __bfloat16_as_ushort(__float2bfloat16_rn(scaled(z, s)));
    return make_uint2((unsigned)bx | ((unsigned)by << 16), (unsigned)bz);
}

template <>
__device__ __forceinline__ uint2 encode_elem<SG_F16>(float x, float y, float z, float s)
{
    const unsigned short hx = __half_as_ushort(__float2half_rn(scaled(x, s)));
    const unsigned short hy = __half_as_ushort(__float2half_rn(scaled(y, s)));
    const unsigned short hz = __half_as_ushort(__float2half_rn(scaled(z, s)));
    return make_uint2((unsigned)hx | ((unsigned)hy << 16), (unsigned)hz);
}

// FX21: q = round-to-nearest-even(v / quantum), clamped to +-(2^20 - 1), stored
// as q + 2^20; the quotient by a power of two is exact.  A non-finite component
// sets the sample's flag (and stores zero).
__device__ __forceinline__ unsigned fx21_code(float v, float quantum, unsigned &flag)
{
    if (!(fabsf(v) < INFINITY)) {
        flag = FX21_FLAG;
        return 1u << 20;
    }
    int q = __float2int_rn(v / quantum);
    q = max(-(1 << 20) + 1, min((1 << 20) - 1, q));
    return (unsigned)(q + (1 << 20));
}

template <>
__device__ __forceinline__ uint2 encode_elem<SG_FX21>(float x, float y, float z, float quantum)
{
    unsigned flag = 0;
    const unsigned ux = fx21_code(x, quantum, flag);
    const unsigned uy = fx21_code(y, quantum, flag);
    const unsigned uz = fx21_code(z, quantum, flag);
    return make_uint2(ux | (uy << 21), (uy >> 11) | flag | (uz << 11));
}

// Source sample of stored coordinate (sx, sy, sz) of brick (bx, by, bz).
__device__ __forceinline__ const float *src_at(const StoreArgs &A, int bx, int by, int bz, int sx, int sy, int sz)
{
    const DevField &F = A.F;
    if (A.src_mode == 1) return A.src + 3 * (((long long)sz * F.S[1] + sy) * F.S[0] + sx);
    const int gx = clampi(bx * F.n[0] - 1 + sx, 0, F.nm1[0]);
    const int gy = clampi(by * F.n[1] - 1 + sy, 0, F.nm1[1]);
    const int gz = clampi(bz * F.n[2] - 1 + sz, 0, F.nm1[2]);
    return A.src + 3 * (((long long)gz * F.dims[1] + gy) * F.dims[0] + gx);
}

// Sample layouts (LINEAR, TILED4): one thread per stored sample.
template <int DT>
__global__ void brick_store_kernel(StoreArgs A, int layout)
{
    using T = typename Elem<DT>::T;
    const DevField &F = A.F;
    const int b = A.brick0 + blockIdx.y;
    const int bx = b % F.B[0], by = (b / F.B[0]) % F.B[1], bz = b / (F.B[0] * F.B[1]);
    T *brick = reinterpret_cast<T *>(A.data + (long long)b * A.brick_bytes);
    const float s = (DT == SG_F32) ? 1.0f : A.scales[b];
    const int total = F.S[0] * F.S[1] * F.S[2];
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < total; r += gridDim.x * blockDim.x) {
        const int sx = r % F.S[0];
        const int t = r / F.S[0];
        const int sy = t % F.S[1];
        const int sz = t / F.S[1];
        const float *src = src_at(A, bx, by, bz, sx, sy, sz);
        brick[storage_index(layout, sx, sy, sz, F)] = encode_elem<DT>(src[0], src[1], src[2], s);
    }
}

// CELL8: one block per row of cell records (fixed y and z, all x), one thread
// per 16-byte chunk of a record (one FP32 corner, or an x pair of 8-byte
// corners), so that the lanes of a warp write whole records side by side
// (coalesced 512-byte stores) and the row's index arithmetic is done once.
// Corner k of a record is (x, y, z) = (k & 1, k >> 1 & 1, k >> 2) from the
// cell's lower corner.
template <int DT>
__global__ void brick_store_cell8_kernel(StoreArgs A)
{
    using T = typename Elem<DT>::T;
    constexpr int CPR = Record<DT>::chunks;         // chunks per record
    constexpr int KPC = 2;                          // corners per chunk (8-byte samples)
    const DevField &F = A.F;
    const int b = A.brick0 + blockIdx.y;
    const int bx = b % F.B[0], by = (b / F.B[0]) % F.B[1], bz = b / (F.B[0] * F.B[1]);
    uint4 *brick = reinterpret_cast<uint4 *>(A.data + (long long)b * A.brick_bytes);
    const float s = (DT == SG_F32) ? 1.0f : A.scales[b];
    const int rows = F.C[1] * F.C[2];
    const int row_chunks = F.C[0] * CPR;
    const int x0 = bx * F.n[0] - 1;
    for (int r = blockIdx.x; r < rows; r += gridDim.x) {
        const int cy = r % F.C[1], cz = r / F.C[1];
        uint4 *dst = brick + (long long)r * row_chunks;
        for (int j = threadIdx.x; j < row_chunks; j += blockDim.x) {
            const int cx = j / CPR, jc = j % CPR;
            // the source sample of corner (dx, dy, dz)
            auto corner = [&](int dx, int dy, int dz) -> const float * {
                if (A.src_mode == 1)
                    return A.src + 3 * (((long long)(cz + dz) * F.S[1] + cy + dy) * F.S[0] + cx + dx);
                const int gx = clampi(x0 + cx + dx, 0, F.nm1[0]);
                const int gy = clampi(by * F.n[1] - 1 + cy + dy, 0, F.nm1[1]);
                const int gz = clampi(bz * F.n[2] - 1 + cz + dz, 0, F.nm1[2]);
                return A.src + 3 * (((long long)gz * F.dims[1] + gy) * F.dims[0] + gx);
            };
            uint4 out;
            if constexpr (DT == SG_F32) {
                // component a = jc / 2 of the four corners with x = jc % 2
                const int a = jc >> 1, dx = jc & 1;
                out = make_uint4(__float_as_uint(corner(dx, 0, 0)[a]), __float_as_uint(corner(dx, 0, 1)[a]),
                                 __float_as_uint(corner(dx, 1, 0)[a]), __float_as_uint(corner(dx, 1, 1)[a]));
            } else {
                T e[KPC];
#pragma unroll
                for (int m = 0; m < KPC; ++m) {
                    const int k = jc * KPC + m;
                    const float *src = corner(k & 1, (k >> 1) & 1, k >> 2);
                    e[m] = encode_elem<DT>(src[0], src[1], src[2], s);
                }
                out = make_uint4(e[0].x, e[0].y, e[1].x, e[1].y);
            }
            dst[j] = out;
        }
    }
}

// CELL8 with the source rows staged: a block builds a strip of STRIP rows of
// cell records (fixed z, y from y0, all x) at a time.  It first copies the
// sample rows those records read ((y0 .. y0 + STRIP) x (z, z + 1), S0
// samples each, ghost shell included) into shared memory with coalesced
// loads, then builds the records from there, one thread per 16-byte chunk,
// with coalesced writes.  The same records as brick_store_cell8_kernel, bit
// for bit.
constexpr int STORE_STRIP = 6;

template <int DT>
__global__ void brick_store_cell8_staged_kernel(StoreArgs A)
{
    using T = typename Elem<DT>::T;
    extern __shared__ float rowbuf[];               // [dz][dy 0..STRIP][3 * S0]
    constexpr int CPR = Record<DT>::chunks;
    const DevField &F = A.F;
    const int b = A.brick0 + blockIdx.y;
    const int bx = b % F.B[0], by = (b / F.B[0]) % F.B[1], bz = b / (F.B[0] * F.B[1]);
    uint4 *brick = reinterpret_cast<uint4 *>(A.data + (long long)b * A.brick_bytes);
    const float s = (DT == SG_F32) ? 1.0f : A.scales[b];
    const int strips = (F.C[1] + STORE_STRIP - 1) / STORE_STRIP;
    const int units = strips * F.C[2];
    const int rowf = 3 * F.S[0];
    const int row_chunks = F.C[0] * CPR;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
    for (int u = blockIdx.x; u < units; u += gridDim.x) {
        const int cz = u / strips, y0 = (u - cz * strips) * STORE_STRIP;
        const int ny = min(STORE_STRIP, F.C[1] - y0);    // record rows in this strip
        const int nrows = ny + 1;                        // sample rows per z layer
        __syncthreads();                                 // the previous strip's records are built
        // sample row k = dy + nrows dz: one warp per row, the lanes along x
        for (int k = warp; k < 2 * nrows; k += nwarps) {
            const int dz = k >= nrows ? 1 : 0;
            const int sy = y0 + k - dz * nrows, sz = cz + dz;
            const float *row;
            int x0 = 0, xhi = F.S[0] - 1;
            if (A.src_mode == 1) {
                row = A.src + 3ll * ((long long)sz * F.S[1] + sy) * F.S[0];
            } else {
                const int gy = clampi(by * F.n[1] - 1 + sy, 0, F.nm1[1]);
                const int gz = clampi(bz * F.n[2] - 1 + sz, 0, F.nm1[2]);
                row = A.src + 3ll * ((long long)gz * F.dims[1] + gy) * F.dims[0];
                x0 = bx * F.n[0] - 1;
                xhi = F.nm1[0];
            }
            float *d = rowbuf + k * rowf;
            for (int sx = lane; sx < F.S[0]; sx += 32) {
                const float *p = row + 3 * clampi(x0 + sx, 0, xhi);
                d[3 * sx] = __ldg(p);
                d[3 * sx + 1] = __ldg(p + 1);
                d[3 * sx + 2] = __ldg(p + 2);
            }
        }
        __syncthreads();
        uint4 *dst = brick + ((long long)cz * F.C[1] + y0) * row_chunks;   // ny consecutive record rows
        int ry = 0, jj = threadIdx.x;                    // record row and chunk within it of chunk j
        while (jj >= row_chunks) {
            jj -= row_chunks;
            ++ry;
        }
        for (int j = threadIdx.x; j < ny * row_chunks; j += blockDim.x) {
            const int cx = jj / CPR, jc = jj - cx * CPR;
            auto smp = [&](int dx, int dy, int dz) {
                return rowbuf + (dz * nrows + ry + dy) * rowf + 3 * (cx + dx);
            };
            uint4 out;
            if constexpr (DT == SG_F32) {
                // component a = jc / 2 of the four corners with x = jc % 2
                const int a = jc >> 1, dx = jc & 1;
                out = make_uint4(__float_as_uint(smp(dx, 0, 0)[a]), __float_as_uint(smp(dx, 0, 1)[a]),
                                 __float_as_uint(smp(dx, 1, 0)[a]), __float_as_uint(smp(dx, 1, 1)[a]));
            } else {
                // corners 2 jc and 2 jc + 1: (0, dy, dz) and (1, dy, dz)
                const int dy = jc & 1, dz = jc >> 1;
                const float *p0 = smp(0, dy, dz), *p1 = smp(1, dy, dz);
                const T e0 = encode_elem<DT>(p0[0], p0[1], p0[2], s);
                const T e1 = encode_elem<DT>(p1[0], p1[1], p1[2], s);
                out = make_uint4(e0.x, e0.y, e1.x, e1.y);
            }
            dst[j] = out;
            jj += blockDim.x;
            while (jj >= row_chunks) {
                jj -= row_chunks;
                ++ry;
            }
        }
    }
}

// Plain copy for the global float3 layout.
__global__ void global_copy_kernel(const float *__restrict__ src, float *__restrict__ dst, long long n)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        dst[i] = src[i];
}

template <int DT>
__global__ void max_speed_kernel(DevField F, long long brick_bytes, int layout, float isx, float isy, float isz,
                                 unsigned *out)
{
    using T = typename Elem<DT>::T;
    const int b = blockIdx.y;
    const long long total = (long long)F.S[0] * F.S[1] * F.S[2];
    const T *brick = reinterpret_cast<const T *>(F.data + (long long)b * brick_bytes);
    const float s = F.scales[b];
    float m = 0.0f;
    for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < total;
         r += (long long)gridDim.x * blockDim.x) {
        const int sx = (int)(r % F.S[0]);
        const int sy = (int)((r / F.S[0]) % F.S[1]);
        const int sz = (int)(r / ((long long)F.S[0] * F.S[1]));
        float3 v;
        if (DT == SG_F32 && layout == SG_LAYOUT_CELL8) {
            const float *bf = reinterpret_cast<const float *>(brick);
            v = make_float3(bf[cell8_f32_index(sx, sy, sz, 0, F)], bf[cell8_f32_index(sx, sy, sz, 1, F)],
                            bf[cell8_f32_index(sx, sy, sz, 2, F)]);
        } else {
            v = decode_elem<DT>(brick[storage_index(layout, sx, sy, sz, F)]);
        }
        const float x = v.x * s * isx, y = v.y * s * isy, z = v.z * s * isz;
        const float sp = sqrtf(x * x + y * y + z * z);
        if (sp < INFINITY && sp > m) m = sp;
    }
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(SG_FULL_MASK, m, o));
    if ((threadIdx.x & 31) == 0 && m > 0.0f) atomicMax(out, __float_as_uint(m));
}

__global__ void max_speed_global_kernel(const float *F, long long n, float isx, float isy, float isz, unsigned *out)
{
    float m = 0.0f;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float x = F[3 * i] * isx, y = F[3 * i + 1] * isy, z = F[3 * i + 2] * isz;
        const float sp = sqrtf(x * x + y * y + z * z);
        if (sp < INFINITY && sp > m) m = sp;
    }
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(SG_FULL_MASK, m, o));
    if ((threadIdx.x & 31) == 0 && m > 0.0f) atomicMax(out, __float_as_uint(m));
}

// ------------------------------------------------------------------ launchers

static int grid_x_for(long long total, int block, int nb, int sm_count)
{
    long long want = (total + block - 1) / block;
    long long cap = (long long)sm_count * 8 / (nb > 0 ? nb : 1) + 1;
    if (want > cap) want = cap;
    if (want < 1) want = 1;
    if (want > 65535) want = 65535;
    return (int)want;
}

sg_status launch_brick_store(sg_field *f, int slot, const float *src, int src_mode, int brick_index, cudaStream_t s)
{
    const sg_field_desc &d = f->desc;
    if (d.layout == SG_FIELD_GLOBAL) {
        const long long n = d.dims[0] * d.dims[1] * d.dims[2] * 3;
        global_copy_kernel<<<f->ctx->sm_count * 4, 256, 0, s>>>(src, reinterpret_cast<float *>(f->slot_data[slot]), n);
        SG_CUDA(cudaGetLastError());
        return SG_OK;
    }
    StoreArgs A;
    A.src = src;
    A.src_mode = src_mode;
    A.F = field_view(f, slot);
    A.data = f->slot_data[slot];
    A.scales = f->slot_scales[slot];
    A.maxbits = f->maxbits;
    A.brick_bytes = (long long)f->brick_bytes;
    const int b0 = src_mode == 1 ? brick_index : 0;
    const int nbr = src_mode == 1 ? 1 : f->nb;
    A.brick0 = b0;
    const long long total = d.layout == SG_LAYOUT_CELL8 ? (long long)A.F.C[0] * A.F.C[1] * A.F.C[2] * 4
                                                        : (long long)A.F.S[0] * A.F.S[1] * A.F.S[2];
    const int block = 256;
    dim3 grid(grid_x_for(total, block, nbr, f->ctx->sm_count), nbr);
    if (d.dtype != SG_F32) {
        brick_maxabs_kernel<<<grid, block, 0, s>>>(A);
        SG_CUDA(cudaGetLastError());
    }
    // FP32 bricks leave the max-abs words at zero, which gives a scale of 1
    brick_scale_kernel<<<(nbr + 255) / 256, 256, 0, s>>>(f->maxbits, A.scales, b0, nbr,
                                                         d.dtype == SG_FX21 ? 1.0f / 1048576.0f : 1.0f);
    SG_CUDA(cudaGetLastError());
    const int rows = A.F.C[1] * A.F.C[2];
    dim3 grid_rows((unsigned)std::min<long long>(rows, std::max(1, f->ctx->sm_count * 16 / nbr)), nbr);
    const int strip_units = (A.F.C[1] + STORE_STRIP - 1) / STORE_STRIP * A.F.C[2];
    dim3 grid_strips((unsigned)std::min<long long>(strip_units, std::max(1, f->ctx->sm_count * 8 / nbr)), nbr);
    const bool ok = with_dtype(d.dtype, [&](auto D) {
        const size_t staged = sizeof(float) * 3 * (size_t)A.F.S[0] * 2 * (STORE_STRIP + 1);   // sample rows of a strip
        if (d.layout == SG_LAYOUT_CELL8 && staged <= 48 * 1024)
            brick_store_cell8_staged_kernel<decltype(D)::value><<<grid_strips, block, staged, s>>>(A);
        else if (d.layout == SG_LAYOUT_CELL8)
            brick_store_cell8_kernel<decltype(D)::value><<<grid_rows, block, 0, s>>>(A);
        else brick_store_kernel<decltype(D)::value><<<grid, block, 0, s>>>(A, d.layout);
    });
    SG_CHECK(ok, SG_ERR_UNSUPPORTED, "unsupported dtype %d", d.dtype);
    SG_CUDA(cudaGetLastError());
    return SG_OK;
}

sg_status launch_max_speed(sg_field *f, int slot, cudaStream_t s)
{
    const sg_field_desc &d = f->desc;
    SG_CUDA(cudaMemsetAsync(f->speed_bits, 0, sizeof(unsigned), s));
    const float isx = (float)(1.0 / d.spacing[0]), isy = (float)(1.0 / d.spacing[1]), isz = (float)(1.0 / d.spacing[2]);
    if (d.layout == SG_FIELD_GLOBAL) {
        const long long n = d.dims[0] * d.dims[1] * d.dims[2];
        max_speed_global_kernel<<<f->ctx->sm_count * 4, 256, 0, s>>>(
            reinterpret_cast<const float *>(f->slot_data[slot]), n, isx, isy, isz, f->speed_bits);
        SG_CUDA(cudaGetLastError());
        return SG_OK;
    }
    DevField F = field_view(f, slot);
    const int block = 256;
    dim3 grid(grid_x_for((long long)F.S[0] * F.S[1] * F.S[2], block, f->nb, f->ctx->sm_count), f->nb);
    with_dtype(d.dtype, [&](auto D) {
        max_speed_kernel<decltype(D)::value><<<grid, block, 0, s>>>(F, (long long)f->brick_bytes, d.layout, isx, isy,
                                                                     isz, f->speed_bits);
    });
    SG_CUDA(cudaGetLastError());
    return SG_OK;
}

}  // namespace sg

// ------------------------------------------------------------------ C ABI: field

using namespace sg;

static sg_status field_layout(const sg_field_desc *d, sg_field *f, size_t *bytes_out, char *base)
{
    SG_CHECK(d != nullptr, SG_ERR_INVALID_ARG, "field desc is NULL");
    for (int a = 0; a < 3; ++a) {
        SG_CHECK(d->dims[a] >= 2 && d->dims[a] < (1ll << 30), SG_ERR_INVALID_ARG, "dims[%d] = %lld out of range", a,
                 (long long)d->dims[a]);
        SG_CHECK(d->spacing[a] > 0.0, SG_ERR_INVALID_ARG, "spacing[%d] must be > 0", a);
        SG_CHECK(d->bricks[a] >= 1, SG_ERR_INVALID_ARG, "bricks[%d] must be >= 1", a);
    }
    SG_CHECK(d->n_slots >= 1 && d->n_slots <= 64, SG_ERR_INVALID_ARG, "n_slots must be in [1, 64]");
    SG_CHECK(d->dtype == SG_F32 || d->dtype == SG_BF16 || d->dtype == SG_F16 || d->dtype == SG_FX21,
             SG_ERR_INVALID_ARG, "bad dtype %d", d->dtype);
    SG_CHECK(d->layout == SG_LAYOUT_LINEAR || d->layout == SG_LAYOUT_TILED4 || d->layout == SG_LAYOUT_CELL8 ||
                 d->layout == SG_FIELD_GLOBAL,
             SG_ERR_INVALID_ARG, "bad layout %d", d->layout);
    SG_CHECK(d->n_slots == 1 || d->slice_dt > 0.0, SG_ERR_INVALID_ARG, "slice_dt must be > 0 for unsteady fields");
    DevField g;
    memset(&g, 0, sizeof g);
    int nb = 1;
    size_t elem = 0, brick_bytes = 0;
    if (d->layout == SG_FIELD_GLOBAL) {
        SG_CHECK(d->bricks[0] == 1 && d->bricks[1] == 1 && d->bricks[2] == 1, SG_ERR_INVALID_ARG,
                 "the global float3 layout has one brick");
        SG_CHECK(d->dtype == SG_F32, SG_ERR_UNSUPPORTED, "the global float3 layout stores FP32");
        for (int a = 0; a < 3; ++a) {
            g.dims[a] = (int)d->dims[a];
            g.nm1[a] = g.dims[a] - 1;
            g.n[a] = g.nm1[a];
            g.B[a] = 1;
            g.S[a] = g.dims[a];
            g.T[a] = 0;
        }
        elem = 12;
        g.brick_elems = d->dims[0] * d->dims[1] * d->dims[2];
        brick_bytes = align_up((size_t)g.brick_elems * elem, 256);
    } else {
        SG_CHECK(d->ghost == 1, SG_ERR_UNSUPPORTED, "ghost must be 1 (got %d)", d->ghost);
        for (int a = 0; a < 3; ++a) {
            const long long cells = d->dims[a] - 1;
            const long long n = (cells + d->bricks[a] - 1) / d->bricks[a];
            SG_CHECK((long long)(d->bricks[a] - 1) * n < cells, SG_ERR_INVALID_ARG,
                     "bricks[%d] = %d leaves the last brick without a cell", a, d->bricks[a]);
            g.dims[a] = (int)d->dims[a];
            g.nm1[a] = g.dims[a] - 1;
            g.n[a] = (int)n;
            g.B[a] = d->bricks[a];
            g.S[a] = (int)n + 3;
            g.T[a] = (g.S[a] + 3) / 4;
            g.C[a] = (int)n + 2;
            nb *= d->bricks[a];
        }
        elem = d->dtype == SG_F32 ? 16 : 8;
        if (d->layout == SG_LAYOUT_LINEAR) g.brick_elems = (long long)g.S[0] * g.S[1] * g.S[2];
        else if (d->layout == SG_LAYOUT_TILED4) g.brick_elems = (long long)g.T[0] * g.T[1] * g.T[2] * 64;
        else g.brick_elems = (long long)g.C[0] * g.C[1] * g.C[2] * (d->dtype == SG_F32 ? record_elems<SG_F32>()
                                                                                      : record_elems<SG_F16>());
        SG_CHECK(g.brick_elems < (1ll << 31) - 1, SG_ERR_UNSUPPORTED, "a brick holds more than 2^31 samples");
        SG_CHECK(nb <= 65535, SG_ERR_UNSUPPORTED, "more than 65535 bricks");
        brick_bytes = align_up((size_t)g.brick_elems * elem, 256);
    }
    g.brick_stride = (long long)(brick_bytes / elem);
    for (int a = 0; a < 3; ++a) {
        g.origin[a] = (float)d->origin[a];
        g.spacing[a] = (float)d->spacing[a];
    }
    Carve c{base, 0, 0};
    char *slot_data[64];
    float *slot_scales[64];
    for (int s = 0; s < d->n_slots; ++s) {
        slot_data[s] = (char *)c.take(brick_bytes * nb);
        slot_scales[s] = (float *)c.take(sizeof(float) * nb);
    }
    unsigned *maxbits = (unsigned *)c.take(sizeof(unsigned) * nb);
    unsigned *speed = (unsigned *)c.take(sizeof(unsigned) * 4);
    float *staging = nullptr;
    if (d->n_slots > 1) staging = (float *)c.take(sizeof(float) * 3 * (size_t)(d->dims[0] * d->dims[1] * d->dims[2]));
    *bytes_out = c.off;
    if (f) {
        f->geom = g;
        f->nb = nb;
        f->elem_bytes = elem;
        f->brick_bytes = brick_bytes;
        for (int s = 0; s < d->n_slots; ++s) {
            f->slot_data[s] = slot_data[s];
            f->slot_scales[s] = slot_scales[s];
            f->slot_slice[s] = -1;
        }
        f->maxbits = maxbits;
        f->speed_bits = speed;
        f->staging = staging;
    }
    return SG_OK;
}

extern "C" sg_status sg_field_required_bytes(const sg_field_desc *desc, size_t *bytes)
{
    SG_CHECK(bytes != nullptr, SG_ERR_INVALID_ARG, "bytes is NULL");
    return field_layout(desc, nullptr, bytes, nullptr);
}

extern "C" sg_status sg_field_create(sg_context *ctx, const sg_field_desc *desc, void *storage, size_t bytes,
                                     sg_field **out)
{
    SG_CHECK(ctx && desc && out, SG_ERR_INVALID_ARG, "NULL argument");
    SG_CHECK(storage != nullptr, SG_ERR_INVALID_ARG, "storage is NULL");
    SG_CHECK(((uintptr_t)storage & 255) == 0, SG_ERR_INVALID_ARG, "storage must be 256-byte aligned");
    size_t need = 0;
    sg_status st = field_layout(desc, nullptr, &need, nullptr);
    if (st) return st;
    SG_CHECK(bytes >= need, SG_ERR_OOM, "field needs %zu bytes, got %zu", need, bytes);
    SG_CHECK(pointer_kind(storage) == PTR_DEVICE, SG_ERR_INVALID_ARG, "field storage must be device memory");
    SG_CUDA(cudaSetDevice(ctx->device));
    sg_field *f = new sg_field;
    memset(f, 0, sizeof *f);
    f->ctx = ctx;
    f->desc = *desc;
    f->storage = (char *)storage;
    f->bytes = bytes;
    field_layout(desc, f, &need, (char *)storage);
    for (int s = 0; s < desc->n_slots; ++s) {
        cudaError_t e = cudaEventCreateWithFlags(&f->slot_ready[s], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&f->slot_used[s], cudaEventDisableTiming);
        if (e != cudaSuccess) {
            for (int k = 0; k <= s; ++k) {
                if (f->slot_ready[k]) cudaEventDestroy(f->slot_ready[k]);
                if (f->slot_used[k]) cudaEventDestroy(f->slot_used[k]);
            }
            delete f;
            return cuda_error(e, "cudaEventCreateWithFlags");
        }
    }
    // scratch words start at zero; scales start at 1
    cudaError_t e = cudaMemset(f->maxbits, 0, sizeof(unsigned) * f->nb);
    if (e != cudaSuccess) {
        for (int k = 0; k < desc->n_slots; ++k) cudaEventDestroy(f->slot_ready[k]);
        delete f;
        return cuda_error(e, "cudaMemset");
    }
    *out = f;
    return SG_OK;
}

extern "C" sg_status sg_field_destroy(sg_field *f)
{
    if (!f) return SG_OK;
    for (int s = 0; s < f->desc.n_slots; ++s) {
        if (f->slot_ready[s]) cudaEventDestroy(f->slot_ready[s]);
        if (f->slot_used[s]) cudaEventDestroy(f->slot_used[s]);
    }
    delete f;
    return SG_OK;
}

extern "C" sg_status sg_field_brick_cells(const sg_field *f, int64_t n_out[3])
{
    SG_CHECK(f && n_out, SG_ERR_INVALID_ARG, "NULL argument");
    for (int a = 0; a < 3; ++a) n_out[a] = f->geom.n[a];
    return SG_OK;
}

static sg_status check_src(const void *p)
{
    const int k = pointer_kind(p);
    SG_CHECK(k == PTR_DEVICE || k == PTR_PINNED, SG_ERR_INVALID_ARG,
             "source must be device or page-locked host memory (kind %d)", k);
    return SG_OK;
}

extern "C" sg_status sg_field_set_global(sg_field *f, int32_t slot, const float *vec3, void *stream)
{
    SG_CHECK(f && vec3, SG_ERR_INVALID_ARG, "NULL argument");
    SG_CHECK(slot >= 0 && slot < f->desc.n_slots, SG_ERR_INVALID_ARG, "slot %d out of range", slot);
    sg_status st = check_src(vec3);
    if (st) return st;
    SG_CUDA(cudaSetDevice(f->ctx->device));
    st = launch_brick_store(f, slot, vec3, 0, 0, (cudaStream_t)stream);
    if (st) return st;
    f->slot_slice[slot] = slot;
    SG_CUDA(cudaEventRecord(f->slot_ready[slot], (cudaStream_t)stream));
    return SG_OK;
}

extern "C" sg_status sg_field_set_brick(sg_field *f, int32_t slot, int32_t bx, int32_t by, int32_t bz,
                                        const float *vec3_with_halo, void *stream)
{
    SG_CHECK(f && vec3_with_halo, SG_ERR_INVALID_ARG, "NULL argument");
    SG_CHECK(f->desc.layout != SG_FIELD_GLOBAL, SG_ERR_UNSUPPORTED, "the global layout has no bricks");
    SG_CHECK(slot >= 0 && slot < f->desc.n_slots, SG_ERR_INVALID_ARG, "slot %d out of range", slot);
    SG_CHECK(bx >= 0 && bx < f->geom.B[0] && by >= 0 && by < f->geom.B[1] && bz >= 0 && bz < f->geom.B[2],
             SG_ERR_INVALID_ARG, "brick (%d,%d,%d) out of range", bx, by, bz);
    sg_status st = check_src(vec3_with_halo);
    if (st) return st;
    SG_CUDA(cudaSetDevice(f->ctx->device));
    const int b = (bz * f->geom.B[1] + by) * f->geom.B[0] + bx;
    st = launch_brick_store(f, slot, vec3_with_halo, 1, b, (cudaStream_t)stream);
    if (st) return st;
    f->slot_slice[slot] = slot;
    SG_CUDA(cudaEventRecord(f->slot_ready[slot], (cudaStream_t)stream));
    return SG_OK;
}

extern "C" sg_status sg_field_stream_slice(sg_field *f, int32_t slice, const float *pinned_host, void *stream)
{
    SG_CHECK(f && pinned_host, SG_ERR_INVALID_ARG, "NULL argument");
    SG_CHECK(f->desc.n_slots > 1, SG_ERR_STATE, "streaming needs a field with n_slots > 1");
    SG_CHECK(slice >= 0, SG_ERR_INVALID_ARG, "negative slice");
    const int k = pointer_kind(pinned_host);
    SG_CHECK(k == PTR_PINNED, SG_ERR_INVALID_ARG, "slices stream from page-locked host memory (kind %d)", k);
    SG_CUDA(cudaSetDevice(f->ctx->device));
    cudaStream_t s = (cudaStream_t)stream;
    const int slot = slice % f->desc.n_slots;
    const size_t bytes = sizeof(float) * 3 * (size_t)(f->desc.dims[0] * f->desc.dims[1] * f->desc.dims[2]);
    SG_CUDA(cudaMemcpyAsync(f->staging, pinned_host, bytes, cudaMemcpyHostToDevice, s));
    // the slot is rewritten only after every queued step that reads it
    SG_CUDA(cudaStreamWaitEvent(s, f->slot_used[slot], 0));
    sg_status st = launch_brick_store(f, slot, f->staging, 0, 0, s);
    if (st) return st;
    f->slot_slice[slot] = slice;
    SG_CUDA(cudaEventRecord(f->slot_ready[slot], s));
    return SG_OK;
}

extern "C" sg_status sg_field_max_speed(sg_field *f, int32_t slot, double *cells_per_time, void *stream)
{
    SG_CHECK(f && cells_per_time, SG_ERR_INVALID_ARG, "NULL argument");
    SG_CHECK(slot >= 0 && slot < f->desc.n_slots, SG_ERR_INVALID_ARG, "slot %d out of range", slot);
    SG_CUDA(cudaSetDevice(f->ctx->device));
    cudaStream_t s = (cudaStream_t)stream;
    sg_status st = launch_max_speed(f, slot, s);
    if (st) return st;
    unsigned bits = 0;
    SG_CUDA(cudaMemcpyAsync(&bits, f->speed_bits, sizeof bits, cudaMemcpyDeviceToHost, s));
    SG_CUDA(cudaStreamSynchronize(s));
    float v;
    memcpy(&v, &bits, sizeof v);
    *cells_per_time = (double)v;
    return SG_OK;
}

extern "C" sg_status sg_field_read_brick(sg_field *f, int32_t slot, int32_t bx, int32_t by, int32_t bz, void *out,
                                         float *scale, void *stream)
{
    SG_CHECK(f && out, SG_ERR_INVALID_ARG, "NULL argument");
    SG_CHECK(f->desc.layout != SG_FIELD_GLOBAL, SG_ERR_UNSUPPORTED, "the global layout has no bricks");
    SG_CHECK(slot >= 0 && slot < f->desc.n_slots, SG_ERR_INVALID_ARG, "slot %d out of range", slot);
    const DevField &g = f->geom;
    SG_CHECK(bx >= 0 && bx < g.B[0] && by >= 0 && by < g.B[1] && bz >= 0 && bz < g.B[2], SG_ERR_INVALID_ARG,
             "brick out of range");
    SG_CUDA(cudaSetDevice(f->ctx->device));
    cudaStream_t s = (cudaStream_t)stream;
    const int b = (bz * g.B[1] + by) * g.B[0] + bx;
    const size_t raw_bytes = (size_t)g.brick_elems * f->elem_bytes;
    char *raw = (char *)malloc(raw_bytes);
    SG_CHECK(raw != nullptr, SG_ERR_OOM, "host allocation of %zu bytes failed", raw_bytes);
    float sc = 1.0f;
    cudaError_t e = cudaMemcpyAsync(raw, f->slot_data[slot] + (size_t)b * f->brick_bytes, raw_bytes,
                                    cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&sc, f->slot_scales[slot] + b, sizeof(float), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        free(raw);
        return cuda_error(e, "read_brick copy");
    }
    if (scale) *scale = sc;
    for (int z = 0; z < g.S[2]; ++z)
        for (int y = 0; y < g.S[1]; ++y)
            for (int x = 0; x < g.S[0]; ++x) {
                const long long src = storage_index(f->desc.layout, x, y, z, g);
                const long long dst = 3 * (((long long)z * g.S[1] + y) * g.S[0] + x);
                if (f->desc.dtype == SG_F32 && f->desc.layout == SG_LAYOUT_CELL8) {
                    const float *v = reinterpret_cast<const float *>(raw);
                    float *o = reinterpret_cast<float *>(out) + dst;
                    for (int a = 0; a < 3; ++a) o[a] = v[cell8_f32_index(x, y, z, a, g)];
                } else if (f->desc.dtype == SG_F32) {
                    const float *v = reinterpret_cast<const float *>(raw) + 4 * src;
                    float *o = reinterpret_cast<float *>(out) + dst;
                    o[0] = v[0];
                    o[1] = v[1];
                    o[2] = v[2];
                } else if (f->desc.dtype == SG_FX21) {
                    const uint32_t *v = reinterpret_cast<const uint32_t *>(raw) + 2 * src;
                    int32_t *o = reinterpret_cast<int32_t *>(out) + dst;
                    const uint32_t lo = v[0], hi = v[1];
                    const bool bad = (hi & 0x400u) != 0;
                    o[0] = bad ? INT32_MIN : (int32_t)(lo & 0x1FFFFFu) - (1 << 20);
                    o[1] = bad ? INT32_MIN : (int32_t)(((lo >> 21) | (hi << 11)) & 0x1FFFFFu) - (1 << 20);
                    o[2] = bad ? INT32_MIN : (int32_t)(hi >> 11) - (1 << 20);
                } else {
                    const uint16_t *v = reinterpret_cast<const uint16_t *>(raw) + 4 * src;
                    uint16_t *o = reinterpret_cast<uint16_t *>(out) + dst;
                    o[0] = v[0];
                    o[1] = v[1];
                    o[2] = v[2];
                }
            }
    free(raw);
    return SG_OK;
}
