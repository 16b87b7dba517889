// Seed points from control shapes, generated on the device: the low-level
// interface's convenience kernels that place seeds uniformly on lines and
// planes (Sec. 3.1).  Positions are computed in double precision with
// explicit round-to-nearest operations (no contraction) and rounded once to
// float32, so the same inputs give the same bits on any device.
//
//   rake:  n points evenly spaced on the segment a..b, both ends included
//   plane: nu x nv points evenly spaced on the parallelogram o + s u + t v,
//          s, t in [0, 1], point (i, j) at index j * nu + i
//   box:   n points uniform at random in [lo, hi] (per axis), from the
//          counter-based SplitMix64 (Steele, Lea, Flood 2014): value k of
//          stream s under seed z is mix64(key + (k + 1) G), key =
//          mix64(z G + C (s + 1)), G = 0x9E3779B97F4A7C15,
//          C = 0x632BE59BD9B4E019; a uniform double takes the top 53 bits;
//          point i uses values 3i, 3i+1, 3i+2 for x, y, z
#include "tracer.cuh"

namespace sg {

namespace {

struct V3 {
    double v[3];
};

__device__ __forceinline__ unsigned long long mix64(unsigned long long z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

constexpr unsigned long long GOLDEN = 0x9E3779B97F4A7C15ull;

__device__ __forceinline__ double frac_of(long long i, long long n)
{
    return n > 1 ? __ddiv_rn((double)i, (double)(n - 1)) : 0.0;
}

__global__ void rake_kernel(V3 a, V3 d, long long n, float *out)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const double t = frac_of(i, n);
#pragma unroll
        for (int c = 0; c < 3; ++c) out[3 * i + c] = __double2float_rn(__dadd_rn(a.v[c], __dmul_rn(d.v[c], t)));
    }
}

__global__ void plane_kernel(V3 o, V3 u, V3 v, long long nu, long long nv, float *out)
{
    const long long n = nu * nv;
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        const long long j = k / nu, i = k - j * nu;
        const double s = frac_of(i, nu), t = frac_of(j, nv);
#pragma unroll
        for (int c = 0; c < 3; ++c)
            out[3 * k + c] =
                __double2float_rn(__dadd_rn(__dadd_rn(o.v[c], __dmul_rn(u.v[c], s)), __dmul_rn(v.v[c], t)));
    }
}

__global__ void box_kernel(V3 lo, V3 d, long long n, unsigned long long key, float *out)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const unsigned long long k = (unsigned long long)(3 * i + c);
            const double u = (double)(mix64(key + (k + 1ull) * GOLDEN) >> 11) * 0x1.0p-53;
            out[3 * i + c] = __double2float_rn(__dadd_rn(lo.v[c], __dmul_rn(d.v[c], u)));
        }
    }
}

unsigned long long mix64_host(unsigned long long z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

V3 v3(const double *p)
{
    V3 r;
    for (int c = 0; c < 3; ++c) r.v[c] = p[c];
    return r;
}

unsigned grid_for(long long n)
{
    const long long g = (n + 255) / 256;
    return (unsigned)(g < 1 ? 1 : (g > 4096 ? 4096 : g));
}

sg_status check_seed_out(const float *out, long long n)
{
    SG_CHECK(n >= 0, SG_ERR_INVALID_ARG, "negative point count");
    SG_CHECK(n == 0 || out != nullptr, SG_ERR_INVALID_ARG, "out is NULL");
    if (n > 0) {
        const int k = pointer_kind(out);
        SG_CHECK(k == PTR_DEVICE || k == PTR_PINNED, SG_ERR_INVALID_ARG,
                 "out must be device or page-locked host memory");
    }
    return SG_OK;
}

}  // namespace

}  // namespace sg

using namespace sg;

extern "C" sg_status sg_seeds_rake(const double a[3], const double b[3], int64_t n, float *out, void *stream)
{
    SG_CHECK(a && b, SG_ERR_INVALID_ARG, "NULL endpoint");
    sg_status st = check_seed_out(out, n);
    if (st || n == 0) return st;
    V3 d;
    for (int c = 0; c < 3; ++c) d.v[c] = b[c] - a[c];
    rake_kernel<<<grid_for(n), 256, 0, (cudaStream_t)stream>>>(v3(a), d, n, out);
    SG_CUDA(cudaGetLastError());
    return SG_OK;
}

extern "C" sg_status sg_seeds_plane(const double origin[3], const double u[3], const double v[3], int64_t nu,
                                    int64_t nv, float *out, void *stream)
{
    SG_CHECK(origin && u && v, SG_ERR_INVALID_ARG, "NULL vector");
    SG_CHECK(nu >= 0 && nv >= 0 && (nv == 0 || nu <= (1ll << 40) / nv), SG_ERR_INVALID_ARG, "bad point counts");
    sg_status st = check_seed_out(out, nu * nv);
    if (st || nu * nv == 0) return st;
    plane_kernel<<<grid_for(nu * nv), 256, 0, (cudaStream_t)stream>>>(v3(origin), v3(u), v3(v), nu, nv, out);
    SG_CUDA(cudaGetLastError());
    return SG_OK;
}

extern "C" sg_status sg_seeds_box(const double lo[3], const double hi[3], int64_t n, uint64_t seed, uint64_t stream_id,
                                  float *out, void *stream)
{
    SG_CHECK(lo && hi, SG_ERR_INVALID_ARG, "NULL corner");
    sg_status st = check_seed_out(out, n);
    if (st || n == 0) return st;
    SG_CHECK(n <= (1ll << 60), SG_ERR_INVALID_ARG, "too many points");
    V3 d;
    for (int c = 0; c < 3; ++c) d.v[c] = hi[c] - lo[c];
    const unsigned long long key = mix64_host(seed * GOLDEN + 0x632BE59BD9B4E019ull * (stream_id + 1ull));
    box_kernel<<<grid_for(n), 256, 0, (cudaStream_t)stream>>>(v3(lo), d, n, key, out);
    SG_CUDA(cudaGetLastError());
    return SG_OK;
}
