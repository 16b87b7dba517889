// Line output: compaction of the per-line vertex slabs into CSR (getLines of
// Sec. 3.2 / Fig. 4; assembleOutput of Listing 2).
//
// Each line owns a slab of max_steps+1 vertices while it is traced, so a step
// writes its vertex without any allocation.  Readback scans the line lengths
// (exclusive scan to int64 offsets) and gathers every line's vertices to its
// offset; the destination may be device or page-locked host memory.
#include <mutex>

#include "tracer.cuh"

namespace sg {

constexpr int SCAN_THREADS = 1024;
constexpr int SCAN_ITEMS = 4;
constexpr int SCAN_CHUNK = SCAN_THREADS * SCAN_ITEMS;

// Block-wide inclusive scan of one 64-bit value per thread; returns the
// inclusive prefix; *total receives the block total.
__device__ __forceinline__ unsigned long long block_scan_u64(unsigned long long v, unsigned long long *total)
{
    __shared__ unsigned long long ws[32];
    const unsigned lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
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
    const unsigned long long r = x + (warp ? ws[warp - 1] : 0ull);
    *total = ws[(blockDim.x >> 5) - 1];
    __syncthreads();
    return r;
}

// Phase 1: per-chunk sums of the lengths (and of nonempty lines, packed in the
// high 24 bits: at most 4096 lines per chunk).
__global__ void scan_reduce_kernel(const uint32_t *len, long long n, unsigned long long *block_sums)
{
    const long long base = (long long)blockIdx.x * SCAN_CHUNK;
    unsigned long long s = 0;
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        const long long i = base + (long long)k * SCAN_THREADS + threadIdx.x;
        if (i < n) {
            const uint32_t l = len[i];
            s += (unsigned long long)l + (l ? (1ull << 40) : 0ull);
        }
    }
    unsigned long long tot;
    block_scan_u64(s, &tot);
    if (threadIdx.x == 0) block_sums[blockIdx.x] = tot;
}

// Phase 2 (one block): exclusive scan of the chunk sums, in passes of 1024.
__global__ void scan_blocks_kernel(unsigned long long *block_sums, long long nblocks, int64_t *totals, int64_t *offsets,
                                   long long n)
{
    __shared__ unsigned long long carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (long long base = 0; base < nblocks; base += blockDim.x) {
        const long long i = base + threadIdx.x;
        const unsigned long long v = i < nblocks ? block_sums[i] : 0ull;
        unsigned long long tot;
        const unsigned long long incl = block_scan_u64(v, &tot);
        const unsigned long long c = carry;
        if (i < nblocks) block_sums[i] = c + incl - v;
        __syncthreads();
        if (threadIdx.x == 0) carry = c + tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const unsigned long long all = carry;
        const long long verts = (long long)(all & ((1ull << 40) - 1));
        const long long nonempty = (long long)(all >> 40);
        totals[0] = verts;
        totals[1] = n;
        totals[2] = verts - nonempty;
        offsets[n] = verts;
    }
}

// Phase 3: offsets of every line.
__global__ void scan_apply_kernel(const uint32_t *len, long long n, const unsigned long long *block_sums,
                                  int64_t *offsets)
{
    const long long base = (long long)blockIdx.x * SCAN_CHUNK;
    const unsigned long long off0 = block_sums[blockIdx.x] & ((1ull << 40) - 1);
    uint32_t v[SCAN_ITEMS];
    unsigned long long s = 0;
    // each thread takes SCAN_ITEMS consecutive lines
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        const long long i = base + (long long)threadIdx.x * SCAN_ITEMS + k;
        v[k] = i < n ? len[i] : 0u;
        s += v[k];
    }
    unsigned long long tot;
    const unsigned long long incl = block_scan_u64(s, &tot);
    unsigned long long run = off0 + incl - s;
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        const long long i = base + (long long)threadIdx.x * SCAN_ITEMS + k;
        if (i < n) offsets[i] = (int64_t)run;
        run += v[k];
    }
}

// One warp per line: copy its vertices (contiguous floats on both sides).
__global__ void gather_lines_kernel(const float *__restrict__ slab, long long W, const uint32_t *__restrict__ len,
                                    const int64_t *__restrict__ off, long long n, float *__restrict__ vertices,
                                    const uint8_t *__restrict__ st_in, uint8_t *st_out, const float *__restrict__ mg_in,
                                    float *mg_out, int64_t *off_out)
{
    const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    const unsigned lane = threadIdx.x & 31;
    for (long long i = warp; i < n; i += nwarps) {
        const long long cnt = 3ll * len[i];
        if (vertices) {
            const float *s = slab + i * W * 3;
            float *d = vertices + 3ll * off[i];
            // eight independent loads in flight per lane before the stores:
            // enough bytes in flight to stream at HBM rate
            long long k = lane;
            for (; k + 7 * 32 < cnt; k += 8 * 32) {
                float v[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) v[u] = __ldcs(s + k + u * 32);
#pragma unroll
                for (int u = 0; u < 8; ++u) d[k + u * 32] = v[u];
            }
            for (; k < cnt; k += 32) d[k] = __ldcs(s + k);
        }
        if (lane == 0) {
            if (st_out) st_out[i] = st_in[i];
            if (mg_out) mg_out[i] = mg_in[i];
            if (off_out) off_out[i] = off[i];
        }
    }
    if (off_out && blockIdx.x == 0 && threadIdx.x == 0) off_out[n] = off[n];
}

// Lines [a, b) into a staging buffer: line i lands at float 3 * (off[i] - base).
__global__ void gather_chunk_kernel(const float *__restrict__ slab, long long W, const uint32_t *__restrict__ len,
                                    const int64_t *__restrict__ off, long long a, long long b, long long base,
                                    float *__restrict__ dst)
{
    const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    const unsigned lane = threadIdx.x & 31;
    for (long long i = a + warp; i < b; i += nwarps) {
        const long long cnt = 3ll * len[i];
        const float *s = slab + i * W * 3;
        float *d = dst + 3ll * (off[i] - base);
        long long k = lane;
        for (; k + 7 * 32 < cnt; k += 8 * 32) {
            float v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) v[u] = __ldcs(s + k + u * 32);
#pragma unroll
            for (int u = 0; u < 8; ++u) d[k + u * 32] = v[u];
        }
        for (; k < cnt; k += 32) d[k] = __ldcs(s + k);
    }
}

sg_status launch_gather_chunk(const sg_tracer *t, long long a, long long b, long long base, float *dst, cudaStream_t s)
{
    gather_chunk_kernel<<<t->ctx->sm_count * 8, 256, 0, s>>>(t->slab, slab_stride(t->p.max_steps), t->line_len,
                                                              t->offsets, a, b, base, dst);
    SG_CUDA(cudaGetLastError());
    return SG_OK;
}

// ------------------------------------------------------------------ bidirectional lines

// Joined polyline lengths: the backward line (seed excluded) then the forward
// line; 0 for an OUT seed (both lines empty).
__global__ void join_len_kernel(const uint32_t *__restrict__ len, long long n, uint32_t *__restrict__ jlen)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const uint32_t lf = len[i], lb = len[n + i];
        jlen[i] = lf == 0u ? 0u : lb - 1u + lf;
    }
}

// One warp per seed: the backward line's vertices lb-1 .. 1, then the
// forward line's vertices 0 .. lf-1.
__global__ void join_gather_kernel(const float *__restrict__ slab, long long W, const uint32_t *__restrict__ len,
                                   const int64_t *__restrict__ joff, long long n, int64_t *off_out,
                                   float *__restrict__ vertices, int64_t *seed_vertex)
{
    const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    const unsigned lane = threadIdx.x & 31;
    for (long long i = warp; i < n; i += nwarps) {
        const long long lf = len[i], lb = len[n + i];
        const long long o = joff[i];
        if (vertices && lf > 0) {
            float *d = vertices + 3 * o;
            const float *sb = slab + (n + i) * W * 3;
            const long long nb = 3 * (lb - 1);
            for (long long k = lane; k < nb; k += 32) {
                const long long j = k / 3, c = k - 3 * j;
                d[k] = __ldcs(sb + 3 * (lb - 1 - j) + c);
            }
            const float *sf = slab + i * W * 3;
            for (long long k = lane; k < 3 * lf; k += 32) d[nb + k] = __ldcs(sf + k);
        }
        if (lane == 0) {
            if (off_out) off_out[i] = o;
            if (seed_vertex) seed_vertex[i] = lf > 0 ? lb - 1 : -1;
        }
    }
    if (off_out && blockIdx.x == 0 && threadIdx.x == 0) off_out[n] = joff[n];
}

static sg_status launch_scan(const uint32_t *len, long long n, unsigned long long *block_sums, int64_t *totals,
                             int64_t *offsets, cudaStream_t s)
{
    const long long nblocks = (n + SCAN_CHUNK - 1) / SCAN_CHUNK;
    if (nblocks > 0) {
        scan_reduce_kernel<<<(unsigned)nblocks, SCAN_THREADS, 0, s>>>(len, n, block_sums);
        SG_CUDA(cudaGetLastError());
    }
    scan_blocks_kernel<<<1, SCAN_THREADS, 0, s>>>(block_sums, nblocks, totals, offsets, n);
    SG_CUDA(cudaGetLastError());
    if (nblocks > 0) {
        scan_apply_kernel<<<(unsigned)nblocks, SCAN_THREADS, 0, s>>>(len, n, block_sums, offsets);
        SG_CUDA(cudaGetLastError());
    }
    return SG_OK;
}

sg_status launch_join_scan(sg_tracer *t, cudaStream_t s)
{
    const long long n = t->n_seeds;
    if (n > 0) {
        join_len_kernel<<<(unsigned)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096), 256, 0, s>>>(t->line_len, n,
                                                                                                 t->join_len);
        SG_CUDA(cudaGetLastError());
    }
    return launch_scan(t->join_len, n, t->block_sums, t->join_tot, t->join_off, s);
}

sg_status launch_join(sg_tracer *t, int64_t *offsets, float *vertices, int64_t *seed_vertex, cudaStream_t s)
{
    const long long n = t->n_seeds;
    if (n == 0) {
        if (offsets) SG_CUDA(cudaMemsetAsync(offsets, 0, sizeof(int64_t), s));
        return SG_OK;
    }
    join_gather_kernel<<<t->ctx->sm_count * 8, 256, 0, s>>>(t->slab, slab_stride(t->p.max_steps), t->line_len,
                                                             t->join_off, n, offsets, vertices, seed_vertex);
    SG_CUDA(cudaGetLastError());
    return SG_OK;
}

sg_status launch_scan_lengths(sg_tracer *t, cudaStream_t s)
{
    const long long n = t->n_lines;
    const long long nblocks = (n + SCAN_CHUNK - 1) / SCAN_CHUNK;
    if (nblocks > 0) {
        scan_reduce_kernel<<<(unsigned)nblocks, SCAN_THREADS, 0, s>>>(t->line_len, n, t->block_sums);
        SG_CUDA(cudaGetLastError());
    }
    scan_blocks_kernel<<<1, SCAN_THREADS, 0, s>>>(t->block_sums, nblocks, t->totals, t->offsets, n);
    SG_CUDA(cudaGetLastError());
    if (nblocks > 0) {
        scan_apply_kernel<<<(unsigned)nblocks, SCAN_THREADS, 0, s>>>(t->line_len, n, t->block_sums, t->offsets);
        SG_CUDA(cudaGetLastError());
    }
    return SG_OK;
}

sg_status launch_gather_lines(sg_tracer *t, int64_t *offsets, float *vertices, uint8_t *status, float *margin,
                              cudaStream_t s)
{
    const long long n = t->n_lines;
    int grid = t->ctx->sm_count * 8;
    gather_lines_kernel<<<grid, 256, 0, s>>>(t->slab, slab_stride(t->p.max_steps), t->line_len, t->offsets, n,
                                             vertices, t->line_status, status, t->line_margin, margin, offsets);
    SG_CUDA(cudaGetLastError());
    return SG_OK;
}

// Scan + gather for a contiguous range of lines whose slabs start at `slab`
// (the request lines of a batch).  scan_only: offsets and totals only.
sg_status launch_compact_range(const uint32_t *len, long long n, const float *slab, long long W, const uint8_t *st_in,
                               const float *mg_in, unsigned long long *block_sums, int64_t *dev_offsets,
                               int64_t *totals, int64_t *offsets_out, float *vertices, uint8_t *status_out,
                               float *margin_out, int sm_count, bool scan_only, cudaStream_t s)
{
    const long long nblocks = (n + SCAN_CHUNK - 1) / SCAN_CHUNK;
    if (scan_only) {
        if (nblocks > 0) {
            scan_reduce_kernel<<<(unsigned)nblocks, SCAN_THREADS, 0, s>>>(len, n, block_sums);
            SG_CUDA(cudaGetLastError());
        }
        scan_blocks_kernel<<<1, SCAN_THREADS, 0, s>>>(block_sums, nblocks, totals, dev_offsets, n);
        SG_CUDA(cudaGetLastError());
        if (nblocks > 0) {
            scan_apply_kernel<<<(unsigned)nblocks, SCAN_THREADS, 0, s>>>(len, n, block_sums, dev_offsets);
            SG_CUDA(cudaGetLastError());
        }
        return SG_OK;
    }
    gather_lines_kernel<<<sm_count * 8, 256, 0, s>>>(slab, W, len, dev_offsets, n, vertices, st_in, status_out, mg_in,
                                                     margin_out, offsets_out);
    SG_CUDA(cudaGetLastError());
    return SG_OK;
}

// ------------------------------------------------------------------ compaction with caller-owned scratch

namespace {

sg_status compact_lines(const float *slab, long long W, const uint32_t *lengths, long long n,
                        unsigned long long *scratch, int64_t *offsets, float *vertices, cudaStream_t s)
{
    const long long nblocks = (n + SCAN_CHUNK - 1) / SCAN_CHUNK;
    int64_t *totals = reinterpret_cast<int64_t *>(scratch + nblocks);
    if (nblocks > 0) {
        scan_reduce_kernel<<<(unsigned)nblocks, SCAN_THREADS, 0, s>>>(lengths, n, scratch);
        SG_CUDA(cudaGetLastError());
    }
    scan_blocks_kernel<<<1, SCAN_THREADS, 0, s>>>(scratch, nblocks, totals, offsets, n);
    SG_CUDA(cudaGetLastError());
    if (nblocks > 0) {
        scan_apply_kernel<<<(unsigned)nblocks, SCAN_THREADS, 0, s>>>(lengths, n, scratch, offsets);
        SG_CUDA(cudaGetLastError());
        if (vertices) {
            int dev = 0, sms = 0;
            SG_CUDA(cudaGetDevice(&dev));
            SG_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
            gather_lines_kernel<<<sms * 8, 256, 0, s>>>(slab, W, lengths, offsets, n, vertices, nullptr, nullptr,
                                                        nullptr, nullptr, nullptr);
            SG_CUDA(cudaGetLastError());
        }
    }
    return SG_OK;
}

}  // namespace

// ------------------------------------------------------------------ allocation-free compaction
//
// Scratch of sg_lines_compact_static: one 64-bit sum per chunk of SCAN_CHUNK
// lines plus the totals written by the middle scan pass.  It lives in the
// library's own device memory (a file-scope array every GPU that loads the
// library holds until the process exits), so the entry point needs no
// allocation.  Every entry the scan reads is written earlier in the same call,
// so nothing has to start at zero.
constexpr long long STATIC_MAX_CHUNKS = 4096;
constexpr long long STATIC_MAX_LINES = STATIC_MAX_CHUNKS * SCAN_CHUNK;   // 16,777,216 lines
static __device__ __align__(256) unsigned long long g_compact_scratch[STATIC_MAX_CHUNKS + 8];

// Host code may not use the array's name as a device address: its device
// address is looked up once per device, with that device current.
static std::mutex g_scratch_mu;
static unsigned long long *g_scratch_dev[1024];

static sg_status static_scratch(unsigned long long **out)
{
    int dev = 0;
    SG_CUDA(cudaGetDevice(&dev));
    SG_CHECK(dev >= 0 && dev < 1024, SG_ERR_UNSUPPORTED, "device ordinal %d out of range", dev);
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_dev[dev]) {
        void *p = nullptr;
        SG_CUDA(cudaGetSymbolAddress(&p, g_compact_scratch));
        g_scratch_dev[dev] = (unsigned long long *)p;
    }
    *out = g_scratch_dev[dev];
    return SG_OK;
}

}  // namespace sg

using namespace sg;

extern "C" sg_status sg_lines_compact_static(const float *slab, int64_t max_vertices_per_line, const uint32_t *lengths,
                                             int64_t n_lines, int64_t *offsets, float *vertices, void *stream)
{
    SG_CHECK(n_lines >= 0, SG_ERR_INVALID_ARG, "n_lines must be >= 0");
    SG_CHECK(n_lines <= STATIC_MAX_LINES, SG_ERR_INVALID_ARG,
             "n_lines = %lld exceeds the limit of the allocation-free compaction (%lld lines)", (long long)n_lines,
             (long long)STATIC_MAX_LINES);
    SG_CHECK(max_vertices_per_line >= 1 && max_vertices_per_line < (1ll << 28), SG_ERR_INVALID_ARG,
             "max_vertices_per_line must be in [1, 2^28)");
    SG_CHECK(offsets != nullptr, SG_ERR_INVALID_ARG, "offsets is NULL");
    SG_CHECK(n_lines == 0 || (lengths != nullptr && (slab != nullptr || vertices == nullptr)), SG_ERR_INVALID_ARG,
             "NULL input");
    unsigned long long *scratch = nullptr;
    sg_status st = static_scratch(&scratch);
    if (st) return st;
    // the totals go after the chunk sums' maximum extent, as the array is laid out
    const long long n = n_lines;
    const long long nblocks = (n + SCAN_CHUNK - 1) / SCAN_CHUNK;
    cudaStream_t s = (cudaStream_t)stream;
    int64_t *totals = reinterpret_cast<int64_t *>(scratch + STATIC_MAX_CHUNKS);
    if (nblocks > 0) {
        scan_reduce_kernel<<<(unsigned)nblocks, SCAN_THREADS, 0, s>>>(lengths, n, scratch);
        SG_CUDA(cudaGetLastError());
    }
    scan_blocks_kernel<<<1, SCAN_THREADS, 0, s>>>(scratch, nblocks, totals, offsets, n);
    SG_CUDA(cudaGetLastError());
    if (nblocks > 0) {
        scan_apply_kernel<<<(unsigned)nblocks, SCAN_THREADS, 0, s>>>(lengths, n, scratch, offsets);
        SG_CUDA(cudaGetLastError());
        if (vertices) {
            int dev = 0, sms = 0;
            SG_CUDA(cudaGetDevice(&dev));
            SG_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
            gather_lines_kernel<<<sms * 8, 256, 0, s>>>(slab, (long long)max_vertices_per_line, lengths, offsets, n,
                                                        vertices, nullptr, nullptr, nullptr, nullptr, nullptr);
            SG_CUDA(cudaGetLastError());
        }
    }
    return SG_OK;
}

extern "C" sg_status sg_lines_compact_scratch_bytes(int64_t n_lines, size_t *bytes)
{
    SG_CHECK(n_lines >= 0, SG_ERR_INVALID_ARG, "n_lines must be >= 0");
    SG_CHECK(bytes != nullptr, SG_ERR_INVALID_ARG, "bytes is NULL");
    const long long nblocks = (n_lines + SCAN_CHUNK - 1) / SCAN_CHUNK;
    *bytes = (size_t)(nblocks + 8) * sizeof(unsigned long long);
    return SG_OK;
}

extern "C" sg_status sg_lines_compact(const float *slab, int64_t max_vertices_per_line, const uint32_t *lengths,
                                      int64_t n_lines, void *scratch, size_t scratch_bytes, int64_t *offsets,
                                      float *vertices, void *stream)
{
    SG_CHECK(n_lines >= 0, SG_ERR_INVALID_ARG, "n_lines must be >= 0");
    SG_CHECK(n_lines < (1ll << 40), SG_ERR_INVALID_ARG, "n_lines too large");
    SG_CHECK(max_vertices_per_line >= 1 && max_vertices_per_line < (1ll << 28), SG_ERR_INVALID_ARG,
             "max_vertices_per_line must be in [1, 2^28)");
    SG_CHECK(offsets != nullptr && scratch != nullptr, SG_ERR_INVALID_ARG, "NULL offsets or scratch");
    SG_CHECK(((uintptr_t)scratch & 7u) == 0, SG_ERR_INVALID_ARG, "scratch must be 8-byte aligned");
    SG_CHECK(n_lines == 0 || (lengths != nullptr && (slab != nullptr || vertices == nullptr)), SG_ERR_INVALID_ARG,
             "NULL input");
    size_t need = 0;
    sg_status st = sg_lines_compact_scratch_bytes(n_lines, &need);
    if (st) return st;
    SG_CHECK(scratch_bytes >= need, SG_ERR_INVALID_ARG, "scratch of %zu bytes, %zu needed", scratch_bytes, need);
    return compact_lines(slab, (long long)max_vertices_per_line, lengths, (long long)n_lines,
                         reinterpret_cast<unsigned long long *>(scratch), offsets, vertices, (cudaStream_t)stream);
}
