// Line output: compaction of the per-line vertex slabs into CSR (getLines of
// Sec. 3.2 / Fig. 4; assembleOutput of Listing 2).
//
// Each line owns a slab of max_steps+1 vertices while it is traced, so a step
// writes its vertex without any allocation.  Readback scans the line lengths
// (exclusive scan to int64 offsets) and gathers every line's vertices to its
// offset; the destination may be device or page-locked host memory.
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
            for (long long k = lane; k < cnt; k += 32) d[k] = s[k];
        }
        if (lane == 0) {
            if (st_out) st_out[i] = st_in[i];
            if (mg_out) mg_out[i] = mg_in[i];
            if (off_out) off_out[i] = off[i];
        }
    }
    if (off_out && blockIdx.x == 0 && threadIdx.x == 0) off_out[n] = off[n];
}

sg_status launch_scan_lengths(sg_tracer *t, cudaStream_t s)
{
    const long long n = t->n_seeds;
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
    const long long n = t->n_seeds;
    int grid = t->ctx->sm_count * 8;
    gather_lines_kernel<<<grid, 256, 0, s>>>(t->slab, (long long)t->p.max_steps + 1, t->line_len, t->offsets, n,
                                             vertices, t->line_status, status, t->line_margin, margin, offsets);
    SG_CUDA(cudaGetLastError());
    return SG_OK;
}

}  // namespace sg
