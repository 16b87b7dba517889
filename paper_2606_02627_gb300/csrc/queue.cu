// Per-brick particle queues: the exchange step between rounds.
//
// The paper forwards particles between GPUs with RaFI: emitOutgoing() buffers
// a particle for its destination rank and a collective all-to-all moves the
// buffers; the host learns whether any particle is left anywhere
// (Sec. 3.1.2, Listing 2).  Here every brick lives on the same GPU, so the
// exchange is a counting sort of the outgoing records by destination brick
// (histogram, exclusive scan, scatter) into the next round's queue, and the
// "any particle left" reduction is the queue length, which a device-side
// control kernel turns into the condition of the CUDA graph's while-node.
#include "tracer.cuh"

namespace sg {

__device__ __forceinline__ int brick_key(const BinArgs &A, uint32_t line, int cx, int cy, int cz)
{
    if (A.line_req) {
        const ReqDev &R = A.reqs[A.line_req[line]];
        const int bx = min(cx / R.F.n[0], R.F.B[0] - 1);
        const int by = min(cy / R.F.n[1], R.F.B[1] - 1);
        const int bz = min(cz / R.F.n[2], R.F.B[2] - 1);
        return (int)R.brick_base + (bz * R.F.B[1] + by) * R.F.B[0] + bx;
    }
    const int bx = min(cx / A.n[0], A.B[0] - 1);
    const int by = min(cy / A.n[1], A.B[1] - 1);
    const int bz = min(cz / A.n[2], A.B[2] - 1);
    const int b = (bz * A.B[1] + by) * A.B[0] + bx;
    return A.key_map ? A.key_map[b] : b;
}

// Histogram of destination bricks (shared-memory counters when they fit).
__global__ void bin_count_kernel(BinArgs A)
{
    extern __shared__ uint32_t hist[];
    const bool local = A.nb <= 8192;
    if (local)
        for (int b = threadIdx.x; b < A.nb; b += blockDim.x) hist[b] = 0;
    __syncthreads();
    const uint32_t n = *A.src_count;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float4 a = reinterpret_cast<const float4 *>(A.src + i)[0];
        const int4 c = reinterpret_cast<const int4 *>(A.src + i)[1];
        const int b = brick_key(A, __float_as_uint(a.w), c.x, c.y, c.z);
        if (local) atomicAdd(hist + b, 1u);
        else atomicAdd(A.brick_count + b, 1u);
    }
    __syncthreads();
    if (local)
        for (int b = threadIdx.x; b < A.nb; b += blockDim.x)
            if (hist[b]) atomicAdd(A.brick_count + b, hist[b]);
}

// Exclusive scan of the brick histogram (one block): queue offsets per brick,
// the round's queue length; clears the histogram for the next use.
__global__ void bin_scan_kernel(BinArgs A)
{
    __shared__ uint32_t warp_sums[32];
    __shared__ uint32_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const unsigned lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int base = 0; base < A.nb; base += blockDim.x) {
        const int b = base + threadIdx.x;
        const uint32_t v = b < A.nb ? A.brick_count[b] : 0u;
        uint32_t x = v;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(SG_FULL_MASK, x, o);
            if ((int)lane >= o) x += y;
        }
        if (lane == 31) warp_sums[warp] = x;
        __syncthreads();
        if (warp == 0) {
            uint32_t w = lane < (blockDim.x >> 5) ? warp_sums[lane] : 0u;
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(SG_FULL_MASK, w, o);
                if ((int)lane >= o) w += y;
            }
            warp_sums[lane] = w;
        }
        __syncthreads();
        const uint32_t before = carry + (warp ? warp_sums[warp - 1] : 0u) + x - v;
        if (b < A.nb) {
            A.brick_cursor[b] = before;
            A.brick_count[b] = 0;
            if (b == A.n_local) A.ctrl->q_count = before;           // the local keys' records
            if (b >= A.n_local && A.key_start) A.key_start[b - A.n_local] = before;
        }
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry = before + v;
        __syncthreads();
    }
    if (threadIdx.x == 0 && A.n_local >= A.nb) A.ctrl->q_count = carry;
}

// Scatter each record to its brick's segment; lanes with the same brick share
// one atomicAdd (__match_any_sync).
__global__ void bin_scatter_kernel(BinArgs A)
{
    const uint32_t n = *A.src_count;
    const unsigned lane = threadIdx.x & 31;
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t base = (blockIdx.x * blockDim.x + threadIdx.x) & ~31u; base < n; base += stride) {
        const uint32_t i = base + lane;
        const bool valid = i < n;
        const unsigned vm = __ballot_sync(SG_FULL_MASK, valid);
        if (!valid) continue;
        const int4 *s = reinterpret_cast<const int4 *>(A.src + i);
        const int4 r0 = s[0], r1 = s[1];
        const int b = brick_key(A, (uint32_t)r0.w, r1.x, r1.y, r1.z);
        const unsigned peers = __match_any_sync(vm, b);
        const int leader = __ffs(peers) - 1;
        uint32_t pos = 0;
        if ((int)lane == leader) pos = atomicAdd(A.brick_cursor + b, (uint32_t)__popc(peers));
        pos = __shfl_sync(peers, pos, leader) + __popc(peers & ((1u << lane) - 1u));
        int4 *d = reinterpret_cast<int4 *>(A.dst + pos);
        d[0] = r0;
        d[1] = r1;
    }
}

// After a scatter: the source buffer is empty, the queue cursor rewinds, and
// the loop continues while the queue holds particles and the round cap is not
// reached.  mode 0: after binning the parked records (start of a call);
// mode 1: after binning a round's outgoing records.  With a brick window the
// next round's part of the queue is the segments of the next window bricks
// that hold particles (brick_cursor[b] is the end of brick b's segment once
// the scatter is done); the others are carried (carry_kernel).
__global__ void ctrl_kernel(Ctrl *ctrl, uint32_t *src_count, int mode, cudaGraphConditionalHandle h, int use_graph,
                            const uint32_t *brick_cursor, int nb)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    *src_count = 0;
    ctrl->q_head = 0;
    if (mode == 1) ctrl->round += 1;
    const uint32_t total = ctrl->q_count;
    ctrl->q_total = total;
    ctrl->win_start = 0;
    const uint32_t w = ctrl->window;
    if (w > 0 && total > 0 && (uint32_t)nb > w) {
        uint32_t lo = ctrl->win_lo < (uint32_t)nb ? ctrl->win_lo : 0u;
        uint32_t start = 0, end = 0;
        for (int tries = 0; tries <= nb; ++tries) {        // a non-empty window exists: total > 0
            const uint32_t hi = min(lo + w, (uint32_t)nb);
            start = lo == 0 ? 0u : brick_cursor[lo - 1];
            end = brick_cursor[hi - 1];
            lo = hi >= (uint32_t)nb ? 0u : hi;
            if (end > start) break;
        }
        ctrl->win_lo = lo;
        ctrl->win_start = start;
        ctrl->q_head = start;
        ctrl->q_count = end;
    }
    const bool more = total > 0;
    const bool capped = ctrl->round >= ctrl->max_rounds;
    if (more && capped) ctrl->err |= CTRL_ERR_ROUND_LIMIT;
    if (!more || capped) ctrl->last_rounds = ctrl->round;
    if (use_graph) cudaGraphSetConditional(h, (more && !capped) ? 1u : 0u);
}

// After a round that advanced one brick window: the queue's records outside
// the window, [0, win_start) and [q_count, q_total), join the round's
// outgoing records, to be binned with them for the next round; then the
// outgoing count takes them in (carry_fix_kernel, one thread, after every
// copy is done).
__global__ void carry_kernel(const Ctrl *ctrl, const Particle *q, Particle *o)
{
    if (ctrl->window == 0) return;
    const uint32_t s = ctrl->win_start, e = ctrl->q_count, tot = ctrl->q_total, base = ctrl->o_count;
    const uint32_t n = s + (tot - e);
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const uint32_t src = i < s ? i : e + (i - s);
        const int4 *a = reinterpret_cast<const int4 *>(q + src);
        int4 *d = reinterpret_cast<int4 *>(o + base + i);
        d[0] = a[0];
        d[1] = a[1];
    }
}

__global__ void carry_fix_kernel(Ctrl *ctrl)
{
    if (threadIdx.x != 0 || blockIdx.x != 0 || ctrl->window == 0) return;
    ctrl->o_count += ctrl->win_start + (ctrl->q_total - ctrl->q_count);
}

sg_status launch_carry(sg_tracer *t, cudaStream_t s)
{
    carry_kernel<<<t->ctx->sm_count * 2, 256, 0, s>>>(t->ctrl, t->q, t->o);
    SG_CUDA(cudaGetLastError());
    carry_fix_kernel<<<1, 32, 0, s>>>(t->ctrl);
    SG_CUDA(cudaGetLastError());
    return SG_OK;
}

// After the round loop of a call: if the round cap stopped it with particles
// left, those particles (the next round's queue) are parked for the next call,
// and each one's line length is brought up to the vertices written so far, so
// that the partial lines read back consistently and a later trace() or step()
// continues them from where they stopped.  One block: the counters move once
// every record has been copied.
__global__ void __launch_bounds__(1024) park_rest_kernel(Ctrl *ctrl, const Particle *q, Particle *park,
                                                         uint32_t *line_len)
{
    if (!(ctrl->err & CTRL_ERR_ROUND_LIMIT)) return;
    const uint32_t n = ctrl->q_total, base = ctrl->p_count;
    for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) {
        const int4 *s = reinterpret_cast<const int4 *>(q + i);
        const int4 r0 = s[0], r1 = s[1];
        int4 *d = reinterpret_cast<int4 *>(park + base + i);
        d[0] = r0;
        d[1] = r1;
        line_len[(uint32_t)r0.w] = (uint32_t)r1.w + 1u;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        ctrl->p_count = base + n;
        ctrl->q_count = 0;
        ctrl->q_total = 0;
    }
}

sg_status launch_park_rest(sg_tracer *t, cudaStream_t s)
{
    park_rest_kernel<<<1, 1024, 0, s>>>(t->ctrl, t->q, t->park, t->line_len);
    SG_CUDA(cudaGetLastError());
    return SG_OK;
}

__global__ void prepare_kernel(Ctrl *ctrl, uint32_t horizon, uint32_t max_rounds, uint32_t window)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    ctrl->window = window;
    ctrl->win_lo = 0;
    ctrl->win_start = 0;
    ctrl->q_total = 0;
    ctrl->q_count = 0;
    ctrl->q_head = 0;
    ctrl->o_count = 0;
    ctrl->round = 0;
    ctrl->err = 0;
    ctrl->horizon = horizon;
    ctrl->max_rounds = max_rounds;
}

sg_status launch_prepare_call(sg_tracer *t, uint32_t horizon, uint32_t max_rounds, cudaStream_t s)
{
    // brick windows for the persistent kernels (they pop from the window's
    // start); the one-launch-per-step kernel and partitioned tracers take
    // every brick each round
    const bool windowed = t->pod_world == 0 &&
                          (t->p.kernel == SG_KERNEL_PERSISTENT || t->p.kernel == SG_KERNEL_LOCKSTEP);
    prepare_kernel<<<1, 32, 0, s>>>(t->ctrl, horizon, max_rounds, windowed ? (uint32_t)t->p.brick_window : 0u);
    SG_CUDA(cudaGetLastError());
    return SG_OK;
}

sg_status launch_bin_args(const BinArgs &A, int sm_count, cudaStream_t s, bool in_graph, unsigned long long cond_handle,
                          int mode)
{
    const int grid = sm_count * 2;
    const size_t smem = A.nb <= 8192 ? sizeof(uint32_t) * A.nb : 0;
    bin_count_kernel<<<grid, 512, smem, s>>>(A);
    SG_CUDA(cudaGetLastError());
    bin_scan_kernel<<<1, 1024, 0, s>>>(A);
    SG_CUDA(cudaGetLastError());
    bin_scatter_kernel<<<grid, 512, 0, s>>>(A);
    SG_CUDA(cudaGetLastError());
    ctrl_kernel<<<1, 32, 0, s>>>(A.ctrl, A.src_count, mode, (cudaGraphConditionalHandle)cond_handle, in_graph ? 1 : 0,
                                 A.brick_cursor, A.n_local);
    SG_CUDA(cudaGetLastError());
    return SG_OK;
}

// mode 0: bin parked records (start of a call); mode 1: bin outgoing records.
sg_status launch_bin(sg_tracer *t, Particle *src, uint32_t *src_count, cudaStream_t s, bool in_graph,
                     unsigned long long cond_handle, int mode)
{
    BinArgs A;
    A.line_req = nullptr;
    A.reqs = nullptr;
    A.src = src;
    A.src_count = src_count;
    A.dst = t->q;
    A.brick_count = t->brick_count;
    A.brick_cursor = t->brick_cursor;
    A.ctrl = t->ctrl;
    for (int a = 0; a < 3; ++a) {
        A.n[a] = t->field->geom.n[a];
        A.B[a] = t->field->geom.B[a];
    }
    A.nb = t->nb;
    A.key_map = nullptr;
    A.n_local = t->nb;
    A.key_start = nullptr;
    if (t->pod_world > 0) {
        A.key_map = t->pod_key_map;
        A.n_local = t->pod_local;
        A.nb = t->pod_local + t->pod_world;
        A.key_start = t->pod_key_start;
    }
    return launch_bin_args(A, t->ctx->sm_count, s, in_graph, cond_handle, mode);
}

__global__ void fill_inf_kernel(float *dst, long long n)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        dst[i] = INFINITY;
}

sg_status launch_fill_inf(float *dst, long long n, cudaStream_t s)
{
    if (n <= 0) return SG_OK;
    fill_inf_kernel<<<(unsigned)((n + 255) / 256 < 8192 ? (n + 255) / 256 : 8192), 256, 0, s>>>(dst, n);
    SG_CUDA(cudaGetLastError());
    return SG_OK;
}

__global__ void set_q_count_kernel(Ctrl *ctrl, uint32_t n)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        ctrl->q_count = n;
        ctrl->q_head = 0;
    }
}

sg_status launch_set_q_count(Ctrl *ctrl, uint32_t n, cudaStream_t s)
{
    set_q_count_kernel<<<1, 32, 0, s>>>(ctrl, n);
    SG_CUDA(cudaGetLastError());
    return SG_OK;
}

// dst[i] = i mod period (the seed of streamline i)
__global__ void iota_kernel(int32_t *dst, long long n, long long period)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        dst[i] = (int32_t)(i % period);
}

sg_status launch_iota(int32_t *dst, int64_t n, int64_t period, cudaStream_t s)
{
    iota_kernel<<<(unsigned)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096), 256, 0, s>>>(dst, n, period);
    SG_CUDA(cudaGetLastError());
    return SG_OK;
}

}  // namespace sg
