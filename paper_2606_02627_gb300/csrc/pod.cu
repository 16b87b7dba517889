// Partition over data (POD): the bricks of a field are owned by ranks, one GPU
// each; a rank advects the particles of its own bricks and forwards the
// particles that leave them to the owning ranks between rounds (the paper's
// RaFI particle forwarding: emitOutgoing into per-destination buffers, then
// one all-to-all exchange, and a reduction of the particles left to decide
// whether another round runs; Sec. 3.1.2, Listing 2).
//
// Here the forwarding rides on the binning that already sorts a round's
// outgoing records by brick: with an ownership table the sort key of a brick
// this rank owns is its local index, and the key of any other brick is one
// export key per destination rank, so that after the sort the round's local
// queue comes first and each destination's records follow as one contiguous
// segment.  The exchange itself (NCCL or gloo all-to-all-v) and the
// termination reduction are the caller's (paper_2606_02627_gb300/pod.py):
// these calls only hand out and take in 32-byte particle records.
#include <vector>

#include "tracer.cuh"

using namespace sg;

extern "C" sg_status sg_tracer_pod_setup(sg_tracer *t, const int32_t *brick_owner, int32_t rank, int32_t world)
{
    SG_CHECK(t && brick_owner, SG_ERR_INVALID_ARG, "NULL argument");
    SG_CHECK(t->p.mode == SG_STREAMLINE, SG_ERR_UNSUPPORTED, "partition over data is for streamlines");
    SG_CHECK(t->p.kernel == SG_KERNEL_PERSISTENT || t->p.kernel == SG_KERNEL_LOCKSTEP, SG_ERR_UNSUPPORTED,
             "partition over data needs a persistent kernel");
    SG_CHECK(world >= 1 && world <= 64 && rank >= 0 && rank < world, SG_ERR_INVALID_ARG, "bad rank %d / world %d",
             rank, world);
    const int nb = t->nb;
    std::vector<int> key(nb);
    int local = 0;
    for (int b = 0; b < nb; ++b) {
        SG_CHECK(brick_owner[b] >= 0 && brick_owner[b] < world, SG_ERR_INVALID_ARG, "brick %d: owner %d out of range",
                 b, brick_owner[b]);
        if (brick_owner[b] == rank) key[b] = local++;
    }
    for (int b = 0; b < nb; ++b)
        if (brick_owner[b] != rank) key[b] = local + brick_owner[b];
    SG_CUDA(cudaSetDevice(t->ctx->device));
    SG_CUDA(cudaMemcpy(t->pod_key_map, key.data(), sizeof(int) * nb, cudaMemcpyHostToDevice));
    t->pod_world = world;
    t->pod_rank = rank;
    t->pod_local = local;
    for (int r = 0; r < 64; ++r) t->pod_export_start[r] = t->pod_export_count[r] = 0;
    t->graph_ready = false;              // the graph form is not used with a partition
    return SG_OK;
}

extern "C" sg_status sg_tracer_pod_begin(sg_tracer *t, int64_t *local_count, void *stream)
{
    SG_CHECK(t && t->pod_world > 0, SG_ERR_STATE, "sg_tracer_pod_setup first");
    SG_CUDA(cudaSetDevice(t->ctx->device));
    cudaStream_t s = (cudaStream_t)stream;
    t->horizon = (uint32_t)t->p.max_steps;
    sg_status st = launch_prepare_call(t, (uint32_t)t->p.max_steps, 0xffffffffu, s);
    if (st) return st;
    // every rank uploaded every seed: a seed in another rank's brick is that
    // rank's (its export segment is dropped here)
    st = launch_bin(t, t->park, &t->ctrl->p_count, s, false, 0ull, 0);
    if (st) return st;
    Ctrl c;
    SG_CUDA(cudaMemcpyAsync(&c, t->ctrl, sizeof c, cudaMemcpyDeviceToHost, s));
    SG_CUDA(cudaStreamSynchronize(s));
    for (int r = 0; r < 64; ++r) t->pod_export_count[r] = 0;
    t->pod_queued = c.q_count;
    t->scanned = false;
    if (local_count) *local_count = c.q_count;
    return SG_OK;
}

extern "C" sg_status sg_tracer_pod_round(sg_tracer *t, int64_t *local_count, int64_t *export_counts, void *stream)
{
    SG_CHECK(t && t->pod_world > 0, SG_ERR_STATE, "sg_tracer_pod_setup first");
    SG_CUDA(cudaSetDevice(t->ctx->device));
    cudaStream_t s = (cudaStream_t)stream;
    sg_status st = launch_round(t, s);
    if (st) return st;
    st = launch_bin(t, t->o, &t->ctrl->o_count, s, false, 0ull, 1);
    if (st) return st;
    const int W = t->pod_world;
    Ctrl c;
    uint32_t start[64], end[64];
    SG_CUDA(cudaMemcpyAsync(&c, t->ctrl, sizeof c, cudaMemcpyDeviceToHost, s));
    SG_CUDA(cudaMemcpyAsync(start, t->pod_key_start, sizeof(uint32_t) * W, cudaMemcpyDeviceToHost, s));
    SG_CUDA(cudaMemcpyAsync(end, t->brick_cursor + t->pod_local, sizeof(uint32_t) * W, cudaMemcpyDeviceToHost, s));
    SG_CUDA(cudaStreamSynchronize(s));
    if (c.err & CTRL_ERR_TIMEOUT) {
        set_error("a record copy of the advection kernel did not complete in time");
        return SG_ERR_TIMEOUT;
    }
    for (int r = 0; r < W; ++r) {
        t->pod_export_start[r] = start[r];
        t->pod_export_count[r] = r == t->pod_rank ? 0 : (int64_t)end[r] - (int64_t)start[r];
        if (export_counts) export_counts[r] = t->pod_export_count[r];
    }
    t->pod_queued = c.q_count;
    t->scanned = false;
    if (local_count) *local_count = c.q_count;
    return SG_OK;
}

extern "C" sg_status sg_tracer_pod_export(sg_tracer *t, int32_t dest, void *records, void *stream)
{
    SG_CHECK(t && t->pod_world > 0, SG_ERR_STATE, "sg_tracer_pod_setup first");
    SG_CHECK(dest >= 0 && dest < t->pod_world, SG_ERR_INVALID_ARG, "bad destination %d", dest);
    const int64_t n = t->pod_export_count[dest];
    if (n == 0) return SG_OK;
    SG_CHECK(records && pointer_kind(records) == PTR_DEVICE, SG_ERR_INVALID_ARG, "records must be device memory");
    SG_CUDA(cudaSetDevice(t->ctx->device));
    SG_CUDA(cudaMemcpyAsync(records, t->q + t->pod_export_start[dest], sizeof(Particle) * (size_t)n,
                            cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
    return SG_OK;
}

extern "C" sg_status sg_tracer_pod_import(sg_tracer *t, const void *records, int64_t count, void *stream)
{
    SG_CHECK(t && t->pod_world > 0, SG_ERR_STATE, "sg_tracer_pod_setup first");
    SG_CHECK(count >= 0, SG_ERR_INVALID_ARG, "negative count");
    if (count == 0) return SG_OK;
    SG_CHECK(records && pointer_kind(records) == PTR_DEVICE, SG_ERR_INVALID_ARG, "records must be device memory");
    SG_CHECK(t->pod_queued + count <= t->n_lines, SG_ERR_INVALID_ARG,
             "more particles than lines: %lld queued + %lld imported", (long long)t->pod_queued, (long long)count);
    SG_CUDA(cudaSetDevice(t->ctx->device));
    cudaStream_t s = (cudaStream_t)stream;
    // after this rank's exports were handed out: the imports join the local queue
    SG_CUDA(cudaMemcpyAsync(t->q + t->pod_queued, records, sizeof(Particle) * (size_t)count, cudaMemcpyDeviceToDevice,
                            s));
    t->pod_queued += count;
    for (int r = 0; r < 64; ++r) t->pod_export_count[r] = 0;
    return launch_set_q_count(t->ctrl, (uint32_t)t->pod_queued, s);
}

extern "C" sg_status sg_tracer_pod_queued(const sg_tracer *t, int64_t *count)
{
    SG_CHECK(t && count, SG_ERR_INVALID_ARG, "NULL argument");
    *count = t->pod_world > 0 ? t->pod_queued : 0;
    return SG_OK;
}

extern "C" sg_status sg_tracer_line_buffers(sg_tracer *t, float **slab, uint32_t **length, uint8_t **status,
                                            float **margin, int64_t *n_lines, int64_t *max_vertices)
{
    SG_CHECK(t != nullptr, SG_ERR_INVALID_ARG, "tracer is NULL");
    SG_CHECK(t->p.mode != SG_STREAKLINE, SG_ERR_UNSUPPORTED, "streaklines keep particles, not line slabs");
    if (slab) *slab = t->slab;
    if (length) *length = t->line_len;
    if (status) *status = t->line_status;
    if (margin) *margin = t->line_margin;
    if (n_lines) *n_lines = t->n_lines;
    if (max_vertices) *max_vertices = (int64_t)slab_stride(t->p.max_steps);
    t->scanned = false;                  // the caller may rewrite them (a merge across ranks)
    return SG_OK;
}
