// C ABI: errors, context, tracer (Tracer of Sec. 3.2 / Fig. 4).
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <string>
#include <vector>

#include "tracer.cuh"

namespace sg {

static thread_local std::string g_last_error;

void set_error(const char *fmt, ...)
{
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
}

sg_status cuda_error(cudaError_t e, const char *what)
{
    set_error("%s: %s (%s)", what, cudaGetErrorString(e), cudaGetErrorName(e));
    return SG_ERR_CUDA;
}

int pointer_kind(const void *p)
{
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return -1;
    }
    switch (a.type) {
    case cudaMemoryTypeDevice:
    case cudaMemoryTypeManaged: return PTR_DEVICE;
    case cudaMemoryTypeHost: return PTR_PINNED;
    default: return PTR_PAGEABLE;
    }
}

LineParams line_params(const sg_tracer *t)
{
    LineParams P;
    memset(&P, 0, sizeof P);
    const sg_field *f = t->field;
    P.F = field_view(f, 0);
    P.seeds = t->seeds;
    P.q = t->q;
    P.o = t->o;
    P.park = t->park;
    P.ctrl = t->ctrl;
    P.slab = t->slab;
    P.line_len = t->line_len;
    P.line_status = t->line_status;
    P.line_margin = t->line_margin;
    P.W = slab_stride(t->p.max_steps);
    P.n_lines = t->n_lines;
    P.n_seed = t->n_seeds;
    P.n_fwd = t->p.direction == SG_DIR_FORWARD ? t->n_lines : (t->p.direction == SG_DIR_BACKWARD ? 0 : t->n_seeds);
    for (int a = 0; a < 3; ++a) {
        P.dtc[a] = (float)(t->p.dt / f->desc.spacing[a]);
        P.origin_d[a] = f->desc.origin[a];
        P.spacing_d[a] = f->desc.spacing[a];
    }
    P.eps = t->p.eps;
    P.tie_cells = t->p.tie_cells;
    P.tie_eps_rel = t->p.tie_eps_rel;
    P.max_steps = (uint32_t)t->p.max_steps;
    P.steps_per_round = (uint32_t)t->p.steps_per_round;
    P.drain_steps = (uint32_t)t->p.drain_steps;
    return P;
}

}  // namespace sg

using namespace sg;

extern "C" size_t sg_last_error(char *buf, size_t n)
{
    const std::string &s = g_last_error;
    if (buf && n) {
        size_t k = s.size() < n - 1 ? s.size() : n - 1;
        memcpy(buf, s.data(), k);
        buf[k] = 0;
    }
    return s.size();
}

extern "C" int32_t sg_version(void) { return 100; }

// ------------------------------------------------------------------ context

extern "C" sg_status sg_context_create(int32_t device, sg_context **out)
{
    SG_CHECK(out != nullptr, SG_ERR_INVALID_ARG, "out is NULL");
    int count = 0;
    SG_CUDA(cudaGetDeviceCount(&count));
    SG_CHECK(device >= 0 && device < count, SG_ERR_INVALID_ARG, "device %d out of range (%d devices)", device, count);
    SG_CUDA(cudaSetDevice(device));
    cudaDeviceProp prop;
    SG_CUDA(cudaGetDeviceProperties(&prop, device));
    sg_context *c = new sg_context;
    c->device = device;
    c->sm_count = prop.multiProcessorCount;
    c->max_threads_per_sm = prop.maxThreadsPerMultiProcessor;
    c->max_smem_optin = (int)prop.sharedMemPerBlockOptin;
    c->l2_bytes = prop.l2CacheSize;
    *out = c;
    return SG_OK;
}

extern "C" sg_status sg_context_destroy(sg_context *ctx)
{
    delete ctx;
    return SG_OK;
}

extern "C" sg_status sg_context_sm_count(const sg_context *ctx, int32_t *out)
{
    SG_CHECK(ctx && out, SG_ERR_INVALID_ARG, "NULL argument");
    *out = ctx->sm_count;
    return SG_OK;
}

// ------------------------------------------------------------------ tracer

extern "C" sg_status sg_tracer_params_default(sg_tracer_params *p)
{
    SG_CHECK(p != nullptr, SG_ERR_INVALID_ARG, "NULL argument");
    memset(p, 0, sizeof *p);
    p->mode = SG_STREAMLINE;
    p->kernel = SG_KERNEL_PERSISTENT;
    p->dt = 0.0;
    p->max_steps = 1000;
    p->eps = 1e-6f;
    p->tie_cells = 1e-3f;
    p->tie_eps_rel = 1e-3f;
    p->inject_steps = 1;
    return SG_OK;
}

static sg_status check_params(const sg_field *f, const sg_tracer_params *p)
{
    SG_CHECK(p->mode == SG_STREAMLINE || p->mode == SG_STREAKLINE || p->mode == SG_PATHLINE, SG_ERR_INVALID_ARG,
             "bad mode %d", p->mode);
    SG_CHECK(p->dt > 0.0 && p->dt < 1e30, SG_ERR_INVALID_ARG, "dt must be > 0");
    SG_CHECK(p->eps >= 0.0f, SG_ERR_INVALID_ARG, "eps must be >= 0");
    // every streamline kernel is built for at most 256 threads per CTA (its
    // register budget): a larger block would fail at launch, inside the
    // capture of the round loop's graph
    SG_CHECK(p->block_size >= 0 && p->block_size <= 256 && p->block_size % 32 == 0, SG_ERR_INVALID_ARG,
             "block_size must be a multiple of 32 in [0, 256]");
    SG_CHECK(p->blocks_per_sm >= 0 && p->blocks_per_sm <= 32, SG_ERR_INVALID_ARG, "blocks_per_sm in [0, 32]");
    SG_CHECK(p->steps_per_round >= 0, SG_ERR_INVALID_ARG, "steps_per_round must be >= 0");
    SG_CHECK(p->max_rounds >= 0, SG_ERR_INVALID_ARG, "max_rounds must be >= 0");
    SG_CHECK(p->brick_window >= 0, SG_ERR_INVALID_ARG, "brick_window must be >= 0");
    SG_CHECK(p->direction >= SG_DIR_FORWARD && p->direction <= SG_DIR_BOTH, SG_ERR_INVALID_ARG, "bad direction %d",
             p->direction);
    if (p->mode == SG_STREAMLINE) {
        SG_CHECK(p->max_steps >= 0 && p->max_steps < (1 << 27), SG_ERR_INVALID_ARG, "max_steps out of range");
        SG_CHECK(p->kernel == SG_KERNEL_PERSISTENT || p->kernel == SG_KERNEL_PER_SEED ||
                     p->kernel == SG_KERNEL_PER_STEP || p->kernel == SG_KERNEL_LOCKSTEP,
                 SG_ERR_INVALID_ARG, "bad kernel %d", p->kernel);
        if (p->kernel == SG_KERNEL_PER_SEED)
            SG_CHECK(f->desc.layout == SG_FIELD_GLOBAL, SG_ERR_UNSUPPORTED,
                     "the per-seed kernel samples the global float3 layout");
        else
            SG_CHECK(f->desc.layout != SG_FIELD_GLOBAL, SG_ERR_UNSUPPORTED, "this kernel samples a bricked field");
    } else if (p->mode == SG_PATHLINE) {
        SG_CHECK(p->direction == SG_DIR_FORWARD, SG_ERR_UNSUPPORTED, "path lines advance forward in time");
        SG_CHECK(p->max_steps >= 0 && p->max_steps < (1 << 27), SG_ERR_INVALID_ARG, "max_steps out of range");
        SG_CHECK(f->desc.n_slots >= 2, SG_ERR_INVALID_ARG, "path lines need a field with >= 2 slots");
        SG_CHECK(f->desc.layout != SG_FIELD_GLOBAL, SG_ERR_UNSUPPORTED, "path lines sample a bricked field");
    } else {
        SG_CHECK(p->direction == SG_DIR_FORWARD, SG_ERR_UNSUPPORTED, "streaklines advance forward in time");
        SG_CHECK(p->inject_steps >= 1, SG_ERR_INVALID_ARG, "inject_steps must be >= 1");
        SG_CHECK(f->desc.n_slots >= 2, SG_ERR_INVALID_ARG, "streaklines need a field with >= 2 slots");
        SG_CHECK(f->desc.layout != SG_FIELD_GLOBAL, SG_ERR_UNSUPPORTED, "streaklines sample a bricked field");
    }
    return SG_OK;
}

// Carves the tracer's buffers; with t == NULL only the size is computed.
static size_t tracer_layout(const sg_field *f, const sg_tracer_params *p, int64_t cap, sg_tracer *t, char *base)
{
    Carve c{base, 0, 0};
    const int nb = f->nb;
    if (p->mode == SG_STREAMLINE || p->mode == SG_PATHLINE) {
        const long long W = slab_stride(p->max_steps);
        const int64_t lc = cap * (p->direction == SG_DIR_BOTH ? 2 : 1);   // line slots
        float *seeds = (float *)c.take(sizeof(float) * 3 * cap);
        float *slab = (float *)c.take(sizeof(float) * 3 * (size_t)W * lc);
        uint32_t *len = (uint32_t *)c.take(sizeof(uint32_t) * lc);
        uint8_t *st = (uint8_t *)c.take(lc);
        float *mg = (float *)c.take(sizeof(float) * lc);
        Particle *q = nullptr, *o = nullptr, *pk = nullptr;
        if (p->kernel != SG_KERNEL_PER_SEED || p->mode == SG_PATHLINE) {
            q = (Particle *)c.take(sizeof(Particle) * lc);
            o = (Particle *)c.take(sizeof(Particle) * lc);
            pk = (Particle *)c.take(sizeof(Particle) * lc);
        }
        Ctrl *ctrl = (Ctrl *)c.take(sizeof(Ctrl));
        // binning keys: the bricks, or (partition over data) the local bricks
        // plus one export key per rank (at most 64 ranks)
        uint32_t *bc = (uint32_t *)c.take(sizeof(uint32_t) * (nb + 64));
        uint32_t *bcur = (uint32_t *)c.take(sizeof(uint32_t) * (nb + 64));
        int *kmap = (int *)c.take(sizeof(int) * nb);
        uint32_t *kstart = (uint32_t *)c.take(sizeof(uint32_t) * 64);
        int64_t *off = (int64_t *)c.take(sizeof(int64_t) * (lc + 1));
        unsigned long long *bs = (unsigned long long *)c.take(sizeof(unsigned long long) * (lc / 4096 + 2));
        int64_t *tot = (int64_t *)c.take(sizeof(int64_t) * 4);
        uint32_t *jlen = nullptr;
        int64_t *joff = nullptr, *jtot = nullptr;
        if (p->direction == SG_DIR_BOTH) {
            jlen = (uint32_t *)c.take(sizeof(uint32_t) * cap);
            joff = (int64_t *)c.take(sizeof(int64_t) * (cap + 1));
            jtot = (int64_t *)c.take(sizeof(int64_t) * 4);
        }
        // two staging buffers for readback into host memory, each at least one line
        size_t stage = (size_t)256 << 20;
        const size_t line_bytes = sizeof(float) * 3 * (size_t)W;
        if (stage < line_bytes) stage = line_bytes;
        const size_t slab_bytes = sizeof(float) * 3 * (size_t)W * lc;
        if (stage > slab_bytes) stage = slab_bytes > line_bytes ? slab_bytes : line_bytes;
        stage = align_up(stage, 256);
        float *st0 = (float *)c.take(stage);
        float *st1 = (float *)c.take(stage);
        if (t) {
            t->staging[0] = st0;
            t->staging[1] = st1;
            t->staging_bytes = stage;
            t->seeds = seeds;
            t->slab = slab;
            t->line_len = len;
            t->line_status = st;
            t->line_margin = mg;
            t->q = q;
            t->o = o;
            t->park = pk;
            t->ctrl = ctrl;
            t->brick_count = bc;
            t->brick_cursor = bcur;
            t->pod_key_map = kmap;
            t->pod_key_start = kstart;
            t->offsets = off;
            t->block_sums = bs;
            t->totals = tot;
            t->join_len = jlen;
            t->join_off = joff;
            t->join_tot = jtot;
        }
    } else {
        const long long inj = p->inject_steps;
        float *seeds = (float *)c.take(sizeof(float) * 3 * cap);
        Particle *state = (Particle *)c.take(sizeof(Particle) * cap * inj);
        uint8_t *st = (uint8_t *)c.take((size_t)cap * inj);
        float *mg = (float *)c.take(sizeof(float) * cap * inj);
        uint32_t *seg = (uint32_t *)c.take(sizeof(uint32_t) * cap * inj);
        int64_t *off = (int64_t *)c.take(sizeof(int64_t) * (cap * inj + 1));
        unsigned long long *bs = (unsigned long long *)c.take(sizeof(unsigned long long) * (cap + 2));
        int64_t *tot = (int64_t *)c.take(sizeof(int64_t) * 4);
        if (t) {
            t->seeds = seeds;
            t->sk_state = state;
            t->sk_status = st;
            t->sk_margin = mg;
            t->sk_seglen = seg;
            t->offsets = off;
            t->block_sums = bs;
            t->totals = tot;
        }
    }
    return c.off;
}

extern "C" sg_status sg_tracer_required_bytes(const sg_context *ctx, const sg_field *f, const sg_tracer_params *p,
                                              int64_t capacity, size_t *bytes)
{
    SG_CHECK(ctx && f && p && bytes, SG_ERR_INVALID_ARG, "NULL argument");
    SG_CHECK(capacity >= 0 && capacity < (1ll << 32), SG_ERR_INVALID_ARG, "capacity out of range");
    sg_status st = check_params(f, p);
    if (st) return st;
    *bytes = tracer_layout(f, p, capacity, nullptr, nullptr);
    return SG_OK;
}

extern "C" sg_status sg_tracer_create(sg_context *ctx, sg_field *f, const sg_tracer_params *p, int64_t capacity,
                                      void *workspace, size_t bytes, sg_tracer **out)
{
    SG_CHECK(ctx && f && p && out, SG_ERR_INVALID_ARG, "NULL argument");
    SG_CHECK(workspace != nullptr && ((uintptr_t)workspace & 255) == 0, SG_ERR_INVALID_ARG,
             "workspace must be non-NULL and 256-byte aligned");
    SG_CHECK(capacity >= 0 && capacity < (1ll << 32), SG_ERR_INVALID_ARG, "capacity out of range");
    sg_status st = check_params(f, p);
    if (st) return st;
    const size_t need = tracer_layout(f, p, capacity, nullptr, nullptr);
    SG_CHECK(bytes >= need, SG_ERR_OOM, "tracer needs %zu bytes, got %zu", need, bytes);
    SG_CHECK(pointer_kind(workspace) == PTR_DEVICE, SG_ERR_INVALID_ARG, "workspace must be device memory");
    SG_CUDA(cudaSetDevice(ctx->device));
    sg_tracer *t = new sg_tracer;
    memset(t, 0, sizeof *t);
    t->ctx = ctx;
    t->field = f;
    t->p = *p;
    t->capacity = capacity;
    t->line_mult = (p->mode == SG_STREAMLINE && p->direction == SG_DIR_BOTH) ? 2 : 1;
    t->ws = (char *)workspace;
    t->ws_bytes = bytes;
    t->nb = f->nb;
    tracer_layout(f, p, capacity, t, (char *)workspace);
    t->block = p->block_size > 0 ? p->block_size : 256;
    // default resident threads per SM (measured on GB300): 512 for the kernels
    // that read every sample through L1, where more particles per SM thrash the
    // L1 that holds their cell records; 768 for the decoupled-lane kernel,
    // whose records sit in shared memory and which is built for 3 CTAs of 256
    // threads per SM (up to 85 registers: at 64 registers, for 1024 threads,
    // the FP32 form spills and ran 13 % slower)
    const bool decoupled = decoupled_lanes(p, f);
    const int threads_per_sm = decoupled ? 768 : 512;
    // round length (measured on GB300): with many more particles than resident
    // lanes the decoupled kernel gains from long rounds whose ends are cut
    // short once the queue is empty (1024 steps: +2 % over 256 for FP32 on
    // 512^3, 1M seeds, 2000 steps); with few, the shorter rounds spread the
    // particles over more warps at each re-binning (1024 seeds on a 64^3
    // brick: 256 steps 12 % faster than 1024)
    const long long resident = (long long)ctx->sm_count * threads_per_sm;
    if (t->p.steps_per_round <= 0)
        t->p.steps_per_round = decoupled ? (capacity >= 4 * resident ? 1024 : 256) : 128;
    if (t->p.drain_steps == 0) t->p.drain_steps = decoupled ? 128 : 0x7fffffff;
    else if (t->p.drain_steps < 0) t->p.drain_steps = 0x7fffffff;
    const int per_sm = p->blocks_per_sm > 0 ? p->blocks_per_sm : (threads_per_sm + t->block - 1) / t->block;
    t->grid = ctx->sm_count * (per_sm > 0 ? per_sm : 1);
    if (t->p.mode == SG_STREAMLINE) {
        sg_status pst = prepare_round(t);
        if (pst) {
            delete t;
            return pst;
        }
    }
    if (t->p.mode != SG_STREAKLINE) {
        cudaError_t ce = cudaStreamCreateWithFlags(&t->copy_stream, cudaStreamNonBlocking);
        for (int k = 0; k < 2 && ce == cudaSuccess; ++k) {
            ce = cudaEventCreateWithFlags(&t->ev_gathered[k], cudaEventDisableTiming);
            if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&t->ev_copied[k], cudaEventDisableTiming);
        }
        if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&t->ev_ovl_gathered, cudaEventDisableTiming);
        for (int k = 0; k < 2 && ce == cudaSuccess; ++k) {
            ce = cudaEventCreateWithFlags(&t->ev_ovl_copied[k], cudaEventDisableTiming);
            if (ce == cudaSuccess) ce = cudaEventRecord(t->ev_ovl_copied[k], t->copy_stream);
        }
        if (ce != cudaSuccess) {
            sg_tracer_destroy(t);
            return cuda_error(ce, "readback stream");
        }
    }
    cudaError_t e = cudaMemset(t->ctrl ? (void *)t->ctrl : (void *)t->totals, 0,
                               t->ctrl ? sizeof(Ctrl) : sizeof(int64_t) * 4);
    if (e == cudaSuccess && t->brick_count) e = cudaMemset(t->brick_count, 0, sizeof(uint32_t) * (t->nb + 64));
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        delete t;
        return cuda_error(e, "tracer init");
    }
    *out = t;
    return SG_OK;
}

extern "C" sg_status sg_tracer_destroy(sg_tracer *t)
{
    if (!t) return SG_OK;
    if (t->exec) cudaGraphExecDestroy(t->exec);
    if (t->graph) cudaGraphDestroy(t->graph);
    for (int k = 0; k < 2; ++k) {
        if (t->ev_gathered[k]) cudaEventDestroy(t->ev_gathered[k]);
        if (t->ev_copied[k]) cudaEventDestroy(t->ev_copied[k]);
    }
    for (int k = 0; k < 2; ++k) {
        if (t->ovl_buf[k]) {
            if (t->ev_ovl_copied[k]) cudaEventSynchronize(t->ev_ovl_copied[k]);
            cudaFree(t->ovl_buf[k]);
        }
        if (t->ev_ovl_copied[k]) cudaEventDestroy(t->ev_ovl_copied[k]);
    }
    if (t->ev_ovl_gathered) cudaEventDestroy(t->ev_ovl_gathered);
    if (t->copy_stream) cudaStreamDestroy(t->copy_stream);
    delete t;
    return SG_OK;
}

extern "C" sg_status sg_tracer_upload_seeds(sg_tracer *t, const float *xyz, int64_t n, void *stream)
{
    SG_CHECK(t != nullptr, SG_ERR_INVALID_ARG, "tracer is NULL");
    SG_CHECK(n >= 0 && n <= t->capacity, SG_ERR_INVALID_ARG, "n = %lld exceeds capacity %lld", (long long)n,
             (long long)t->capacity);
    SG_CHECK(n == 0 || xyz != nullptr, SG_ERR_INVALID_ARG, "xyz is NULL");
    SG_CUDA(cudaSetDevice(t->ctx->device));
    cudaStream_t s = (cudaStream_t)stream;
    if (n > 0) {
        const int k = pointer_kind(xyz);
        SG_CHECK(k >= 0, SG_ERR_INVALID_ARG, "cannot classify the seed pointer");
        SG_CUDA(cudaMemcpyAsync(t->seeds, xyz, sizeof(float) * 3 * (size_t)n, cudaMemcpyDefault, s));
    }
    t->n_seeds = n;
    t->n_lines = n * t->line_mult;
    t->scanned = false;
    t->traced = false;
    t->horizon = 0;
    if (t->p.mode == SG_STREAKLINE) return streak_upload(t, s);
    if (t->p.mode == SG_PATHLINE) return path_upload(t, s);
    if (t->ctrl) SG_CUDA(cudaMemsetAsync(t->ctrl, 0, sizeof(Ctrl), s));
    if (t->pod_world > 0) {
        // every rank's slab starts at +inf so that the ranks' partial lines
        // merge by an elementwise minimum (each vertex written by one rank)
        sg_status st = launch_fill_inf(t->slab, 3 * slab_stride(t->p.max_steps) * t->n_lines, s);
        if (st) return st;
    }
    return launch_upload(t, s);
}

// Builds the CUDA graph of one call: bin the parked particles, then a while
// node whose body is one round plus the binning of its outgoing records.
static sg_status build_graph(sg_tracer *t)
{
    cudaStream_t cs;
    SG_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaGraph_t g = nullptr;
    cudaGraphConditionalHandle h;
    sg_status st = SG_OK;
    cudaError_t e = cudaGraphCreate(&g, 0);
    if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&h, g, 0, 0);
    if (e == cudaSuccess) e = cudaStreamBeginCaptureToGraph(cs, g, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
        st = cuda_error(e, "graph setup");
    } else {
        st = launch_bin(t, t->park, &t->ctrl->p_count, cs, true, (unsigned long long)h, 0);
        cudaStreamCaptureStatus cst;
        const cudaGraphNode_t *deps = nullptr;
        size_t ndeps = 0;
        cudaGraphNode_t cond = nullptr;
        cudaGraphNodeParams cp = {};
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = h;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        if (st == SG_OK) {
            e = cudaStreamGetCaptureInfo(cs, &cst, nullptr, nullptr, &deps, nullptr, &ndeps);
            if (e == cudaSuccess) e = cudaGraphAddNode(&cond, g, deps, nullptr, ndeps, &cp);
            if (e == cudaSuccess) e = cudaStreamUpdateCaptureDependencies(cs, &cond, nullptr, 1, cudaStreamSetCaptureDependencies);
            if (e != cudaSuccess) st = cuda_error(e, "conditional node");
        }
        if (st == SG_OK) st = launch_park_rest(t, cs);
        cudaGraph_t g2 = nullptr;
        cudaError_t e2 = cudaStreamEndCapture(cs, &g2);
        if (st == SG_OK && e2 != cudaSuccess) st = cuda_error(e2, "cudaStreamEndCapture");
        if (st == SG_OK) {
            cudaGraph_t body = cp.conditional.phGraph_out[0];
            e = cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
            if (e != cudaSuccess) {
                st = cuda_error(e, "body capture");
            } else {
                st = launch_round(t, cs);
                if (st == SG_OK) st = launch_carry(t, cs);
                if (st == SG_OK) st = launch_bin(t, t->o, &t->ctrl->o_count, cs, true, (unsigned long long)h, 1);
                cudaGraph_t b2 = nullptr;
                e2 = cudaStreamEndCapture(cs, &b2);
                if (st == SG_OK && e2 != cudaSuccess) st = cuda_error(e2, "body end capture");
            }
        }
        if (st == SG_OK) {
            e = cudaGraphInstantiate(&t->exec, g, 0);
            if (e != cudaSuccess) st = cuda_error(e, "cudaGraphInstantiate");
        }
    }
    cudaStreamDestroy(cs);
    if (st != SG_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    t->graph = g;
    t->graph_ready = true;
    return SG_OK;
}

// Round cap of a call that advances particles up to `horizon` steps: every
// round advances each particle of its brick window by at least one step, no
// particle starts a call below step 0 (a call that the round cap stopped
// leaves particles behind the horizon), and a sweep over the bricks takes
// ceil(bricks / window) rounds, so (horizon + 2) sweeps finish a call; the cap
// only guards against a fault unless the caller sets max_rounds.
static uint64_t round_guard(const sg_tracer *t, uint32_t horizon)
{
    const uint64_t w = (uint64_t)(t->p.brick_window > 0 ? t->p.brick_window : t->nb);
    const uint64_t sweeps = ((uint64_t)t->nb + w - 1) / w;
    return ((uint64_t)horizon + 2) * (sweeps > 0 ? sweeps : 1);
}

static sg_status run_call(sg_tracer *t, uint32_t horizon, uint32_t n_steps, cudaStream_t s)
{
    if (!t->graph_ready) {
        sg_status st = build_graph(t);
        if (st) return st;
    }
    (void)n_steps;
    uint64_t cap = round_guard(t, horizon);
    if (t->p.max_rounds > 0 && (uint64_t)t->p.max_rounds < cap) cap = (uint64_t)t->p.max_rounds;
    if (cap > 0xffffffffull) cap = 0xffffffffull;
    sg_status st = launch_prepare_call(t, horizon, (uint32_t)cap, s);
    if (st) return st;
    SG_CUDA(cudaGraphLaunch(t->exec, s));
    t->scanned = false;
    return SG_OK;
}

extern "C" sg_status sg_tracer_trace(sg_tracer *t, void *stream)
{
    SG_CHECK(t != nullptr, SG_ERR_INVALID_ARG, "tracer is NULL");
    SG_CHECK(t->p.mode == SG_STREAMLINE, SG_ERR_STATE, "trace() is for streamlines; streak and path lines use step()");
    SG_CHECK(t->pod_world == 0, SG_ERR_STATE, "a partitioned tracer advances with the sg_tracer_pod_* calls");
    SG_CUDA(cudaSetDevice(t->ctx->device));
    cudaStream_t s = (cudaStream_t)stream;
    if (t->n_seeds == 0) return SG_OK;
    if (t->p.kernel == SG_KERNEL_PER_SEED) {
        SG_CHECK(!t->traced, SG_ERR_STATE, "the per-seed kernel traces once per upload");
        sg_status st = launch_per_seed(t, s);
        if (st) return st;
        t->traced = true;
        t->scanned = false;
        return SG_OK;
    }
    const uint32_t target = (uint32_t)t->p.max_steps;
    const uint32_t n = target > t->horizon ? target - t->horizon : 0;
    t->horizon = target;
    return run_call(t, target, n, s);
}

extern "C" sg_status sg_tracer_trace_timed(sg_tracer *t, double *kernel_ms, int32_t *launches, float *round_ms,
                                           uint32_t *round_particles, int32_t max_records, void *stream)
{
    SG_CHECK(t != nullptr, SG_ERR_INVALID_ARG, "tracer is NULL");
    SG_CHECK(t->p.mode == SG_STREAMLINE, SG_ERR_STATE, "trace() is for streamlines");
    SG_CHECK(t->pod_world == 0, SG_ERR_STATE, "a partitioned tracer advances with the sg_tracer_pod_* calls");
    SG_CUDA(cudaSetDevice(t->ctx->device));
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t e0, e1;
    SG_CUDA(cudaEventCreate(&e0));
    cudaError_t ce = cudaEventCreate(&e1);
    if (ce != cudaSuccess) {
        cudaEventDestroy(e0);
        return cuda_error(ce, "cudaEventCreate");
    }
    double total = 0.0;
    int32_t n_launch = 0;
    sg_status st = SG_OK;
    if (t->n_seeds > 0 && t->p.kernel == SG_KERNEL_PER_SEED) {
        if (t->traced) {
            set_error("the per-seed kernel traces once per upload");
            st = SG_ERR_STATE;
        }
        if (st == SG_OK && (ce = cudaEventRecord(e0, s)) != cudaSuccess) st = cuda_error(ce, "cudaEventRecord");
        if (st == SG_OK) st = launch_per_seed(t, s);
        if (st == SG_OK && (ce = cudaEventRecord(e1, s)) != cudaSuccess) st = cuda_error(ce, "cudaEventRecord");
        if (st == SG_OK && (ce = cudaEventSynchronize(e1)) != cudaSuccess) st = cuda_error(ce, "cudaEventSynchronize");
        float ms = 0.f;
        if (st == SG_OK && (ce = cudaEventElapsedTime(&ms, e0, e1)) != cudaSuccess) st = cuda_error(ce, "elapsed");
        total = ms;
        n_launch = 1;
        t->traced = true;
        t->scanned = false;
    } else if (t->n_seeds > 0) {
        const uint32_t target = (uint32_t)t->p.max_steps;
        const uint32_t n = target > t->horizon ? target - t->horizon : 0;
        t->horizon = target;
        (void)n;
        uint64_t cap = round_guard(t, target);
        if (t->p.max_rounds > 0 && (uint64_t)t->p.max_rounds < cap) cap = (uint64_t)t->p.max_rounds;
        if (cap > 0xffffffffull) cap = 0xffffffffull;
        st = launch_prepare_call(t, target, (uint32_t)cap, s);
        if (st == SG_OK) st = launch_bin(t, t->park, &t->ctrl->p_count, s, false, 0ull, 0);
        Ctrl c;
        while (st == SG_OK) {
            if ((ce = cudaMemcpyAsync(&c, t->ctrl, sizeof c, cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
                (ce = cudaStreamSynchronize(s)) != cudaSuccess) {
                st = cuda_error(ce, "ctrl readback");
                break;
            }
            if (c.q_count == 0 || c.round >= c.max_rounds) break;
            if ((ce = cudaEventRecord(e0, s)) != cudaSuccess) { st = cuda_error(ce, "cudaEventRecord"); break; }
            st = launch_round(t, s);
            if (st) break;
            if ((ce = cudaEventRecord(e1, s)) != cudaSuccess) { st = cuda_error(ce, "cudaEventRecord"); break; }
            st = launch_carry(t, s);
            if (st) break;
            st = launch_bin(t, t->o, &t->ctrl->o_count, s, false, 0ull, 1);
            if (st) break;
            if ((ce = cudaEventSynchronize(e1)) != cudaSuccess) { st = cuda_error(ce, "cudaEventSynchronize"); break; }
            float ms = 0.f;
            if ((ce = cudaEventElapsedTime(&ms, e0, e1)) != cudaSuccess) { st = cuda_error(ce, "elapsed"); break; }
            total += ms;
            if (round_ms && round_particles && n_launch < max_records) {
                round_ms[n_launch] = ms;
                round_particles[n_launch] = c.q_count - c.win_start;
            }
            ++n_launch;
        }
        t->scanned = false;
        if (st == SG_OK) st = launch_park_rest(t, s);
        if (st == SG_OK && c.q_count > 0) {
            set_error("the round cap stopped the trace with particles left");
            st = SG_ERR_ROUND_LIMIT;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (kernel_ms) *kernel_ms = total;
    if (launches) *launches = n_launch;
    return st;
}

extern "C" sg_status sg_tracer_step(sg_tracer *t, int32_t n_steps, int32_t *any_active, void *stream)
{
    SG_CHECK(t != nullptr, SG_ERR_INVALID_ARG, "tracer is NULL");
    SG_CHECK(n_steps >= 0, SG_ERR_INVALID_ARG, "n_steps must be >= 0");
    SG_CUDA(cudaSetDevice(t->ctx->device));
    cudaStream_t s = (cudaStream_t)stream;
    if (t->p.mode == SG_STREAKLINE) return streak_step(t, n_steps, any_active, s);
    if (t->p.mode == SG_PATHLINE) return path_step(t, n_steps, any_active, s);
    SG_CHECK(t->pod_world == 0, SG_ERR_STATE, "a partitioned tracer advances with the sg_tracer_pod_* calls");
    SG_CHECK(t->p.kernel != SG_KERNEL_PER_SEED, SG_ERR_UNSUPPORTED, "the per-seed kernel only traces to the end");
    uint64_t target = (uint64_t)t->horizon + (uint64_t)n_steps;
    if (target > (uint64_t)t->p.max_steps) target = (uint64_t)t->p.max_steps;
    const uint32_t n = (uint32_t)(target - t->horizon);
    t->horizon = (uint32_t)target;
    if (t->n_seeds > 0) {
        sg_status st = run_call(t, (uint32_t)target, n, s);
        if (st) return st;
    }
    if (any_active) {
        Ctrl c;
        SG_CUDA(cudaMemcpyAsync(&c, t->ctrl, sizeof c, cudaMemcpyDeviceToHost, s));
        SG_CUDA(cudaStreamSynchronize(s));
        *any_active = (t->n_seeds > 0 && c.p_count > 0) ? 1 : 0;
        if (c.err & CTRL_ERR_TIMEOUT) {
            set_error("a record copy of the advection kernel did not complete in time");
            return SG_ERR_TIMEOUT;
        }
        if (c.err & CTRL_ERR_ROUND_LIMIT) {
            set_error("the round cap stopped the call with particles left");
            return SG_ERR_ROUND_LIMIT;
        }
    }
    return SG_OK;
}

extern "C" sg_status sg_tracer_check(sg_tracer *t, int32_t *rounds, void *stream)
{
    SG_CHECK(t != nullptr, SG_ERR_INVALID_ARG, "tracer is NULL");
    SG_CUDA(cudaSetDevice(t->ctx->device));
    cudaStream_t s = (cudaStream_t)stream;
    if (!t->ctrl) {
        SG_CUDA(cudaStreamSynchronize(s));
        if (rounds) *rounds = 1;
        return SG_OK;
    }
    Ctrl c;
    SG_CUDA(cudaMemcpyAsync(&c, t->ctrl, sizeof c, cudaMemcpyDeviceToHost, s));
    SG_CUDA(cudaStreamSynchronize(s));
    if (rounds) *rounds = (int32_t)c.last_rounds;
    if (c.err & CTRL_ERR_TIMEOUT) {
        set_error("a record copy of the advection kernel did not complete in time");
        return SG_ERR_TIMEOUT;
    }
    if (c.err & CTRL_ERR_ROUND_LIMIT) {
        set_error("the round cap stopped the trace with particles left");
        return SG_ERR_ROUND_LIMIT;
    }
    return SG_OK;
}

static sg_status ensure_scanned(sg_tracer *t, cudaStream_t s)
{
    if (t->scanned) return SG_OK;
    sg_status st;
    if (t->p.mode == SG_STREAKLINE) st = launch_streak_scan(t, s);
    else st = launch_scan_lengths(t, s);
    if (st) return st;
    t->scanned = true;
    return SG_OK;
}

static sg_status read_totals(sg_tracer *t, int64_t out[3], cudaStream_t s)
{
    int64_t h[4];
    SG_CUDA(cudaMemcpyAsync(h, t->totals, sizeof h, cudaMemcpyDeviceToHost, s));
    SG_CUDA(cudaStreamSynchronize(s));
    out[0] = h[0];
    out[1] = h[1];
    out[2] = h[2];
    return SG_OK;
}

static sg_status check_out_ptr(const void *p, const char *what)
{
    if (!p) return SG_OK;
    const int k = pointer_kind(p);
    SG_CHECK(k == PTR_DEVICE || k == PTR_PINNED, SG_ERR_INVALID_ARG,
             "%s must be device or page-locked host memory", what);
    return SG_OK;
}

extern "C" sg_status sg_tracer_get_lines(sg_tracer *t, int64_t *n_lines, int64_t *n_vertices, int64_t *offsets,
                                         float *vertices, uint8_t *status, float *margin, int32_t *line_source,
                                         void *stream)
{
    SG_CHECK(t != nullptr, SG_ERR_INVALID_ARG, "tracer is NULL");
    SG_CUDA(cudaSetDevice(t->ctx->device));
    cudaStream_t s = (cudaStream_t)stream;
    sg_status st = ensure_scanned(t, s);
    if (st) return st;
    const bool query = !offsets && !vertices && !status && !margin && !line_source;
    if (query || n_lines || n_vertices) {
        int64_t tot[3];
        st = read_totals(t, tot, s);
        if (st) return st;
        if (n_lines) *n_lines = tot[1];
        if (n_vertices) *n_vertices = tot[0];
        if (query) return SG_OK;
    }
    if ((st = check_out_ptr(offsets, "offsets")) || (st = check_out_ptr(vertices, "vertices")) ||
        (st = check_out_ptr(status, "status")) || (st = check_out_ptr(margin, "margin")) ||
        (st = check_out_ptr(line_source, "line_source")))
        return st;
    if (t->p.mode == SG_STREAKLINE) return launch_streak_gather(t, offsets, vertices, status, margin, line_source, s);
    if (line_source && t->n_lines > 0) {
        st = launch_iota(line_source, t->n_lines, t->n_seeds, s);
        if (st) return st;
    }
    if (vertices && pointer_kind(vertices) == PTR_PINNED && t->n_lines > 0) {
        // host destination: gather chunks of lines into device staging buffers
        // and copy each to the host on the copy stream, overlapping the next
        // chunk's gather (DMA copies beat kernel stores over the host link)
        st = launch_gather_lines(t, offsets, nullptr, status, margin, s);
        if (st) return st;
        std::vector<int64_t> off((size_t)t->n_lines + 1);
        SG_CUDA(cudaMemcpyAsync(off.data(), t->offsets, sizeof(int64_t) * off.size(), cudaMemcpyDeviceToHost, s));
        SG_CUDA(cudaStreamSynchronize(s));
        const long long cap_v = (long long)(t->staging_bytes / (3 * sizeof(float)));
        long long a = 0;
        int k = 0;
        while (a < t->n_lines) {
            long long b = a + 1;
            while (b < t->n_lines && off[b + 1] - off[a] <= cap_v) ++b;
            const int buf = k & 1;
            SG_CUDA(cudaStreamWaitEvent(s, t->ev_copied[buf], 0));          // the buffer's last copy is done
            st = launch_gather_chunk(t, a, b, off[a], t->staging[buf], s);
            if (st) return st;
            SG_CUDA(cudaEventRecord(t->ev_gathered[buf], s));
            SG_CUDA(cudaStreamWaitEvent(t->copy_stream, t->ev_gathered[buf], 0));
            const size_t bytes = sizeof(float) * 3 * (size_t)(off[b] - off[a]);
            if (bytes)
                SG_CUDA(cudaMemcpyAsync(vertices + 3 * off[a], t->staging[buf], bytes, cudaMemcpyDeviceToHost,
                                        t->copy_stream));
            SG_CUDA(cudaEventRecord(t->ev_copied[buf], t->copy_stream));
            a = b;
            ++k;
        }
        for (int buf = 0; buf < 2; ++buf) SG_CUDA(cudaStreamWaitEvent(s, t->ev_copied[buf], 0));
        return SG_OK;
    }
    return launch_gather_lines(t, offsets, vertices, status, margin, s);
}

extern "C" sg_status sg_tracer_get_lines_overlapped(sg_tracer *t, int64_t *n_lines, int64_t *n_vertices,
                                                    int64_t *offsets, float *vertices, uint8_t *status, float *margin,
                                                    void *stream)
{
    SG_CHECK(t != nullptr, SG_ERR_INVALID_ARG, "tracer is NULL");
    SG_CHECK(t->p.mode != SG_STREAKLINE, SG_ERR_STATE, "overlapped readout is for streamline and path-line tracers");
    for (const void *q : {(const void *)offsets, (const void *)vertices, (const void *)status, (const void *)margin})
        SG_CHECK(!q || pointer_kind(q) == PTR_PINNED, SG_ERR_INVALID_ARG,
                 "overlapped readout buffers must be page-locked host memory");
    SG_CUDA(cudaSetDevice(t->ctx->device));
    cudaStream_t s = (cudaStream_t)stream;
    sg_status st = ensure_scanned(t, s);
    if (st) return st;
    int64_t tot[3];
    if ((st = read_totals(t, tot, s))) return st;   // synchronises `stream`: the trace is done
    if (n_lines) *n_lines = tot[1];
    if (n_vertices) *n_vertices = tot[0];
    if (!offsets && !vertices && !status && !margin) return SG_OK;
    const size_t nl = (size_t)t->n_lines, nv = (size_t)tot[0];
    const size_t o_off = 0, o_vert = align_up(sizeof(int64_t) * (nl + 1), 256);
    const size_t o_st = o_vert + align_up(sizeof(float) * 3 * nv, 256);
    const size_t o_mg = o_st + align_up(nl, 256);
    const size_t need = o_mg + align_up(sizeof(float) * nl, 256);
    const size_t bytes = align_up(need, (size_t)2 << 20);
    // this readout's staging buffer: the two alternate; if the second cannot
    // be allocated, the first serves every readout
    int k = t->ovl_single ? 0 : t->ovl_next;
    if (need > t->ovl_bytes[k]) {
        // the copy of the readout that used this buffer still reads it
        SG_CUDA(cudaEventSynchronize(t->ev_ovl_copied[k]));
        if (t->ovl_buf[k]) SG_CUDA(cudaFree(t->ovl_buf[k]));
        t->ovl_buf[k] = nullptr;
        t->ovl_bytes[k] = 0;
        cudaError_t ae = cudaMalloc(&t->ovl_buf[k], bytes);
        if (ae != cudaSuccess) t->ovl_buf[k] = nullptr;   // nothing to free later
        if (ae == cudaErrorMemoryAllocation && k == 1) {
            (void)cudaGetLastError();            // not sticky: the first buffer serves from now on
            t->ovl_single = true;
            k = 0;
            if (need > t->ovl_bytes[0]) {
                SG_CUDA(cudaEventSynchronize(t->ev_ovl_copied[0]));
                if (t->ovl_buf[0]) SG_CUDA(cudaFree(t->ovl_buf[0]));
                t->ovl_buf[0] = nullptr;
                t->ovl_bytes[0] = 0;
                const cudaError_t a0 = cudaMalloc(&t->ovl_buf[0], bytes);
                if (a0 != cudaSuccess) t->ovl_buf[0] = nullptr;
                SG_CUDA(a0);
                t->ovl_bytes[0] = bytes;
            }
        } else {
            SG_CUDA(ae);
            t->ovl_bytes[k] = bytes;
        }
    }
    t->ovl_next = k ^ 1;
    t->ovl_last = k;
    char *b = t->ovl_buf[k];
    // the gather overwrites the staging memory only after the copy of the
    // readout that used it last has read it
    SG_CUDA(cudaStreamWaitEvent(s, t->ev_ovl_copied[k], 0));
    st = launch_gather_lines(t, (int64_t *)(b + o_off), (float *)(b + o_vert), (uint8_t *)(b + o_st),
                             (float *)(b + o_mg), s);
    if (st) return st;
    SG_CUDA(cudaEventRecord(t->ev_ovl_gathered, s));
    SG_CUDA(cudaStreamWaitEvent(t->copy_stream, t->ev_ovl_gathered, 0));
    if (offsets)
        SG_CUDA(cudaMemcpyAsync(offsets, b + o_off, sizeof(int64_t) * (nl + 1), cudaMemcpyDeviceToHost,
                                t->copy_stream));
    if (vertices && nv)
        SG_CUDA(cudaMemcpyAsync(vertices, b + o_vert, sizeof(float) * 3 * nv, cudaMemcpyDeviceToHost, t->copy_stream));
    if (status && nl) SG_CUDA(cudaMemcpyAsync(status, b + o_st, nl, cudaMemcpyDeviceToHost, t->copy_stream));
    if (margin && nl)
        SG_CUDA(cudaMemcpyAsync(margin, b + o_mg, sizeof(float) * nl, cudaMemcpyDeviceToHost, t->copy_stream));
    SG_CUDA(cudaEventRecord(t->ev_ovl_copied[k], t->copy_stream));
    return SG_OK;
}

extern "C" sg_status sg_tracer_wait_lines(sg_tracer *t, void *stream)
{
    SG_CHECK(t != nullptr, SG_ERR_INVALID_ARG, "tracer is NULL");
    SG_CHECK(t->p.mode != SG_STREAKLINE, SG_ERR_STATE, "overlapped readout is for streamline and path-line tracers");
    SG_CUDA(cudaSetDevice(t->ctx->device));
    // the copies run in order on the copy stream: the last one covers them all
    SG_CUDA(cudaStreamWaitEvent((cudaStream_t)stream, t->ev_ovl_copied[t->ovl_last], 0));
    return SG_OK;
}

extern "C" sg_status sg_tracer_get_joined(sg_tracer *t, int64_t *n_lines, int64_t *n_vertices, int64_t *offsets,
                                          float *vertices, int64_t *seed_vertex, void *stream)
{
    SG_CHECK(t != nullptr, SG_ERR_INVALID_ARG, "tracer is NULL");
    SG_CHECK(t->p.mode == SG_STREAMLINE && t->p.direction == SG_DIR_BOTH, SG_ERR_STATE,
             "joined lines need a streamline tracer created with SG_DIR_BOTH");
    SG_CUDA(cudaSetDevice(t->ctx->device));
    cudaStream_t s = (cudaStream_t)stream;
    sg_status st = launch_join_scan(t, s);
    if (st) return st;
    const bool query = !offsets && !vertices && !seed_vertex;
    if (query || n_lines || n_vertices) {
        int64_t h[4];
        SG_CUDA(cudaMemcpyAsync(h, t->join_tot, sizeof h, cudaMemcpyDeviceToHost, s));
        SG_CUDA(cudaStreamSynchronize(s));
        if (n_lines) *n_lines = t->n_seeds;
        if (n_vertices) *n_vertices = t->n_seeds > 0 ? h[0] : 0;
        if (query) return SG_OK;
    }
    for (const void *q : {(const void *)offsets, (const void *)vertices, (const void *)seed_vertex})
        SG_CHECK(!q || pointer_kind(q) == PTR_DEVICE, SG_ERR_INVALID_ARG, "joined-line buffers must be device memory");
    return launch_join(t, offsets, vertices, seed_vertex, s);
}

extern "C" sg_status sg_tracer_total_steps(sg_tracer *t, int64_t *steps, void *stream)
{
    SG_CHECK(t && steps, SG_ERR_INVALID_ARG, "NULL argument");
    SG_CUDA(cudaSetDevice(t->ctx->device));
    cudaStream_t s = (cudaStream_t)stream;
    sg_status st = ensure_scanned(t, s);
    if (st) return st;
    int64_t tot[3];
    st = read_totals(t, tot, s);
    if (st) return st;
    *steps = tot[2];
    return SG_OK;
}
