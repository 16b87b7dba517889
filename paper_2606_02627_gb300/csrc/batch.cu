// Request batch: continuous batching of streamline requests over resident
// fields (the serving form of the interactive seed-placement application of
// Sec. 4).  The particles of every admitted request share one brick-sorted
// queue and one persistent kernel; each lane reads its own request's field,
// storage type, step size and step cap.  Rounds run as one CUDA graph (a
// while-node, as for a tracer); requests join between runs and leave as soon
// as their last line stops.
#include <string.h>

#include <map>
#include <vector>

#include "rk4.cuh"

namespace sg {

struct BatchParams {
    Particle *q;
    Particle *o;
    Ctrl *ctrl;
    const ReqDev *reqs;
    const uint32_t *line_req;
    uint32_t *active;
    float *slab;
    uint32_t *line_len;
    uint8_t *line_status;
    float *line_margin;
    uint32_t steps_per_round;
    uint32_t drain_steps;
};

// A brick of any storage type: the typed view is made at the call.
struct BrickAny {
    const char *data;
    float scale;
    int lo[3];
    int hi[3];
};

template <int DT>
__device__ __forceinline__ BrickRef<DT> as_ref(const BrickAny &b)
{
    BrickRef<DT> r;
    r.data = reinterpret_cast<const typename Elem<DT>::T *>(b.data);
    r.scale = b.scale;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        r.lo[a] = b.lo[a];
        r.hi[a] = b.hi[a];
    }
    return r;
}

__device__ __forceinline__ void brick_any(const DevField &F, int dtype, const int c[3], BrickAny &br)
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
    const long long elem = dtype == SG_F32 ? 16 : 8;
    br.data = F.data + (long long)id * F.brick_stride * elem;
    br.scale = dtype == SG_F32 ? 1.0f : __ldg(F.scales + id);
}

template <int LAYOUT>
__device__ __forceinline__ int rk4_any(int dtype, const DevField &F, const float dtc[3], float eps, const BrickAny &br,
                                       int c[3], float f[3], float &margin)
{
    switch (dtype) {
    case SG_BF16: return rk4_bricked<SG_BF16, LAYOUT>(F, dtc, eps, as_ref<SG_BF16>(br), c, f, margin);
    case SG_F16: return rk4_bricked<SG_F16, LAYOUT>(F, dtc, eps, as_ref<SG_F16>(br), c, f, margin);
    case SG_FX21: return rk4_bricked<SG_FX21, LAYOUT>(F, dtc, eps, as_ref<SG_FX21>(br), c, f, margin);
    default: return rk4_bricked<SG_F32, LAYOUT>(F, dtc, eps, as_ref<SG_F32>(br), c, f, margin);
    }
}

// The persistent round of a batch: the tracer's round kernel with every
// request parameter read per lane when a particle is popped.
template <int LAYOUT>
__global__ void __launch_bounds__(256) batch_round_kernel(const __grid_constant__ BatchParams P)
{
    const unsigned lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    const uint32_t q_count = P.ctrl->q_count;
    bool active = false;
    bool drained = q_count == 0;
    int c[3] = {0, 0, 0};
    float f[3] = {0.f, 0.f, 0.f};
    uint32_t line = 0, step = 0, here = 0, r = 0, max_steps = 0;
    int dtype = SG_F32;
    float dtc[3] = {0.f, 0.f, 0.f}, eps = 0.f;
    float *vslab = nullptr;
    const ReqDev *R = P.reqs;
    BrickAny br;
    br.data = nullptr;
    br.scale = 1.0f;
    for (int a = 0; a < 3; ++a) br.lo[a] = br.hi[a] = 0;

    while (true) {
        const unsigned need = __ballot_sync(SG_FULL_MASK, !active);
        if (need && !drained) {
            const int leader = __ffs(need) - 1;
            uint32_t base = 0;
            if ((int)lane == leader) base = atomicAdd(&P.ctrl->q_head, (uint32_t)__popc(need));
            base = __shfl_sync(SG_FULL_MASK, base, leader);
            if (base + (uint32_t)__popc(need) >= q_count) drained = true;
            if (!active) {
                const uint32_t my = base + __popc(need & lt);
                if (my < q_count) {
                    load_particle(P.q + my, c, f, line, step);
                    r = P.line_req[line];
                    R = P.reqs + r;
                    dtype = R->dtype;
                    max_steps = R->max_steps;
                    eps = R->eps;
#pragma unroll
                    for (int a = 0; a < 3; ++a) dtc[a] = R->dtc[a];
                    vslab = P.slab + R->slab_base + (long long)(line - R->line_base) * R->W * 3;
                    brick_any(R->F, dtype, c, br);
                    active = true;
                    here = 0;
                }
            }
        }
        if (__ballot_sync(SG_FULL_MASK, active) == 0) break;

        int ev = EV_NONE, st = SG_LINE_ACTIVE;
        float margin = INFINITY;
        if (active) {
            if (step >= max_steps) {
                ev = EV_STOP;
                st = SG_LINE_MAXSTEPS;
            } else if (here >= P.steps_per_round) {
                ev = EV_APPEND;
            } else {
                const DevField &F = R->F;
                st = rk4_any<LAYOUT>(dtype, F, dtc, eps, br, c, f, margin);
                if (st != SG_LINE_ACTIVE) {
                    ev = EV_STOP;
                } else {
                    ++step;
                    ++here;
                    float *o = vslab + 3ll * step;
                    st_na(o, fmaf(F.spacing[0], (float)c[0] + f[0], F.origin[0]));
                    st_na(o + 1, fmaf(F.spacing[1], (float)c[1] + f[1], F.origin[1]));
                    st_na(o + 2, fmaf(F.spacing[2], (float)c[2] + f[2], F.origin[2]));
                    if (step >= max_steps) {
                        ev = EV_STOP;
                        st = SG_LINE_MAXSTEPS;
                    } else if (c[0] < br.lo[0] || c[0] >= br.hi[0] || c[1] < br.lo[1] || c[1] >= br.hi[1] ||
                               c[2] < br.lo[2] || c[2] >= br.hi[2]) {
                        ev = EV_APPEND;
                    }
                }
            }
        }
        warp_append(ev == EV_APPEND, P.o, &P.ctrl->o_count, c, f, line, step);
        if (ev == EV_STOP) {
            P.line_len[line] = step + 1;
            P.line_status[line] = stop_code_t(st, margin, R->tie_cells, R->tie_eps_rel);
            P.line_margin[line] = margin;
            atomicSub(P.active + r, 1u);
        }
        if (ev != EV_NONE) active = false;
    }
}

// The same round with the lanes of a warp decoupled (CELL8 layout), as the
// tracer's round_async_kernel: a pass runs up to four RK4 stages, unrolled
// (iteration s runs stage s for the lanes at stage s whose record is at
// hand); each lane keeps the FP32 cell record of its current sample point in
// a shared-memory slot and fetches another with one TMA bulk copy completing
// on its own mbarrier; the 8-byte formats' records land in a separate area
// and are decoded into the slot once, with the storage type of the lane's own
// request; vertices are staged and leave as 48-byte runs.  Stage arithmetic as
// rk4_bricked's, so a request's lines are the tracer's bits.
//
// Shared memory per thread: the FP32 slot (6 chunks) and a pad holding the
// brick's first owned cell and two extents; the landing area (4 chunks) and a
// pad holding the eps^2 threshold, brick scale and step cap; the vertex
// staging (4 chunks) and a pad holding the slab row pointer, the first vertex
// this lane writes and the third extent; one mbarrier.  Strides of 7, 5 and 5
// chunks keep eight consecutive lanes' 16-byte accesses in different banks.
struct BatchLayout {
    static constexpr int NCH = Record<SG_F32>::chunks;
    static constexpr unsigned SLOT = (NCH + 1) * 16;
    static constexpr unsigned LAND = (Record<SG_F16>::chunks + 1) * 16;
    static constexpr unsigned VBUF = 80;
    static constexpr unsigned PER_THREAD = SLOT + LAND + VBUF + 8;
};
// Consecutive passes a lane may wait for one record copy (each pass takes at
// least ~100 cycles: well over a second in all), as in the tracer's kernel.
constexpr unsigned BATCH_COPY_WAIT_PASSES = 1u << 24;

template <int DT>
__device__ __forceinline__ void decode_face(const uint4 *land, int dx, float3 cr[4], unsigned &flags)
{
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const uint4 w = land[j];
        const uint2 e = dx ? make_uint2(w.z, w.w) : make_uint2(w.x, w.y);
        cr[j] = decode_elem<DT>(e);
        flags |= elem_flag<DT>(e);
    }
}

__global__ void __launch_bounds__(256, 3) batch_async_kernel(const __grid_constant__ BatchParams P)
{
    using L = BatchLayout;
    constexpr int NCH = L::NCH;
    extern __shared__ uint4 slots[];
    const unsigned tid = threadIdx.x, nthr = blockDim.x;
    const unsigned lane = tid & 31;
    uint4 *my_slot = slots + tid * (L::SLOT / 16);
    uint4 *my_land = slots + nthr * (L::SLOT / 16) + tid * (L::LAND / 16);
    uint4 *vbuf = slots + nthr * ((L::SLOT + L::LAND) / 16) + tid * (L::VBUF / 16);
    const uint32_t bar =
        smem_addr(reinterpret_cast<uint64_t *>(slots + nthr * ((L::SLOT + L::LAND + L::VBUF) / 16)) + tid);
    const uint32_t slot_f32 = smem_addr(my_slot), slot_raw = smem_addr(my_land);
    mbar_init(bar, 1);
    mbar_init_fence();
    __syncwarp();

    const uint32_t *q_count_p = &P.ctrl->q_count;
    bool active = false, pending = false;
    bool inflight = false;                                 // a copy may still land in the slot
    bool drained = __ldg(q_count_p) == 0;
    uint32_t drain_left = P.drain_steps;                   // one pass per step
    unsigned parity = 0, waited = 0;
    int c[3] = {0, 0, 0}, q[3] = {0, 0, 0};
    float f[3] = {0.f, 0.f, 0.f}, g[3] = {0.f, 0.f, 0.f};
    float k1x = 0.f, k1y = 0.f, k1z = 0.f;
    float k23x = 0.f, k23y = 0.f, k23z = 0.f;
    float dsx = 0.f, dsy = 0.f, dsz = 0.f;
    uint32_t line = 0, step = 0, stage = 0, r = 0;
    int dtype = SG_F32;
    int left = 0;                        // steps before max_steps or the round's step budget stops the lane
    uint32_t held = 0xffffffffu;         // cell of the record in (or on its way to) the slot
    bool rec_bad = false;                // FX21: a corner of the slot's record is flagged
    const char *bdata = nullptr;         // the brick's records
    int cbase = 0, C0 = 0, C1 = 0;       // record index of cell q: (q.z C1 + q.y) C0 + q.x + cbase
    int box_lo[3] = {0, 0, 0};
    unsigned box_span[3] = {0u, 0u, 0u};

    auto cell_of = [&]() { return (uint32_t)((q[2] * C1 + q[1]) * C0 + q[0] + cbase); };
    auto fetch = [&](uint32_t cell) {
        const uint32_t bytes = dtype == SG_F32 ? (uint32_t)(NCH * 16) : (uint32_t)(Record<SG_F16>::chunks * 16);
        bulk_copy_arrive(dtype == SG_F32 ? slot_f32 : slot_raw, bdata + (long long)cell * bytes, bytes, bar);
        inflight = true;
        held = cell;
        pending = true;
        waited = 0;
    };

    while (true) {
        const unsigned need = __ballot_sync(SG_FULL_MASK, !active);
        if (need == SG_FULL_MASK && drained) break;
        if (need && !drained) {
            const int leader = __ffs(need) - 1;
            uint32_t base = 0;
            if ((int)lane == leader) base = atomicAdd(&P.ctrl->q_head, (uint32_t)__popc(need));
            base = __shfl_sync(SG_FULL_MASK, base, leader);
            const uint32_t q_count = __ldg(q_count_p);
            if (base + (uint32_t)__popc(need) >= q_count) drained = true;
            if (!active) {
                const uint32_t my = base + __popc(need & ((1u << lane) - 1u));
                if (my < q_count) {
                    load_particle(P.q + my, c, f, line, step);
                    r = P.line_req[line];
                    const ReqDev *R = P.reqs + r;
                    dtype = R->dtype;
                    const uint32_t max_steps = R->max_steps;
                    const DevField &F = R->F;
                    BrickAny br;
                    brick_any(F, dtype, c, br);
                    bdata = br.data;
                    float ds[3];
#pragma unroll
                    for (int a = 0; a < 3; ++a) {
                        ds[a] = dtype == SG_F32 ? R->dtc[a] : __fmul_rn(R->dtc[a], br.scale);
                        q[a] = c[a];
                        g[a] = f[a];
                    }
                    dsx = ds[0];
                    dsy = ds[1];
                    dsz = ds[2];
#pragma unroll
                    for (int a = 0; a < 3; ++a) {
                        const int lo = max(br.lo[a] - 1, 0);
                        const int hi = min(br.lo[a] + F.S[a] - 3, F.nm1[a] - 1);
                        box_lo[a] = hi >= lo ? lo : 0x7fffffff;   // empty: every point takes the full tests
                        box_span[a] = hi >= lo ? (unsigned)(hi - lo) : 0u;
                    }
                    C0 = F.C[0];
                    C1 = F.C[1];
                    cbase = -(((br.lo[2] - 1) * C1 + (br.lo[1] - 1)) * C0 + (br.lo[0] - 1));
                    {
                        // |v|^2 at or above the threshold (before the brick scale) means |v| >= eps
                        const float e = dtype == SG_F32 ? R->eps : __fdiv_ru(R->eps, br.scale);
                        my_land[4] = make_uint4(__float_as_uint(__fmul_ru(e, e)), __float_as_uint(br.scale),
                                                max_steps, 0u);
                        const unsigned long long row = reinterpret_cast<unsigned long long>(
                            P.slab + R->slab_base + (long long)(line - R->line_base) * R->W * 3);
                        const uint32_t sp0 = (uint32_t)(br.hi[0] - br.lo[0]), sp1 = (uint32_t)(br.hi[1] - br.lo[1]);
                        vbuf[4] = make_uint4((uint32_t)row, (uint32_t)(row >> 32), step + 1,
                                             (uint32_t)(br.hi[2] - br.lo[2]));
                        my_slot[NCH] = make_uint4((uint32_t)br.lo[0], (uint32_t)br.lo[1], (uint32_t)br.lo[2],
                                                  sp0 | (sp1 << 16));
                    }
                    left = step >= max_steps ? 0 : (int)min(max_steps - step, P.steps_per_round);
                    active = true;
                    stage = 0;
                    fetch(cell_of());
                }
            }
        }
        if (drained) {
            if (drain_left == 0) left = 0;
            else --drain_left;
        }
        bool gave_up = false;
        if (pending) {
            if (mbar_done(bar, parity)) {
                parity ^= 1u;
                pending = false;
                inflight = false;
                if (dtype != SG_F32) {
                    // decode the landed record once into the FP32 slot, one x face at
                    // a time, with the lane's own storage type
                    unsigned flags = 0u;
#pragma unroll
                    for (int dx = 0; dx < 2; ++dx) {
                        float3 cr[4];                // (dy, dz) = (0,0), (1,0), (0,1), (1,1)
                        if (dtype == SG_BF16) decode_face<SG_BF16>(my_land, dx, cr, flags);
                        else if (dtype == SG_F16) decode_face<SG_F16>(my_land, dx, cr, flags);
                        else decode_face<SG_FX21>(my_land, dx, cr, flags);
                        my_slot[dx] = make_uint4(__float_as_uint(cr[0].x), __float_as_uint(cr[2].x),
                                                 __float_as_uint(cr[1].x), __float_as_uint(cr[3].x));
                        my_slot[2 + dx] = make_uint4(__float_as_uint(cr[0].y), __float_as_uint(cr[2].y),
                                                     __float_as_uint(cr[1].y), __float_as_uint(cr[3].y));
                        my_slot[4 + dx] = make_uint4(__float_as_uint(cr[0].z), __float_as_uint(cr[2].z),
                                                     __float_as_uint(cr[1].z), __float_as_uint(cr[3].z));
                    }
                    rec_bad = flags != 0u;
                }
            } else if (++waited >= BATCH_COPY_WAIT_PASSES) {
                atomicOr(&P.ctrl->err, CTRL_ERR_TIMEOUT);
                active = false;
                pending = false;
                gave_up = true;
            }
        }
        if (__any_sync(SG_FULL_MASK, gave_up)) drained = true;

        int ev = EV_NONE, st = SG_LINE_ACTIVE;
        float margin = INFINITY;
        bool go = active && !pending;
        bool run_done = false;                       // this pass completed vertex 4j+3 of the row
        if (go && stage == 0 && left <= 0) {
            if (step >= my_land[4].z) {
                ev = EV_STOP;
                st = SG_LINE_MAXSTEPS;
            } else {
                ev = EV_APPEND;                   // the round's step budget is spent
            }
            go = false;
        }
#pragma unroll
        for (int S = 0; S < 4; ++S) {
            if (go && stage == (uint32_t)S) {
                Record<SG_F32> Rc;
#pragma unroll
                for (int k = 0; k < NCH; ++k) Rc.r[k] = my_slot[k];
                bool bad_flag;
                const float3 v = interp_record<SG_F32>(Rc, g[0], g[1], g[2], bad_flag);
                const float kx = __fmul_rn(v.x, dsx), ky = __fmul_rn(v.y, dsy), kz = __fmul_rn(v.z, dsz);
                float dx, dy, dz;                    // offset of the next point from P0
                if (S == 0) {
                    k1x = kx;
                    k1y = ky;
                    k1z = kz;
                } else if (S == 1) {
                    k23x = kx;
                    k23y = ky;
                    k23z = kz;
                } else if (S == 2) {
                    k23x = __fadd_rn(k23x, kx);
                    k23y = __fadd_rn(k23y, ky);
                    k23z = __fadd_rn(k23z, kz);
                }
                if (S < 3) {
                    const float w = S < 2 ? 0.5f : 1.0f;   // P1, P2 = P0 + k/2; P3 = P0 + k3
                    dx = __fmul_rn(w, kx);
                    dy = __fmul_rn(w, ky);
                    dz = __fmul_rn(w, kz);
                } else {
                    dx = __fmul_rn(__fadd_rn(__fadd_rn(k1x, kx), __fmul_rn(2.0f, k23x)), 1.0f / 6.0f);
                    dy = __fmul_rn(__fadd_rn(__fadd_rn(k1y, ky), __fmul_rn(2.0f, k23y)), 1.0f / 6.0f);
                    dz = __fmul_rn(__fadd_rn(__fadd_rn(k1z, kz), __fmul_rn(2.0f, k23z)), 1.0f / 6.0f);
                }
                locate(f[0], dx, c[0], q[0], g[0]);
                locate(f[1], dy, c[1], q[1], g[1]);
                locate(f[2], dz, c[2], q[2], g[2]);
                const bool in_box = (unsigned)(q[0] - box_lo[0]) <= box_span[0] &&
                                    (unsigned)(q[1] - box_lo[1]) <= box_span[1] &&
                                    (unsigned)(q[2] - box_lo[2]) <= box_span[2];
                const float s2 = __fadd_rn(__fadd_rn(__fmul_rn(v.x, v.x), __fmul_rn(v.y, v.y)), __fmul_rn(v.z, v.z));
                const bool maybe_bad = dtype == SG_FX21 ? rec_bad : !(s2 < INFINITY);
                if (maybe_bad || (S == 0 && !(s2 >= __uint_as_float(my_land[4].x))) || !in_box) {
                    // the tests in full (rare)
                    const ReqDev *R = P.reqs + r;
                    const DevField &F = R->F;
                    const bool bad = dtype == SG_FX21 ? rec_bad : bad3(v);
                    float sp = sqrtf(s2);
                    if (dtype != SG_F32) sp = __fmul_rn(sp, __uint_as_float(my_land[4].y));
                    const float eps = R->eps;
                    if (bad) {
                        st = SG_LINE_NANFIELD;
                    } else if (S == 0 && sp < eps) {
                        margin = (eps - sp) / eps;
                        st = SG_LINE_STAGNANT;
                    } else if (!in_domain(F, q, g)) {
                        margin = out_dist(F, q, g);
                        st = SG_LINE_EXIT;
                    } else if (S < 3) {
                        const uint4 bl = my_slot[NCH];
                        if ((unsigned)(q[0] - (int)bl.x + 1) > (unsigned)(F.S[0] - 2) ||
                            (unsigned)(q[1] - (int)bl.y + 1) > (unsigned)(F.S[1] - 2) ||
                            (unsigned)(q[2] - (int)bl.z + 1) > (unsigned)(F.S[2] - 2))
                            st = SG_LINE_HALO;
                    }
                }
                if (st != SG_LINE_ACTIVE) {
                    ev = EV_STOP;
                    go = false;
                } else if (S == 3) {
#pragma unroll
                    for (int a = 0; a < 3; ++a) {
                        c[a] = q[a];
                        f[a] = g[a];
                    }
                    ++step;
                    --left;
                    {
                        const DevField &F = P.reqs[r].F;
                        vbuf[step & 3u] = make_uint4(__float_as_uint(fmaf(F.spacing[0], (float)c[0] + f[0], F.origin[0])),
                                                     __float_as_uint(fmaf(F.spacing[1], (float)c[1] + f[1], F.origin[1])),
                                                     __float_as_uint(fmaf(F.spacing[2], (float)c[2] + f[2], F.origin[2])),
                                                     0u);
                    }
                    run_done = (step & 3u) == 3u;
                    stage = 0;
                    const uint4 bl = my_slot[NCH];
                    const bool out = (unsigned)(c[0] - (int)bl.x) >= (bl.w & 0xffffu) ||
                                     (unsigned)(c[1] - (int)bl.y) >= (bl.w >> 16) ||
                                     (unsigned)(c[2] - (int)bl.z) >= vbuf[4].w;
                    if (left <= 0 || out) {
                        go = false;
                        if (step >= my_land[4].z) {
                            ev = EV_STOP;
                            st = SG_LINE_MAXSTEPS;
                        } else {
                            ev = EV_APPEND;           // another brick, or the round's step budget is spent
                        }
                    }
                } else {
                    stage = S + 1;
                }
                if (go) {
                    const uint32_t next = cell_of();
                    if (next != held) {
                        fetch(next);
                        go = false;
                    }
                }
            }
        }
        if (run_done) {
            const uint4 rw = vbuf[4];
            float *vrow = reinterpret_cast<float *>(((unsigned long long)rw.y << 32) | rw.x);
            if (step - 3u >= rw.z) {
                // the row's run 4j .. 4j+3 is this lane's: 48 bytes at a 16-byte boundary
                uint4 *o = reinterpret_cast<uint4 *>(vrow + 3ll * (step - 3u));
                const uint4 a = vbuf[0], b = vbuf[1];
                st_na4(o, make_uint4(a.x, a.y, a.z, b.x));
                const uint4 cc = vbuf[2];
                st_na4(o + 1, make_uint4(b.y, b.z, cc.x, cc.y));
                const uint4 d = vbuf[3];
                st_na4(o + 2, make_uint4(cc.z, d.x, d.y, d.z));
            } else {
                for (uint32_t u = rw.z; u <= step; ++u) {
                    const uint4 a = vbuf[u & 3u];
                    float *o = vrow + 3ll * u;
                    st_na(o, __uint_as_float(a.x));
                    st_na(o + 1, __uint_as_float(a.y));
                    st_na(o + 2, __uint_as_float(a.z));
                }
            }
        }
        if (__any_sync(SG_FULL_MASK, ev != EV_NONE)) {
            if (ev != EV_NONE && (step & 3u) != 3u) {
                // the particle leaves: the staged vertices of its unfinished run
                const uint4 rw = vbuf[4];
                float *vrow = reinterpret_cast<float *>(((unsigned long long)rw.y << 32) | rw.x);
                for (uint32_t u = max(rw.z, step & ~3u); u <= step; ++u) {
                    const uint4 a = vbuf[u & 3u];
                    float *o = vrow + 3ll * u;
                    st_na(o, __uint_as_float(a.x));
                    st_na(o + 1, __uint_as_float(a.y));
                    st_na(o + 2, __uint_as_float(a.z));
                }
            }
            warp_append(ev == EV_APPEND, P.o, &P.ctrl->o_count, c, f, line, step);
            if (ev == EV_STOP) {
                const ReqDev *R = P.reqs + r;
                P.line_len[line] = step + 1;
                P.line_status[line] = stop_code_t(st, margin, R->tie_cells, R->tie_eps_rel);
                P.line_margin[line] = margin;
                atomicSub(P.active + r, 1u);
            }
            if (ev != EV_NONE) active = false;
        }
    }
    // a copy left in flight after a wait ran out: wait for it once more, with a limit
    for (unsigned i = 0; inflight && i < BATCH_COPY_WAIT_PASSES; ++i)
        if (mbar_done(bar, parity)) inflight = false;
}

// Seeds of request r -> particles appended to the outgoing buffer, first
// vertices, line arrays and the request's count of lines still moving.
__global__ void batch_upload_kernel(BatchParams P, const float *seeds, uint32_t r, ReqDev Rh)
{
    const long long n = Rh.n_lines;
    const unsigned lane = threadIdx.x & 31;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long base = (long long)blockIdx.x * blockDim.x + threadIdx.x - lane; base < n; base += stride) {
        const long long i = base + lane;
        bool keep = false;
        int c[3] = {0, 0, 0};
        float f[3] = {0.f, 0.f, 0.f};
        const uint32_t line = Rh.line_base + (uint32_t)i;
        if (i < n) {
            const float *sd = seeds + 3ll * line;
            double p[3];
            bool inside = true;
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                p[a] = ((double)sd[a] - Rh.origin_d[a]) / Rh.spacing_d[a];
                inside = inside && (p[a] >= 0.0 && p[a] <= (double)Rh.F.nm1[a]);
            }
            P.line_margin[line] = INFINITY;
            if (!inside) {
                P.line_len[line] = 0;
                P.line_status[line] = SG_LINE_OUT;
            } else {
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    const double fl = floor(p[a]);
                    c[a] = (int)fl;
                    f[a] = (float)(p[a] - fl);
                    if (f[a] >= 1.0f) {
                        f[a] = 0.0f;
                        c[a] += 1;
                    }
                }
                float *o = P.slab + Rh.slab_base + i * Rh.W * 3;
                o[0] = sd[0];
                o[1] = sd[1];
                o[2] = sd[2];
                P.line_len[line] = 1;
                P.line_status[line] = SG_LINE_ACTIVE;
                keep = true;
            }
        }
        const unsigned m = __ballot_sync(SG_FULL_MASK, keep);
        if (m && lane == (unsigned)(__ffs(m) - 1)) atomicAdd(P.active + r, (uint32_t)__popc(m));
        warp_append(keep, P.o, &P.ctrl->o_count, c, f, line, 0u);
    }
}

__global__ void fill_u32_kernel(uint32_t *dst, long long n, uint32_t v)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        dst[i] = v;
}

// Start of a run: the particles left in the queue by a capped run join the
// outgoing buffer (where new requests' particles already are), to be binned
// together.
__global__ void batch_merge_kernel(const Particle *q, Particle *o, const Ctrl *ctrl)
{
    const uint32_t nq = ctrl->q_count, base = ctrl->o_count;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < nq; i += gridDim.x * blockDim.x) {
        const int4 *s = reinterpret_cast<const int4 *>(q + i);
        int4 *d = reinterpret_cast<int4 *>(o + base + i);
        d[0] = s[0];
        d[1] = s[1];
    }
}

__global__ void batch_merge_fix_kernel(Ctrl *ctrl)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        ctrl->o_count += ctrl->q_count;
        ctrl->q_count = 0;
        ctrl->q_head = 0;
    }
}

__global__ void batch_prepare_kernel(Ctrl *ctrl, uint32_t max_rounds)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        ctrl->round = 0;
        ctrl->err = 0;
        ctrl->max_rounds = max_rounds;
    }
}

// ------------------------------------------------------------------ host side

// First-fit allocator of [0, size) in units, coalescing on release.
class RangeAlloc {
  public:
    void reset(long long size)
    {
        free_.clear();
        if (size > 0) free_[0] = size;
    }
    bool alloc(long long len, long long align, long long *off)
    {
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            const long long start = (it->first + align - 1) / align * align;
            const long long end = it->first + it->second;
            if (start + len <= end) {
                const long long s0 = it->first;
                free_.erase(it);
                if (start > s0) free_[s0] = start - s0;
                if (end > start + len) free_[start + len] = end - (start + len);
                *off = start;
                return true;
            }
        }
        return false;
    }
    void release(long long off, long long len)
    {
        auto it = free_.emplace(off, len).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
    long long largest() const
    {
        long long m = 0;
        for (auto &kv : free_) m = kv.second > m ? kv.second : m;
        return m;
    }
    long long total() const
    {
        long long t = 0;
        for (auto &kv : free_) t += kv.second;
        return t;
    }

  private:
    std::map<long long, long long> free_;
};

struct ReqHost {
    bool in_use = false;
    bool listed = false;
    uint32_t gen = 0;
    long long line_base = 0, n = 0;
    long long slab_off = 0, slab_len = 0;   // floats
    long long W = 0;
    int field = -1;
};

}  // namespace sg

struct sg_batch {
    sg_context *ctx;
    sg_batch_desc d;
    char *ws;
    size_t bytes;
    float *slab;
    float *seeds;
    uint32_t *line_len;
    uint8_t *line_status;
    float *line_margin;
    uint32_t *line_req;
    sg::Particle *q;
    sg::Particle *o;
    sg::Ctrl *ctrl;
    uint32_t *brick_count;
    uint32_t *brick_cursor;
    sg::ReqDev *reqs;
    uint32_t *active;
    int64_t *offsets;
    unsigned long long *block_sums;
    int64_t *totals;
    sg::RangeAlloc lines, slabs;
    std::vector<sg::ReqHost> req;
    std::vector<sg_field *> fields;
    std::vector<uint32_t> field_base;
    uint32_t next_brick;
    int64_t scanned_id;
    int grid, block;
    cudaGraph_t graph;
    cudaGraphExec_t exec;
};

namespace sg {

static size_t batch_layout(const sg_batch_desc *d, sg_batch *b, char *base)
{
    Carve c{base, 0, 0};
    const long long L = d->max_lines;
    float *slab = (float *)c.take((size_t)d->slab_bytes);
    float *seeds = (float *)c.take(sizeof(float) * 3 * L);
    uint32_t *len = (uint32_t *)c.take(sizeof(uint32_t) * L);
    uint8_t *st = (uint8_t *)c.take(L);
    float *mg = (float *)c.take(sizeof(float) * L);
    uint32_t *lr = (uint32_t *)c.take(sizeof(uint32_t) * L);
    Particle *q = (Particle *)c.take(sizeof(Particle) * L);
    Particle *o = (Particle *)c.take(sizeof(Particle) * L);
    Ctrl *ctrl = (Ctrl *)c.take(sizeof(Ctrl));
    uint32_t *bc = (uint32_t *)c.take(sizeof(uint32_t) * d->max_bricks);
    uint32_t *bcur = (uint32_t *)c.take(sizeof(uint32_t) * d->max_bricks);
    ReqDev *reqs = (ReqDev *)c.take(sizeof(ReqDev) * d->max_requests);
    uint32_t *act = (uint32_t *)c.take(sizeof(uint32_t) * d->max_requests);
    int64_t *off = (int64_t *)c.take(sizeof(int64_t) * (L + 1));
    unsigned long long *bs = (unsigned long long *)c.take(sizeof(unsigned long long) * (L / 4096 + 2));
    int64_t *tot = (int64_t *)c.take(sizeof(int64_t) * 4);
    if (b) {
        b->slab = slab;
        b->seeds = seeds;
        b->line_len = len;
        b->line_status = st;
        b->line_margin = mg;
        b->line_req = lr;
        b->q = q;
        b->o = o;
        b->ctrl = ctrl;
        b->brick_count = bc;
        b->brick_cursor = bcur;
        b->reqs = reqs;
        b->active = act;
        b->offsets = off;
        b->block_sums = bs;
        b->totals = tot;
    }
    return c.off;
}

static sg_status check_desc(const sg_batch_desc *d)
{
    SG_CHECK(d != nullptr, SG_ERR_INVALID_ARG, "desc is NULL");
    SG_CHECK(d->max_lines >= 1 && d->max_lines < (1ll << 32), SG_ERR_INVALID_ARG, "max_lines out of range");
    SG_CHECK(d->slab_bytes >= 0, SG_ERR_INVALID_ARG, "slab_bytes must be >= 0");
    SG_CHECK(d->max_requests >= 1 && d->max_requests <= (1 << 20), SG_ERR_INVALID_ARG, "max_requests out of range");
    SG_CHECK(d->max_fields >= 1 && d->max_fields <= 64, SG_ERR_INVALID_ARG, "max_fields out of range");
    SG_CHECK(d->max_bricks >= 1 && d->max_bricks <= 65536, SG_ERR_INVALID_ARG, "max_bricks out of range");
    SG_CHECK(d->layout == SG_LAYOUT_LINEAR || d->layout == SG_LAYOUT_TILED4 || d->layout == SG_LAYOUT_CELL8,
             SG_ERR_INVALID_ARG, "a batch samples bricked layouts");
    SG_CHECK(d->block_size >= 0 && d->block_size <= 256 && d->block_size % 32 == 0, SG_ERR_INVALID_ARG,
             "block_size must be a multiple of 32 in [0, 256]");
    SG_CHECK(d->blocks_per_sm >= 0 && d->blocks_per_sm <= 32, SG_ERR_INVALID_ARG, "bad blocks_per_sm");
    SG_CHECK(d->steps_per_round >= 0, SG_ERR_INVALID_ARG, "bad steps_per_round");
    return SG_OK;
}

static size_t batch_async_smem(int block) { return (size_t)block * BatchLayout::PER_THREAD; }

static BatchParams batch_params(const sg_batch *b)
{
    BatchParams P;
    P.q = b->q;
    P.o = b->o;
    P.ctrl = b->ctrl;
    P.reqs = b->reqs;
    P.line_req = b->line_req;
    P.active = b->active;
    P.slab = b->slab;
    P.line_len = b->line_len;
    P.line_status = b->line_status;
    P.line_margin = b->line_margin;
    P.steps_per_round = (uint32_t)(b->d.steps_per_round > 0 ? b->d.steps_per_round
                                                            : (b->d.layout == SG_LAYOUT_CELL8 ? 256 : 128));
    const int ds = b->d.drain_steps;
    P.drain_steps = ds < 0 ? 0x7fffffffu : (ds > 0 ? (uint32_t)ds : (b->d.layout == SG_LAYOUT_CELL8 ? 128u : 0x7fffffffu));
    return P;
}

static BinArgs batch_bin_args(const sg_batch *b)
{
    BinArgs A;
    A.src = b->o;
    A.src_count = &b->ctrl->o_count;
    A.dst = b->q;
    A.brick_count = b->brick_count;
    A.brick_cursor = b->brick_cursor;
    A.ctrl = b->ctrl;
    for (int a = 0; a < 3; ++a) {
        A.n[a] = 1;
        A.B[a] = 1;
    }
    A.nb = b->d.max_bricks;
    A.line_req = b->line_req;
    A.reqs = b->reqs;
    A.key_map = nullptr;
    A.n_local = A.nb;
    A.key_start = nullptr;
    return A;
}

static sg_status launch_batch_round(const sg_batch *b, cudaStream_t s)
{
    BatchParams P = batch_params(b);
    if (b->d.layout == SG_LAYOUT_CELL8) {
        batch_async_kernel<<<b->grid, b->block, batch_async_smem(b->block), s>>>(P);
        SG_CUDA(cudaGetLastError());
        return SG_OK;
    }
    bool ok = with_layout(b->d.layout, [&](auto Lay) {
        batch_round_kernel<decltype(Lay)::value><<<b->grid, b->block, 0, s>>>(P);
    });
    SG_CHECK(ok, SG_ERR_UNSUPPORTED, "no batch kernel for layout %d", b->d.layout);
    SG_CUDA(cudaGetLastError());
    return SG_OK;
}

static sg_status build_batch_graph(sg_batch *b)
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
        st = cuda_error(e, "batch graph setup");
    } else {
        const int sm = b->ctx->sm_count;
        batch_merge_kernel<<<sm * 4, 256, 0, cs>>>(b->q, b->o, b->ctrl);
        batch_merge_fix_kernel<<<1, 32, 0, cs>>>(b->ctrl);
        e = cudaGetLastError();
        if (e != cudaSuccess) st = cuda_error(e, "merge launch");
        if (st == SG_OK) st = launch_bin_args(batch_bin_args(b), sm, cs, true, (unsigned long long)h, 0);
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
            if (e == cudaSuccess)
                e = cudaStreamUpdateCaptureDependencies(cs, &cond, nullptr, 1, cudaStreamSetCaptureDependencies);
            if (e != cudaSuccess) st = cuda_error(e, "batch conditional node");
        }
        cudaGraph_t g2 = nullptr;
        cudaError_t e2 = cudaStreamEndCapture(cs, &g2);
        if (st == SG_OK && e2 != cudaSuccess) st = cuda_error(e2, "cudaStreamEndCapture");
        if (st == SG_OK) {
            cudaGraph_t body = cp.conditional.phGraph_out[0];
            e = cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
            if (e != cudaSuccess) {
                st = cuda_error(e, "batch body capture");
            } else {
                st = launch_batch_round(b, cs);
                if (st == SG_OK) st = launch_bin_args(batch_bin_args(b), sm, cs, true, (unsigned long long)h, 1);
                cudaGraph_t b2 = nullptr;
                e2 = cudaStreamEndCapture(cs, &b2);
                if (st == SG_OK && e2 != cudaSuccess) st = cuda_error(e2, "batch body end capture");
            }
        }
        if (st == SG_OK) {
            e = cudaGraphInstantiate(&b->exec, g, 0);
            if (e != cudaSuccess) st = cuda_error(e, "cudaGraphInstantiate");
        }
    }
    cudaStreamDestroy(cs);
    if (st != SG_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    b->graph = g;
    return SG_OK;
}

template <int LAYOUT>
static cudaError_t batch_prefer_l1()
{
    return cudaFuncSetAttribute(batch_round_kernel<LAYOUT>, cudaFuncAttributePreferredSharedMemoryCarveout, 0);
}

}  // namespace sg

using namespace sg;

extern "C" sg_status sg_batch_required_bytes(const sg_context *ctx, const sg_batch_desc *desc, size_t *bytes)
{
    SG_CHECK(ctx && bytes, SG_ERR_INVALID_ARG, "NULL argument");
    sg_status st = check_desc(desc);
    if (st) return st;
    *bytes = batch_layout(desc, nullptr, nullptr);
    return SG_OK;
}

extern "C" sg_status sg_batch_create(sg_context *ctx, const sg_batch_desc *desc, void *workspace, size_t bytes,
                                     sg_batch **out)
{
    SG_CHECK(ctx && out, SG_ERR_INVALID_ARG, "NULL argument");
    sg_status st = check_desc(desc);
    if (st) return st;
    SG_CHECK(workspace && ((uintptr_t)workspace & 255) == 0, SG_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
    const size_t need = batch_layout(desc, nullptr, nullptr);
    SG_CHECK(bytes >= need, SG_ERR_OOM, "batch needs %zu bytes, got %zu", need, bytes);
    SG_CHECK(pointer_kind(workspace) == PTR_DEVICE, SG_ERR_INVALID_ARG, "workspace must be device memory");
    SG_CUDA(cudaSetDevice(ctx->device));
    sg_batch *b = new sg_batch();
    b->ctx = ctx;
    b->d = *desc;
    b->ws = (char *)workspace;
    b->bytes = bytes;
    batch_layout(desc, b, (char *)workspace);
    b->lines.reset(desc->max_lines);
    b->slabs.reset(desc->slab_bytes / (long long)sizeof(float));
    b->req.resize(desc->max_requests);
    b->next_brick = 0;
    b->scanned_id = -1;
    b->block = desc->block_size > 0 ? desc->block_size : 256;
    // resident threads per SM as for a tracer: 768 with decoupled lanes (CELL8), else 512
    const int threads_per_sm = desc->layout == SG_LAYOUT_CELL8 ? 768 : 512;
    const int per_sm = desc->blocks_per_sm > 0 ? desc->blocks_per_sm : (threads_per_sm + b->block - 1) / b->block;
    b->grid = ctx->sm_count * per_sm;
    b->graph = nullptr;
    b->exec = nullptr;
    cudaError_t e = cudaMemset(b->ctrl, 0, sizeof(Ctrl));
    if (e == cudaSuccess) e = cudaMemset(b->brick_count, 0, sizeof(uint32_t) * desc->max_bricks);
    if (e == cudaSuccess) e = cudaMemset(b->active, 0, sizeof(uint32_t) * desc->max_requests);
    if (e == cudaSuccess) {
        if (desc->layout == SG_LAYOUT_CELL8) {
            const size_t smem = batch_async_smem(b->block);
            e = cudaFuncSetAttribute(batch_async_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            const size_t total = (smem + 1024) * (size_t)per_sm;
            int pct = (int)((total * 100 + 228 * 1024 - 1) / (228 * 1024));
            if (pct > 100) pct = 100;
            if (e == cudaSuccess)
                e = cudaFuncSetAttribute(batch_async_kernel, cudaFuncAttributePreferredSharedMemoryCarveout, pct);
        } else {
            with_layout(desc->layout, [&](auto Lay) { e = batch_prefer_l1<decltype(Lay)::value>(); });
        }
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        delete b;
        return cuda_error(e, "batch init");
    }
    *out = b;
    return SG_OK;
}

extern "C" sg_status sg_batch_destroy(sg_batch *b)
{
    if (!b) return SG_OK;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    delete b;
    return SG_OK;
}

extern "C" sg_status sg_batch_capacity(const sg_batch *b, int64_t *free_lines, int64_t *largest_slab_bytes,
                                       int32_t *free_requests)
{
    SG_CHECK(b != nullptr, SG_ERR_INVALID_ARG, "batch is NULL");
    if (free_lines) *free_lines = b->lines.total();
    if (largest_slab_bytes) *largest_slab_bytes = b->slabs.largest() * (int64_t)sizeof(float);
    if (free_requests) {
        int32_t k = 0;
        for (auto &r : b->req) k += !r.in_use;
        *free_requests = k;
    }
    return SG_OK;
}

static bool decode_id(const sg_batch *b, int64_t id, int *slot)
{
    const int64_t s = id & ((1 << 20) - 1);
    const uint32_t gen = (uint32_t)(id >> 20);
    if (id < 0 || s >= (int64_t)b->req.size()) return false;
    const ReqHost &r = b->req[s];
    if (!r.in_use || r.gen != gen) return false;
    *slot = (int)s;
    return true;
}

extern "C" sg_status sg_batch_submit(sg_batch *b, sg_field *f, const float *xyz, int64_t n, const sg_tracer_params *p,
                                     int64_t *request_id, void *stream)
{
    SG_CHECK(b && f && p && request_id, SG_ERR_INVALID_ARG, "NULL argument");
    SG_CHECK(n >= 0 && (n == 0 || xyz), SG_ERR_INVALID_ARG, "bad seeds");
    SG_CHECK(p->mode == SG_STREAMLINE, SG_ERR_UNSUPPORTED, "a batch traces streamlines");
    SG_CHECK(p->direction == SG_DIR_FORWARD || p->direction == SG_DIR_BACKWARD, SG_ERR_UNSUPPORTED,
             "a batch request traces one direction");
    SG_CHECK(p->dt > 0.0 && p->dt < 1e30, SG_ERR_INVALID_ARG, "dt must be > 0");
    SG_CHECK(p->max_steps >= 0 && p->max_steps < (1 << 27), SG_ERR_INVALID_ARG, "max_steps out of range");
    SG_CHECK(f->desc.layout == b->d.layout, SG_ERR_INVALID_ARG, "the field's layout differs from the batch's");
    SG_CHECK(f->ctx == b->ctx, SG_ERR_INVALID_ARG, "field of another context");
    SG_CUDA(cudaSetDevice(b->ctx->device));
    cudaStream_t s = (cudaStream_t)stream;
    // field key range
    int fi = -1;
    for (size_t k = 0; k < b->fields.size(); ++k)
        if (b->fields[k] == f) fi = (int)k;
    const bool new_field = fi < 0;
    if (new_field) {
        if ((int)b->fields.size() >= b->d.max_fields || (int64_t)b->next_brick + f->nb > b->d.max_bricks) {
            set_error("no room for another field in the batch");
            return SG_ERR_OOM;
        }
    }
    int slot = -1;
    for (size_t k = 0; k < b->req.size(); ++k)
        if (!b->req[k].in_use) {
            slot = (int)k;
            break;
        }
    if (slot < 0) {
        set_error("the request table is full");
        return SG_ERR_OOM;
    }
    const long long W = slab_stride(p->max_steps);    // rows of whole 4-vertex runs
    long long line_base = 0, slab_off = 0;
    const long long slab_len = (long long)n * W * 3;
    if (n > 0 && !b->lines.alloc(n, 1, &line_base)) {
        set_error("not enough free line slots (%lld needed)", (long long)n);
        return SG_ERR_OOM;
    }
    if (n > 0 && !b->slabs.alloc(slab_len, 4, &slab_off)) {
        b->lines.release(line_base, n);
        set_error("not enough free slab memory (%lld bytes needed)", slab_len * 4);
        return SG_ERR_OOM;
    }
    if (new_field) {
        fi = (int)b->fields.size();
        b->fields.push_back(f);
        b->field_base.push_back(b->next_brick);
        b->next_brick += f->nb;
    }
    ReqHost &rh = b->req[slot];
    rh.in_use = true;
    rh.listed = false;
    rh.gen += 1;
    rh.line_base = line_base;
    rh.n = n;
    rh.slab_off = slab_off;
    rh.slab_len = slab_len;
    rh.W = W;
    rh.field = fi;
    ReqDev R;
    memset(&R, 0, sizeof R);
    R.F = field_view(f, 0);
    for (int a = 0; a < 3; ++a) {
        R.dtc[a] = (float)(p->dt / f->desc.spacing[a]) * (p->direction == SG_DIR_BACKWARD ? -1.0f : 1.0f);
        R.origin_d[a] = f->desc.origin[a];
        R.spacing_d[a] = f->desc.spacing[a];
    }
    R.eps = p->eps;
    R.tie_cells = p->tie_cells;
    R.tie_eps_rel = p->tie_eps_rel;
    R.max_steps = (uint32_t)p->max_steps;
    R.W = (uint32_t)W;
    R.slab_base = slab_off;
    R.line_base = (uint32_t)line_base;
    R.n_lines = (uint32_t)n;
    R.brick_base = b->field_base[fi];
    R.dtype = f->desc.dtype;
    // the table entry is a plain host copy (pageable: the copy completes before this call returns)
    SG_CUDA(cudaMemcpyAsync(b->reqs + slot, &R, sizeof R, cudaMemcpyHostToDevice, s));
    SG_CUDA(cudaMemsetAsync(b->active + slot, 0, sizeof(uint32_t), s));
    if (n > 0) {
        SG_CUDA(cudaMemcpyAsync(b->seeds + 3 * line_base, xyz, sizeof(float) * 3 * (size_t)n, cudaMemcpyDefault, s));
        const int grid = (int)((n + 255) / 256 < b->ctx->sm_count * 16 ? (n + 255) / 256 : b->ctx->sm_count * 16);
        fill_u32_kernel<<<grid, 256, 0, s>>>(b->line_req + line_base, n, (uint32_t)slot);
        SG_CUDA(cudaGetLastError());
        batch_upload_kernel<<<grid, 256, 0, s>>>(batch_params(b), b->seeds, (uint32_t)slot, R);
        SG_CUDA(cudaGetLastError());
    }
    *request_id = ((int64_t)rh.gen << 20) | slot;
    return SG_OK;
}

extern "C" sg_status sg_batch_run(sg_batch *b, int32_t max_rounds, void *stream)
{
    SG_CHECK(b != nullptr, SG_ERR_INVALID_ARG, "batch is NULL");
    SG_CUDA(cudaSetDevice(b->ctx->device));
    cudaStream_t s = (cudaStream_t)stream;
    if (!b->exec) {
        sg_status st = build_batch_graph(b);
        if (st) return st;
    }
    batch_prepare_kernel<<<1, 32, 0, s>>>(b->ctrl, max_rounds > 0 ? (uint32_t)max_rounds : 0xffffffffu);
    SG_CUDA(cudaGetLastError());
    SG_CUDA(cudaGraphLaunch(b->exec, s));
    b->scanned_id = -1;
    return SG_OK;
}

extern "C" sg_status sg_batch_finished(sg_batch *b, int64_t *ids, int32_t cap, int32_t *count, void *stream)
{
    SG_CHECK(b && count && (cap <= 0 || ids), SG_ERR_INVALID_ARG, "NULL argument");
    SG_CUDA(cudaSetDevice(b->ctx->device));
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<uint32_t> act(b->req.size());
    Ctrl c;
    SG_CUDA(cudaMemcpyAsync(act.data(), b->active, sizeof(uint32_t) * act.size(), cudaMemcpyDeviceToHost, s));
    SG_CUDA(cudaMemcpyAsync(&c, b->ctrl, sizeof c, cudaMemcpyDeviceToHost, s));
    SG_CUDA(cudaStreamSynchronize(s));
    if (c.err & CTRL_ERR_TIMEOUT) {
        set_error("a record copy of the batch kernel did not complete in time");
        return SG_ERR_TIMEOUT;
    }
    int32_t k = 0;
    for (size_t i = 0; i < b->req.size() && k < cap; ++i) {
        ReqHost &r = b->req[i];
        if (r.in_use && !r.listed && act[i] == 0) {
            r.listed = true;
            ids[k++] = ((int64_t)r.gen << 20) | (int64_t)i;
        }
    }
    *count = k;
    return SG_OK;
}

extern "C" sg_status sg_batch_get_lines(sg_batch *b, int64_t request_id, int64_t *n_lines, int64_t *n_vertices,
                                        int64_t *offsets, float *vertices, uint8_t *status, float *margin,
                                        void *stream)
{
    SG_CHECK(b != nullptr, SG_ERR_INVALID_ARG, "batch is NULL");
    int slot;
    SG_CHECK(decode_id(b, request_id, &slot), SG_ERR_INVALID_ARG, "unknown request id %lld", (long long)request_id);
    SG_CUDA(cudaSetDevice(b->ctx->device));
    cudaStream_t s = (cudaStream_t)stream;
    const ReqHost &r = b->req[slot];
    const int sm = b->ctx->sm_count;
    if (b->scanned_id != request_id) {
        sg_status st = launch_compact_range(b->line_len + r.line_base, r.n, nullptr, r.W, nullptr, nullptr,
                                            b->block_sums, b->offsets, b->totals, nullptr, nullptr, nullptr, nullptr,
                                            sm, true, s);
        if (st) return st;
        b->scanned_id = request_id;
    }
    const bool query = !offsets && !vertices && !status && !margin;
    if (query || n_lines || n_vertices) {
        int64_t h[4];
        SG_CUDA(cudaMemcpyAsync(h, b->totals, sizeof h, cudaMemcpyDeviceToHost, s));
        SG_CUDA(cudaStreamSynchronize(s));
        if (n_lines) *n_lines = h[1];
        if (n_vertices) *n_vertices = h[0];
        if (query) return SG_OK;
    }
    for (const void *ptr : {(const void *)offsets, (const void *)vertices, (const void *)status, (const void *)margin}) {
        if (!ptr) continue;
        const int k = pointer_kind(ptr);
        SG_CHECK(k == PTR_DEVICE || k == PTR_PINNED, SG_ERR_INVALID_ARG,
                 "outputs must be device or page-locked host memory");
    }
    return launch_compact_range(b->line_len + r.line_base, r.n, b->slab + r.slab_off, r.W, b->line_status + r.line_base,
                                b->line_margin + r.line_base, b->block_sums, b->offsets, b->totals, offsets, vertices,
                                status, margin, sm, false, s);
}

extern "C" sg_status sg_batch_release(sg_batch *b, int64_t request_id, void *stream)
{
    SG_CHECK(b != nullptr, SG_ERR_INVALID_ARG, "batch is NULL");
    int slot;
    SG_CHECK(decode_id(b, request_id, &slot), SG_ERR_INVALID_ARG, "unknown request id %lld", (long long)request_id);
    SG_CUDA(cudaSetDevice(b->ctx->device));
    SG_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    ReqHost &r = b->req[slot];
    if (r.n > 0) {
        b->lines.release(r.line_base, r.n);
        b->slabs.release(r.slab_off, r.slab_len);
    }
    r.in_use = false;
    r.listed = false;
    if (b->scanned_id == request_id) b->scanned_id = -1;
    return SG_OK;
}
