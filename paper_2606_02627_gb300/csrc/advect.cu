// Streamline advection kernels.
//
//  * round_kernel: the persistent form.  Each warp pops particles from the
//    brick-sorted queue of the round (warp-aggregated atomics on one cursor),
//    advances each lane by RK4 steps inside its brick, and refills lanes whose
//    particle stopped, left the brick or used its steps for the round
//    (__ballot_sync / __shfl_sync).  A particle that leaves its brick is
//    appended to the outgoing buffer, from which the binning kernels build the
//    destination bricks' queues for the next round: the paper's emitOutgoing /
//    particle forwarding (Sec. 3.1.2) as an exchange inside one GPU.
//  * per_step_kernel: Listing 1 as written: one thread per particle, one RK4
//    step per launch, every particle emitted to the queue of its destination
//    brick (which may be its own).
//  * per_seed_kernel: one thread per seed to termination on the global float3
//    field; no bricks, no queues.
//  * upload_kernel: seeds to particles; writes each line's first vertex.
//
// RK4 (Listing 1): k1 = dt v(P0), P1 = P0 + k1/2, k2 = dt v(P1),
// P2 = P0 + k2/2, k3 = dt v(P2), P3 = P0 + k3, k4 = dt v(P3),
// P' = P0 + (k1 + 2 k2 + 2 k3 + k4)/6, with v in cells per unit time.
#include <math.h>

#include "rk4.cuh"

namespace sg {

__device__ __forceinline__ void write_vertex(const LineParams &P, uint32_t line, uint32_t step, const int c[3],
                                             const float f[3])
{
    float *o = P.slab + ((long long)line * P.W + step) * 3;
    st_na(o, fmaf(P.F.spacing[0], (float)c[0] + f[0], P.F.origin[0]));
    st_na(o + 1, fmaf(P.F.spacing[1], (float)c[1] + f[1], P.F.origin[1]));
    st_na(o + 2, fmaf(P.F.spacing[2], (float)c[2] + f[2], P.F.origin[2]));
}

__device__ __forceinline__ uint8_t stop_code(const LineParams &P, int st, float margin)
{
    return stop_code_t(st, margin, P.tie_cells, P.tie_eps_rel);
}

// ------------------------------------------------------------------ persistent round kernel

template <int DT, int LAYOUT>
__global__ void __launch_bounds__(256) round_kernel(const __grid_constant__ LineParams P)
{
    const unsigned lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    const uint32_t q_count = P.ctrl->q_count;
    const uint32_t horizon = P.ctrl->horizon;
    bool active = false;
    bool drained = q_count == 0;
    uint32_t drain_left = P.drain_steps;   // warp-uniform; counts down once the queue is empty
    int c[3] = {0, 0, 0};
    float f[3] = {0.f, 0.f, 0.f};
    uint32_t line = 0, step = 0, here = 0;
    float dtc[3] = {0.f, 0.f, 0.f};          // dt/h of this lane's line (negated backward)
    BrickRef<DT> br;
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
                    brick_of<DT>(P.F, c, br);
                    line_dtc(P, line, dtc);
                    active = true;
                    here = 0;
                }
            }
        }
        if (__ballot_sync(SG_FULL_MASK, active) == 0) break;
        // the queue is empty: give the warp's runs a few more steps, then hand
        // them to the next round instead of holding the round open
        if (drained) {
            if (drain_left == 0) here = P.steps_per_round;
            else --drain_left;
        }

        int ev = EV_NONE, st = SG_LINE_ACTIVE;
        float margin = INFINITY;
        if (active) {
            if (step >= horizon) {
                if (step >= P.max_steps) {
                    ev = EV_STOP;
                    st = SG_LINE_MAXSTEPS;
                } else {
                    ev = EV_PARK;
                }
            } else if (here >= P.steps_per_round) {
                ev = EV_APPEND;
            } else {
                st = rk4_bricked<DT, LAYOUT>(P.F, dtc, P.eps, br, c, f, margin);
                if (st != SG_LINE_ACTIVE) {
                    ev = EV_STOP;
                } else {
                    ++step;
                    ++here;
                    write_vertex(P, line, step, c, f);
                    if (step >= horizon) {
                        if (step >= P.max_steps) {
                            ev = EV_STOP;
                            st = SG_LINE_MAXSTEPS;
                        } else {
                            ev = EV_PARK;
                        }
                    } else if (c[0] < br.lo[0] || c[0] >= br.hi[0] || c[1] < br.lo[1] || c[1] >= br.hi[1] ||
                               c[2] < br.lo[2] || c[2] >= br.hi[2]) {
                        ev = EV_APPEND;       // destinationID(new position) != this brick
                    }
                }
            }
        }
        warp_append(ev == EV_APPEND, P.o, &P.ctrl->o_count, c, f, line, step);
        warp_append(ev == EV_PARK, P.park, &P.ctrl->p_count, c, f, line, step);
        if (ev == EV_STOP) {
            P.line_len[line] = step + 1;
            P.line_status[line] = stop_code(P, st, margin);
            P.line_margin[line] = margin;
        } else if (ev == EV_PARK) {
            P.line_len[line] = step + 1;
        }
        if (ev != EV_NONE) active = false;
    }
}

// ------------------------------------------------------------------ persistent round kernel, decoupled lanes

// Consecutive passes a lane may wait for one record copy (each pass of a warp
// takes at least ~100 cycles: well over a second in all).
constexpr unsigned COPY_WAIT_PASSES = 1u << 24;

// Shared memory of the decoupled-lane kernel, per thread, in this order over
// the block: every storage type interpolates an FP32 record (6 chunks of 16 B)
// in the lane's slot, followed by a 16-byte pad; the 8-byte formats' 64-byte
// records land in a separate area and are decoded into the slot once, when
// the copy lands (that area's fifth chunk holds the brick scale and the eps^2
// threshold); the vertex staging area holds four 16-byte vertices, then the
// line's slab row pointer, the first vertex this lane writes and a brick
// extent; then one 8-byte mbarrier.  Every stride is a multiple of 16 bytes
// and an odd number of 16-byte chunks, so that the 16-byte accesses of eight
// consecutive lanes fall in eight different bank groups.
template <int DT>
struct AsyncLayout {
    static constexpr int NCH = Record<SG_F32>::chunks;                 // chunks of the FP32 record
    static constexpr int RAW = Record<DT>::chunks;                     // chunks one copy brings
    static constexpr unsigned SLOT = (NCH + 1) * 16;
    static constexpr unsigned LAND = (DT == SG_F32) ? 0u : (RAW + 1) * 16;
    static constexpr unsigned VBUF = 80;
    static constexpr unsigned BAR = 8;
    static constexpr unsigned PER_THREAD = SLOT + LAND + VBUF + BAR;
};

// The same round as round_kernel for the CELL8 layout, with the lanes of a
// warp no longer waiting for one another at each sample.  In round_kernel
// every one of the four samples of a step is a load that the whole warp
// waits for, so the warp runs at the pace of its slowest lane: at nearly
// every sample some lane has just entered a cell whose record is not in L1.
//
// Here each lane keeps the record of the cell of its current sample point in
// its own shared-memory slot.  A pass of the warp's loop runs the four RK4
// stages in order, unrolled: iteration s runs stage s for every lane that is
// at stage s and holds the record its sample point needs, so a lane that
// starts the pass at stage 0 completes a whole step, and the end of the step
// (new P0, vertex, brick test) runs for those lanes together.  When a stage
// point falls in another cell (about one sample in seventeen at h = 0.5
// cell), the lane starts one bulk copy of that record by the TMA engine
// (cp.async.bulk) into its slot, completing on its own mbarrier, and sits out
// the rest of the pass; the next pass it resumes at that stage.  The per-pass
// bookkeeping (refill vote, copy completion, hand-off appends) is shared by
// the up to four stages of a pass.  A slot is the record plus 16 bytes of
// padding (112 bytes for FP32, 80 for the 8-byte formats): with that stride
// the 16-byte reads of eight consecutive lanes fall in eight different bank
// groups.  The stage arithmetic is rk4_bricked's, operation for operation, so
// both kernels produce the same bits.
//
// Vertices leave in 48-byte runs: every lane of a warp ends its step in the
// same iteration, and three scattered 4-byte stores per lane at that point
// (one per component, 32 lines at once) stall the load/store pipe that the
// next stage's slot reads go through.  Instead each lane stages its line's
// vertices in shared memory (16 bytes per vertex, four of them) and writes
// the four vertices of a slab row position 4j .. 4j+3 as three 16-byte
// stores once the last of them is done (slab rows are a multiple of four
// vertices long, so such a run starts at a 16-byte boundary).  Vertices of a
// run that another lane (or the upload) wrote, and the vertices of an
// unfinished run when the particle leaves the lane, go out as 4-byte stores.
template <int DT>
__global__ void __launch_bounds__(256, 3) round_async_kernel(const __grid_constant__ LineParams P)
{
    using L = AsyncLayout<DT>;
    constexpr int NCH = L::NCH, RAW = L::RAW;
    constexpr unsigned SLOT = L::SLOT, LAND = L::LAND, VBUF = L::VBUF;
    extern __shared__ uint4 slots[];
    const unsigned tid = threadIdx.x, nthr = blockDim.x;
    const unsigned lane = tid & 31;
    uint4 *my_slot = slots + tid * (SLOT / 16);
    uint4 *my_land = slots + nthr * (SLOT / 16) + tid * (LAND / 16);
    uint4 *vbuf = slots + nthr * ((SLOT + LAND) / 16) + tid * (VBUF / 16);
    const uint32_t bar = smem_addr(reinterpret_cast<uint64_t *>(slots + nthr * ((SLOT + LAND + VBUF) / 16)) + tid);
    const uint32_t slot = smem_addr(DT == SG_F32 ? my_slot : my_land);   // where a copy lands
    mbar_init(bar, 1);
    mbar_init_fence();
    __syncwarp();

    const DevField &F = P.F;
    // the round's queue length and step horizon: constant while the kernel
    // runs, read where they are needed (refills, particle events) rather than
    // held in registers across the loop
    const uint32_t *q_count_p = &P.ctrl->q_count;
    const uint32_t *horizon_p = &P.ctrl->horizon;
    bool active = false, pending = false;
    bool inflight = false;                                 // a copy may still land in the slot
    bool drained = __ldg(q_count_p) == 0;
    // one pass per step once a lane's records are at hand
    uint32_t drain_left = P.drain_steps;
    unsigned parity = 0, waited = 0;
    int c[3] = {0, 0, 0}, q[3] = {0, 0, 0};               // P0 and the current sample point
    float f[3] = {0.f, 0.f, 0.f}, g[3] = {0.f, 0.f, 0.f};
    // k1 and k2 (k2 + k3 after stage 2) and the step factor, per component.
    // The stage arithmetic and this state are scalar: with the x and y
    // components carried across the unrolled stages as packed register pairs,
    // about one step in 500 came out one unit in the last place away from
    // rk4_bricked's result; scalar they give its bits, at the same speed.  The
    // interpolation keeps its packed pairs.
    float k1x = 0.f, k1y = 0.f, k1z = 0.f;
    float k23x = 0.f, k23y = 0.f, k23z = 0.f;
    float dsx = 0.f, dsy = 0.f, dsz = 0.f;
    uint32_t line = 0, step = 0, stage = 0;
    // steps the lane may take before its step horizon or the round's step
    // budget stops it: min(horizon - step, steps_per_round - steps this round)
    int left = 0;
    uint32_t held = 0xffffffffu;                           // cell of the record in (or on its way to) the slot
    bool rec_bad = false;                                  // FX21: a corner of the slot's record is flagged
    BrickRef<DT> br;
    br.data = nullptr;
    br.scale = 1.0f;
    for (int a = 0; a < 3; ++a) br.lo[a] = br.hi[a] = 0;
    // the record index of cell q in the brick is q.z C1 C0 + q.y C0 + q.x + cbase;
    // the brick's first owned cell and its extent (lo, span per axis) sit in
    // the 16-byte pad after the lane's record slot (the bulk copy writes only
    // the record) and in the vertex staging area: the per-step brick test
    // reads them there
    int cbase = 0;
    // cells [box_lo, box_lo + box_span] per axis lie inside the domain's
    // cells (not on its last sample layer) and inside the brick's ghost
    // shell: a stage point there needs neither the EXIT nor the HALO test
    int box_lo[3] = {0, 0, 0};
    unsigned box_span[3] = {0u, 0u, 0u};

    // the cell of sample point q within the brick's records
    auto cell_of = [&]() { return (uint32_t)((q[2] * F.C[1] + q[1]) * F.C[0] + q[0] + cbase); };
    // copy the record of `cell` into the slot
    auto fetch = [&](uint32_t cell) {
        bulk_copy_arrive(slot, br.data + (long long)cell * record_elems<DT>(), RAW * 16u, bar);
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
                    const uint32_t horizon = __ldg(horizon_p);
                    load_particle(P.q + my, c, f, line, step);
                    brick_of<DT>(F, c, br);
                    float dtc[3];
                    line_dtc(P, line, dtc);
                    float ds[3];
#pragma unroll
                    for (int a = 0; a < 3; ++a) {
                        ds[a] = (DT == SG_F32) ? dtc[a] : __fmul_rn(dtc[a], br.scale);
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
                        box_lo[a] = lo;
                        box_span[a] = hi >= lo ? (unsigned)(hi - lo) : 0u;
                        if (hi < lo) box_lo[a] = 0x7fffffff;   // empty: every point takes the full tests
                    }
                    if constexpr (DT != SG_F32) {
                        // |v|^2 at or above e2min (before the brick scale) means |v| >= eps
                        const float e = __fdiv_ru(P.eps, br.scale);
                        my_land[RAW] = make_uint4(__float_as_uint(__fmul_ru(e, e)), __float_as_uint(br.scale), 0u, 0u);
                    }
                    {
                        const unsigned long long row =
                            reinterpret_cast<unsigned long long>(P.slab + (long long)line * P.W * 3);
                        const uint32_t sp0 = (uint32_t)(br.hi[0] - br.lo[0]), sp1 = (uint32_t)(br.hi[1] - br.lo[1]);
                        vbuf[4] = make_uint4((uint32_t)row, (uint32_t)(row >> 32), step + 1,
                                             (uint32_t)(br.hi[2] - br.lo[2]));
                        my_slot[NCH] = make_uint4((uint32_t)br.lo[0], (uint32_t)br.lo[1], (uint32_t)br.lo[2],
                                                  sp0 | (sp1 << 16));
                        cbase = -(((br.lo[2] - 1) * F.C[1] + (br.lo[1] - 1)) * F.C[0] + (br.lo[0] - 1));
                    }
                    left = step >= horizon ? 0 : (int)min(horizon - step, P.steps_per_round);
                    active = true;
                    stage = 0;
                    fetch(cell_of());                // another brick: the slot's record is stale
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
                if constexpr (DT != SG_F32) {
                    // decode the landed record once into the FP32 slot, one x face at a
                    // time: corner (dx, dy, dz) is sample dx of raw chunk dy + 2 dz, and
                    // its component a goes to f32_record_index(a, dx, dy, dz)
                    unsigned flags = 0u;
#pragma unroll
                    for (int dx = 0; dx < 2; ++dx) {
                        float3 cr[4];                // (dy, dz) = (0,0), (1,0), (0,1), (1,1)
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            const uint4 w = my_land[j];
                            const uint2 e = dx ? make_uint2(w.z, w.w) : make_uint2(w.x, w.y);
                            cr[j] = decode_elem<DT>(e);
                            flags |= elem_flag<DT>(e);
                        }
                        my_slot[dx] = make_uint4(__float_as_uint(cr[0].x), __float_as_uint(cr[2].x),
                                                 __float_as_uint(cr[1].x), __float_as_uint(cr[3].x));
                        my_slot[2 + dx] = make_uint4(__float_as_uint(cr[0].y), __float_as_uint(cr[2].y),
                                                     __float_as_uint(cr[1].y), __float_as_uint(cr[3].y));
                        my_slot[4 + dx] = make_uint4(__float_as_uint(cr[0].z), __float_as_uint(cr[2].z),
                                                     __float_as_uint(cr[1].z), __float_as_uint(cr[3].z));
                    }
                    rec_bad = flags != 0u;
                }
            } else if (++waited >= COPY_WAIT_PASSES) {
                // the particle is dropped and the call fails; the warp takes
                // no other particle while this lane's barrier may still complete
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
            if (step >= __ldg(horizon_p)) {
                if (step >= P.max_steps) {
                    ev = EV_STOP;
                    st = SG_LINE_MAXSTEPS;
                } else {
                    ev = EV_PARK;
                }
            } else {
                ev = EV_APPEND;                   // the round's step budget is spent
            }
            go = false;
        }
        // the four stages; iteration S runs stage S: sample, k = v dt/h, and
        // the next point P0 + k1/2, P0 + k2/2, P0 + k3 or P'
#pragma unroll
        for (int S = 0; S < 4; ++S) {
            if (go && stage == (uint32_t)S) {
                Record<SG_F32> R;
#pragma unroll
                for (int k = 0; k < NCH; ++k) R.r[k] = my_slot[k];
                bool bad_flag;                       // a non-finite corner (FX21: a flagged one)
                const float3 v = interp_record<SG_F32>(R, g[0], g[1], g[2], bad_flag);
                if constexpr (DT == SG_FX21) bad_flag = rec_bad;
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
                // |v|^2 of the stage-0 sample, and of any sample whose values may
                // not be finite: a non-finite component makes it non-finite
                float s2 = 0.f;
                bool maybe_bad;
                if constexpr (DT == SG_FX21) {
                    maybe_bad = bad_flag;
                    if (S == 0)
                        s2 = __fadd_rn(__fadd_rn(__fmul_rn(v.x, v.x), __fmul_rn(v.y, v.y)), __fmul_rn(v.z, v.z));
                } else {
                    s2 = __fadd_rn(__fadd_rn(__fmul_rn(v.x, v.x), __fmul_rn(v.y, v.y)), __fmul_rn(v.z, v.z));
                    maybe_bad = !(s2 < INFINITY);
                }
                float e2 = 0.f;
                if (S == 0) e2 = (DT == SG_F32) ? __fmul_ru(P.eps, P.eps) : __uint_as_float(my_land[RAW].x);
                if (maybe_bad || (S == 0 && !(s2 >= e2)) || !in_box) {
                    // the tests in full (rare): a sample that may not be finite, a
                    // speed that may be below eps, a point near the domain or
                    // brick boundary
                    const bool bad = (DT == SG_FX21) ? bad_flag : bad3(v);
                    float sp = sqrtf(s2);
                    if (DT != SG_F32) sp = __fmul_rn(sp, __uint_as_float(my_land[RAW].y));
                    if (bad) {
                        st = SG_LINE_NANFIELD;
                    } else if (S == 0 && sp < P.eps) {
                        margin = (P.eps - sp) / P.eps;
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
                    vbuf[step & 3u] = make_uint4(__float_as_uint(fmaf(F.spacing[0], (float)c[0] + f[0], F.origin[0])),
                                                 __float_as_uint(fmaf(F.spacing[1], (float)c[1] + f[1], F.origin[1])),
                                                 __float_as_uint(fmaf(F.spacing[2], (float)c[2] + f[2], F.origin[2])),
                                                 0u);
                    run_done = (step & 3u) == 3u;
                    stage = 0;
                    const uint4 bl = my_slot[NCH];
                    const bool out = (unsigned)(c[0] - (int)bl.x) >= (bl.w & 0xffffu) ||
                                     (unsigned)(c[1] - (int)bl.y) >= (bl.w >> 16) ||
                                     (unsigned)(c[2] - (int)bl.z) >= vbuf[4].w;
                    if (left <= 0 || out) {
                        go = false;
                        if (step >= __ldg(horizon_p)) {
                            ev = step >= P.max_steps ? EV_STOP : EV_PARK;
                            st = step >= P.max_steps ? SG_LINE_MAXSTEPS : st;
                        } else {
                            // destinationID(new position) != this brick, or the
                            // round's step budget is spent
                            ev = EV_APPEND;
                        }
                    }
                } else {
                    stage = S + 1;
                }
                if (go) {
                    // the record of the next sample point q
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
            warp_append(ev == EV_PARK, P.park, &P.ctrl->p_count, c, f, line, step);
            if (ev == EV_STOP) {
                P.line_len[line] = step + 1;
                P.line_status[line] = stop_code(P, st, margin);
                P.line_margin[line] = margin;
            } else if (ev == EV_PARK) {
                P.line_len[line] = step + 1;
            }
            if (ev != EV_NONE) active = false;
        }
    }
    // only after a copy wait ran out can one be in flight: wait for it once
    // more, again with a limit, before the slot's memory is released
    for (unsigned i = 0; inflight && i < COPY_WAIT_PASSES; ++i)
        if (mbar_done(bar, parity)) inflight = false;
}

// ------------------------------------------------------------------ Listing 1: one launch per step

template <int DT, int LAYOUT>
__global__ void __launch_bounds__(256) per_step_kernel(const __grid_constant__ LineParams P)
{
    const uint32_t q_count = P.ctrl->q_count;
    const uint32_t horizon = P.ctrl->horizon;
    const uint32_t stride = gridDim.x * blockDim.x;
    // warp-uniform trip count: each warp takes 32 consecutive particles per pass
    for (uint32_t base = (blockIdx.x * blockDim.x + threadIdx.x) & ~31u; base < q_count; base += stride) {
        const uint32_t idx = base + (threadIdx.x & 31);
        const bool valid = idx < q_count;
        int c[3] = {0, 0, 0};
        float f[3] = {0.f, 0.f, 0.f};
        uint32_t line = 0, step = 0;
        int ev = EV_NONE, st = SG_LINE_ACTIVE;
        float margin = INFINITY;
        if (valid) {
            load_particle(P.q + idx, c, f, line, step);       // getIncoming(particleID)
            if (step >= horizon) {
                if (step >= P.max_steps) {
                    ev = EV_STOP;
                    st = SG_LINE_MAXSTEPS;
                } else {
                    ev = EV_PARK;
                }
            } else {
                BrickRef<DT> br;
                brick_of<DT>(P.F, c, br);
                float dtc[3];
                line_dtc(P, line, dtc);
                st = rk4_bricked<DT, LAYOUT>(P.F, dtc, P.eps, br, c, f, margin);
                if (st != SG_LINE_ACTIVE) {
                    ev = EV_STOP;
                } else {
                    ++step;
                    write_vertex(P, line, step, c, f);
                    if (step >= P.max_steps) {
                        ev = EV_STOP;
                        st = SG_LINE_MAXSTEPS;
                    } else {
                        ev = (step >= horizon) ? EV_PARK : EV_APPEND;   // emitOutgoing(p, destinationID(P'))
                    }
                }
            }
        }
        warp_append(ev == EV_APPEND, P.o, &P.ctrl->o_count, c, f, line, step);
        warp_append(ev == EV_PARK, P.park, &P.ctrl->p_count, c, f, line, step);
        if (ev == EV_STOP) {
            P.line_len[line] = step + 1;
            P.line_status[line] = stop_code(P, st, margin);
            P.line_margin[line] = margin;
        } else if (ev == EV_PARK) {
            P.line_len[line] = step + 1;
        }
    }
}

// ------------------------------------------------------------------ per-seed kernel (global float3 field)

// Trilinear sample of the global float3 AoS array at cell c, fraction f (a
// point inside the domain).  On the upper face (c = dims-1, f = 0) the upper
// corner repeats the last sample, as a brick's clamped ghost layer does, so the
// sample is that sample exactly.
__device__ __forceinline__ float3 sample_global(const float *__restrict__ Fg, const DevField &F, const int c[3],
                                                const float f[3])
{
    const long long sy = 3ll * F.dims[0], sz = sy * F.dims[1];
    const long long x0 = 3ll * c[0], x1 = 3ll * min(c[0] + 1, F.nm1[0]);
    const long long y0 = sy * c[1], y1 = sy * min(c[1] + 1, F.nm1[1]);
    const long long z0 = sz * c[2], z1 = sz * min(c[2] + 1, F.nm1[2]);
    float r[3];
#pragma unroll
    for (int comp = 0; comp < 3; ++comp) {
        const float *b = Fg + comp;
        const float v000 = __ldg(b + z0 + y0 + x0), v100 = __ldg(b + z0 + y0 + x1);
        const float v010 = __ldg(b + z0 + y1 + x0), v110 = __ldg(b + z0 + y1 + x1);
        const float v001 = __ldg(b + z1 + y0 + x0), v101 = __ldg(b + z1 + y0 + x1);
        const float v011 = __ldg(b + z1 + y1 + x0), v111 = __ldg(b + z1 + y1 + x1);
        r[comp] = lerpf(lerpf(lerpf(v000, v100, f[0]), lerpf(v010, v110, f[0]), f[1]),
                        lerpf(lerpf(v001, v101, f[0]), lerpf(v011, v111, f[0]), f[1]), f[2]);
    }
    return make_float3(r[0], r[1], r[2]);
}

// One RK4 step (Listing 1) on the global array, with rk4_bricked's operations
// in the same order: stage points are formed relative to the particle's cell,
// so the position keeps ~2^-24 cells of rounding anywhere in the grid.
__device__ __forceinline__ int rk4_global(const float *__restrict__ Fg, const DevField &F, const float ds[3], float eps,
                                          int c[3], float f[3], float &margin)
{
    float3 v = sample_global(Fg, F, c, f);
    if (bad3(v)) return SG_LINE_NANFIELD;
    const float sp = sqrtf(__fadd_rn(__fadd_rn(__fmul_rn(v.x, v.x), __fmul_rn(v.y, v.y)), __fmul_rn(v.z, v.z)));
    if (sp < eps) {
        margin = (eps - sp) / eps;
        return SG_LINE_STAGNANT;
    }
    float k[4][3];
    const float w[3] = {0.5f, 0.5f, 1.0f};     // P1, P2 = P0 + k/2; P3 = P0 + k3
    int q[3];
    float g[3];
#pragma unroll
    for (int s = 0; s < 3; ++s) {
        k[s][0] = __fmul_rn(v.x, ds[0]);
        k[s][1] = __fmul_rn(v.y, ds[1]);
        k[s][2] = __fmul_rn(v.z, ds[2]);
#pragma unroll
        for (int a = 0; a < 3; ++a) locate(f[a], w[s] * k[s][a], c[a], q[a], g[a]);
        if (!in_domain(F, q, g)) {
            margin = out_dist(F, q, g);
            return SG_LINE_EXIT;
        }
        v = sample_global(Fg, F, q, g);
        if (bad3(v)) return SG_LINE_NANFIELD;
    }
    k[3][0] = __fmul_rn(v.x, ds[0]);
    k[3][1] = __fmul_rn(v.y, ds[1]);
    k[3][2] = __fmul_rn(v.z, ds[2]);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float d = __fmul_rn(__fadd_rn(__fadd_rn(k[0][a], k[3][a]), __fmul_rn(2.0f, __fadd_rn(k[1][a], k[2][a]))),
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

// A grid-stride loop over the seeds: the grid sets how many seeds are in
// flight per SM (as for the persistent kernel), each thread traces its seeds
// one after the other to termination.
__global__ void __launch_bounds__(256) per_seed_kernel(const __grid_constant__ LineParams P)
{
    const float *Fg = reinterpret_cast<const float *>(P.F.data);
    const DevField &F = P.F;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < P.n_lines;
         i += (long long)gridDim.x * blockDim.x) {
        // seed to cell + fraction, converted in double precision (as the upload)
        const float *sd = P.seeds + 3 * seed_of(P, i);
        float ds[3];
        line_dtc(P, i, ds);
        double p[3];
        bool inside = true;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            p[a] = ((double)sd[a] - P.origin_d[a]) / P.spacing_d[a];
            inside = inside && (p[a] >= 0.0 && p[a] <= (double)F.nm1[a]);
        }
        if (!inside) {
            P.line_len[i] = 0;
            P.line_status[i] = SG_LINE_OUT;
            P.line_margin[i] = INFINITY;
            continue;
        }
        int c[3];
        float f[3];
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
        float *out = P.slab + (long long)i * P.W * 3;
        out[0] = sd[0];
        out[1] = sd[1];
        out[2] = sd[2];
        uint32_t step = 0;
        int st = SG_LINE_MAXSTEPS;
        float margin = INFINITY;
        while (step < P.max_steps) {
            const int r = rk4_global(Fg, F, ds, P.eps, c, f, margin);
            if (r != SG_LINE_ACTIVE) {
                st = r;
                break;
            }
            ++step;
            float *o = out + 3ll * step;
            st_na(o, fmaf(F.spacing[0], (float)c[0] + f[0], F.origin[0]));
            st_na(o + 1, fmaf(F.spacing[1], (float)c[1] + f[1], F.origin[1]));
            st_na(o + 2, fmaf(F.spacing[2], (float)c[2] + f[2], F.origin[2]));
        }
        P.line_len[i] = step + 1;
        P.line_status[i] = stop_code(P, st, margin);
        P.line_margin[i] = margin;
    }
}

// ------------------------------------------------------------------ seed upload

__global__ void upload_kernel(const __grid_constant__ LineParams P)
{
    const long long n = P.n_lines;
    const unsigned lane = threadIdx.x & 31;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long base = (long long)blockIdx.x * blockDim.x + threadIdx.x - lane; base < n; base += stride) {
        const long long i = base + lane;
        bool keep = false;
        int c[3] = {0, 0, 0};
        float f[3] = {0.f, 0.f, 0.f};
        if (i < n) {
            const float *sd = P.seeds + 3 * seed_of(P, i);
            double p[3];
            bool inside = true;
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                p[a] = ((double)sd[a] - P.origin_d[a]) / P.spacing_d[a];
                inside = inside && (p[a] >= 0.0 && p[a] <= (double)P.F.nm1[a]);
            }
            if (!inside) {
                P.line_len[i] = 0;
                P.line_status[i] = SG_LINE_OUT;
                P.line_margin[i] = INFINITY;
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
                float *o = P.slab + (long long)i * P.W * 3;
                o[0] = sd[0];
                o[1] = sd[1];
                o[2] = sd[2];
                P.line_len[i] = 1;
                P.line_status[i] = SG_LINE_ACTIVE;
                P.line_margin[i] = INFINITY;
                keep = true;
            }
        }
        warp_append(keep, P.park, &P.ctrl->p_count, c, f, (uint32_t)i, 0u);
    }
}

// ------------------------------------------------------------------ launchers

sg_status launch_upload(sg_tracer *t, cudaStream_t s)
{
    LineParams P = line_params(t);
    if (t->p.kernel == SG_KERNEL_PER_SEED) return SG_OK;   // the per-seed kernel reads the seeds itself
    int grid = (int)((t->n_lines + 255) / 256);
    if (grid > t->ctx->sm_count * 16) grid = t->ctx->sm_count * 16;
    if (grid < 1) grid = 1;
    upload_kernel<<<grid, 256, 0, s>>>(P);
    SG_CUDA(cudaGetLastError());
    return SG_OK;
}

sg_status launch_per_seed(sg_tracer *t, cudaStream_t s)
{
    LineParams P = line_params(t);
    if (t->n_lines == 0) return SG_OK;
    const int block = t->block;
    long long grid = (t->n_lines + block - 1) / block;
    if (grid > t->grid) grid = t->grid;
    per_seed_kernel<<<(unsigned)grid, block, 0, s>>>(P);
    SG_CUDA(cudaGetLastError());
    return SG_OK;
}

// The decoupled-lane form runs for the CELL8 layout when every brick spans
// fewer than 2^16 cells per axis (it keeps two of its spans in 16-bit
// halves); SG_KERNEL_LOCKSTEP, the other layouts and larger bricks take
// round_kernel, which gives the same bits.
static bool spans_fit(const DevField &F)
{
    for (int a = 0; a < 3; ++a) {
        const long long last = (long long)F.dims[a] - (long long)(F.B[a] - 1) * F.n[a];
        if (F.n[a] >= 65536 || last >= 65536) return false;
    }
    return true;
}

static bool use_async(int kernel, int layout, const DevField &F)
{
    return kernel == SG_KERNEL_PERSISTENT && layout == SG_LAYOUT_CELL8 && spans_fit(F);
}

bool decoupled_lanes(const sg_tracer_params *p, const sg_field *f)
{
    return use_async(p->kernel, f->desc.layout, f->geom);
}

// dynamic shared memory of the decoupled-lane kernel (AsyncLayout)
template <int DT>
static size_t async_smem(int block)
{
    return (size_t)block * AsyncLayout<DT>::PER_THREAD;
}

template <int DT, int LAYOUT>
static void launch_round_t(const LineParams &P, int grid, int block, int kernel, cudaStream_t s)
{
    if (kernel == SG_KERNEL_PER_STEP) per_step_kernel<DT, LAYOUT><<<grid, block, 0, s>>>(P);
    else if (use_async(kernel, LAYOUT, P.F)) round_async_kernel<DT><<<grid, block, async_smem<DT>(block), s>>>(P);
    else round_kernel<DT, LAYOUT><<<grid, block, 0, s>>>(P);
}

// The lockstep and Listing-1 kernels use no shared memory: ask for the whole
// unified L1/shared array as L1, which holds the particles' current cell
// records.  The decoupled-lane kernel asks for the smallest shared part that
// holds its record slots at the tracer's blocks per SM.
template <int DT, int LAYOUT>
static cudaError_t prefer_l1_t(int kernel, int block, int blocks_per_sm, const DevField &F)
{
    if (kernel == SG_KERNEL_PER_STEP)
        return cudaFuncSetAttribute(per_step_kernel<DT, LAYOUT>, cudaFuncAttributePreferredSharedMemoryCarveout, 0);
    if (use_async(kernel, LAYOUT, F)) {
        const size_t per_block = async_smem<DT>(block);
        cudaError_t e = cudaFuncSetAttribute(round_async_kernel<DT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)per_block);
        if (e != cudaSuccess) return e;
        const size_t total = per_block * (size_t)blocks_per_sm + 1024 * (size_t)blocks_per_sm;
        int pct = (int)((total * 100 + 228 * 1024 - 1) / (228 * 1024));
        if (pct > 100) pct = 100;
        return cudaFuncSetAttribute(round_async_kernel<DT>, cudaFuncAttributePreferredSharedMemoryCarveout, pct);
    }
    return cudaFuncSetAttribute(round_kernel<DT, LAYOUT>, cudaFuncAttributePreferredSharedMemoryCarveout, 0);
}

sg_status prepare_round(sg_tracer *t)
{
    if (t->p.kernel == SG_KERNEL_PER_SEED) {
        SG_CUDA(cudaFuncSetAttribute(per_seed_kernel, cudaFuncAttributePreferredSharedMemoryCarveout, 0));
        return SG_OK;
    }
    cudaError_t e = cudaSuccess;
    with_dtype(t->field->desc.dtype, [&](auto D) {
        with_layout(t->field->desc.layout,
                    [&](auto Lay) {
                        e = prefer_l1_t<decltype(D)::value, decltype(Lay)::value>(
                            t->p.kernel, t->block, t->grid / t->ctx->sm_count, t->field->geom);
                    });
    });
    SG_CUDA(e);
    return SG_OK;
}

sg_status launch_round(sg_tracer *t, cudaStream_t s)
{
    LineParams P = line_params(t);
    const int k = t->p.kernel;
    bool ok = false;
    with_dtype(t->field->desc.dtype, [&](auto D) {
        ok = with_layout(t->field->desc.layout, [&](auto Lay) {
            launch_round_t<decltype(D)::value, decltype(Lay)::value>(P, t->grid, t->block, k, s);
        });
    });
    SG_CHECK(ok, SG_ERR_UNSUPPORTED, "no advection kernel for dtype %d layout %d", t->field->desc.dtype,
             t->field->desc.layout);
    SG_CUDA(cudaGetLastError());
    return SG_OK;
}

}  // namespace sg
