// Internal state of a tracer and the launchers shared by its translation units.
#pragma once

#include "common.cuh"

namespace sg {

// Everything a streamline kernel needs, passed by value (__grid_constant__).
struct LineParams {
    DevField F;                  // field slot
    const float *seeds;          // n x 3 world (per-seed kernel)
    Particle *q;                 // brick-sorted queue of the round
    Particle *o;                 // outgoing records (hand-offs, re-queues)
    Particle *park;              // records that reached the step horizon
    Ctrl *ctrl;
    float *slab;                 // [line][W][3] world vertices
    uint32_t *line_len;          // vertices per line
    uint8_t *line_status;
    float *line_margin;
    long long W;                 // slab row stride in vertices: max_steps + 1 rounded up to a multiple of 4
    long long n_lines;
    long long n_seed;            // seeds uploaded: line l starts at seed l (l < n_seed) or l - n_seed
    long long n_fwd;             // lines [0, n_fwd) integrate forward, the rest backward (-dt)
    float dtc[3];                // dt / spacing: cells per unit velocity
    float eps;
    float tie_cells;
    float tie_eps_rel;
    uint32_t max_steps;
    uint32_t steps_per_round;
    uint32_t drain_steps;        // steps left to a warp's lanes once the round's queue is empty
    double origin_d[3];
    double spacing_d[3];
};

enum { EV_NONE = 0, EV_STOP = 1, EV_APPEND = 2, EV_PARK = 3 };

// The seed a line starts from, and its direction of integration (the step
// factor dt/h negated for backward lines: exact).
__device__ __forceinline__ long long seed_of(const LineParams &P, long long line)
{
    return line >= P.n_seed ? line - P.n_seed : line;
}

__device__ __forceinline__ void line_dtc(const LineParams &P, long long line, float dtc[3])
{
    const bool fwd = line < P.n_fwd;
#pragma unroll
    for (int a = 0; a < 3; ++a) dtc[a] = fwd ? P.dtc[a] : -P.dtc[a];
}

// One request of a batch (device copy).  Its lines occupy the global line
// slots [line_base, line_base + n_lines); its vertex slabs start at float
// slab_base of the batch's slab pool, W vertices per line.
struct ReqDev {
    DevField F;                  // slot 0 of the request's field
    float dtc[3];
    float eps;
    float tie_cells;
    float tie_eps_rel;
    uint32_t max_steps;
    uint32_t W;                  // slab row stride in vertices (max_steps + 1 rounded up to a multiple of 4)
    long long slab_base;
    uint32_t line_base;
    uint32_t n_lines;
    uint32_t brick_base;         // first global brick key of the request's field
    int dtype;
    double origin_d[3];          // the field's geometry in double (seed conversion)
    double spacing_d[3];
};

// Arguments of the binning kernels (counting sort of particle records by
// brick).  With line_req set, the key of a record is its request's
// brick_base plus its brick in the request's field; otherwise its brick in
// the single field (n, B).
struct BinArgs {
    const Particle *src;
    uint32_t *src_count;
    Particle *dst;
    uint32_t *brick_count;
    uint32_t *brick_cursor;
    Ctrl *ctrl;
    int n[3];
    int B[3];
    int nb;                      // number of keys
    const uint32_t *line_req;    // batch: request of each line slot (else NULL)
    const ReqDev *reqs;
    // partition over data (bricks owned by ranks): key = key_map[brick]; keys
    // [0, n_local) are this rank's bricks, the rest one per destination rank
    // (exports); the round's queue is the local keys' part
    const int *key_map;          // NULL: key = brick
    int n_local;                 // == nb without a key map
    uint32_t *key_start;         // start of every export key's segment [nb - n_local]
};

}  // namespace sg

struct sg_tracer {
    sg_context *ctx;
    sg_field *field;
    sg_tracer_params p;
    int64_t capacity;            // seeds
    int64_t n_seeds;
    int64_t n_lines;             // n_seeds, or 2 n_seeds for SG_DIR_BOTH
    int line_mult;               // lines per seed (1, or 2 for SG_DIR_BOTH)
    uint32_t *join_len;          // SG_DIR_BOTH: joined polyline lengths [capacity]
    int64_t *join_off;           // SG_DIR_BOTH: their offsets [capacity + 1]
    int64_t *join_tot;           // SG_DIR_BOTH: totals of the joined scan [4]
    char *ws;
    size_t ws_bytes;
    int nb;
    // streamline state
    float *seeds;
    float *slab;
    uint32_t *line_len;
    uint8_t *line_status;
    float *line_margin;
    sg::Particle *q;
    sg::Particle *o;
    sg::Particle *park;
    sg::Ctrl *ctrl;
    uint32_t *brick_count;
    uint32_t *brick_cursor;
    // compaction
    int64_t *offsets;            // capacity + 1
    unsigned long long *block_sums;
    int64_t *totals;             // [0] vertices, [1] lines, [2] steps
    int64_t *host_totals;        // page-locked copy of totals
    bool scanned;
    // readback into page-locked host memory: gather into device staging
    // buffers, copy each to the host on a second stream (double buffered)
    float *staging[2];
    size_t staging_bytes;
    cudaStream_t copy_stream;
    cudaEvent_t ev_gathered[2];
    cudaEvent_t ev_copied[2];
    // overlapped readout: the whole CSR gathered into device memory, then
    // copied to the host on copy_stream while the caller's stream moves on;
    // two staging buffers used in turn (the second only once it could be
    // allocated), so a readout waits for the copy of the one two back
    char *ovl_buf[2];            // device, grown on demand
    size_t ovl_bytes[2];
    cudaEvent_t ev_ovl_gathered;
    cudaEvent_t ev_ovl_copied[2];
    int ovl_next;                // staging buffer of the next readout
    int ovl_last;                // staging buffer of the last readout
    bool ovl_single;             // the second buffer could not be allocated
    // streaklines
    int64_t n_release;
    int32_t births;              // births released so far
    int32_t steps_done;          // advection steps done
    sg::Particle *sk_state;      // [release][inject] particle state (cell, frac, steps in .step)
    uint8_t *sk_status;          // [release][inject]
    float *sk_margin;            // [release][inject]
    uint32_t *sk_seglen;         // [release][inject]: run length at each run start, else 0
    // schedule
    int block;
    int grid;
    uint32_t horizon;            // step horizon of the next call
    bool traced;
    // partition over data: this rank advects the particles of its own bricks
    int pod_world;               // 0: every brick is local
    int pod_rank;
    int pod_local;               // bricks this rank owns (local binning keys)
    int *pod_key_map;            // device [nb]
    uint32_t *pod_key_start;     // device [pod_world]
    int64_t pod_queued;          // records in the local queue (host copy)
    int64_t pod_export_start[64];
    int64_t pod_export_count[64];
    // CUDA graph of the round loop
    cudaGraph_t graph;
    cudaGraphExec_t exec;
    bool graph_ready;
};

namespace sg {

// Row stride (vertices) of a streamline or path-line tracer's vertex slab:
// max_steps + 1 rounded up to a multiple of 4, so that every run of four
// vertices starting at a multiple of 4 is 48 bytes at a 16-byte boundary.
inline long long slab_stride(int32_t max_steps) { return ((long long)max_steps + 4) / 4 * 4; }

// Whether a streamline tracer with these parameters runs the decoupled-lane
// advection kernel on this field.
bool decoupled_lanes(const sg_tracer_params *p, const sg_field *f);

sg_status launch_upload(sg_tracer *t, cudaStream_t s);
sg_status launch_join_scan(sg_tracer *t, cudaStream_t s);
sg_status launch_join(sg_tracer *t, int64_t *offsets, float *vertices, int64_t *seed_vertex, cudaStream_t s);
sg_status launch_per_seed(sg_tracer *t, cudaStream_t s);
sg_status launch_bin(sg_tracer *t, Particle *src, uint32_t *src_count, cudaStream_t s, bool in_graph,
                     unsigned long long cond_handle, int mode);
sg_status launch_bin_args(const BinArgs &A, int sm_count, cudaStream_t s, bool in_graph, unsigned long long cond_handle,
                          int mode);
sg_status launch_compact_range(const uint32_t *len, long long n, const float *slab, long long W, const uint8_t *st_in,
                               const float *mg_in, unsigned long long *block_sums, int64_t *dev_offsets,
                               int64_t *totals, int64_t *offsets_out, float *vertices, uint8_t *status_out,
                               float *margin_out, int sm_count, bool scan_only, cudaStream_t s);
sg_status launch_round(sg_tracer *t, cudaStream_t s);
sg_status prepare_round(sg_tracer *t);
sg_status launch_prepare_call(sg_tracer *t, uint32_t horizon, uint32_t max_rounds, cudaStream_t s);
sg_status launch_park_rest(sg_tracer *t, cudaStream_t s);
sg_status launch_carry(sg_tracer *t, cudaStream_t s);
sg_status launch_iota(int32_t *dst, int64_t n, int64_t period, cudaStream_t s);
sg_status launch_fill_inf(float *dst, long long n, cudaStream_t s);
sg_status launch_set_q_count(Ctrl *ctrl, uint32_t n, cudaStream_t s);
sg_status streak_upload(sg_tracer *t, cudaStream_t s);
sg_status path_upload(sg_tracer *t, cudaStream_t s);
sg_status path_step(sg_tracer *t, int32_t n_steps, int32_t *any_active, cudaStream_t s);
sg_status streak_step(sg_tracer *t, int32_t n_steps, int32_t *any_active, cudaStream_t s);
sg_status launch_scan_lengths(sg_tracer *t, cudaStream_t s);
sg_status launch_gather_lines(sg_tracer *t, int64_t *offsets, float *vertices, uint8_t *status, float *margin,
                              cudaStream_t s);
sg_status launch_gather_chunk(const sg_tracer *t, long long a, long long b, long long base, float *dst, cudaStream_t s);
sg_status launch_streak_release(sg_tracer *t, int birth, cudaStream_t s);
sg_status launch_streak_scan(sg_tracer *t, cudaStream_t s);
sg_status launch_streak_gather(sg_tracer *t, int64_t *offsets, float *vertices, uint8_t *status, float *margin,
                               int32_t *source, cudaStream_t s);
LineParams line_params(const sg_tracer *t);

}  // namespace sg
