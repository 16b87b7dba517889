/*
 * streamgb — field-line advection on one GB300 (sm_103a), C ABI.
 *
 * The calls follow the problem statement of Zellmann et al., "Streami: An MPI
 * Data-Parallel Library to Compute Field Lines on GPUs":
 *   - a vector field made of macrocells (here: bricks) with a halo, created
 *     per brick or from a global array (Sec. 3.1.1, Sec. 3.3);
 *   - seeds given as positions, each tracked by a unique ID (Sec. 3.1.2);
 *   - step / trace / getLines of the Tracer (Sec. 3.2, Fig. 4, Listing 2),
 *     in streamline, streakline or path-line mode (the Mode enumeration of
 *     Fig. 4, with path lines added).
 *
 * Conventions
 *   - Every call returns sg_status: SG_OK (0) or a negative error.  No call
 *     throws or aborts.  sg_last_error() gives a message for the last error
 *     raised on the calling host thread.
 *   - Handles are opaque.  Large device buffers are owned by the caller: each
 *     *_required_bytes query comes before the matching *_create, which carves
 *     its state out of the caller's buffer and allocates no device memory of
 *     its own (except the CUDA graph objects of a tracer).  The caller keeps
 *     the buffer alive until the handle is destroyed.
 *   - Streams are cudaStream_t passed as void* (0 = legacy default stream).
 *     A call is asynchronous on its stream unless it says otherwise; it
 *     returns before the GPU work ends.  Host pointers given to an
 *     asynchronous call must stay valid until the stream reaches that point.
 *   - Positions are world coordinates, float32 xyz triples (AoS).  Index
 *     space: world = origin + spacing * index per axis; the sampled domain is
 *     the closed box [0, dims-1] per axis.
 *   - "host or device" pointers are classified with cudaPointerGetAttributes.
 *     Pointers that a kernel writes or reads directly must be device memory or
 *     page-locked host memory (cudaHostAlloc / cudaHostRegister); pageable
 *     host memory is accepted only where the argument says so.
 */
#ifndef STREAMGB_H
#define STREAMGB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t sg_status;

enum {
    SG_OK = 0,
    SG_ERR_INVALID_ARG = -1,   /* a NULL handle, a bad size, an unsupported combination */
    SG_ERR_OOM = -2,           /* the caller's buffer is smaller than *_required_bytes */
    SG_ERR_CUDA = -3,          /* a CUDA runtime call failed; see sg_last_error */
    SG_ERR_ROUND_LIMIT = -4,   /* a trace hit its round cap with particles left */
    SG_ERR_TIMEOUT = -5,       /* a bounded wait ran out */
    SG_ERR_STATE = -6,         /* the call does not fit the object's state */
    SG_ERR_UNSUPPORTED = -7    /* not built for this mode / dtype / layout */
};

/* Field storage type.  SG_F32 stores the samples as given; SG_BF16 and SG_F16
 * store code = round-to-nearest-even(v / s_b) with one scale s_b per brick,
 * s_b the smallest power of two >= the largest finite |component| among the
 * brick's stored samples (ghosts included), and decode as code * s_b.
 * SG_FX21 stores the three components as 21-bit signed fixed-point integers
 * q = round-to-nearest-even(v / s_b * 2^20), clamped to +-(2^20 - 1), packed
 * with a non-finite flag in the same 8 bytes a BF16 sample takes (x: bits
 * 0-20, y: bits 21-41, flag: bit 42, z: bits 43-63, each as q + 2^20); it
 * decodes as q * s_b * 2^-20 (the per-brick scale it reports is that quantum),
 * an absolute error of at most s_b * 2^-21, and a sample with a non-finite
 * component decodes as NaN.  Interpolation and integration are FP32 in every
 * case. */
enum { SG_F32 = 0, SG_BF16 = 1, SG_F16 = 2, SG_FX21 = 3 };

/* Sample layout inside a brick.  A LINEAR or TILED4 sample is x, y, z and one
 * pad: 16 B in FP32, 8 B in BF16/FP16 (FX21: three 21-bit components and a
 * flag in 8 B).  LINEAR is x-fastest; TILED4 groups 4x4x4 samples
 * contiguously (tile-major, x-fastest inside a tile).  CELL8 stores, for every
 * cell of the brick (ghost cells included, (n+2)^3 of them), the eight corner
 * samples of that cell contiguously, so that one interpolation reads one
 * record instead of eight scattered samples: a 96-B FP32 record holds the 24
 * components without padding (x, then y, then z; each as the four corners of
 * the cell's x = 0 face, then the four of its x = 1 face, in (y, z) order
 * (0,0), (0,1), (1,0), (1,1)); a 64-B record of an 8-byte format holds the
 * eight samples in corner order (x fastest, then y, then z). */
enum { SG_LAYOUT_LINEAR = 0, SG_LAYOUT_TILED4 = 1, SG_LAYOUT_CELL8 = 2 };

/* Line status (uint8 per line).  Bit 7 (SG_LINE_TIE) marks a boundary tie: a
 * line that stopped by EXIT with its offending point less than tie_cells
 * outside the domain, or by STAGNANT with (eps - |v|)/eps < tie_eps_rel. */
enum {
    SG_LINE_ACTIVE = 0,    /* not stopped yet (after sg_tracer_step)          */
    SG_LINE_MAXSTEPS = 1,  /* reached max_steps                                */
    SG_LINE_EXIT = 2,      /* a stage point or the new position left the domain */
    SG_LINE_STAGNANT = 3,  /* |v(P0)| < eps in world units, before a step       */
    SG_LINE_NANFIELD = 4,  /* a sample was not finite                           */
    SG_LINE_OUT = 5,       /* the seed lies outside the domain (no vertex)      */
    SG_LINE_HALO = 6,      /* a stage point left the brick's ghost shell: dt *
                              max speed exceeded one cell                        */
    SG_LINE_TIE = 0x80
};

/* Line modes (Fig. 4's Mode): streamlines in a steady field; streaklines
 * (one release per seed per step, Sec. 3.2); path lines: every seed released
 * once at time 0 and followed through the time-dependent field, one vertex
 * per step (the paper notes they follow from the same machinery, Sec. 3.2).
 * Streak and path lines advance with sg_tracer_step and sample a field whose
 * time slices are streamed into resident slots (sg_field_stream_slice). */
enum { SG_STREAMLINE = 0, SG_STREAKLINE = 1, SG_PATHLINE = 2 };

/* Direction of streamline integration (the paper's Tracer advects forward
 * only; backward lines follow -v, the same RK4 with -dt).  With
 * SG_DIR_BOTH a tracer holds two lines per seed: line i forward and line
 * n + i backward from seed i (n seeds uploaded); sg_tracer_get_joined joins
 * them into one polyline through the seed. */
enum { SG_DIR_FORWARD = 0, SG_DIR_BACKWARD = 1, SG_DIR_BOTH = 2 };

/* Advection kernel of a streamline tracer. */
enum {
    SG_KERNEL_PERSISTENT = 0,  /* bricked field; persistent warps refill lanes from
                                  per-brick queues; rounds run as one CUDA graph  */
    SG_KERNEL_PER_SEED = 1,    /* one thread per seed to termination on a global
                                  FP32 field (layout SG_FIELD_GLOBAL only)         */
    SG_KERNEL_PER_STEP = 2,    /* Listing 1: one launch per advection step, one
                                  thread per particle, forwarding between launches */
    SG_KERNEL_LOCKSTEP = 3     /* the persistent kernel with the lanes of a warp in
                                  lockstep (every sample a load the warp waits
                                  for).  SG_KERNEL_PERSISTENT on a CELL8 field
                                  decouples the lanes instead: each holds its
                                  current cell record and fetches the next one
                                  asynchronously; both give the same bits.    */
};

typedef struct sg_context sg_context;
typedef struct sg_field sg_field;
typedef struct sg_tracer sg_tracer;
typedef struct sg_batch sg_batch;

/* Copies the last error message of the calling thread into buf (NUL-terminated,
 * truncated to n bytes).  Returns the length of the full message. */
size_t sg_last_error(char *buf, size_t n);

/* Library version: major * 10000 + minor * 100 + patch. */
int32_t sg_version(void);

/* ------------------------------------------------------------------ context */

/* Makes `device` current and records its properties (SM count, shared memory,
 * L2 size).  One context per device; it holds no device memory. */
sg_status sg_context_create(int32_t device, sg_context **out);
sg_status sg_context_destroy(sg_context *ctx);
/* Number of SMs of the context's device (for grid sizing by callers). */
sg_status sg_context_sm_count(const sg_context *ctx, int32_t *out);

/* -------------------------------------------------------------------- field */

/* A structured vector field on a uniform grid, split into a uniform grid of
 * bricks (the paper's macrocells, Sec. 3.1.1 and Sec. 3.3).
 *
 * Brick b = (bx, by, bz) owns n = ceil((dims-1)/bricks) cells per axis, the
 * index interval [b*n, b*n+n), and the last brick also the upper face; a
 * position on an interior face belongs to the upper brick (this is the
 * field's destinationID).  Each brick stores the samples b*n-1 .. b*n+n+1
 * (n+3 per axis, clamped to [0, dims-1]): the owned cells plus a one-cell
 * ghost shell, the macrocell's halo.  A step whose displacement is at most
 * one cell (dt * max speed <= 1) samples only its own brick.
 *
 * layout SG_FIELD_GLOBAL (bricks must be 1x1x1, dtype SG_F32) instead keeps
 * the paper's plain float3 AoS voxel array, sampled by offsets into it; it
 * is the field of SG_KERNEL_PER_SEED.
 *
 * n_slots resident copies (time slices) share the geometry; steady fields
 * use 1.  Unsteady fields map time slice s (time s * slice_dt) to slot
 * s % n_slots when it is streamed in. */
enum { SG_FIELD_GLOBAL = 16 };

typedef struct {
    int64_t dims[3];      /* samples per axis, each >= 2                        */
    double origin[3];     /* world position of sample (0, 0, 0)                 */
    double spacing[3];    /* world distance between samples, > 0                */
    int32_t bricks[3];    /* bricks per axis, >= 1; the last brick must own a cell */
    int32_t ghost;        /* ghost layers; must be 1                            */
    int32_t dtype;        /* SG_F32, SG_BF16, SG_F16                            */
    int32_t layout;       /* SG_LAYOUT_LINEAR / _TILED4 / _CELL8, SG_FIELD_GLOBAL */
    int32_t n_slots;      /* resident slices, >= 1                              */
    double slice_dt;      /* time between slices (unsteady fields), > 0         */
} sg_field_desc;

/* Device bytes needed by a field with this description (all slots plus a
 * staging area of one global FP32 slice for streamed slices). */
sg_status sg_field_required_bytes(const sg_field_desc *desc, size_t *bytes);

/* Creates a field in the caller's device buffer `storage` of `bytes` bytes
 * (256-byte aligned).  The field does not own the buffer. */
sg_status sg_field_create(sg_context *ctx, const sg_field_desc *desc, void *storage, size_t bytes,
                          sg_field **out);
sg_status sg_field_destroy(sg_field *f);

/* Owned cells per brick per axis (n above). */
sg_status sg_field_brick_cells(const sg_field *f, int64_t n_out[3]);

/* Sets slot `slot` from a global FP32 AoS array [dims2][dims1][dims0][3]
 * (device or page-locked host memory): cuts the bricks, fills the ghost
 * shells and encodes BF16/FP16 with per-brick scales.  The paper's setField
 * with a structured field of float3 voxels (Sec. 3.2, Sec. 3.3), here cut
 * into the macrocells with their halos (Sec. 3.1.1) by the library.
 * Errors: SG_ERR_INVALID_ARG for a NULL pointer or a slot out of range,
 * SG_ERR_CUDA for a failed launch or copy.  Asynchronous. */
sg_status sg_field_set_global(sg_field *f, int32_t slot, const float *vec3, void *stream);

/* Sets one brick of slot `slot` from its own (n+3)^3 FP32 AoS samples,
 * ghost shell included, as the application holds it (device or page-locked
 * host memory); samples are those at global indices b*n-1 .. b*n+n+1 per
 * axis, which the caller clamps (or fills) at the domain faces itself.  This
 * is the paper's per-rank field creation: each macrocell's data with its
 * user-defined halo, assembled by the application from its own
 * decomposition (Sec. 3.1.1, Sec. 3.2).  Errors: SG_ERR_INVALID_ARG for a
 * brick or slot out of range or a NULL pointer, SG_ERR_CUDA for a failed
 * launch or copy.  Asynchronous. */
sg_status sg_field_set_brick(sg_field *f, int32_t slot, int32_t bx, int32_t by, int32_t bz,
                             const float *vec3_with_halo, void *stream);

/* Streams time slice `slice` from page-locked host memory (global FP32 AoS)
 * into slot slice % n_slots on `stream`, and records that the slot holds the
 * slice once the stream reaches the end of the copy.  A tracer step that
 * needs the slice waits for it on its own stream (cudaStreamWaitEvent).  The
 * paper's unsteady input: one field per time step, set with setField(f,
 * timeStep) and selected by the simulation time in step() (Sec. 3.2, Listing
 * 2).  Errors: SG_ERR_INVALID_ARG for pageable or NULL memory or a negative
 * slice, SG_ERR_CUDA for a failed copy.  Asynchronous. */
sg_status sg_field_stream_slice(sg_field *f, int32_t slice, const float *pinned_host, void *stream);

/* Largest |v / spacing| over the stored (decoded) samples of `slot`, in cells
 * per unit time; dt = h / max_speed makes every step at most h cells.
 * Synchronous on `stream`. */
sg_status sg_field_max_speed(sg_field *f, int32_t slot, double *cells_per_time, void *stream);

/* Copies brick (bx,by,bz) of `slot` back in a canonical form (z, y, x,
 * component order): FP32 stores give (n+3)^3*3 floats, BF16/FP16 stores
 * (n+3)^3*3 uint16 codes, FX21 stores (n+3)^3*3 int32 codes q (INT32_MIN in
 * every component of a sample flagged non-finite), and the brick scale.
 * `out` is host memory of at least (n+3)^3*3*(4, 2 or 4) bytes.  Synchronous. */
sg_status sg_field_read_brick(sg_field *f, int32_t slot, int32_t bx, int32_t by, int32_t bz,
                              void *out, float *scale, void *stream);

/* ------------------------------------------------------------------- tracer */

typedef struct {
    int32_t mode;          /* SG_STREAMLINE or SG_STREAKLINE                       */
    int32_t kernel;        /* SG_KERNEL_* (streamlines)                             */
    double dt;             /* time step (k_i = dt * v / spacing, in cells)          */
    int32_t max_steps;     /* streamlines: steps per line (>= 0)                    */
    float eps;             /* stop when |v(P0)| < eps (world units); 1e-6 typical   */
    float tie_cells;       /* tie threshold for EXIT (cells); 0 turns ties off      */
    float tie_eps_rel;     /* tie threshold for STAGNANT (relative)                 */
    int32_t inject_steps;  /* streaklines: particles released per release point     */
    /* schedule of the persistent kernel (0 = default) */
    int32_t block_size;    /* threads per CTA (multiple of 32, <= 256: the kernels'
                              register budget)                                   */
    int32_t blocks_per_sm; /* CTAs per SM of the persistent grid                     */
    int32_t steps_per_round; /* steps a particle may take in one round before it is
                                re-queued in its own brick (0 = default: for the
                                decoupled-lane kernel 1024 when the capacity is at
                                least 4 x SMs x 768 particles, else 256; 128 for
                                the other kernels)                                  */
    int32_t max_rounds;    /* round cap of one trace / step call (0 = max_steps + 2,
                              which only a fault can reach).  A call stopped by it
                              returns (or its sg_tracer_check reports)
                              SG_ERR_ROUND_LIMIT; its lines stay consistent: every
                              particle left keeps the vertices written so far
                              (status SG_LINE_ACTIVE, length = steps + 1) and the
                              next trace / step call continues it             */
    int32_t drain_steps;   /* once a warp finds the round's queue empty, its lanes take
                              at most this many more steps before re-queueing their
                              particles for the next round: shortens the end of a
                              round at the price of more rounds.  0 = library
                              default (128 for the decoupled-lane kernel, no limit
                              otherwise); negative = no limit                      */
    int32_t direction;     /* SG_DIR_* (streamlines; 0 = forward)                   */
    int32_t brick_window;  /* rounds policy of the persistent kernels (streamlines):
                              0 = every round advances the particles of all
                              bricks; w > 0 = brick-major: a round advances only
                              the particles of w consecutive bricks (round-robin
                              over the bricks, skipping empty ones) and carries
                              the others to the next round, so that a round's
                              field accesses stay within w bricks (L2 locality
                              for fields larger than L2).  The lines are the same
                              bits either way.  Ignored by SG_KERNEL_PER_STEP and
                              by partitioned tracers.                            */
} sg_tracer_params;

/* Fills p with the defaults (streamline, persistent kernel, eps 1e-6,
 * tie_cells 1e-3, tie_eps_rel 1e-3, automatic schedule). */
sg_status sg_tracer_params_default(sg_tracer_params *p);

/* Device bytes of a tracer for up to `capacity` seeds (streamlines) or
 * release points (streaklines): particle queues, the per-line vertex slabs
 * (capacity * W * 12 B for streamlines and path lines, W = max_steps + 1
 * rounded up to a multiple of 4, so that runs of four vertices are 48 bytes at
 * a 16-byte boundary), per-line lengths and status, and the scan scratch of
 * the compaction. */
sg_status sg_tracer_required_bytes(const sg_context *ctx, const sg_field *f, const sg_tracer_params *p,
                                   int64_t capacity, size_t *bytes);

sg_status sg_tracer_create(sg_context *ctx, sg_field *f, const sg_tracer_params *p, int64_t capacity,
                           void *workspace, size_t bytes, sg_tracer **out);
sg_status sg_tracer_destroy(sg_tracer *t);

/* Seeds (streamlines) or release points (streaklines): n world xyz float32
 * triples, host (pageable or page-locked) or device memory; n <= capacity.
 * Line i is seed i (the unique particle ID of Sec. 3.1.2).  Bins the seeds
 * into per-brick queues and writes each line's first vertex; a seed outside
 * the domain gets status SG_LINE_OUT and no vertex.  Streaklines release
 * birth 0 at every release point.  Resets any previous trace.  Asynchronous. */
sg_status sg_tracer_upload_seeds(sg_tracer *t, const float *xyz, int64_t n, void *stream);

/* Advances by n_steps steps (Listing 2's step(), called n_steps times):
 * streamlines advance every active line by up to n_steps more steps;
 * streaklines advance every released particle by one step of the time-
 * dependent field and then release the next birth, n_steps times; path
 * lines advance every moving line by one step of the time-dependent field
 * (step j from time (j-1) dt to j dt), n_steps times or until max_steps.
 * Streak and path steps need the slices of their stage times resident
 * (SG_ERR_STATE otherwise).  any_active (nullable, host) receives 1 if a
 * particle can still move; when it is non-NULL the call synchronises the
 * stream.  Returns SG_ERR_ROUND_LIMIT if the round cap stopped the call
 * early. */
sg_status sg_tracer_step(sg_tracer *t, int32_t n_steps, int32_t *any_active, void *stream);

/* Streamlines: advances until every line has stopped (Sec. 3.2's trace()).
 * The persistent kernel runs as one CUDA graph launch whose conditional
 * while-node repeats rounds until the queues are empty.  Asynchronous;
 * sg_tracer_check reports a round-cap stop afterwards. */
sg_status sg_tracer_trace(sg_tracer *t, void *stream);

/* Synchronises `stream` and returns SG_ERR_ROUND_LIMIT if a previous
 * asynchronous trace stopped at its round cap, else SG_OK.  rounds (nullable)
 * receives the number of rounds of the last trace. */
sg_status sg_tracer_check(sg_tracer *t, int32_t *rounds, void *stream);

/* Measurement form of sg_tracer_trace: the same kernels on the same data, but
 * the rounds are driven from the host with a CUDA event pair around every
 * advection-kernel launch, so that the kernel's own time can be read (event
 * record nodes cannot sit inside the graph's while-node).  Synchronous.
 * kernel_ms receives the summed advection-kernel time, launches the number of
 * advection-kernel launches (both nullable).  When round_ms and
 * round_particles are given (host arrays of max_records entries), round r's
 * kernel time and the particles its queue started with are stored for
 * r < max_records. */
sg_status sg_tracer_trace_timed(sg_tracer *t, double *kernel_ms, int32_t *launches, float *round_ms,
                                uint32_t *round_particles, int32_t max_records, void *stream);

/* Line readback (getLines of Fig. 4), compacted to CSR: line i's vertices
 * are vertices[offsets[i] .. offsets[i+1]) (world xyz float32).  For
 * streamlines there is one line per seed; for streaklines one line per run of
 * consecutive live particles of a release point, oldest birth first, and
 * line_source gives its release point.  Two calls: with offsets and vertices
 * NULL it only returns n_lines and n_vertices (synchronising the stream);
 * then with buffers of n_lines+1 int64 offsets, 3*n_vertices floats, n_lines
 * status bytes, n_lines float margins and n_lines int32 sources (each
 * nullable, device or page-locked host memory).  margin: EXIT distance
 * outside (cells), STAGNANT relative margin, else +inf.  Asynchronous when
 * the buffers are given. */
sg_status sg_tracer_get_lines(sg_tracer *t, int64_t *n_lines, int64_t *n_vertices, int64_t *offsets,
                              float *vertices, uint8_t *status, float *margin, int32_t *line_source,
                              void *stream);

/* Overlapped line readback into page-locked host memory (streamline and
 * path-line tracers): the same CSR as sg_tracer_get_lines, but the copy to
 * the host runs on the tracer's own copy stream, so that work enqueued on
 * `stream` after this call (the next upload and trace, which may reuse every
 * tracer buffer) overlaps it.  The call synchronises `stream` (the sizes are
 * read), gathers the CSR into device staging memory owned by the tracer
 * (grown on demand, freed by sg_tracer_destroy) on `stream`, and returns
 * without waiting for the copy.  The tracer keeps two staging buffers of
 * the CSR's size and uses them in turn, so that the gather of one readout
 * does not wait for the copy of the one before (if the second cannot be
 * allocated, the first serves every readout).  n_lines / n_vertices (host, nullable)
 * receive the sizes; with every buffer NULL the call stops there.  Buffers
 * (each nullable, page-locked host memory, else SG_ERR_INVALID_ARG): n_lines+1
 * int64 offsets, 3*n_vertices floats, n_lines status bytes, n_lines float
 * margins, as in sg_tracer_get_lines.  They are complete once a stream made
 * to wait by sg_tracer_wait_lines has reached that point; a later overlapped
 * readout waits (on `stream`) for the copy of the readout that last used the
 * same staging buffer before reusing it.  SG_ERR_STATE for streakline
 * tracers. */
sg_status sg_tracer_get_lines_overlapped(sg_tracer *t, int64_t *n_lines, int64_t *n_vertices, int64_t *offsets,
                                         float *vertices, uint8_t *status, float *margin, void *stream);

/* Makes `stream` wait for the host copies of the last
 * sg_tracer_get_lines_overlapped (no wait if there was none); synchronising
 * `stream` afterwards guarantees the host buffers are complete.  Does not
 * block the host.  SG_ERR_STATE for streakline tracers. */
sg_status sg_tracer_wait_lines(sg_tracer *t, void *stream);

/* Bidirectional readback (SG_DIR_BOTH): one polyline per seed, the backward
 * line reversed (the seed not repeated) followed by the forward line, so that
 * polyline i runs along the flow through seed i.  Two calls, as
 * sg_tracer_get_lines: with offsets and vertices NULL it only returns n_lines
 * (= seeds) and n_vertices (synchronising the stream); then with device
 * buffers of n_lines+1 int64 offsets, 3*n_vertices floats and n_lines int64
 * seed_vertex (nullable: the index of the seed within its polyline, -1 for
 * an OUT seed).  Per-direction status and margin come from
 * sg_tracer_get_lines (lines i and n + i).  SG_ERR_STATE unless the tracer
 * was created with SG_DIR_BOTH; asynchronous when the buffers are given. */
sg_status sg_tracer_get_joined(sg_tracer *t, int64_t *n_lines, int64_t *n_vertices, int64_t *offsets,
                               float *vertices, int64_t *seed_vertex, void *stream);

/* Successful RK4 steps of the current trace summed over all lines (the unit of
 * the particle-steps/s metric).  Synchronous. */
sg_status sg_tracer_total_steps(sg_tracer *t, int64_t *steps, void *stream);

/* ------------------------------------------------- partition over data (POD) */

/* The paper's data-parallel mode (Sec. 3.1.2, Listing 2): the bricks of the
 * field are owned by ranks (one GPU each); a rank advects the particles of
 * its own bricks, and the particles that leave them are forwarded to the
 * owning ranks between rounds (emitOutgoing + an all-to-all exchange), until
 * a reduction finds no particle left anywhere.  These calls are the rank-local
 * side; the exchange and the reduction are the caller's (NCCL or gloo
 * all-to-all-v, paper_2606_02627_gb300/pod.py).  Records are the library's
 * 32-byte particle records (fraction 3 x f32, line u32, cell 3 x i32, step
 * u32), exchanged as opaque bytes between tracers with the same field
 * geometry and parameters.  Lines are assembled by merging every rank's line
 * buffers (sg_tracer_line_buffers): slab by elementwise minimum (each vertex
 * is written by one rank, the others hold +inf), length and status by
 * maximum, margin by minimum.  Synchronous where stated. */

/* Before sg_tracer_upload_seeds: brick_owner (host, one entry per brick of
 * the field, linear brick index (bz * By + by) * Bx + bx) gives each brick's
 * rank in [0, world); this tracer is rank `rank`; world <= 64.  Every rank
 * then uploads every seed (each keeps the seeds in its own bricks); trace and
 * step are refused while a partition is set (SG_ERR_STATE). */
sg_status sg_tracer_pod_setup(sg_tracer *t, const int32_t *brick_owner, int32_t rank, int32_t world);

/* After the upload: sorts this rank's particles into its local queue;
 * *local_count (host, nullable) receives its length.  Synchronous. */
sg_status sg_tracer_pod_begin(sg_tracer *t, int64_t *local_count, void *stream);

/* One round over the local queue, then the sort of the round's outgoing
 * particles: the local queue of the next round, and one export segment per
 * other rank.  local_count (host, nullable) and export_counts (host, world
 * entries, nullable; 0 for this rank) receive the sizes.  Synchronous. */
sg_status sg_tracer_pod_round(sg_tracer *t, int64_t *local_count, int64_t *export_counts, void *stream);

/* Copies the export segment of rank `dest` (export_counts[dest] records of
 * 32 B) into records (device).  Call for every destination before any
 * import of the same round. */
sg_status sg_tracer_pod_export(sg_tracer *t, int32_t dest, void *records, void *stream);

/* Appends count records (device, 32 B each, all in this rank's bricks) to
 * the local queue of the next round. */
sg_status sg_tracer_pod_import(sg_tracer *t, const void *records, int64_t count, void *stream);

/* Length of the local queue (host bookkeeping, no synchronisation). */
sg_status sg_tracer_pod_queued(const sg_tracer *t, int64_t *count);

/* Device pointers of the tracer's line buffers inside its workspace (each
 * nullable): slab (n_lines x max_vertices x 3 floats; max_vertices is the
 * row stride, max_steps + 1 rounded up to a multiple of 4), length (u32),
 * status (u8), margin (f32).  For merging the ranks' partial lines; the next
 * sg_tracer_get_lines rescans them. */
sg_status sg_tracer_line_buffers(sg_tracer *t, float **slab, uint32_t **length, uint8_t **status, float **margin,
                                 int64_t *n_lines, int64_t *max_vertices);

/* ------------------------------------------------------ unstructured fields */

/* The second field type of Sec. 3.3: an unstructured mesh of tetrahedra,
 * pyramids, prisms (wedges) and hexahedra with the velocity at its vertices,
 * interpolated with each cell's isoparametric shape functions (VTK vertex
 * orders: tet 0-3; pyramid base 0-3, apex 4; wedge triangles 0-2 and 3-5;
 * hexahedron bottom 0-3, top 4-7).  A point lies in a cell when the
 * parametric solution of sum N_i(r) x_i = p (Newton's method in FP32) maps
 * back onto p and lies in the cell's reference domain within tau.  Cells are
 * found through a bounding volume hierarchy built on the host at creation
 * (median splits, at most 4 cells per leaf).  Steady streamlines in world
 * coordinates: RK4 of Listing 1, one thread per particle in rounds of at
 * most 128 steps (sg_umesh_trace); a stage point or new
 * position in no cell stops the line (EXIT, margin = how far outside the
 * particle's cell, in parametric units). */
typedef struct sg_umesh sg_umesh;
enum { SG_CELL_TET = 4, SG_CELL_PYRAMID = 5, SG_CELL_PRISM = 6, SG_CELL_HEX = 8 };

/* Workspace bytes of a mesh of n_cells cells (256 B per cell record, 32 B per
 * cell of hierarchy: at most one node per cell, 4 B of index). */
sg_status sg_umesh_required_bytes(int64_t n_cells, size_t *bytes);

/* vertices, velocity: host, n_vertices x 3 floats (world); cell_vertices,
 * cell_offsets (n_cells + 1), cell_types (SG_CELL_*, the vertex count): host;
 * tau: containment tolerance (0: 1e-5); workspace: device, 256-byte aligned,
 * sg_umesh_required_bytes, kept alive by the caller.  Synchronous (the
 * hierarchy is built on the host).  SG_ERR_INVALID_ARG on a bad type, count
 * or index. */
sg_status sg_umesh_create(sg_context *ctx, const float *vertices, const float *velocity, int64_t n_vertices,
                          const int32_t *cell_vertices, const int64_t *cell_offsets, const uint8_t *cell_types,
                          int64_t n_cells, float tau, void *workspace, size_t bytes, sg_umesh **out);
sg_status sg_umesh_destroy(sg_umesh *m);

/* Velocity at n world points (device, 3 floats each; NaN where no cell
 * contains the point) and the containing cell's index (device, nullable, -1
 * for none).  Asynchronous. */
sg_status sg_umesh_sample(sg_umesh *m, const float *points, int64_t n, float *velocity, int64_t *cell, void *stream);

/* Streamlines from n seeds (device, world; n < 2^31): line i's vertices go
 * to slab + 3 i (max_steps + 1) (device), its vertex count to length[i], its
 * status (SG_LINE_*, tie bit for EXIT margins < 1e-3) and margin likewise
 * (all device).  The particles advance in rounds of at most 128 steps; with
 * max_steps above 128 the call takes its two particle queues (128 B per
 * seed) from the device's stream-ordered memory pool on `stream`
 * (cudaMallocAsync) and returns them there.  Compact with sg_lines_compact.
 * Asynchronous. */
sg_status sg_umesh_trace(sg_umesh *m, const float *seeds, int64_t n, double dt, int32_t max_steps, float eps,
                         float *slab, uint32_t *length, uint8_t *status, float *margin, void *stream);

/* ------------------------------------------------------- seed-shape kernels */

/* Seed points from control shapes, generated on the device (the low-level
 * interface's convenience kernels for seeds placed uniformly on lines and
 * planes, Sec. 3.1).  World coordinates; positions are computed in double
 * precision with explicit round-to-nearest operations and rounded once to
 * float32.  out: device or page-locked host memory, 3 floats per point
 * (x, y, z), caller-owned.  Asynchronous on stream; SG_ERR_INVALID_ARG on
 * NULL vectors, negative counts or an unusable out pointer. */

/* n points evenly spaced on the segment a..b, both ends included
 * (point i at a + (b - a) i / (n - 1); n = 1 gives a). */
sg_status sg_seeds_rake(const double a[3], const double b[3], int64_t n, float *out, void *stream);

/* nu x nv points evenly spaced on the parallelogram origin + s u + t v,
 * s, t in [0, 1] (s = i / (nu - 1), t = j / (nv - 1)); point (i, j) at index
 * j nu + i. */
sg_status sg_seeds_plane(const double origin[3], const double u[3], const double v[3], int64_t nu, int64_t nv,
                         float *out, void *stream);

/* n points uniform at random in the box [lo, hi] (per axis): coordinate c of
 * point i is lo + (hi - lo) u with u the top 53 bits of value 3i + c of the
 * counter-based SplitMix64 stream (seed, stream_id) (Steele, Lea, Flood
 * 2014: value k = mix64(key + (k + 1) G), key = mix64(seed G +
 * 0x632BE59BD9B4E019 (stream_id + 1)), G = 0x9E3779B97F4A7C15). */
sg_status sg_seeds_box(const double lo[3], const double hi[3], int64_t n, uint64_t seed, uint64_t stream_id,
                       float *out, void *stream);

/* -------------------------------------------------------------- request batch */

/* Continuous batching of streamline requests over resident fields: the
 * serving form of the paper's interactive seed-placement application
 * (Sec. 4), where seed regions arrive while earlier ones are being traced.
 * Requests (seeds + tracer parameters + one resident field) are admitted
 * while line slots and slab memory are free, and their particles share the
 * per-brick queues and the persistent kernel of one CUDA-graph launch per
 * sg_batch_run; a request's lines are read back as soon as its last line
 * stops, and its memory then serves later requests.  Every particle's
 * arithmetic is the same as in a tracer: a request's lines are identical
 * whether it runs alone or among others.
 *
 * All fields of a batch must share one layout (desc.layout); their storage
 * types may differ (each lane decodes its own request's type). */
typedef struct {
    int64_t max_lines;       /* line slots: lines of admitted, not yet released requests */
    int64_t slab_bytes;      /* vertex slab pool: W * 12 B per line of a request, W =
                                max_steps + 1 rounded up to a multiple of 4      */
    int32_t max_requests;    /* request table entries (<= 1048576) */
    int32_t max_fields;      /* distinct fields used by requests (<= 64) */
    int32_t max_bricks;      /* bricks summed over those fields (<= 65536) */
    int32_t layout;          /* field layout of every request's field */
    int32_t block_size;      /* schedule of the persistent kernel (0 = default), */
    int32_t blocks_per_sm;   /* as the fields of sg_tracer_params                */
    int32_t steps_per_round;
    int32_t drain_steps;
} sg_batch_desc;

/* Device bytes of a batch (slab pool, line arrays, queues, request table,
 * scan scratch). */
sg_status sg_batch_required_bytes(const sg_context *ctx, const sg_batch_desc *desc, size_t *bytes);
sg_status sg_batch_create(sg_context *ctx, const sg_batch_desc *desc, void *workspace, size_t bytes,
                          sg_batch **out);
sg_status sg_batch_destroy(sg_batch *b);

/* Free line slots and the largest free slab extent (bytes), for admission. */
sg_status sg_batch_capacity(const sg_batch *b, int64_t *free_lines, int64_t *largest_slab_bytes,
                            int32_t *free_requests);

/* Admits a request: n seeds (world xyz float32, host or device memory) traced
 * on field f with p (dt, max_steps, eps, tie thresholds; mode must be
 * SG_STREAMLINE; the schedule fields are ignored).  Returns SG_ERR_OOM,
 * leaving the batch unchanged, when the request does not fit now (line
 * slots, slab pool, request table or brick keys); the caller keeps it queued
 * and retries after releasing finished requests.  The seeds are copied and
 * binned on `stream`; they join the next sg_batch_run. */
sg_status sg_batch_submit(sg_batch *b, sg_field *f, const float *xyz, int64_t n, const sg_tracer_params *p,
                          int64_t *request_id, void *stream);

/* Runs up to max_rounds rounds of the persistent kernel over all admitted
 * requests (one CUDA-graph launch; max_rounds <= 0 runs until every queue is
 * empty).  Asynchronous. */
sg_status sg_batch_run(sg_batch *b, int32_t max_rounds, void *stream);

/* Synchronises `stream` and lists requests whose lines have all stopped and
 * that were not listed before: up to cap ids into ids (host), *count set. */
sg_status sg_batch_finished(sg_batch *b, int64_t *ids, int32_t cap, int32_t *count, void *stream);

/* Lines of a request, as sg_tracer_get_lines (two calls: sizes with NULL
 * buffers, then the buffers; device or page-locked host). */
sg_status sg_batch_get_lines(sg_batch *b, int64_t request_id, int64_t *n_lines, int64_t *n_vertices,
                             int64_t *offsets, float *vertices, uint8_t *status, float *margin, void *stream);

/* Frees a request's line slots and slab once the work queued on `stream`
 * (its readback) is done.  Its id becomes invalid. */
sg_status sg_batch_release(sg_batch *b, int64_t request_id, void *stream);

/* ------------------------------------------------------- line compaction */

/* Bytes of scan scratch sg_lines_compact needs for n_lines lines: one 8-byte
 * sum per 4096 lines plus 64 bytes. */
sg_status sg_lines_compact_scratch_bytes(int64_t n_lines, size_t *bytes);

/* Compacts per-line vertex slabs into CSR: getLines / assembleOutput (Fig. 4,
 * Listing 2) for slabs a caller holds itself (the unstructured field's trace,
 * a partitioned trace's merged lines).  Same arguments as
 * sg_lines_compact_static below, plus a caller-owned device scratch buffer
 * (8-byte aligned, at least sg_lines_compact_scratch_bytes(n_lines) bytes)
 * that the call uses on `stream` and that may be reused once the stream has
 * passed it.  Calls with separate scratch buffers may run concurrently.
 * Errors: SG_ERR_INVALID_ARG for a NULL or short buffer or sizes out of
 * range.  Asynchronous on `stream`. */
sg_status sg_lines_compact(const float *slab, int64_t max_vertices_per_line, const uint32_t *lengths,
                           int64_t n_lines, void *scratch, size_t scratch_bytes, int64_t *offsets, float *vertices,
                           void *stream);

/* ------------------------------------------------ allocation-free compaction */

/* The paper has no counterpart to this call: it is a service for callers that
 * must not allocate device memory, such as a simulation that has handed all
 * of HBM to its own pool and lends its buffers to the field-line pass in
 * situ, or a loop that cannot take the device-wide synchronisation that
 * cudaMalloc/cudaFree may cause.
 *
 * Compacts per-line vertex slabs into CSR, as sg_tracer_get_lines does, but
 * its scan scratch lives in a fixed array inside the library's device memory
 * (32 KB on every GPU that loads the library, held until the process exits),
 * so it calls no cudaMalloc, cudaFree or allocating routine.
 *   slab      device, n_lines x max_vertices_per_line x 3 floats (line i's
 *             vertices start at slab + 3 * i * max_vertices_per_line)
 *   lengths   device, n_lines uint32 vertex counts, each <= max_vertices_per_line
 *             (larger values are not checked and read past the slab)
 *   offsets   out, n_lines + 1 int64 (device or page-locked host):
 *             offsets[i] = sum of lengths before i, offsets[n_lines] = total
 *   vertices  out, 3 * total floats (device or page-locked host), or NULL to
 *             compute only the offsets
 * n_lines above 16,777,216 (4096 chunks of 4096 lines), or
 * max_vertices_per_line of 2^28 or more, is rejected with SG_ERR_INVALID_ARG.  The first call on a device looks up the scratch
 * array's device address (cudaGetSymbolAddress) with that device current; make
 * that first call before any stream capture.  The address stays cached for the
 * life of the process: after a cudaDeviceReset of that device (which frees
 * the library's copy of the array with the context) the call must not be used
 * on it again in the same process.  All calls on a device share the
 * one scratch array and it keeps the last call's contents: calls that overlap
 * on the GPU (issued on different streams) race and must be ordered by the
 * caller.  Asynchronous on `stream`. */
sg_status sg_lines_compact_static(const float *slab, int64_t max_vertices_per_line, const uint32_t *lengths,
                                  int64_t n_lines, int64_t *offsets, float *vertices, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* STREAMGB_H */
