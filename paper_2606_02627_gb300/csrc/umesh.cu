// Unstructured fields (the second field type of Sec. 3.3): a mesh of
// tetrahedra, pyramids, prisms and hexahedra (VTK vertex orders) carrying the
// velocity at its vertices, interpolated with each cell's isoparametric
// shape functions; cells are located with a bounding volume hierarchy and a
// point-in-cell test (the parametric solution of sum N_i(r) x_i = p, found by
// Newton's method, inside the cell's reference domain within tau).
//
// Layout (caller's workspace): one 256-byte record per cell, the eight
// vertex positions (float4, the cell type in the first w, the neighbours
// across the cell's faces in the next six w words) and the eight vertex
// velocities (float4), so that testing and interpolating a cell reads one
// contiguous record; the cells are stored in the order of the BVH's leaves,
// each leaf a contiguous range; BVH nodes are 32 bytes (box with the child /
// range in the w words).  The hierarchy and the face neighbours (faces
// matched by their vertex sets) are built on the host at creation (median
// split of the cell centroids along the widest axis, at most 4 cells per
// leaf).
//
// Tracing: one thread per seed to termination (Listing 1's RK4 in world
// coordinates, positions in FP64, samples in FP32 relative to the cell).  A
// point is looked for in the cell of the previous sample first, then by
// walking from it across the face whose parametric bound the point violates
// most (a few cells at most), and only then in the BVH.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "rk4.cuh"

namespace sg {

struct __align__(16) UCell {
    float4 x[8];                 // vertex positions; x[0].w holds the cell type (4, 5, 6, 8)
    float4 v[8];                 // vertex velocities
};

struct __align__(16) UNode {
    float4 lo;                   // w: leaf: first cell (int bits); inner: left child
    float4 hi;                   // w: leaf: cell count (> 0); inner: -(right child) (int bits)
};

constexpr int UMESH_LEAF = 4;
constexpr int UMESH_STACK = 64;
constexpr int UMESH_NEWTON = 12;
constexpr int UMESH_WALK = 6;                  // cells visited by a walk before the BVH takes over
constexpr int UMESH_SEGMENT = 128;             // steps per particle per round of a trace

// Faces of each cell type (VTK vertex order), in the order of the parametric
// bounds that exit_face reports: hexahedron a<0, a>1, b<0, b>1, c<0, c>1;
// tetrahedron a<0, b<0, c<0, a+b+c>1; prism a<0, b<0, a+b>1, c<0, c>1;
// pyramid a<0, a>1, b<0, b>1, c<0 (its apex has no face).  -1 pads a
// triangle.
struct UFaces {
    int n;
    int v[6][4];
};
static const UFaces UFACES_TET = {4, {{0, 2, 3, -1}, {0, 1, 3, -1}, {0, 1, 2, -1}, {1, 2, 3, -1}}};
static const UFaces UFACES_PYR = {5, {{0, 3, 4, -1}, {1, 2, 4, -1}, {0, 1, 4, -1}, {2, 3, 4, -1}, {0, 1, 2, 3}}};
static const UFaces UFACES_PRI = {5, {{0, 2, 5, 3}, {0, 1, 4, 3}, {1, 2, 5, 4}, {0, 1, 2, -1}, {3, 4, 5, -1}}};
static const UFaces UFACES_HEX = {6, {{0, 3, 7, 4}, {1, 2, 6, 5}, {0, 1, 5, 4}, {3, 2, 6, 7}, {0, 1, 2, 3}, {4, 5, 6, 7}}};

}  // namespace sg

struct sg_umesh {
    sg_context *ctx;
    int64_t n_cells;
    int64_t n_nodes;
    float tau;
    sg::UCell *cells;
    sg::UNode *nodes;
    int32_t *orig;               // original index of every stored cell
    float lo[3], hi[3];          // bounds of the mesh
};

namespace sg {

__device__ __forceinline__ void ushape(int type, float a, float b, float c, float N[8], float dN[8][3])
{
    if (type == 4) {
        N[0] = 1.f - a - b - c; N[1] = a; N[2] = b; N[3] = c;
#pragma unroll
        for (int i = 0; i < 4; ++i) dN[i][0] = dN[i][1] = dN[i][2] = 0.f;
        dN[0][0] = dN[0][1] = dN[0][2] = -1.f;
        dN[1][0] = 1.f; dN[2][1] = 1.f; dN[3][2] = 1.f;
    } else if (type == 5) {
        N[0] = (1 - a) * (1 - b) * (1 - c); N[1] = a * (1 - b) * (1 - c);
        N[2] = a * b * (1 - c); N[3] = (1 - a) * b * (1 - c); N[4] = c;
        dN[0][0] = -(1 - b) * (1 - c); dN[0][1] = -(1 - a) * (1 - c); dN[0][2] = -(1 - a) * (1 - b);
        dN[1][0] = (1 - b) * (1 - c);  dN[1][1] = -a * (1 - c);       dN[1][2] = -a * (1 - b);
        dN[2][0] = b * (1 - c);        dN[2][1] = a * (1 - c);        dN[2][2] = -a * b;
        dN[3][0] = -b * (1 - c);       dN[3][1] = (1 - a) * (1 - c);  dN[3][2] = -(1 - a) * b;
        dN[4][0] = 0.f;                dN[4][1] = 0.f;                dN[4][2] = 1.f;
    } else if (type == 6) {
        N[0] = (1 - a - b) * (1 - c); N[1] = a * (1 - c); N[2] = b * (1 - c);
        N[3] = (1 - a - b) * c;       N[4] = a * c;       N[5] = b * c;
        dN[0][0] = -(1 - c); dN[0][1] = -(1 - c); dN[0][2] = -(1 - a - b);
        dN[1][0] = (1 - c);  dN[1][1] = 0.f;      dN[1][2] = -a;
        dN[2][0] = 0.f;      dN[2][1] = (1 - c);  dN[2][2] = -b;
        dN[3][0] = -c;       dN[3][1] = -c;       dN[3][2] = (1 - a - b);
        dN[4][0] = c;        dN[4][1] = 0.f;      dN[4][2] = a;
        dN[5][0] = 0.f;      dN[5][1] = c;        dN[5][2] = b;
    } else {
        N[0] = (1 - a) * (1 - b) * (1 - c); N[1] = a * (1 - b) * (1 - c);
        N[2] = a * b * (1 - c);             N[3] = (1 - a) * b * (1 - c);
        N[4] = (1 - a) * (1 - b) * c;       N[5] = a * (1 - b) * c;
        N[6] = a * b * c;                   N[7] = (1 - a) * b * c;
        dN[0][0] = -(1 - b) * (1 - c); dN[0][1] = -(1 - a) * (1 - c); dN[0][2] = -(1 - a) * (1 - b);
        dN[1][0] = (1 - b) * (1 - c);  dN[1][1] = -a * (1 - c);       dN[1][2] = -a * (1 - b);
        dN[2][0] = b * (1 - c);        dN[2][1] = a * (1 - c);        dN[2][2] = -a * b;
        dN[3][0] = -b * (1 - c);       dN[3][1] = (1 - a) * (1 - c);  dN[3][2] = -(1 - a) * b;
        dN[4][0] = -(1 - b) * c;       dN[4][1] = -(1 - a) * c;       dN[4][2] = (1 - a) * (1 - b);
        dN[5][0] = (1 - b) * c;        dN[5][1] = -a * c;             dN[5][2] = a * (1 - b);
        dN[6][0] = b * c;              dN[6][1] = a * c;              dN[6][2] = a * b;
        dN[7][0] = -b * c;             dN[7][1] = (1 - a) * c;        dN[7][2] = (1 - a) * b;
    }
}

__device__ __forceinline__ float uviolation(int type, const float r[3])
{
    float v = fmaxf(-r[0], fmaxf(-r[1], -r[2]));
    if (type == 4) v = fmaxf(v, r[0] + r[1] + r[2] - 1.f);
    else if (type == 6) v = fmaxf(v, fmaxf(r[0] + r[1] - 1.f, r[2] - 1.f));
    else v = fmaxf(v, fmaxf(r[0] - 1.f, fmaxf(r[1] - 1.f, r[2] - 1.f)));
    return v;
}

// Parametric coordinates of p in the cell (Newton's method from its centre),
// in coordinates relative to the cell's first vertex so that FP32 keeps its
// precision relative to the cell's size; returns how far outside the
// reference domain they lie (<= tau: inside).
// warm: r already holds a guess (the previous sample's coordinates in this
// cell), else Newton starts from the cell's centre.  Not inlined: one copy
// serves every call site, and its loops run over the 8 vertex slots
// unrolled, so the shape functions stay in registers.
__device__ __noinline__ float ucell_param(const UCell &C, double3 pw, float r[3], bool warm = false)
{
    const int type = __float_as_int(C.x[0].w);
    const float4 X0 = C.x[0];
    const float3 p = make_float3((float)(pw.x - (double)X0.x), (float)(pw.y - (double)X0.y),
                                 (float)(pw.z - (double)X0.z));
    if (!warm) {
        r[0] = r[1] = r[2] = type == 4 ? 0.25f : (type == 6 ? (1.f / 3.f) : 0.5f);
        if (type == 6) r[2] = 0.5f;
        if (type == 5) r[2] = 0.2f;
    }
    for (int it = 0; it < UMESH_NEWTON; ++it) {
        float N[8], dN[8][3];
        ushape(type, r[0], r[1], r[2], N, dN);
        float x0 = -p.x, x1 = -p.y, x2 = -p.z;
        float J[3][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            if (i >= type) break;
            const float4 Xw = C.x[i];
            const float3 X = make_float3(Xw.x - X0.x, Xw.y - X0.y, Xw.z - X0.z);
            x0 = fmaf(N[i], X.x, x0);
            x1 = fmaf(N[i], X.y, x1);
            x2 = fmaf(N[i], X.z, x2);
#pragma unroll
            for (int l = 0; l < 3; ++l) {
                J[0][l] = fmaf(X.x, dN[i][l], J[0][l]);
                J[1][l] = fmaf(X.y, dN[i][l], J[1][l]);
                J[2][l] = fmaf(X.z, dN[i][l], J[2][l]);
            }
        }
        const float c00 = J[1][1] * J[2][2] - J[1][2] * J[2][1];
        const float c01 = J[1][2] * J[2][0] - J[1][0] * J[2][2];
        const float c02 = J[1][0] * J[2][1] - J[1][1] * J[2][0];
        const float det = J[0][0] * c00 + J[0][1] * c01 + J[0][2] * c02;
        if (!(fabsf(det) > 0.f)) break;
        const float inv = 1.f / det;
        // d = J^-1 F (adjugate)
        const float d0 = (c00 * x0 + (J[0][2] * J[2][1] - J[0][1] * J[2][2]) * x1 + (J[0][1] * J[1][2] - J[0][2] * J[1][1]) * x2) * inv;
        const float d1 = (c01 * x0 + (J[0][0] * J[2][2] - J[0][2] * J[2][0]) * x1 + (J[0][2] * J[1][0] - J[0][0] * J[1][2]) * x2) * inv;
        const float d2 = (c02 * x0 + (J[0][1] * J[2][0] - J[0][0] * J[2][1]) * x1 + (J[0][0] * J[1][1] - J[0][1] * J[1][0]) * x2) * inv;
        r[0] -= d0;
        r[1] -= d1;
        r[2] -= d2;
        // converged to well inside the containment tolerance (FP32 rounding
        // keeps the update near 1e-7 for coordinates of order one, so a
        // tighter test would run every iteration)
        if (fabsf(d0) + fabsf(d1) + fabsf(d2) < 3e-6f) break;
        if (fabsf(r[0]) + fabsf(r[1]) + fabsf(r[2]) > 1e6f) break;
    }
    // a parametric point counts only if it maps back onto p (Newton converged)
    float N[8], dN[8][3];
    ushape(type, r[0], r[1], r[2], N, dN);
    float x0 = -p.x, x1 = -p.y, x2 = -p.z, ext = 0.f;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        if (i >= type) break;
        const float4 Xw = C.x[i];
        const float3 X = make_float3(Xw.x - X0.x, Xw.y - X0.y, Xw.z - X0.z);
        x0 = fmaf(N[i], X.x, x0);
        x1 = fmaf(N[i], X.y, x1);
        x2 = fmaf(N[i], X.z, x2);
        ext = fmaxf(ext, fmaxf(fabsf(X.x), fmaxf(fabsf(X.y), fabsf(X.z))));
    }
    if (!(fabsf(x0) + fabsf(x1) + fabsf(x2) <= 1e-4f * ext)) return INFINITY;
    return uviolation(type, r);
}

__device__ float3 ucell_value(const UCell &C, const float r[3])
{
    const int type = __float_as_int(C.x[0].w);
    float N[8], dN[8][3];
    ushape(type, r[0], r[1], r[2], N, dN);
    float3 v = make_float3(0.f, 0.f, 0.f);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        if (i >= type) break;
        const float4 V = C.v[i];
        v.x = fmaf(N[i], V.x, v.x);
        v.y = fmaf(N[i], V.y, v.y);
        v.z = fmaf(N[i], V.z, v.z);
    }
    return v;
}

struct UMeshView {
    const UCell *cells;
    const UNode *nodes;
    long long n_cells;
    float tau;
};

// The face (in UFaces order) whose parametric bound the point r violates
// most, or -1 (a pyramid's apex).
__device__ __forceinline__ int exit_face(int type, const float r[3])
{
    const float a = r[0], b = r[1], c = r[2];
    float best;
    int f;
    if (type == 4) {
        best = -a, f = 0;
        if (-b > best) best = -b, f = 1;
        if (-c > best) best = -c, f = 2;
        if (a + b + c - 1.f > best) f = 3;
        return f;
    }
    if (type == 6) {
        best = -a, f = 0;
        if (-b > best) best = -b, f = 1;
        if (a + b - 1.f > best) best = a + b - 1.f, f = 2;
        if (-c > best) best = -c, f = 3;
        if (c - 1.f > best) f = 4;
        return f;
    }
    best = -a, f = 0;
    if (a - 1.f > best) best = a - 1.f, f = 1;
    if (-b > best) best = -b, f = 2;
    if (b - 1.f > best) best = b - 1.f, f = 3;
    if (-c > best) best = -c, f = 4;
    if (c - 1.f > best) f = type == 8 ? 5 : -1;
    return f;
}

// The stored cell containing p, or -1: the hint cell, then a walk across the
// faces from it, then the hierarchy.  r holds the parametric coordinates of
// the previous sample in the hint cell (the warm start) and receives those
// of p.
__device__ long long ulocate(const UMeshView &M, double3 pw, long long hint, float r[3], bool warm = false)
{
    for (int hop = 0; hint >= 0 && hop < UMESH_WALK; ++hop) {
        const UCell &C = M.cells[hint];
        const float viol = ucell_param(C, pw, r, warm);
        if (viol <= M.tau) return hint;
        if (!(viol < INFINITY)) break;             // no parametric solution: the hierarchy decides
        const int f = exit_face(__float_as_int(C.x[0].w), r);
        hint = f >= 0 ? __float_as_int(C.x[1 + f].w) : -1;
        warm = false;
    }
    const float3 p = make_float3((float)pw.x, (float)pw.y, (float)pw.z);
    if (M.n_cells == 0) return -1;
    int stack[UMESH_STACK];
    int top = 0;
    stack[top++] = 0;
    while (top > 0) {
        const UNode n = M.nodes[stack[--top]];
        if (p.x < n.lo.x || p.y < n.lo.y || p.z < n.lo.z || p.x > n.hi.x || p.y > n.hi.y || p.z > n.hi.z) continue;
        const int a = __float_as_int(n.lo.w), b = __float_as_int(n.hi.w);
        if (b > 0) {
            for (int k = 0; k < b; ++k)
                if (ucell_param(M.cells[a + k], pw, r) <= M.tau) return a + k;
        } else if (top + 2 <= UMESH_STACK) {
            stack[top++] = -b;
            stack[top++] = a;
        }
    }
    return -1;
}

__global__ void umesh_sample_kernel(UMeshView M, const int32_t *orig, const float *pts, long long n, float *vel,
                                    int64_t *cell)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const double3 p = make_double3(pts[3 * i], pts[3 * i + 1], pts[3 * i + 2]);
        float r[3];
        const long long c = ulocate(M, p, -1, r);
        float3 v = make_float3(NAN, NAN, NAN);
        if (c >= 0) v = ucell_value(M.cells[c], r);
        vel[3 * i] = v.x;
        vel[3 * i + 1] = v.y;
        vel[3 * i + 2] = v.z;
        if (cell) cell[i] = c >= 0 ? orig[c] : -1;
    }
}

struct UTraceArgs {
    const float *seeds;
    long long n;
    float dt;
    float eps;
    uint32_t max_steps;
    long long W;
    float *slab;
    uint32_t *len;
    uint8_t *status;
    float *margin;
    float tie_cells, tie_eps_rel;
};

// One RK4 step (Listing 1) in world coordinates; returns the status
// (SG_LINE_ACTIVE on success with pn set).  Positions are kept in FP64 (a
// handful of additions per step); the samples are FP32.  P0 comes located:
// its cell (hint), its coordinates there (rp) and its velocity (v0), from
// the previous step's locate of its new position; on success they are
// replaced by those of pn.
__device__ int urk4(const UMeshView &M, double3 p, float dt, float eps, long long &hint, float rp[3], float3 &v0,
                    double3 &pn, float &margin)
{
    float r[3], r0[3];
    const long long c0 = hint;
    long long c = c0;
    r0[0] = rp[0];
    r0[1] = rp[1];
    r0[2] = rp[2];
    float3 v = v0;
    if (bad3(v)) return SG_LINE_NANFIELD;
    const float sp = sqrtf(v.x * v.x + v.y * v.y + v.z * v.z);
    if (sp < eps) {
        margin = (eps - sp) / eps;
        return SG_LINE_STAGNANT;
    }
    float3 k[4];
    k[0] = make_float3(dt * v.x, dt * v.y, dt * v.z);
    const float w[3] = {0.5f, 0.5f, 1.0f};
    for (int s = 1; s < 4; ++s) {
        const double3 q = make_double3(p.x + (double)(w[s - 1] * k[s - 1].x), p.y + (double)(w[s - 1] * k[s - 1].y),
                                       p.z + (double)(w[s - 1] * k[s - 1].z));
        // stage points lie near P0: start from P0's coordinates in its cell
        long long cs = c0;
        float rs[3] = {r0[0], r0[1], r0[2]};
        cs = ulocate(M, q, cs, rs, true);
        if (cs < 0) {
            float rr[3] = {r0[0], r0[1], r0[2]};
            margin = ucell_param(M.cells[c0], q, rr, true);
            return SG_LINE_EXIT;
        }
        c = cs;
        v = ucell_value(M.cells[cs], rs);
        if (bad3(v)) return SG_LINE_NANFIELD;
        k[s] = make_float3(dt * v.x, dt * v.y, dt * v.z);
    }
    pn = make_double3(p.x + (double)((k[0].x + 2.f * k[1].x + 2.f * k[2].x + k[3].x) * (1.f / 6.f)),
                      p.y + (double)((k[0].y + 2.f * k[1].y + 2.f * k[2].y + k[3].y) * (1.f / 6.f)),
                      p.z + (double)((k[0].z + 2.f * k[1].z + 2.f * k[2].z + k[3].z) * (1.f / 6.f)));
    r[0] = r0[0];
    r[1] = r0[1];
    r[2] = r0[2];
    c = ulocate(M, pn, c0, r, true);
    if (c < 0) {
        float rr[3] = {r0[0], r0[1], r0[2]};
        margin = ucell_param(M.cells[c0], pn, rr, true);
        return SG_LINE_EXIT;
    }
    hint = c;
    rp[0] = r[0];
    rp[1] = r[1];
    rp[2] = r[2];
    v0 = ucell_value(M.cells[c], r);
    return SG_LINE_ACTIVE;
}

// A particle between rounds: its FP64 position, the cell found for it, its
// coordinates and velocity there (what the next step starts from), its line
// and its step count.
struct UPart {
    double p[3];
    float r[3];
    float v[3];
    int32_t hint;
    uint32_t line;
    uint32_t step;
    uint32_t pad;
};
static_assert(sizeof(UPart) == 64, "UPart");

// One round of the unstructured trace: every particle of the round's queue
// (round 0: the seeds, located here) takes at most `seg` steps; a particle
// that neither stopped nor reached max_steps goes to the next round's queue.
// Lines end at different lengths, so a launch that traced every line to its
// end would run as long as the longest line of each warp; rounds of a bounded
// number of steps keep the lanes of a warp busy until the last round.  A
// particle's state carries over whole, so its steps are the same as in one
// uninterrupted loop.
struct URound {
    const UPart *in;             // nullptr: the seeds
    const uint32_t *in_count;
    UPart *out;
    uint32_t *out_count;
    uint32_t seg;
};

// Built for 3 CTAs of 256 per SM (80 registers, with some spill): the
// kernel waits on dependent loads, and 24 warps per SM hide more of that than
// the 16 that 127 registers allow (measured on GB300: 5 % faster).
__global__ void __launch_bounds__(256, 3) umesh_round_kernel(UMeshView M, UTraceArgs A, URound R)
{
    const long long n = R.in ? (long long)*R.in_count : A.n;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        double3 p;
        long long hint;
        float r[3];
        float3 v0;
        uint32_t line, step;
        if (!R.in) {
            line = (uint32_t)i;
            step = 0;
            p = make_double3(A.seeds[3 * i], A.seeds[3 * i + 1], A.seeds[3 * i + 2]);
            hint = ulocate(M, p, -1, r);
            A.margin[i] = INFINITY;
            if (hint < 0) {
                A.len[i] = 0;
                A.status[i] = SG_LINE_OUT;
                continue;
            }
            float *o = A.slab + i * A.W * 3;
            o[0] = A.seeds[3 * i];
            o[1] = A.seeds[3 * i + 1];
            o[2] = A.seeds[3 * i + 2];
            v0 = ucell_value(M.cells[hint], r);
        } else {
            const UPart &q = R.in[i];
            p = make_double3(q.p[0], q.p[1], q.p[2]);
            hint = q.hint;
            r[0] = q.r[0];
            r[1] = q.r[1];
            r[2] = q.r[2];
            v0 = make_float3(q.v[0], q.v[1], q.v[2]);
            line = q.line;
            step = q.step;
        }
        float *out = A.slab + (long long)line * A.W * 3;
        float margin = INFINITY;
        int st = SG_LINE_ACTIVE;
        const uint32_t stop = step + min(R.seg, A.max_steps - step);
        while (step < stop) {
            double3 pn;
            const int s = urk4(M, p, A.dt, A.eps, hint, r, v0, pn, margin);
            if (s != SG_LINE_ACTIVE) {
                st = s;
                break;
            }
            p = pn;
            ++step;
            st_na(out + 3ll * step, (float)p.x);
            st_na(out + 3ll * step + 1, (float)p.y);
            st_na(out + 3ll * step + 2, (float)p.z);
        }
        if (st == SG_LINE_ACTIVE && step >= A.max_steps) st = SG_LINE_MAXSTEPS;
        if (st != SG_LINE_ACTIVE) {
            A.len[line] = step + 1;
            A.status[line] = stop_code_t(st, margin, A.tie_cells, A.tie_eps_rel);
            A.margin[line] = margin;
        } else {
            // warp-aggregated append to the next round's queue
            const unsigned m = __activemask();
            const int leader = __ffs(m) - 1;
            const unsigned lane = threadIdx.x & 31u;
            uint32_t base = 0;
            if ((int)lane == leader) base = atomicAdd(R.out_count, (uint32_t)__popc(m));
            base = __shfl_sync(m, base, leader);
            UPart &q = R.out[base + __popc(m & ((1u << lane) - 1u))];
            q.p[0] = p.x;
            q.p[1] = p.y;
            q.p[2] = p.z;
            q.r[0] = r[0];
            q.r[1] = r[1];
            q.r[2] = r[2];
            q.v[0] = v0.x;
            q.v[1] = v0.y;
            q.v[2] = v0.z;
            q.hint = (int32_t)hint;
            q.line = line;
            q.step = step;
            q.pad = 0u;
        }
    }
}

// ------------------------------------------------------------------ host: hierarchy build

struct BuildItem {
    int node, first, count;
};

// The median split turns a node of more than UMESH_LEAF (4) cells into two
// of at least 2, so every leaf of a hierarchy over n >= 2 cells holds 2 to 4
// cells: at most n / 2 leaves and n - 1 nodes.
static int64_t max_nodes(int64_t n_cells) { return n_cells > 1 ? n_cells : 1; }

}  // namespace sg

using namespace sg;

static size_t umesh_bytes(int64_t n_cells)
{
    return align_up(sizeof(UCell) * (size_t)n_cells, 256) + align_up(sizeof(UNode) * (size_t)max_nodes(n_cells), 256) +
           align_up(sizeof(int32_t) * (size_t)n_cells, 256);
}

extern "C" sg_status sg_umesh_required_bytes(int64_t n_cells, size_t *bytes)
{
    SG_CHECK(bytes && n_cells >= 0 && n_cells < (1ll << 30), SG_ERR_INVALID_ARG, "bad cell count");
    *bytes = umesh_bytes(n_cells);
    return SG_OK;
}

extern "C" sg_status sg_umesh_create(sg_context *ctx, const float *vertices, const float *velocity, int64_t n_vertices,
                                     const int32_t *cell_vertices, const int64_t *cell_offsets, const uint8_t *cell_types,
                                     int64_t n_cells, float tau, void *workspace, size_t bytes, sg_umesh **out)
{
    SG_CHECK(ctx && out && n_vertices >= 0 && n_cells >= 0 && n_cells < (1ll << 30), SG_ERR_INVALID_ARG,
             "bad arguments");
    SG_CHECK(n_cells == 0 || (vertices && velocity && cell_vertices && cell_offsets && cell_types), SG_ERR_INVALID_ARG,
             "NULL mesh array");
    SG_CHECK(workspace && ((uintptr_t)workspace & 255) == 0 && bytes >= umesh_bytes(n_cells), SG_ERR_OOM,
             "workspace of %zu bytes (256-byte aligned) needed", umesh_bytes(n_cells));
    SG_CHECK(pointer_kind(workspace) == PTR_DEVICE, SG_ERR_INVALID_ARG, "workspace must be device memory");
    SG_CHECK(tau >= 0.f && tau < 0.5f, SG_ERR_INVALID_ARG, "tau must be in [0, 0.5)");
    const float tol = tau > 0.f ? tau : 1e-5f;
    // cell records and boxes
    std::vector<UCell> rec((size_t)n_cells);
    std::vector<float> box((size_t)n_cells * 6), cen((size_t)n_cells * 3);
    float glo[3] = {INFINITY, INFINITY, INFINITY}, ghi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t c = 0; c < n_cells; ++c) {
        const int type = cell_types[c];
        SG_CHECK(type == 4 || type == 5 || type == 6 || type == 8, SG_ERR_INVALID_ARG, "cell %lld: type %d",
                 (long long)c, type);
        SG_CHECK(cell_offsets[c + 1] - cell_offsets[c] == type, SG_ERR_INVALID_ARG,
                 "cell %lld: %lld vertices for type %d", (long long)c,
                 (long long)(cell_offsets[c + 1] - cell_offsets[c]), type);
        UCell &u = rec[(size_t)c];
        memset(&u, 0, sizeof u);
        float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
        for (int i = 0; i < type; ++i) {
            const int64_t vi = cell_vertices[cell_offsets[c] + i];
            SG_CHECK(vi >= 0 && vi < n_vertices, SG_ERR_INVALID_ARG, "cell %lld: vertex %lld out of range",
                     (long long)c, (long long)vi);
            u.x[i] = make_float4(vertices[3 * vi], vertices[3 * vi + 1], vertices[3 * vi + 2], 0.f);
            u.v[i] = make_float4(velocity[3 * vi], velocity[3 * vi + 1], velocity[3 * vi + 2], 0.f);
            const float *X = vertices + 3 * vi;
            for (int a = 0; a < 3; ++a) {
                lo[a] = std::min(lo[a], X[a]);
                hi[a] = std::max(hi[a], X[a]);
            }
        }
        int tbits = type;
        memcpy(&u.x[0].w, &tbits, 4);
        for (int a = 0; a < 3; ++a) {
            // boxes grow by the containment tolerance (relative to the cell)
            const float pad = (hi[a] - lo[a]) * tol + 1e-30f;
            box[6 * c + a] = lo[a] - pad;
            box[6 * c + 3 + a] = hi[a] + pad;
            cen[3 * c + a] = 0.5f * (lo[a] + hi[a]);
            glo[a] = std::min(glo[a], lo[a]);
            ghi[a] = std::max(ghi[a], hi[a]);
        }
    }
    // hierarchy: median split of the centroids along the widest axis
    std::vector<int32_t> order((size_t)n_cells);
    for (int64_t c = 0; c < n_cells; ++c) order[(size_t)c] = (int32_t)c;
    std::vector<UNode> nodes;
    nodes.reserve((size_t)max_nodes(n_cells));
    if (n_cells > 0) {
        nodes.push_back(UNode());
        std::vector<BuildItem> todo{{0, 0, (int)n_cells}};
        while (!todo.empty()) {
            const BuildItem it = todo.back();
            todo.pop_back();
            float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
            float clo[3] = {INFINITY, INFINITY, INFINITY}, chi[3] = {-INFINITY, -INFINITY, -INFINITY};
            for (int k = it.first; k < it.first + it.count; ++k) {
                const int c = order[(size_t)k];
                for (int a = 0; a < 3; ++a) {
                    lo[a] = std::min(lo[a], box[6 * c + a]);
                    hi[a] = std::max(hi[a], box[6 * c + 3 + a]);
                    clo[a] = std::min(clo[a], cen[3 * c + a]);
                    chi[a] = std::max(chi[a], cen[3 * c + a]);
                }
            }
            UNode &nd = nodes[(size_t)it.node];
            nd.lo = make_float4(lo[0], lo[1], lo[2], 0.f);
            nd.hi = make_float4(hi[0], hi[1], hi[2], 0.f);
            if (it.count <= UMESH_LEAF) {
                int a = it.first, b = it.count;
                memcpy(&nd.lo.w, &a, 4);
                memcpy(&nd.hi.w, &b, 4);
                continue;
            }
            int ax = 0;
            for (int a = 1; a < 3; ++a)
                if (chi[a] - clo[a] > chi[ax] - clo[ax]) ax = a;
            const int mid = it.first + it.count / 2;
            std::nth_element(order.begin() + it.first, order.begin() + mid, order.begin() + it.first + it.count,
                             [&](int32_t p, int32_t q) { return cen[3 * p + ax] < cen[3 * q + ax]; });
            const int left = (int)nodes.size(), right = left + 1;
            nodes.push_back(UNode());
            nodes.push_back(UNode());
            UNode &nd2 = nodes[(size_t)it.node];        // the push_backs may have moved it
            int l = left, r = -right;
            memcpy(&nd2.lo.w, &l, 4);
            memcpy(&nd2.hi.w, &r, 4);
            todo.push_back({right, mid, it.first + it.count - mid});
            todo.push_back({left, it.first, mid - it.first});
        }
    }
    std::vector<UCell> sorted((size_t)n_cells);
    for (int64_t k = 0; k < n_cells; ++k) sorted[(size_t)k] = rec[(size_t)order[(size_t)k]];
    // face neighbours: faces matched by their sorted vertex ids; stored as
    // the neighbour's position in the stored order (-1: on the boundary)
    {
        std::vector<int32_t> pos((size_t)n_cells);
        for (int64_t k = 0; k < n_cells; ++k) pos[(size_t)order[(size_t)k]] = (int32_t)k;
        struct FaceKey {
            uint64_t k0, k1;
            int32_t cell;
            int32_t slot;
        };
        std::vector<FaceKey> faces;
        faces.reserve((size_t)n_cells * 6);
        for (int64_t c = 0; c < n_cells; ++c) {
            const int type = cell_types[c];
            const UFaces &F = type == 4 ? UFACES_TET : type == 5 ? UFACES_PYR : type == 6 ? UFACES_PRI : UFACES_HEX;
            for (int f = 0; f < F.n; ++f) {
                uint32_t v[4];
                for (int i = 0; i < 4; ++i)
                    v[i] = F.v[f][i] < 0 ? 0xffffffffu : (uint32_t)cell_vertices[cell_offsets[c] + F.v[f][i]];
                std::sort(v, v + 4);
                faces.push_back({((uint64_t)v[0] << 32) | v[1], ((uint64_t)v[2] << 32) | v[3], (int32_t)c, f});
            }
        }
        std::sort(faces.begin(), faces.end(), [](const FaceKey &p, const FaceKey &q) {
            return p.k0 != q.k0 ? p.k0 < q.k0 : (p.k1 != q.k1 ? p.k1 < q.k1 : p.cell < q.cell);
        });
        for (int64_t k = 0; k < n_cells; ++k)
            for (int f = 0; f < 6; ++f) {
                const int none = -1;
                memcpy(&sorted[(size_t)k].x[1 + f].w, &none, 4);
            }
        for (size_t i = 0; i + 1 < faces.size(); ++i) {
            const FaceKey &p = faces[i], &q = faces[i + 1];
            if (p.k0 != q.k0 || p.k1 != q.k1) continue;
            if (i + 2 < faces.size() && faces[i + 2].k0 == p.k0 && faces[i + 2].k1 == p.k1) continue;   // not manifold
            if (i > 0 && faces[i - 1].k0 == p.k0 && faces[i - 1].k1 == p.k1) continue;
            const int32_t a = pos[(size_t)p.cell], b = pos[(size_t)q.cell];
            memcpy(&sorted[(size_t)a].x[1 + p.slot].w, &b, 4);
            memcpy(&sorted[(size_t)b].x[1 + q.slot].w, &a, 4);
        }
    }
    SG_CHECK((int64_t)nodes.size() <= max_nodes(n_cells), SG_ERR_STATE, "hierarchy of %zu nodes exceeds its bound",
             nodes.size());
    SG_CUDA(cudaSetDevice(ctx->device));
    Carve cv{(char *)workspace, 0, 0};
    UCell *dcells = (UCell *)cv.take(sizeof(UCell) * (size_t)n_cells);
    UNode *dnodes = (UNode *)cv.take(sizeof(UNode) * (size_t)max_nodes(n_cells));
    int32_t *dorig = (int32_t *)cv.take(sizeof(int32_t) * (size_t)n_cells);
    if (n_cells > 0) {
        SG_CUDA(cudaMemcpy(dcells, sorted.data(), sizeof(UCell) * (size_t)n_cells, cudaMemcpyHostToDevice));
        SG_CUDA(cudaMemcpy(dnodes, nodes.data(), sizeof(UNode) * nodes.size(), cudaMemcpyHostToDevice));
        SG_CUDA(cudaMemcpy(dorig, order.data(), sizeof(int32_t) * (size_t)n_cells, cudaMemcpyHostToDevice));
    }
    sg_umesh *m = new sg_umesh;
    m->ctx = ctx;
    m->n_cells = n_cells;
    m->n_nodes = (int64_t)nodes.size();
    m->tau = tol;
    m->cells = dcells;
    m->nodes = dnodes;
    m->orig = dorig;
    for (int a = 0; a < 3; ++a) {
        m->lo[a] = glo[a];
        m->hi[a] = ghi[a];
    }
    *out = m;
    return SG_OK;
}

extern "C" sg_status sg_umesh_destroy(sg_umesh *m)
{
    delete m;
    return SG_OK;
}

static UMeshView view_of(const sg_umesh *m)
{
    UMeshView M;
    M.cells = m->cells;
    M.nodes = m->nodes;
    M.n_cells = m->n_cells;
    M.tau = m->tau;
    return M;
}

extern "C" sg_status sg_umesh_sample(sg_umesh *m, const float *points, int64_t n, float *velocity, int64_t *cell,
                                     void *stream)
{
    SG_CHECK(m && n >= 0 && (n == 0 || (points && velocity)), SG_ERR_INVALID_ARG, "bad arguments");
    if (n == 0) return SG_OK;
    SG_CHECK(pointer_kind(points) == PTR_DEVICE && pointer_kind(velocity) == PTR_DEVICE &&
                 (!cell || pointer_kind(cell) == PTR_DEVICE),
             SG_ERR_INVALID_ARG, "points, velocity and cell must be device memory");
    SG_CUDA(cudaSetDevice(m->ctx->device));
    const long long g = (n + 255) / 256;
    umesh_sample_kernel<<<(unsigned)(g < 65535 ? g : 65535), 256, 0, (cudaStream_t)stream>>>(view_of(m), m->orig,
                                                                                          points, n, velocity, cell);
    SG_CUDA(cudaGetLastError());
    return SG_OK;
}

extern "C" sg_status sg_umesh_trace(sg_umesh *m, const float *seeds, int64_t n, double dt, int32_t max_steps, float eps,
                                    float *slab, uint32_t *length, uint8_t *status, float *margin, void *stream)
{
    SG_CHECK(m && n >= 0 && n <= 0x7fffffff && max_steps >= 0 && max_steps < (1 << 27), SG_ERR_INVALID_ARG,
             "bad arguments");
    SG_CHECK(dt > 0.0 && dt < 1e30 && eps >= 0.f, SG_ERR_INVALID_ARG, "bad dt or eps");
    if (n == 0) return SG_OK;
    for (const void *p : {(const void *)seeds, (const void *)slab, (const void *)length, (const void *)status,
                          (const void *)margin})
        SG_CHECK(p && pointer_kind(p) == PTR_DEVICE, SG_ERR_INVALID_ARG, "trace buffers must be device memory");
    SG_CUDA(cudaSetDevice(m->ctx->device));
    UTraceArgs A;
    A.seeds = seeds;
    A.n = n;
    A.dt = (float)dt;
    A.eps = eps;
    A.max_steps = (uint32_t)max_steps;
    A.W = (long long)max_steps + 1;
    A.slab = slab;
    A.len = length;
    A.status = status;
    A.margin = margin;
    A.tie_cells = 1e-3f;
    A.tie_eps_rel = 1e-3f;
    long long g = (n + 255) / 256;
    const long long cap = (long long)m->ctx->sm_count * 8;
    if (g > cap) g = cap;
    // rounds of at most UMESH_SEGMENT steps per particle; after
    // ceil(max_steps / UMESH_SEGMENT) of them (at least one) every line has
    // ended, so the queue lengths stay on the device
    cudaStream_t s = (cudaStream_t)stream;
    const int rounds = max_steps > 0 ? (max_steps + UMESH_SEGMENT - 1) / UMESH_SEGMENT : 1;
    const size_t qbytes = align_up(sizeof(UPart) * (size_t)n, 256);
    char *buf = nullptr;
    if (rounds > 1) SG_CUDA(cudaMallocAsync((void **)&buf, 2 * qbytes + 256, s));
    UPart *q[2] = {buf ? (UPart *)buf : nullptr, buf ? (UPart *)(buf + qbytes) : nullptr};
    uint32_t *cnt = buf ? (uint32_t *)(buf + 2 * qbytes) : nullptr;
    cudaError_t e = cudaSuccess;
    for (int r = 0; r < rounds && e == cudaSuccess; ++r) {
        URound R;
        R.in = r == 0 ? nullptr : q[(r - 1) & 1];
        R.in_count = r == 0 ? nullptr : cnt + ((r - 1) & 1);
        R.out = q[r & 1];
        R.out_count = cnt ? cnt + (r & 1) : nullptr;
        R.seg = rounds > 1 ? (uint32_t)UMESH_SEGMENT : (uint32_t)max_steps;
        if (R.out_count) e = cudaMemsetAsync(R.out_count, 0, sizeof(uint32_t), s);
        if (e == cudaSuccess) {
            umesh_round_kernel<<<(unsigned)g, 256, 0, s>>>(view_of(m), A, R);
            e = cudaGetLastError();
        }
    }
    if (buf) {
        const cudaError_t f = cudaFreeAsync(buf, s);
        if (e == cudaSuccess) e = f;
    }
    SG_CUDA(e);
    return SG_OK;
}
