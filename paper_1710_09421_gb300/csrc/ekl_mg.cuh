// Multigrid-preconditioned conjugate gradients for the Poisson equation of
// the step (Eqs. 2-3, the same 7-point finite-volume operator on the fluid
// nodes as the red-black SOR of Sec. II.C): an alternative solver whose cost
// per decade of residual does not grow with the lattice.
//
// Operator: (A phi)_i = deg_i phi_i - sum_{open faces} phi_j, A phi = b.  It is
// symmetric positive semi-definite (constants span its null space when no
// face is fixed), so CG applies with a symmetric preconditioner:
//   * hierarchy: cell-centred 2x2x2 aggregation; the coarse face conductance
//     is half the sum of the fine conductances crossing the coarse face (the
//     rediscretised Laplacian at twice the spacing; a pure Galerkin product
//     with piecewise-constant transfer would double it), restriction sums the
//     children, prolongation injects;
//   * smoother: red-black Gauss-Seidel, nu sweeps red->black before the coarse
//     correction and the mirror sequence black->red after it; the coarsest
//     level takes (R B)^k R half sweeps on a zero-mean right-hand side and
//     returns a zero-mean correction, so the whole V-cycle is a fixed
//     symmetric linear operator;
//   * precision: the V-cycle and the CG vectors are FP32; the potential, the
//     source and the true residual b - A phi are in the path's potential type
//     (FP64, or 64-bit fixed point with an exact integer residual).  CG runs
//     until its recurrence residual has dropped by `inner_red` (or under the
//     tolerance), then the true residual is formed, tested against
//     tol ||b||, and CG restarts from it when needed (iterative refinement).
//
// One cooperative launch runs the whole solve: lattice-sized phases are
// spread over the grid and separated by the bounded grid barrier; coarse
// levels from `tile_from` on are smoothed in shared-memory tiles (one barrier
// per smoothing pass); levels at and below `cta_from` are handled by block 0
// alone while the other blocks wait at the next barrier.  Every load of data written inside the launch
// goes through L2 (__ldcg: L1 is not coherent across SMs) or, for data
// that no block writes during the current phase, through L1 (mg_ldl): the
// acquire fence of the grid barrier that opens the phase discards stale L1
// lines, and the phase itself never rewrites what it reads.
#pragma once
#include "ekl_kernels.cuh"

namespace ekl {

struct MgArgs {
    float *r, *z, *q, *p[2];
    double *part;         // [4][gridDim.x]
    const float *dense;   // pseudo-inverse of the coarsest operator [N][N], or null
    const uint8_t *link;  // per-node link byte of the lattice level (mg_link_of)
    void *phi_prev;       // potential of the step before the last (PhiT[N])
    int have_prev;        // phi_prev holds phi(t-2) and phi holds phi(t-1)
    int nlev, cta_from, nu, nu_c, coarse_sweeps;  // smoothing sweeps: lattice level, coarse levels
    float inner_red;
    int tile_from;                // first tiled coarse level (cta_from: none)
    int tile_off;                 // tile region offset (floats) in the dynamic shared memory
    int tile[MG_MAXLEV][3];       // owned cells per tile, per level
    MgLevel lev[MG_MAXLEV];
};

// Scalar state of a split solve (ekl_mgs.cuh) in device memory: written by
// its one-block control kernels, read by its lattice kernels.
struct MgCtl {
    double tol, bb, tol2, rr_true, rr_ref, rz_old;
    int max_iter, fixed_iter, limit, it, pi;
    int fresh;      // next search direction starts from z (beta = 0)
    int current;    // rr_true belongs to the present phi
    int converged, stop, need_true;
    int skip;       // zero source: nothing to solve, nothing to report
    int done;       // batches: this replica's loop has ended
};

// 4-byte words of shared memory for a tile region of Rx x Ry x Rz cells:
// e and f (each padded to 16 bytes), the float4 conductances, and the
// wrapped level coordinates of the region's columns, rows and planes
__host__ __device__ inline size_t mg_tile_words(int Rx, int Ry, int Rz)
{
    const size_t RN = (size_t)Rx * Ry * Rz, RN4 = (RN + 3) & ~(size_t)3;
    return 2 * RN4 + 4 * RN + (size_t)Rx + Ry + Rz;
}

// The blocks that solve one problem: all blocks of a single-handle launch, or
// the blocks a batched launch assigns to one replica (each replica then runs
// at its own pace with its own barrier).
struct MgGrid {
    int t0, nt;      // this thread's index and the thread count of the set
    int nblk, blk;   // block count of the set and this block's index in it
    unsigned *bar;   // the set's barrier words
};

__device__ __forceinline__ float mg_inv_deg(int d)
{
    return d == 6 ? (1.f / 6.f) : d == 5 ? 0.2f : d == 4 ? 0.25f : d == 3 ? (1.f / 3.f) : d == 2 ? 0.5f : 1.f;
}
// The lattice-level passes read, per node, either the link word (bit 31 on
// wall nodes, bit f + 1 when face f, in the order -x, +x, -y, +y, -z, +z,
// is closed) or the link byte made from it (MgArgs::link: the same face bits,
// the wall bit moved to bit 7), a quarter of the word's bytes.  L is the
// type read.
constexpr unsigned MG_LINK_SOLID = 0x80u;
__device__ __forceinline__ uint8_t mg_link_of(uint32_t m)
{
    return (uint8_t)((m & 0x7Eu) | ((m & SOLID_BIT) ? MG_LINK_SOLID : 0u));
}
template <typename L> __device__ __forceinline__ bool mg_wall(unsigned m)
{
    if constexpr (sizeof(L) == 1) return (m & MG_LINK_SOLID) != 0;
    else return (m & SOLID_BIT) != 0;
}
constexpr unsigned MG_NO_NODE = ~0u;  // a link value that reads as a wall in either type
// open faces of a fluid node, bit f in face order
__device__ __forceinline__ unsigned mg_open(unsigned m) { return (~(m >> 1)) & 63u; }

// The pair h of a level's red-black iteration: the two nodes (2 xh, 2 xh + 1)
// of one x-row; `x` takes colour c, `xo` the other colour.
struct Pair {
    int x, xo, y, z, row;
};
__device__ __forceinline__ Pair mg_pair(int h, int hx, int ny, int c)
{
    Pair p;
    p.row = h / hx;
    const int xh = h - p.row * hx;
    p.z = p.row / ny;
    p.y = p.row - p.z * ny;
    const int s = (c + p.y + p.z) & 1;
    p.x = 2 * xh + s;
    p.xo = 2 * xh + (s ^ 1);
    return p;
}

// load of a value no block writes during the current phase (L1-cached)
template <typename T> __device__ __forceinline__ T mg_ldl(const T *p) { return __ldca(p); }

template <bool SH> __device__ __forceinline__ float mg_ld(const float *p)
{
    if constexpr (SH) return *p;
    else return mg_ldl(p);
}
template <bool SH> __device__ __forceinline__ void mg_st(float *p, float v)
{
    if constexpr (SH) *p = v;
    else __stcg(p, v);
}
// conductances: read-only global memory, or block 0's shared-memory copy
template <bool SH> __device__ __forceinline__ float4 mg_sig(const float4 *p)
{
    if constexpr (SH) return *p;
    else return __ldg(p);
}
template <bool SH> __device__ __forceinline__ float mg_sx(const float4 *p)
{
    if constexpr (SH) return p->x;
    else return __ldg(&p->x);
}
template <bool SH> __device__ __forceinline__ float mg_sy(const float4 *p)
{
    if constexpr (SH) return p->y;
    else return __ldg(&p->y);
}
template <bool SH> __device__ __forceinline__ float mg_sz(const float4 *p)
{
    if constexpr (SH) return p->z;
    else return __ldg(&p->z);
}
template <bool SH> __device__ __forceinline__ float mg_sw(const float4 *p)
{
    if constexpr (SH) return p->w;
    else return __ldg(&p->w);
}

// ------------------------------------------------------------ lattice level
// The first half sweep of every smoothing pass starts from zero, so it only
// sets the colour-0 nodes to r / deg (colour-1 values are overwritten before
// they are read); it is fused into the phase that produces r.  Likewise a
// red-black update never reads the node's own old value, so the coarse-grid
// correction is added on the fly where the first post-smoothing half sweep
// (colour 1) reads its colour-0 neighbours, and colour-0 nodes take the
// corrected neighbours in the next half sweep: no separate prolongation pass.

// neighbour across face f (order -x, +x, -y, +y, -z, +z), wrapped
__device__ __forceinline__ void mg_face_coord(int nx, int ny, int nz, int x, int y, int z, int f, int &X, int &Y,
                                              int &Z)
{
    X = x;
    Y = y;
    Z = z;
    if (f == 0) X = x == 0 ? nx - 1 : x - 1;
    if (f == 1) X = x == nx - 1 ? 0 : x + 1;
    if (f == 2) Y = y == 0 ? ny - 1 : y - 1;
    if (f == 3) Y = y == ny - 1 ? 0 : y + 1;
    if (f == 4) Z = z == 0 ? nz - 1 : z - 1;
    if (f == 5) Z = z == nz - 1 ? 0 : z + 1;
}
__device__ __forceinline__ int mg_parent(const MgLevel &C, int x, int y, int z)
{
    return (x >> 1) + C.nx * ((y >> 1) + C.ny * (z >> 1));
}

// Half sweep of colour c of z <- (r + sum_open z_j) / deg.  PRO: the
// neighbours' values include the level-1 correction C.e(parent).  RZ: add
// r_i z_i of both nodes of each pair (the last half sweep of a V-cycle, when
// the other colour is final).  A thread takes U pairs per trip (h, h + nt,
// ...) and issues the loads of all of them before the first update, so
// their memory round trips overlap; the updates, and the order of the r.z
// sum, are those of one pair per trip.
constexpr int MG_FINE_U = 1;
template <bool RZ, bool PRO, int U = MG_FINE_U, typename L>
static __device__ void fine_half(const Grid3 &g, const L *__restrict__ link, const float *r, float *z,
                                 const MgLevel &C, int c, int t0, int nt, float &rz)
{
    const int hx = (g.nx + 1) >> 1, np = hx * g.ny * g.nz;
    for (int h0 = t0; h0 < np; h0 += U * nt) {
        float zn[U][6], ri[U], ro[U], zo[U];
        unsigned mk[U], mo[U];
        int ii[U];
#pragma unroll
        for (int u = 0; u < U; u++) {
            const int h = h0 + u * nt;
            mk[u] = mo[u] = MG_NO_NODE;
            ii[u] = 0;
            ri[u] = ro[u] = zo[u] = 0.f;
            if (h >= np) continue;
            const Pair p = mg_pair(h, hx, g.ny, c);
            if (p.x < g.nx) {
                // every load is issued before the link byte is known (neighbour
                // indices are always valid; closed faces are masked afterwards)
                const int i = p.x + g.nx * p.row;
                ii[u] = i;
                int nb[6];
                face_nbrs(g, p.x, p.y, p.z, i, nb);
#pragma unroll
                for (int f = 0; f < 6; f++) {
                    zn[u][f] = mg_ldl(z + nb[f]);
                    if (PRO) {
                        int X, Y, Z;
                        mg_face_coord(g.nx, g.ny, g.nz, p.x, p.y, p.z, f, X, Y, Z);
                        zn[u][f] += mg_ldl(C.e + mg_parent(C, X, Y, Z));
                    }
                }
                ri[u] = mg_ldl(r + i);
                mk[u] = __ldg(link + i);
            }
            if (RZ && p.xo < g.nx) {
                const int io = p.xo + g.nx * p.row;
                ro[u] = mg_ldl(r + io);
                zo[u] = mg_ldl(z + io);
                mo[u] = __ldg(link + io);
            }
        }
#pragma unroll
        for (int u = 0; u < U; u++) {
            const unsigned o = mg_open(mk[u]);
            if (!mg_wall<L>(mk[u]) && o) {
                float v = ri[u];
#pragma unroll
                for (int f = 0; f < 6; f++)
                    if ((o >> f) & 1u) v += zn[u][f];
                v *= mg_inv_deg(__popc(o));
                __stcg(z + ii[u], v);
                if (RZ) rz += ri[u] * v;
            }
            if (RZ && !mg_wall<L>(mo[u]) && mg_open(mo[u])) rz += ro[u] * zo[u];
        }
    }
}

// Warp-shuffle restrictions (fine_restrict_warp, coarse_restrict): a warp
// takes 8 consecutive coarse cells; lane = X + 8 k computes the two
// x-children (dx = 0, 1) in the (dy, dz) = (k & 1, k >> 1) row of cell X;
// the four rows of a cell are summed by shuffles.  The loops are
// warp-uniform.
__device__ __forceinline__ float mg_sum_rows(float v)
{
    v += __shfl_xor_sync(0xffffffffu, v, 8);
    v += __shfl_xor_sync(0xffffffffu, v, 16);
    return v;
}

// The loads of one node's residual r - A z, issued before any is used
template <typename L> struct ResidIn {
    float zn[6], ri, zi;
    unsigned m;
};
template <typename L>
__device__ __forceinline__ void fine_resid_load(const Grid3 &g, const L *__restrict__ link, const float *r,
                                                const float *z, int x, int y, int zz, ResidIn<L> &o)
{
    o.m = MG_NO_NODE;
    if (x >= g.nx || y >= g.ny || zz >= g.nz) return;
    const int i = x + g.nx * (y + g.ny * zz);
    int nb[6];
    face_nbrs(g, x, y, zz, i, nb);
#pragma unroll
    for (int f = 0; f < 6; f++) o.zn[f] = mg_ldl(z + nb[f]);
    o.ri = mg_ldl(r + i);
    o.zi = mg_ldl(z + i);
    o.m = __ldg(link + i);
}
template <typename L> __device__ __forceinline__ float fine_resid_eval(const ResidIn<L> &o)
{
    const unsigned open = mg_open(o.m);
    if (mg_wall<L>(o.m) || !open) return 0.f;
    float acc = o.ri - (float)__popc(open) * o.zi;
#pragma unroll
    for (int f = 0; f < 6; f++)
        if ((open >> f) & 1u) acc += o.zn[f];
    return acc;
}

// C.f = sum over the children of each level-1 cell of (r - A z); FIRST: also
// start level 1's pre-smoothing (colour-0 cells take f / diag).  A thread
// takes whole cells (consecutive threads, consecutive cells of a row), so a
// warp reads 64 consecutive nodes of a fine row per load; the children of a
// cell are visited one z-plane at a time, the loads of its four nodes issued
// before any is used.  The sum is formed as (row (0,0) + row (1,0)) +
// (row (0,1) + row (1,1)) over the (dy, dz) rows, each row the x-pair's sum.
template <bool FIRST, typename L>
static __device__ void fine_restrict_cells(const Grid3 &g, const L *__restrict__ link, const float *r,
                                     const float *z, const MgLevel &C, int t0, int nt)
{
    for (int I = t0; I < C.N; I += nt) {
        const int X = I % C.nx, t = I / C.nx, Y = t % C.ny, Z = t / C.ny;
        float row[2][2];
#pragma unroll
        for (int dz = 0; dz < 2; dz++) {
            ResidIn<L> in[2][2];
#pragma unroll
            for (int dy = 0; dy < 2; dy++)
#pragma unroll
                for (int dx = 0; dx < 2; dx++)
                    fine_resid_load(g, link, r, z, 2 * X + dx, 2 * Y + dy, 2 * Z + dz, in[dy][dx]);
#pragma unroll
            for (int dy = 0; dy < 2; dy++) row[dy][dz] = fine_resid_eval(in[dy][0]) + fine_resid_eval(in[dy][1]);
        }
        const float f = (row[0][0] + row[1][0]) + (row[0][1] + row[1][1]);
        __stcg(C.f + I, f);
        if (FIRST && !((X + Y + Z) & 1)) __stcg(C.e + I, f * __ldg(&C.sig[I].w));
    }
}

// residual r - A z of one fluid node of the lattice (0 elsewhere)
template <typename L>
__device__ __forceinline__ float fine_resid(const Grid3 &g, const L *__restrict__ link, const float *r,
                                            const float *z, int x, int y, int zz)
{
    if (x >= g.nx || y >= g.ny || zz >= g.nz) return 0.f;
    const int i = x + g.nx * (y + g.ny * zz);
    int nb[6];
    face_nbrs(g, x, y, zz, i, nb);
    float zn[6];
#pragma unroll
    for (int f = 0; f < 6; f++) zn[f] = mg_ldl(z + nb[f]);
    const float ri = mg_ldl(r + i), zi = mg_ldl(z + i);
    const unsigned m = __ldg(link + i);
    const unsigned o = mg_open(m);
    if (mg_wall<L>(m) || !o) return 0.f;
    float acc = ri - (float)__popc(o) * zi;
#pragma unroll
    for (int f = 0; f < 6; f++)
        if ((o >> f) & 1u) acc += zn[f];
    return acc;
}

// The same restriction for the single cooperative launch (fewer registers):
// a warp takes 8 consecutive coarse cells, lane = X + 8 k computes the two
// x-children in the (dy, dz) = (k & 1, k >> 1) row of cell X, and the four
// rows are summed by shuffles in the same order as fine_restrict_cells (same
// result bit for bit).  The loop is warp-uniform.
template <bool FIRST, typename L>
static __device__ void fine_restrict_warp(const Grid3 &g, const L *__restrict__ link, const float *r,
                                     const float *z, const MgLevel &C, int t0, int nt)
{
    const int lane = threadIdx.x & 31, total = ((C.N + 7) >> 3) * 32;
    for (int base = t0 - lane; base < total; base += nt) {
        const int I = (base >> 2) + (lane & 7), k = lane >> 3;
        float acc = 0.f;
        int X = 0, Y = 0, Z = 0;
        if (I < C.N) {
            X = I % C.nx;
            const int t = I / C.nx;
            Y = t % C.ny;
            Z = t / C.ny;
            const int y0 = 2 * Y + (k & 1), z0 = 2 * Z + (k >> 1);
            acc = fine_resid(g, link, r, z, 2 * X, y0, z0) + fine_resid(g, link, r, z, 2 * X + 1, y0, z0);
        }
        const float sum = mg_sum_rows(acc);
        if (I < C.N && k == 0) {
            __stcg(C.f + I, sum);
            if (FIRST && !((X + Y + Z) & 1)) __stcg(C.e + I, sum * __ldg(&C.sig[I].w));
        }
    }
}

// ------------------------------------------------------------ coarse levels
// SH: the level's e and f live in shared memory (block 0's part of the cycle);
// the conductances always come from global memory.
struct CNbr {
    int xm, xp, ym, yp, zm, zp;
};
__device__ __forceinline__ CNbr coarse_nbrs(const MgLevel &L, int x, int y, int z, int i)
{
    const int nxy = L.nx * L.ny;
    CNbr n;
    n.xm = x == 0 ? i + L.nx - 1 : i - 1;
    n.xp = x == L.nx - 1 ? i - L.nx + 1 : i + 1;
    n.ym = y == 0 ? i + nxy - L.nx : i - L.nx;
    n.yp = y == L.ny - 1 ? i - nxy + L.nx : i + L.nx;
    n.zm = z == 0 ? i + L.N - nxy : i - nxy;
    n.zp = z == L.nz - 1 ? i - L.N + nxy : i + nxy;
    return n;
}

// value of neighbour j (coordinates X, Y, Z), with the coarser correction when PRO
template <bool SH, bool PRO>
__device__ __forceinline__ float coarse_val(const MgLevel &L, const MgLevel &C, int j, int X, int Y, int Z)
{
    float v = mg_ld<SH>(L.e + j);
    if (PRO) v += mg_ld<SH>(C.e + mg_parent(C, X, Y, Z));
    return v;
}

// The coarse-level update e_i = (f_i + sum_j sigma_ij e_j) / diag_i and the
// residual f_i - (A e)_i from the cell's own conductances s (+x, +y, +z
// faces, 1/diag), those of its -x, -y, -z faces and the six neighbour
// values; one definition serves the global and the tiled sweeps, so both
// round identically.
__device__ __forceinline__ float mg_relax(float f, float4 s, float sxm, float sym, float szm, float vxp,
                                          float vxm, float vyp, float vym, float vzp, float vzm)
{
    float acc = f;
    acc += s.x * vxp + sxm * vxm;
    acc += s.y * vyp + sym * vym;
    acc += s.z * vzp + szm * vzm;
    return acc * s.w;
}
__device__ __forceinline__ float mg_cresid(float f, float e, float4 s, float sxm, float sym, float szm, float exp_,
                                           float exm, float eyp, float eym, float ezp, float ezm)
{
    const float diag = s.x + s.y + s.z + sxm + sym + szm;
    float acc = f - diag * e;
    acc += s.x * exp_ + sxm * exm;
    acc += s.y * eyp + sym * eym;
    acc += s.z * ezp + szm * ezm;
    return acc;
}

// Half sweep of colour c of e <- (f + sum sigma e_j) / diag.  Faces beyond a
// closed side carry sigma = 0 and inactive cells keep e = 0, so wrapped or
// inactive neighbours contribute nothing.  Every load of a cell is issued
// before its activity (1/diag = 0 on inactive cells) is known, so a cell
// costs one memory round trip, not two; a thread takes U cells per trip
// (h, h + nt, ...) with all their loads issued first.
template <bool SH, bool PRO, int U = 1>
static __device__ void coarse_half(const MgLevel &L, const MgLevel &C, int c, int t0, int nt)
{
    const int hx = (L.nx + 1) >> 1, np = hx * L.ny * L.nz;
    for (int h0 = t0; h0 < np; h0 += U * nt) {
        float v[U], w[U];
        int ii[U];
#pragma unroll
        for (int u = 0; u < U; u++) {
            const int h = h0 + u * nt;
            w[u] = 0.f;
            v[u] = 0.f;
            ii[u] = 0;
            if (h >= np) continue;
            const Pair p = mg_pair(h, hx, L.ny, c);
            if (p.x >= L.nx) continue;
            const int i = p.x + L.nx * p.row;
            ii[u] = i;
            const CNbr n = coarse_nbrs(L, p.x, p.y, p.z, i);
            const int xm = p.x == 0 ? L.nx - 1 : p.x - 1, xp = p.x == L.nx - 1 ? 0 : p.x + 1;
            const int ym = p.y == 0 ? L.ny - 1 : p.y - 1, yp = p.y == L.ny - 1 ? 0 : p.y + 1;
            const int zm = p.z == 0 ? L.nz - 1 : p.z - 1, zp = p.z == L.nz - 1 ? 0 : p.z + 1;
            const float4 s = mg_sig<SH>(L.sig + i);
            w[u] = s.w;
            v[u] = mg_relax(mg_ld<SH>(L.f + i), s, mg_sx<SH>(L.sig + n.xm), mg_sy<SH>(L.sig + n.ym),
                            mg_sz<SH>(L.sig + n.zm), coarse_val<SH, PRO>(L, C, n.xp, xp, p.y, p.z),
                            coarse_val<SH, PRO>(L, C, n.xm, xm, p.y, p.z),
                            coarse_val<SH, PRO>(L, C, n.yp, p.x, yp, p.z),
                            coarse_val<SH, PRO>(L, C, n.ym, p.x, ym, p.z),
                            coarse_val<SH, PRO>(L, C, n.zp, p.x, p.y, zp),
                            coarse_val<SH, PRO>(L, C, n.zm, p.x, p.y, zm));
        }
#pragma unroll
        for (int u = 0; u < U; u++)
            if (w[u] != 0.f) mg_st<SH>(L.e + ii[u], v[u]);
    }
}

template <bool SH>
__device__ __forceinline__ float coarse_resid(const MgLevel &L, int x, int y, int z)
{
    if (x >= L.nx || y >= L.ny || z >= L.nz) return 0.f;
    const int i = x + L.nx * (y + L.ny * z);
    const float4 sg = mg_sig<SH>(L.sig + i);
    const CNbr n = coarse_nbrs(L, x, y, z, i);
    // formed before the activity test, so all its loads are in flight at once
    const float res = mg_cresid(mg_ld<SH>(L.f + i), mg_ld<SH>(L.e + i), sg, mg_sx<SH>(L.sig + n.xm),
                                mg_sy<SH>(L.sig + n.ym), mg_sz<SH>(L.sig + n.zm), mg_ld<SH>(L.e + n.xp),
                                mg_ld<SH>(L.e + n.xm), mg_ld<SH>(L.e + n.yp), mg_ld<SH>(L.e + n.ym),
                                mg_ld<SH>(L.e + n.zp), mg_ld<SH>(L.e + n.zm));
    return sg.w == 0.f ? 0.f : res;
}

// C.f = sum over the children of each cell of level l+1 of (f - A e) on
// level l; FIRST: also start C's pre-smoothing
template <bool SH, bool FIRST>
static __device__ void coarse_restrict(const MgLevel &L, const MgLevel &C, int t0, int nt)
{
    const int lane = threadIdx.x & 31, total = ((C.N + 7) >> 3) * 32;
    for (int base = t0 - lane; base < total; base += nt) {
        const int I = (base >> 2) + (lane & 7), k = lane >> 3;
        float acc = 0.f;
        int X = 0, Y = 0, Z = 0;
        if (I < C.N) {
            X = I % C.nx;
            const int t = I / C.nx;
            Y = t % C.ny;
            Z = t / C.ny;
            const int y0 = 2 * Y + (k & 1), z0 = 2 * Z + (k >> 1);
            acc = coarse_resid<SH>(L, 2 * X, y0, z0) + coarse_resid<SH>(L, 2 * X + 1, y0, z0);
        }
        const float sum = mg_sum_rows(acc);
        if (I < C.N && k == 0) {
            mg_st<SH>(C.f + I, sum);
            if (FIRST && !((X + Y + Z) & 1)) mg_st<SH>(C.e + I, sum * mg_sw<SH>(C.sig + I));
        }
    }
}

// ------------------------------------------------------------ tiled coarse smoothing
// A block takes whole tiles of a level (tx x ty x tz owned cells, even, tile
// origins even) and runs a complete smoothing pass on the tile plus a halo of
// H = 2 nu_c cells held in shared memory: the k-th half sweep updates the
// cells within H - k (pre) or H - 1 - k (post) layers of the tile, so each
// half sweep reads only values already final for that stage, and the halo
// is recomputed by every tile that needs it.  The region is indexed by
// wrapped level coordinates (a region larger than the level simply repeats
// cells, which all take the same values), and every update and residual
// uses mg_relax / mg_cresid on the same inputs as the global sweeps: results
// are identical, at one grid barrier per smoothing pass.
constexpr int TILE_LOADS = 4;  // region cells a thread loads per round
struct TileSm {
    float *e, *f;
    float4 *s;
    int *wx, *wy, *wz;
    int Rx, Ry, Rz;
};
__device__ __forceinline__ TileSm tile_sm(float *sm, int Rx, int Ry, int Rz)
{
    TileSm T;
    const int RN = Rx * Ry * Rz, RN4 = (RN + 3) & ~3;
    T.e = sm;
    T.f = sm + RN4;
    T.s = (float4 *)(sm + 2 * RN4);
    T.wx = (int *)(T.s + RN);
    T.wy = T.wx + Rx;
    T.wz = T.wy + Ry;
    T.Rx = Rx;
    T.Ry = Ry;
    T.Rz = Rz;
    return T;
}

// region index k -> (a, b, c) for rows of nx cells and planes of ny rows
__device__ __forceinline__ void tsplit(int k, int nx, int ny, float inx, float iny, int &a, int &b, int &c)
{
    const int r = tdiv(k, inx);
    a = k - r * nx;
    c = tdiv(r, iny);
    b = r - c * ny;
}
__device__ __forceinline__ int mg_wrap(int v, int n)
{
    while (v < 0) v += n;
    while (v >= n) v -= n;
    return v;
}

// wrapped level coordinates of the region that starts at (x0, y0, z0)
__device__ __forceinline__ void tile_coords(const TileSm &T, const MgLevel &L, int x0, int y0, int z0)
{
    for (int a = threadIdx.x; a < T.Rx + T.Ry + T.Rz; a += blockDim.x) {
        if (a < T.Rx) T.wx[a] = mg_wrap(x0 + a, L.nx);
        else if (a < T.Rx + T.Ry) T.wy[a - T.Rx] = mg_wrap(y0 + a - T.Rx, L.ny);
        else T.wz[a - T.Rx - T.Ry] = mg_wrap(z0 + a - T.Rx - T.Ry, L.nz);
    }
}

// Half sweep of colour col over the region cells at least `lo` layers from
// the region's faces.  Colours follow the region coordinates (parity base at
// the region origin): they equal the level's colours everywhere the owned
// cells' results depend on, since periodic extents are even and a closed
// side decouples the wrapped cells beyond it (zero conductance).  A thread
// takes an x-pair and updates its colour-col cell.
static __device__ void tile_half(const TileSm &T, int lo, int col, int base)
{
    const int bx = T.Rx - 2 * lo, by = T.Ry - 2 * lo, bz = T.Rz - 2 * lo;
    const int bxh = (bx + 1) >> 1, np = bxh * by * bz;
    const float ibxh = 1.f / (float)bxh, iby = 1.f / (float)by;
    const int sy = T.Rx, sz = T.Rx * T.Ry, amax = T.Rx - lo;
    for (int h = threadIdx.x; h < np; h += blockDim.x) {
        int xh, b, c;
        tsplit(h, bxh, by, ibxh, iby, xh, b, c);
        b += lo;
        c += lo;
        const int a0 = lo + 2 * xh;
        const int a = a0 + ((a0 + b + c + base + col) & 1);
        if (a >= amax) continue;
        const int k = a + sy * b + sz * c;
        const float4 s = T.s[k];
        if (s.w == 0.f) continue;
        T.e[k] = mg_relax(T.f[k], s, T.s[k - 1].x, T.s[k - sy].y, T.s[k - sz].z, T.e[k + 1], T.e[k - 1],
                          T.e[k + sy], T.e[k - sy], T.e[k + sz], T.e[k - sz]);
    }
}

// tile origin (owned cells) of tile number t of a level
__device__ __forceinline__ void tile_origin(const MgLevel &L, const int *tdim, int t, int &x0, int &y0, int &z0)
{
    const int ntx = (L.nx + tdim[0] - 1) / tdim[0], nty = (L.ny + tdim[1] - 1) / tdim[1];
    const int tz = t / (ntx * nty), rem = t - tz * ntx * nty, ty = rem / ntx;
    x0 = (rem - ty * ntx) * tdim[0];
    y0 = ty * tdim[1];
    z0 = tz * tdim[2];
}
__device__ __forceinline__ int tile_count(const MgLevel &L, const int *tdim)
{
    return ((L.nx + tdim[0] - 1) / tdim[0]) * ((L.ny + tdim[1] - 1) / tdim[1]) * ((L.nz + tdim[2] - 1) / tdim[2]);
}

// Pre-smoothing of level L from its right-hand side (colour 0 from zero, then
// 2 nu_c - 1 half sweeps), the smoothed correction of the owned cells into
// L.t, and the restricted residual of the owned parents into C.f.
static __device__ void coarse_pre_tiles(const MgLevel &L, const MgLevel &C, const int *tdim, int H, int blk,
                                        int nblk, float *sm)
{
    const int tx = tdim[0], ty = tdim[1], tz = tdim[2];
    const TileSm T = tile_sm(sm, tx + 2 * H, ty + 2 * H, tz + 2 * H);
    const int RN = T.Rx * T.Ry * T.Rz, sy = T.Rx, sz = T.Rx * T.Ry;
    const float iRx = 1.f / (float)T.Rx, iRy = 1.f / (float)T.Ry, itx = 1.f / (float)tx, ity = 1.f / (float)ty;
    const int px = tx >> 1, py = ty >> 1, pz = tz >> 1;
    const float ipx = 1.f / (float)px, ipy = 1.f / (float)py;
    const int ntiles = tile_count(L, tdim);
    for (int t = blk; t < ntiles; t += nblk) {
        int x0, y0, z0;
        tile_origin(L, tdim, t, x0, y0, z0);
        const int base = (x0 + y0 + z0 - 3 * H) & 1;
        tile_coords(T, L, x0 - H, y0 - H, z0 - H);
        __syncthreads();
        // TILE_LOADS cells per thread in flight at once (the loads of one
        // round are independent: one L2 round trip per round, not per cell)
        for (int k0 = threadIdx.x; k0 < RN; k0 += TILE_LOADS * blockDim.x) {
            float4 sv[TILE_LOADS];
            float fv[TILE_LOADS];
            int col[TILE_LOADS];
#pragma unroll
            for (int j = 0; j < TILE_LOADS; j++) {
                const int k = k0 + j * blockDim.x;
                if (k < RN) {
                    int a, b, c;
                    tsplit(k, T.Rx, T.Ry, iRx, iRy, a, b, c);
                    const int i = T.wx[a] + L.nx * (T.wy[b] + L.ny * T.wz[c]);
                    sv[j] = __ldg(L.sig + i);
                    fv[j] = __ldcg(L.f + i);
                    col[j] = (a + b + c + base) & 1;
                }
            }
#pragma unroll
            for (int j = 0; j < TILE_LOADS; j++) {
                const int k = k0 + j * blockDim.x;
                if (k < RN) {
                    T.s[k] = sv[j];
                    T.f[k] = fv[j];
                    T.e[k] = col[j] ? 0.f : fv[j] * sv[j].w;
                }
            }
        }
        __syncthreads();
        for (int h = 1; h < H; h++) {
            tile_half(T, h, h & 1, base);
            __syncthreads();
        }
        // residual of the owned cells (in place of f), and their correction
        for (int k = threadIdx.x; k < tx * ty * tz; k += blockDim.x) {
            int a, b, c;
            tsplit(k, tx, ty, itx, ity, a, b, c);
            const int X = x0 + a, Y = y0 + b, Z = z0 + c;
            const int q = (a + H) + sy * (b + H) + sz * (c + H);
            float res = 0.f;
            if (X < L.nx && Y < L.ny && Z < L.nz) {
                const float4 s = T.s[q];
                if (s.w != 0.f)
                    res = mg_cresid(T.f[q], T.e[q], s, T.s[q - 1].x, T.s[q - sy].y, T.s[q - sz].z, T.e[q + 1],
                                    T.e[q - 1], T.e[q + sy], T.e[q - sy], T.e[q + sz], T.e[q - sz]);
                __stcg(L.t + X + L.nx * (Y + L.ny * Z), T.e[q]);
            }
            T.f[q] = res;
        }
        __syncthreads();
        // children summed as the global restriction does: each (dy, dz) row's
        // two x-children, then rows (0 + 1) + (2 + 3) with row = dy + 2 dz
        for (int k = threadIdx.x; k < px * py * pz; k += blockDim.x) {
            int a, b, c;
            tsplit(k, px, py, ipx, ipy, a, b, c);
            const int X = (x0 >> 1) + a, Y = (y0 >> 1) + b, Z = (z0 >> 1) + c;
            if (X >= C.nx || Y >= C.ny || Z >= C.nz) continue;
            const int q = (2 * a + H) + sy * (2 * b + H) + sz * (2 * c + H);
            const float r0 = T.f[q] + T.f[q + 1], r1 = T.f[q + sy] + T.f[q + sy + 1];
            const float r2 = T.f[q + sz] + T.f[q + sz + 1], r3 = T.f[q + sz + sy] + T.f[q + sz + sy + 1];
            __stcg(C.f + X + C.nx * (Y + C.ny * Z), (r0 + r1) + (r2 + r3));
        }
        __syncthreads();
    }
}

// Post-smoothing of level L: colour-0 cells start from their pre-smoothed
// correction plus the coarser correction C.e of their parent (what the first
// global post half sweep reads), then 2 nu_c half sweeps; the owned active
// cells' result goes to L.e.
static __device__ void coarse_post_tiles(const MgLevel &L, const MgLevel &C, const int *tdim, int H, int blk,
                                         int nblk, float *sm)
{
    const int tx = tdim[0], ty = tdim[1], tz = tdim[2];
    const TileSm T = tile_sm(sm, tx + 2 * H, ty + 2 * H, tz + 2 * H);
    const int RN = T.Rx * T.Ry * T.Rz, sy = T.Rx, sz = T.Rx * T.Ry;
    const float iRx = 1.f / (float)T.Rx, iRy = 1.f / (float)T.Ry, itx = 1.f / (float)tx, ity = 1.f / (float)ty;
    const int ntiles = tile_count(L, tdim);
    for (int t = blk; t < ntiles; t += nblk) {
        int x0, y0, z0;
        tile_origin(L, tdim, t, x0, y0, z0);
        const int base = (x0 + y0 + z0 - 3 * H) & 1;
        tile_coords(T, L, x0 - H, y0 - H, z0 - H);
        __syncthreads();
        for (int k0 = threadIdx.x; k0 < RN; k0 += TILE_LOADS * blockDim.x) {
            float4 sv[TILE_LOADS];
            float fv[TILE_LOADS], tv[TILE_LOADS], cv[TILE_LOADS];
#pragma unroll
            for (int j = 0; j < TILE_LOADS; j++) {
                const int k = k0 + j * blockDim.x;
                if (k < RN) {
                    int a, b, c;
                    tsplit(k, T.Rx, T.Ry, iRx, iRy, a, b, c);
                    const int gx = T.wx[a], gy = T.wy[b], gz = T.wz[c];
                    const int i = gx + L.nx * (gy + L.ny * gz);
                    sv[j] = __ldg(L.sig + i);
                    fv[j] = __ldcg(L.f + i);
                    tv[j] = 0.f;
                    cv[j] = 0.f;
                    if (!((a + b + c + base) & 1)) {
                        tv[j] = __ldcg(L.t + i);
                        cv[j] = __ldcg(C.e + mg_parent(C, gx, gy, gz));
                    }
                }
            }
#pragma unroll
            for (int j = 0; j < TILE_LOADS; j++) {
                const int k = k0 + j * blockDim.x;
                if (k < RN) {
                    T.s[k] = sv[j];
                    T.f[k] = fv[j];
                    float v = tv[j];
                    v += cv[j];
                    T.e[k] = v;
                }
            }
        }
        __syncthreads();
        for (int h = 0; h < H; h++) {
            tile_half(T, h + 1, (h & 1) ^ 1, base);
            __syncthreads();
        }
        for (int k = threadIdx.x; k < tx * ty * tz; k += blockDim.x) {
            int a, b, c;
            tsplit(k, tx, ty, itx, ity, a, b, c);
            const int X = x0 + a, Y = y0 + b, Z = z0 + c;
            const int q = (a + H) + sy * (b + H) + sz * (c + H);
            if (X < L.nx && Y < L.ny && Z < L.nz && T.s[q].w != 0.f) __stcg(L.e + X + L.nx * (Y + L.ny * Z), T.e[q]);
        }
        __syncthreads();
    }
}

// mean of v over the active cells of level L (block-wide, every thread gets it)
static __device__ float coarse_mean(const MgLevel &L, const float *v, double *sh, double *bc)
{
    double s = 0.0, n = 0.0;
    for (int i = threadIdx.x; i < L.N; i += blockDim.x)
        if (L.sig[i].w != 0.f) {
            s += (double)v[i];
            n += 1.0;
        }
    const double ts = block_sum(s, sh);
    const double tn = block_sum(n, sh);
    if (threadIdx.x == 0) bc[0] = tn > 0 ? ts / tn : 0.0;
    __syncthreads();
    const float mean = (float)bc[0];
    __syncthreads();
    return mean;
}

// Shared-memory layout of block 0's levels (l >= cta_from): per level e[N]
// and f[N] (floats, padded to 16 bytes) then sig[N] (float4).
__device__ __forceinline__ void mg_cta_levels(const MgArgs &m, float *sm, MgLevel *Ls)
{
    size_t off = 0;
    for (int l = m.cta_from; l < m.nlev; l++) {
        Ls[l] = m.lev[l];
        const size_t n2 = (2 * (size_t)Ls[l].N + 3) & ~(size_t)3;
        Ls[l].e = sm + off;
        Ls[l].f = sm + off + Ls[l].N;
        Ls[l].sig = (float4 *)(sm + off + n2);
        off += n2 + 4 * (size_t)Ls[l].N;
    }
}

// block 0, once per launch: the conductances of its levels into shared memory
static __device__ void mg_cta_load(const MgArgs &m, float *sm)
{
    MgLevel Ls[MG_MAXLEV];
    mg_cta_levels(m, sm, Ls);
    for (int l = m.cta_from; l < m.nlev; l++)
        for (int i = threadIdx.x; i < Ls[l].N; i += blockDim.x) Ls[l].sig[i] = __ldg(m.lev[l].sig + i);
    __syncthreads();
}

// Block 0 alone: the V-cycle at and below level m.cta_from in shared memory.
// On entry the level's right-hand side is in global memory; on exit its
// correction is written back there.
static __device__ void mg_cta_cycle(const MgArgs &m, float *sm, double *sh, double *bc)
{
    const int t0 = threadIdx.x, nt = blockDim.x;
    const int k0 = m.cta_from, last = m.nlev - 1;
    MgLevel Ls[MG_MAXLEV];
    mg_cta_levels(m, sm, Ls);
    // the right-hand side, and the first half sweep unless k0 is the coarsest
    {
        const MgLevel &L = Ls[k0];
        for (int i = t0; i < L.N; i += nt) {
            const float f = __ldcg(m.lev[k0].f + i);
            L.f[i] = f;
            L.e[i] = k0 < last ? f * L.sig[i].w : 0.f;  // colour 1 is overwritten first
        }
        __syncthreads();
    }
    for (int l = k0; l < last; l++) {
        for (int s = 1; s < 2 * m.nu_c; s++) {
            coarse_half<true, false>(Ls[l], Ls[l], s & 1, t0, nt);
            __syncthreads();
        }
        if (l + 1 < last) coarse_restrict<true, true>(Ls[l], Ls[l + 1], t0, nt);
        else coarse_restrict<true, false>(Ls[l], Ls[l + 1], t0, nt);
        __syncthreads();
    }
    // coarsest: zero-mean right-hand side, (R B)^k R from zero, zero-mean result
    {
        const MgLevel &L = Ls[last];
        const float mean = coarse_mean(L, L.f, sh, bc);
        for (int i = t0; i < L.N; i += nt) {
            const float w = L.sig[i].w;
            const float f = w != 0.f ? L.f[i] - mean : 0.f;
            L.f[i] = f;
            L.e[i] = f * w;  // colour 0 from zero; colour 1 is overwritten first
        }
        __syncthreads();
        for (int s = 1; s < 2 * m.coarse_sweeps + 1; s++) {
            coarse_half<true, false>(L, L, s & 1, t0, nt);
            __syncthreads();
        }
        const float emean = coarse_mean(L, L.e, sh, bc);
        for (int i = t0; i < L.N; i += nt)
            if (L.sig[i].w != 0.f) L.e[i] -= emean;
        __syncthreads();
    }
    for (int l = last - 1; l >= k0; l--) {
        coarse_half<true, true>(Ls[l], Ls[l + 1], 1, t0, nt);
        __syncthreads();
        for (int s = 1; s < 2 * m.nu_c; s++) {
            coarse_half<true, false>(Ls[l], Ls[l], (s & 1) ^ 1, t0, nt);
            __syncthreads();
        }
    }
    for (int i = t0; i < Ls[k0].N; i += nt) __stcg(m.lev[k0].e + i, Ls[k0].e[i]);
}

// Exact coarsest-level solve e = A^+ f with the host-computed pseudo-inverse
// (symmetric; it removes the null-space part of f and returns a zero-mean e
// on every connected part): one warp per row, grid-wide.
static __device__ void mg_dense_solve(const MgArgs &m, int t0, int nt)
{
    const MgLevel &L = m.lev[m.nlev - 1];
    const int n = L.N, lane = threadIdx.x & 31;
    for (int I = t0 >> 5; I < n; I += nt >> 5) {
        const float *row = m.dense + (size_t)I * n;
        float acc = 0.f;
        for (int J = lane; J < n; J += 32) acc += __ldg(row + J) * mg_ldl(L.f + J);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) __stcg(L.e + I, acc);
    }
}

// Coarse part of a V-cycle over the grid, from level `from` (1, or 2 when
// level 1 is smoothed by separate launches): entered with level from's
// right-hand side restricted (and, when that level is grid-wide and not
// block 0's, its pre-smoothing started); leaves level from's correction in
// lev[from].e for the prolongating half sweep of the level above.  False on
// a barrier abort.
template <bool TILES>
__device__ bool mg_coarse_cycle(const MgArgs &m, const MgGrid &G, unsigned &bar_k, int *status, float *sm,
                                double *sh, double *bc, int from = 1)
{
    const int t0 = G.t0, nt = G.nt;
#define MG_BAR()                                                          \
    do {                                                                  \
        if (!grid_barrier(G.bar, (unsigned)G.nblk, bar_k, status)) return false; \
    } while (0)
    float *tsm = sm + m.tile_off;  // coarse tile regions
    for (int l = from; l < m.cta_from; l++) {
        if (TILES && l >= m.tile_from) {
            coarse_pre_tiles(m.lev[l], m.lev[l + 1], m.tile[l], 2 * m.nu_c, G.blk, G.nblk, tsm);
            MG_BAR();
            continue;
        }
        for (int s = 1; s < 2 * m.nu_c; s++) {
            coarse_half<false, false>(m.lev[l], m.lev[l], s & 1, t0, nt);
            MG_BAR();
        }
        if (l + 1 < m.cta_from) coarse_restrict<false, true>(m.lev[l], m.lev[l + 1], t0, nt);
        else coarse_restrict<false, false>(m.lev[l], m.lev[l + 1], t0, nt);
        MG_BAR();
    }
    if (m.dense) mg_dense_solve(m, t0, nt);
    else if (G.blk == 0) mg_cta_cycle(m, sm, sh, bc);
    MG_BAR();
    for (int l = m.cta_from - 1; l >= from; l--) {
        if (TILES && l >= m.tile_from) {
            coarse_post_tiles(m.lev[l], m.lev[l + 1], m.tile[l], 2 * m.nu_c, G.blk, G.nblk, tsm);
            MG_BAR();
            continue;
        }
        coarse_half<false, true>(m.lev[l], m.lev[l + 1], 1, t0, nt);
        MG_BAR();
        for (int s = 1; s < 2 * m.nu_c; s++) {
            coarse_half<false, false>(m.lev[l], m.lev[l], (s & 1) ^ 1, t0, nt);
            MG_BAR();
        }
    }
#undef MG_BAR
    return true;
}

// One V-cycle z = M^-1 r over the grid, entered with z's colour-0 nodes
// already set to r / deg; returns this block's partial of r.z in thread 0
// (through rz_block), or false on a barrier abort.
template <typename S, typename R, typename PhiT, bool TILES>
__device__ bool mg_vcycle(const StepArgs<S, R, PhiT> &a, const MgArgs &m, const MgGrid &G, unsigned &bar_k,
                          float *sm, double *sh, double *bc, double &rz_block)
{
    const Grid3 g = a.g;
    const int t0 = G.t0, nt = G.nt;
    float dummy = 0.f;
#define MG_BAR()                                                          \
    do {                                                                  \
        if (!grid_barrier(G.bar, (unsigned)G.nblk, bar_k, a.status)) return false; \
    } while (0)
    // lattice level: rest of the pre-smoothing, residual restricted to level 1
    for (int s = 1; s < 2 * m.nu; s++) {
        fine_half<false, false>(g, a.mask, m.r, m.z, m.lev[1], s & 1, t0, nt, dummy);
        MG_BAR();
    }
    if (m.cta_from > 1) fine_restrict_warp<true>(g, a.mask, m.r, m.z, m.lev[1], t0, nt);
    else fine_restrict_warp<false>(g, a.mask, m.r, m.z, m.lev[1], t0, nt);
    MG_BAR();
    if (!mg_coarse_cycle<TILES>(m, G, bar_k, a.status, sm, sh, bc)) return false;
    fine_half<false, true>(g, a.mask, m.r, m.z, m.lev[1], 1, t0, nt, dummy);
    MG_BAR();
    float rz = 0.f;
    for (int s = 1; s < 2 * m.nu; s++) {
        const int c = (s & 1) ^ 1;
        if (s == 2 * m.nu - 1) {
            fine_half<true, false>(g, a.mask, m.r, m.z, m.lev[1], c, t0, nt, rz);
        } else {
            fine_half<false, false>(g, a.mask, m.r, m.z, m.lev[1], c, t0, nt, dummy);
            MG_BAR();
        }
    }
#undef MG_BAR
    rz_block = block_sum_lanes0(warp_sum_ff_lane0(rz), sh);
    return true;
}

// true residual r = b - A phi (exact in the potential type), as FP32, with
// the first pre-smoothing half sweep (colour-0 z = r / deg); returns this
// block's sum of r^2 (thread 0).  A thread takes MG_RES_U nodes per trip (one
// per grid stride) with all their loads issued first; its nodes are still
// summed in increasing order.
constexpr int MG_RES_U = 2;
template <typename PhiT, typename L>
__device__ double mg_true_residual(const Grid3 &g, const L *__restrict__ link, const PhiT *phi,
                                   const PhiT *b, float *r, float *z, int t0, int nt, double *sh)
{
    float rr = 0.f;
    const int N = (int)g.N;
    for (long long i0 = t0; i0 < N; i0 += (long long)MG_RES_U * nt) {
        PhiT pn[MG_RES_U][6], bi[MG_RES_U], phii[MG_RES_U];
        unsigned mk[MG_RES_U];
        int xyz[MG_RES_U];
#pragma unroll
        for (int k = 0; k < MG_RES_U; k++) {
            const long long il = i0 + (long long)k * nt;
            mk[k] = MG_NO_NODE;
            if (il >= N) continue;
            const int i = (int)il;
            const int x = i % g.nx, t = i / g.nx, y = t % g.ny, zz = t / g.ny;
            xyz[k] = x + y + zz;
            int nb[6];
            face_nbrs(g, x, y, zz, i, nb);
#pragma unroll
            for (int f = 0; f < 6; f++) pn[k][f] = mg_ldl(phi + nb[f]);
            bi[k] = mg_ldl(b + i);
            phii[k] = mg_ldl(phi + i);
            mk[k] = __ldg(link + i);
        }
#pragma unroll
        for (int k = 0; k < MG_RES_U; k++) {
            const int i = (int)(i0 + (long long)k * nt);
            if (mg_wall<L>(mk[k])) continue;  // also every node past N
            const unsigned o = mg_open(mk[k]);
            float rv = 0.f;
            if (o) {
                PhiT acc = bi[k];
#pragma unroll
                for (int f = 0; f < 6; f++)
                    if ((o >> f) & 1u) acc += pn[k][f];
                acc -= (PhiT)__popc(o) * phii[k];
                if constexpr (((PhiT)0.5) != 0) rv = (float)acc;
                else rv = ll_to_float(acc) * (float)PHI_INV;
                if (!(xyz[k] & 1)) __stcg(z + i, rv * mg_inv_deg(__popc(o)));
            }
            __stcg(r + i, rv);
            rr += rv * rv;
        }
    }
    return block_sum_lanes0(warp_sum_ff_lane0(rr), sh);
}

// The CG passes walk the lattice by pairs (2 xh, 2 xh + 1) of one x-row: one
// division chain per two nodes and the loads of both issued together.

// p = z + beta p_old and q = A p on the fluid nodes: the loads of one node
template <typename L> struct PqIn {
    float zj[6], pj[6], zi, pi;
    unsigned m;
};
template <bool FRESH, typename L>
__device__ __forceinline__ void mg_pq_load(const Grid3 &g, const L *__restrict__ link, const float *z,
                                           const float *pold, int x, int y, int zz, int i, PqIn<L> &o)
{
    int nb[6];
    face_nbrs(g, x, y, zz, i, nb);
#pragma unroll
    for (int f = 0; f < 6; f++) {
        o.zj[f] = mg_ldl(z + nb[f]);
        if (!FRESH) o.pj[f] = mg_ldl(pold + nb[f]);
    }
    o.zi = mg_ldl(z + i);
    if (!FRESH) o.pi = mg_ldl(pold + i);
    o.m = __ldg(link + i);
}
template <bool FRESH, typename L>
__device__ __forceinline__ void mg_pq_eval(const PqIn<L> &o, float beta, float &pn, float &qv, bool &live)
{
    const unsigned open = mg_open(o.m);
    live = !mg_wall<L>(o.m);
    pn = 0.f;
    qv = 0.f;
    if (!live || !open) return;
    pn = FRESH ? o.zi : o.zi + beta * o.pi;
    float acc = 0.f;
#pragma unroll
    for (int f = 0; f < 6; f++)
        if ((open >> f) & 1u) acc += FRESH ? o.zj[f] : o.zj[f] + beta * o.pj[f];
    qv = (float)__popc(open) * pn - acc;
}

// U pairs per thread and trip (loads of all first); returns sum p q in the
// order of one pair per trip
template <bool FRESH, typename L, int U = 1>
__device__ float mg_pq_pass(const Grid3 &g, const L *__restrict__ link, const float *z, const float *pold,
                            float *pnew, float *q, float beta, int t0, int nt)
{
    const int hx = (g.nx + 1) >> 1, np = hx * g.ny * g.nz;
    float pq = 0.f;
    for (int h0 = t0; h0 < np; h0 += U * nt) {
        PqIn<L> in[U][2];
        int i0[U];
#pragma unroll
        for (int u = 0; u < U; u++) {
            const int h = h0 + u * nt;
            in[u][0].m = in[u][1].m = MG_NO_NODE;
            i0[u] = 0;
            if (h >= np) continue;
            const int row = h / hx, xh = h - row * hx;
            const int zz = row / g.ny, y = row - zz * g.ny;
            const int x0 = 2 * xh;
            i0[u] = x0 + g.nx * row;
            mg_pq_load<FRESH>(g, link, z, pold, x0, y, zz, i0[u], in[u][0]);
            if (x0 + 1 < g.nx) mg_pq_load<FRESH>(g, link, z, pold, x0 + 1, y, zz, i0[u] + 1, in[u][1]);
        }
#pragma unroll
        for (int u = 0; u < U; u++) {
            float pn0, q0, pn1, q1;
            bool l0, l1;
            mg_pq_eval<FRESH>(in[u][0], beta, pn0, q0, l0);
            mg_pq_eval<FRESH>(in[u][1], beta, pn1, q1, l1);
            if (l0) {
                __stcg(pnew + i0[u], pn0);
                __stcg(q + i0[u], q0);
            }
            if (l1) {
                __stcg(pnew + i0[u] + 1, pn1);
                __stcg(q + i0[u] + 1, q1);
            }
            pq += pn0 * q0 + pn1 * q1;
        }
    }
    return pq;
}

// The same p/q pass for the single cooperative launch, one pair per trip
// with the neighbours' p formed as they arrive (fewer registers; the same
// values and the same order of the p.q sum as mg_pq_pass)
template <bool FRESH, typename L>
__device__ __forceinline__ void mg_pq_node_lean(const Grid3 &g, const L *__restrict__ link, const float *z,
                                           const float *pold, float beta, int x, int y, int zz, int i, float &pn,
                                           float &qv, bool &live)
{
    int nb[6];
    face_nbrs(g, x, y, zz, i, nb);
    float pj[6];
#pragma unroll
    for (int f = 0; f < 6; f++) pj[f] = FRESH ? mg_ldl(z + nb[f]) : mg_ldl(z + nb[f]) + beta * mg_ldl(pold + nb[f]);
    const float pi_ = FRESH ? mg_ldl(z + i) : mg_ldl(z + i) + beta * mg_ldl(pold + i);
    const unsigned mk = __ldg(link + i);
    const unsigned o = mg_open(mk);
    live = !mg_wall<L>(mk);
    pn = 0.f;
    qv = 0.f;
    if (!live || !o) return;
    pn = pi_;
    float acc = 0.f;
#pragma unroll
    for (int f = 0; f < 6; f++)
        if ((o >> f) & 1u) acc += pj[f];
    qv = (float)__popc(o) * pn - acc;
}

template <bool FRESH, typename L>
__device__ float mg_pq_pass_lean(const Grid3 &g, const L *__restrict__ link, const float *z, const float *pold,
                            float *pnew, float *q, float beta, int t0, int nt)
{
    const int hx = (g.nx + 1) >> 1, np = hx * g.ny * g.nz;
    float pq = 0.f;
    for (int h = t0; h < np; h += nt) {
        const int row = h / hx, xh = h - row * hx;
        const int zz = row / g.ny, y = row - zz * g.ny;
        const int x0 = 2 * xh, i0 = x0 + g.nx * row;
        const bool two = x0 + 1 < g.nx;
        float pn0, q0, pn1 = 0.f, q1 = 0.f;
        bool l0, l1 = false;
        mg_pq_node_lean<FRESH>(g, link, z, pold, beta, x0, y, zz, i0, pn0, q0, l0);
        if (two) mg_pq_node_lean<FRESH>(g, link, z, pold, beta, x0 + 1, y, zz, i0 + 1, pn1, q1, l1);
        if (l0) {
            __stcg(pnew + i0, pn0);
            __stcg(q + i0, q0);
        }
        if (l1) {
            __stcg(pnew + i0 + 1, pn1);
            __stcg(q + i0 + 1, q1);
        }
        pq += pn0 * q0 + pn1 * q1;
    }
    return pq;
}

// phi += alpha p, r -= alpha q and colour-0 z = r / deg on the fluid nodes
// with an open face; returns sum r^2
template <typename PhiT, typename L>
__device__ float mg_update_pass(const Grid3 &g, const L *__restrict__ link, PhiT *phi, const float *p,
                                const float *q, float *r, float *z, double alpha, int t0, int nt)
{
    const int hx = (g.nx + 1) >> 1, np = hx * g.ny * g.nz;
    const float af = (float)alpha;
    const float afx = (float)(alpha * PHI_SCALE);
    float rr = 0.f;
    for (int h = t0; h < np; h += nt) {
        const int row = h / hx, xh = h - row * hx;
        const int zz = row / g.ny, y = row - zz * g.ny;
        const int x0 = 2 * xh, i0 = x0 + g.nx * row;
        const int nk = x0 + 1 < g.nx ? 2 : 1;
        unsigned mk[2];
        float pv[2], qv[2], rv[2];
        PhiT ph[2];
#pragma unroll
        for (int k = 0; k < 2; k++) {
            mk[k] = MG_NO_NODE;
            pv[k] = qv[k] = rv[k] = 0.f;
            ph[k] = (PhiT)0;
            if (k < nk) {
                mk[k] = __ldg(link + i0 + k);
                pv[k] = __ldcg(p + i0 + k);
                qv[k] = __ldcg(q + i0 + k);
                rv[k] = __ldcg(r + i0 + k);
                ph[k] = __ldcg(phi + i0 + k);
            }
        }
#pragma unroll
        for (int k = 0; k < 2; k++) {
            const unsigned o = mg_open(mk[k]);
            if (mg_wall<L>(mk[k]) || !o) continue;
            const int i = i0 + k;
            if constexpr (((PhiT)0.5) != 0) __stcg(phi + i, ph[k] + (double)af * (double)pv[k]);
            else __stcg(phi + i, ph[k] + float_to_ll(afx * pv[k]));
            const float rn = rv[k] - af * qv[k];
            __stcg(r + i, rn);
            rr += rn * rn;
            if (!((x0 + k + y + zz) & 1)) __stcg(z + i, rn * mg_inv_deg(__popc(o)));
        }
    }
    return rr;
}

// Start of a solve, one pass: the starting guess phi <- 2 phi(t-1) - phi(t-2),
// the linear extrapolation of the last two potentials (exact in the
// fixed-point type; phi(t-1) is kept for the next step), and the source b.
// A thread takes MG_START_U nodes per trip (one per grid stride) and issues
// all their loads before it uses any, so their memory round trips overlap;
// each thread still visits its nodes in increasing order, which keeps the
// b^2 sum bit-identical to form_source's.  Returns the block's sum of b^2
// (thread 0).
constexpr int MG_START_U = 4;
template <typename S, typename R, typename PhiT, typename L>
__device__ double mg_start_pass(const StepArgs<S, R, PhiT> &a, const MgArgs &m, const L *__restrict__ link, int tid,
                                int nthr, double *sh, double *bc)
{
    const SrcMean sm = source_mean(a, bc);
    const int N = (int)a.g.N;
    PhiT *prev = (PhiT *)m.phi_prev;
    const bool extrap = m.have_prev != 0;
    double bl = 0.0;
    float blf = 0.f;
    for (long long i0 = tid; i0 < N; i0 += (long long)MG_START_U * nthr) {
        unsigned mk[MG_START_U];
        PhiT cur[MG_START_U], pv[MG_START_U];
        R rho[MG_START_U];
#pragma unroll
        for (int k = 0; k < MG_START_U; k++) {
            const long long i = i0 + (long long)k * nthr;
            mk[k] = MG_NO_NODE;
            cur[k] = pv[k] = (PhiT)0;
            rho[k] = (R)0;
            if (i < N) {
                mk[k] = __ldg(link + i);
                cur[k] = __ldcg(a.phi + i);
                if (extrap) pv[k] = __ldcg(prev + i);
                rho[k] = __ldcg(a.rho + i);
            }
        }
#pragma unroll
        for (int k = 0; k < MG_START_U; k++) {
            const long long i = i0 + (long long)k * nthr;
            if (i >= N) continue;
            PhiT bv = (PhiT)0;
            if (!mg_wall<L>(mk[k])) {
                if (extrap) __stcg(a.phi + i, (PhiT)2 * cur[k] - pv[k]);
                __stcg(prev + i, cur[k]);
                bv = source_value<R, PhiT>(rho[k], i, a.c4, sm, bl, blf);
            }
            __stcg(a.b + i, bv);
        }
    }
    return source_norm<PhiT>(bl, blf, sh);
}

template <typename S, typename R, typename PhiT, bool TILES>
__device__ void mg_solve(const StepArgs<S, R, PhiT> &a, const MgArgs &m, const MgGrid &G, float *mg_sm, double *sh,
                         double *bc)
{
    const Grid3 g = a.g;
    const int nblk = G.nblk;
    const int tid = G.t0, nthr = G.nt;
    const int N = (int)g.N;
    unsigned bar_k = 0;
    int slot = 0;
    // every reduction writes its own rotating slot: a block may run ahead
    // into the next reduction while another still reads the previous one
    auto reduce = [&](double block_value, double &out) -> bool {
        double *p = m.part + (size_t)(slot & 3) * nblk;
        slot++;
        if (threadIdx.x == 0) p[G.blk] = block_value;
        if (!grid_barrier(G.bar, (unsigned)nblk, bar_k, a.status)) return false;
        out = sum_partials(p, nblk, bc);
        return true;
    };
    if (G.blk == 0 && !m.dense) mg_cta_load(m, mg_sm);
    double bb;
    if (!reduce(mg_start_pass(a, m, a.mask, tid, nthr, sh, bc), bb)) return;
    if (a.fixed_iter <= 0 && bb == 0.0) {
        if (tid == 0) {
            *a.pois_iters = 0;
            *a.pois_res = 0.0;
        }
        return;
    }
    const double tol2 = a.tol * a.tol * bb;
    const int limit = a.fixed_iter > 0 ? a.fixed_iter : a.max_iter;
    double rr_true;
    if (!reduce(mg_true_residual<PhiT>(g, a.mask, a.phi, a.b, m.r, m.z, tid, nthr, sh), rr_true)) return;
    double rr_ref = rr_true;
    bool current = true;  // rr_true belongs to the present phi
    bool converged = a.fixed_iter <= 0 && rr_true <= tol2;
    int it = 0, pi = 0;
    bool fresh = true;
    double rz_old = 1.0;
    while (!converged && it < limit) {
        double rzb = 0.0, rz;
        if (!mg_vcycle<S, R, PhiT, TILES>(a, m, G, bar_k, mg_sm, sh, bc, rzb)) return;
        if (!reduce(rzb, rz)) return;
        if (!(rz > 0.0)) break;
        const float beta = fresh ? 0.f : (float)(rz / rz_old);
        rz_old = rz;
        // p = z + beta p_old and q = A p in one pass (p of the neighbours is
        // formed from their z and p_old)
        const float *pold = m.p[pi];
        float *pnew = m.p[pi ^ 1];
        float pq_t = fresh ? mg_pq_pass_lean<true>(g, a.mask, m.z, pold, pnew, m.q, beta, tid, nthr)
                           : mg_pq_pass_lean<false>(g, a.mask, m.z, pold, pnew, m.q, beta, tid, nthr);
        pi ^= 1;
        double pq;
        if (!reduce(block_sum_lanes0(warp_sum_ff_lane0(pq_t), sh), pq)) return;
        if (!(pq > 0.0)) break;
        const double alpha = rz / pq;
        // phi += alpha p, r -= alpha q, and the next V-cycle's first half
        // sweep (colour-0 z = r / deg)
        const float rr_t = mg_update_pass<PhiT>(g, a.mask, a.phi, m.p[pi], m.q, m.r, m.z, alpha, tid, nthr);
        double rr;
        if (!reduce(block_sum_lanes0(warp_sum_ff_lane0(rr_t), sh), rr)) return;
        it++;
        fresh = false;
        current = false;
        if (a.fixed_iter > 0) continue;
        if (rr <= 0.25 * tol2 || rr <= (double)m.inner_red * m.inner_red * rr_ref || it == limit) {
            if (!reduce(mg_true_residual<PhiT>(g, a.mask, a.phi, a.b, m.r, m.z, tid, nthr, sh), rr_true)) return;
            current = true;
            if (rr_true <= tol2) {
                converged = true;
                break;
            }
            rr_ref = rr_true;
            fresh = true;
        }
    }
    if (!current)
        if (!reduce(mg_true_residual<PhiT>(g, a.mask, a.phi, a.b, m.r, m.z, tid, nthr, sh), rr_true)) return;
    if (tid == 0) {
        *a.pois_iters = it;
        a.pois_total[0] += it;
        *a.pois_res = sqrt(rr_true / bb);
        if (a.fixed_iter <= 0 && !(converged || rr_true <= tol2)) atomicOr(a.status, ST_NOCONV);
    }
}

template <typename S, typename R, typename PhiT>
__global__ void __launch_bounds__(MG_THREADS, 1) poisson_mg_kernel(StepArgs<S, R, PhiT> a, MgArgs m)
{
    __shared__ double sh[MG_THREADS / 32];
    __shared__ double bc[1];
    extern __shared__ float mg_sm[];  // block 0: the levels it handles alone
    const MgGrid G{(int)(blockIdx.x * blockDim.x + threadIdx.x), (int)(gridDim.x * blockDim.x), (int)gridDim.x,
                   (int)blockIdx.x, a.barrier};
    mg_solve<S, R, PhiT, true>(a, m, G, mg_sm, sh, bc);
}

// Batched form: block b solves replica block_rep[b] together with the other
// rep_blocks[r] blocks of that replica (local index block_local[b]); each
// replica has its own barrier words bars[4 r ..] and converges on its own.
template <typename S, typename R, typename PhiT>
__global__ void __launch_bounds__(MG_BATCH_THREADS, 1)
    poisson_mg_batch_kernel(const StepArgs<S, R, PhiT> *reps, const MgArgs *mgs, PoisBatch pb, unsigned *bars)
{
    __shared__ double sh[MG_BATCH_THREADS / 32];
    __shared__ double bc[1];
    extern __shared__ float mg_sm[];
    const int r = pb.block_rep[blockIdx.x];
    const int lb = pb.block_local[blockIdx.x], nb = pb.rep_blocks[r];
    const MgGrid G{(int)(lb * blockDim.x + threadIdx.x), (int)(nb * blockDim.x), nb, lb, bars + 4 * r};
    mg_solve<S, R, PhiT, false>(reps[r], mgs[r], G, mg_sm, sh, bc);  // replicas are not tiled
}

}  // namespace ekl
