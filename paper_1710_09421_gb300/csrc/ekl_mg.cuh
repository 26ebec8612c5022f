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
// spread over the grid and separated by the bounded grid barrier; levels at
// and below `cta_from` are handled by block 0 alone while the other blocks
// wait at the next barrier.  Every load of data written inside the launch
// goes through L2 (__ldcg): L1 is not coherent across SMs.
#pragma once
#include "ekl_kernels.cuh"

namespace ekl {

struct MgArgs {
    float *r, *z, *q, *p[2];
    double *part;  // [4][gridDim.x]
    int nlev, cta_from, nu, coarse_sweeps;
    float inner_red;
    MgLevel lev[MG_MAXLEV];
};

__device__ __forceinline__ float mg_inv_deg(int d)
{
    return d == 6 ? (1.f / 6.f) : d == 5 ? 0.2f : d == 4 ? 0.25f : d == 3 ? (1.f / 3.f) : d == 2 ? 0.5f : 1.f;
}
// open faces of a fluid node, bit f in face order (-x, +x, -y, +y, -z, +z)
__device__ __forceinline__ unsigned mg_open(uint32_t m) { return (~(m >> 1)) & 63u; }

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

// ------------------------------------------------------------ lattice level
// Half sweep of colour c of z <- (r + sum_open z_j) / deg.  `first`: z starts
// from zero (colour c takes r / deg, the other colour 0).  `rz`: add r_i z_i
// of both nodes of each pair (only meaningful on the last half sweep of a
// V-cycle, when the other colour is final).
template <bool RZ>
static __device__ void fine_half(const Grid3 &g, const uint32_t *__restrict__ mask, const float *r, float *z, int c,
                          bool first, int t0, int nt, float &rz)
{
    const int hx = (g.nx + 1) >> 1, np = hx * g.ny * g.nz;
    for (int h = t0; h < np; h += nt) {
        const Pair p = mg_pair(h, hx, g.ny, c);
        if (p.x < g.nx) {
            const int i = p.x + g.nx * p.row;
            const uint32_t m = __ldg(mask + i);
            if (!(m & SOLID_BIT)) {
                const unsigned o = mg_open(m);
                const float ri = __ldcg(r + i);
                float v = ri;
                if (!first) {
                    int nb[6];
                    face_nbrs(g, p.x, p.y, p.z, i, nb);
#pragma unroll
                    for (int f = 0; f < 6; f++)
                        if ((o >> f) & 1u) v += __ldcg(z + nb[f]);
                }
                v = o ? v * mg_inv_deg(__popc(o)) : 0.f;
                __stcg(z + i, v);
                if (RZ) rz += ri * v;
            }
        }
        if (p.xo < g.nx) {
            const int io = p.xo + g.nx * p.row;
            if (first) {
                __stcg(z + io, 0.f);
            } else if (RZ) {
                const uint32_t m = __ldg(mask + io);
                if (!(m & SOLID_BIT) && mg_open(m)) rz += __ldcg(r + io) * __ldcg(z + io);
            }
        }
    }
}

// f1 = sum over the children of each level-1 cell of (r - A z)
static __device__ void fine_restrict(const Grid3 &g, const uint32_t *__restrict__ mask, const float *r, const float *z,
                              const MgLevel &C, int t0, int nt)
{
    for (int I = t0; I < C.N; I += nt) {
        const int X = I % C.nx, t = I / C.nx, Y = t % C.ny, Z = t / C.ny;
        float s = 0.f;
        for (int dz = 0; dz < 2; dz++) {
            const int z0 = 2 * Z + dz;
            if (z0 >= g.nz) continue;
            for (int dy = 0; dy < 2; dy++) {
                const int y0 = 2 * Y + dy;
                if (y0 >= g.ny) continue;
                for (int dx = 0; dx < 2; dx++) {
                    const int x0 = 2 * X + dx;
                    if (x0 >= g.nx) continue;
                    const int i = x0 + g.nx * (y0 + g.ny * z0);
                    const uint32_t m = __ldg(mask + i);
                    if (m & SOLID_BIT) continue;
                    const unsigned o = mg_open(m);
                    if (!o) continue;
                    int nb[6];
                    face_nbrs(g, x0, y0, z0, i, nb);
                    float acc = __ldcg(r + i) - (float)__popc(o) * __ldcg(z + i);
#pragma unroll
                    for (int f = 0; f < 6; f++)
                        if ((o >> f) & 1u) acc += __ldcg(z + nb[f]);
                    s += acc;
                }
            }
        }
        __stcg(C.f + I, s);
    }
}

// z += e1(parent) on the fluid nodes
static __device__ void fine_prolong(const Grid3 &g, const uint32_t *__restrict__ mask, float *z, const MgLevel &C, int t0,
                             int nt)
{
    const int N = (int)g.N;
    for (int i = t0; i < N; i += nt) {
        const uint32_t m = __ldg(mask + i);
        if ((m & SOLID_BIT) || !mg_open(m)) continue;
        const int x = i % g.nx, t = i / g.nx, y = t % g.ny, zz = t / g.ny;
        const int I = (x >> 1) + C.nx * ((y >> 1) + C.ny * (zz >> 1));
        __stcg(z + i, __ldcg(z + i) + __ldcg(C.e + I));
    }
}

// ------------------------------------------------------------ coarse levels
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

// Half sweep of colour c of e <- (f + sum sigma e_j) / diag.  Faces beyond a
// closed side carry sigma = 0, so the wrapped neighbour contributes nothing.
static __device__ void coarse_half(const MgLevel &L, int c, bool first, int t0, int nt)
{
    const int hx = (L.nx + 1) >> 1, np = hx * L.ny * L.nz;
    for (int h = t0; h < np; h += nt) {
        const Pair p = mg_pair(h, hx, L.ny, c);
        if (p.x < L.nx) {
            const int i = p.x + L.nx * p.row;
            const float4 s = __ldg(L.sig + i);
            if (first) {
                __stcg(L.e + i, s.w != 0.f ? __ldcg(L.f + i) * s.w : 0.f);
            } else if (s.w != 0.f) {
                const CNbr n = coarse_nbrs(L, p.x, p.y, p.z, i);
                float acc = __ldcg(L.f + i);
                acc += s.x * __ldcg(L.e + n.xp) + __ldg(&L.sig[n.xm].x) * __ldcg(L.e + n.xm);
                acc += s.y * __ldcg(L.e + n.yp) + __ldg(&L.sig[n.ym].y) * __ldcg(L.e + n.ym);
                acc += s.z * __ldcg(L.e + n.zp) + __ldg(&L.sig[n.zm].z) * __ldcg(L.e + n.zm);
                __stcg(L.e + i, acc * s.w);
            }
        }
        if (first && p.xo < L.nx) __stcg(L.e + p.xo + L.nx * p.row, 0.f);
    }
}

// C.f = sum over the children of each cell of level l+1 of (f - A e) on level l
static __device__ void coarse_restrict(const MgLevel &L, const MgLevel &C, int t0, int nt)
{
    for (int I = t0; I < C.N; I += nt) {
        const int X = I % C.nx, t = I / C.nx, Y = t % C.ny, Z = t / C.ny;
        float s = 0.f;
        for (int dz = 0; dz < 2; dz++) {
            const int z0 = 2 * Z + dz;
            if (z0 >= L.nz) continue;
            for (int dy = 0; dy < 2; dy++) {
                const int y0 = 2 * Y + dy;
                if (y0 >= L.ny) continue;
                for (int dx = 0; dx < 2; dx++) {
                    const int x0 = 2 * X + dx;
                    if (x0 >= L.nx) continue;
                    const int i = x0 + L.nx * (y0 + L.ny * z0);
                    const float4 sg = __ldg(L.sig + i);
                    if (sg.w == 0.f) continue;
                    const CNbr n = coarse_nbrs(L, x0, y0, z0, i);
                    const float sxm = __ldg(&L.sig[n.xm].x), sym = __ldg(&L.sig[n.ym].y),
                                szm = __ldg(&L.sig[n.zm].z);
                    const float diag = sg.x + sg.y + sg.z + sxm + sym + szm;
                    float acc = __ldcg(L.f + i) - diag * __ldcg(L.e + i);
                    acc += sg.x * __ldcg(L.e + n.xp) + sxm * __ldcg(L.e + n.xm);
                    acc += sg.y * __ldcg(L.e + n.yp) + sym * __ldcg(L.e + n.ym);
                    acc += sg.z * __ldcg(L.e + n.zp) + szm * __ldcg(L.e + n.zm);
                    s += acc;
                }
            }
        }
        __stcg(C.f + I, s);
    }
}

// e_l += e_{l+1}(parent) on the active cells of level l
static __device__ void coarse_prolong(const MgLevel &L, const MgLevel &C, int t0, int nt)
{
    for (int i = t0; i < L.N; i += nt) {
        if (__ldg(&L.sig[i].w) == 0.f) continue;
        const int x = i % L.nx, t = i / L.nx, y = t % L.ny, z = t / L.ny;
        const int I = (x >> 1) + C.nx * ((y >> 1) + C.ny * (z >> 1));
        __stcg(L.e + i, __ldcg(L.e + i) + __ldcg(C.e + I));
    }
}

// subtract the mean over the active cells of level L from v (block-wide)
static __device__ void coarse_project(const MgLevel &L, float *v, double *sh, double *bc)
{
    double s = 0.0, n = 0.0;
    for (int i = threadIdx.x; i < L.N; i += blockDim.x)
        if (__ldg(&L.sig[i].w) != 0.f) {
            s += (double)__ldcg(v + i);
            n += 1.0;
        }
    const double ts = block_sum(s, sh);
    const double tn = block_sum(n, sh);
    if (threadIdx.x == 0) bc[0] = tn > 0 ? ts / tn : 0.0;
    __syncthreads();
    const float mean = (float)bc[0];
    for (int i = threadIdx.x; i < L.N; i += blockDim.x)
        if (__ldg(&L.sig[i].w) != 0.f) __stcg(v + i, __ldcg(v + i) - mean);
    __syncthreads();
}

// Block 0 alone: the V-cycle below (and including) level m.cta_from.
static __device__ void mg_cta_cycle(const MgArgs &m, double *sh, double *bc)
{
    const int t0 = threadIdx.x, nt = blockDim.x;
    const int last = m.nlev - 1;
    for (int l = m.cta_from; l < last; l++) {
        for (int s = 0; s < 2 * m.nu; s++) {
            coarse_half(m.lev[l], s & 1, s == 0, t0, nt);
            __syncthreads();
        }
        coarse_restrict(m.lev[l], m.lev[l + 1], t0, nt);
        __syncthreads();
    }
    const MgLevel &L = m.lev[last];
    coarse_project(L, L.f, sh, bc);
    for (int s = 0; s < 2 * m.coarse_sweeps + 1; s++) {
        coarse_half(L, s & 1, s == 0, t0, nt);
        __syncthreads();
    }
    coarse_project(L, L.e, sh, bc);
    for (int l = last - 1; l >= m.cta_from; l--) {
        coarse_prolong(m.lev[l], m.lev[l + 1], t0, nt);
        __syncthreads();
        for (int s = 0; s < 2 * m.nu; s++) {
            coarse_half(m.lev[l], (s & 1) ^ 1, false, t0, nt);
            __syncthreads();
        }
    }
}

// One V-cycle z = M^-1 r over the grid; returns this block's partial of r.z
// in thread 0 (through *rz_block) or false on a barrier abort.
template <typename S, typename R, typename PhiT>
__device__ bool mg_vcycle(const StepArgs<S, R, PhiT> &a, const MgArgs &m, unsigned &bar_k, double *sh, double *bc,
                          double &rz_block)
{
    const Grid3 g = a.g;
    const unsigned nblk = gridDim.x;
    const int t0 = blockIdx.x * blockDim.x + threadIdx.x, nt = nblk * blockDim.x;
    float dummy = 0.f;
    // lattice level: pre-smoothing from zero, residual restricted to level 1
    for (int s = 0; s < 2 * m.nu; s++) {
        fine_half<false>(g, a.mask, m.r, m.z, s & 1, s == 0, t0, nt, dummy);
        if (!grid_barrier(a.barrier, nblk, bar_k, a.status)) return false;
    }
    fine_restrict(g, a.mask, m.r, m.z, m.lev[1], t0, nt);
    if (!grid_barrier(a.barrier, nblk, bar_k, a.status)) return false;
    // grid-wide coarse levels
    for (int l = 1; l < m.cta_from; l++) {
        for (int s = 0; s < 2 * m.nu; s++) {
            coarse_half(m.lev[l], s & 1, s == 0, t0, nt);
            if (!grid_barrier(a.barrier, nblk, bar_k, a.status)) return false;
        }
        coarse_restrict(m.lev[l], m.lev[l + 1], t0, nt);
        if (!grid_barrier(a.barrier, nblk, bar_k, a.status)) return false;
    }
    if (blockIdx.x == 0) mg_cta_cycle(m, sh, bc);
    if (!grid_barrier(a.barrier, nblk, bar_k, a.status)) return false;
    for (int l = m.cta_from - 1; l >= 1; l--) {
        coarse_prolong(m.lev[l], m.lev[l + 1], t0, nt);
        if (!grid_barrier(a.barrier, nblk, bar_k, a.status)) return false;
        for (int s = 0; s < 2 * m.nu; s++) {
            coarse_half(m.lev[l], (s & 1) ^ 1, false, t0, nt);
            if (!grid_barrier(a.barrier, nblk, bar_k, a.status)) return false;
        }
    }
    fine_prolong(g, a.mask, m.z, m.lev[1], t0, nt);
    if (!grid_barrier(a.barrier, nblk, bar_k, a.status)) return false;
    float rz = 0.f;
    for (int s = 0; s < 2 * m.nu; s++) {
        const int c = (s & 1) ^ 1;
        if (s == 2 * m.nu - 1) fine_half<true>(g, a.mask, m.r, m.z, c, false, t0, nt, rz);
        else fine_half<false>(g, a.mask, m.r, m.z, c, false, t0, nt, dummy);
        if (s < 2 * m.nu - 1 && !grid_barrier(a.barrier, nblk, bar_k, a.status)) return false;
    }
    rz_block = block_sum_lanes0(warp_sum_ff_lane0(rz), sh);
    return true;
}

// true residual r = b - A phi (exact in the potential type), as FP32, and
// this block's sum of r^2 (thread 0)
template <typename PhiT>
__device__ double mg_true_residual(const Grid3 &g, const uint32_t *__restrict__ mask, const PhiT *phi,
                                   const PhiT *b, float *r, int t0, int nt, double *sh)
{
    float rr = 0.f;
    const int N = (int)g.N;
    for (int i = t0; i < N; i += nt) {
        const uint32_t m = __ldg(mask + i);
        if (m & SOLID_BIT) continue;
        const unsigned o = mg_open(m);
        float rv = 0.f;
        if (o) {
            const int x = i % g.nx, t = i / g.nx, y = t % g.ny, z = t / g.ny;
            int nb[6];
            face_nbrs(g, x, y, z, i, nb);
            PhiT acc = __ldcg(b + i);
#pragma unroll
            for (int f = 0; f < 6; f++)
                if ((o >> f) & 1u) acc += __ldcg(phi + nb[f]);
            acc -= (PhiT)__popc(o) * __ldcg(phi + i);
            if constexpr (((PhiT)0.5) != 0) rv = (float)acc;
            else rv = ll_to_float(acc) * (float)PHI_INV;
        }
        __stcg(r + i, rv);
        rr += rv * rv;
    }
    return block_sum_lanes0(warp_sum_ff_lane0(rr), sh);
}

template <typename S, typename R, typename PhiT>
__global__ void __launch_bounds__(POIS_THREADS, 1) poisson_mg_kernel(StepArgs<S, R, PhiT> a, MgArgs m)
{
    __shared__ double sh[POIS_THREADS / 32];
    __shared__ double bc[1];
    const Grid3 g = a.g;
    const unsigned nblk = gridDim.x;
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    const int nthr = nblk * blockDim.x;
    const int N = (int)g.N;
    unsigned bar_k = 0;
    int slot = 0;
    // every reduction writes its own rotating slot: a block may run ahead
    // into the next reduction while another still reads the previous one
    auto reduce = [&](double block_value, double &out) -> bool {
        double *p = m.part + (size_t)(slot & 3) * nblk;
        slot++;
        if (threadIdx.x == 0) p[blockIdx.x] = block_value;
        if (!grid_barrier(a.barrier, nblk, bar_k, a.status)) return false;
        out = sum_partials(p, (int)nblk, bc);
        return true;
    };
    double bb;
    if (!reduce(form_source(a, tid, nthr, sh, bc), bb)) return;
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
    if (!reduce(mg_true_residual<PhiT>(g, a.mask, a.phi, a.b, m.r, tid, nthr, sh), rr_true)) return;
    double rr_ref = rr_true;
    bool current = true;  // rr_true belongs to the present phi
    bool converged = a.fixed_iter <= 0 && rr_true <= tol2;
    int it = 0, pi = 0;
    bool fresh = true;
    double rz_old = 1.0;
    while (!converged && it < limit) {
        double rzb = 0.0, rz;
        if (!mg_vcycle(a, m, bar_k, sh, bc, rzb)) return;
        if (!reduce(rzb, rz)) return;
        if (!(rz > 0.0)) break;
        const float beta = fresh ? 0.f : (float)(rz / rz_old);
        rz_old = rz;
        // p = z + beta p_old and q = A p in one pass (p of the neighbours is
        // formed from their z and p_old)
        const float *pold = m.p[pi];
        float *pnew = m.p[pi ^ 1];
        float pq_t = 0.f;
        for (int i = tid; i < N; i += nthr) {
            const uint32_t mk = __ldg(a.mask + i);
            if (mk & SOLID_BIT) continue;
            const unsigned o = mg_open(mk);
            if (!o) {
                __stcg(pnew + i, 0.f);
                __stcg(m.q + i, 0.f);
                continue;
            }
            const int x = i % g.nx, t = i / g.nx, y = t % g.ny, z = t / g.ny;
            int nb[6];
            face_nbrs(g, x, y, z, i, nb);
            const float pn = fresh ? __ldcg(m.z + i) : __ldcg(m.z + i) + beta * __ldcg(pold + i);
            float qv = (float)__popc(o) * pn;
#pragma unroll
            for (int f = 0; f < 6; f++)
                if ((o >> f) & 1u)
                    qv -= fresh ? __ldcg(m.z + nb[f]) : __ldcg(m.z + nb[f]) + beta * __ldcg(pold + nb[f]);
            __stcg(pnew + i, pn);
            __stcg(m.q + i, qv);
            pq_t += pn * qv;
        }
        pi ^= 1;
        double pq;
        if (!reduce(block_sum_lanes0(warp_sum_ff_lane0(pq_t), sh), pq)) return;
        if (!(pq > 0.0)) break;
        const double alpha = rz / pq;
        // phi += alpha p, r -= alpha q
        const float alpha_f = (float)alpha;
        const float alpha_fx = (float)(alpha * PHI_SCALE);
        float rr_t = 0.f;
        for (int i = tid; i < N; i += nthr) {
            const uint32_t mk = __ldg(a.mask + i);
            if ((mk & SOLID_BIT) || !mg_open(mk)) continue;
            const float pv = __ldcg(m.p[pi] + i);
            if constexpr (((PhiT)0.5) != 0) __stcg(a.phi + i, __ldcg(a.phi + i) + (double)alpha_f * (double)pv);
            else __stcg(a.phi + i, __ldcg(a.phi + i) + float_to_ll(alpha_fx * pv));
            const float rv = __ldcg(m.r + i) - alpha_f * __ldcg(m.q + i);
            __stcg(m.r + i, rv);
            rr_t += rv * rv;
        }
        double rr;
        if (!reduce(block_sum_lanes0(warp_sum_ff_lane0(rr_t), sh), rr)) return;
        it++;
        fresh = false;
        current = false;
        if (a.fixed_iter > 0) continue;
        if (rr <= 0.25 * tol2 || rr <= (double)m.inner_red * m.inner_red * rr_ref || it == limit) {
            if (!reduce(mg_true_residual<PhiT>(g, a.mask, a.phi, a.b, m.r, tid, nthr, sh), rr_true)) return;
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
        if (!reduce(mg_true_residual<PhiT>(g, a.mask, a.phi, a.b, m.r, tid, nthr, sh), rr_true)) return;
    if (tid == 0) {
        *a.pois_iters = it;
        a.pois_total[0] += it;
        *a.pois_res = sqrt(rr_true / bb);
        if (a.fixed_iter <= 0 && !(converged || rr_true <= tol2)) atomicOr(a.status, ST_NOCONV);
    }
}

}  // namespace ekl
