// Kernels of one electrokinetic LB-MD time step (Sec. II.C algorithm):
//   bead_bin   : bead -> node stencils, deterministic patch list, bead charge
//   charge     : ion densities pulled from the post-collision state, charge
//                density (Eq. 2) with wall and bead charge, FP64 block sums
//   poisson    : persistent red-black Chebyshev SOR for Eq. 3, FP64 residual
//   bead_md    : fluid -> bead interpolation, Langevin sub-steps (Eqs. 7-9),
//                bead drag spread back to the patch nodes
//   lb_fused   : pull-stream with bounce-back + moments + forces (Eqs. 5-6)
//                + BGK collision with forcing (Eqs. 10, 12, 13), one pass
// Template parameters: S = population storage type, R = arithmetic type,
// DEV = populations stored as deviations from w_p n_ref, PhiT = potential
// storage (double, or 64-bit fixed point).
#pragma once
#include <cooperative_groups.h>

#include "ekl_dev.cuh"

namespace ekl {

template <typename R> struct Consts {
    static constexpr R KT = R(1.0) / R(3.0);
    static constexpr R VT2 = R(1.0) / R(3.0);
};

// ============================================================== arguments
template <typename S, typename R, typename PhiT> struct StepArgs {
    Grid3 g;
    int per[3];
    const uint32_t *__restrict__ mask;
    const S *__restrict__ fin;  // post-collision populations of the previous step
    S *__restrict__ fout;       // post-collision populations of this step
    PhiT *phi;
    PhiT *b;
    R *rho;
    const R *__restrict__ wall_share;  // null when no wall carries charge
    const R *__restrict__ src_wall;
    R n_ref[NS];
    R zv[NS];        // valences as reals
    R wd[NS];        // omega_drag
    R om[NS];        // 1 / tau
    R body[NS][3];
    R E[3];
    R c4;            // 4 pi l_B
    int flags;
    // bead patch
    const int *patch_count;
    const uint32_t *patch_bits;  // bit i set when node i is in the patch list
    const int *patch_node;
    const R *patch_q;
    const R *patch_f;
    // reductions / status
    double *part_charge;
    long long *part_charge_q;  // fixed-point paths: exact sum of rho * 2^40 per block
    // totals of those partials (charge_totals), or null: the solve then sums
    // the partials itself
    double *charge_tot;
    long long *charge_tot_q;
    double *part_mass;
    double *part_pois;
    unsigned *barrier;
    int *status;
    int *pois_iters;
    long long *pois_total;
    double *pois_res;
    // Poisson controls
    const void *omegas;  // Chebyshev schedule per half sweep (double, or float for fixed point)
    double tol;
    int max_iter, check_every, fixed_iter;
    double rJ;
    double n_fluid;  // number of fluid nodes (mean charge divisor)
    int nblocks_charge;
    // fluctuating term (Eq. 14)
    const R *wchi;   // w_p chi_kp, [19][19] row k (k = 4..18 used)
    R fluct_m;       // thermal mass m (0: off)
    uint32_t key0, key1;
    long long step;
};

// pull of the 19 populations of species s at node i (bounce-back on set bits)
template <typename S, typename R>
__device__ __forceinline__ void pull19(const S *__restrict__ f, long long N, int s, long long i,
                                       uint32_t m, const Nbr &nb, R v[Q])
{
    // 32-bit offsets inside one species block (19 N < 2^31)
    const S *fs = f + (size_t)s * Q * (size_t)N;
    const int n = (int)N, ii = (int)i;
#pragma unroll
    for (int p = 0; p < Q; p++) {
        const int off = ((m >> p) & 1u) ? opp_(p) * n + ii : p * n + nb.pull(p);
        v[p] = (R)Store<S>::ld(fs + off);
    }
}

// ------------------------------------------------------------ node gradient
// Central differences of phi; a wall (or closed-box) face neighbour takes the
// Neumann ghost value phi_i + 4 pi l_B sigma_face (Sec. II.A boundary condition).
template <typename R, typename PhiT>
__device__ __forceinline__ void node_gradient(const PhiT *phi, const R *wall_share, R c4,
                                              long long i, uint32_t m, const Nbr &nb,
                                              const int out_lo[3], const int out_hi[3], R g[3])
{
    PhiT pi = phi[i];
#pragma unroll
    for (int a = 0; a < 3; a++) {
        int fm = 2 * a, fp = 2 * a + 1;  // minus and plus faces
        bool sm = (m >> (fm + 1)) & 1u, sp = (m >> (fp + 1)) & 1u;
        long long jm = face_idx(nb, fm), jp = face_idx(nb, fp);
        // a face beyond a closed box side is a wall without charge
        const R *wsm = out_lo[a] ? nullptr : wall_share;
        const R *wsp = out_hi[a] ? nullptr : wall_share;
        if constexpr (sizeof(PhiT) == 8 && ((PhiT)0.5) != 0) {
            // FP64: the ghost value enters the difference exactly as written
            double vm = sm ? (double)pi + (wsm ? (double)c4 * (double)wsm[jm] : 0.0)
                           : (double)phi[jm];
            double vp = sp ? (double)pi + (wsp ? (double)c4 * (double)wsp[jp] : 0.0)
                           : (double)phi[jp];
            g[a] = (R)((vp - vm) * 0.5);
        } else {
            PhiT vm = sm ? pi : phi[jm];
            PhiT vp = sp ? pi : phi[jp];
            R d = (R)PhiOps<PhiT>::diff(vp, vm) * R(0.5);
            if (sp && wsp) d += R(0.5) * c4 * wsp[jp];
            if (sm && wsm) d -= R(0.5) * c4 * wsm[jm];
            g[a] = d;
        }
    }
}

// which faces of node (x, y, z) lie beyond a closed box side
__device__ __forceinline__ void closed_faces(const Grid3 &g, const int per[3], int x, int y, int z,
                                             int lo[3], int hi[3])
{
    lo[0] = !per[0] && x == 0; hi[0] = !per[0] && x == g.nx - 1;
    lo[1] = !per[1] && y == 0; hi[1] = !per[1] && y == g.ny - 1;
    lo[2] = !per[2] && z == 0; hi[2] = !per[2] && z == g.nz - 1;
}

// ============================================================== init
template <typename S, typename R, bool DEV>
__global__ void init_kernel(Grid3 g, const uint32_t *__restrict__ mask,
                            const double *__restrict__ n_init, S *__restrict__ f, R n0, R n1, R n2)
{
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= g.N) return;
    bool solid = mask[i] & SOLID_BIT;
    R nref[NS] = {n0, n1, n2};
    for (int s = 0; s < NS; s++) {
        double n = solid ? 0.0 : (n_init ? n_init[(long long)s * g.N + i] : (double)nref[s]);
#pragma unroll
        for (int p = 0; p < Q; p++) {
            double v;
            if (solid) v = 0.0;
            else if (DEV) v = w_(p) * (n - (double)nref[s]);
            else v = w_(p) * n;
            Store<S>::st(f + (long long)(s * Q + p) * g.N + i, (R)v);
        }
    }
}

// ============================================================== charge
// rho_i = sum_a z^a n^a + wall charge + bead charge (Eq. 2), n^a pulled from
// the post-collision state (the streamed densities of this step, Eq. 15).
template <typename S, typename R, typename PhiT, bool DEV>
__device__ __forceinline__ void charge_body(const StepArgs<S, R, PhiT> &a, long long blk)
{
    const Grid3 g = a.g;
    const long long i = blk * (long long)blockDim.x + threadIdx.x;
    R mine = R(0);
    if (i < g.N) {
        const uint32_t m = a.mask[i];
        R rho = R(0);
        if (!(m & SOLID_BIT)) {
            int x, y, z;
            coords_of(g, i, x, y, z);
            Nbr nb = make_nbr(g, x, y, z);
            R v[2][Q];
            pull19<S, R>(a.fin, g.N, 1, i, m, nb, v[0]);
            pull19<S, R>(a.fin, g.N, 2, i, m, nb, v[1]);
            R r = R(0);
            r += a.zv[0] * R(0);  // solvent carries no charge
            for (int s = 1; s < NS; s++) {
                R n = R(0);
#pragma unroll
                for (int p = 0; p < Q; p++) n += v[s - 1][p];
                // Deviation storage: sum_a z^a n^a = sum_a z^a n_ref^a + sum_a z^a dn^a.
                // The first term is the same constant on every fluid node and
                // cancels in the neutralising mean subtraction, so only the
                // deviations enter (no cancellation between two close ion
                // densities in reduced precision).
                r += a.zv[s] * n;
            }
            rho = r + (a.src_wall ? a.src_wall[i] : R(0));
            if ((__ldg(a.patch_bits + (i >> 5)) >> (i & 31)) & 1u) {
                const int pc = *a.patch_count;
                int k = lower_bound_i(a.patch_node, pc, i);
                if (k < pc && a.patch_node[k] == i) rho = rho + a.patch_q[k];
            }
            mine = rho;
        }
        a.rho[i] = rho;
    }
    // one FP64 partial per block (fixed shuffle tree per warp, warps in
    // order), so that the Poisson launch sums few partials
    __shared__ double csh[CHARGE_THREADS / 32];
    double t;
    if constexpr (sizeof(R) == 8) t = warp_sum((double)mine);
    else t = warp_sum_ff_lane0((float)mine);
    t = block_sum_lanes0(t, csh);
    if (threadIdx.x == 0) a.part_charge[blk] = t;
    if constexpr (!(((PhiT)0.5) != 0)) {
        // the fixed-point source's exact total: sum of rho * 2^40 as the
        // Poisson launch rounds it (integer, order-independent)
        __shared__ long long qsh[CHARGE_THREADS / 32];
        long long qv = (i < g.N) ? float_to_ll((float)mine * (float)PHI_SCALE) : 0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) qv += __shfl_xor_sync(0xffffffffu, qv, o);
        if ((threadIdx.x & 31) == 0) qsh[threadIdx.x >> 5] = qv;
        __syncthreads();
        if (threadIdx.x == 0) {
            long long s = 0;
            for (int w = 0; w < (int)(blockDim.x >> 5); w++) s += qsh[w];
            a.part_charge_q[blk] = s;
        }
    }
}

// Totals of the charge pass's block partials, for the Poisson solve, in a
// fixed order, the same for a single run and for a batch replica: block b of
// CHARGE_TOTAL_BLOCKS sums the partials of its contiguous chunk (thread t
// keeps eight running sums, t + 1024 (8 j + u) going to sum u, added in a
// fixed tree; then a fixed shuffle tree per warp and the warps in order); the
// block that finishes last sums the chunk totals in chunk order and resets
// the arrival counter.  FIXED: also the exact integer total of rho * 2^40.
constexpr int CHARGE_TOTAL_BLOCKS = 64;
constexpr size_t CHARGE_CHUNK_BYTES = CHARGE_TOTAL_BLOCKS * (sizeof(double) + sizeof(long long)) + 16;
struct ChargeTotals {
    const double *part;
    const long long *part_q;
    int n;
    double *tot;
    long long *tot_q;
    double *chunk;         // [CHARGE_TOTAL_BLOCKS]
    long long *chunk_q;    // [CHARGE_TOTAL_BLOCKS]
    unsigned *arrived;     // zero between launches
};

template <bool FIXED> __device__ void charge_totals(const ChargeTotals &T)
{
    __shared__ double sh[32];
    __shared__ long long shq[32];
    __shared__ int last;
    constexpr int U = 8;
    const int per = (T.n + CHARGE_TOTAL_BLOCKS - 1) / CHARGE_TOTAL_BLOCKS;
    const int k_beg = blockIdx.x * per, k_end = min(T.n, k_beg + per);
    double v[U];
    long long q = 0;
#pragma unroll
    for (int u = 0; u < U; u++) v[u] = 0.0;
    for (int k0 = k_beg + threadIdx.x; k0 < k_end; k0 += U * blockDim.x) {
#pragma unroll
        for (int u = 0; u < U; u++) {
            const int k = k0 + u * blockDim.x;
            if (k < k_end) {
                v[u] += __ldcg(T.part + k);
                if (FIXED) q += __ldcg(T.part_q + k);
            }
        }
    }
    auto block_ll = [&](long long x) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        __syncthreads();
        if ((threadIdx.x & 31) == 0) shq[threadIdx.x >> 5] = x;
        __syncthreads();
        long long r = 0;
        if (threadIdx.x == 0)
            for (int w = 0; w < (int)(blockDim.x >> 5); w++) r += shq[w];
        return r;
    };
    const double t = block_sum(((v[0] + v[1]) + (v[2] + v[3])) + ((v[4] + v[5]) + (v[6] + v[7])), sh);
    const long long tq = FIXED ? block_ll(q) : 0;
    if (threadIdx.x == 0) {
        __stcg(T.chunk + blockIdx.x, t);
        if (FIXED) __stcg(T.chunk_q + blockIdx.x, tq);
        __threadfence();
        last = atomicAdd(T.arrived, 1u) == CHARGE_TOTAL_BLOCKS - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    const double c = threadIdx.x < CHARGE_TOTAL_BLOCKS ? __ldcg(T.chunk + threadIdx.x) : 0.0;
    const long long cq = (FIXED && threadIdx.x < CHARGE_TOTAL_BLOCKS) ? __ldcg(T.chunk_q + threadIdx.x) : 0;
    const double tt = block_sum(c, sh);
    const long long ttq = FIXED ? block_ll(cq) : 0;
    if (threadIdx.x == 0) {
        *T.tot = tt;
        if (FIXED) *T.tot_q = ttq;
        *T.arrived = 0;
    }
}

template <bool FIXED> __global__ void __launch_bounds__(1024) charge_total_kernel(ChargeTotals T)
{
    charge_totals<FIXED>(T);
}

// the same for every replica of a batch (blockIdx.y: replica)
template <bool FIXED> __global__ void __launch_bounds__(1024) charge_total_batch_kernel(const ChargeTotals *T)
{
    charge_totals<FIXED>(T[blockIdx.y]);
}

template <typename S, typename R, typename PhiT, bool DEV>
__global__ void __launch_bounds__(CHARGE_THREADS) charge_kernel(StepArgs<S, R, PhiT> a)
{
    charge_body<S, R, PhiT, DEV>(a, blockIdx.x);
}

// every replica of a batch in one launch: blockIdx.y selects the replica
template <typename S, typename R, typename PhiT, bool DEV>
__global__ void __launch_bounds__(CHARGE_THREADS) charge_batch_kernel(const StepArgs<S, R, PhiT> *reps)
{
    const StepArgs<S, R, PhiT> &a = reps[blockIdx.y];
    if ((long long)blockIdx.x * blockDim.x >= a.g.N) return;
    charge_body<S, R, PhiT, DEV>(a, blockIdx.x);
}

// ============================================================== Poisson
// Red-black successive over-relaxation with Chebyshev acceleration on the
// 7-point fluid-only finite-volume Laplacian (Eq. 3; Sec. II.C):
//   r_i = b_i + sum_{fluid faces j} phi_j - deg_i phi_i,  phi_i += omega r_i / deg_i
//   omega: 1, 1/(1 - rJ^2/2), then 1/(1 - rJ^2 omega / 4) per half sweep.
// One persistent cooperative launch runs the source set-up, every sweep and
// every convergence test; the residual norm is accumulated from the nodes'
// residuals as they are updated, in FP64, and all blocks reach the same
// decision from the same block partials summed in the same order.
template <typename PhiT> struct PoisUpd;
template <> struct PoisUpd<double> {
    typedef double acc_t;
    typedef double om_t;
    __device__ static double resid(double acc, int deg, double pi) { return acc - deg * pi; }
    __device__ static double apply(double pi, double omega, double r, int deg)
    {
        return pi + omega * r / deg;
    }
    __device__ static double r2(double r) { return r * r; }
};
template <> struct PoisUpd<long long> {
    typedef float acc_t;
    typedef float om_t;
    __device__ static long long resid(long long acc, int deg, long long pi) { return acc - deg * pi; }
    __device__ static long long apply(long long pi, float omega, long long r, int deg)
    {
        const float inv = deg == 6 ? (1.f / 6.f) : deg == 5 ? 0.2f : deg == 4 ? 0.25f
                        : deg == 3 ? (1.f / 3.f) : deg == 2 ? 0.5f : 1.f;
        return pi + float_to_ll(omega * ll_to_float(r) * inv);
    }
    __device__ static float r2(long long r)
    {
        float v = ll_to_float(r) * (float)PHI_INV;
        return v * v;
    }
};

// Neighbour indices of node i = (x, y, z) across its six faces (-x, +x,
// -y, +y, -z, +z), wrapped; faces beyond a closed side are never read (their
// link bit is set).
__device__ __forceinline__ void face_nbrs(const Grid3 &g, int x, int y, int z, int i, int nb[6])
{
    const int nx = g.nx, nxy = g.nx * g.ny;
    nb[0] = x == 0 ? i + nx - 1 : i - 1;
    nb[1] = x == nx - 1 ? i - nx + 1 : i + 1;
    nb[2] = y == 0 ? i + nxy - nx : i - nx;
    nb[3] = y == g.ny - 1 ? i - nxy + nx : i + nx;
    nb[4] = z == 0 ? i + (int)g.N - nxy : i - nxy;
    nb[5] = z == g.nz - 1 ? i - (int)g.N + nxy : i + nxy;
}

// SOR update of one node from its loaded neighbours (acc starts at b_i)
template <typename PhiT>
__device__ __forceinline__ void sor_apply(PhiT *phi, int i, uint32_t m, PhiT bi, PhiT pi, const PhiT v[6],
                                          typename PoisUpd<PhiT>::om_t omega,
                                          typename PoisUpd<PhiT>::acc_t &r2)
{
    PhiT acc = bi;
    int deg = 0;
#pragma unroll
    for (int f = 0; f < 6; f++)
        if (!((m >> (f + 1)) & 1u)) {
            acc += v[f];
            deg++;
        }
    if (deg == 0) return;
    PhiT r = PoisUpd<PhiT>::resid(acc, deg, pi);
    __stcg(phi + i, PoisUpd<PhiT>::apply(pi, omega, r, deg));
    r2 += PoisUpd<PhiT>::r2(r);
}

constexpr int POIS_KMAX = 2;  // nodes per colour a thread keeps in registers

// Poisson source of the step, b = 4 pi l_B (rho - <rho>_fluid) on fluid
// nodes and 0 on walls (Eqs. 2-3 with the neutralising mean of Sec. III).
// SrcMean holds the mean in the forms the per-node formula needs.
struct SrcMean {
    double mean;             // FP64 path: the mean charge over the fluid nodes
    long long mean_lo, C_int;  // fixed-point path: see source_value
    float C_frac;
};

// Every thread of the block must call it (the charge pass's block partials
// are summed by the block).
template <typename S, typename R, typename PhiT>
__device__ SrcMean source_mean(const StepArgs<S, R, PhiT> &a, double *bc)
{
    SrcMean sm{0.0, 0, 0, 0.f};
    const double csum = a.charge_tot ? __ldcg(a.charge_tot) : sum_partials(a.part_charge, a.nblocks_charge, bc);
    const double nfl = a.n_fluid;
    sm.mean = nfl > 0 ? csum / nfl : 0.0;
    // fixed point: the exact total S of rho * 2^40 over the fluid nodes,
    // S / n = mean_lo + frac with 0 <= frac < 1, and C = c4 frac split into
    // integer and fraction
    if constexpr (!(((PhiT)0.5) != 0)) {
        const long long Sq = a.charge_tot ? __ldcg(a.charge_tot_q) : sum_partials_ll(a.part_charge_q, a.nblocks_charge);
        const long long n = (long long)nfl;
        if (n > 0) {
            long long mean_lo = Sq / n;
            long long rem = Sq - mean_lo * n;
            if (rem < 0) {
                mean_lo -= 1;
                rem += n;
            }
            const double C = (double)(float)a.c4 * ((double)rem / (double)n);
            sm.mean_lo = mean_lo;
            sm.C_int = (long long)floor(C);
            sm.C_frac = (float)(C - (double)sm.C_int);
        }
    }
    return sm;
}

// b of one fluid node i with charge density rho; adds b^2 to bl (FP64 path)
// or blf (fixed-point path, in units of the potential)
template <typename R, typename PhiT>
__device__ __forceinline__ PhiT source_value(R rho, long long i, R c4, const SrcMean &sm, double &bl, float &blf)
{
    if constexpr (((PhiT)0.5) != 0) {
        const double v = (double)c4 * ((double)rho - sm.mean);
        bl += v * v;
        return (PhiT)v;
    } else {
        // Fixed point throughout, without FP64 per node.  rho * 2^40 is
        // exact (a power-of-two scaling of an FP32 value; rounded to the
        // nearest 2^-40 below 2^-17) and its total S over the fluid nodes
        // comes exactly from the charge pass; d = q - floor(S / n) is an
        // integer, c4 d is formed as an unevaluated float pair (the
        // product's rounding error recovered by an FMA), the fractional
        // mean enters as C = c4 frac, and x = c4 d - C is rounded to an
        // integer stochastically, floor(x + u) with u uniform per node.
        // The source then sums to zero up to a random walk of unit
        // roundings.  Any rounding shared by many nodes (the mean rounded
        // once, or the same rounding of c4 d on the many nodes that carry
        // the same charge) would instead leave a net source of up to half
        // a unit per node, which a periodic or all-Neumann problem cannot
        // absorb: on 33.5 M nodes it stalled CG near a relative residual
        // of 1e-6.
        const long long d = float_to_ll((float)rho * (float)PHI_SCALE) - sm.mean_lo;
        const float d_hi = ll_to_float(d);
        const float d_lo = ll_to_float(d - float_to_ll(d_hi));  // exact remainder
        const float c4f = (float)c4;
        const float p = c4f * d_hi;
        const float lo = fmaf(c4f, d_hi, -p) + c4f * d_lo;
        const float fp = floorf(p), fl = floorf(lo);
        const float F = (p - fp) + (lo - fl) - sm.C_frac + node_uniform(i);
        const PhiT bv = float_to_ll(fp) + float_to_ll(fl) - sm.C_int + (long long)floorf(F);
        const float v = ll_to_float(bv) * (float)PHI_INV;
        blf += v * v;
        return bv;
    }
}

// block total of the per-thread b^2 sums (valid in thread 0)
template <typename PhiT> __device__ __forceinline__ double source_norm(double bl, float blf, double *sh)
{
    if constexpr (((PhiT)0.5) != 0) return block_sum(bl, sh);
    else return block_sum_lanes0(warp_sum_ff_lane0(blf), sh);
}

// Writes the source to a.b; returns this block's sum of b^2 (valid in
// thread 0).  Every thread of the block must call it.
template <typename S, typename R, typename PhiT>
__device__ double form_source(const StepArgs<S, R, PhiT> &a, int tid, int nthr, double *sh, double *bc)
{
    const SrcMean sm = source_mean(a, bc);
    double bl = 0.0;
    float blf = 0.f;
    for (long long i = tid; i < a.g.N; i += nthr) {
        const uint32_t m = a.mask[i];
        const PhiT bv = (m & SOLID_BIT) ? (PhiT)0 : source_value<R, PhiT>(a.rho[i], i, a.c4, sm, bl, blf);
        __stcg(a.b + i, bv);
    }
    return source_norm<PhiT>(bl, blf, sh);
}

template <typename S, typename R, typename PhiT>
__global__ void __launch_bounds__(POIS_THREADS, 1) poisson_kernel(StepArgs<S, R, PhiT> a)
{
    __shared__ double sh[POIS_THREADS / 32];
    __shared__ double bc[1];
    __shared__ int cflag;
    const Grid3 g = a.g;
    const unsigned nblk = gridDim.x;
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    const int nthr = nblk * blockDim.x;
    unsigned bar_k = 0;
    // --- source: subtract the mean charge over fluid nodes (neutralisation)
    const double t = form_source(a, tid, nthr, sh, bc);
    if (threadIdx.x == 0) a.part_pois[blockIdx.x] = t;
    if (!grid_barrier(a.barrier, nblk, bar_k, a.status)) return;
    const double bn2 = sum_partials(a.part_pois, (int)nblk, bc);
    const double bnorm = sqrt(bn2);
    const int limit = a.fixed_iter > 0 ? a.fixed_iter : a.max_iter;
    if (a.fixed_iter <= 0 && bnorm == 0.0) {
        if (tid == 0) {
            *a.pois_iters = 0;
            *a.pois_res = 0.0;
        }
        return;
    }
    const int hx = (g.nx + 1) >> 1;
    const int nhalf = hx * g.ny * g.nz;
    // register cache of this thread's nodes (both colours) when they fit:
    // node index, link word and packed coordinates
    const bool cached = (nhalf + nthr - 1) / nthr <= POIS_KMAX && g.nx < 2048 && g.ny < 1024 && g.nz < 2048;
    int ci[2][POIS_KMAX], cxyz[2][POIS_KMAX];
    uint32_t cm[2][POIS_KMAX];
    if (cached) {
#pragma unroll
        for (int colour = 0; colour < 2; colour++)
#pragma unroll
            for (int k = 0; k < POIS_KMAX; k++) {
                const int h = tid + k * nthr;
                ci[colour][k] = 0;
                cxyz[colour][k] = 0;
                cm[colour][k] = SOLID_BIT;
                if (h >= nhalf) continue;
                const int row = h / hx, xh = h - row * hx;
                const int z = row / g.ny, y = row - z * g.ny;
                const int x = 2 * xh + ((colour + y + z) & 1);
                if (x >= g.nx) continue;
                const int i = x + g.nx * row;
                ci[colour][k] = i;
                cxyz[colour][k] = x | (y << 11) | (z << 21);
                cm[colour][k] = a.mask[i];
            }
    }
    int it = 0, converged = 0;
    double r2tot = 0.0;
    const double tolb = a.tol * bnorm;
    const typename PoisUpd<PhiT>::om_t *oms = (const typename PoisUpd<PhiT>::om_t *)a.omegas;
    for (it = 0; it < limit; it++) {
        typename PoisUpd<PhiT>::acc_t r2 = 0;
#pragma unroll
        for (int colour = 0; colour < 2; colour++) {
            // Chebyshev relaxation factor of this half sweep (host-computed schedule)
            const typename PoisUpd<PhiT>::om_t omega = __ldg(oms + 2 * it + colour);
            if (cached) {
                // all loads of this thread's nodes first, then the updates
                PhiT v[POIS_KMAX][6], bb[POIS_KMAX], pp[POIS_KMAX];
#pragma unroll
                for (int k = 0; k < POIS_KMAX; k++) {
                    const uint32_t m = cm[colour][k];
                    const int i = ci[colour][k], q = cxyz[colour][k];
                    int nb[6];
                    face_nbrs(g, q & 2047, (q >> 11) & 1023, q >> 21, i, nb);
                    const bool live = !(m & SOLID_BIT);
#pragma unroll
                    for (int f = 0; f < 6; f++)
                        v[k][f] = (live && !((m >> (f + 1)) & 1u)) ? __ldcg(a.phi + nb[f]) : (PhiT)0;
                    bb[k] = live ? __ldcg(a.b + i) : (PhiT)0;
                    pp[k] = live ? __ldcg(a.phi + i) : (PhiT)0;
                }
#pragma unroll
                for (int k = 0; k < POIS_KMAX; k++)
                    if (!(cm[colour][k] & SOLID_BIT))
                        sor_apply<PhiT>(a.phi, ci[colour][k], cm[colour][k], bb[k], pp[k], v[k], omega, r2);
            } else {
                for (int h = tid; h < nhalf; h += nthr) {
                    const int row = h / hx, xh = h - row * hx;
                    const int z = row / g.ny, y = row - z * g.ny;
                    const int x = 2 * xh + ((colour + y + z) & 1);
                    if (x >= g.nx) continue;
                    const int i = x + g.nx * row;
                    const uint32_t m = a.mask[i];
                    if (m & SOLID_BIT) continue;
                    int nb[6];
                    face_nbrs(g, x, y, z, i, nb);
                    PhiT v[6];
#pragma unroll
                    for (int f = 0; f < 6; f++) v[f] = ((m >> (f + 1)) & 1u) ? (PhiT)0 : __ldcg(a.phi + nb[f]);
                    sor_apply<PhiT>(a.phi, i, m, __ldcg(a.b + i), __ldcg(a.phi + i), v, omega, r2);
                }
            }
            // the residual norm is only needed on the sweeps that test it
            const bool need = (a.fixed_iter <= 0 && ((it + 1) % a.check_every) == 0) || it + 1 == limit;
            if (colour == 1 && need) {
                double wsum;
                if constexpr (((PhiT)0.5) != 0) wsum = warp_sum((double)r2);
                else wsum = warp_sum_ff_lane0((float)r2);
                double tb = block_sum_lanes0(wsum, sh);
                if (threadIdx.x == 0) a.part_pois[blockIdx.x] = tb;
            }
            if (!grid_barrier(a.barrier, nblk, bar_k, a.status)) return;
        }
        const bool test = a.fixed_iter <= 0 && ((it + 1) % a.check_every) == 0;
        if (test || it + 1 == limit) {
            if (test_partials(a.part_pois, (int)nblk, tolb, bc, &cflag, r2tot) && test) {
                converged = 1;
                it++;
                break;
            }
        }
    }
    if (tid == 0) {
        *a.pois_iters = it;
        a.pois_total[0] += it;
        *a.pois_res = sqrt(r2tot) / bnorm;
        if (a.fixed_iter <= 0 && !converged) atomicOr(a.status, ST_NOCONV);
    }
}

// ---------------------------------------------------------------- tiled SOR
// Shared-memory-resident variant for lattices whose (y, z) tiles fit one SM
// each: block t owns the full-x slab tile T = [y0, y0+ty) x [z0, z0+tz) and
// keeps T plus a 2-deep (y, z) halo of phi, the source and the link words in
// shared memory for the whole solve.  A sweep updates the red nodes of T and
// of the first halo layer (the halo red values are recomputed from the same
// inputs as their owner's, so they are bitwise the owner's), then the black
// nodes of T, writes T to global memory and passes one grid barrier; the
// next sweep reloads only the halo.  Results are bitwise those of the
// global-memory kernel (same node updates, same schedule).
struct TileGeom {
    int ty, tz, nty, ntz;  // tile extents and tile counts along y and z
};

template <typename PhiT>
__device__ __forceinline__ void tile_update(PhiT *ps, const PhiT *bs, const uint32_t *ms, int nx, int ey,
                                            int e, int x, uint32_t m, typename PoisUpd<PhiT>::om_t omega,
                                            typename PoisUpd<PhiT>::acc_t &r2, bool count)
{
    const int ex = nx * ey;  // stride of lz
    // face neighbours in the extended frame (x wraps inside the row)
    const int nb[6] = {x == 0 ? e + nx - 1 : e - 1, x == nx - 1 ? e - nx + 1 : e + 1, e - nx, e + nx,
                       e - ex, e + ex};
    PhiT acc = bs[e];
    int deg = 0;
#pragma unroll
    for (int f = 0; f < 6; f++)
        if (!((m >> (f + 1)) & 1u)) {
            acc += ps[nb[f]];
            deg++;
        }
    if (deg == 0) return;
    const PhiT pi = ps[e];
    const PhiT r = PoisUpd<PhiT>::resid(acc, deg, pi);
    ps[e] = PoisUpd<PhiT>::apply(pi, omega, r, deg);
    if (count) r2 += PoisUpd<PhiT>::r2(r);
}

template <typename S, typename R, typename PhiT>
__global__ void __launch_bounds__(POIS_THREADS, 1) poisson_tiled_kernel(StepArgs<S, R, PhiT> a, TileGeom tg)
{
    extern __shared__ __align__(16) unsigned char tsm[];
    __shared__ double sh[POIS_THREADS / 32];
    __shared__ double bc[1];
    __shared__ int cflag;
    const Grid3 g = a.g;
    const unsigned nblk = gridDim.x;
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    const int nthr = nblk * blockDim.x;
    unsigned bar_k = 0;
    const int nx = g.nx, ey = tg.ty + 4, ez = tg.tz + 4, E = nx * ey * ez;
    PhiT *ps = (PhiT *)tsm;
    PhiT *bs = ps + E;
    uint32_t *ms = (uint32_t *)(bs + E);
    const int by = blockIdx.x % tg.nty, bz = blockIdx.x / tg.nty;
    const int y0 = by * tg.ty - 2, z0 = bz * tg.tz - 2;  // global coordinates of the extended origin
    // --- source (grid-wide, as in the global kernel)
    const double t = form_source(a, tid, nthr, sh, bc);
    if (threadIdx.x == 0) a.part_pois[blockIdx.x] = t;
    if (!grid_barrier(a.barrier, nblk, bar_k, a.status)) return;
    const double bn2 = sum_partials(a.part_pois, (int)nblk, bc);
    const double bnorm = sqrt(bn2);
    const int limit = a.fixed_iter > 0 ? a.fixed_iter : a.max_iter;
    if (a.fixed_iter <= 0 && bnorm == 0.0) {
        if (tid == 0) {
            *a.pois_iters = 0;
            *a.pois_res = 0.0;
        }
        return;
    }
    // --- load the extended tile: link words, source, potential.  Loops run
    // one warp per (ly, lz) row and one lane per x, so the row decomposition
    // costs one division per row.
    auto gidx = [&](int ly, int lz, int &gi) -> bool {
        int y = y0 + ly, z = z0 + lz;
        if (y < 0 || y >= g.ny) {
            if (!a.per[1]) return false;
            y = (y % g.ny + g.ny) % g.ny;
        }
        if (z < 0 || z >= g.nz) {
            if (!a.per[2]) return false;
            z = (z % g.nz + g.nz) % g.nz;
        }
        gi = nx * (y + g.ny * z);
        return true;
    };
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int rows = ey * ez;
    for (int row = warp; row < rows; row += nwarps) {
        const int ly = row % ey, lz = row / ey;
        int gi;
        const bool in = gidx(ly, lz, gi);
        const int e0 = nx * row;
        for (int x = lane; x < nx; x += 32) {
            ms[e0 + x] = in ? a.mask[gi + x] : SOLID_BIT;
            bs[e0 + x] = in ? __ldcg(a.b + gi + x) : (PhiT)0;
            ps[e0 + x] = in ? __ldcg(a.phi + gi + x) : (PhiT)0;
        }
    }
    __syncthreads();
    int it = 0, converged = 0;
    double r2tot = 0.0;
    const double tolb = a.tol * bnorm;
    const typename PoisUpd<PhiT>::om_t *oms = (const typename PoisUpd<PhiT>::om_t *)a.omegas;
    const int ty = tg.ty, tz = tg.tz;
    const int hx = (nx + 1) >> 1;
    for (it = 0; it < limit; it++) {
        typename PoisUpd<PhiT>::acc_t r2 = 0;
        if (it > 0) {
            // reload the halo rows (rows outside the owned tile)
            for (int row = warp; row < rows; row += nwarps) {
                const int ly = row % ey, lz = row / ey;
                if (ly >= 2 && ly < ty + 2 && lz >= 2 && lz < tz + 2) continue;
                int gi;
                if (!gidx(ly, lz, gi)) continue;
                const int e0 = nx * row;
                for (int x = lane; x < nx; x += 32) ps[e0 + x] = __ldcg(a.phi + gi + x);
            }
            __syncthreads();
        }
        const typename PoisUpd<PhiT>::om_t om_r = __ldg(oms + 2 * it), om_b = __ldg(oms + 2 * it + 1);
        // red nodes of T and of the first halo layer
        {
            const int ny1 = ty + 2, nrow = ny1 * (tz + 2);
            for (int rr = warp; rr < nrow; rr += nwarps) {
                const int ly = 1 + rr % ny1, lz = 1 + rr / ny1;
                const int par = (y0 + ly + z0 + lz) & 1;   // red: (x + y + z) even
                const bool own = ly >= 2 && ly < ty + 2 && lz >= 2 && lz < tz + 2;
                const int e0 = nx * (ly + ey * lz);
                for (int xh = lane; xh < hx; xh += 32) {
                    const int x = 2 * xh + par;
                    if (x >= nx) continue;
                    const uint32_t m = ms[e0 + x];
                    if (m & SOLID_BIT) continue;
                    tile_update<PhiT>(ps, bs, ms, nx, ey, e0 + x, x, m, om_r, r2, own);
                }
            }
        }
        __syncthreads();
        // black nodes of T
        {
            const int nrow = ty * tz;
            for (int rr = warp; rr < nrow; rr += nwarps) {
                const int ly = 2 + rr % ty, lz = 2 + rr / ty;
                const int par = (y0 + ly + z0 + lz + 1) & 1;  // black: (x + y + z) odd
                const int e0 = nx * (ly + ey * lz);
                for (int xh = lane; xh < hx; xh += 32) {
                    const int x = 2 * xh + par;
                    if (x >= nx) continue;
                    const uint32_t m = ms[e0 + x];
                    if (m & SOLID_BIT) continue;
                    tile_update<PhiT>(ps, bs, ms, nx, ey, e0 + x, x, m, om_b, r2, true);
                }
            }
        }
        __syncthreads();
        // owned rows back to global memory
        for (int rr = warp; rr < ty * tz; rr += nwarps) {
            const int ly = 2 + rr % ty, lz = 2 + rr / ty;
            const int gi = nx * ((y0 + ly) + g.ny * (z0 + lz));
            const int e0 = nx * (ly + ey * lz);
            for (int x = lane; x < nx; x += 32) __stcg(a.phi + gi + x, ps[e0 + x]);
        }
        const bool need = (a.fixed_iter <= 0 && ((it + 1) % a.check_every) == 0) || it + 1 == limit;
        if (need) {
            double wsum;
            if constexpr (((PhiT)0.5) != 0) wsum = warp_sum((double)r2);
            else wsum = warp_sum_ff_lane0((float)r2);
            double tb = block_sum_lanes0(wsum, sh);
            if (threadIdx.x == 0) a.part_pois[blockIdx.x] = tb;
        }
        if (!grid_barrier(a.barrier, nblk, bar_k, a.status)) return;
        const bool test = a.fixed_iter <= 0 && ((it + 1) % a.check_every) == 0;
        if (test || it + 1 == limit) {
            if (test_partials(a.part_pois, (int)nblk, tolb, bc, &cflag, r2tot) && test) {
                converged = 1;
                it++;
                break;
            }
        }
    }
    if (tid == 0) {
        *a.pois_iters = it;
        a.pois_total[0] += it;
        *a.pois_res = sqrt(r2tot) / bnorm;
        if (a.fixed_iter <= 0 && !converged) atomicOr(a.status, ST_NOCONV);
    }
}

// ---------------------------------------------------------------- batched SOR
// Every replica of a batch in one persistent cooperative launch.  Blocks are
// split among replicas (block_rep / block_local, rep_blocks per replica); all
// replicas sweep in lockstep behind one grid barrier per half sweep, each with
// its own Chebyshev schedule, tolerance and iteration cap, and a replica that
// has converged (or reached its cap) stops updating.  Every block evaluates
// every replica's residual test from the same partials in the same order, so
// all blocks agree on who is still active without extra synchronisation.
constexpr int MAX_REPS = 256;

struct PoisBatch {
    int nrep;
    const int *block_rep;
    const int *block_local;
    const int *rep_blocks;
    unsigned *barrier;
    int *status;
};

template <typename S, typename R, typename PhiT>
__global__ void __launch_bounds__(POIS_THREADS, 1) poisson_batch_kernel(const StepArgs<S, R, PhiT> *reps, PoisBatch pb)
{
    __shared__ double sh[POIS_THREADS / 32];
    __shared__ double s_tolb[MAX_REPS], s_bnorm[MAX_REPS], s_res[MAX_REPS];
    __shared__ int s_active[MAX_REPS], s_iters[MAX_REPS], s_conv[MAX_REPS], s_any;
    const int rep = pb.block_rep[blockIdx.x], lb = pb.block_local[blockIdx.x], kr = pb.rep_blocks[rep];
    const StepArgs<S, R, PhiT> &a = reps[rep];
    const Grid3 g = a.g;
    const int tid = lb * blockDim.x + threadIdx.x, nthr = kr * blockDim.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    unsigned bar_k = 0;
    // --- source of this replica (mean over its fluid nodes)
    __shared__ double bc[1];
    const double t = form_source(a, tid, nthr, sh, bc);
    if (threadIdx.x == 0) a.part_pois[lb] = t;
    if (!grid_barrier(pb.barrier, gridDim.x, bar_k, pb.status)) return;
    // every replica's source norm and activity, in every block
    for (int r = threadIdx.x; r < pb.nrep; r += blockDim.x) {
        const StepArgs<S, R, PhiT> &q = reps[r];
        double v = 0.0;
        for (int k = 0; k < pb.rep_blocks[r]; k++) v += __ldcg(q.part_pois + k);
        const double bn = sqrt(v);
        s_bnorm[r] = bn;
        s_tolb[r] = q.tol * bn;
        s_active[r] = !(q.fixed_iter <= 0 && bn == 0.0);
        s_iters[r] = 0;
        s_res[r] = 0.0;
        s_conv[r] = 0;
    }
    __syncthreads();
    const int hx = (g.nx + 1) >> 1;
    const int rows = g.ny * g.nz;
    const typename PoisUpd<PhiT>::om_t *oms = (const typename PoisUpd<PhiT>::om_t *)a.omegas;
    for (int it = 0;; it++) {
        // who is still sweeping: within its cap and not converged
        if (threadIdx.x == 0) {
            int any = 0;
            for (int r = 0; r < pb.nrep; r++) {
                const StepArgs<S, R, PhiT> &q = reps[r];
                const int lim = q.fixed_iter > 0 ? q.fixed_iter : q.max_iter;
                if (s_active[r] && it >= lim) s_active[r] = 0;
                any |= s_active[r];
            }
            s_any = any;
        }
        __syncthreads();
        if (!s_any) break;
        const bool mine = s_active[rep] != 0;
        const bool need = mine && ((a.fixed_iter <= 0 && ((it + 1) % a.check_every) == 0) ||
                                   it + 1 == (a.fixed_iter > 0 ? a.fixed_iter : a.max_iter));
        typename PoisUpd<PhiT>::acc_t r2 = 0;
#pragma unroll
        for (int colour = 0; colour < 2; colour++) {
            if (mine) {
                const typename PoisUpd<PhiT>::om_t omega = __ldg(oms + 2 * it + colour);
                for (int row = lb * nwarps + warp; row < rows; row += kr * nwarps) {
                    const int z = row / g.ny, y = row - z * g.ny;
                    const int par = (colour + y + z) & 1;
                    for (int xh = lane; xh < hx; xh += 32) {
                        const int x = 2 * xh + par;
                        if (x >= g.nx) continue;
                        const int i = x + g.nx * row;
                        const uint32_t m = a.mask[i];
                        if (m & SOLID_BIT) continue;
                        int nb[6];
                        face_nbrs(g, x, y, z, i, nb);
                        PhiT v[6];
#pragma unroll
                        for (int f = 0; f < 6; f++) v[f] = ((m >> (f + 1)) & 1u) ? (PhiT)0 : __ldcg(a.phi + nb[f]);
                        sor_apply<PhiT>(a.phi, i, m, __ldcg(a.b + i), __ldcg(a.phi + i), v, omega, r2);
                    }
                }
            }
            if (colour == 1 && need) {
                double wsum;
                if constexpr (((PhiT)0.5) != 0) wsum = warp_sum((double)r2);
                else wsum = warp_sum_ff_lane0((float)r2);
                double tb = block_sum_lanes0(wsum, sh);
                if (threadIdx.x == 0) a.part_pois[lb] = tb;
            }
            if (!grid_barrier(pb.barrier, gridDim.x, bar_k, pb.status)) return;
        }
        // residual tests of every replica that tests at this sweep
        for (int r = threadIdx.x; r < pb.nrep; r += blockDim.x) {
            if (!s_active[r]) continue;
            const StepArgs<S, R, PhiT> &q = reps[r];
            const int lim = q.fixed_iter > 0 ? q.fixed_iter : q.max_iter;
            const bool test = q.fixed_iter <= 0 && ((it + 1) % q.check_every) == 0;
            if (!test && it + 1 != lim) continue;
            double v = 0.0;
            for (int k = 0; k < pb.rep_blocks[r]; k++) v += __ldcg(q.part_pois + k);
            s_res[r] = v;
            s_iters[r] = it + 1;
            if (test && sqrt(v) <= s_tolb[r]) {
                s_active[r] = 0;
                s_conv[r] = 1;
            }
        }
        for (int r = threadIdx.x; r < pb.nrep; r += blockDim.x)
            if (s_active[r]) s_iters[r] = it + 1;
        __syncthreads();
    }
    if (lb == 0 && threadIdx.x == 0) {
        const int itr = s_iters[rep];
        *a.pois_iters = itr;
        a.pois_total[0] += itr;
        *a.pois_res = s_bnorm[rep] > 0 ? sqrt(s_res[rep]) / s_bnorm[rep] : 0.0;
        if (a.fixed_iter <= 0 && !s_conv[rep] && s_bnorm[rep] > 0.0) atomicOr(a.status, ST_NOCONV);
    }
}

template <typename PhiT> inline size_t tile_smem_bytes(int nx, const TileGeom &tg)
{
    return (size_t)nx * (tg.ty + 4) * (tg.tz + 4) * (2 * sizeof(PhiT) + sizeof(uint32_t));
}

// ============================================================== beads
// Bead positions are FP64 in every precision: a float position near x = 64
// has an ulp of 7.6e-6, too coarse for sub-step displacements of ~1e-4.
// Velocities, forces and the drag use the arithmetic type R.
template <typename R> struct BeadArgs {
    Grid3 g;
    int per[3];
    const uint32_t *__restrict__ mask;
    int nb;
    double *Rb;
    R *Vb;
    const R *qb;
    const int *chain;
    int *patch_count;
    uint32_t *patch_bits;
    int *patch_node;
    R *patch_q;
    R *patch_f;
    R *patch_mom;
    int *entry_slot;
    R *entry_w;
    int *sorted_entry;
    int *slot_first;
    int *status;
};

// Trilinear weights of the 8 nodes around a bead, wall nodes weighted zero
// and the rest renormalised (the interpolation kernel of Sec. II.C).
// Slot order k = ox + 2 oy + 4 oz.  Returns false when all 8 are wall.
template <typename R>
__device__ bool bead_stencil(const Grid3 &g, const int per[3], const uint32_t *mask, const double Rb[3],
                             long long nodes[8], R w[8])
{
    int base[3];
    R fr[3];
    int dims[3] = {g.nx, g.ny, g.nz};
    for (int c = 0; c < 3; c++)
        if (!(fabs(Rb[c]) < 1e6)) return false;  // non-finite or absurd position
    for (int c = 0; c < 3; c++) {
        double fl = floor(Rb[c]);
        base[c] = (int)fl;
        fr[c] = (R)(Rb[c] - fl);
    }
    // node ids first (a position in [0, L) on a periodic axis puts every
    // corner within one period, so a single add or subtract wraps it), then
    // all eight link words are loaded together
    uint32_t mk[8];
#pragma unroll
    for (int k = 0; k < 8; k++) {
        const int o[3] = {k & 1, (k >> 1) & 1, (k >> 2) & 1};
        int q[3];
        bool in = true;
        for (int c = 0; c < 3; c++) {
            int v = base[c] + o[c];
            if (per[c]) {
                if (v >= dims[c]) v -= dims[c];
                else if (v < 0) v += dims[c];
                if (v < 0 || v >= dims[c]) {  // far outside the box: the general wrap
                    v %= dims[c];
                    if (v < 0) v += dims[c];
                }
            } else if (v < 0 || v >= dims[c]) {
                in = false;
            }
            q[c] = v;
        }
        nodes[k] = in ? (long long)q[0] + (long long)g.nx * (q[1] + (long long)g.ny * q[2]) : -1;
    }
#pragma unroll
    for (int k = 0; k < 8; k++) mk[k] = nodes[k] >= 0 ? mask[nodes[k]] : SOLID_BIT;
    R W = R(0);
#pragma unroll
    for (int k = 0; k < 8; k++) {
        const int o[3] = {k & 1, (k >> 1) & 1, (k >> 2) & 1};
        R wk = R(1);
        for (int c = 0; c < 3; c++) wk *= o[c] ? fr[c] : R(1) - fr[c];
        w[k] = (mk[k] & SOLID_BIT) ? R(0) : wk;
        W += w[k];
    }
    if (!(W > R(0))) return false;
    for (int k = 0; k < 8; k++) w[k] = w[k] / W;
    return true;
}

// One block: stencils of all beads, entries sorted by (node, bead) with a
// bitonic sort in shared memory, unique nodes -> patch slots (ascending node
// id), the sorted entry list with each slot's first position, and the bead
// charge per slot summed in bead order.
template <typename R> __device__ void bead_bin_body(const BeadArgs<R> &a)
{
    __shared__ unsigned long long key[MAX_ENTRIES];
    __shared__ int flag[MAX_ENTRIES];
    const int ne = a.nb * 8;
    int npow = 1;
    while (npow < ne) npow <<= 1;
    // clear the previous step's patch bits (the list is rewritten below,
    // after several block barriers)
    {
        const int old = *a.patch_count;
        for (int k = threadIdx.x; k < old; k += blockDim.x) {
            const int nd = a.patch_node[k];
            atomicAnd(a.patch_bits + (nd >> 5), ~(1u << (nd & 31)));
        }
    }
    for (int b = threadIdx.x; b < a.nb; b += blockDim.x) {
        double Rb[3] = {a.Rb[3 * b], a.Rb[3 * b + 1], a.Rb[3 * b + 2]};
        long long nd[8];
        R w[8];
        bool ok = bead_stencil<R>(a.g, a.per, a.mask, Rb, nd, w);
        if (!ok) atomicOr(a.status, ST_BEAD);
        for (int k = 0; k < 8; k++) {
            int e = b * 8 + k;
            a.entry_w[e] = ok ? w[k] : R(0);
            bool use = ok && nd[k] >= 0 && !(a.mask[nd[k]] & SOLID_BIT);
            key[e] = use ? (((unsigned long long)nd[k] << 20) | (unsigned)e) : ~0ull;
        }
    }
    for (int e = ne + threadIdx.x; e < npow; e += blockDim.x) key[e] = ~0ull;
    __syncthreads();
    for (int k = 2; k <= npow; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int t = threadIdx.x; t < npow; t += blockDim.x) {
                int ixj = t ^ j;
                if (ixj > t) {
                    unsigned long long u = key[t], v = key[ixj];
                    bool up = (t & k) == 0;
                    if ((u > v) == up) {
                        key[t] = v;
                        key[ixj] = u;
                    }
                }
            }
            __syncthreads();
        }
    }
    // slots: an entry starts a slot when its node differs from the previous
    // entry's; slot index = inclusive prefix count of starts - 1 (block scan:
    // each thread takes a contiguous chunk, warps scan their chunk totals by
    // shuffles, warp totals are scanned once); unused keys (~0) sort last
    {
        __shared__ int wtot[BEAD_THREADS / 32];
        __shared__ int s_nvalid;
        const int per = (npow + blockDim.x - 1) / blockDim.x;
        const int t0 = threadIdx.x * per, t1 = min(t0 + per, npow);
        int local = 0;
        for (int t = t0; t < t1; t++) {
            const unsigned long long u = key[t];
            local += (u != ~0ull) && (t == 0 || (key[t - 1] >> 20) != (u >> 20));
        }
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
        int incl = local;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        if (lane == 31) wtot[wid] = incl;
        if (threadIdx.x == 0) s_nvalid = npow;
        __syncthreads();
        int before = 0;
        for (int w = 0; w < wid; w++) before += wtot[w];
        int run = before + incl - local;  // starts before this thread's chunk
        for (int t = t0; t < t1; t++) {
            const unsigned long long u = key[t];
            if (u == ~0ull) {
                flag[t] = -1;
                if (t == 0 || key[t - 1] != ~0ull) s_nvalid = t;  // first unused key
                continue;
            }
            if (t == 0 || (key[t - 1] >> 20) != (u >> 20)) {
                a.slot_first[run] = t;
                run++;
            }
            flag[t] = run - 1;
        }
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) {
            int c = 0;
            for (int w = 0; w < (int)(blockDim.x >> 5); w++) c += wtot[w];
            a.slot_first[c] = s_nvalid;
            *a.patch_count = c;
        }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < ne; t += blockDim.x) a.entry_slot[t] = -1;
    __syncthreads();
    for (int t = threadIdx.x; t < npow; t += blockDim.x) {
        unsigned long long u = key[t];
        if (u == ~0ull) continue;
        int e = (int)(u & 0xFFFFFu);
        a.entry_slot[e] = flag[t];
        a.sorted_entry[t] = e;
        if (t == 0 || (key[t - 1] >> 20) != (u >> 20)) {
            const int nd = (int)(u >> 20);
            a.patch_node[flag[t]] = nd;
            atomicOr(a.patch_bits + (nd >> 5), 1u << (nd & 31));
        }
    }
    __syncthreads();
    const int pc = *a.patch_count;
    for (int k = threadIdx.x; k < pc; k += blockDim.x) {
        R acc = R(0);
        for (int t = a.slot_first[k]; t < a.slot_first[k + 1]; t++) {
            int e = a.sorted_entry[t];
            R w = a.entry_w[e];
            if (w != R(0)) acc += a.qb[e >> 3] * w;
        }
        a.patch_q[k] = acc;
    }
}

template <typename R> __global__ void __launch_bounds__(BEAD_THREADS) bead_bin_kernel(BeadArgs<R> a)
{
    bead_bin_body<R>(a);
}

template <typename R> __global__ void __launch_bounds__(BEAD_THREADS) bead_bin_batch_kernel(const BeadArgs<R> *reps)
{
    const BeadArgs<R> &a = reps[blockIdx.y];
    if (a.nb == 0) return;
    bead_bin_body<R>(a);
}

template <typename R>
__device__ __forceinline__ void wca_add(R eps, R sig, const R d[3], R F[3])
{
    R r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    // 2^(1/3) sigma^2 is the squared WCA cut-off
    R rc2 = (R)1.2599210498948732 * sig * sig;
    if (r2 >= rc2) return;
    R mag;
    if constexpr (sizeof(R) == 8) {  // FP64: divisions as the oracle writes them
        R sr2 = sig * sig / r2;
        R sr6 = sr2 * sr2 * sr2;
        mag = R(24) * eps * (R(2) * sr6 * sr6 - sr6) / r2;
    } else {
        const R inv = R(1) / r2;
        R sr2 = sig * sig * inv;
        R sr6 = sr2 * sr2 * sr2;
        mag = R(24) * eps * (R(2) * sr6 * sr6 - sr6) * inv;
    }
    for (int c = 0; c < 3; c++) F[c] += mag * d[c];
}

// separation Rb - Rc in FP64 with the minimum image on periodic axes
// (|d| < L because positions are kept in [0, L) on periodic axes)
template <typename R>
__device__ __forceinline__ void separation(const Grid3 &g, const int per[3], const double *Rb,
                                           const double *Rc, R d[3])
{
    const double L[3] = {(double)g.nx, (double)g.ny, (double)g.nz};
    for (int c = 0; c < 3; c++) {
        double v = Rb[c] - Rc[c];
        if (per[c]) {
            if (v > 0.5 * L[c]) v -= L[c];
            else if (v < -0.5 * L[c]) v += L[c];
        }
        d[c] = (R)v;
    }
}

// Reduced-precision paths: inside the MD kernel bead positions are signed
// 64-bit fixed point with 40 fractional bits, so separations, wraps and the
// position update stay on the integer pipe (GB300's FP64 rate would
// otherwise dominate the sub-steps); the separation is then converted to FP32.
__device__ __forceinline__ void separation(const Grid3 &g, const int per[3], const long long *Rb,
                                           const long long *Rc, float d[3])
{
    const long long L[3] = {(long long)g.nx << 40, (long long)g.ny << 40, (long long)g.nz << 40};
    for (int c = 0; c < 3; c++) {
        long long v = Rb[c] - Rc[c];
        if (per[c]) {
            if (v > (L[c] >> 1)) v -= L[c];
            else if (v < -(L[c] >> 1)) v += L[c];
        }
        d[c] = ll_to_float(v) * (float)PHI_INV;
    }
}

template <typename S, typename R, typename PhiT, bool DEV> struct MdArgs {
    StepArgs<S, R, PhiT> s;
    BeadArgs<R> b;
    int md_substeps;
    R xi, mass, bead_kT;
    int bond_kind;
    R bond_k, bond_r0, bond_l0, wca_eps, wca_sigma, wall_eps, wall_sigma;
    uint32_t key0, key1;
    long long step;
};

// Solid flags of a WALL_BOX^3 block of nodes around each bead, cached in
// shared memory for the sub-steps (bit (z*WALL_BOX + y)*WALL_BOX + x of the
// bead's words, origin org).
constexpr int WALL_BOX = 6;
constexpr int WALL_WORDS = (WALL_BOX * WALL_BOX * WALL_BOX + 31) / 32;

__device__ __forceinline__ bool wall_solid(const Grid3 &g, const int per[3], const uint32_t *mask,
                                           int x, int y, int z, const int *org, const uint32_t *bits,
                                           bool &in)
{
    // inside the cached block the bit already encodes the wrap and the box
    // faces (a node beyond a closed face was cached as fluid)
    const int ox = x - org[0], oy = y - org[1], oz = z - org[2];
    if (ox >= 0 && ox < WALL_BOX && oy >= 0 && oy < WALL_BOX && oz >= 0 && oz < WALL_BOX) {
        in = true;
        const int bit = (oz * WALL_BOX + oy) * WALL_BOX + ox;
        return (bits[bit >> 5] >> (bit & 31)) & 1u;
    }
    int q[3] = {x, y, z};
    const int dims[3] = {g.nx, g.ny, g.nz};
    in = true;
    for (int c = 0; c < 3; c++) {
        if (per[c]) {
            q[c] %= dims[c];
            if (q[c] < 0) q[c] += dims[c];
        } else if (q[c] < 0 || q[c] >= dims[c]) {
            in = false;
        }
    }
    if (!in) return false;
    long long id = (long long)q[0] + (long long)g.nx * (q[1] + (long long)g.ny * q[2]);
    return mask[id] & SOLID_BIT;
}

// bond force on bead b from the pair (lo, lo+1); side 0: b = lo+1, side 1: b = lo
template <typename S, typename R, typename PhiT, bool DEV, typename P>
__device__ __forceinline__ bool bond_add(const MdArgs<S, R, PhiT, DEV> &A, const P *Rs, const int *chain, int b,
                                         int side, R F[3])
{
    const int lo = side == 0 ? b - 1 : b;
    if (lo < 0 || lo + 1 >= A.b.nb || chain[lo] != chain[lo + 1]) return true;
    R d[3];
    separation(A.b.g, A.b.per, &Rs[3 * lo], &Rs[3 * (lo + 1)], d);
    R r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    R fac;
    bool ok = true;
    if (A.bond_kind == EKL_BOND_FENE) {
        R x = r2 / (A.bond_r0 * A.bond_r0);
        if (!(x < R(1))) ok = false;
        fac = -A.bond_k / (R(1) - x);
    } else {
        R r = sqrt(r2);
        fac = -A.bond_k * (r - A.bond_l0) / r;
    }
    for (int c = 0; c < 3; c++) {
        if (side == 0) F[c] -= fac * d[c];
        else F[c] += fac * d[c];
    }
    return ok;
}

// Conservative force on bead b, summed serially in the oracle's order: bond
// with b-1, bond with b+1 (Eq. 9c, FENE option), WCA with every other bead in
// index order except bonded neighbours when the bond is harmonic (Eq. 9a),
// WCA against wall nodes in z, y, x order.
template <typename S, typename R, typename PhiT, bool DEV>
__device__ bool bead_force_serial(const MdArgs<S, R, PhiT, DEV> &A, const double *Rs, int b, R F[3],
                                  const int *org, const uint32_t *bits)
{
    const Grid3 &g = A.b.g;
    const int nb = A.b.nb;
    F[0] = F[1] = F[2] = R(0);
    bool ok = bond_add(A, Rs, A.b.chain, b, 0, F);
    ok = bond_add(A, Rs, A.b.chain, b, 1, F) && ok;
    for (int c2 = 0; c2 < nb; c2++) {
        if (c2 == b) continue;
        int lo = c2 < b ? c2 : b, hi = c2 < b ? b : c2;
        if (A.bond_kind == EKL_BOND_HARMONIC && A.b.chain[lo] == A.b.chain[hi] && hi - lo <= 1)
            continue;
        R d[3];
        separation(g, A.b.per, &Rs[3 * lo], &Rs[3 * hi], d);
        R Fp[3] = {R(0), R(0), R(0)};
        wca_add<R>(A.wca_eps, A.wca_sigma, d, Fp);
        for (int c = 0; c < 3; c++) {
            if (c2 < b) F[c] -= Fp[c];
            else F[c] += Fp[c];
        }
    }
    const double rc = 1.122462048309373 * (double)A.wall_sigma;  // 2^(1/6) sigma
    for (int c = 0; c < 3; c++)
        if (!(fabs(Rs[3 * b + c]) < 1e6) || !(rc < 16.0)) return false;  // keeps the scan bounded
    int lo[3], hi[3];
    for (int c = 0; c < 3; c++) {
        lo[c] = (int)floor(Rs[3 * b + c] - rc);
        hi[c] = (int)floor(Rs[3 * b + c] + rc) + 1;
    }
    for (int z = lo[2]; z <= hi[2]; z++)
        for (int y = lo[1]; y <= hi[1]; y++)
            for (int x = lo[0]; x <= hi[0]; x++) {
                bool in;
                if (!wall_solid(g, A.b.per, A.b.mask, x, y, z, org, bits, in)) continue;
                R d[3] = {(R)(Rs[3 * b] - x), (R)(Rs[3 * b + 1] - y), (R)(Rs[3 * b + 2] - z)};
                wca_add<R>(A.wall_eps, A.wall_sigma, d, F);
            }
    return ok;
}

// Same forces with the 32 lanes of a warp sharing the partner and wall loops
// (reduced-precision paths); the result is reduced with a fixed xor tree and
// is valid in every lane.
template <typename S, typename R, typename PhiT, bool DEV>
__device__ bool bead_force_warp(const MdArgs<S, R, PhiT, DEV> &A, const long long *Rq, const float *Rf,
                                const float *Rloc, const int *wlo, const int *wn, const int *chain, int b, R F[3],
                                const int *org, const uint32_t *bits)
{
    const Grid3 &g = A.b.g;
    const int nb = A.b.nb;
    const int lane = threadIdx.x & 31;
    R f[3] = {R(0), R(0), R(0)};
    bool ok = true;
    // the bond with b - 1 in lane 0, with b + 1 in lane 1 (one pass)
    if (lane < 2) ok = bond_add(A, Rq, chain, b, lane, f);
    const float Lf[3] = {(float)g.nx, (float)g.ny, (float)g.nz};
    const float cut2 = 1.2599210498948732f * (float)A.wca_sigma * (float)A.wca_sigma;
    for (int c2 = lane; c2 < nb; c2 += 32) {
        if (c2 == b) continue;
        int lo = c2 < b ? c2 : b, hi = c2 < b ? b : c2;
        if (A.bond_kind == EKL_BOND_HARMONIC && chain[lo] == chain[hi] && hi - lo <= 1) continue;
        // float screen, FP64 separation only for pairs near the cut-off
        float q2 = 0.f;
        for (int c = 0; c < 3; c++) {
            float v = Rf[3 * b + c] - Rf[3 * c2 + c];
            if (A.b.per[c]) {
                if (v > 0.5f * Lf[c]) v -= Lf[c];
                else if (v < -0.5f * Lf[c]) v += Lf[c];
            }
            q2 += v * v;
        }
        if (q2 > 1.1f * cut2 + 0.01f) continue;
        R d[3];
        separation(g, A.b.per, &Rq[3 * lo], &Rq[3 * hi], d);
        R Fp[3] = {R(0), R(0), R(0)};
        wca_add<R>(A.wca_eps, A.wca_sigma, d, Fp);
        for (int c = 0; c < 3; c++) {
            if (c2 < b) f[c] -= Fp[c];
            else f[c] += Fp[c];
        }
    }
    // wall nodes in the scan box; coordinates relative to the cached box origin
    const int n0 = wn[3 * b], n1 = wn[3 * b + 1], n2 = wn[3 * b + 2];
    const int cells = n0 * n1 * n2;
    const float i0 = 1.f / (float)n0, i1 = 1.f / (float)n1;
    for (int t = lane; t < cells; t += 32) {
        const int r = tdiv(t, i0), zz = tdiv(r, i1);
        const int x = wlo[3 * b] + t - r * n0, y = wlo[3 * b + 1] + r - zz * n1, z = wlo[3 * b + 2] + zz;
        bool in;
        if (!wall_solid(g, A.b.per, A.b.mask, x, y, z, org, bits, in)) continue;
        R d[3] = {(R)(Rloc[3 * b] - (float)(x - org[0])), (R)(Rloc[3 * b + 1] - (float)(y - org[1])),
                  (R)(Rloc[3 * b + 2] - (float)(z - org[2]))};
        wca_add<R>(A.wall_eps, A.wall_sigma, d, f);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        for (int c = 0; c < 3; c++) f[c] += __shfl_xor_sync(0xffffffffu, f[c], o);
    for (int c = 0; c < 3; c++) F[c] = f[c];
    return __all_sync(0xffffffffu, ok);
}

// Per-bead wall scan box [floor(R - rc), floor(R + rc) + 1] and coordinates
// local to the cached block (one thread per coordinate, FP64 once per sub-step)
__device__ __forceinline__ void scan_bounds(double r, double rc, int org, int &lo, int &n, float &loc,
                                            int &bad)
{
    if (!(fabs(r) < 1e6) || !(rc < 16.0)) {
        bad = 1;
        lo = 0;
        n = 0;
        loc = 0.f;
        return;
    }
    lo = (int)floor(r - rc);
    n = (int)floor(r + rc) + 2 - lo;
    loc = (float)(r - (double)org);
}
// the same from a fixed-point position rq and cut-off rcq (40 fractional bits)
__device__ __forceinline__ void scan_bounds_q(long long rq, long long rcq, int org, int &lo, int &n, float &loc,
                                              int &bad)
{
    if (!(rq < (1ll << 60) && rq > -(1ll << 60)) || !(rcq < (16ll << 40))) {
        bad = 1;
        lo = 0;
        n = 0;
        loc = 0.f;
        return;
    }
    lo = (int)((rq - rcq) >> 40);
    n = (int)((rq + rcq) >> 40) + 2 - lo;
    loc = ll_to_float(rq - ((long long)org << 40)) * (float)PHI_INV;
}

// One block: moments and field at the patch nodes, interpolation to beads,
// md_substeps Langevin sub-steps with implicit friction, spreading of the
// sub-step-averaged drag g^a_i = -gamma^a (u^a(R_i) - V_i) as a force per
// particle on the patch nodes.  Readings as in the oracle: gamma^a = xi n^a/n
// (or xi), fluid/field held at R(t) over the sub-steps, R(t) weights both ways.
// FP64 instantiation: one thread per bead, serial sums in the oracle's order.
// Reduced-precision instantiations: one warp per bead.
template <typename R> inline size_t md_smem_bytes(int nb)
{
    return (size_t)nb * (3 * sizeof(double) + 27 * sizeof(R) + 6 * sizeof(float) + 10 * sizeof(int) +
                         WALL_WORDS * sizeof(uint32_t));
}

template <typename R> struct MdThreads {
    static constexpr int value = sizeof(R) == 8 ? BEAD_THREADS : 1024;
};

template <typename S, typename R, typename PhiT, bool DEV>
__device__ void bead_md_body(const MdArgs<S, R, PhiT, DEV> &A)
{
    constexpr bool SERIAL = sizeof(R) == 8;
    const StepArgs<S, R, PhiT> &a = A.s;
    const BeadArgs<R> &B = A.b;
    const Grid3 g = a.g;
    const int nb = B.nb;
    const int pc = *B.patch_count;
    // dynamic shared memory, sized for nb beads (md_smem_bytes)
    extern __shared__ __align__(16) unsigned char md_smem[];
    double *Rs = (double *)md_smem;              // positions, FP64 path
    long long *Rq = (long long *)md_smem;        // positions, fixed point (other paths)
    R *sV = (R *)(Rs + 3 * nb);
    R *sU = sV + 3 * nb;
    R *sG = sU + 9 * nb;
    R *sGam = sG + 3 * nb;
    R *sAcc = sGam + 3 * nb;
    float *Rf = (float *)(sAcc + 9 * nb);
    float *Rloc = Rf + 3 * nb;
    int *worg = (int *)(Rloc + 3 * nb);
    int *wlo = worg + 3 * nb;
    int *wn = wlo + 3 * nb;
    int *sChain = wn + 3 * nb;  // chain ids (read every sub-step)
    uint32_t *wbits = (uint32_t *)(sChain + nb);
    __shared__ int sBad;
    if (threadIdx.x == 0) sBad = 0;
    // moments at the patch nodes: thread (k, s) takes species s of node k,
    // thread (k, 3) the potential gradient (one memory round trip each)
    for (int t = threadIdx.x; t < 4 * pc; t += blockDim.x) {
        const int k = t >> 2, s = t & 3;
        long long i = B.patch_node[k];
        uint32_t m = a.mask[i];
        int x, y, z;
        coords_of(g, i, x, y, z);
        Nbr nbr = make_nbr(g, x, y, z);
        R *out = B.patch_mom + (long long)k * 15;
        if (s < NS) {
            R v[Q];
            pull19<S, R>(a.fin, g.N, s, i, m, nbr, v);
            R n = R(0), jx = R(0), jy = R(0), jz = R(0);
#pragma unroll
            for (int p = 0; p < Q; p++) {
                n += v[p];
                if (cx_(p) == 1) jx += v[p];
                if (cx_(p) == -1) jx -= v[p];
                if (cy_(p) == 1) jy += v[p];
                if (cy_(p) == -1) jy -= v[p];
                if (cz_(p) == 1) jz += v[p];
                if (cz_(p) == -1) jz -= v[p];
            }
            if (DEV) n = a.n_ref[s] + n;
            out[s] = n;
            out[3 + 3 * s + 0] = jx / n;
            out[3 + 3 * s + 1] = jy / n;
            out[3 + 3 * s + 2] = jz / n;
        } else {
            R gr[3];
            int olo[3], ohi[3];
            closed_faces(g, a.per, x, y, z, olo, ohi);
            node_gradient<R, PhiT>(a.phi, a.wall_share, a.c4, i, m, nbr, olo, ohi, gr);
            out[12] = gr[0];
            out[13] = gr[1];
            out[14] = gr[2];
        }
    }
    for (int t = threadIdx.x; t < 3 * nb; t += blockDim.x) {
        const double r = B.Rb[t];
        if constexpr (SERIAL) Rs[t] = r;
        else Rq[t] = __double2ll_rn(r * PHI_SCALE);
        Rf[t] = (float)r;
        sV[t] = B.Vb[t];
    }
    for (int t = threadIdx.x; t < nb; t += blockDim.x) sChain[t] = B.chain[t];
    for (int t = threadIdx.x; t < 9 * nb; t += blockDim.x) sAcc[t] = R(0);
    const double rcw = 1.122462048309373 * (double)A.wall_sigma;  // 2^(1/6) sigma
    const long long rcq = rcw < 16.0 ? __double2ll_rn(rcw * PHI_SCALE) : (16ll << 40);
    int bad0 = 0;  // raised into sBad after the barrier that orders its reset
    for (int t = threadIdx.x; t < 3 * nb; t += blockDim.x) {
        const double r = B.Rb[t];
        worg[t] = fabs(r) < 1e6 ? (int)floor(r) - WALL_BOX / 2 + 1 : 0;
        int bad = 0;
        scan_bounds(r, rcw, worg[t], wlo[t], wn[t], Rloc[t], bad);
        bad0 |= bad;
    }
    __syncthreads();
    if (bad0) sBad = 1;
    {
        // one word (32 cells of one bead's block) per warp and round, built by
        // a ballot; WALL_ROUNDS rounds' link words are loaded before any is used
        constexpr int WALL_ROUNDS = 8;
        const int dims[3] = {g.nx, g.ny, g.nz};
        const int cells = WALL_BOX * WALL_BOX * WALL_BOX;
        const int words = nb * WALL_WORDS;
        const int wid = threadIdx.x >> 5, ln = threadIdx.x & 31, nw = blockDim.x >> 5;
        for (int w0 = wid; w0 < words; w0 += WALL_ROUNDS * nw) {
            bool solid[WALL_ROUNDS];
#pragma unroll
            for (int u = 0; u < WALL_ROUNDS; u++) {
                const int w = w0 + u * nw;
                solid[u] = false;
                const int bb = w / WALL_WORDS, cell = (w - bb * WALL_WORDS) * 32 + ln;
                if (w >= words || cell >= cells) continue;
                const int ox = cell % WALL_BOX, oy = (cell / WALL_BOX) % WALL_BOX, oz = cell / (WALL_BOX * WALL_BOX);
                int q[3] = {worg[3 * bb] + ox, worg[3 * bb + 1] + oy, worg[3 * bb + 2] + oz};
                bool in = true;
                for (int c = 0; c < 3; c++) {
                    if (B.per[c]) {
                        // the block reaches at most WALL_BOX nodes beyond the box
                        if (q[c] >= dims[c]) q[c] -= dims[c];
                        else if (q[c] < 0) q[c] += dims[c];
                        if (q[c] < 0 || q[c] >= dims[c]) {
                            q[c] %= dims[c];
                            if (q[c] < 0) q[c] += dims[c];
                        }
                    } else if (q[c] < 0 || q[c] >= dims[c]) {
                        in = false;
                    }
                }
                if (in) solid[u] = a.mask[(long long)q[0] + (long long)g.nx * (q[1] + (long long)g.ny * q[2])] & SOLID_BIT;
            }
#pragma unroll
            for (int u = 0; u < WALL_ROUNDS; u++) {
                const int w = w0 + u * nw;  // warp-uniform
                const unsigned word = __ballot_sync(0xffffffffu, solid[u]);
                if (ln == 0 && w < words) wbits[w] = word;
            }
        }
    }
    // interpolation.  FP64: one thread per bead, entries in slot order k (the
    // oracle's order).  Reduced precision: eight lanes per bead, one entry
    // each (all loads in flight at once), summed over the lanes by shuffles.
    auto interp_out = [&](int b, const R *v) {  // v: n^a (3), u^a (9), grad phi (3)
        const R ntot = v[0] + v[1] + v[2];
        for (int s = 0; s < NS; s++) {
            sGam[3 * b + s] = (a.flags & EKL_GAMMA_LITERAL) ? A.xi : A.xi * v[s] / ntot;
            for (int c = 0; c < 3; c++) sU[9 * b + 3 * s + c] = v[3 + 3 * s + c];
        }
        const R qb = B.qb[b];
        for (int c = 0; c < 3; c++) {
            sG[3 * b + c] = v[12 + c];
            if (fabs(qb * v[12 + c]) >= R(1)) atomicOr(a.status, ST_CFL);
        }
    };
    if constexpr (SERIAL) {
        for (int b = threadIdx.x; b < nb; b += blockDim.x) {
            R v[15];
            for (int j = 0; j < 15; j++) v[j] = R(0);
            for (int k = 0; k < 8; k++) {
                R w = B.entry_w[b * 8 + k];
                if (w == R(0)) continue;
                int slot = B.entry_slot[b * 8 + k];
                const R *mo = B.patch_mom + (long long)slot * 15;
                for (int j = 0; j < 15; j++) v[j] += w * mo[j];
            }
            interp_out(b, v);
        }
    } else {
        const int total = (8 * nb + 31) & ~31;  // whole warps: the shuffles below are warp-wide
        for (int t = threadIdx.x; t < total; t += blockDim.x) {
            const int b = t >> 3, k = t & 7;
            R v[15];
#pragma unroll
            for (int j = 0; j < 15; j++) v[j] = R(0);
            if (b < nb) {
                const R w = B.entry_w[b * 8 + k];
                if (w != R(0)) {
                    const R *mo = B.patch_mom + (long long)B.entry_slot[b * 8 + k] * 15;
#pragma unroll
                    for (int j = 0; j < 15; j++) v[j] = w * mo[j];
                }
            }
#pragma unroll
            for (int j = 0; j < 15; j++)
#pragma unroll
                for (int o = 1; o < 8; o <<= 1) v[j] += __shfl_xor_sync(0xffffffffu, v[j], o);
            if (k == 0 && b < nb) interp_out(b, v);
        }
    }
    __syncthreads();
    const int nsub = A.md_substeps;
    const R dt = R(1) / (R)nsub;
    const bool noise = A.bead_kT > R(0) && !(a.flags & EKL_NO_BEAD_NOISE);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
    // Reduced-precision instantiations: with one bead per warp and at most
    // 32 sub-steps, lane s draws the sub-step-s noise of its warp's bead up
    // front (the draws are independent of the dynamics)
    const bool pre = !SERIAL && noise && nb <= nwarps && nsub <= 32;
    float xpre[3] = {0.f, 0.f, 0.f};
    if (pre && warp < nb && lane < nsub) {
        uint32_t ctr[4] = {(uint32_t)warp, (uint32_t)lane | (1u << 24), (uint32_t)A.step,
                           (uint32_t)((uint64_t)A.step >> 32)};
        philox4x32_10(ctr, A.key0, A.key1);
        for (int c = 0; c < 3; c++) xpre[c] = unit_variate_f32(ctr[c]);
    }
    for (int sub = 0; sub < nsub; sub++) {
        // force from the positions at the start of the sub-step, then the
        // bead's own velocity and drag update (positions move after the barrier)
        const int first = SERIAL ? (int)threadIdx.x : warp;
        const int stride = SERIAL ? (int)blockDim.x : nwarps;
        for (int b = first; b < nb; b += stride) {
            R F[3];
            bool okf;
            if constexpr (SERIAL) okf = bead_force_serial(A, Rs, b, F, &worg[3 * b], &wbits[b * WALL_WORDS]);
            else okf = bead_force_warp(A, Rq, Rf, Rloc, wlo, wn, sChain, b, F, &worg[3 * b], &wbits[b * WALL_WORDS]);
            if (!okf) sBad = 1;
            R xi_[3] = {R(0), R(0), R(0)};
            if (noise) {
                if (pre) {
                    for (int c = 0; c < 3; c++) xi_[c] = __shfl_sync(0xffffffffu, xpre[c], sub);
                } else {
                    uint32_t ctr[4] = {(uint32_t)b, (uint32_t)sub | (1u << 24), (uint32_t)A.step,
                                       (uint32_t)((uint64_t)A.step >> 32)};
                    philox4x32_10(ctr, A.key0, A.key1);
                    for (int c = 0; c < 3; c++) {
                        if constexpr (SERIAL) xi_[c] = unit_variate<R>(ctr[c]);
                        else xi_[c] = unit_variate_f32(ctr[c]);
                    }
                }
            }
            // the serial instantiation updates the three components in turn;
            // the warp instantiation updates component `lane` in lanes 0-2
            const int c0 = SERIAL ? 0 : lane, c1 = SERIAL ? 3 : lane + 1;
            if (c0 >= 3) continue;
            const R *gam = &sGam[3 * b];
            R gtot = gam[0] + gam[1] + gam[2];
            R amp = noise ? sqrt(R(2) * gtot * A.bead_kT / dt) : R(0);
            R qb = B.qb[b];
            for (int c = c0; c < c1; c++) {
                const R Fc = c == 0 ? F[0] : c == 1 ? F[1] : F[2];
                const R xc = c == 0 ? xi_[0] : c == 1 ? xi_[1] : xi_[2];
                R Fe = -qb * Consts<R>::KT * sG[3 * b + c] + qb * Consts<R>::KT * a.E[c];
                R num = A.mass * sV[3 * b + c] / dt;
                for (int s2 = 0; s2 < NS; s2++) num += gam[s2] * sU[9 * b + 3 * s2 + c];
                num += Fc + Fe + amp * xc;
                R Vn = num / (A.mass / dt + gtot);
                for (int s2 = 0; s2 < NS; s2++)
                    sAcc[9 * b + 3 * s2 + c] += dt * (-gam[s2] * (sU[9 * b + 3 * s2 + c] - Vn));
                sV[3 * b + c] = Vn;
            }
        }
        __syncthreads();
        // positions, wrapped into [0, L) on periodic axes
        for (int t = threadIdx.x; t < 3 * nb; t += blockDim.x) {
            const int c = t % 3;
            const int Li = c == 0 ? g.nx : (c == 1 ? g.ny : g.nz);
            int bad = 0;
            if constexpr (SERIAL) {
                const double L = Li;
                double r = Rs[t] + (double)(dt * sV[t]);
                if (B.per[c]) {
                    if (r < 0.0) r += L;
                    else if (r >= L) r -= L;
                }
                Rs[t] = r;
                Rf[t] = (float)r;
                scan_bounds(r, rcw, worg[t], wlo[t], wn[t], Rloc[t], bad);
            } else {
                const long long L = (long long)Li << 40;
                long long r = Rq[t] + float_to_ll((float)(dt * sV[t]) * (float)PHI_SCALE);
                if (B.per[c]) {
                    if (r < 0) r += L;
                    else if (r >= L) r -= L;
                }
                Rq[t] = r;
                Rf[t] = ll_to_float(r) * (float)PHI_INV;
                scan_bounds_q(r, rcq, worg[t], wlo[t], wn[t], Rloc[t], bad);
            }
            if (bad) sBad = 1;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0 && sBad) atomicOr(a.status, ST_BEAD);
    for (int t = threadIdx.x; t < 3 * nb; t += blockDim.x) {
        if constexpr (SERIAL) B.Rb[t] = Rs[t];
        else B.Rb[t] = __ll2double_rn(Rq[t]) * PHI_INV;
        B.Vb[t] = sV[t];
    }
    // spread: per slot, entries in bead order (ascending b), then per particle
    for (int k = threadIdx.x; k < pc; k += blockDim.x) {
        R acc[9];
        for (int t = 0; t < 9; t++) acc[t] = R(0);
        const int t0 = B.slot_first[k], t1 = B.slot_first[k + 1];
        // entries in rounds of eight: their ids, then their weights, loaded
        // before any is summed (in the same order as one at a time)
        for (int tb = t0; tb < t1; tb += 8) {
            int e[8];
            R w[8];
#pragma unroll
            for (int j = 0; j < 8; j++) e[j] = tb + j < t1 ? B.sorted_entry[tb + j] : -1;
#pragma unroll
            for (int j = 0; j < 8; j++) w[j] = e[j] >= 0 ? B.entry_w[e[j]] : R(0);
#pragma unroll
            for (int j = 0; j < 8; j++) {
                if (w[j] == R(0)) continue;
                const int bb = e[j] >> 3;
                for (int u = 0; u < 9; u++) acc[u] += sAcc[bb * 9 + u] * w[j];
            }
        }
        const R *mo = B.patch_mom + (long long)k * 15;
        for (int s = 0; s < NS; s++)
            for (int c = 0; c < 3; c++) {
                R v = acc[3 * s + c];
                B.patch_f[(long long)k * 9 + 3 * s + c] = v != R(0) ? v / mo[s] : R(0);
            }
    }
}

template <typename S, typename R, typename PhiT, bool DEV>
__global__ void __launch_bounds__(MdThreads<R>::value) bead_md_kernel(MdArgs<S, R, PhiT, DEV> A)
{
    bead_md_body<S, R, PhiT, DEV>(A);
}

template <typename S, typename R, typename PhiT, bool DEV>
__global__ void __launch_bounds__(MdThreads<R>::value)
    bead_md_batch_kernel(const MdArgs<S, R, PhiT, DEV> *reps, long long step)
{
    MdArgs<S, R, PhiT, DEV> A = reps[blockIdx.y];
    if (A.b.nb == 0) return;
    A.step = step;
    bead_md_body<S, R, PhiT, DEV>(A);
}

// ============================================================== fused LB
// Per fluid node: pull the 3 x 19 populations (halfway bounce-back on set
// link bits), moments (Eqs. 15-16), force per particle (Eq. 5: external,
// field -z k_B T grad phi + z k_B T E, bead drag, and the friction of Eq. 6
// evaluated at the half-force velocities by the closed form below), BGK
// relaxation to f_eq(n, u^a*) (Eq. 10) plus (1 - omega/2) S (Eq. 13), store.
//   a^a = j^a/n^a + G^a/2, h^a = omega_d^a/2,
//   u* = sum n a/(1+h) / sum n/(1+h), u^a* = (a^a + h^a u*)/(1+h^a),
//   Phi^a = G^a - omega_d^a (u^a* - u*).
template <typename S, typename R, typename PhiT, bool DEV, bool FLUCT>
__device__ __forceinline__ void lb_body(const StepArgs<S, R, PhiT> &a, long long blk, long long step)
{
    const Grid3 g = a.g;
    const long long i = blk * (long long)blockDim.x + threadIdx.x;
    int bad = 0, cfl = 0;
    if (i < g.N) {
        const uint32_t m = a.mask[i];
        if (!(m & SOLID_BIT)) {
            int x, y, z;
            coords_of(g, i, x, y, z);
            const Nbr nb = make_nbr(g, x, y, z);
            R f[NS][Q];
#pragma unroll
            for (int s = 0; s < NS; s++) pull19<S, R>(a.fin, g.N, s, i, m, nb, f[s]);
            R gphi[3];
            int olo[3], ohi[3];
            closed_faces(g, a.per, x, y, z, olo, ohi);
            node_gradient<R, PhiT>(a.phi, a.wall_share, a.c4, i, m, nb, olo, ohi, gphi);
            for (int c = 0; c < 3; c++)
                if (fabs(gphi[c]) >= R(1)) cfl = 1;
            int slot = -1;
            if ((__ldg(a.patch_bits + (i >> 5)) >> (i & 31)) & 1u) {
                const int pc = *a.patch_count;
                int k = lower_bound_i(a.patch_node, pc, i);
                if (k < pc && a.patch_node[k] == i) slot = k;
            }
            R n[NS], dn[NS], av[NS][3], G[NS][3], h[NS], ih[NS];
#pragma unroll
            for (int s = 0; s < NS; s++) {
                R nn = R(0), jx = R(0), jy = R(0), jz = R(0);
#pragma unroll
                for (int p = 0; p < Q; p++) {
                    R v = f[s][p];
                    nn += v;
                    if (cx_(p) == 1) jx += v;
                    if (cx_(p) == -1) jx -= v;
                    if (cy_(p) == 1) jy += v;
                    if (cy_(p) == -1) jy -= v;
                    if (cz_(p) == 1) jz += v;
                    if (cz_(p) == -1) jz -= v;
                }
                dn[s] = nn;
                n[s] = DEV ? a.n_ref[s] + nn : nn;
                if (!(n[s] > R(0)) || !isfinite(n[s])) bad = 1;
                h[s] = R(0.5) * a.wd[s];
                ih[s] = R(1) / (R(1) + h[s]);
                // reduced-precision paths multiply by reciprocals; the FP64
                // path divides exactly as the oracle does
                const R in_ = DEV ? R(1) / n[s] : R(0);
                R j[3] = {jx, jy, jz};
                for (int c = 0; c < 3; c++) {
                    R zk = a.zv[s] * Consts<R>::KT;
                    R Gc = a.body[s][c] - zk * gphi[c] + zk * a.E[c];
                    if (slot >= 0) Gc = Gc + a.patch_f[(long long)slot * 9 + 3 * s + c];
                    G[s][c] = Gc;
                    av[s][c] = (DEV ? j[c] * in_ : j[c] / n[s]) + R(0.5) * Gc;
                }
            }
            R num[3] = {R(0), R(0), R(0)}, den = R(0), us[3];
#pragma unroll
            for (int s = 0; s < NS; s++) {
                if constexpr (DEV) {
                    den += n[s] * ih[s];
                    for (int c = 0; c < 3; c++) num[c] += n[s] * av[s][c] * ih[s];
                } else {
                    den += n[s] / (R(1) + h[s]);
                    for (int c = 0; c < 3; c++) num[c] += n[s] * av[s][c] / (R(1) + h[s]);
                }
            }
            if constexpr (DEV) {
                const R iden = R(1) / den;
                for (int c = 0; c < 3; c++) us[c] = num[c] * iden;
            } else {
                for (int c = 0; c < 3; c++) us[c] = num[c] / den;
            }
#pragma unroll
            for (int s = 0; s < NS; s++) {
                R ue[3], Ph[3];
                for (int c = 0; c < 3; c++) {
                    R ua = DEV ? (av[s][c] + h[s] * us[c]) * ih[s] : (av[s][c] + h[s] * us[c]) / (R(1) + h[s]);
                    Ph[c] = G[s][c] - a.wd[s] * (ua - us[c]);
                    ue[c] = (a.flags & EKL_EQ_BARYCENTRIC) ? us[c] : ua;
                }
                const R om = a.om[s];
                const R u2 = ue[0] * ue[0] + ue[1] * ue[1] + ue[2] * ue[2];
                const R Fu = Ph[0] * ue[0] + Ph[1] * ue[1] + Ph[2] * ue[2];
                const R cS = R(1) - R(0.5) * om;
                S *out = a.fout + (long long)(s * Q) * g.N + i;
                // fluctuating term (Eq. 14): 15 zero-mean unit-variance N_k
                // from Philox (counter: node, 2^25 | species << 4 | call, step)
                R Nk[FLUCT ? 16 : 1];
                R amp = R(0);
                if constexpr (FLUCT) {
#pragma unroll
                    for (int call = 0; call < 4; call++) {
                        uint32_t ctr[4] = {(uint32_t)i, (2u << 24) | ((uint32_t)s << 4) | (uint32_t)call,
                                           (uint32_t)step, (uint32_t)((uint64_t)step >> 32)};
                        philox4x32_10(ctr, a.key0, a.key1);
#pragma unroll
                        for (int j = 0; j < 4; j++) {
                            if constexpr (sizeof(R) == 8) Nk[4 * call + j] = unit_variate<R>(ctr[j]);
                            else Nk[4 * call + j] = unit_variate_f32(ctr[j]);
                        }
                    }
                    amp = sqrt(a.fluct_m * n[s] * om * (R(2) - om));
                }
                // v plus the noise of population p (v itself without the term)
                auto noisy = [&](R v, int p) -> R {
                    if constexpr (!FLUCT) return v;
                    else {
                        R d = R(0);
#pragma unroll
                        for (int k = 4; k < Q; k++) d += __ldg(a.wchi + k * Q + p) * Nk[k - 4];
                        return v + amp * d;
                    }
                };
                if constexpr (!DEV) {
#pragma unroll
                    for (int p = 0; p < Q; p++) {
                        const R cu = (R)cx_(p) * ue[0] + (R)cy_(p) * ue[1] + (R)cz_(p) * ue[2];
                        const R cF = (R)cx_(p) * Ph[0] + (R)cy_(p) * Ph[1] + (R)cz_(p) * Ph[2];
                        const R w = (R)w_(p);
                        const R VT2 = Consts<R>::VT2;
                        R feq = w * n[s] * (R(1) + cu / VT2 + (cu * cu - VT2 * u2) / (R(2) * VT2 * VT2));
                        R Sp = w * n[s] * (cF / VT2 + (cu * cF - VT2 * Fu) / (VT2 * VT2));
                        R fs = f[s][p] - om * (f[s][p] - feq) + cS * Sp;
                        Store<S>::st(out + (long long)p * g.N, noisy(fs, p));
                    }
                } else {
                    // deviation form, s_eq = f_eq - w n_ref:
                    //   out = (1 - om) f + om s_eq + cS S
                    //   s_eq = w (dn + n (3 cu + 4.5 cu^2 - 1.5 u^2)), S = w n (3 cF + 9 cu cF - 3 F.u)
                    // a velocity and its opposite share the parts even in c
                    const R keep = R(1) - om;
                    const R w0 = (R)w_(0);
                    Store<S>::st(out, noisy(keep * f[s][0] + w0 * (om * (dn[s] - R(1.5) * n[s] * u2) - cS * R(3) * n[s] * Fu), 0));
#pragma unroll
                    for (int p = 1; p < Q; p += 2) {
                        const int q = p + 1;  // opposite of p
                        const R cu = (R)cx_(p) * ue[0] + (R)cy_(p) * ue[1] + (R)cz_(p) * ue[2];
                        const R cF = (R)cx_(p) * Ph[0] + (R)cy_(p) * Ph[1] + (R)cz_(p) * Ph[2];
                        const R w = (R)w_(p);
                        const R wn = w * n[s];
                        const R even = om * (R(4.5) * cu * cu - R(1.5) * u2) + cS * (R(9) * cu * cF - R(3) * Fu);
                        const R odd = R(3) * (om * cu + cS * cF);
                        const R base = om * w * dn[s];
                        Store<S>::st(out + (long long)p * g.N, noisy(keep * f[s][p] + (base + wn * (even + odd)), p));
                        Store<S>::st(out + (long long)q * g.N, noisy(keep * f[s][q] + (base + wn * (even - odd)), q));
                    }
                }
            }
        }
    }
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(a.status, ST_UNSTABLE);
    if (__any_sync(0xffffffffu, cfl) && (threadIdx.x & 31) == 0) atomicOr(a.status, ST_CFL);
}

template <typename S, typename R, typename PhiT, bool DEV, bool FLUCT>
__global__ void __launch_bounds__(LB_THREADS, sizeof(R) == 4 ? 4 : 1) lb_fused_kernel(StepArgs<S, R, PhiT> a)
{
    lb_body<S, R, PhiT, DEV, FLUCT>(a, blockIdx.x, a.step);
}

template <typename S, typename R, typename PhiT, bool DEV, bool FLUCT>
__global__ void __launch_bounds__(LB_THREADS, sizeof(R) == 4 ? 4 : 1)
    lb_fused_batch_kernel(const StepArgs<S, R, PhiT> *reps, long long step)
{
    const StepArgs<S, R, PhiT> &a = reps[blockIdx.y];
    if ((long long)blockIdx.x * blockDim.x >= a.g.N) return;
    lb_body<S, R, PhiT, DEV, FLUCT>(a, blockIdx.x, step);
}

// ============================================================== outputs
template <typename S, typename R, typename PhiT, bool DEV>
__global__ void fields_kernel(StepArgs<S, R, PhiT> a, double *n_out, double *j_out, double *phi_out)
{
    const Grid3 g = a.g;
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= g.N) return;
    uint32_t m = a.mask[i];
    bool solid = m & SOLID_BIT;
    int x, y, z;
    coords_of(g, i, x, y, z);
    Nbr nb = make_nbr(g, x, y, z);
    for (int s = 0; s < NS; s++) {
        double n = 0, jx = 0, jy = 0, jz = 0;
        if (!solid) {
            R v[Q];
            pull19<S, R>(a.fin, g.N, s, i, m, nb, v);
            R nn = R(0), ax = R(0), ay = R(0), az = R(0);
#pragma unroll
            for (int p = 0; p < Q; p++) {
                nn += v[p];
                if (cx_(p) == 1) ax += v[p];
                if (cx_(p) == -1) ax -= v[p];
                if (cy_(p) == 1) ay += v[p];
                if (cy_(p) == -1) ay -= v[p];
                if (cz_(p) == 1) az += v[p];
                if (cz_(p) == -1) az -= v[p];
            }
            n = DEV ? (double)a.n_ref[s] + (double)nn : (double)nn;
            jx = ax; jy = ay; jz = az;
        }
        if (n_out) n_out[(long long)s * g.N + i] = n;
        if (j_out) {
            j_out[((long long)s * 3 + 0) * g.N + i] = jx;
            j_out[((long long)s * 3 + 1) * g.N + i] = jy;
            j_out[((long long)s * 3 + 2) * g.N + i] = jz;
        }
    }
    if (phi_out) {
        double v;
        if constexpr (((PhiT)0.5) != 0) v = (double)a.phi[i];
        else v = (double)a.phi[i] * PHI_INV;
        phi_out[i] = solid ? 0.0 : v;
    }
}

// Species fluxes through the lattice plane {coordinate `axis` == plane}:
// per fluid node of the plane the bare current component sum_p c_p,axis f_p
// of the streamed populations (Eq. 16), summed in FP64; one partial per
// block and species.
template <typename S, typename R, typename PhiT, bool DEV>
__global__ void current_kernel(StepArgs<S, R, PhiT> a, int axis, int plane, double *part)
{
    __shared__ double sh[256 / 32];
    const Grid3 g = a.g;
    const int n1 = axis == 0 ? g.ny : g.nx, n2 = axis == 2 ? g.ny : g.nz;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    double acc[NS] = {0.0, 0.0, 0.0};
    if (t < n1 * n2) {
        const int u = t % n1, v = t / n1;
        int x, y, z;
        if (axis == 0) { x = plane; y = u; z = v; }
        else if (axis == 1) { x = u; y = plane; z = v; }
        else { x = u; y = v; z = plane; }
        const long long i = x + (long long)g.nx * (y + (long long)g.ny * z);
        const uint32_t m = a.mask[i];
        if (!(m & SOLID_BIT)) {
            const Nbr nb = make_nbr(g, x, y, z);
            for (int s = 0; s < NS; s++) {
                R v19[Q];
                pull19<S, R>(a.fin, g.N, s, i, m, nb, v19);
                double j = 0.0;
#pragma unroll
                for (int p = 0; p < Q; p++) {
                    const int c = axis == 0 ? cx_(p) : (axis == 1 ? cy_(p) : cz_(p));
                    if (c == 1) j += (double)v19[p];
                    if (c == -1) j -= (double)v19[p];
                }
                acc[s] = j;
            }
        }
    }
    for (int s = 0; s < NS; s++) {
        const double b = block_sum(acc[s], sh);
        if (threadIdx.x == 0) part[(size_t)blockIdx.x * NS + s] = b;
    }
}

// Per-species mass of the post-collision populations (the collision keeps
// each node's density, so this is the total of the last step's densities),
// one FP64 partial per block; computed only when statistics are requested.
template <typename S, typename R, typename PhiT, bool DEV>
__global__ void mass_kernel(StepArgs<S, R, PhiT> a)
{
    __shared__ double sh[256 / 32];
    const Grid3 g = a.g;
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    double v[NS] = {0.0, 0.0, 0.0};
    if (i < g.N && !(a.mask[i] & SOLID_BIT))
        for (int s = 0; s < NS; s++) {
            double t = 0.0;
            for (int p = 0; p < Q; p++) t += (double)Store<S>::ld(a.fin + (long long)(s * Q + p) * g.N + i);
            v[s] = DEV ? t + (double)a.n_ref[s] : t;
        }
    for (int s = 0; s < NS; s++) {
        const double b = block_sum(v[s], sh);
        if (threadIdx.x == 0) a.part_mass[(size_t)blockIdx.x * NS + s] = b;
    }
}

template <typename S, typename R, typename PhiT, bool DEV>
__global__ void state_kernel(StepArgs<S, R, PhiT> a, double *f_io, double *phi_io, int to_host)
{
    const Grid3 g = a.g;
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= g.N) return;
    bool solid = a.mask[i] & SOLID_BIT;
    for (int s = 0; s < NS; s++)
        for (int p = 0; p < Q; p++) {
            long long k = (long long)(s * Q + p) * g.N + i;
            double off = DEV ? w_(p) * (double)a.n_ref[s] : 0.0;
            if (to_host) {
                f_io[k] = solid ? 0.0 : (double)Store<S>::ld((const S *)a.fin + k) + off;
            } else {
                Store<S>::st((S *)a.fin + k, (R)(solid ? 0.0 : f_io[k] - off));
            }
        }
    if (phi_io) {
        if (to_host) {
            if constexpr (((PhiT)0.5) != 0) phi_io[i] = (double)a.phi[i];
            else phi_io[i] = (double)a.phi[i] * PHI_INV;
        } else {
            if constexpr (((PhiT)0.5) != 0) a.phi[i] = (PhiT)phi_io[i];
            else a.phi[i] = __double2ll_rn(phi_io[i] * PHI_SCALE);
        }
    }
}

}  // namespace ekl
