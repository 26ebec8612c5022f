// The multigrid-preconditioned CG solve of ekl_mg.cuh in split form: every
// lattice-level pass is its own launch (level 1 too when it is grid-wide),
// the remaining coarse levels of each V-cycle are one cooperative launch, and
// the CG loop runs on the device as a CUDA graph with a conditional WHILE
// node, so a step's solve needs no host round trip.
//
// Why split: inside the single cooperative launch every pass shares the
// register budget of the whole solve (64 a thread at 1024 threads), and a
// lattice pass cannot keep the loads of several nodes in flight; on its own
// launch it can (MGS_U node pairs per thread and trip), and a lattice pass is
// bound by memory latency at one pair.  On small lattices a graph node also
// costs less than a grid barrier.
//
// The passes, their thread-to-node maps and the block partials of every
// reduction are those of the single-launch solve with the same grid (nblk
// blocks of the single launch's block size: 1024 threads on lattices of at
// least MG_WIDE_NODES_PER_SM nodes per SM, else 512), and the partials are
// summed the same way, so both forms return the same potential bit for bit.  The scalar recurrences
// (beta, alpha, the convergence test, the restart from the true residual)
// live in MgCtl in device memory: the lattice kernels read it, one-block
// control kernels write it and set the loop's condition.
#pragma once
#include "ekl_mg.cuh"

namespace ekl {

constexpr int MGS_THREADS = 1024;  // the largest block size of the split kernels
constexpr int MGS_U = 4;   // node pairs per thread and trip in the lattice half sweeps
constexpr int MGS_PQU = 1; // p/q pass node pairs per thread and trip
constexpr int MGS_CU = 1;  // level-1 cells per thread and trip in its half sweeps

// block-partial slots (nblk doubles each) in MgArgs::part
enum { MGS_BB = 0, MGS_RES = 1, MGS_RZ = 2, MGS_PQ = 3, MGS_RR = 4, MGS_SLOTS = 5 };
static_assert(MGS_SLOTS == MGS_PART_SLOTS, "batch partial buffers are sized by MGS_PART_SLOTS");

// Programmatic dependent launch: the loop's lattice kernels are launched so
// that they may start while the kernel before them drains; each waits here,
// before touching anything that kernel wrote, until it has completed and its
// writes are visible (a no-op when launched without the attribute).
__device__ __forceinline__ void mgs_wait_previous() { cudaGridDependencySynchronize(); }

__device__ __forceinline__ double *mgs_slot(const MgArgs &m, int slot, int nblk) { return m.part + (size_t)slot * nblk; }

// Start of the solve: guess, source and its block partials of b^2; block 0
// records the step's solver settings.
template <typename S, typename R, typename PhiT>
__global__ void __launch_bounds__(MGS_THREADS, 1) mgs_start_kernel(StepArgs<S, R, PhiT> a, MgArgs m, MgCtl *ctl)
{
    mgs_wait_previous();
    __shared__ double sh[MGS_THREADS / 32];
    __shared__ double bc[1];
    const int tid = blockIdx.x * blockDim.x + threadIdx.x, nthr = gridDim.x * blockDim.x;
    const double t = mg_start_pass(a, m, m.link, tid, nthr, sh, bc);
    if (threadIdx.x == 0) mgs_slot(m, MGS_BB, gridDim.x)[blockIdx.x] = t;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        ctl->tol = a.tol;
        ctl->max_iter = a.max_iter;
        ctl->fixed_iter = a.fixed_iter;
    }
}

// True residual with its block partials of r^2.  when: 0 always, 1 when the
// control state asks for one, 2 when phi moved since the last one.
template <typename PhiT>
__global__ void __launch_bounds__(MGS_THREADS, 1)
    mgs_residual_kernel(Grid3 g, MgArgs m, const PhiT *phi, const PhiT *b, const MgCtl *ctl, int when)
{
    mgs_wait_previous();
    __shared__ double sh[MGS_THREADS / 32];
    if (when == 1 && !ctl->need_true) return;
    if (when == 2 && (ctl->current || ctl->skip)) return;
    const int tid = blockIdx.x * blockDim.x + threadIdx.x, nthr = gridDim.x * blockDim.x;
    const double t = mg_true_residual<PhiT>(g, m.link, phi, b, m.r, m.z, tid, nthr, sh);
    if (threadIdx.x == 0) mgs_slot(m, MGS_RES, gridDim.x)[blockIdx.x] = t;
}

// Control kernels: one block of 32 threads.
static __global__ void mgs_init_kernel(MgArgs m, MgCtl *ctl, int nblk, cudaGraphConditionalHandle loop,
                                       int *pois_iters, double *pois_res)
{
    mgs_wait_previous();
    __shared__ double bc[1];
    const double bb = sum_partials(mgs_slot(m, MGS_BB, nblk), nblk, bc);
    const double rr = sum_partials(mgs_slot(m, MGS_RES, nblk), nblk, bc);
    if (threadIdx.x != 0) return;
    MgCtl c = *ctl;
    c.bb = bb;
    c.it = 0;
    c.pi = 0;
    c.fresh = 1;
    c.current = 1;
    c.stop = 0;
    c.need_true = 0;
    c.skip = 0;
    c.rz_old = 1.0;
    c.limit = c.fixed_iter > 0 ? c.fixed_iter : c.max_iter;
    c.tol2 = c.tol * c.tol * bb;
    c.rr_true = rr;
    c.rr_ref = rr;
    c.converged = c.fixed_iter <= 0 && rr <= c.tol2;
    if (c.fixed_iter <= 0 && bb == 0.0) {
        *pois_iters = 0;
        *pois_res = 0.0;
        c.skip = 1;
        c.converged = 1;
    }
    *ctl = c;
    cudaGraphSetConditional(loop, (!c.converged && c.it < c.limit) ? 1u : 0u);
}

// After the update pass: the CG scalars of the iteration, and whether the
// true residual is due (the recurrence residual fell by inner_red, or under
// a quarter of the tolerance, or the iteration limit is reached).
static __global__ void mgs_mid_kernel(MgArgs m, MgCtl *ctl, int nblk)
{
    mgs_wait_previous();
    __shared__ double bc[1];
    const double rz = sum_partials(mgs_slot(m, MGS_RZ, nblk), nblk, bc);
    const double pq = sum_partials(mgs_slot(m, MGS_PQ, nblk), nblk, bc);
    const double rr = sum_partials(mgs_slot(m, MGS_RR, nblk), nblk, bc);
    if (threadIdx.x != 0) return;
    MgCtl c = *ctl;
    c.need_true = 0;
    if (!(rz > 0.0) || !(pq > 0.0)) {
        c.stop = 1;  // breakdown: phi was not moved in this iteration
    } else {
        c.rz_old = rz;
        c.pi ^= 1;
        c.it++;
        c.fresh = 0;
        c.current = 0;
        if (c.fixed_iter <= 0 &&
            (rr <= 0.25 * c.tol2 || rr <= (double)m.inner_red * m.inner_red * c.rr_ref || c.it == c.limit))
            c.need_true = 1;
    }
    *ctl = c;
}

// After the (conditional) true residual: convergence test, restart, and the
// loop's condition.
static __global__ void mgs_end_kernel(MgArgs m, MgCtl *ctl, int nblk, cudaGraphConditionalHandle loop,
                                      const int *status)
{
    mgs_wait_previous();
    __shared__ double bc[1];
    const double rt = sum_partials(mgs_slot(m, MGS_RES, nblk), nblk, bc);
    if (threadIdx.x != 0) return;
    MgCtl c = *ctl;
    if (c.need_true) {
        c.rr_true = rt;
        c.current = 1;
        if (rt <= c.tol2) {
            c.converged = 1;
        } else {
            c.rr_ref = rt;
            c.fresh = 1;
        }
        c.need_true = 0;
    }
    *ctl = c;
    const bool go = !c.stop && !c.converged && c.it < c.limit && !(*(volatile const int *)status & ST_TIMEOUT);
    cudaGraphSetConditional(loop, go ? 1u : 0u);
}

// Iterations, final relative residual and the non-convergence flag.
static __global__ void mgs_report_kernel(MgArgs m, const MgCtl *ctl, int nblk, int *pois_iters,
                                         long long *pois_total, double *pois_res, int *status)
{
    mgs_wait_previous();
    __shared__ double bc[1];
    const double rt = sum_partials(mgs_slot(m, MGS_RES, nblk), nblk, bc);
    if (threadIdx.x != 0) return;
    const MgCtl c = *ctl;
    if (c.skip) return;
    // a final true residual was formed exactly when phi moved after the last one
    const double rr_true = c.current ? c.rr_true : rt;
    *pois_iters = c.it;
    pois_total[0] += c.it;
    *pois_res = sqrt(rr_true / c.bb);
    if (c.fixed_iter <= 0 && !(c.converged || rr_true <= c.tol2)) atomicOr(status, ST_NOCONV);
}

// V-cycle on the lattice level: one red-black half sweep (RZ: the last one,
// with the block partials of r.z; PRO: the prolongating one)
template <bool RZ, bool PRO>
__global__ void __launch_bounds__(MGS_THREADS, 1) mgs_half_kernel(Grid3 g, MgArgs m, int c)
{
    mgs_wait_previous();
    __shared__ double sh[MGS_THREADS / 32];
    const int tid = blockIdx.x * blockDim.x + threadIdx.x, nthr = gridDim.x * blockDim.x;
    float rz = 0.f;
    fine_half<RZ, PRO, MGS_U>(g, m.link, m.r, m.z, m.lev[1], c, tid, nthr, rz);
    if constexpr (RZ) {
        const double t = block_sum_lanes0(warp_sum_ff_lane0(rz), sh);
        if (threadIdx.x == 0) mgs_slot(m, MGS_RZ, gridDim.x)[blockIdx.x] = t;
    }
}

template <bool FIRST> __global__ void __launch_bounds__(MGS_THREADS, 1) mgs_restrict_kernel(Grid3 g, MgArgs m)
{
    mgs_wait_previous();
    fine_restrict_cells<FIRST>(g, m.link, m.r, m.z, m.lev[1], (int)(blockIdx.x * blockDim.x + threadIdx.x),
                         (int)(gridDim.x * blockDim.x));
}

// Level 1, when grid-wide, in separate launches like the lattice: one
// red-black half sweep (PRO: prolongating from level 2) ...
template <bool PRO> __global__ void __launch_bounds__(MGS_THREADS, 1) mgs_chalf_kernel(MgArgs m, int c)
{
    mgs_wait_previous();
    coarse_half<false, PRO, MGS_CU>(m.lev[1], m.lev[2], c, (int)(blockIdx.x * blockDim.x + threadIdx.x),
                            (int)(gridDim.x * blockDim.x));
}
// ... and its restriction to level 2 (FIRST: level 2 is grid-wide or tiled)
template <bool FIRST> __global__ void __launch_bounds__(MGS_THREADS, 1) mgs_crestrict_kernel(MgArgs m)
{
    mgs_wait_previous();
    coarse_restrict<false, FIRST>(m.lev[1], m.lev[2], (int)(blockIdx.x * blockDim.x + threadIdx.x),
                                  (int)(gridDim.x * blockDim.x));
}

// The coarse levels of one V-cycle from level `from` (cooperative launch;
// `bar` zeroed before it)
static __global__ void __launch_bounds__(MGS_THREADS, 1) mgs_coarse_kernel(MgArgs m, unsigned *bar, int *status,
                                                                          int from)
{
    mgs_wait_previous();
    __shared__ double sh[MGS_THREADS / 32];
    __shared__ double bc[1];
    extern __shared__ float mg_sm[];
    const MgGrid G{(int)(blockIdx.x * blockDim.x + threadIdx.x), (int)(gridDim.x * blockDim.x), (int)gridDim.x,
                   (int)blockIdx.x, bar};
    if (G.blk == 0 && !m.dense) mg_cta_load(m, mg_sm);
    unsigned bar_k = 0;
    mg_coarse_cycle<true>(m, G, bar_k, status, mg_sm, sh, bc, from);
}

// p = z + beta p_old, q = A p with the block partials of p.q
static __global__ void __launch_bounds__(MGS_THREADS, 1) mgs_pq_kernel(Grid3 g, MgArgs m, const MgCtl *ctl)
{
    mgs_wait_previous();
    __shared__ double sh[MGS_THREADS / 32];
    __shared__ double bc[1];
    const int nblk = gridDim.x;
    const double rz = sum_partials(mgs_slot(m, MGS_RZ, nblk), nblk, bc);
    if (!(rz > 0.0)) return;
    const int tid = blockIdx.x * blockDim.x + threadIdx.x, nthr = gridDim.x * blockDim.x;
    const int fresh = ctl->fresh, pi = ctl->pi;
    const float beta = fresh ? 0.f : (float)(rz / ctl->rz_old);
    const float *pold = m.p[pi];
    float *pnew = m.p[pi ^ 1];
    const float t = fresh ? mg_pq_pass<true, uint8_t, MGS_PQU>(g, m.link, m.z, pold, pnew, m.q, beta, tid, nthr)
                          : mg_pq_pass<false, uint8_t, MGS_PQU>(g, m.link, m.z, pold, pnew, m.q, beta, tid, nthr);
    const double pq = block_sum_lanes0(warp_sum_ff_lane0(t), sh);
    if (threadIdx.x == 0) mgs_slot(m, MGS_PQ, nblk)[blockIdx.x] = pq;
}

// phi += alpha p, r -= alpha q (and the next V-cycle's first half sweep)
// with the block partials of r^2
template <typename PhiT>
__global__ void __launch_bounds__(MGS_THREADS, 1) mgs_update_kernel(Grid3 g, MgArgs m, PhiT *phi, const MgCtl *ctl)
{
    mgs_wait_previous();
    __shared__ double sh[MGS_THREADS / 32];
    __shared__ double bc[1];
    const int nblk = gridDim.x;
    const double rz = sum_partials(mgs_slot(m, MGS_RZ, nblk), nblk, bc);
    const double pq = sum_partials(mgs_slot(m, MGS_PQ, nblk), nblk, bc);
    if (!(rz > 0.0) || !(pq > 0.0)) return;
    const int tid = blockIdx.x * blockDim.x + threadIdx.x, nthr = gridDim.x * blockDim.x;
    const double alpha = rz / pq;
    const float t = mg_update_pass<PhiT>(g, m.link, phi, m.p[ctl->pi ^ 1], m.q, m.r, m.z, alpha, tid, nthr);
    const double rr = block_sum_lanes0(warp_sum_ff_lane0(t), sh);
    if (threadIdx.x == 0) mgs_slot(m, MGS_RR, nblk)[blockIdx.x] = rr;
}

}  // namespace ekl

// ------------------------------------------------------------------ batches
// The split solve for a batch of replicas: every kernel runs over all
// replicas at once, block b working for replica block_rep[b] as its block
// block_local[b] of rep_blocks[r], with one MgCtl per replica; a replica
// that has converged skips its work, and the loop runs while any replica
// has not.  The lattice passes and the coarse launch have tables of their
// own: the coarse launch is cooperative (the cooperative batch solve's
// blocks, one per SM), while the lattice passes may take several times as
// many blocks, which evens out the load of replicas of uneven size.  With
// the same tables for both, thread maps and partials are those of the
// cooperative batch solve and the results are the same bit for bit.
// Replicas do not tile their coarse levels.
namespace ekl {

struct MgsBatch {
    const MgArgs *mg;  // [nrep]
    const Grid3 *grid; // [nrep] lattice of each replica
    MgCtl *ctl;        // [nrep]
    PoisBatch pb;      // blocks of the lattice passes
    PoisBatch cpb;     // blocks of the cooperative coarse launch
    double *part;      // block partials: replica r, slot s at part + (r MGS_SLOTS + s) stride
    int stride;
    int *loops;        // iterations the batch loop has run (launch accounting)
};

__device__ __forceinline__ double *mgsb_slot(const MgsBatch &B, int r, int slot)
{
    return B.part + ((size_t)r * MGS_SLOTS + slot) * B.stride;
}

// A replica's descriptors live in global memory, where the passes' own
// stores could alias them as far as the compiler knows: read through a
// reference there, a field would be loaded again after every store.  The
// kernels therefore take value copies (the lattice and level 1 in
// registers) or, for the whole descriptor, a copy in shared memory.
template <typename T> __device__ __forceinline__ void mgsb_copy(const T *src, T &dst)
{
    static_assert(sizeof(T) % sizeof(int) == 0, "descriptor copied as 4-byte words");
    const int *s = (const int *)src;
    int *d = (int *)&dst;
    for (int i = threadIdx.x; i < (int)(sizeof(T) / sizeof(int)); i += blockDim.x) d[i] = __ldg(s + i);
    __syncthreads();
}

struct BRep {
    int r, lb, nb, t0, nt;
};
__device__ __forceinline__ BRep mgsb_rep(const PoisBatch &pb)
{
    BRep x;
    x.r = pb.block_rep[blockIdx.x];
    x.lb = pb.block_local[blockIdx.x];
    x.nb = pb.rep_blocks[x.r];
    x.t0 = x.lb * blockDim.x + threadIdx.x;
    x.nt = x.nb * blockDim.x;
    return x;
}

template <typename S, typename R, typename PhiT>
__global__ void __launch_bounds__(MGS_THREADS, 1)
    mgsb_start_kernel(const StepArgs<S, R, PhiT> *reps, MgsBatch B)
{
    mgs_wait_previous();
    __shared__ double sh[MGS_THREADS / 32];
    __shared__ double bc[1];
    __shared__ StepArgs<S, R, PhiT> s_a;
    __shared__ MgArgs s_m;
    const BRep x = mgsb_rep(B.pb);
    mgsb_copy(reps + x.r, s_a);
    mgsb_copy(B.mg + x.r, s_m);
    const StepArgs<S, R, PhiT> &a = s_a;
    const MgArgs &m = s_m;
    const double t = mg_start_pass(a, m, m.link, x.t0, x.nt, sh, bc);
    if (threadIdx.x == 0) mgsb_slot(B, x.r, MGS_BB)[x.lb] = t;
    if (x.lb == 0 && threadIdx.x == 0) {
        MgCtl &c = B.ctl[x.r];
        c.tol = a.tol;
        c.max_iter = a.max_iter;
        c.fixed_iter = a.fixed_iter;
    }
}

template <typename S, typename R, typename PhiT>
__global__ void __launch_bounds__(MGS_THREADS, 1)
    mgsb_residual_kernel(const StepArgs<S, R, PhiT> *reps, MgsBatch B, int when)
{
    mgs_wait_previous();
    __shared__ double sh[MGS_THREADS / 32];
    const BRep x = mgsb_rep(B.pb);
    const MgCtl &c = B.ctl[x.r];
    if (when == 1 && (c.done || !c.need_true)) return;
    if (when == 2 && (c.current || c.skip)) return;
    const Grid3 g = B.grid[x.r];
    const MgArgs &m = B.mg[x.r];
    const double t = mg_true_residual<PhiT>(g, m.link, reps[x.r].phi, reps[x.r].b, m.r, m.z, x.t0, x.nt, sh);
    if (threadIdx.x == 0) mgsb_slot(B, x.r, MGS_RES)[x.lb] = t;
}

// one block of 32 threads per replica
template <typename S, typename R, typename PhiT>
__global__ void mgsb_init_kernel(const StepArgs<S, R, PhiT> *reps, MgsBatch B)
{
    mgs_wait_previous();
    __shared__ double bc[1];
    const int r = blockIdx.x, nb = B.pb.rep_blocks[r];
    const MgArgs &m = B.mg[r];
    const double bb = sum_partials(mgsb_slot(B, r, MGS_BB), nb, bc);
    const double rr = sum_partials(mgsb_slot(B, r, MGS_RES), nb, bc);
    if (threadIdx.x != 0) return;
    MgCtl c = B.ctl[r];
    c.bb = bb;
    c.it = 0;
    c.pi = 0;
    c.fresh = 1;
    c.current = 1;
    c.stop = 0;
    c.need_true = 0;
    c.skip = 0;
    c.rz_old = 1.0;
    c.limit = c.fixed_iter > 0 ? c.fixed_iter : c.max_iter;
    c.tol2 = c.tol * c.tol * bb;
    c.rr_true = rr;
    c.rr_ref = rr;
    c.converged = c.fixed_iter <= 0 && rr <= c.tol2;
    if (c.fixed_iter <= 0 && bb == 0.0) {
        *reps[r].pois_iters = 0;
        *reps[r].pois_res = 0.0;
        c.skip = 1;
        c.converged = 1;
    }
    c.done = c.converged || c.it >= c.limit;
    B.ctl[r] = c;
}

// one block: the loop goes on while any replica is not done
__global__ static void mgsb_cond_kernel(MgsBatch B, cudaGraphConditionalHandle loop, int count)
{
    mgs_wait_previous();
    __shared__ int any;
    if (threadIdx.x == 0) any = 0;
    __syncthreads();
    int mine = 0;
    for (int r = threadIdx.x; r < B.pb.nrep; r += blockDim.x) mine |= !B.ctl[r].done;
    if (mine) atomicOr(&any, 1);
    __syncthreads();
    if (threadIdx.x == 0) {
        cudaGraphSetConditional(loop, any ? 1u : 0u);
        if (count && any) *B.loops += 1;
    }
}

template <bool RZ, bool PRO>
__global__ void __launch_bounds__(MGS_THREADS, 1) mgsb_half_kernel(MgsBatch B, int c)
{
    mgs_wait_previous();
    __shared__ double sh[MGS_THREADS / 32];
    const BRep x = mgsb_rep(B.pb);
    if (B.ctl[x.r].done) return;
    const MgArgs &m = B.mg[x.r];
    float rz = 0.f;
    const Grid3 g = B.grid[x.r];
    const MgLevel l1 = m.lev[1];
    fine_half<RZ, PRO, MGS_U>(g, m.link, m.r, m.z, l1, c, x.t0, x.nt, rz);
    if constexpr (RZ) {
        const double t = block_sum_lanes0(warp_sum_ff_lane0(rz), sh);
        if (threadIdx.x == 0) mgsb_slot(B, x.r, MGS_RZ)[x.lb] = t;
    }
}

__global__ static void __launch_bounds__(MGS_THREADS, 1) mgsb_restrict_kernel(MgsBatch B)
{
    mgs_wait_previous();
    const BRep x = mgsb_rep(B.pb);
    if (B.ctl[x.r].done) return;
    const MgArgs &m = B.mg[x.r];
    const Grid3 g = B.grid[x.r];
    const MgLevel l1 = m.lev[1];
    if (m.cta_from > 1) fine_restrict_cells<true>(g, m.link, m.r, m.z, l1, x.t0, x.nt);
    else fine_restrict_cells<false>(g, m.link, m.r, m.z, l1, x.t0, x.nt);
}

// the coarse levels of every active replica (cooperative; `bars` zeroed)
template <typename S, typename R, typename PhiT>
__global__ void __launch_bounds__(MGS_THREADS, 1)
    mgsb_coarse_kernel(const StepArgs<S, R, PhiT> *reps, MgsBatch B, unsigned *bars)
{
    mgs_wait_previous();
    __shared__ double sh[MGS_THREADS / 32];
    __shared__ double bc[1];
    extern __shared__ float mg_sm[];
    const BRep x = mgsb_rep(B.cpb);
    if (B.ctl[x.r].done) return;  // every block of that replica
    __shared__ MgArgs s_m;
    mgsb_copy(B.mg + x.r, s_m);
    const MgArgs &m = s_m;
    const MgGrid G{x.t0, x.nt, x.nb, x.lb, bars + 4 * x.r};
    if (G.blk == 0 && !m.dense) mg_cta_load(m, mg_sm);
    unsigned bar_k = 0;
    mg_coarse_cycle<false>(m, G, bar_k, reps[x.r].status, mg_sm, sh, bc, 1);
}

__global__ static void __launch_bounds__(MGS_THREADS, 1) mgsb_pq_kernel(MgsBatch B)
{
    mgs_wait_previous();
    __shared__ double sh[MGS_THREADS / 32];
    __shared__ double bc[1];
    const BRep x = mgsb_rep(B.pb);
    const MgCtl &c = B.ctl[x.r];
    if (c.done) return;
    const MgArgs &m = B.mg[x.r];
    const double rz = sum_partials(mgsb_slot(B, x.r, MGS_RZ), x.nb, bc);
    if (!(rz > 0.0)) return;
    const int fresh = c.fresh, pi = c.pi;
    const float beta = fresh ? 0.f : (float)(rz / c.rz_old);
    const float *pold = m.p[pi];
    float *pnew = m.p[pi ^ 1];
    const Grid3 g = B.grid[x.r];
    const float t = fresh ? mg_pq_pass<true, uint8_t, MGS_PQU>(g, m.link, m.z, pold, pnew, m.q, beta, x.t0, x.nt)
                          : mg_pq_pass<false, uint8_t, MGS_PQU>(g, m.link, m.z, pold, pnew, m.q, beta, x.t0, x.nt);
    const double pq = block_sum_lanes0(warp_sum_ff_lane0(t), sh);
    if (threadIdx.x == 0) mgsb_slot(B, x.r, MGS_PQ)[x.lb] = pq;
}

template <typename S, typename R, typename PhiT>
__global__ void __launch_bounds__(MGS_THREADS, 1) mgsb_update_kernel(const StepArgs<S, R, PhiT> *reps, MgsBatch B)
{
    mgs_wait_previous();
    __shared__ double sh[MGS_THREADS / 32];
    __shared__ double bc[1];
    const BRep x = mgsb_rep(B.pb);
    const MgCtl &c = B.ctl[x.r];
    if (c.done) return;
    const MgArgs &m = B.mg[x.r];
    const double rz = sum_partials(mgsb_slot(B, x.r, MGS_RZ), x.nb, bc);
    const double pq = sum_partials(mgsb_slot(B, x.r, MGS_PQ), x.nb, bc);
    if (!(rz > 0.0) || !(pq > 0.0)) return;
    const double alpha = rz / pq;
    const Grid3 g = B.grid[x.r];
    const float t = mg_update_pass<PhiT>(g, m.link, reps[x.r].phi, m.p[c.pi ^ 1], m.q, m.r, m.z, alpha,
                                         x.t0, x.nt);
    const double rr = block_sum_lanes0(warp_sum_ff_lane0(t), sh);
    if (threadIdx.x == 0) mgsb_slot(B, x.r, MGS_RR)[x.lb] = rr;
}

// one block of 32 threads per replica (active replicas only)
__global__ static void mgsb_mid_kernel(MgsBatch B)
{
    mgs_wait_previous();
    __shared__ double bc[1];
    const int r = blockIdx.x, nb = B.pb.rep_blocks[r];
    if (B.ctl[r].done) return;
    const MgArgs &m = B.mg[r];
    const double rz = sum_partials(mgsb_slot(B, r, MGS_RZ), nb, bc);
    const double pq = sum_partials(mgsb_slot(B, r, MGS_PQ), nb, bc);
    const double rr = sum_partials(mgsb_slot(B, r, MGS_RR), nb, bc);
    if (threadIdx.x != 0) return;
    MgCtl c = B.ctl[r];
    c.need_true = 0;
    if (!(rz > 0.0) || !(pq > 0.0)) {
        c.stop = 1;
    } else {
        c.rz_old = rz;
        c.pi ^= 1;
        c.it++;
        c.fresh = 0;
        c.current = 0;
        if (c.fixed_iter <= 0 &&
            (rr <= 0.25 * c.tol2 || rr <= (double)m.inner_red * m.inner_red * c.rr_ref || c.it == c.limit))
            c.need_true = 1;
    }
    B.ctl[r] = c;
}

template <typename S, typename R, typename PhiT>
__global__ void mgsb_end_kernel(const StepArgs<S, R, PhiT> *reps, MgsBatch B)
{
    mgs_wait_previous();
    __shared__ double bc[1];
    const int r = blockIdx.x, nb = B.pb.rep_blocks[r];
    if (B.ctl[r].done) return;
    const MgArgs &m = B.mg[r];
    const double rt = sum_partials(mgsb_slot(B, r, MGS_RES), nb, bc);
    if (threadIdx.x != 0) return;
    MgCtl c = B.ctl[r];
    if (c.need_true) {
        c.rr_true = rt;
        c.current = 1;
        if (rt <= c.tol2) {
            c.converged = 1;
        } else {
            c.rr_ref = rt;
            c.fresh = 1;
        }
        c.need_true = 0;
    }
    c.done = c.stop || c.converged || c.it >= c.limit || (*(volatile const int *)reps[r].status & ST_TIMEOUT);
    B.ctl[r] = c;
}

template <typename S, typename R, typename PhiT>
__global__ void mgsb_report_kernel(const StepArgs<S, R, PhiT> *reps, MgsBatch B)
{
    mgs_wait_previous();
    __shared__ double bc[1];
    const int r = blockIdx.x, nb = B.pb.rep_blocks[r];
    const MgArgs &m = B.mg[r];
    const double rt = sum_partials(mgsb_slot(B, r, MGS_RES), nb, bc);
    if (threadIdx.x != 0) return;
    const MgCtl c = B.ctl[r];
    if (c.skip) return;
    const double rr_true = c.current ? c.rr_true : rt;
    const StepArgs<S, R, PhiT> &a = reps[r];
    *a.pois_iters = c.it;
    a.pois_total[0] += c.it;
    *a.pois_res = sqrt(rr_true / c.bb);
    if (c.fixed_iter <= 0 && !(c.converged || rr_true <= c.tol2)) atomicOr(a.status, ST_NOCONV);
}

}  // namespace ekl
