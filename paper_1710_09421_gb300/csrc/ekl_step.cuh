// Host orchestration of the step for one (storage, arithmetic, potential)
// combination; included by the instantiation units.
#pragma once
#include <cooperative_groups.h>

#include <algorithm>
#include <vector>

#include "ekl_kernels.cuh"
#include "ekl_mg.cuh"
#include "ekl_mgs.cuh"

namespace ekl {

template <typename S, typename R, typename PhiT>
static StepArgs<S, R, PhiT> make_args(Ctx &c, int parity = -1)
{
    StepArgs<S, R, PhiT> a;
    const int cur = parity < 0 ? c.cur : parity;
    a.g = make_grid3(c.nx, c.ny, c.nz);
    for (int k = 0; k < 3; k++) a.per[k] = c.per[k];
    a.mask = c.mask;
    a.fin = (const S *)c.f[cur];
    a.fout = (S *)c.f[1 - cur];
    a.phi = (PhiT *)c.phi;
    a.b = (PhiT *)c.b;
    a.rho = (R *)c.rho;
    a.wall_share = (const R *)c.wall_share;
    a.src_wall = (const R *)c.src_wall;
    for (int s = 0; s < NS; s++) {
        a.n_ref[s] = (R)c.P.n_ref[s];
        a.zv[s] = (R)c.P.valence[s];
        a.wd[s] = (R)c.wd[s];
        a.om[s] = (R)c.om[s];
        for (int k = 0; k < 3; k++) a.body[s][k] = (R)c.P.body_force[s][k];
    }
    for (int k = 0; k < 3; k++) a.E[k] = (R)c.P.E_app[k];
    a.c4 = (R)c.c4;
    a.flags = c.P.flags;
    a.patch_count = c.patch_count;
    a.patch_bits = c.patch_bits;
    a.patch_node = c.patch_node;
    a.patch_q = (const R *)c.patch_q;
    a.patch_f = (const R *)c.patch_f;
    a.part_charge = c.part_charge;
    a.part_charge_q = c.part_charge_q;
    a.charge_tot = c.charge_tot;
    a.charge_tot_q = c.charge_tot_q;
    a.part_mass = c.part_mass;
    a.part_pois = c.part_pois;
    a.barrier = c.barrier;
    a.status = c.status;
    a.pois_iters = c.pois_iters;
    a.pois_total = c.pois_total;
    a.pois_res = c.pois_res;
    a.tol = c.P.poisson_tol;
    a.max_iter = c.P.poisson_max_iter;
    a.check_every = c.P.poisson_check_every < 1 ? 1 : c.P.poisson_check_every;
    a.fixed_iter = c.P.poisson_fixed_iter;
    a.rJ = c.rJ;
    a.omegas = c.omegas;
    a.n_fluid = (double)c.n_fluid;
    a.wchi = (const R *)c.wchi;
    a.fluct_m = (R)c.P.fluct_mass;
    a.key0 = (uint32_t)c.P.seed;
    a.key1 = (uint32_t)(c.P.seed >> 32);
    a.step = c.step;
    a.nblocks_charge = c.charge_blocks;  // one partial per block
    return a;
}

template <typename R> static BeadArgs<R> make_bead_args(Ctx &c)
{
    BeadArgs<R> b;
    b.g = make_grid3(c.nx, c.ny, c.nz);
    for (int k = 0; k < 3; k++) b.per[k] = c.per[k];
    b.mask = c.mask;
    b.nb = c.nb;
    b.Rb = (double *)c.R;
    b.Vb = (R *)c.V;
    b.qb = (const R *)c.q;
    b.chain = c.chain;
    b.patch_count = c.patch_count;
    b.patch_bits = c.patch_bits;
    b.patch_node = c.patch_node;
    b.patch_q = (R *)c.patch_q;
    b.patch_f = (R *)c.patch_f;
    b.patch_mom = (R *)c.patch_mom;
    b.entry_slot = c.entry_slot;
    b.entry_w = (R *)c.entry_w;
    b.sorted_entry = c.sorted_entry;
    b.slot_first = c.slot_first;
    b.status = c.status;
    return b;
}

template <typename S, typename R, typename PhiT, bool DEV>
static MdArgs<S, R, PhiT, DEV> make_md_args(Ctx &c, const StepArgs<S, R, PhiT> &a, const BeadArgs<R> &ba)
{
    MdArgs<S, R, PhiT, DEV> md;
    md.s = a;
    md.b = ba;
    md.md_substeps = c.P.md_substeps < 1 ? 1 : c.P.md_substeps;
    md.xi = (R)c.P.bead_xi;
    md.mass = (R)c.P.bead_mass;
    md.bead_kT = (R)c.P.bead_kT;
    md.bond_kind = c.P.bond_kind;
    md.bond_k = (R)c.P.bond_k;
    md.bond_r0 = (R)c.P.bond_r0;
    md.bond_l0 = (R)c.P.bond_l0;
    md.wca_eps = (R)c.P.wca_eps;
    md.wca_sigma = (R)c.P.wca_sigma;
    md.wall_eps = (R)c.P.wall_eps;
    md.wall_sigma = (R)c.P.wall_sigma;
    md.key0 = (uint32_t)c.P.seed;
    md.key1 = (uint32_t)(c.P.seed >> 32);
    md.step = c.step;
    return md;
}

// The multigrid solve of poisson_mg_kernel with 1024-thread blocks (64
// registers a thread), for lattices of at least MG_WIDE_NODES_PER_SM nodes
// per SM: their lattice passes are bound by memory throughput and gain from
// twice the warps in flight (17 against 23 ms per step on a 256x256x512
// pore), where a small lattice is bound by barrier latency and runs faster
// at 512 threads with 128 registers (0.68 against 0.75 ms on 64x64x128).
template <typename S, typename R, typename PhiT>
__global__ void __launch_bounds__(MG_WIDE_THREADS, 1) poisson_mg_wide_kernel(StepArgs<S, R, PhiT> a, MgArgs m)
{
    __shared__ double sh[MG_WIDE_THREADS / 32];
    __shared__ double bc[1];
    extern __shared__ float mg_sm[];
    const MgGrid G{(int)(blockIdx.x * blockDim.x + threadIdx.x), (int)(gridDim.x * blockDim.x), (int)gridDim.x,
                   (int)blockIdx.x, a.barrier};
    mg_solve<S, R, PhiT, true>(a, m, G, mg_sm, sh, bc);
}

static inline MgArgs make_mg_args(const Ctx &c)
{
    MgArgs m;
    m.r = c.mg_r;
    m.z = c.mg_z;
    m.q = c.mg_q;
    m.p[0] = c.mg_p[0];
    m.p[1] = c.mg_p[1];
    m.part = c.mg_part;
    m.link = c.mg_link;
    m.dense = c.mg_dense;
    m.phi_prev = c.mg_phi_prev;
    // with a learned warm start installed the network supplies the guess
    m.have_prev = c.mg_have_prev && !c.net;
    m.nlev = c.mg_nlev;
    m.cta_from = c.mg_cta_from;
    m.nu = MG_NU;
    m.nu_c = MG_NU_COARSE;
    m.coarse_sweeps = MG_COARSE_SWEEPS;
    m.inner_red = MG_INNER_RED;
    m.tile_from = c.mg_tile_from;
    m.tile_off = (int)c.mg_tile_off;
    for (int l = 0; l < MG_MAXLEV; l++) {
        m.lev[l] = c.mg_lev[l];
        for (int k = 0; k < 3; k++) m.tile[l][k] = c.mg_tile[l][k];
    }
    return m;
}

// Graph of a split multigrid solve (ekl_mgs.cuh), launched after the step's
// start kernel:
//   true residual -> init -> WHILE (condition set by init / end) {
//     pre-smoothing half sweeps, restriction, [level 1: half sweeps and
//     restriction], coarse levels (cooperative), [level 1: prolongating and
//     post-smoothing half sweeps], lattice prolongating and post-smoothing
//     half sweeps, p/q, update, mid, true residual when due, end }
//   -> true residual when phi moved after the last one -> report.
// Every argument is fixed for the life of the handle; the step's tolerance
// and iteration limits reach the graph through MgCtl.
template <typename PhiT> static cudaError_t mgs_build(Ctx &c, const MgArgs &m0, Grid3 g, bool pdl)
{
    MgArgs m = m0;
    const int nb = c.pois_blocks, nt = c.mgs_threads;
    MgCtl *ctl = (MgCtl *)c.mgs_ctl;
    const PhiT *phi = (const PhiT *)c.phi, *b = (const PhiT *)c.b;
    PhiT *phiw = (PhiT *)c.phi;
    int when0 = 0, when2 = 2, nblk = nb;
    cudaGraph_t G = nullptr;
    cudaStream_t cs = nullptr;
    cudaGraphConditionalHandle loop;
    cudaGraphNode_t nres0, ninit, nloop, nres2, nrep;
    cudaError_t e = cudaGraphCreate(&G, 0);
    auto kernel_node = [&](cudaGraphNode_t *out, cudaGraphNode_t *dep, const void *fn, int grid, int block,
                           void **args) {
        cudaKernelNodeParams kp = {};
        kp.func = (void *)fn;
        kp.gridDim = dim3(grid);
        kp.blockDim = dim3(block);
        kp.kernelParams = args;
        return cudaGraphAddKernelNode(out, G, dep, dep ? 1 : 0, &kp);
    };
    if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&loop, G, 0, cudaGraphCondAssignDefault);
    if (e == cudaSuccess) {
        void *args[] = {&g, &m, &phi, &b, &ctl, &when0};
        e = kernel_node(&nres0, nullptr, (const void *)mgs_residual_kernel<PhiT>, nb, nt, args);
    }
    if (e == cudaSuccess) {
        void *args[] = {&m, &ctl, &nblk, &loop, &c.pois_iters, &c.pois_res};
        e = kernel_node(&ninit, &nres0, (const void *)mgs_init_kernel, 1, 32, args);
    }
    cudaGraph_t body = nullptr;
    if (e == cudaSuccess) {
        cudaGraphNodeParams cp = {};
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = loop;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        e = cudaGraphAddNode(&nloop, G, &ninit, nullptr, 1, &cp);
        if (e == cudaSuccess) body = cp.conditional.phGraph_out[0];
    }
    if (e == cudaSuccess && c.mg_smem > 48 * 1024)
        e = cudaFuncSetAttribute(mgs_coarse_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)c.mg_smem);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
    if (e == cudaSuccess) {
        // every lattice kernel but the first of the body and the one after
        // the cooperative launch may start while its predecessor drains
        // (programmatic dependent launch; each waits for its predecessor
        // before touching its output)
        cudaLaunchAttribute dep[1];
        dep[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        dep[0].val.programmaticStreamSerializationAllowed = 1;
        cudaError_t el = cudaSuccess;
        auto go = [&](bool overlap, unsigned grid, unsigned block, auto kern, auto... args) {
            cudaLaunchConfig_t lc = {};
            lc.gridDim = dim3(grid);
            lc.blockDim = dim3(block);
            lc.stream = cs;
            lc.attrs = dep;
            lc.numAttrs = (overlap && pdl) ? 1 : 0;
            const cudaError_t r = cudaLaunchKernelEx(&lc, kern, args...);
            if (el == cudaSuccess) el = r;
        };
        for (int s = 1; s < 2 * MG_NU; s++) go(s > 1, nb, nt, mgs_half_kernel<false, false>, g, m, s & 1);
        if (m.cta_from > 1) go(true, nb, nt, mgs_restrict_kernel<true>, g, m);
        else go(true, nb, nt, mgs_restrict_kernel<false>, g, m);
        // level 1 smoothed and restricted by separate launches when grid-wide
        const int from = c.mgs_l1 ? 2 : 1;
        if (c.mgs_l1) {
            for (int s = 1; s < 2 * MG_NU_COARSE; s++) go(true, nb, nt, mgs_chalf_kernel<false>, m, s & 1);
            if (m.cta_from > 2) go(true, nb, nt, mgs_crestrict_kernel<true>, m);
            else go(true, nb, nt, mgs_crestrict_kernel<false>, m);
        }
        cudaMemsetAsync(c.barrier, 0, 4 * sizeof(unsigned), cs);
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute coop[1];
        coop[0].id = cudaLaunchAttributeCooperative;
        coop[0].val.cooperative = 1;
        cfg.gridDim = dim3(nb);
        cfg.blockDim = dim3(nt);
        cfg.dynamicSmemBytes = c.mg_smem;
        cfg.stream = cs;
        cfg.attrs = coop;
        cfg.numAttrs = 1;
        const cudaError_t ecoop = cudaLaunchKernelEx(&cfg, mgs_coarse_kernel, m, c.barrier, c.status, from);
        if (el == cudaSuccess) el = ecoop;
        if (c.mgs_l1) {
            go(false, nb, nt, mgs_chalf_kernel<true>, m, 1);
            for (int s = 1; s < 2 * MG_NU_COARSE; s++) go(true, nb, nt, mgs_chalf_kernel<false>, m, (s & 1) ^ 1);
        }
        go(c.mgs_l1 != 0, nb, nt, mgs_half_kernel<false, true>, g, m, 1);
        for (int s = 1; s < 2 * MG_NU; s++) {
            const int col = (s & 1) ^ 1;
            if (s == 2 * MG_NU - 1) go(true, nb, nt, mgs_half_kernel<true, false>, g, m, col);
            else go(true, nb, nt, mgs_half_kernel<false, false>, g, m, col);
        }
        go(true, nb, nt, mgs_pq_kernel, g, m, (const MgCtl *)ctl);
        go(true, nb, nt, mgs_update_kernel<PhiT>, g, m, phiw, (const MgCtl *)ctl);
        go(true, 1, 32, mgs_mid_kernel, m, ctl, nb);
        go(true, nb, nt, mgs_residual_kernel<PhiT>, g, m, phi, b, (const MgCtl *)ctl, 1);
        go(true, 1, 32, mgs_end_kernel, m, ctl, nb, loop, (const int *)c.status);
        cudaError_t ek = cudaGetLastError();
        cudaError_t ec = cudaStreamEndCapture(cs, &body);
        e = el != cudaSuccess ? el : ek != cudaSuccess ? ek : ec;
    }
    if (cs) cudaStreamDestroy(cs);
    if (e == cudaSuccess) {
        void *args[] = {&g, &m, &phi, &b, &ctl, &when2};
        e = kernel_node(&nres2, &nloop, (const void *)mgs_residual_kernel<PhiT>, nb, nt, args);
    }
    if (e == cudaSuccess) {
        void *args[] = {&m, &ctl, &nblk, &c.pois_iters, &c.pois_total, &c.pois_res, &c.status};
        e = kernel_node(&nrep, &nres2, (const void *)mgs_report_kernel, 1, 32, args);
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&c.mgs_exec, G, 0);
    if (e != cudaSuccess) {
        if (G) cudaGraphDestroy(G);
        c.mgs_exec = nullptr;
        return e;
    }
    c.mgs_graph = G;
    return cudaSuccess;
}

static inline ChargeTotals charge_totals_args(const Ctx &c)
{
    ChargeTotals T;
    T.part = c.part_charge;
    T.part_q = c.part_charge_q;
    T.n = c.charge_blocks;
    T.tot = c.charge_tot;
    T.tot_q = c.charge_tot_q;
    T.chunk = (double *)c.charge_chunks;
    T.chunk_q = (long long *)(T.chunk + CHARGE_TOTAL_BLOCKS);
    T.arrived = (unsigned *)(T.chunk_q + CHARGE_TOTAL_BLOCKS);
    return T;
}

static inline int cuda_ok(cudaError_t e) { return e == cudaSuccess ? EKL_OK : EKL_ERR_CUDA; }

static inline void phase_begin(Ctx &c, int ph)
{
    if (c.timing) timing_record(c, ph, 1);
}
static inline void phase_end(Ctx &c, int ph)
{
    if (c.timing) timing_record(c, ph, 0);
}

template <typename S, typename R, typename PhiT, bool DEV> int init_impl(Ctx &c, const double *d_n)
{
    int blocks = (int)((c.N + 255) / 256);
    init_kernel<S, R, DEV><<<blocks, 256, 0, c.stream>>>(make_grid3(c.nx, c.ny, c.nz), c.mask, d_n,
                                                         (S *)c.f[c.cur], (R)c.P.n_ref[0],
                                                         (R)c.P.n_ref[1], (R)c.P.n_ref[2]);
    c.launches++;
    return cuda_ok(cudaGetLastError());
}

template <typename S, typename R, typename PhiT, bool DEV> int steps_impl(Ctx &c, int nsteps)
{
    for (int k = 0; k < nsteps; k++) {
        StepArgs<S, R, PhiT> a = make_args<S, R, PhiT>(c);
        BeadArgs<R> ba = make_bead_args<R>(c);
        // 1. bead -> node stencils and bead charge (positions R(t))
        phase_begin(c, PH_BIN);
        if (c.nb > 0) {
            bead_bin_kernel<R><<<1, BEAD_THREADS, 0, c.stream>>>(ba);
            c.launches++;
        }
        phase_end(c, PH_BIN);
        // 2. charge density from the streamed ion densities
        phase_begin(c, PH_CHARGE);
        charge_kernel<S, R, PhiT, DEV><<<c.charge_blocks, CHARGE_THREADS, 0, c.stream>>>(a);
        charge_total_kernel<!(((PhiT)0.5) != 0)>
            <<<CHARGE_TOTAL_BLOCKS, 1024, 0, c.stream>>>(charge_totals_args(c));
        c.launches += 2;
        phase_end(c, PH_CHARGE);
        // 3. Poisson: one cooperative launch for all sweeps (after the learned
        //    warm start, when one is installed)
        if (c.net) {
            phase_begin(c, PH_OTHER);
            int rc = warmstart_before_poisson(c);
            phase_end(c, PH_OTHER);
            if (rc != EKL_OK) return rc;
        }
        phase_begin(c, PH_POISSON);
        cudaMemsetAsync(c.barrier, 0, 4 * sizeof(unsigned), c.stream);
        if (c.mg && c.mg_split) {
            MgArgs m = make_mg_args(c);
            mgs_start_kernel<S, R, PhiT><<<c.pois_blocks, c.mgs_threads, 0, c.stream>>>(a, m, (MgCtl *)c.mgs_ctl);
            c.launches++;
            // the graph with programmatic dependent launches, else without
            if (!c.mgs_exec && mgs_build<PhiT>(c, m, a.g, true) != cudaSuccess) {
                cudaGetLastError();
                if (mgs_build<PhiT>(c, m, a.g, false) != cudaSuccess) return EKL_ERR_CUDA;
            }
            if (cudaGraphLaunch(c.mgs_exec, c.stream) != cudaSuccess) return EKL_ERR_CUDA;
            c.launches += 4;  // the loop's kernels are counted from its iterations
            c.mg_have_prev = 1;
        } else if (c.mg) {
            MgArgs m = make_mg_args(c);
            void *args[] = {&a, &m};
            const void *kern = c.mg_wide ? (const void *)poisson_mg_wide_kernel<S, R, PhiT>
                                         : (const void *)poisson_mg_kernel<S, R, PhiT>;
            static size_t attr_bytes[2] = {0, 0};
            if (c.mg_smem > attr_bytes[c.mg_wide]) {
                cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)c.mg_smem);
                attr_bytes[c.mg_wide] = c.mg_smem;
            }
            cudaError_t e = cudaLaunchCooperativeKernel(kern, dim3(c.pois_blocks),
                                                        dim3(c.mg_wide ? MG_WIDE_THREADS : MG_THREADS), args,
                                                        c.mg_smem, c.stream);
            c.launches++;
            if (e != cudaSuccess) return EKL_ERR_CUDA;
            c.mg_have_prev = 1;
        } else if (c.pois_tiled) {
            TileGeom tg{c.tile_ty, c.tile_tz, c.tile_nty, c.tile_ntz};
            const size_t smem = tile_smem_bytes<PhiT>(c.nx, tg);
            static size_t attr_bytes = 0;
            if (smem > attr_bytes) {
                cudaFuncSetAttribute(poisson_tiled_kernel<S, R, PhiT>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
                attr_bytes = smem;
            }
            void *args[] = {&a, &tg};
            cudaError_t e = cudaLaunchCooperativeKernel((const void *)poisson_tiled_kernel<S, R, PhiT>,
                                                        dim3(c.tile_nty * c.tile_ntz), dim3(POIS_THREADS),
                                                        args, smem, c.stream);
            c.launches++;
            if (e != cudaSuccess) return EKL_ERR_CUDA;
        } else {
            void *args[] = {&a};
            cudaError_t e = cudaLaunchCooperativeKernel((const void *)poisson_kernel<S, R, PhiT>,
                                                        dim3(c.pois_blocks), dim3(POIS_THREADS),
                                                        args, 0, c.stream);
            c.launches++;
            if (e != cudaSuccess) return EKL_ERR_CUDA;
        }
        phase_end(c, PH_POISSON);
        if (c.net) {
            int rc = warmstart_after_poisson(c);
            if (rc != EKL_OK) return rc;
        }
        // 4. beads: interpolate, Langevin sub-steps, spread
        phase_begin(c, PH_MD);
        if (c.nb > 0) {
            MdArgs<S, R, PhiT, DEV> md = make_md_args<S, R, PhiT, DEV>(c, a, ba);
            static bool attr_set = false;
            if (!attr_set) {
                cudaFuncSetAttribute(bead_md_kernel<S, R, PhiT, DEV>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)md_smem_bytes<R>(MAX_BEADS));
                attr_set = true;
            }
            bead_md_kernel<S, R, PhiT, DEV><<<1, MdThreads<R>::value, md_smem_bytes<R>(c.nb), c.stream>>>(md);
            c.launches++;
        }
        phase_end(c, PH_MD);
        // 5. fused pull-collide-stream
        phase_begin(c, PH_LB);
        if (c.P.fluct_mass > 0.0)
            lb_fused_kernel<S, R, PhiT, DEV, true><<<c.lb_blocks, LB_THREADS, 0, c.stream>>>(a);
        else
            lb_fused_kernel<S, R, PhiT, DEV, false><<<c.lb_blocks, LB_THREADS, 0, c.stream>>>(a);
        c.launches++;
        phase_end(c, PH_LB);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return EKL_ERR_CUDA;
        c.cur = 1 - c.cur;
        c.step++;
    }
    return EKL_OK;
}

template <typename S, typename R, typename PhiT, bool DEV>
int fields_impl(Ctx &c, double *d_n, double *d_j, double *d_phi)
{
    StepArgs<S, R, PhiT> a = make_args<S, R, PhiT>(c);
    int blocks = (int)((c.N + 255) / 256);
    fields_kernel<S, R, PhiT, DEV><<<blocks, 256, 0, c.stream>>>(a, d_n, d_j, d_phi);
    c.launches++;
    return cuda_ok(cudaGetLastError());
}

template <typename S, typename R, typename PhiT, bool DEV>
int state_impl(Ctx &c, double *d_f, double *d_phi, int to_host)
{
    StepArgs<S, R, PhiT> a = make_args<S, R, PhiT>(c);
    int blocks = (int)((c.N + 255) / 256);
    state_kernel<S, R, PhiT, DEV><<<blocks, 256, 0, c.stream>>>(a, d_f, d_phi, to_host);
    c.launches++;
    return cuda_ok(cudaGetLastError());
}

// per-block plane-current partials into `part`; returns the block count (< 0 on error)
template <typename S, typename R, typename PhiT, bool DEV> int current_impl(Ctx &c, int axis, int plane, double *part)
{
    StepArgs<S, R, PhiT> a = make_args<S, R, PhiT>(c);
    const int n1 = axis == 0 ? c.ny : c.nx, n2 = axis == 2 ? c.ny : c.nz;
    const int blocks = (n1 * n2 + 255) / 256;
    current_kernel<S, R, PhiT, DEV><<<blocks, 256, 0, c.stream>>>(a, axis, plane, part);
    c.launches++;
    return cudaGetLastError() == cudaSuccess ? blocks : EKL_ERR_CUDA;
}

// per-block mass partials into c.part_mass; returns the block count (< 0 on error)
template <typename S, typename R, typename PhiT, bool DEV> int mass_impl(Ctx &c)
{
    StepArgs<S, R, PhiT> a = make_args<S, R, PhiT>(c);
    const int blocks = (int)((c.N + 255) / 256);
    mass_kernel<S, R, PhiT, DEV><<<blocks, 256, 0, c.stream>>>(a);
    c.launches++;
    return cudaGetLastError() == cudaSuccess ? blocks : EKL_ERR_CUDA;
}

// ------------------------------------------------------------------ batch
static inline int charge_batch_tables(Batch &B)
{
    std::vector<ChargeTotals> t(B.nrep);
    for (int r = 0; r < B.nrep; r++) t[r] = charge_totals_args(*B.reps[r]);
    if (cudaMemcpyAsync(B.d_ctot, t.data(), t.size() * sizeof(ChargeTotals), cudaMemcpyHostToDevice, B.stream) !=
        cudaSuccess)
        return EKL_ERR_CUDA;
    return cudaStreamSynchronize(B.stream) == cudaSuccess ? EKL_OK : EKL_ERR_CUDA;
}

static inline int mg_batch_tables(Batch &B)
{
    std::vector<MgArgs> t(B.nrep);
    std::vector<Grid3> g(B.nrep);
    for (int r = 0; r < B.nrep; r++) {
        t[r] = make_mg_args(*B.reps[r]);
        g[r] = make_grid3(B.reps[r]->nx, B.reps[r]->ny, B.reps[r]->nz);
    }
    if (cudaMemcpyAsync(B.d_mgargs, t.data(), t.size() * sizeof(MgArgs), cudaMemcpyHostToDevice, B.stream) !=
            cudaSuccess ||
        cudaMemcpyAsync(B.d_grids, g.data(), g.size() * sizeof(Grid3), cudaMemcpyHostToDevice, B.stream) !=
            cudaSuccess)
        return EKL_ERR_CUDA;
    return cudaStreamSynchronize(B.stream) == cudaSuccess ? EKL_OK : EKL_ERR_CUDA;
}

template <typename S, typename R, typename PhiT, bool DEV> int batch_tables(Batch &B)
{
    const int n = B.nrep;
    std::vector<StepArgs<S, R, PhiT>> args(n);
    std::vector<BeadArgs<R>> bargs(n);
    std::vector<MdArgs<S, R, PhiT, DEV>> md(n);
    for (int q = 0; q < 2; q++) {
        for (int r = 0; r < n; r++) {
            Ctx &c = *B.reps[r];
            args[r] = make_args<S, R, PhiT>(c, q);
            bargs[r] = make_bead_args<R>(c);
            md[r] = make_md_args<S, R, PhiT, DEV>(c, args[r], bargs[r]);
        }
        if (cudaMemcpyAsync(B.d_args[q], args.data(), n * sizeof(args[0]), cudaMemcpyHostToDevice, B.stream) != cudaSuccess ||
            cudaMemcpyAsync(B.d_bargs[q], bargs.data(), n * sizeof(bargs[0]), cudaMemcpyHostToDevice, B.stream) != cudaSuccess ||
            cudaMemcpyAsync(B.d_mdargs[q], md.data(), n * sizeof(md[0]), cudaMemcpyHostToDevice, B.stream) != cudaSuccess)
            return EKL_ERR_CUDA;
    }
    // Poisson blocks: at least one per replica, the rest in proportion to
    // the replica's (fluid) node count, largest remainders first
    std::vector<double> w(n);
    double W = 0.0;
    for (int r = 0; r < n; r++) {
        w[r] = (double)(B.weight_fluid ? B.reps[r]->n_fluid : B.reps[r]->N);
        W += w[r];
    }
    std::vector<int> k, brep, bloc, lk, lrep, lloc;
    auto share_out = [&](int total, std::vector<int> &k, std::vector<int> &brep, std::vector<int> &bloc) {
        k.assign(n, 1);
        int used = n;
        std::vector<std::pair<double, int>> frac;
        for (int r = 0; r < n; r++) {
            double share = (total - n) * w[r] / W;
            int extra = (int)share;
            k[r] += extra;
            used += extra;
            frac.push_back({share - extra, r});
        }
        std::sort(frac.begin(), frac.end(),
                  [](auto &x, auto &y) { return x.first > y.first || (x.first == y.first && x.second < y.second); });
        for (int t = 0; used < total && t < n; t++, used++) k[frac[t].second]++;
        for (int r = 0; r < n; r++)
            for (int j = 0; j < k[r]; j++) {
                brep.push_back(r);
                bloc.push_back(j);
            }
    };
    share_out(B.pois_blocks, k, brep, bloc);
    B.pois_blocks = (int)brep.size();
    if (cudaMemcpyAsync(B.d_block_rep, brep.data(), brep.size() * 4, cudaMemcpyHostToDevice, B.stream) != cudaSuccess ||
        cudaMemcpyAsync(B.d_block_local, bloc.data(), bloc.size() * 4, cudaMemcpyHostToDevice, B.stream) != cudaSuccess ||
        cudaMemcpyAsync(B.d_rep_blocks, k.data(), n * 4, cudaMemcpyHostToDevice, B.stream) != cudaSuccess)
        return EKL_ERR_CUDA;
    if (B.mg && B.mgs_split) {
        // the split solve's lattice passes: mgs_factor times the blocks
        // (factor 1: the same tables)
        share_out(B.pois_blocks * B.mgs_factor, lk, lrep, lloc);
        B.mgs_lblocks = (int)lrep.size();
        if (cudaMemcpyAsync(B.d_lrep, lrep.data(), lrep.size() * 4, cudaMemcpyHostToDevice, B.stream) != cudaSuccess ||
            cudaMemcpyAsync(B.d_lloc, lloc.data(), lloc.size() * 4, cudaMemcpyHostToDevice, B.stream) != cudaSuccess ||
            cudaMemcpyAsync(B.d_lrb, lk.data(), n * 4, cudaMemcpyHostToDevice, B.stream) != cudaSuccess)
            return EKL_ERR_CUDA;
        // the coarse launch: with the finer lattice tables, two 512-thread
        // blocks per SM when both are resident (its block-wide sums then run
        // over 512 threads; factor 1 keeps the cooperative solve's blocks and
        // results)
        int occ = 0;
        if (B.mg_smem > 48 * 1024)
            cudaFuncSetAttribute(mgsb_coarse_kernel<S, R, PhiT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)B.mg_smem);
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, mgsb_coarse_kernel<S, R, PhiT>, MGS_THREADS / 2,
                                                          B.mg_smem) != cudaSuccess)
            occ = 0;
        cudaGetLastError();
        const int per_sm = (B.mgs_factor > 1 && occ >= 2) ? 2 : 1;
        B.mgs_cthreads = MGS_THREADS / per_sm;
        std::vector<int> ck, crep, cloc;
        share_out(B.pois_blocks * per_sm, ck, crep, cloc);
        B.mgs_cgrid = (int)crep.size();
        if (cudaMemcpyAsync(B.d_crep, crep.data(), crep.size() * 4, cudaMemcpyHostToDevice, B.stream) != cudaSuccess ||
            cudaMemcpyAsync(B.d_cloc, cloc.data(), cloc.size() * 4, cudaMemcpyHostToDevice, B.stream) != cudaSuccess ||
            cudaMemcpyAsync(B.d_crb, ck.data(), n * 4, cudaMemcpyHostToDevice, B.stream) != cudaSuccess)
            return EKL_ERR_CUDA;
    }
    if (cudaStreamSynchronize(B.stream) != cudaSuccess) return EKL_ERR_CUDA;
    if (charge_batch_tables(B) != EKL_OK) return EKL_ERR_CUDA;
    if (B.mg && mg_batch_tables(B) != EKL_OK) return EKL_ERR_CUDA;
    B.max_nb = 0;
    B.fluct = 0;
    for (int r = 0; r < n; r++)
        if (B.reps[r]->P.fluct_mass > 0.0) B.fluct = 1;
    B.max_lb_blocks = B.max_charge_blocks = 0;
    for (int r = 0; r < n; r++) {
        B.max_nb = std::max(B.max_nb, B.reps[r]->nb);
        B.max_lb_blocks = std::max(B.max_lb_blocks, B.reps[r]->lb_blocks);
        B.max_charge_blocks = std::max(B.max_charge_blocks, B.reps[r]->charge_blocks);
    }
    B.ready = 1;
    return EKL_OK;
}

// Graph of the batched split solve (ekl_mgs.cuh), launched after the step's
// start kernel: true residuals -> init -> loop condition -> WHILE (any
// replica not done) { the passes of one CG iteration over every replica,
// a replica that is done skipping them; loop condition } -> final true
// residuals -> report.  The descriptors it reads (parity 0: the solve does
// not touch the populations) keep their addresses for the batch's life; the
// graph is rebuilt when the Poisson grid changes.
static inline MgsBatch mgsb_args(const Batch &B)
{
    return MgsBatch{(const MgArgs *)B.d_mgargs,
                    (const Grid3 *)B.d_grids,
                    (MgCtl *)B.d_ctl,
                    PoisBatch{B.nrep, B.d_lrep, B.d_lloc, B.d_lrb, B.barrier, B.status},
                    PoisBatch{B.nrep, B.d_crep, B.d_cloc, B.d_crb, B.barrier, B.status},
                    B.d_mgs_part,
                    B.mgs_part_stride,
                    B.d_loops};
}

template <typename S, typename R, typename PhiT> static cudaError_t mgsb_build(Batch &B, bool pdl)
{
    const int n = B.nrep, nb = B.mgs_lblocks, ncb = B.mgs_cgrid, nt = MGS_THREADS;
    const StepArgs<S, R, PhiT> *reps = (const StepArgs<S, R, PhiT> *)B.d_args[0];
    MgsBatch mb = mgsb_args(B);
    unsigned *bars = B.mg_bars;
    int when0 = 0, when2 = 2, one = 1;
    cudaGraph_t G = nullptr;
    cudaStream_t cs = nullptr;
    cudaGraphConditionalHandle loop;
    cudaGraphNode_t nres0, ninit, ncond, nloop, nres2, nrep;
    cudaError_t e = cudaGraphCreate(&G, 0);
    auto kernel_node = [&](cudaGraphNode_t *out, cudaGraphNode_t *dep, const void *fn, int grid, int block,
                           void **args) {
        cudaKernelNodeParams kp = {};
        kp.func = (void *)fn;
        kp.gridDim = dim3(grid);
        kp.blockDim = dim3(block);
        kp.kernelParams = args;
        return cudaGraphAddKernelNode(out, G, dep, dep ? 1 : 0, &kp);
    };
    if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&loop, G, 0, cudaGraphCondAssignDefault);
    if (e == cudaSuccess) {
        void *args[] = {&reps, &mb, &when0};
        e = kernel_node(&nres0, nullptr, (const void *)mgsb_residual_kernel<S, R, PhiT>, nb, nt, args);
    }
    if (e == cudaSuccess) {
        void *args[] = {&reps, &mb};
        e = kernel_node(&ninit, &nres0, (const void *)mgsb_init_kernel<S, R, PhiT>, n, 32, args);
    }
    if (e == cudaSuccess) {
        void *args[] = {&mb, &loop, &one};
        e = kernel_node(&ncond, &ninit, (const void *)mgsb_cond_kernel, 1, 256, args);
    }
    cudaGraph_t body = nullptr;
    if (e == cudaSuccess) {
        cudaGraphNodeParams cp = {};
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = loop;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        e = cudaGraphAddNode(&nloop, G, &ncond, nullptr, 1, &cp);
        if (e == cudaSuccess) body = cp.conditional.phGraph_out[0];
    }
    if (e == cudaSuccess && B.mg_smem > 48 * 1024)
        e = cudaFuncSetAttribute(mgsb_coarse_kernel<S, R, PhiT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)B.mg_smem);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
    if (e == cudaSuccess) {
        cudaLaunchAttribute dep[1];
        dep[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        dep[0].val.programmaticStreamSerializationAllowed = 1;
        cudaError_t el = cudaSuccess;
        auto go = [&](bool overlap, unsigned grid, unsigned block, auto kern, auto... args) {
            cudaLaunchConfig_t lc = {};
            lc.gridDim = dim3(grid);
            lc.blockDim = dim3(block);
            lc.stream = cs;
            lc.attrs = dep;
            lc.numAttrs = (overlap && pdl) ? 1 : 0;
            const cudaError_t r = cudaLaunchKernelEx(&lc, kern, args...);
            if (el == cudaSuccess) el = r;
        };
        for (int s = 1; s < 2 * MG_NU; s++) go(s > 1, nb, nt, mgsb_half_kernel<false, false>, mb, s & 1);
        go(true, nb, nt, mgsb_restrict_kernel, mb);
        cudaMemsetAsync(bars, 0, 4 * sizeof(unsigned) * (size_t)n, cs);
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute coop[1];
        coop[0].id = cudaLaunchAttributeCooperative;
        coop[0].val.cooperative = 1;
        cfg.gridDim = dim3(ncb);
        cfg.blockDim = dim3(B.mgs_cthreads);
        cfg.dynamicSmemBytes = B.mg_smem;
        cfg.stream = cs;
        cfg.attrs = coop;
        cfg.numAttrs = 1;
        const cudaError_t ecoop = cudaLaunchKernelEx(&cfg, mgsb_coarse_kernel<S, R, PhiT>, reps, mb, bars);
        if (el == cudaSuccess) el = ecoop;
        go(false, nb, nt, mgsb_half_kernel<false, true>, mb, 1);
        for (int s = 1; s < 2 * MG_NU; s++) {
            const int col = (s & 1) ^ 1;
            if (s == 2 * MG_NU - 1) go(true, nb, nt, mgsb_half_kernel<true, false>, mb, col);
            else go(true, nb, nt, mgsb_half_kernel<false, false>, mb, col);
        }
        go(true, nb, nt, mgsb_pq_kernel, mb);
        go(true, nb, nt, mgsb_update_kernel<S, R, PhiT>, reps, mb);
        go(true, n, 32, mgsb_mid_kernel, mb);
        go(true, nb, nt, mgsb_residual_kernel<S, R, PhiT>, reps, mb, 1);
        go(true, n, 32, mgsb_end_kernel<S, R, PhiT>, reps, mb);
        go(true, 1, 256, mgsb_cond_kernel, mb, loop, 1);
        cudaError_t ek = cudaGetLastError();
        cudaError_t ec = cudaStreamEndCapture(cs, &body);
        e = el != cudaSuccess ? el : ek != cudaSuccess ? ek : ec;
    }
    if (cs) cudaStreamDestroy(cs);
    if (e == cudaSuccess) {
        void *args[] = {&reps, &mb, &when2};
        e = kernel_node(&nres2, &nloop, (const void *)mgsb_residual_kernel<S, R, PhiT>, nb, nt, args);
    }
    if (e == cudaSuccess) {
        void *args[] = {&reps, &mb};
        e = kernel_node(&nrep, &nres2, (const void *)mgsb_report_kernel<S, R, PhiT>, n, 32, args);
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&B.mgs_exec, G, 0);
    if (e != cudaSuccess) {
        if (G) cudaGraphDestroy(G);
        B.mgs_exec = nullptr;
        return e;
    }
    B.mgs_graph = G;
    B.mgs_blocks = nb;
    B.mgs_cblocks = ncb;
    // half sweeps, restriction, coarse, p/q, update, mid, residual, end, condition
    B.mgs_iter_kernels = 2 * (2 * MG_NU - 1) + 1 + 1 + 1 + 6;
    return cudaSuccess;
}

template <typename S, typename R, typename PhiT, bool DEV> int batch_impl(Batch &B, int nsteps)
{
    if (!B.ready) {
        int rc = batch_tables<S, R, PhiT, DEV>(B);
        if (rc != EKL_OK) return rc;
    }
    const int n = B.nrep;
    for (int k = 0; k < nsteps; k++) {
        const int q = B.reps[0]->cur;
        const long long step = B.reps[0]->step;
        if (B.max_nb > 0) {
            bead_bin_batch_kernel<R><<<dim3(1, n), BEAD_THREADS, 0, B.stream>>>((const BeadArgs<R> *)B.d_bargs[q]);
            B.launches++;
        }
        charge_batch_kernel<S, R, PhiT, DEV><<<dim3(B.max_charge_blocks, n), CHARGE_THREADS, 0, B.stream>>>(
            (const StepArgs<S, R, PhiT> *)B.d_args[q]);
        charge_total_batch_kernel<!(((PhiT)0.5) != 0)>
            <<<dim3(CHARGE_TOTAL_BLOCKS, n), 1024, 0, B.stream>>>((const ChargeTotals *)B.d_ctot);
        B.launches += 2;
        cudaMemsetAsync(B.barrier, 0, 4 * sizeof(unsigned), B.stream);
        if (B.mg) {
            cudaMemsetAsync(B.mg_bars, 0, 4 * sizeof(unsigned) * (size_t)n, B.stream);
            PoisBatch pb{n, B.d_block_rep, B.d_block_local, B.d_rep_blocks, B.barrier, B.status};
            const StepArgs<S, R, PhiT> *reps = (const StepArgs<S, R, PhiT> *)B.d_args[q];
            const MgArgs *mgs = (const MgArgs *)B.d_mgargs;
            unsigned *bars = B.mg_bars;
            static size_t attr_bytes = 0;
            if (B.mg_smem > attr_bytes) {
                cudaFuncSetAttribute(poisson_mg_batch_kernel<S, R, PhiT>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)B.mg_smem);
                attr_bytes = B.mg_smem;
            }
            if (B.mgs_split) {
                static_assert(MGS_THREADS == MG_BATCH_THREADS, "split and cooperative batch solves share the grid");
                if (B.mgs_exec && (B.mgs_blocks != B.mgs_lblocks || B.mgs_cblocks != B.mgs_cgrid)) {
                    cudaGraphExecDestroy(B.mgs_exec);
                    cudaGraphDestroy(B.mgs_graph);
                    B.mgs_exec = nullptr;
                    B.mgs_graph = nullptr;
                }
                // the graph with programmatic dependent launches, else without
                if (!B.mgs_exec && mgsb_build<S, R, PhiT>(B, true) != cudaSuccess) {
                    cudaGetLastError();
                    if (mgsb_build<S, R, PhiT>(B, false) != cudaSuccess) return EKL_ERR_CUDA;
                }
                mgsb_start_kernel<S, R, PhiT><<<B.mgs_lblocks, MGS_THREADS, 0, B.stream>>>(reps, mgsb_args(B));
                if (cudaGraphLaunch(B.mgs_exec, B.stream) != cudaSuccess) return EKL_ERR_CUDA;
                B.launches += 6;  // start, residual, init, condition, final residual, report
            } else {
                void *args[] = {&reps, &mgs, &pb, &bars};
                cudaError_t e = cudaLaunchCooperativeKernel((const void *)poisson_mg_batch_kernel<S, R, PhiT>,
                                                            dim3(B.pois_blocks), dim3(MG_BATCH_THREADS), args,
                                                            B.mg_smem, B.stream);
                B.launches++;
                if (e != cudaSuccess) return EKL_ERR_CUDA;
            }
            // from now on every replica extrapolates its starting guess
            bool changed = false;
            for (int r = 0; r < n; r++)
                if (!B.reps[r]->mg_have_prev) {
                    B.reps[r]->mg_have_prev = 1;
                    changed = true;
                }
            if (changed && mg_batch_tables(B) != EKL_OK) return EKL_ERR_CUDA;
        } else {
            PoisBatch pb{n, B.d_block_rep, B.d_block_local, B.d_rep_blocks, B.barrier, B.status};
            const StepArgs<S, R, PhiT> *reps = (const StepArgs<S, R, PhiT> *)B.d_args[q];
            void *args[] = {&reps, &pb};
            cudaError_t e = cudaLaunchCooperativeKernel((const void *)poisson_batch_kernel<S, R, PhiT>,
                                                        dim3(B.pois_blocks), dim3(B.pois_threads), args, 0, B.stream);
            B.launches++;
            if (e != cudaSuccess) return EKL_ERR_CUDA;
        }
        if (B.max_nb > 0) {
            static size_t attr = 0;
            const size_t smem = md_smem_bytes<R>(B.max_nb);
            if (smem > attr) {
                cudaFuncSetAttribute(bead_md_batch_kernel<S, R, PhiT, DEV>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)md_smem_bytes<R>(MAX_BEADS));
                attr = md_smem_bytes<R>(MAX_BEADS);
            }
            bead_md_batch_kernel<S, R, PhiT, DEV><<<dim3(1, n), MdThreads<R>::value, smem, B.stream>>>(
                (const MdArgs<S, R, PhiT, DEV> *)B.d_mdargs[q], step);
            B.launches++;
        }
        if (B.fluct)
            lb_fused_batch_kernel<S, R, PhiT, DEV, true><<<dim3(B.max_lb_blocks, n), LB_THREADS, 0, B.stream>>>(
                (const StepArgs<S, R, PhiT> *)B.d_args[q], step);
        else
            lb_fused_batch_kernel<S, R, PhiT, DEV, false><<<dim3(B.max_lb_blocks, n), LB_THREADS, 0, B.stream>>>(
                (const StepArgs<S, R, PhiT> *)B.d_args[q], step);
        B.launches++;
        if (cudaGetLastError() != cudaSuccess) return EKL_ERR_CUDA;
        for (int r = 0; r < n; r++) {
            B.reps[r]->cur ^= 1;
            B.reps[r]->step++;
        }
    }
    return EKL_OK;
}

// occupancy of the cooperative Poisson kernel for this instantiation
template <typename S, typename R, typename PhiT> int mg_max_blocks_per_sm(size_t smem, int wide)
{
    const void *kern = wide ? (const void *)poisson_mg_wide_kernel<S, R, PhiT>
                            : (const void *)poisson_mg_kernel<S, R, PhiT>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return 0;
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, wide ? MG_WIDE_THREADS : MG_THREADS, smem);
    return nb;
}

template <typename S, typename R, typename PhiT> int mg_batch_max_blocks_per_sm(size_t smem)
{
    if (cudaFuncSetAttribute(poisson_mg_batch_kernel<S, R, PhiT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) != cudaSuccess)
        return 0;
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, poisson_mg_batch_kernel<S, R, PhiT>, MG_BATCH_THREADS, smem);
    return nb;
}

template <typename S, typename R, typename PhiT> int poisson_max_blocks_per_sm()
{
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, poisson_kernel<S, R, PhiT>, POIS_THREADS, 0);
    return nb;
}

}  // namespace ekl

#define EKL_INSTANTIATE(SUFFIX, S, R, PhiT, DEV)                                                   \
    namespace ekl {                                                                              \
    int init_populations_##SUFFIX(Ctx &c, const double *d) { return init_impl<S, R, PhiT, DEV>(c, d); } \
    int run_steps_##SUFFIX(Ctx &c, int n) { return steps_impl<S, R, PhiT, DEV>(c, n); }           \
    int get_fields_##SUFFIX(Ctx &c, double *n, double *j, double *p)                             \
    {                                                                                            \
        return fields_impl<S, R, PhiT, DEV>(c, n, j, p);                                         \
    }                                                                                            \
    int get_state_##SUFFIX(Ctx &c, double *f, double *p) { return state_impl<S, R, PhiT, DEV>(c, f, p, 1); } \
    int set_state_##SUFFIX(Ctx &c, const double *f, const double *p)                             \
    {                                                                                            \
        return state_impl<S, R, PhiT, DEV>(c, (double *)f, (double *)p, 0);                      \
    }                                                                                            \
    int pois_blocks_##SUFFIX() { return poisson_max_blocks_per_sm<S, R, PhiT>(); }                \
    int mass_##SUFFIX(Ctx &c) { return mass_impl<S, R, PhiT, DEV>(c); }                           \
    int current_##SUFFIX(Ctx &c, int ax, int pl, double *p) { return current_impl<S, R, PhiT, DEV>(c, ax, pl, p); } \
    int mg_blocks_##SUFFIX(size_t smem, int wide) { return mg_max_blocks_per_sm<S, R, PhiT>(smem, wide); } \
    int mg_batch_blocks_##SUFFIX(size_t smem) { return mg_batch_max_blocks_per_sm<S, R, PhiT>(smem); } \
    int run_batch_##SUFFIX(Batch &b, int n) { return batch_impl<S, R, PhiT, DEV>(b, n); }         \
    }
