// Host orchestration of the step for one (storage, arithmetic, potential)
// combination; included by the instantiation units.
#pragma once
#include <cooperative_groups.h>

#include "ekl_kernels.cuh"

namespace ekl {

template <typename S, typename R, typename PhiT>
static StepArgs<S, R, PhiT> make_args(Ctx &c)
{
    StepArgs<S, R, PhiT> a;
    a.g = Grid3{c.nx, c.ny, c.nz, c.N};
    for (int k = 0; k < 3; k++) a.per[k] = c.per[k];
    a.mask = c.mask;
    a.fin = (const S *)c.f[c.cur];
    a.fout = (S *)c.f[1 - c.cur];
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
    a.patch_node = c.patch_node;
    a.patch_q = (const R *)c.patch_q;
    a.patch_f = (const R *)c.patch_f;
    a.part_charge = c.part_charge;
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
    a.nblocks_charge = c.charge_blocks * (CHARGE_THREADS / 32);  // one partial per warp
    return a;
}

template <typename R> static BeadArgs<R> make_bead_args(Ctx &c)
{
    BeadArgs<R> b;
    b.g = Grid3{c.nx, c.ny, c.nz, c.N};
    for (int k = 0; k < 3; k++) b.per[k] = c.per[k];
    b.mask = c.mask;
    b.nb = c.nb;
    b.Rb = (double *)c.R;
    b.Vb = (R *)c.V;
    b.qb = (const R *)c.q;
    b.chain = c.chain;
    b.patch_count = c.patch_count;
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
    init_kernel<S, R, DEV><<<blocks, 256, 0, c.stream>>>(Grid3{c.nx, c.ny, c.nz, c.N}, c.mask, d_n,
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
        c.launches++;
        phase_end(c, PH_CHARGE);
        // 3. Poisson: one cooperative launch for all sweeps
        phase_begin(c, PH_POISSON);
        cudaMemsetAsync(c.barrier, 0, 4 * sizeof(unsigned), c.stream);
        if (c.pois_tiled) {
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
        // 4. beads: interpolate, Langevin sub-steps, spread
        phase_begin(c, PH_MD);
        if (c.nb > 0) {
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
        lb_fused_kernel<S, R, PhiT, DEV><<<c.lb_blocks, LB_THREADS, 0, c.stream>>>(a);
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

// occupancy of the cooperative Poisson kernel for this instantiation
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
    }
