/*
 * ekl.h -- C ABI of the GB300 electrokinetic lattice-Boltzmann / MD step.
 *
 * The library advances the method of Datar, Fyta, Marini Bettolo Marconi and
 * Melchionna (arXiv:1710.09421): a ternary mixture (solvent, cation, anion)
 * on a D3Q19 lattice (Sec. II.C), the Poisson equation for the potential
 * (Eq. 3), and a bead-spring polyelectrolyte in Langevin dynamics (Sec. II.B)
 * coupled to the fluid by frictional drag through a trilinear interpolation
 * kernel (Sec. II.C, algorithm).  The caller states the problem as the paper
 * does (Sec. II.C: geometry, boundary conditions, temperature and all fluid
 * and molecular parameters are inputs) and drives it with these calls:
 *
 *   ekl_create      -> grid, wall map, surface charge, species, solver knobs
 *   ekl_set_beads   -> bead positions, velocities, charges, chain ids
 *   ekl_step        -> advance n lattice time steps on the GPU
 *   ekl_get_fields  -> densities, currents, potential, bead state to the host
 *   ekl_get_stats   -> FP64 totals, Poisson iterations / residual, status
 *   ekl_destroy
 *
 * Units: lattice units, dx = dt = 1, m = 1, v_T^2 = 1/3, k_B T = m v_T^2 = 1/3
 * (Sec. II.C).  The reduced potential phi = e psi / k_B T solves
 * lap(phi) = -4 pi l_B rho_e with rho_e in proton charges per node (Eqs. 2-3);
 * E_app is in k_B T / (e dx); wall surface charge in e per wall node.
 *
 * Layout: node id = x + nx (y + ny z); host arrays are row-major [nz][ny][nx];
 * species 0 = solvent, 1 = cation, 2 = anion.
 *
 * Ownership: every input array is copied during the call; the caller keeps
 * it.  Output pointers are caller-allocated HOST memory.  Device memory is
 * owned by the handle (allocated with cudaMalloc, or through the allocator
 * installed with ekl_set_allocator).
 *
 * Errors: every call returns EKL_OK (0), a positive warning bit set or a
 * negative error code; ekl_last_error() returns a message for the calling
 * thread.  A failed ekl_create leaves nothing allocated.  A step that fails
 * with EKL_ERR_UNSTABLE / EKL_ERR_BEAD stops the step loop; the populations
 * of the failing step are already written, so the state is the failed one.
 */
#ifndef EKL_H
#define EKL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* return codes */
#define EKL_OK 0
#define EKL_WARN_NOCONV 1      /* Poisson hit poisson_max_iter before the tolerance */
#define EKL_WARN_CFL 2         /* |z grad phi| >= 1 somewhere: the stability bound of Sec. III */
#define EKL_ERR_ARG (-1)       /* bad sizes, odd periodic extent, null required pointer */
#define EKL_ERR_ALLOC (-2)     /* device allocation failed */
#define EKL_ERR_UNSTABLE (-3)  /* non-finite or non-positive species density */
#define EKL_ERR_BEAD (-4)      /* bead inside walls / outside the box / FENE bond broken */
#define EKL_ERR_TIMEOUT (-5)   /* a bounded device-side wait gave up */
#define EKL_ERR_CUDA (-6)      /* a CUDA runtime call failed */

/* storage precision of the populations */
#define EKL_F64 0      /* FP64 populations, FP64 arithmetic (the oracle's arithmetic) */
#define EKL_F32 1      /* FP32 deviations from w_p n_ref, FP32 arithmetic */
#define EKL_BF16DEV 2  /* BF16 deviations, FP32 arithmetic */
#define EKL_FP16DEV 3  /* FP16 deviations, FP32 arithmetic */

/* flags */
#define EKL_EQ_BARYCENTRIC 1   /* f_eq and S use the barycentric velocity (printed Eq. 10) */
#define EKL_GAMMA_LITERAL 2    /* bead drag gamma^a = xi for every species (literal Sec. II.B) */
#define EKL_NO_BEAD_NOISE 4    /* no Langevin noise on the beads */
#define EKL_POISSON_GLOBAL 8   /* no shared-memory tiles: the global-memory SOR kernel, or (with
                                  EKL_POISSON_MG) coarse-level half sweeps one grid-wide phase each */
/* Solve the Poisson equation of each step by conjugate gradients
 * preconditioned with one geometric multigrid V-cycle (2x2x2 aggregation,
 * red-black Gauss-Seidel smoothing) instead of the Chebyshev SOR of
 * Sec. II.C.  Same operator, source and stopping rule ||r||_2 <= tol ||b||_2,
 * with r = b - A phi the true residual of the returned potential (not the
 * residual met during a sweep).  poisson_max_iter and poisson_fixed_iter
 * then count CG iterations, poisson_check_every and rho_jacobi are unused,
 * and ekl_stats.poisson_iters / poisson_sweeps report CG iterations.
 * Coarse levels small enough per block are smoothed in shared-memory tiles
 * with redundant halos (same results, fewer grid-wide barriers) unless
 * EKL_POISSON_GLOBAL is set.  ekl_create fails with EKL_ERR_ARG when no
 * coarser level exists (a periodic extent that is not a multiple of 4). */
#define EKL_POISSON_MG 16
/* With EKL_POISSON_MG: run the solve as one cooperative launch.  By default
 * the solve runs split (every lattice pass its own launch, the CG loop a
 * CUDA graph with a conditional WHILE node, built at the first step); both
 * forms return the same potential bit for bit.  A batch takes the flag of
 * replica 0: split, each launch serves every replica and the loop runs
 * while any replica is iterating; cooperative, one launch per step for all
 * replicas. */
#define EKL_POISSON_MG_SINGLE 32

#define EKL_BOND_FENE 0
#define EKL_BOND_HARMONIC 1

typedef struct ekl_handle ekl_handle;

/* Problem statement (Sec. II.C: "geometry, boundary conditions, temperature,
 * timesteps and all fluid and molecular parameters are given as input").
 * Pointers are host pointers, read during ekl_create only. */
typedef struct ekl_params {
    int32_t nx, ny, nz;           /* lattice extents, each >= 2 */
    int32_t periodic[3];          /* 1 = periodic axis (extent must be even: red-black) */
    const uint8_t *solid;         /* [nz][ny][nx], 1 = wall node; required */
    const double *surface_charge; /* [nz][ny][nx] e per wall node, or NULL (Sec. II.A) */
    const double *n_init;         /* [3][nz][ny][nx] initial densities, or NULL = n_ref */
    int32_t valence[3];           /* z^a (Sec. II.A); solvent 0 */
    double diffusivity[3];        /* D^a -> omega_drag = v_T^2 / D^a (Eq. 6); <= 0: use D^1 */
    double tau[3];                /* BGK relaxation time per species (Eq. 12: omega = 1/tau) */
    double n_ref[3];              /* reference densities (deviation storage baseline) */
    double body_force[3][3];      /* Phi_ext^a per particle (Eq. 5) */
    double bjerrum;               /* l_B in lattice units */
    double E_app[3];              /* applied field, k_B T / (e dx) */
    double poisson_tol;           /* stop when ||r||_2 <= tol ||b||_2 */
    int32_t poisson_max_iter;     /* cap on red+black sweeps per step */
    int32_t poisson_check_every;  /* test the residual every k sweeps (>= 1) */
    int32_t poisson_fixed_iter;   /* > 0: exactly this many sweeps, no test */
    double rho_jacobi;            /* Jacobi spectral radius for Chebyshev omega; <= 0: box default */
    int32_t md_substeps;          /* MD sub-steps per LB step (Sec. II.B), >= 1 */
    double bead_xi;               /* total bead friction xi (Sec. II.B gamma) */
    double bead_mass;             /* bead mass M */
    int32_t bond_kind;            /* EKL_BOND_FENE or EKL_BOND_HARMONIC (Eq. 9c) */
    double bond_k, bond_r0, bond_l0;           /* spring constant, FENE R0, harmonic rest length */
    double wca_eps, wca_sigma, wall_eps, wall_sigma; /* WCA bead-bead (Eq. 9a), bead-wall */
    uint64_t seed;                /* Philox key of the bead noise */
    double bead_kT;               /* bead thermostat temperature (Eq. 8) */
    int32_t flags;                /* EKL_EQ_BARYCENTRIC | EKL_GAMMA_LITERAL | EKL_NO_BEAD_NOISE */
    int32_t precision;            /* EKL_F64 / EKL_F32 / EKL_BF16DEV / EKL_FP16DEV */
    double fluct_mass;            /* thermal mass m of the fluctuating term of Eq. 14 (Landau-Lifshitz
                                     noise on the momentum flux and higher moments,
                                     Delta_p = sqrt(m n omega (2 - omega)) sum_{k>=4} w_p chi_kp N_k,
                                     N_k from Philox keyed by `seed`); 0 = no fluctuations */
} ekl_params;

typedef struct ekl_stats {
    double mass[3];          /* FP64 per-species total of the last step's densities */
    int64_t step;            /* completed steps */
    int32_t poisson_iters;   /* sweeps of the last step */
    int32_t status;          /* accumulated warning bits of the last ekl_step */
    double poisson_res;      /* ||r|| / ||b|| of the last step */
    double ms_phase[6];      /* per-phase GPU time (ms) accumulated while timing is on:
                                bead bin, charge, Poisson, bead MD, LB, other */
    int64_t launches;        /* kernels launched by the library since creation */
    int64_t poisson_sweeps;  /* red+black sweeps summed over every step since creation */
} ekl_stats;

/* Optional device allocator (e.g. a framework's caching allocator).  Must be
 * installed before ekl_create; NULL restores cudaMalloc/cudaFree.  `stream`
 * is the handle's stream as a cudaStream_t. */
typedef void *(*ekl_alloc_fn)(size_t bytes, void *stream, void *ctx);
typedef void (*ekl_free_fn)(void *ptr, size_t bytes, void *stream, void *ctx);
int ekl_set_allocator(ekl_alloc_fn alloc, ekl_free_fn free_fn, void *ctx);

/* Create a simulation on the current CUDA device.  `stream` is a
 * cudaStream_t (NULL = the legacy default stream) on which every later call
 * of this handle is ordered.  Builds the wall link table, the wall-charge
 * source, and the initial populations w_p n_init (placed as the
 * post-collision state of step -1).  Errors: EKL_ERR_ARG, EKL_ERR_ALLOC,
 * EKL_ERR_CUDA; *out is NULL on error. */
int ekl_create(const ekl_params *params, void *stream, ekl_handle **out);

/* Replace the beads (Sec. II.B): positions R[n][3], velocities V[n][3] (NULL =
 * zero), charges q[n] (e), chain ids chain[n] (NULL = one chain; consecutive
 * beads with equal ids are bonded).  n <= 1024.  Errors: EKL_ERR_ARG. */
int ekl_set_beads(ekl_handle *h, int32_t n, const double *R, const double *V,
                  const double *q, const int32_t *chain);

/* Advance nsteps time steps (Sec. II.C algorithm): charge density, Poisson,
 * bead interpolation + MD + spreading, fused pull-collide-stream.  Work is
 * queued on the handle's stream; the call synchronises once at the end to
 * read the status word.  Returns EKL_OK, warning bits, or an error. */
int ekl_step(ekl_handle *h, int32_t nsteps);

/* Queue nsteps steps without synchronising (status is read by the next
 * ekl_step / ekl_get_stats). */
int ekl_step_async(ekl_handle *h, int32_t nsteps);

/* Copy fields to host memory (any pointer may be NULL).  Arrays of 8 MB and
 * more move through two 64 MB pinned staging buffers that the library
 * allocates at the first such transfer and keeps for the life of the
 * process (the same for ekl_create's initial densities and for
 * ekl_get_state / ekl_set_state); without pinned memory they are plain
 * copies.
 *   n_out[3][N]     species densities n^a of the current populations (Eq. 15)
 *   j_out[3][3][N]  bare currents sum_p c_p f_p (Eq. 16)
 *   phi_out[N]      potential of the last step, fluid mean removed, 0 on walls
 *   R_out, V_out    bead positions / velocities [nb][3] */
int ekl_get_fields(ekl_handle *h, double *n_out, double *j_out, double *phi_out,
                   double *R_out, double *V_out);

/* Self-test of the library's bounded device-side wait (no counterpart in
 * the paper): one block waits at a grid barrier that another block never
 * reaches; the wait gives up after about 2 s and raises the timeout status,
 * as every spin in the library's kernels does.  Returns EKL_ERR_TIMEOUT when
 * the bound works (the expected result), EKL_ERR_CUDA on a CUDA error. */
int ekl_selftest_wait(void);

/* Replace the applied field E_app (k_B T / (e dx)) from the next step on,
 * e.g. to relax a chain at zero field before driving it (Sec. IV.A).
 * Errors: EKL_ERR_ARG (null or non-finite). */
int ekl_set_field(ekl_handle *h, const double E[3]);

/* Flux of each species through the lattice plane {coordinate `axis` ==
 * `plane`} (axis 0/1/2 = x/y/z): out[s] = sum over the plane's fluid nodes of
 * the current component sum_p c_p,axis f^s_p of the streamed populations
 * (Eq. 16, the populations the next step starts from); out[3] = sum_s z^s
 * out[s], the ionic current in e per time step (the conductance observable
 * of Sec. IV.B: G = out[3] / potential difference).  Errors: EKL_ERR_ARG. */
int ekl_get_current(ekl_handle *h, int32_t axis, int32_t plane, double out[4]);

/* Checkpoint: post-collision populations as FP64 f values [3][19][N] and the
 * raw potential [N] (no gauge shift), plus the step counter. */
int ekl_get_state(ekl_handle *h, double *fstar, double *phi, int64_t *step);
int ekl_set_state(ekl_handle *h, const double *fstar, const double *phi, int64_t step);

int ekl_get_stats(ekl_handle *h, ekl_stats *out);

/* Per-phase CUDA-event timing of later steps (adds one event pair per phase). */
int ekl_set_timing(ekl_handle *h, int32_t on);

/* Link table as built on the device: bit p (1..18) set when x - c_p is a wall
 * node or lies beyond a closed face, bit 31 on wall nodes. mask_out[N]. */
int ekl_get_link_mask(ekl_handle *h, uint32_t *mask_out);

/* Lattice table of the library: c[19][3], w[19], opp[19] (host memory). */
void ekl_lattice(int32_t *c, double *w, int32_t *opp);

void ekl_destroy(ekl_handle *h);

/* Every call that takes a handle runs with the handle's device (the device
 * that was current at ekl_create) made current, and restores the caller's
 * device before it returns; a call whose handle device cannot be made
 * current fails with EKL_ERR_ARG and queues no work.
 * Test support (no counterpart in the paper): record `device` as the
 * handle's device without moving anything, so that a one-GPU test can check
 * that refusal.  Not for use by programs. */
int ekl_test_set_device(ekl_handle *h, int32_t device);

/* Message of the last error on this thread ("" if none). */
const char *ekl_last_error(void);

int64_t ekl_sizeof_params(void);

/* ---------------------------------------------------------------------------
 * Batched replicas.  Many independent simulations of uneven size (e.g.
 * translocation events with different boxes, pores, chains and seeds; the
 * paper runs 100 such events, Sec. IV.A) stepped together: each phase of
 * the step is one launch for all replicas, the Poisson solve one persistent
 * cooperative launch whose blocks are shared out among the replicas (each
 * with its own schedule, tolerance and convergence).  With EKL_POISSON_MG
 * (every replica or none) each replica runs its multigrid-CG solve on its own
 * blocks with its own barrier, at its own pace, and its hierarchy goes one
 * level deeper (coarsest level <= 512 cells, solved exactly).  All replicas
 * share the precision of params[0] and the stream.  Replicas are ordinary
 * handles (ekl_batch_replica) for set-up and read-back, but must only be
 * advanced through ekl_batch_step; ekl_set_field on a replica takes effect
 * from the next ekl_batch_step. */
typedef struct ekl_batch ekl_batch;

/* nrep parameter blocks (params[r]); errors as ekl_create, plus
 * EKL_ERR_ARG when nrep exceeds the number of co-resident Poisson blocks. */
int ekl_batch_create(int32_t nrep, const ekl_params *params, void *stream, ekl_batch **out);
/* the same call under the name the batch interface is also known by */
int ekl_create_batch(int32_t nrep, const ekl_params *params, void *stream, ekl_batch **out);

/* beads of replica rep, as ekl_set_beads */
int ekl_batch_set_beads(ekl_batch *b, int32_t rep, int32_t n, const double *R, const double *V,
                        const double *q, const int32_t *chain);

/* advance every replica by nsteps; returns the OR of warning bits, or the
 * first error of any replica */
int ekl_batch_step(ekl_batch *b, int32_t nsteps);

/* handle of replica rep (owned by the batch; for get_fields / get_stats) */
ekl_handle *ekl_batch_replica(ekl_batch *b, int32_t rep);

/* Autotuner: time each Poisson schedule (1024-thread blocks one per SM or
 * 512-thread blocks two per SM; blocks shared by all nodes or by fluid
 * nodes) over trial_steps steps of the live batch (the steps are real: the
 * batch advances by trial_steps per schedule tried) and keep the fastest;
 * *choice_out gets its index (bit 0: 512-thread blocks, bit 1: fluid
 * weighting).  A multigrid batch keeps one 1024-thread block per SM for its
 * coarse levels; bit 0 then puts the split solve's lattice passes on four
 * times the blocks and its coarse launch on two 512-thread blocks per SM
 * (not available to the cooperative form). */
int ekl_batch_autotune(ekl_batch *b, int32_t trial_steps, int32_t *choice_out);

/* Set the Poisson schedule the autotuner would pick as `choice` (0..3; bit 1:
 * blocks shared by fluid nodes, else by all nodes; bit 0: SOR on 512-thread
 * blocks two per SM, or for a split multigrid batch its lattice passes on
 * four times as many blocks and its coarse launch on two 512-thread blocks
 * per SM, whose sums then run in another order than the cooperative
 * form's, so the potentials agree to rounding instead of bit for bit).  Takes effect at the next step.  EKL_ERR_ARG for
 * a choice out of range or not available (bit 0 on a cooperative multigrid
 * batch). */
int ekl_batch_set_schedule(ekl_batch *b, int32_t choice);

/* kernels launched by the batch itself since creation (a split multigrid
 * solve launches its loop from the device: this then reads the device's
 * loop count and waits for the batch's stream; -1 on a CUDA error) */
int64_t ekl_batch_launches(ekl_batch *b);

void ekl_batch_destroy(ekl_batch *b);

/* ---------------------------------------------------------------------------
 * Learned warm start of the Poisson solve (not in the paper): a 3D
 * convolutional network, 3^3 kernels, channels 2 -> 16 -> 16 -> 16 -> 1, ReLU
 * between layers, linear output, mapping (change of the Poisson source,
 * previous potential) to the change of the potential.  Parameters are one
 * FP32 vector of EKL_NET_PARAMS values, per layer W[co][ci][k] then b[co],
 * k = (dz+1)*9 + (dy+1)*3 + (dx+1).  Inputs x[2][N] (channel-major), output
 * y[N]; periodic wrap on periodic axes, zeros beyond closed ones.  The two
 * 16 -> 16 layers run as BF16 implicit GEMMs on tensor cores with FP32
 * accumulation.  All pointers are host memory. */
#define EKL_NET_PARAMS 15169
int ekl_net_eval(const int32_t dims[3], const int32_t periodic[3], const float *x, const float *w,
                 float *y);
/* mean squared error over mask (NULL = all nodes) and its gradient [EKL_NET_PARAMS] */
int ekl_net_loss_grad(const int32_t dims[3], const int32_t periodic[3], const float *x,
                      const float *target, const uint8_t *mask, const float *w, double *loss,
                      float *grad);
/* Adam training on nsamples crops (closed boundaries): x[s][2][N], target[s][N],
 * mask[N] selects the nodes whose receptive field lies inside the crop;
 * w is read and written; loss_out[iters] (may be NULL). */
int ekl_net_train(int32_t nsamples, const int32_t dims[3], const float *x, const float *target,
                  const uint8_t *mask, float *w, int32_t iters, int32_t batch, float lr,
                  uint64_t seed, float *loss_out);

/* Install trained parameters w[EKL_NET_PARAMS] as the warm start of every
 * later step's Poisson solve (NULL switches it off): the network reads
 * scales[0] * (b(t) - b(t-1)) and scales[1] * phi(t-1), b = 4 pi l_B
 * (rho - mean), and phi(t-1) + scales[2] * output starts the iteration, which
 * still runs to poisson_tol.  The first step after installation has no b(t-1)
 * and starts from phi(t-1). */
int ekl_set_warmstart(ekl_handle *h, const float *w, const float scales[3]);

/* Run nsteps plain steps and record training samples.  Network on the
 * lattice (level 0): ncrops crops per step, cubes of crop^3 nodes centred near
 * the beads, out[k][3][crop^3] = (b(t) - b(t-1), phi(t-1), phi(t) - phi(t-1)),
 * unscaled; needs beads.  Network on level L >= 1 (ekl_warmstart_level): one
 * sample per step, the whole coarse grid, out[k][3][NL] = (b(t) - b(t-1)
 * summed over each cell, phi(t-1) and phi(t) - phi(t-1) averaged over the
 * cell's fluid nodes), NL = nx ny nz / 8^L; crop is unused.  *n_out samples
 * written. */
int ekl_warmstart_collect(ekl_handle *h, int32_t nsteps, int32_t crop, int32_t ncrops, uint64_t seed,
                          float *out, int64_t *n_out);

/* The level the warm-start network runs on (not in the paper; the error
 * that sets the solver's iteration count is smooth and box-wide, while the
 * network sees 4 cells around each output).  0: the lattice (default).
 * L >= 1 (at most 4): cells of 2^L x 2^L x 2^L nodes, cell (X, Y, Z) covering
 * nodes 2^L (X, Y, Z) + [0, 2^L)^3; the inputs are the change of the Poisson
 * source summed over each cell (times scales[0]) and phi(t-1) averaged over
 * its fluid nodes (times scales[1]); the output times scales[2] is added to
 * the potential of every fluid node of the cell (piecewise-constant
 * prolongation) before the solve, which still runs to poisson_tol.  Every
 * extent must be a multiple of 2^L.  Changing the level discards the
 * installed parameters; install them (ekl_set_warmstart) afterwards.
 * Errors: EKL_ERR_ARG. */
int ekl_warmstart_level(ekl_handle *h, int32_t level);

/* Tensor-core path of the two 16 -> 16 layers (no counterpart in the paper):
 * 1 = tcgen05.mma implicit GEMM, 128 nodes per block, FP32 accumulator in
 * tensor memory (default); 0 = the warp-level mma.sync form; other values
 * leave it unchanged.  Returns the previous path.  Process-wide; the network
 * calls return EKL_ERR_TIMEOUT if a block gave up waiting for its MMAs. */
int ekl_net_tensor_path(int32_t path);

/* ekl_net_train on a grid whose periodic axes wrap (whole coarse fields of
 * a periodic box); ekl_net_train is this with every axis closed. */
int ekl_net_train_grid(int32_t nsamples, const int32_t dims[3], const int32_t periodic[3], const float *x,
                       const float *target, const uint8_t *mask, float *w, int32_t iters, int32_t batch, float lr,
                       uint64_t seed, float *loss_out);

/* ---------------------------------------------------------------------------
 * Allocation-free field read-back.  The paper has no counterpart: this entry
 * serves callers that may not allocate GPU memory while they run (code
 * running between capture and replay of a CUDA graph on a pool-allocated
 * stream, a real-time loop that reserved all device memory up front, a host
 * framework whose allocator is locked during a solver callback).  It returns
 * the fields of ekl_get_fields bit for bit (both remove phi's fluid mean
 * with the same deterministic device sum), staged
 * through one fixed device array of
 * EKL_NOALLOC_MAX_DOUBLES doubles (16 MiB) that the library reserves on every
 * GPU that loads it, instead of per-call device buffers; it calls no
 * cudaMalloc/cudaFree and no allocator.  A request needing more staging than
 * that (3N + 9N + N + 512 doubles for n_out/j_out/phi_out, 6 per bead for
 * R/V) is
 * rejected with EKL_ERR_ARG.  All calls share the array: calls whose GPU work
 * overlaps race and must be serialised by the caller.  The first call on a
 * device looks up the array's device address (once per device); make it
 * before any stream capture begins.  Output pointers are host memory, as for
 * ekl_get_fields. */
#define EKL_NOALLOC_MAX_DOUBLES 2097152
int ekl_get_fields_noalloc(ekl_handle *h, double *n_out, double *j_out, double *phi_out,
                           double *R_out, double *V_out);

#ifdef __cplusplus
}
#endif

#endif /* EKL_H */
