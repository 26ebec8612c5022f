// Host-side state of one simulation handle (internal to the library).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/ekl.h"

namespace ekl {

constexpr int Q = 19;
constexpr int NS = 3;
constexpr int MAX_BEADS = 256;
constexpr int MAX_ENTRIES = 8 * MAX_BEADS;
constexpr int LB_THREADS = 128;
constexpr int CHARGE_THREADS = 256;
constexpr int POIS_THREADS = 1024;
constexpr int MG_THREADS = 512;     // multigrid launch: one block per SM (latency-bound solve)
constexpr int MG_WIDE_THREADS = 1024;  // the same for lattices of at least MG_WIDE_NODES_PER_SM nodes per SM
constexpr int MG_WIDE_NODES_PER_SM = 16384;
constexpr int MG_BATCH_THREADS = 1024;  // batched multigrid: each block sweeps large replica volumes
constexpr int BEAD_THREADS = 256;
// fixed-point scale of the potential in the reduced-precision paths: 2^40
constexpr double PHI_SCALE = 1099511627776.0;
constexpr double PHI_INV = 1.0 / 1099511627776.0;

// status bits written by kernels (mapped to return codes on the host)
constexpr int ST_NOCONV = 1;
constexpr int ST_CFL = 2;
constexpr int ST_UNSTABLE = 4;
constexpr int ST_BEAD = 8;
constexpr int ST_TIMEOUT = 16;

// Multigrid hierarchy of the Poisson operator (levels >= 1; level 0 is the
// lattice itself).  Cell (X, Y, Z) of level l+1 aggregates the cells
// (2X + {0,1}, 2Y + {0,1}, 2Z + {0,1}) of level l.
constexpr int MG_MAXLEV = 12;
constexpr int MG_NU = 2;                 // red-black smoothing sweeps on the lattice before and after the coarse correction
constexpr int MG_NU_COARSE = 2;          // the same on the coarse levels
constexpr int MG_COARSE_SWEEPS = 8;      // (R B)^k R half sweeps on the coarsest level
constexpr float MG_INNER_RED = 1e-6f;    // CG residual reduction before the true residual is formed (1e-4: 3 % slower per step)
constexpr int MG_COARSEST_CELLS = 1024;  // stop coarsening at or below this many cells
constexpr int MG_COARSEST_CELLS_REPLICA = 512;  // the same for the replicas of a batch
constexpr int MG_DENSE_CELLS = 1024;     // coarsest levels this small are solved exactly (dense pseudo-inverse)
constexpr int MG_CTA_CELLS = 2048;       // levels this small are handled by one block
// Coarse levels with at most this many cells per block of the launch are
// smoothed in shared-memory tiles with redundant halos (one grid barrier per
// smoothing pass instead of one per half sweep); a tile's region (cells plus
// halo) takes at most MG_TILE_BYTES of shared memory.
constexpr int MG_TILE_CELLS_PER_BLOCK = 1024;
constexpr size_t MG_TILE_BYTES = 100 * 1024;
struct MgLevel {
    int nx, ny, nz, N;
    float4 *sig;  // conductances of the +x, +y, +z faces and 1 / diagonal (0: inactive cell)
    float *e;     // correction
    float *f;     // right-hand side (restricted residual)
    float *t;     // pre-smoothed correction of a tiled level (read by its post-smoothing)
};

enum Phase { PH_BIN = 0, PH_CHARGE, PH_POISSON, PH_MD, PH_LB, PH_OTHER, PH_COUNT };

struct Ctx {
    ekl_params P;  // copy; pointer members cleared
    int nx, ny, nz;
    int per[3];
    long long N;
    long long n_fluid;
    int prec;
    cudaStream_t stream;
    int device;
    int num_sms;
    int *batch_ready;  // replica of a batch: its descriptor-table flag, cleared on set-up changes

    // constants (FP64, derived exactly as the paper's formulas state)
    double c4;        // 4 pi l_B
    double wd[NS];    // omega_drag = v_T^2 / D
    double om[NS];    // 1 / tau
    double rJ;        // Jacobi spectral radius of the Chebyshev schedule

    // device buffers
    void *f[2];
    int cur;
    uint32_t *mask;
    void *wall_share;  // Real[N] (wall node's charge per fluid face) or null
    void *src_wall;    // Real[N] (wall charge moved onto fluid nodes) or null
    void *rho;         // Real[N]
    void *b;           // PhiT[N]
    void *phi;         // PhiT[N]
    double *part_charge;  // [charge blocks]
    long long *part_charge_q;  // [charge blocks] fixed-point paths: exact sum of rho * 2^40
    double *charge_tot;        // totals of the two (charge_total_kernel)
    long long *charge_tot_q;
    void *charge_chunks;       // its per-block chunk totals and arrival counter (zeroed)
    double *part_mass;    // [mass blocks][3] (filled on request)
    double *part_pois;    // [poisson blocks][2]
    unsigned *barrier;    // {count, generation, abort}
    int *status;          // device status word
    int *pois_iters;      // last step's sweep count
    long long *pois_total;  // sweeps summed over all steps
    double *pois_res;     // last step's relative residual
    void *omegas;         // Chebyshev relaxation factor per half sweep
    void *wchi;           // Real[19][19] w_p chi_kp of the fluctuating term, or null
    int charge_blocks;
    int lb_blocks;
    int pois_blocks;
    int pois_tiled;          // shared-memory tiled Poisson kernel in use
    int tile_ty, tile_tz, tile_nty, tile_ntz;

    // beads
    int nb;
    void *R, *V, *q;      // Real[nb*3], Real[nb*3], Real[nb]
    int *chain;           // [nb]
    int *patch_count;     // [1]
    uint32_t *patch_bits; // [N/32 + 1] bit per node: in the patch list
    int *patch_node;      // [MAX_ENTRIES]
    void *patch_q;        // Real[MAX_ENTRIES]
    void *patch_f;        // Real[MAX_ENTRIES][9]
    void *patch_mom;      // Real[MAX_ENTRIES][15] scratch: n[3], u[9], grad[3]
    int *entry_slot;      // [MAX_ENTRIES]
    int *sorted_entry;    // [MAX_ENTRIES]
    int *slot_first;      // [MAX_ENTRIES + 1]
    void *entry_w;        // Real[MAX_ENTRIES]

    // multigrid-preconditioned CG Poisson solver (EKL_POISSON_MG)
    int mg;                  // solver in use
    int mg_nlev;             // levels including the lattice
    int mg_cta_from;         // first level handled by one block alone
    int mg_wide;             // launch the solve with MG_WIDE_THREADS-thread blocks
    int mg_tile_from;        // first level smoothed in shared-memory tiles (mg_cta_from: none)
    int mg_tile[MG_MAXLEV][3];  // owned cells per tile of each tiled level
    size_t mg_tile_off;      // offset (floats) of the tile region in the dynamic shared memory
    size_t mg_smem;          // dynamic shared memory of the multigrid launch
    MgLevel mg_lev[MG_MAXLEV];
    float *mg_r, *mg_z, *mg_q, *mg_p[2];  // lattice-level CG vectors
    uint8_t *mg_link;        // per-node link byte of the lattice level (wall bit, closed faces)
    float *mg_dense;         // pseudo-inverse of the coarsest operator, or null
    void *mg_phi_prev;       // potential of the step before the last (starting-guess extrapolation)
    int mg_have_prev;        // mg_phi_prev and phi hold two consecutive potentials
    double *mg_part;         // [8][pois_blocks] reduction partials
    int mg_split;            // the split solve (ekl_mgs.cuh) instead of one cooperative launch
    void *mgs_ctl;           // its scalar state (MgCtl)
    cudaGraph_t mgs_graph;   // its CG loop, built at the first solve
    cudaGraphExec_t mgs_exec;
    int mgs_iter_kernels;    // kernels launched per CG iteration of the loop
    int mgs_l1;              // level 1 grid-wide: smoothed by separate launches in the loop
    int mgs_threads;         // block size of its lattice launches (that of the single launch it matches)

    // learned warm start of the Poisson solve (ekl_net.cu)
    void *net;

    // timing / accounting
    int timing;
    cudaEvent_t ev[2 * PH_COUNT];
    cudaEvent_t *tpool;   // event pairs recorded around phases while timing is on
    int *tphase;
    int tcap, tused;
    double ms_phase[PH_COUNT];
    long long launches;
    long long step;
    int last_status;
};

// deferred phase timing: record now, accumulate after the next synchronisation
void timing_record(Ctx &c, int phase, int begin);
void timing_flush(Ctx &c);

// A batch of independent replicas stepped together (every phase is one
// launch for all replicas).
struct Batch {
    int nrep;
    Ctx **reps;              // replica contexts (owned through their handles)
    void **handles;          // the ekl_handle of each replica
    cudaStream_t stream;
    int prec;
    int ready;               // descriptor tables current
    void *d_args[2], *d_bargs[2], *d_mdargs[2];  // per parity
    int *d_block_rep, *d_block_local, *d_rep_blocks;
    unsigned *barrier;
    int *status;
    int pois_threads, pois_blocks;  // schedule of the batched Poisson launch
    int weight_fluid;        // split Poisson blocks by fluid nodes (1) or all nodes (0)
    int max_lb_blocks, max_charge_blocks, max_nb;
    int fluct;               // some replica has the fluctuating term on
    long long launches;
    // multigrid replicas: one cooperative launch, each replica on its own
    // blocks with its own barrier words
    int mg;
    void *d_mgargs;          // MgArgs per replica
    void *d_ctot;            // ChargeTotals per replica
    unsigned *mg_bars;       // [4 * nrep]
    size_t mg_smem;          // largest replica's shared memory for its coarse levels
    // split form of the batched solve (ekl_mgs.cuh): per-pass launches over
    // all replicas, the CG loop a graph with a conditional WHILE node
    int mgs_split;
    void *d_ctl;             // MgCtl per replica
    void *d_grids;           // Grid3 per replica
    int *d_loops;            // loop iterations run (launch accounting)
    cudaGraph_t mgs_graph;
    cudaGraphExec_t mgs_exec;
    int mgs_blocks, mgs_cblocks;  // lattice and coarse grids the graph was built for
    int mgs_iter_kernels;    // kernels of one loop iteration
    // the lattice passes may split replicas into more blocks than the
    // cooperative coarse launch (mgs_factor times as many; 1: the same
    // blocks, and the same results bit for bit as the cooperative form)
    int mgs_factor;
    int mgs_lblocks;
    int *d_lrep, *d_lloc, *d_lrb;  // block tables of the lattice passes
    // block tables of the cooperative coarse launch: two 512-thread blocks
    // per SM where they fit, so that a replica's coarse levels spread over
    // more SMs (else one 1024-thread block per SM)
    int *d_crep, *d_cloc, *d_crb;
    int mgs_cgrid, mgs_cthreads;
    double *d_mgs_part;      // block partials: per replica MGS_SLOTS x mgs_part_stride
    int mgs_part_stride;
};
constexpr int MGS_MAX_FACTOR = 4;
constexpr int MGS_PART_SLOTS = 5;  // block-partial slots of a split solve (ekl_mgs.cuh)
int run_batch_f64(Batch &b, int nsteps);
int run_batch_f32(Batch &b, int nsteps);
int run_batch_bf16(Batch &b, int nsteps);
int run_batch_fp16(Batch &b, int nsteps);

// learned warm start hooks (ekl_net.cu): before the Poisson launch (inputs,
// network, potential update) and after it (training-crop collection)
int warmstart_before_poisson(Ctx &c);
int warmstart_after_poisson(Ctx &c);
void warmstart_free(Ctx &c);

// Makes a handle's device current for the duration of one C-ABI call and
// restores the caller's device when the call returns, so that every kernel,
// copy and symbol lookup of the call lands on the device the handle's memory
// lives on, whatever device the calling thread had current.  ok() is false
// when that device cannot be made current; the call then fails.
struct DeviceScope {
    int prev = -1;
    bool switched = false;
    bool good = true;
    explicit DeviceScope(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) {
            cudaGetLastError();
            good = false;
            return;
        }
        if (prev == dev) return;
        if (cudaSetDevice(dev) != cudaSuccess) {
            cudaGetLastError();
            good = false;
            return;
        }
        switched = true;
    }
    ~DeviceScope()
    {
        if (switched) cudaSetDevice(prev);
    }
    DeviceScope(const DeviceScope &) = delete;
    DeviceScope &operator=(const DeviceScope &) = delete;
    bool ok() const { return good; }
};

// message returned by ekl_last_error() on this thread
void set_last_error(const char *msg);

// allocation through the installed allocator
void *dev_alloc(Ctx &c, size_t bytes);
void dev_free(Ctx &c, void *p, size_t bytes);

// per-precision entry points (defined in the instantiation units)
int init_populations_f64(Ctx &c, const double *d_n_init);
int run_steps_f64(Ctx &c, int nsteps);
int get_fields_f64(Ctx &c, double *d_n, double *d_j, double *d_phi);
int get_state_f64(Ctx &c, double *d_f, double *d_phi);
int set_state_f64(Ctx &c, const double *d_f, const double *d_phi);
int pois_blocks_f64();
int mass_f64(Ctx &c);
int current_f64(Ctx &c, int axis, int plane, double *part);
int mg_blocks_f64(size_t smem, int wide);
int mg_batch_blocks_f64(size_t smem);

int init_populations_f32(Ctx &c, const double *d_n_init);
int run_steps_f32(Ctx &c, int nsteps);
int get_fields_f32(Ctx &c, double *d_n, double *d_j, double *d_phi);
int get_state_f32(Ctx &c, double *d_f, double *d_phi);
int set_state_f32(Ctx &c, const double *d_f, const double *d_phi);
int pois_blocks_f32();
int mass_f32(Ctx &c);
int current_f32(Ctx &c, int axis, int plane, double *part);
int mg_blocks_f32(size_t smem, int wide);
int mg_batch_blocks_f32(size_t smem);

int init_populations_bf16(Ctx &c, const double *d_n_init);
int run_steps_bf16(Ctx &c, int nsteps);
int get_fields_bf16(Ctx &c, double *d_n, double *d_j, double *d_phi);
int get_state_bf16(Ctx &c, double *d_f, double *d_phi);
int set_state_bf16(Ctx &c, const double *d_f, const double *d_phi);
int pois_blocks_bf16();
int mass_bf16(Ctx &c);
int current_bf16(Ctx &c, int axis, int plane, double *part);
int mg_blocks_bf16(size_t smem, int wide);
int mg_batch_blocks_bf16(size_t smem);

int init_populations_fp16(Ctx &c, const double *d_n_init);
int run_steps_fp16(Ctx &c, int nsteps);
int get_fields_fp16(Ctx &c, double *d_n, double *d_j, double *d_phi);
int get_state_fp16(Ctx &c, double *d_f, double *d_phi);
int set_state_fp16(Ctx &c, const double *d_f, const double *d_phi);
int pois_blocks_fp16();
int mass_fp16(Ctx &c);
int current_fp16(Ctx &c, int axis, int plane, double *part);
int mg_blocks_fp16(size_t smem, int wide);
int mg_batch_blocks_fp16(size_t smem);

size_t real_size(int prec);
size_t store_size(int prec);
size_t phi_size(int prec);

}  // namespace ekl
