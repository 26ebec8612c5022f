/*
 * ORACLE -- test infrastructure only.
 *
 * A plain, slow, double-precision CPU restatement of one time step of the
 * electrokinetic lattice-Boltzmann / molecular-dynamics method of Datar,
 * Fyta, Marini Bettolo Marconi and Melchionna, "Electrokinetic Lattice
 * Boltzmann solver coupled to Molecular Dynamics: application to polymer
 * translocation" (arXiv:1710.09421).  It exists to check the CUDA library.
 * Only the test suite, the package smoke check and the CPU-baseline leg of the
 * benchmark may load it; the library never does.  It shares no source with
 * the CUDA path: its lattice table, geometry code, Poisson solver, bead model
 * and random-number generator are written here, on their own.
 *
 * Every array is a full array; every loop is the textbook loop; the step runs
 * in the order of the paper's algorithm sketch (Sec. II.C, Fig. "algo"):
 *   1. stream the post-collision populations (Eq. 11) with halfway
 *      bounce-back at solid nodes;
 *   2. moments n^a, n^a u^a (Eqs. 15-16);
 *   3. charge density (Eq. 2) + wall charge, neutralising mean removed;
 *   4. Poisson equation (Eq. 3) by red-black SOR with Chebyshev acceleration
 *      (Sec. II.C, last paragraph before the algorithm sketch);
 *   5. beads: interpolate the fluid to the beads, Langevin update (Eqs. 7-9),
 *      spread the bead-fluid drag back to the nodes (Sec. II.C, algorithm);
 *   6. collision (Eqs. 10, 12, 13) with the total force of Eq. 5 and the
 *      drag of Eq. 6.
 * The readings taken where the paper is silent or garbled are listed in the
 * repository's design notes and repeated next to the code they affect.
 *
 * Parity status: every function below is pinned by the CPU tests against
 * closed forms, invariants or brute force (lattice identities, Philox
 * known-answer vector, exact mass and momentum bookkeeping, Poiseuille at the
 * exact relaxation time, Nernst-Einstein drift, discrete Poisson solutions,
 * interpolation identities, Boltzmann equilibrium at a charged wall).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define EKO_Q 19
#define EKO_NS 3

#define EKO_OK 0
#define EKO_WARN_NOCONV 1
#define EKO_WARN_CFL 2
#define EKO_ERR_ARG -1
#define EKO_ERR_ALLOC -2
#define EKO_ERR_UNSTABLE -3
#define EKO_ERR_BEAD -4

#define EKO_FLAG_EQ_BARYCENTRIC 1
#define EKO_FLAG_GAMMA_LITERAL 2
#define EKO_FLAG_NO_BEAD_NOISE 4

#define EKO_BOND_FENE 0
#define EKO_BOND_HARMONIC 1

static const double KT = 1.0 / 3.0;   /* k_B T = m v_T^2, m = 1, v_T^2 = 1/3 (Sec. II.C) */
static const double VT2 = 1.0 / 3.0;

/* D3Q19 velocity set (Sec. II.C): one rest velocity, six |c| = 1 and twelve
 * |c| = sqrt(2).  The weights are the standard D3Q19 ones (1/3, 1/18, 1/36);
 * the paper only calls them "Gaussian weights".  Order: rest, +-x, +-y, +-z,
 * then the xy, xz, yz diagonals, each velocity followed by its opposite. */
static const int CV[EKO_Q][3] = {
    {0, 0, 0},
    {1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1},
    {1, 1, 0}, {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0},
    {1, 0, 1}, {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
    {0, 1, 1}, {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};
static double WV[EKO_Q];
static int OPPV[EKO_Q];
/* Moment basis of the fluctuating term (Eq. 14): CHI[k][p], orthonormal in
 * sum_p w_p CHI[k][p] CHI[l][p]; k = 0 density, 1-3 current, 4-9 momentum
 * flux, 10-18 the remaining moments.  Built by Gram-Schmidt, in that
 * scalar product, of the monomials 1, cx, cy, cz, cx^2, cy^2, cz^2, cx cy,
 * cx cz, cy cz, cx^2 cy, cx cy^2, cx^2 cz, cx cz^2, cy^2 cz, cy cz^2,
 * cx^2 cy^2, cx^2 cz^2, cy^2 cz^2 in this order. */
static double CHI[EKO_Q][EKO_Q];
static int lattice_ready = 0;

static double monomial(int k, const int c[3])
{
    const double x = c[0], y = c[1], z = c[2];
    switch (k) {
    case 0: return 1.0;
    case 1: return x;
    case 2: return y;
    case 3: return z;
    case 4: return x * x;
    case 5: return y * y;
    case 6: return z * z;
    case 7: return x * y;
    case 8: return x * z;
    case 9: return y * z;
    case 10: return x * x * y;
    case 11: return x * y * y;
    case 12: return x * x * z;
    case 13: return x * z * z;
    case 14: return y * y * z;
    case 15: return y * z * z;
    case 16: return x * x * y * y;
    case 17: return x * x * z * z;
    default: return y * y * z * z;
    }
}

static void basis_init(void)
{
    for (int k = 0; k < EKO_Q; k++) {
        double v[EKO_Q];
        for (int p = 0; p < EKO_Q; p++) v[p] = monomial(k, CV[p]);
        for (int l = 0; l < k; l++) {
            double d = 0.0;
            for (int p = 0; p < EKO_Q; p++) d += WV[p] * v[p] * CHI[l][p];
            for (int p = 0; p < EKO_Q; p++) v[p] -= d * CHI[l][p];
        }
        double nrm = 0.0;
        for (int p = 0; p < EKO_Q; p++) nrm += WV[p] * v[p] * v[p];
        nrm = sqrt(nrm);
        for (int p = 0; p < EKO_Q; p++) CHI[k][p] = v[p] / nrm;
    }
}

static void lattice_init(void)
{
    if (lattice_ready) return;
    for (int p = 0; p < EKO_Q; p++) {
        int c2 = CV[p][0] * CV[p][0] + CV[p][1] * CV[p][1] + CV[p][2] * CV[p][2];
        WV[p] = c2 == 0 ? 1.0 / 3.0 : (c2 == 1 ? 1.0 / 18.0 : 1.0 / 36.0);
        for (int q = 0; q < EKO_Q; q++)
            if (CV[q][0] == -CV[p][0] && CV[q][1] == -CV[p][1] && CV[q][2] == -CV[p][2])
                OPPV[p] = q;
    }
    basis_init();
    lattice_ready = 1;
}

typedef struct {
    int32_t nx, ny, nz;
    int32_t periodic[3];
    int32_t valence[3];
    double diffusivity[3];
    double tau[3];
    double n_ref[3];
    double body_force[3][3];
    double bjerrum;
    double E_app[3];
    double poisson_tol;
    int32_t poisson_max_iter;
    int32_t poisson_check_every;
    int32_t poisson_fixed_iter;
    double rho_jacobi;
    int32_t md_substeps;
    double bead_xi;
    double bead_mass;
    int32_t bond_kind;
    double bond_k, bond_r0, bond_l0;
    double wca_eps, wca_sigma, wall_eps, wall_sigma;
    uint64_t seed;
    double bead_kT;
    int32_t flags;
    double fluct_mass;   /* thermal mass m of the fluctuating term (Eq. 14); 0 = none */
} eko_params;

typedef struct {
    eko_params P;
    long N;
    uint8_t *solid;
    double *wall_share;   /* per solid node: its charge / number of fluid faces */
    double *src_wall;     /* per fluid node: wall charge moved onto it */
    double *fstar;        /* [3][19][N] post-collision populations (state) */
    double *f;            /* [3][19][N] streamed populations */
    double *n;            /* [3][N] */
    double *j;            /* [3][3][N] */
    double *rho;          /* [N] */
    double *b;            /* [N] Poisson source 4 pi l_B (rho - mean) */
    double *phi;          /* [N] */
    double *grad;         /* [3][N] */
    double *bead_q;       /* [N] bead charge on nodes */
    double *bead_f;       /* [3][3][N] bead force per particle of each species */
    int nb;
    double *R, *V, *q;
    int32_t *chain;
    int64_t step;
    int poisson_iters;
    double poisson_res;
    int status;
    int threads;
} eko_sim;

/* ------------------------------------------------------------------------ */
/* geometry helpers                                                          */
/* ------------------------------------------------------------------------ */

/* Wrap a coordinate along a periodic axis; on a closed axis report whether it
 * lies inside the box. */
static int wrap_coord(int c, int n, int periodic, int *inside)
{
    if (periodic) {
        c %= n;
        if (c < 0) c += n;
        return c;
    }
    if (c < 0 || c >= n) *inside = 0;
    return c;
}

static long node_id(const eko_sim *s, int x, int y, int z, int *inside)
{
    *inside = 1;
    x = wrap_coord(x, s->P.nx, s->P.periodic[0], inside);
    y = wrap_coord(y, s->P.ny, s->P.periodic[1], inside);
    z = wrap_coord(z, s->P.nz, s->P.periodic[2], inside);
    if (!*inside) return -1;
    return x + (long)s->P.nx * (y + (long)s->P.ny * z);
}

/* A node outside a closed box face counts as wall. */
static int fluid_at(const eko_sim *s, int x, int y, int z)
{
    int in;
    long id = node_id(s, x, y, z, &in);
    return in && !s->solid[id];
}

static void coords(const eko_sim *s, long i, int *x, int *y, int *z)
{
    *x = (int)(i % s->P.nx);
    *y = (int)((i / s->P.nx) % s->P.ny);
    *z = (int)(i / ((long)s->P.nx * s->P.ny));
}

static const int FACE[6][3] = {{-1, 0, 0}, {1, 0, 0}, {0, -1, 0}, {0, 1, 0}, {0, 0, -1}, {0, 0, 1}};

/* ------------------------------------------------------------------------ */
/* Philox-4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), written from its       */
/* published definition: ten rounds of two 32x32->64 multiplies, the key      */
/* bumped by the Weyl constants between rounds.                              */
/* ------------------------------------------------------------------------ */
void eko_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int r = 0; r < 10; r++) {
        if (r > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Zero-mean, unit-variance variate from one 32-bit word: sqrt(3)(2U-1) with
 * U = (x + 1/2) / 2^32; every operation before the last multiply is exact. */
static double unit_variate(uint32_t x)
{
    double t = ((double)(2.0 * (double)x + 1.0) - 4294967296.0) * (1.0 / 4294967296.0);
    return 1.7320508075688772 * t;
}

/* ------------------------------------------------------------------------ */
/* creation                                                                  */
/* ------------------------------------------------------------------------ */

static void *xcalloc(size_t n, size_t sz) { return calloc(n ? n : 1, sz); }

void eko_destroy(eko_sim *s)
{
    if (!s) return;
    free(s->solid); free(s->wall_share); free(s->src_wall); free(s->fstar); free(s->f);
    free(s->n); free(s->j); free(s->rho); free(s->b); free(s->phi); free(s->grad);
    free(s->bead_q); free(s->bead_f); free(s->R); free(s->V); free(s->q); free(s->chain);
    free(s);
}

/* Initial state: the post-collision populations of step -1 are the rest
 * equilibrium w_p n^a(x) of the given densities, so that the first step
 * streams them (Sec. II.C: the fluid is initialised, then densities computed). */
eko_sim *eko_create(const eko_params *P, const uint8_t *solid, const double *surface_charge,
                    const double *n_init, int *err)
{
    lattice_init();
    *err = EKO_ERR_ARG;
    if (P->nx < 2 || P->ny < 2 || P->nz < 2) return NULL;
    for (int a = 0; a < 3; a++) {
        int L = a == 0 ? P->nx : (a == 1 ? P->ny : P->nz);
        if (P->periodic[a] && (L % 2)) return NULL;   /* red-black needs even periods */
    }
    eko_sim *s = (eko_sim *)xcalloc(1, sizeof(eko_sim));
    s->P = *P;
    if (s->P.md_substeps < 1) s->P.md_substeps = 1;
    if (s->P.poisson_check_every < 1) s->P.poisson_check_every = 1;
    long N = (long)P->nx * P->ny * P->nz;
    s->N = N;
    s->threads = 1;
    s->solid = (uint8_t *)xcalloc(N, 1);
    s->wall_share = (double *)xcalloc(N, sizeof(double));
    s->src_wall = (double *)xcalloc(N, sizeof(double));
    s->fstar = (double *)xcalloc((size_t)EKO_NS * EKO_Q * N, sizeof(double));
    s->f = (double *)xcalloc((size_t)EKO_NS * EKO_Q * N, sizeof(double));
    s->n = (double *)xcalloc((size_t)EKO_NS * N, sizeof(double));
    s->j = (double *)xcalloc((size_t)EKO_NS * 3 * N, sizeof(double));
    s->rho = (double *)xcalloc(N, sizeof(double));
    s->b = (double *)xcalloc(N, sizeof(double));
    s->phi = (double *)xcalloc(N, sizeof(double));
    s->grad = (double *)xcalloc(3 * (size_t)N, sizeof(double));
    s->bead_q = (double *)xcalloc(N, sizeof(double));
    s->bead_f = (double *)xcalloc((size_t)EKO_NS * 3 * N, sizeof(double));
    if (!s->solid || !s->wall_share || !s->src_wall || !s->fstar || !s->f || !s->n || !s->j ||
        !s->rho || !s->b || !s->phi || !s->grad || !s->bead_q || !s->bead_f) {
        eko_destroy(s);
        *err = EKO_ERR_ALLOC;
        return NULL;
    }
    memcpy(s->solid, solid, (size_t)N);
    /* Wall charge (Sec. II.A, Neumann condition -grad psi . n = Sigma/eps):
     * each charged wall node splits its charge equally over its fluid faces;
     * the share enters the Poisson source of the fluid node across that face
     * and the ghost value used for the field at that node. */
    if (surface_charge) {
        for (long w = 0; w < N; w++) {
            if (!solid[w] || surface_charge[w] == 0.0) continue;
            int x, y, z, k = 0;
            coords(s, w, &x, &y, &z);
            for (int f = 0; f < 6; f++)
                k += fluid_at(s, x + FACE[f][0], y + FACE[f][1], z + FACE[f][2]);
            if (k > 0) s->wall_share[w] = surface_charge[w] / k;
        }
        for (long i = 0; i < N; i++) {
            if (solid[i]) continue;
            int x, y, z;
            coords(s, i, &x, &y, &z);
            double acc = 0.0;
            for (int f = 0; f < 6; f++) {
                int in;
                long w = node_id(s, x + FACE[f][0], y + FACE[f][1], z + FACE[f][2], &in);
                if (in && solid[w]) acc += s->wall_share[w];
            }
            s->src_wall[i] = acc;
        }
    }
    for (int a = 0; a < EKO_NS; a++)
        for (long i = 0; i < N; i++) {
            if (solid[i]) continue;
            double na = n_init ? n_init[(size_t)a * N + i] : P->n_ref[a];
            for (int p = 0; p < EKO_Q; p++) s->fstar[((size_t)a * EKO_Q + p) * N + i] = WV[p] * na;
        }
    *err = EKO_OK;
    return s;
}

void eko_set_threads(eko_sim *s, int t) { s->threads = t < 1 ? 1 : t; }

int eko_set_beads(eko_sim *s, int nb, const double *R, const double *V, const double *q,
                  const int32_t *chain)
{
    free(s->R); free(s->V); free(s->q); free(s->chain);
    s->nb = nb;
    s->R = (double *)xcalloc(3 * (size_t)nb, sizeof(double));
    s->V = (double *)xcalloc(3 * (size_t)nb, sizeof(double));
    s->q = (double *)xcalloc((size_t)nb, sizeof(double));
    s->chain = (int32_t *)xcalloc((size_t)nb, sizeof(int32_t));
    if (nb > 0) {
        memcpy(s->R, R, 3 * sizeof(double) * nb);
        if (V) memcpy(s->V, V, 3 * sizeof(double) * nb);
        memcpy(s->q, q, sizeof(double) * nb);
        if (chain) memcpy(s->chain, chain, sizeof(int32_t) * nb);
    }
    return EKO_OK;
}

/* ------------------------------------------------------------------------ */
/* 1. streaming (Eq. 11) with halfway bounce-back                            */
/* ------------------------------------------------------------------------ */

/* f_p(x, t+1) = f*_p(x - c_p, t); when x - c_p is a wall node the population
 * that left x towards the wall comes back reversed: f_p(x) = f*_{opp p}(x).
 * (The paper leaves the wall rule to the "boundary conditions" input; the
 * halfway bounce-back rule puts a no-slip wall midway between nodes.) */
static void stream(eko_sim *s)
{
    const long N = s->N;
#pragma omp parallel for schedule(static) num_threads(s->threads)
    for (long i = 0; i < N; i++) {
        if (s->solid[i]) continue;
        int x, y, z;
        coords(s, i, &x, &y, &z);
        for (int p = 0; p < EKO_Q; p++) {
            int in;
            long src = node_id(s, x - CV[p][0], y - CV[p][1], z - CV[p][2], &in);
            int wall = !in || s->solid[src];
            for (int a = 0; a < EKO_NS; a++) {
                double v = wall ? s->fstar[((size_t)a * EKO_Q + OPPV[p]) * N + i]
                                : s->fstar[((size_t)a * EKO_Q + p) * N + src];
                s->f[((size_t)a * EKO_Q + p) * N + i] = v;
            }
        }
    }
}

/* 2. moments (Eqs. 15-16): n^a = sum_p f_p, n^a u^a = sum_p c_p f_p */
static void moments(eko_sim *s)
{
    const long N = s->N;
#pragma omp parallel for schedule(static) num_threads(s->threads)
    for (long i = 0; i < N; i++) {
        for (int a = 0; a < EKO_NS; a++) {
            double n = 0.0, jx = 0.0, jy = 0.0, jz = 0.0;
            if (!s->solid[i]) {
                for (int p = 0; p < EKO_Q; p++) {
                    double v = s->f[((size_t)a * EKO_Q + p) * N + i];
                    n += v;
                    jx += CV[p][0] * v;
                    jy += CV[p][1] * v;
                    jz += CV[p][2] * v;
                }
            }
            s->n[(size_t)a * N + i] = n;
            s->j[((size_t)a * 3 + 0) * N + i] = jx;
            s->j[((size_t)a * 3 + 1) * N + i] = jy;
            s->j[((size_t)a * 3 + 2) * N + i] = jz;
        }
    }
}

/* ------------------------------------------------------------------------ */
/* bead <-> node kernel (Sec. II.C: the same interpolation kernel both ways)  */
/* ------------------------------------------------------------------------ */

/* Trilinear weights of the 8 nodes around R, ordered k = ox + 2 oy + 4 oz.
 * Wall nodes get weight zero and the rest are renormalised to sum to one.
 * Returns 0 when every surrounding node is wall. */
int eko_bead_stencil(const eko_sim *s, const double R[3], long nodes[8], double w[8])
{
    int base[3];
    double fr[3];
    for (int a = 0; a < 3; a++) {
        double fl = floor(R[a]);
        base[a] = (int)fl;
        fr[a] = R[a] - fl;
    }
    double W = 0.0;
    for (int k = 0; k < 8; k++) {
        int o[3] = {k & 1, (k >> 1) & 1, (k >> 2) & 1};
        double wk = 1.0;
        for (int a = 0; a < 3; a++) wk *= o[a] ? fr[a] : 1.0 - fr[a];
        int in;
        long id = node_id(s, base[0] + o[0], base[1] + o[1], base[2] + o[2], &in);
        int fl = in && !s->solid[id];
        nodes[k] = in ? id : -1;
        w[k] = fl ? wk : 0.0;
        W += w[k];
    }
    if (!(W > 0.0)) return 0;
    for (int k = 0; k < 8; k++) w[k] = w[k] / W;
    return 1;
}

/* ------------------------------------------------------------------------ */
/* 3. charge density (Eq. 2) and 4. Poisson (Eq. 3)                           */
/* ------------------------------------------------------------------------ */

static int deposit_beads(eko_sim *s)
{
    memset(s->bead_q, 0, sizeof(double) * s->N);
    for (int b = 0; b < s->nb; b++) {
        long nd[8];
        double w[8];
        if (!eko_bead_stencil(s, &s->R[3 * b], nd, w)) return EKO_ERR_BEAD;
        for (int k = 0; k < 8; k++)
            if (w[k] != 0.0) s->bead_q[nd[k]] += s->q[b] * w[k];
    }
    return EKO_OK;
}

static double default_rho_jacobi(const eko_params *P)
{
    /* Jacobi spectral radius of the 7-point Laplacian for the slowest box mode:
     * (2 + cos theta)/3 with theta = 2 pi / L on a periodic axis and pi / L on
     * a closed one, minimised over the three axes. */
    double th = 1e30;
    int L[3] = {P->nx, P->ny, P->nz};
    for (int a = 0; a < 3; a++) {
        double t = (P->periodic[a] ? 2.0 : 1.0) * M_PI / L[a];
        if (t < th) th = t;
    }
    return (2.0 + cos(th)) / 3.0;
}

/* Solve the 7-point finite-volume Poisson equation on the fluid nodes,
 *   sum_{fluid faces j} (phi_j - phi_i) = -4 pi l_B (rho_i - <rho>),
 * walls being zero-flux faces (their charge is already inside rho), by
 * successive over-relaxation in red-black (checkerboard) order with the
 * Chebyshev sequence of relaxation factors:
 *   omega = 1 for the first half sweep, 1/(1 - rJ^2/2) for the second,
 *   1/(1 - rJ^2 omega/4) afterwards
 * (Press et al., Numerical Recipes, Sec. 19.5; Sec. II.C of the paper).
 * The residual of each node is the one computed when it is updated; the
 * iteration stops after a full (red + black) sweep when
 * ||r||_2 <= tol * ||b||_2, tested every `check_every` sweeps, or after
 * exactly `fixed_iter` sweeps when that is positive.  Returns the sweep count
 * (negative when max_iter was reached without convergence). */
int eko_poisson_solve(eko_sim *s, const double *rho, double *phi, double tol, int max_iter,
                      int check_every, int fixed_iter, double *res_out)
{
    const long N = s->N;
    const eko_params *P = &s->P;
    double sum = 0.0;
    long nf = 0;
    for (long i = 0; i < N; i++)
        if (!s->solid[i]) {
            sum += rho[i];
            nf++;
        }
    double mean = nf ? sum / nf : 0.0;
    double bn2 = 0.0;
    for (long i = 0; i < N; i++) {
        s->b[i] = s->solid[i] ? 0.0 : 4.0 * M_PI * P->bjerrum * (rho[i] - mean);
        bn2 += s->b[i] * s->b[i];
    }
    double bnorm = sqrt(bn2);
    double rJ = P->rho_jacobi > 0.0 ? P->rho_jacobi : default_rho_jacobi(P);
    if (check_every < 1) check_every = 1;
    int limit = fixed_iter > 0 ? fixed_iter : max_iter;
    if (fixed_iter <= 0 && bnorm == 0.0) {
        if (res_out) *res_out = 0.0;
        return 0;
    }
    double omega = 1.0;
    int it;
    double r2 = 0.0;
    int converged = 0;
    for (it = 0; it < limit; it++) {
        r2 = 0.0;
        for (int colour = 0; colour < 2; colour++) {
#pragma omp parallel for schedule(static) reduction(+ : r2) num_threads(s->threads)
            for (long i = 0; i < N; i++) {
                if (s->solid[i]) continue;
                int x, y, z;
                coords(s, i, &x, &y, &z);
                if (((x + y + z) & 1) != colour) continue;
                double acc = s->b[i];
                int deg = 0;
                for (int f = 0; f < 6; f++) {
                    int in;
                    long j = node_id(s, x + FACE[f][0], y + FACE[f][1], z + FACE[f][2], &in);
                    if (in && !s->solid[j]) {
                        acc += phi[j];
                        deg++;
                    }
                }
                if (deg == 0) continue;
                double r = acc - deg * phi[i];
                phi[i] = phi[i] + omega * r / deg;
                r2 += r * r;
            }
            if (it == 0 && colour == 0)
                omega = 1.0 / (1.0 - 0.5 * rJ * rJ);
            else
                omega = 1.0 / (1.0 - 0.25 * rJ * rJ * omega);
        }
        if (fixed_iter <= 0 && ((it + 1) % check_every) == 0 && sqrt(r2) <= tol * bnorm) {
            converged = 1;
            it++;
            break;
        }
    }
    if (res_out) *res_out = bnorm > 0.0 ? sqrt(r2) / bnorm : sqrt(r2);
    if (fixed_iter > 0) return fixed_iter;
    return converged ? it : -it;
}

/* Relative residual ||b - A phi||_2 / ||b||_2 of a potential for the charge
 * density rho, with b = 4 pi l_B (rho - <rho>_fluid) on the fluid nodes and
 * (A phi)_i = sum_{fluid faces j} (phi_i - phi_j): the equation that
 * eko_poisson_solve iterates on (Eqs. 2-3), evaluated once, written out
 * directly.  Nodes without a fluid face are left out, as in the solver. */
double eko_poisson_residual(const eko_sim *s, const double *rho, const double *phi)
{
    const long N = s->N;
    double sum = 0.0;
    long nf = 0;
    for (long i = 0; i < N; i++)
        if (!s->solid[i]) {
            sum += rho[i];
            nf++;
        }
    const double mean = nf ? sum / nf : 0.0;
    double r2 = 0.0, b2 = 0.0;
    for (long i = 0; i < N; i++) {
        if (s->solid[i]) continue;
        const double b = 4.0 * M_PI * s->P.bjerrum * (rho[i] - mean);
        b2 += b * b;
        int x, y, z;
        coords(s, i, &x, &y, &z);
        double Aphi = 0.0;
        int deg = 0;
        for (int f = 0; f < 6; f++) {
            int in;
            long j = node_id(s, x + FACE[f][0], y + FACE[f][1], z + FACE[f][2], &in);
            if (in && !s->solid[j]) {
                Aphi += phi[i] - phi[j];
                deg++;
            }
        }
        if (deg == 0) continue;
        r2 += (b - Aphi) * (b - Aphi);
    }
    return b2 > 0.0 ? sqrt(r2 / b2) : sqrt(r2);
}

/* charge density rho_e of the last step (ions, wall charge, beads) */
void eko_last_rho(const eko_sim *s, double *out) { memcpy(out, s->rho, sizeof(double) * s->N); }

/* Field at the fluid nodes by central differences; a wall (or closed-box)
 * neighbour is replaced by the Neumann ghost phi_i + 4 pi l_B sigma_face,
 * sigma_face being the wall node's charge share on that face (Sec. II.A:
 * -grad psi . n = Sigma / eps at insulating walls). */
void eko_node_gradient(const eko_sim *s, const double *phi, double *grad)
{
    const long N = s->N;
    const double c4 = 4.0 * M_PI * s->P.bjerrum;
    for (long i = 0; i < N; i++) {
        for (int a = 0; a < 3; a++) grad[(size_t)a * N + i] = 0.0;
        if (s->solid[i]) continue;
        int x, y, z;
        coords(s, i, &x, &y, &z);
        for (int a = 0; a < 3; a++) {
            double v[2];
            for (int sgn = 0; sgn < 2; sgn++) {
                int f = 2 * a + sgn; /* sgn 0: minus side, 1: plus side */
                int in;
                long j = node_id(s, x + FACE[f][0], y + FACE[f][1], z + FACE[f][2], &in);
                if (in && !s->solid[j])
                    v[sgn] = phi[j];
                else
                    v[sgn] = phi[i] + c4 * (in ? s->wall_share[j] : 0.0);
            }
            grad[(size_t)a * N + i] = (v[1] - v[0]) * 0.5;
        }
    }
}

/* ------------------------------------------------------------------------ */
/* 5. beads (Sec. II.B): forces, Langevin update, bead-fluid drag             */
/* ------------------------------------------------------------------------ */

static void min_image(const eko_sim *s, double d[3])
{
    int L[3] = {s->P.nx, s->P.ny, s->P.nz};
    for (int a = 0; a < 3; a++)
        if (s->P.periodic[a]) d[a] -= L[a] * nearbyint(d[a] / L[a]);
}

/* WCA force on a particle at separation d (vector from partner to particle):
 * u = 4 eps [(sig/r)^12 - (sig/r)^6] + eps for r < 2^(1/6) sig, else 0
 * (Eq. 9a with the garbled second case read as r >= 2^(1/6) sig). */
static void wca_force(double eps, double sig, const double d[3], double F[3])
{
    double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    double rc2 = pow(2.0, 1.0 / 3.0) * sig * sig;
    if (r2 >= rc2) return;
    double sr2 = sig * sig / r2;
    double sr6 = sr2 * sr2 * sr2;
    double mag = 24.0 * eps * (2.0 * sr6 * sr6 - sr6) / r2;
    for (int a = 0; a < 3; a++) F[a] += mag * d[a];
}

/* Conservative forces on every bead: bond (Eq. 9c; FENE as an option), WCA
 * between beads that are not bonded neighbours (Eq. 9a), WCA against wall
 * nodes (not in the paper: it keeps beads out of the walls). */
static int conservative_forces(const eko_sim *s, const double *R, double *F)
{
    const eko_params *P = &s->P;
    int nb = s->nb;
    memset(F, 0, sizeof(double) * 3 * nb);
    for (int b = 0; b + 1 < nb; b++) {
        if (s->chain[b] != s->chain[b + 1]) continue;
        double d[3] = {R[3 * b] - R[3 * (b + 1)], R[3 * b + 1] - R[3 * (b + 1) + 1],
                       R[3 * b + 2] - R[3 * (b + 1) + 2]};
        min_image(s, d);
        double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
        double fac;
        if (P->bond_kind == EKO_BOND_FENE) {
            double x = r2 / (P->bond_r0 * P->bond_r0);
            if (!(x < 1.0)) return EKO_ERR_BEAD;
            fac = -P->bond_k / (1.0 - x);
        } else {
            double r = sqrt(r2);
            fac = -P->bond_k * (r - P->bond_l0) / r;
        }
        for (int a = 0; a < 3; a++) {
            F[3 * b + a] += fac * d[a];
            F[3 * (b + 1) + a] -= fac * d[a];
        }
    }
    for (int b = 0; b < nb; b++)
        for (int c = b + 1; c < nb; c++) {
            /* Eq. 9 excludes bonded neighbours from the WCA term; that holds for
             * the harmonic bond, whose rest length keeps beads apart.  The FENE
             * bond is purely attractive, so with it the WCA term acts on every
             * pair (Kremer-Grest). */
            if (P->bond_kind == EKO_BOND_HARMONIC && s->chain[b] == s->chain[c] && c - b <= 1) continue;
            double d[3] = {R[3 * b] - R[3 * c], R[3 * b + 1] - R[3 * c + 1], R[3 * b + 2] - R[3 * c + 2]};
            min_image(s, d);
            double Fb[3] = {0, 0, 0};
            wca_force(P->wca_eps, P->wca_sigma, d, Fb);
            for (int a = 0; a < 3; a++) {
                F[3 * b + a] += Fb[a];
                F[3 * c + a] -= Fb[a];
            }
        }
    double rc = pow(2.0, 1.0 / 6.0) * P->wall_sigma;
    for (int b = 0; b < nb; b++) {
        int lo[3], hi[3];
        for (int a = 0; a < 3; a++) {
            lo[a] = (int)floor(R[3 * b + a] - rc);
            hi[a] = (int)floor(R[3 * b + a] + rc) + 1;
        }
        for (int z = lo[2]; z <= hi[2]; z++)
            for (int y = lo[1]; y <= hi[1]; y++)
                for (int x = lo[0]; x <= hi[0]; x++) {
                    int in;
                    long id = node_id(s, x, y, z, &in);
                    if (!in || !s->solid[id]) continue;
                    double d[3] = {R[3 * b] - x, R[3 * b + 1] - y, R[3 * b + 2] - z};
                    wca_force(P->wall_eps, P->wall_sigma, d, &F[3 * b]);
                }
    }
    return EKO_OK;
}

/* Interpolate to every bead, advance it by md_substeps sub-steps of
 * dt = 1/md_substeps, and leave on the nodes the drag it exerts on each
 * species as a force per particle.
 *   g^a_i = -gamma^a [u^a(R_i) - V_i]                                 (Sec. II.B)
 *   M dV/dt = -sum_a g^a_i + F_i + f_i, <f f> = 2 gamma k_B T / dt  (Eqs. 7-8)
 * Readings: gamma^a = xi n^a(R)/n(R) (the total friction xi split by the local
 * composition; the literal gamma^a = xi is a flag); the friction is implicit
 * in V so that M/dt >> xi is not required; the fluid velocity, composition and
 * field are those interpolated at R(t), held over the sub-steps; the drag
 * handed back to the fluid is the sub-step average of g, spread with the R(t)
 * weights, which conserves bead + fluid momentum exactly. */
static int beads_step(eko_sim *s)
{
    const eko_params *P = &s->P;
    const long N = s->N;
    int nb = s->nb;
    memset(s->bead_f, 0, sizeof(double) * EKO_NS * 3 * N);
    if (nb == 0) return EKO_OK;
    long (*nodes)[8] = malloc(sizeof(long[8]) * nb);
    double (*wts)[8] = malloc(sizeof(double[8]) * nb);
    double *uR = malloc(sizeof(double) * nb * EKO_NS * 3);
    double *gam = malloc(sizeof(double) * nb * EKO_NS);
    double *gR = malloc(sizeof(double) * nb * 3);
    double *gacc = calloc((size_t)nb * EKO_NS * 3, sizeof(double));
    double *F = malloc(sizeof(double) * nb * 3);
    int st = EKO_OK;
    for (int b = 0; b < nb; b++) {
        if (!eko_bead_stencil(s, &s->R[3 * b], nodes[b], wts[b])) {
            st = EKO_ERR_BEAD;
            goto done;
        }
        double nR[EKO_NS] = {0, 0, 0};
        for (int a = 0; a < EKO_NS; a++)
            for (int c = 0; c < 3; c++) uR[(b * EKO_NS + a) * 3 + c] = 0.0;
        for (int c = 0; c < 3; c++) gR[3 * b + c] = 0.0;
        for (int k = 0; k < 8; k++) {
            double w = wts[b][k];
            if (w == 0.0) continue;
            long id = nodes[b][k];
            for (int a = 0; a < EKO_NS; a++) {
                double na = s->n[(size_t)a * N + id];
                nR[a] += w * na;
                for (int c = 0; c < 3; c++)
                    uR[(b * EKO_NS + a) * 3 + c] += w * (s->j[((size_t)a * 3 + c) * N + id] / na);
            }
            for (int c = 0; c < 3; c++) gR[3 * b + c] += w * s->grad[(size_t)c * N + id];
        }
        double ntot = nR[0] + nR[1] + nR[2];
        for (int a = 0; a < EKO_NS; a++)
            gam[b * EKO_NS + a] =
                (P->flags & EKO_FLAG_GAMMA_LITERAL) ? P->bead_xi : P->bead_xi * nR[a] / ntot;
        for (int c = 0; c < 3; c++)
            if (fabs(s->q[b] * gR[3 * b + c]) >= 1.0) s->status |= EKO_WARN_CFL;
    }
    {
        int nsub = P->md_substeps;
        double dt = 1.0 / nsub;
        int noise = P->bead_kT > 0.0 && !(P->flags & EKO_FLAG_NO_BEAD_NOISE);
        uint32_t key[2] = {(uint32_t)P->seed, (uint32_t)(P->seed >> 32)};
        for (int sub = 0; sub < nsub; sub++) {
            st = conservative_forces(s, s->R, F);
            if (st != EKO_OK) goto done;
            for (int b = 0; b < nb; b++) {
                double xi[3] = {0, 0, 0};
                if (noise) {
                    uint32_t ctr[4] = {(uint32_t)b, (uint32_t)sub | (1u << 24), (uint32_t)s->step,
                                       (uint32_t)((uint64_t)s->step >> 32)};
                    uint32_t o[4];
                    eko_philox4x32_10(ctr, key, o);
                    for (int c = 0; c < 3; c++) xi[c] = unit_variate(o[c]);
                }
                double gtot = gam[b * EKO_NS + 0] + gam[b * EKO_NS + 1] + gam[b * EKO_NS + 2];
                double amp = noise ? sqrt(2.0 * gtot * P->bead_kT / dt) : 0.0;
                for (int c = 0; c < 3; c++) {
                    double Fe = -s->q[b] * KT * gR[3 * b + c] + s->q[b] * KT * P->E_app[c];
                    double num = P->bead_mass * s->V[3 * b + c] / dt;
                    for (int a = 0; a < EKO_NS; a++) num += gam[b * EKO_NS + a] * uR[(b * EKO_NS + a) * 3 + c];
                    num += F[3 * b + c] + Fe + amp * xi[c];
                    double Vn = num / (P->bead_mass / dt + gtot);
                    for (int a = 0; a < EKO_NS; a++)
                        gacc[(b * EKO_NS + a) * 3 + c] +=
                            dt * (-gam[b * EKO_NS + a] * (uR[(b * EKO_NS + a) * 3 + c] - Vn));
                    s->V[3 * b + c] = Vn;
                }
            }
            int L[3] = {P->nx, P->ny, P->nz};
            for (int b = 0; b < nb; b++)
                for (int c = 0; c < 3; c++) {
                    double r = s->R[3 * b + c] + dt * s->V[3 * b + c];
                    if (P->periodic[c]) {
                        if (r < 0.0) r += L[c];
                        else if (r >= L[c]) r -= L[c];
                    }
                    s->R[3 * b + c] = r;
                }
        }
    }
    /* spread: force density sum_i g^a_i w_ik, then per particle of species a */
    for (int b = 0; b < nb; b++)
        for (int k = 0; k < 8; k++) {
            double w = wts[b][k];
            if (w == 0.0) continue;
            long id = nodes[b][k];
            for (int a = 0; a < EKO_NS; a++)
                for (int c = 0; c < 3; c++)
                    s->bead_f[((size_t)a * 3 + c) * N + id] += gacc[(b * EKO_NS + a) * 3 + c] * w;
        }
    for (long i = 0; i < N; i++) {
        if (s->solid[i]) continue;
        for (int a = 0; a < EKO_NS; a++)
            for (int c = 0; c < 3; c++) {
                size_t k = ((size_t)a * 3 + c) * N + i;
                if (s->bead_f[k] != 0.0) s->bead_f[k] = s->bead_f[k] / s->n[(size_t)a * N + i];
            }
    }
done:
    free(nodes); free(wts); free(uR); free(gam); free(gR); free(gacc); free(F);
    return st;
}

/* ------------------------------------------------------------------------ */
/* 6. collision (Eqs. 5, 6, 10, 12, 13)                                      */
/* ------------------------------------------------------------------------ */

/* Per node and species the force per particle is (Eq. 5)
 *   Phi^a = Phi_ext^a - z^a k_B T grad(phi) + z^a k_B T E_app + bead drag
 *           + Phi_drag^a,
 * with the inter-species friction of Eq. 6, Phi_drag^a = -omega_d^a (u^a - u)
 * (m = 1, sum_b n^b (u^a - u^b)/n = u^a - u).  Readings (see design notes):
 * the forces enter the currents by half (Guo et al. 2002), u^a* = j^a/n^a +
 * Phi^a/2, and the source carries (1 - omega/2); the friction is evaluated at
 * the half-step velocities, which gives the closed form
 *   a^a = j^a/n^a + G^a/2,  h^a = omega_d^a/2,
 *   u*  = sum_a n^a a^a/(1+h^a) / sum_a n^a/(1+h^a),
 *   u^a* = (a^a + h^a u*)/(1+h^a),  Phi^a = G^a - omega_d^a (u^a* - u*);
 * f_eq and S use the species velocity u^a* (the barycentric u* is a flag).
 *   f*_p = f_p - omega (f_p - f_eq_p) + (1 - omega/2) S_p          (Eq. 12)
 *   f_eq_p = w_p n [1 + c.u/vT2 + ((c.u)^2 - vT2 u^2)/(2 vT2^2)]      (Eq. 10)
 *   S_p = w_p n [c.Phi/vT2 + ((c.u)(c.Phi) - vT2 Phi.u)/vT2^2]        (Eq. 13) */
static int collide(eko_sim *s)
{
    const eko_params *P = &s->P;
    const long N = s->N;
    int bad = 0, cfl = 0;
#pragma omp parallel for schedule(static) reduction(| : bad, cfl) num_threads(s->threads)
    for (long i = 0; i < N; i++) {
        if (s->solid[i]) continue;
        double n[EKO_NS], a_[EKO_NS][3], G[EKO_NS][3], h[EKO_NS], wd[EKO_NS];
        double gphi[3] = {s->grad[i], s->grad[(size_t)N + i], s->grad[2 * (size_t)N + i]};
        for (int c = 0; c < 3; c++)
            if (fabs(gphi[c]) >= 1.0) cfl = 1;
        for (int a = 0; a < EKO_NS; a++) {
            n[a] = s->n[(size_t)a * N + i];
            if (!(n[a] > 0.0) || !isfinite(n[a])) bad = 1;
            double D = P->diffusivity[a] > 0.0 ? P->diffusivity[a] : P->diffusivity[1];
            wd[a] = VT2 / D;
            h[a] = 0.5 * wd[a];
            for (int c = 0; c < 3; c++) {
                double z = P->valence[a];
                G[a][c] = P->body_force[a][c] - z * KT * gphi[c] + z * KT * P->E_app[c] +
                          s->bead_f[((size_t)a * 3 + c) * N + i];
                a_[a][c] = s->j[((size_t)a * 3 + c) * N + i] / n[a] + 0.5 * G[a][c];
            }
        }
        double us[3], num[3] = {0, 0, 0}, den = 0.0;
        for (int a = 0; a < EKO_NS; a++) {
            den += n[a] / (1.0 + h[a]);
            for (int c = 0; c < 3; c++) num[c] += n[a] * a_[a][c] / (1.0 + h[a]);
        }
        for (int c = 0; c < 3; c++) us[c] = num[c] / den;
        for (int a = 0; a < EKO_NS; a++) {
            double ua[3], Phi[3], ue[3];
            for (int c = 0; c < 3; c++) {
                ua[c] = (a_[a][c] + h[a] * us[c]) / (1.0 + h[a]);
                Phi[c] = G[a][c] - wd[a] * (ua[c] - us[c]);
                ue[c] = (P->flags & EKO_FLAG_EQ_BARYCENTRIC) ? us[c] : ua[c];
            }
            double om = 1.0 / P->tau[a];
            double u2 = ue[0] * ue[0] + ue[1] * ue[1] + ue[2] * ue[2];
            double Fu = Phi[0] * ue[0] + Phi[1] * ue[1] + Phi[2] * ue[2];
            for (int p = 0; p < EKO_Q; p++) {
                double cu = CV[p][0] * ue[0] + CV[p][1] * ue[1] + CV[p][2] * ue[2];
                double cF = CV[p][0] * Phi[0] + CV[p][1] * Phi[1] + CV[p][2] * Phi[2];
                double feq = WV[p] * n[a] * (1.0 + cu / VT2 + (cu * cu - VT2 * u2) / (2.0 * VT2 * VT2));
                double S = WV[p] * n[a] * (cF / VT2 + (cu * cF - VT2 * Fu) / (VT2 * VT2));
                size_t k = ((size_t)a * EKO_Q + p) * N + i;
                s->fstar[k] = s->f[k] - om * (s->f[k] - feq) + (1.0 - 0.5 * om) * S;
            }
            if (P->fluct_mass > 0.0) {
                /* Eq. 14: Delta_p = sqrt(m n omega (2 - omega)) sum_{k=4}^{18}
                 * w_p CHI_kp N_k, N_k zero mean and unit variance, drawn
                 * from Philox with counter (node, 2^25 | species << 4 | call,
                 * step) and the run's seed as key */
                double Nk[16];
                for (int call = 0; call < 4; call++) {
                    uint32_t ctr[4] = {(uint32_t)i, (2u << 24) | ((uint32_t)a << 4) | (uint32_t)call,
                                       (uint32_t)s->step, (uint32_t)((uint64_t)s->step >> 32)};
                    uint32_t key[2] = {(uint32_t)P->seed, (uint32_t)(P->seed >> 32)}, out[4];
                    eko_philox4x32_10(ctr, key, out);
                    for (int j = 0; j < 4; j++) Nk[4 * call + j] = unit_variate(out[j]);
                }
                double amp = sqrt(P->fluct_mass * n[a] * om * (2.0 - om));
                for (int p = 0; p < EKO_Q; p++) {
                    double d = 0.0;
                    for (int k = 4; k < EKO_Q; k++) d += CHI[k][p] * Nk[k - 4];
                    s->fstar[((size_t)a * EKO_Q + p) * N + i] += amp * WV[p] * d;
                }
            }
        }
    }
    if (cfl) s->status |= EKO_WARN_CFL;
    return bad ? EKO_ERR_UNSTABLE : EKO_OK;
}

/* ------------------------------------------------------------------------ */
/* one step                                                                  */
/* ------------------------------------------------------------------------ */

static int one_step(eko_sim *s)
{
    const long N = s->N;
    stream(s);
    moments(s);
    int st = deposit_beads(s);
    if (st != EKO_OK) return st;
    for (long i = 0; i < N; i++) {
        if (s->solid[i]) {
            s->rho[i] = 0.0;
            continue;
        }
        double r = 0.0;
        for (int a = 0; a < EKO_NS; a++) r += s->P.valence[a] * s->n[(size_t)a * N + i];
        s->rho[i] = r + s->src_wall[i] + s->bead_q[i];
    }
    double res = 0.0;
    int it = eko_poisson_solve(s, s->rho, s->phi, s->P.poisson_tol, s->P.poisson_max_iter,
                               s->P.poisson_check_every, s->P.poisson_fixed_iter, &res);
    s->poisson_iters = it < 0 ? -it : it;
    s->poisson_res = res;
    if (it < 0) s->status |= EKO_WARN_NOCONV;
    eko_node_gradient(s, s->phi, s->grad);
    st = beads_step(s);
    if (st != EKO_OK) return st;
    st = collide(s);
    if (st != EKO_OK) return st;
    s->step++;
    return EKO_OK;
}

int eko_step(eko_sim *s, int nsteps)
{
    s->status = 0;
    for (int k = 0; k < nsteps; k++) {
        int st = one_step(s);
        if (st < 0) return st;
    }
    return s->status;
}

/* ------------------------------------------------------------------------ */
/* outputs                                                                   */
/* ------------------------------------------------------------------------ */

/* Densities and (bare) currents of the streamed populations f(t), the
 * potential of the last step with its fluid mean removed, bead state. */
void eko_get_fields(eko_sim *s, double *n_out, double *j_out, double *phi_out, double *R_out,
                    double *V_out)
{
    const long N = s->N;
    stream(s);
    moments(s);
    if (n_out) memcpy(n_out, s->n, sizeof(double) * EKO_NS * N);
    if (j_out) memcpy(j_out, s->j, sizeof(double) * EKO_NS * 3 * N);
    if (phi_out) {
        double sum = 0.0;
        long nf = 0;
        for (long i = 0; i < N; i++)
            if (!s->solid[i]) {
                sum += s->phi[i];
                nf++;
            }
        double mean = nf ? sum / nf : 0.0;
        for (long i = 0; i < N; i++) phi_out[i] = s->solid[i] ? 0.0 : s->phi[i] - mean;
    }
    if (R_out && s->nb) memcpy(R_out, s->R, sizeof(double) * 3 * s->nb);
    if (V_out && s->nb) memcpy(V_out, s->V, sizeof(double) * 3 * s->nb);
}

void eko_get_state(const eko_sim *s, double *fstar, double *phi, int64_t *step)
{
    if (fstar) memcpy(fstar, s->fstar, sizeof(double) * EKO_NS * EKO_Q * s->N);
    if (phi) memcpy(phi, s->phi, sizeof(double) * s->N);
    if (step) *step = s->step;
}

/* replace the applied field from the next step on */
void eko_set_field(eko_sim *s, const double E[3])
{
    for (int a = 0; a < 3; a++) s->P.E_app[a] = E[a];
}

void eko_set_state(eko_sim *s, const double *fstar, const double *phi, int64_t step)
{
    if (fstar) memcpy(s->fstar, fstar, sizeof(double) * EKO_NS * EKO_Q * s->N);
    if (phi) memcpy(s->phi, phi, sizeof(double) * s->N);
    s->step = step;
}

/* stats: [mass_0..2, momentum_x,y,z (fluid, bare), poisson_iters, poisson_res,
 *         bead momentum x,y,z] */
void eko_get_stats(eko_sim *s, double *out)
{
    const long N = s->N;
    stream(s);
    moments(s);
    for (int k = 0; k < 12; k++) out[k] = 0.0;
    for (int a = 0; a < EKO_NS; a++)
        for (long i = 0; i < N; i++) {
            out[a] += s->n[(size_t)a * N + i];
            for (int c = 0; c < 3; c++) out[3 + c] += s->j[((size_t)a * 3 + c) * N + i];
        }
    out[6] = s->poisson_iters;
    out[7] = s->poisson_res;
    for (int b = 0; b < s->nb; b++)
        for (int c = 0; c < 3; c++) out[8 + c] += s->P.bead_mass * s->V[3 * b + c];
}

/* Link bits: bit p (1..18) set when x - c_p is wall or outside a closed face;
 * bit 31 set on wall nodes (all other bits clear there). */
void eko_link_mask(const eko_sim *s, uint32_t *mask)
{
    for (long i = 0; i < s->N; i++) {
        if (s->solid[i]) {
            mask[i] = 0x80000000u;
            continue;
        }
        int x, y, z;
        coords(s, i, &x, &y, &z);
        uint32_t m = 0;
        for (int p = 1; p < EKO_Q; p++)
            if (!fluid_at(s, x - CV[p][0], y - CV[p][1], z - CV[p][2])) m |= 1u << p;
        mask[i] = m;
    }
}

void eko_wall_source(const eko_sim *s, double *out) { memcpy(out, s->src_wall, sizeof(double) * s->N); }

void eko_basis(double *chi)
{
    lattice_init();
    memcpy(chi, CHI, sizeof(CHI));
}

void eko_lattice(int32_t *c, double *w, int32_t *opp)
{
    lattice_init();
    for (int p = 0; p < EKO_Q; p++) {
        for (int a = 0; a < 3; a++) c[3 * p + a] = CV[p][a];
        w[p] = WV[p];
        opp[p] = OPPV[p];
    }
}

double eko_default_rho_jacobi(const eko_sim *s) { return default_rho_jacobi(&s->P); }

int64_t eko_sizeof_params(void) { return (int64_t)sizeof(eko_params); }
