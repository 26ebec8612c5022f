// C ABI of the library: handle life cycle, argument checks, geometry set-up,
// dispatch to the per-precision step implementations, host transfers.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <condition_variable>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "ekl_kernels.cuh"
#include "ekl_gauge.cuh"
#include "ekl_mg.cuh"

using namespace ekl;

struct ekl_handle {
    Ctx c;
};

struct ekl_batch {
    Batch b;
};

namespace {

thread_local char g_err[512] = "";
ekl_alloc_fn g_alloc = nullptr;
ekl_free_fn g_free = nullptr;
void *g_alloc_ctx = nullptr;

int fail(int code, const char *msg)
{
    snprintf(g_err, sizeof g_err, "%s", msg);
    return code;
}

int fail_cuda(cudaError_t e, const char *where)
{
    snprintf(g_err, sizeof g_err, "%s: %s", where, cudaGetErrorString(e));
    return EKL_ERR_CUDA;
}

struct PrecOps {
    int (*init)(Ctx &, const double *);
    int (*run)(Ctx &, int);
    int (*fields)(Ctx &, double *, double *, double *);
    int (*get_state)(Ctx &, double *, double *);
    int (*set_state)(Ctx &, const double *, const double *);
    int (*pois_blocks)();
    int (*mg_blocks)(size_t, int);
    int (*mass)(Ctx &);
    int (*mg_batch_blocks)(size_t);
    int (*current)(Ctx &, int, int, double *);
};

const PrecOps &ops(int prec)
{
    static const PrecOps t[4] = {
        {init_populations_f64, run_steps_f64, get_fields_f64, get_state_f64, set_state_f64, pois_blocks_f64, mg_blocks_f64, mass_f64, mg_batch_blocks_f64, current_f64},
        {init_populations_f32, run_steps_f32, get_fields_f32, get_state_f32, set_state_f32, pois_blocks_f32, mg_blocks_f32, mass_f32, mg_batch_blocks_f32, current_f32},
        {init_populations_bf16, run_steps_bf16, get_fields_bf16, get_state_bf16, set_state_bf16, pois_blocks_bf16, mg_blocks_bf16, mass_bf16, mg_batch_blocks_bf16, current_bf16},
        {init_populations_fp16, run_steps_fp16, get_fields_fp16, get_state_fp16, set_state_fp16, pois_blocks_fp16, mg_blocks_fp16, mass_fp16, mg_batch_blocks_fp16, current_fp16},
    };
    return t[prec];
}

// Link bits of every node (integer work, bit-exact against the oracle):
// bit p set when x - c_p is a wall node or beyond a closed face; bit 31 on walls.
// Self-test of the bounded device-side wait: block 1 never reaches the
// barrier, so block 0's wait has to give up on its own.
__global__ void wait_selftest_kernel(unsigned *bar, int *status)
{
    if (blockIdx.x != 0) return;
    unsigned k = 0;
    grid_barrier(bar, gridDim.x, k, status);
}

// The multigrid lattice level's link byte of every node (see mg_link_of).
__global__ void mg_link_kernel(const uint32_t *__restrict__ mask, uint8_t *__restrict__ link, long long N)
{
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < N) link[i] = mg_link_of(mask[i]);
}

__global__ void mask_kernel(Grid3 g, int px, int py, int pz, const uint8_t *__restrict__ solid,
                            uint32_t *__restrict__ mask)
{
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= g.N) return;
    if (solid[i]) {
        mask[i] = SOLID_BIT;
        return;
    }
    int x, y, z;
    coords_of(g, i, x, y, z);
    uint32_t m = 0;
#pragma unroll
    for (int p = 1; p < Q; p++) {
        int X = x - cx_(p), Y = y - cy_(p), Z = z - cz_(p);
        bool in = true;
        if (X < 0 || X >= g.nx) {
            if (px) X = (X + g.nx) % g.nx;
            else in = false;
        }
        if (Y < 0 || Y >= g.ny) {
            if (py) Y = (Y + g.ny) % g.ny;
            else in = false;
        }
        if (Z < 0 || Z >= g.nz) {
            if (pz) Z = (Z + g.nz) % g.nz;
            else in = false;
        }
        if (!in || solid[(long long)X + (long long)g.nx * (Y + (long long)g.ny * Z)]) m |= 1u << p;
    }
    mask[i] = m;
}

void release(Ctx &c)
{
    size_t rs = real_size(c.prec);
    dev_free(c, c.f[0], 0);
    dev_free(c, c.f[1], 0);
    dev_free(c, c.mask, 0);
    dev_free(c, c.wall_share, 0);
    dev_free(c, c.src_wall, 0);
    dev_free(c, c.rho, 0);
    dev_free(c, c.b, 0);
    dev_free(c, c.phi, 0);
    dev_free(c, c.part_charge, 0);
    dev_free(c, c.part_charge_q, 0);
    dev_free(c, c.charge_tot, 0);
    dev_free(c, c.charge_tot_q, 0);
    dev_free(c, c.charge_chunks, 0);
    dev_free(c, c.part_mass, 0);
    dev_free(c, c.part_pois, 0);
    dev_free(c, c.barrier, 0);
    dev_free(c, c.status, 0);
    dev_free(c, c.pois_iters, 0);
    dev_free(c, c.pois_total, 0);
    dev_free(c, c.pois_res, 0);
    dev_free(c, c.omegas, 0);
    dev_free(c, c.wchi, 0);
    dev_free(c, c.R, 0);
    dev_free(c, c.V, 0);
    dev_free(c, c.q, 0);
    dev_free(c, c.chain, 0);
    dev_free(c, c.patch_count, 0);
    dev_free(c, c.patch_bits, 0);
    dev_free(c, c.patch_node, 0);
    dev_free(c, c.patch_q, 0);
    dev_free(c, c.patch_f, 0);
    dev_free(c, c.patch_mom, 0);
    dev_free(c, c.entry_slot, 0);
    dev_free(c, c.sorted_entry, 0);
    dev_free(c, c.slot_first, 0);
    dev_free(c, c.entry_w, 0);
    for (int l = 1; l < MG_MAXLEV; l++) {
        dev_free(c, c.mg_lev[l].sig, 0);
        dev_free(c, c.mg_lev[l].e, 0);
        dev_free(c, c.mg_lev[l].f, 0);
        dev_free(c, c.mg_lev[l].t, 0);
    }
    dev_free(c, c.mg_r, 0);
    dev_free(c, c.mg_link, 0);
    dev_free(c, c.mg_z, 0);
    dev_free(c, c.mg_q, 0);
    dev_free(c, c.mg_p[0], 0);
    dev_free(c, c.mg_p[1], 0);
    dev_free(c, c.mg_part, 0);
    dev_free(c, c.mgs_ctl, 0);
    if (c.mgs_exec) cudaGraphExecDestroy(c.mgs_exec);
    if (c.mgs_graph) cudaGraphDestroy(c.mgs_graph);
    c.mgs_exec = nullptr;
    c.mgs_graph = nullptr;
    dev_free(c, c.mg_dense, 0);
    dev_free(c, c.mg_phi_prev, 0);
    warmstart_free(c);
    (void)rs;
    for (int k = 0; k < 2 * PH_COUNT; k++)
        if (c.ev[k]) cudaEventDestroy(c.ev[k]);
    for (int k = 0; k < c.tcap; k++) cudaEventDestroy(c.tpool[k]);
    free(c.tpool);
    free(c.tphase);
}

int status_to_code(int st)
{
    if (st & ST_TIMEOUT) return fail(EKL_ERR_TIMEOUT, "a device-side wait timed out");
    if (st & ST_UNSTABLE) return fail(EKL_ERR_UNSTABLE, "non-finite or non-positive species density");
    if (st & ST_BEAD) return fail(EKL_ERR_BEAD, "bead in a wall, outside the box, or FENE bond broken");
    int w = 0;
    if (st & ST_NOCONV) w |= EKL_WARN_NOCONV;
    if (st & ST_CFL) w |= EKL_WARN_CFL;
    return w;
}

}  // namespace

namespace ekl {

void set_last_error(const char *msg) { fail(0, msg); }

void timing_record(Ctx &c, int phase, int begin)
{
    if (c.tused + 1 > c.tcap) {
        int ncap = c.tcap ? 2 * c.tcap : 256;
        cudaEvent_t *np = (cudaEvent_t *)realloc(c.tpool, ncap * sizeof(cudaEvent_t));
        int *nph = (int *)realloc(c.tphase, ncap * sizeof(int));
        if (!np || !nph) {
            if (np) c.tpool = np;
            if (nph) c.tphase = nph;
            return;
        }
        c.tpool = np;
        c.tphase = nph;
        for (int k = c.tcap; k < ncap; k++) cudaEventCreate(&c.tpool[k]);
        c.tcap = ncap;
    }
    cudaEventRecord(c.tpool[c.tused], c.stream);
    c.tphase[c.tused] = begin ? phase : -1 - phase;
    c.tused++;
}

// call after the stream has been synchronised
void timing_flush(Ctx &c)
{
    for (int k = 0; k + 1 < c.tused; k++) {
        if (c.tphase[k] >= 0 && c.tphase[k + 1] == -1 - c.tphase[k]) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, c.tpool[k], c.tpool[k + 1]) == cudaSuccess)
                c.ms_phase[c.tphase[k]] += ms;
            k++;
        }
    }
    c.tused = 0;
}

size_t real_size(int prec) { return prec == EKL_F64 ? 8 : 4; }
size_t store_size(int prec) { return prec == EKL_F64 ? 8 : (prec == EKL_F32 ? 4 : 2); }
size_t phi_size(int prec) { return 8; }

void *dev_alloc(Ctx &c, size_t bytes)
{
    if (bytes == 0) bytes = 16;
    if (g_alloc) return g_alloc(bytes, (void *)c.stream, g_alloc_ctx);
    void *p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) return nullptr;
    return p;
}

void dev_free(Ctx &c, void *p, size_t bytes)
{
    if (!p) return;
    if (g_free) g_free(p, bytes, (void *)c.stream, g_alloc_ctx);
    else cudaFree(p);
}

}  // namespace ekl

namespace {

// Moment basis of the fluctuating term (Eq. 14), returned as w_p chi_kp:
// the monomials 1, cx, cy, cz, cx^2, cy^2, cz^2, cx cy, cx cz, cy cz,
// cx^2 cy, cx cy^2, cx^2 cz, cx cz^2, cy^2 cz, cy cz^2, cx^2 cy^2, cx^2 cz^2,
// cy^2 cz^2 on the 19 velocities, made orthonormal in order (classical
// Gram-Schmidt) in the scalar product sum_p w_p a_p b_p; rows 0-3 then span
// density and current, 4-9 the momentum flux, 10-18 the rest.
static void fluct_basis(double wchi[Q][Q])
{
    double chi[Q][Q];
    for (int k = 0; k < Q; k++) {
        double v[Q];
        for (int p = 0; p < Q; p++) {
            const double x = cx_(p), y = cy_(p), z = cz_(p);
            const double mono[Q] = {1.0,       x,         y,         z,         x * x,     y * y,     z * z,
                                    x * y,     x * z,     y * z,     x * x * y, x * y * y, x * x * z, x * z * z,
                                    y * y * z, y * z * z, x * x * y * y, x * x * z * z, y * y * z * z};
            v[p] = mono[k];
        }
        for (int l = 0; l < k; l++) {
            double dot = 0.0;
            for (int p = 0; p < Q; p++) dot += w_(p) * v[p] * chi[l][p];
            for (int p = 0; p < Q; p++) v[p] -= dot * chi[l][p];
        }
        double norm2 = 0.0;
        for (int p = 0; p < Q; p++) norm2 += w_(p) * v[p] * v[p];
        const double inv = 1.0 / sqrt(norm2);
        for (int p = 0; p < Q; p++) chi[k][p] = v[p] * inv;
    }
    for (int k = 0; k < Q; k++)
        for (int p = 0; p < Q; p++) wchi[k][p] = w_(p) * chi[k][p];
}

// fn(t) for t in [0, count) on the host's cores (interleaved, so that rows of
// growing length spread evenly); runs inline when count is small
template <typename Fn> static void host_parallel(int count, Fn fn)
{
    const int hw = (int)std::thread::hardware_concurrency();
    const int T = std::max(1, std::min({hw, 32, count / 16}));
    if (T <= 1) {
        for (int t = 0; t < count; t++) fn(t);
        return;
    }
    std::vector<std::thread> pool;
    for (int w = 0; w < T; w++)
        pool.emplace_back([&, w]() {
            for (int t = w; t < count; t += T) fn(t);
        });
    for (auto &th : pool) th.join();
}

// Copies of large pageable host arrays run at about 12 GB/s; through two
// pinned staging buffers, with the host side of each chunk copied on several
// cores while the DMA of the next chunk runs, they run several times faster.
// The buffers are allocated once per process and shared under a lock.
static constexpr size_t STAGE_BYTES = (size_t)64 << 20;
static std::mutex g_stage_lock;
static void *g_stage[2] = {nullptr, nullptr};
static cudaEvent_t g_stage_ev[2];
static int g_stage_dev = -1;

// Host copies of a staged transfer: a crew of threads, made once per
// transfer, copies each chunk in equal slices (one per thread) while the
// transfer's next DMA runs.
class CopyCrew {
  public:
    explicit CopyCrew(size_t bytes)
    {
        const int hw = (int)std::thread::hardware_concurrency();
        const int T = (int)std::max<size_t>(1, std::min<size_t>({(size_t)std::max(1, hw), 16, bytes >> 22}));
        // slices are set by the threads actually made (T_ is read by the
        // workers only after the first copy() publishes a job under m_)
        for (int t = 1; t < T; t++) {
            try {
                th_.emplace_back([this, t]() { work(t); });
            } catch (...) {
                break;
            }
        }
        T_ = (int)th_.size() + 1;
    }
    ~CopyCrew()
    {
        {
            std::lock_guard<std::mutex> lk(m_);
            stop_ = true;
        }
        go_.notify_all();
        for (auto &t : th_) t.join();
    }
    // dst <- src (n bytes), the calling thread taking slice 0
    void copy(void *dst, const void *src, size_t n)
    {
        {
            std::lock_guard<std::mutex> lk(m_);
            dst_ = (char *)dst;
            src_ = (const char *)src;
            n_ = n;
            pending_ = T_ - 1;
            gen_++;
        }
        go_.notify_all();
        slice(0, (char *)dst, (const char *)src, n);
        std::unique_lock<std::mutex> lk(m_);
        done_.wait(lk, [this]() { return pending_ == 0; });
    }

  private:
    void slice(int t, char *dst, const char *src, size_t n) const
    {
        const size_t part = (n + T_ - 1) / T_, off = part * t;
        if (off < n) memcpy(dst + off, src + off, std::min(part, n - off));
    }
    void work(int t)
    {
        long seen = 0;
        for (;;) {
            std::unique_lock<std::mutex> lk(m_);
            go_.wait(lk, [&]() { return stop_ || gen_ != seen; });
            if (stop_) return;
            seen = gen_;
            char *d = dst_;
            const char *s = src_;
            const size_t n = n_;
            lk.unlock();
            slice(t, d, s, n);
            lk.lock();
            if (--pending_ == 0) done_.notify_one();
        }
    }
    int T_ = 1;
    std::vector<std::thread> th_;
    std::mutex m_;
    std::condition_variable go_, done_;
    long gen_ = 0;
    int pending_ = 0;
    bool stop_ = false;
    char *dst_ = nullptr;
    const char *src_ = nullptr;
    size_t n_ = 0;
};

// dst <- src, bytes long, one side on the device (to_host: src is device
// memory); ordered on the stream and complete on return
static cudaError_t staged_copy(cudaStream_t stream, int device, void *dst, const void *src, size_t bytes,
                               bool to_host)
{
    auto plain = [&]() {  // one pageable copy
        cudaError_t e = cudaMemcpyAsync(dst, src, bytes, to_host ? cudaMemcpyDeviceToHost : cudaMemcpyHostToDevice,
                                        stream);
        return e == cudaSuccess ? cudaStreamSynchronize(stream) : e;
    };
    if (bytes < ((size_t)8 << 20)) return plain();
    std::lock_guard<std::mutex> lock(g_stage_lock);
    cudaError_t e = cudaSuccess;
    if (g_stage_dev != device) {
        for (int b = 0; b < 2; b++)
            if (g_stage[b]) {
                cudaFreeHost(g_stage[b]);
                cudaEventDestroy(g_stage_ev[b]);
                g_stage[b] = nullptr;
            }
        g_stage_dev = -1;
        bool ev_made[2] = {false, false};
        for (int b = 0; b < 2 && e == cudaSuccess; b++) {
            e = cudaMallocHost(&g_stage[b], STAGE_BYTES);
            if (e != cudaSuccess) g_stage[b] = nullptr;
            else if ((e = cudaEventCreateWithFlags(&g_stage_ev[b], cudaEventDisableTiming)) == cudaSuccess)
                ev_made[b] = true;
        }
        if (e != cudaSuccess) {  // no pinned memory to be had: the plain copy
            for (int b = 0; b < 2; b++) {
                if (g_stage[b]) cudaFreeHost(g_stage[b]);
                if (ev_made[b]) cudaEventDestroy(g_stage_ev[b]);
                g_stage[b] = nullptr;
            }
            cudaGetLastError();
            return plain();
        }
        g_stage_dev = device;
    }
    const size_t nch = (bytes + STAGE_BYTES - 1) / STAGE_BYTES;
    auto len = [&](size_t k) { return std::min(STAGE_BYTES, bytes - k * STAGE_BYTES); };
    CopyCrew crew(std::min(bytes, STAGE_BYTES));
    if (to_host) {
        // DMA of chunk k into buffer k % 2 while the host copies chunk k - 1 out
        for (size_t k = 0; k <= nch && e == cudaSuccess; k++) {
            if (k < nch) {
                e = cudaMemcpyAsync(g_stage[k & 1], (const char *)src + k * STAGE_BYTES, len(k),
                                    cudaMemcpyDeviceToHost, stream);
                if (e == cudaSuccess) e = cudaEventRecord(g_stage_ev[k & 1], stream);
            }
            if (k >= 1 && e == cudaSuccess) {
                e = cudaEventSynchronize(g_stage_ev[(k - 1) & 1]);
                if (e == cudaSuccess) crew.copy((char *)dst + (k - 1) * STAGE_BYTES, g_stage[(k - 1) & 1], len(k - 1));
            }
        }
    } else {
        // host copy of chunk k into buffer k % 2 once that buffer's DMA (chunk
        // k - 2) is done, then its DMA
        for (size_t k = 0; k < nch && e == cudaSuccess; k++) {
            if (k >= 2) e = cudaEventSynchronize(g_stage_ev[k & 1]);
            if (e != cudaSuccess) break;
            crew.copy(g_stage[k & 1], (const char *)src + k * STAGE_BYTES, len(k));
            e = cudaMemcpyAsync((char *)dst + k * STAGE_BYTES, g_stage[k & 1], len(k), cudaMemcpyHostToDevice, stream);
            if (e == cudaSuccess) e = cudaEventRecord(g_stage_ev[k & 1], stream);
        }
    }
    return e == cudaSuccess ? cudaStreamSynchronize(stream) : e;
}

// Pseudo-inverse of the coarsest multigrid operator A (cells with conductances
// sig: +x, +y, +z faces, 1/diag; inactive cells have none).  A is the graph
// Laplacian of the active cells, symmetric positive semi-definite with the
// constants of each connected part as null space, so
//   A^+ = (A + sum_parts 1_p 1_p^T / n_p)^-1 - sum_parts 1_p 1_p^T / n_p,
// the bracket being positive definite (Cholesky, FP64).  Returns row-major
// FP32 [n][n] with zero rows and columns on inactive cells.
// sum of a[k] b[k] over k0 <= k < k1 in four interleaved partial sums (a
// fixed order: the same on every host), so that the products' additions
// need not wait on one another
static inline double dot4(const double *a, const double *b, int k0, int k1)
{
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
    int k = k0;
    for (; k + 4 <= k1; k += 4) {
        s0 += a[k] * b[k];
        s1 += a[k + 1] * b[k + 1];
        s2 += a[k + 2] * b[k + 2];
        s3 += a[k + 3] * b[k + 3];
    }
    for (; k < k1; k++) s0 += a[k] * b[k];
    return (s0 + s1) + (s2 + s3);
}

static std::vector<float> coarse_pinv(int nx, int ny, int nz, const std::vector<float4> &sig)
{
    const int n = nx * ny * nz;
    std::vector<double> B((size_t)n * n, 0.0);
    auto at = [&](int i, int j) -> double & { return B[(size_t)i * n + j]; };
    std::vector<int> act(n), part(n, -1);
    for (int i = 0; i < n; i++) act[i] = sig[i].w != 0.f;
    auto nbr = [&](int i, int a) {
        int x = i % nx, y = (i / nx) % ny, z = i / (nx * ny);
        if (a == 0) x = (x + 1) % nx;
        if (a == 1) y = (y + 1) % ny;
        if (a == 2) z = (z + 1) % nz;
        return x + nx * (y + ny * z);
    };
    for (int i = 0; i < n; i++) {
        const float s3[3] = {sig[i].x, sig[i].y, sig[i].z};
        for (int a = 0; a < 3; a++) {
            if (s3[a] == 0.f) continue;
            const int j = nbr(i, a);
            at(i, i) += s3[a];
            at(j, j) += s3[a];
            at(i, j) -= s3[a];
            at(j, i) -= s3[a];
        }
    }
    // connected parts of the active cells (faces with sigma > 0)
    std::vector<int> count, stack;
    for (int i = 0; i < n; i++) {
        if (!act[i] || part[i] >= 0) continue;
        const int p = (int)count.size();
        count.push_back(0);
        stack.assign(1, i);
        part[i] = p;
        while (!stack.empty()) {
            const int u = stack.back();
            stack.pop_back();
            count[p]++;
            for (int j = 0; j < n; j++)
                if (j != u && at(u, j) != 0.0 && part[j] < 0) {
                    part[j] = p;
                    stack.push_back(j);
                }
        }
    }
    for (int i = 0; i < n; i++) {
        if (!act[i]) {
            at(i, i) = 1.0;
            continue;
        }
        for (int j = 0; j < n; j++)
            if (act[j] && part[j] == part[i]) at(i, j) += 1.0 / count[part[i]];
    }
    // Cholesky B = L L^T (lower triangle in place), blocked right-looking:
    // per block column, factor the diagonal block, solve the panel below it,
    // update the trailing matrix; panel and update rows go to host threads
    const int NB = 64;
    bool spd = true;
    for (int kb = 0; kb < n && spd; kb += NB) {
        const int e = std::min(kb + NB, n);
        for (int j = kb; j < e && spd; j++) {
            double d = at(j, j);
            for (int k = kb; k < j; k++) d -= at(j, k) * at(j, k);
            if (!(d > 0.0)) {
                spd = false;
                break;
            }
            d = sqrt(d);
            at(j, j) = d;
            for (int i = j + 1; i < e; i++) {
                double v = at(i, j);
                for (int k = kb; k < j; k++) v -= at(i, k) * at(j, k);
                at(i, j) = v / d;
            }
        }
        if (!spd) break;
        host_parallel(n - e, [&](int t) {
            const int i = e + t;
            double *ri = &B[(size_t)i * n];
            for (int j = kb; j < e; j++) {
                const double *rj = &B[(size_t)j * n];
                ri[j] = (ri[j] - dot4(ri, rj, kb, j)) / rj[j];
            }
        });
        host_parallel(n - e, [&](int t) {
            const int i = e + t;
            double *ri = &B[(size_t)i * n];
            for (int j = e; j <= i; j++) ri[j] -= dot4(ri, &B[(size_t)j * n], kb, e);
        });
    }
    if (!spd) return {};
    // Wt = (L^-1)^T (upper, row j = column j of L^-1), then B^-1 = Wt Wt^T
    std::vector<double> Wt((size_t)n * n, 0.0);
    host_parallel(n, [&](int j) {
        double *w = &Wt[(size_t)j * n];
        w[j] = 1.0 / at(j, j);
        for (int i = j + 1; i < n; i++) {
            const double *ri = &B[(size_t)i * n];
            w[i] = -dot4(ri, w, j, i) / ri[i];
        }
    });
    std::vector<float> M((size_t)n * n, 0.f);
    host_parallel(n, [&](int i) {
        if (!act[i]) return;
        const double *wi = &Wt[(size_t)i * n];
        for (int j = 0; j <= i; j++) {
            if (!act[j]) continue;
            double v = dot4(wi, &Wt[(size_t)j * n], i, n);
            if (part[i] == part[j]) v -= 1.0 / count[part[i]];
            M[(size_t)i * n + j] = M[(size_t)j * n + i] = (float)v;
        }
    });
    return M;
}

// Tile of a coarse level for the shared-memory smoothing (even extents up to
// tmax; halo H; region within max_bytes):
// minimises the rounds of tiles over the launch's blocks times a tile's cost,
// taken as a fixed part (load latency and the block-wide barriers, worth
// about 6000 region cells) plus its region's cell count.
static void mg_pick_tile(const int ex[3], int H, int nblk, int tmax, size_t max_bytes, int T[3], size_t &words)
{
    int lim[3];
    for (int a = 0; a < 3; a++) lim[a] = std::min(tmax, std::max(2, (ex[a] + 1) & ~1));
    double best = 1e300;
    size_t wbest = 0;
    for (int tx = 2; tx <= lim[0]; tx += 2)
        for (int ty = 2; ty <= lim[1]; ty += 2)
            for (int tz = 2; tz <= lim[2]; tz += 2) {
                const size_t w = mg_tile_words(tx + 2 * H, ty + 2 * H, tz + 2 * H);
                if (w * sizeof(float) > max_bytes) continue;
                const long long nt = (long long)((ex[0] + tx - 1) / tx) * ((ex[1] + ty - 1) / ty) * ((ex[2] + tz - 1) / tz);
                const double rounds = (double)((nt + nblk - 1) / nblk);
                const double cost = rounds * (6000.0 + (double)(tx + 2 * H) * (ty + 2 * H) * (tz + 2 * H));
                if (cost < best) {
                    best = cost;
                    T[0] = tx;
                    T[1] = ty;
                    T[2] = tz;
                    wbest = w;
                }
            }
    words = std::max(words, wbest);
}

// Multigrid hierarchy of the Poisson operator (EKL_POISSON_MG): levels halve
// every extent (rounding up) while each periodic extent stays even, down to
// MG_COARSEST_CELLS cells.  Face conductances: 1 on the lattice's open faces
// (fluid to fluid, inside or across a periodic side); on level l+1, half the
// sum of the level-l conductances crossing the aggregated face.  `tiles`:
// smooth the grid-wide coarse levels of at most MG_TILE_CELLS_PER_BLOCK cells
// per block in shared-memory tiles.  `split`: run the solve of a large
// lattice in split form (ekl_mgs.cuh).  Returns an error message, or null.
template <typename Alloc>
static const char *build_multigrid(Ctx &c, const uint8_t *solid, Alloc &A, long long coarsest_cells, bool tiles,
                                   bool split)
{
    int d[MG_MAXLEV][3];
    d[0][0] = c.nx;
    d[0][1] = c.ny;
    d[0][2] = c.nz;
    int nlev = 1;
    while (nlev < MG_MAXLEV) {
        const int *p = d[nlev - 1];
        if ((long long)p[0] * p[1] * p[2] <= coarsest_cells) break;
        bool ok = true;
        for (int a = 0; a < 3; a++)
            if (p[a] < 2 || (c.per[a] && p[a] % 4)) ok = false;
        if (!ok) break;
        for (int a = 0; a < 3; a++) d[nlev][a] = (p[a] + 1) / 2;
        nlev++;
    }
    if (nlev < 2) return "multigrid needs a coarser level: periodic extents must be multiples of 4";
    // lattice conductances of the +x, +y, +z faces (every entry written by
    // the plane loops: the arrays are not cleared first)
    const long long N = c.N;
    std::unique_ptr<float[]> sg[3];
    for (int a = 0; a < 3; a++) sg[a].reset(new (std::nothrow) float[N]);
    if (!sg[0] || !sg[1] || !sg[2]) return "host allocation failed";
    host_parallel(c.nz, [&](int z) {  // planes on the host's cores (disjoint writes)
        for (int y = 0; y < c.ny; y++)
            for (int x = 0; x < c.nx; x++) {
                const long long i = x + (long long)c.nx * (y + (long long)c.ny * z);
                for (int a = 0; a < 3; a++) sg[a][i] = 0.f;
                if (solid[i]) continue;
                const int q[3] = {x, y, z}, L[3] = {c.nx, c.ny, c.nz};
                for (int a = 0; a < 3; a++) {
                    int r[3] = {q[0], q[1], q[2]};
                    r[a]++;
                    if (r[a] == L[a]) {
                        if (!c.per[a]) continue;
                        r[a] = 0;
                    }
                    const long long j = r[0] + (long long)c.nx * (r[1] + (long long)c.ny * r[2]);
                    if (!solid[j]) sg[a][i] = 1.f;
                }
            }
    });
    for (int l = 1; l < nlev; l++) {
        const int *F = d[l - 1], *C = d[l];
        const long long NC = (long long)C[0] * C[1] * C[2];
        std::unique_ptr<float[]> cs[3];  // every entry written below
        for (int a = 0; a < 3; a++) cs[a].reset(new (std::nothrow) float[NC]);
        if (!cs[0] || !cs[1] || !cs[2]) return "host allocation failed";
        host_parallel(C[2], [&](int Z) {
            for (int Y = 0; Y < C[1]; Y++)
                for (int X = 0; X < C[0]; X++) {
                    const long long I = X + (long long)C[0] * (Y + (long long)C[1] * Z);
                    const int Q3[3] = {X, Y, Z};
                    for (int a = 0; a < 3; a++) {
                        // fine faces crossing the coarse +a face: the +a faces of
                        // the children at coordinate 2 Q + 1 along a
                        double acc = 0.0;
                        for (int u = 0; u < 2; u++)
                            for (int v = 0; v < 2; v++) {
                                int f[3];
                                f[a] = 2 * Q3[a] + 1;
                                f[(a + 1) % 3] = 2 * Q3[(a + 1) % 3] + u;
                                f[(a + 2) % 3] = 2 * Q3[(a + 2) % 3] + v;
                                if (f[0] >= F[0] || f[1] >= F[1] || f[2] >= F[2]) continue;
                                acc += sg[a][f[0] + (long long)F[0] * (f[1] + (long long)F[1] * f[2])];
                            }
                        cs[a][I] = (float)(0.5 * acc);
                    }
                }
        });
        std::vector<float4> h4(NC);
        host_parallel(C[2], [&](int Z) {
            for (int Y = 0; Y < C[1]; Y++)
                for (int X = 0; X < C[0]; X++) {
                    const long long I = X + (long long)C[0] * (Y + (long long)C[1] * Z);
                    const long long xm = X == 0 ? I + C[0] - 1 : I - 1;
                    const long long ym = Y == 0 ? I + (long long)C[0] * (C[1] - 1) : I - C[0];
                    const long long zm = Z == 0 ? I + (long long)C[0] * C[1] * (C[2] - 1) : I - (long long)C[0] * C[1];
                    const double diag = (double)cs[0][I] + cs[1][I] + cs[2][I] + cs[0][xm] + cs[1][ym] + cs[2][zm];
                    h4[I] = make_float4(cs[0][I], cs[1][I], cs[2][I], diag > 0.0 ? (float)(1.0 / diag) : 0.f);
                }
        });
        MgLevel &ml = c.mg_lev[l];
        ml.nx = C[0];
        ml.ny = C[1];
        ml.nz = C[2];
        ml.N = (int)NC;
        ml.sig = (float4 *)A(NC * sizeof(float4));
        ml.e = (float *)A(NC * sizeof(float));
        ml.f = (float *)A(NC * sizeof(float));
        ml.t = (float *)A(NC * sizeof(float));
        if (!ml.sig || !ml.e || !ml.f || !ml.t) return nullptr;
        // inactive cells are never written and must read as 0
        if (cudaMemset(ml.e, 0, NC * sizeof(float)) != cudaSuccess ||
            cudaMemset(ml.t, 0, NC * sizeof(float)) != cudaSuccess)
            return "multigrid setup failed";
        if (staged_copy(c.stream, c.device, ml.sig, h4.data(), NC * sizeof(float4), false) != cudaSuccess)
            return "multigrid upload failed";
        if (l == nlev - 1 && NC <= MG_DENSE_CELLS) {
            const std::vector<float> M = coarse_pinv(C[0], C[1], C[2], h4);
            if (M.empty()) return "coarsest multigrid operator is not semi-definite";
            c.mg_dense = (float *)A(M.size() * sizeof(float));
            if (!c.mg_dense) return nullptr;
            if (cudaMemcpy(c.mg_dense, M.data(), M.size() * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess)
                return "multigrid upload failed";
        }
        for (int a = 0; a < 3; a++) sg[a].swap(cs[a]);
    }
    c.mg_lev[0].nx = c.nx;
    c.mg_lev[0].ny = c.ny;
    c.mg_lev[0].nz = c.nz;
    c.mg_lev[0].N = (int)N;
    c.mg_nlev = nlev;
    // block 0 takes every level from the first one of at most MG_CTA_CELLS
    // cells (their e and f in its shared memory); at least the coarsest
    int maxdyn = 0;
    cudaDeviceGetAttribute(&maxdyn, cudaDevAttrMaxSharedMemoryPerBlockOptin, c.device);
    c.mg_cta_from = nlev - 1;
    // per level: e and f (padded to 16 bytes) and the float4 conductances
    auto cta_bytes = [&](int from) {
        size_t bytes = 0;
        for (int k = from; k < nlev; k++)
            bytes += sizeof(float) * (((2 * (size_t)c.mg_lev[k].N + 3) & ~(size_t)3) + 4 * (size_t)c.mg_lev[k].N);
        return bytes;
    };
    for (int l = 1; l < nlev; l++)
        if (c.mg_lev[l].N <= MG_CTA_CELLS && cta_bytes(l) + 4096 <= (size_t)maxdyn) {
            c.mg_cta_from = l;
            break;
        }
    c.mg_smem = cta_bytes(c.mg_cta_from);
    if (c.mg_dense) {  // exact coarsest solve: every other level is grid-wide
        c.mg_cta_from = nlev - 1;
        c.mg_smem = 0;
    }
    // tiled smoothing from the first grid-wide coarse level small enough per
    // block; its region follows block 0's levels in the dynamic shared memory
    c.mg_tile_from = c.mg_cta_from;
    c.mg_tile_off = c.mg_smem / sizeof(float);
    size_t tile_words = 0;
    for (int l = 1; tiles && l < c.mg_cta_from; l++) {
        if ((long long)c.mg_lev[l].N > (long long)MG_TILE_CELLS_PER_BLOCK * c.pois_blocks) continue;
        if (c.mg_tile_from == c.mg_cta_from) c.mg_tile_from = l;
        const int ex[3] = {c.mg_lev[l].nx, c.mg_lev[l].ny, c.mg_lev[l].nz};
        mg_pick_tile(ex, 2 * MG_NU_COARSE, c.pois_blocks, 16, MG_TILE_BYTES, c.mg_tile[l], tile_words);
    }
    c.mg_smem += tile_words * sizeof(float);
    if (c.mg_smem + 4096 > (size_t)maxdyn) return "coarsest multigrid level too large for shared memory";
    // large lattices per SM make the lattice passes bandwidth-bound: twice the
    // warps in flight (1024-thread blocks) then beat the 512-thread launch
    // that keeps 128 registers a thread for the latency-bound small solve
    c.mg_wide = N >= (long long)MG_WIDE_NODES_PER_SM * c.num_sms;  // (replicas use the batched solve)
    // the solve runs split into per-pass launches (measured faster on every
    // lattice size tried: 64x64x128 0.53 against 0.57 ms, 256x256x512 8.3
    // against 14.4 ms), with the block size of the single launch it matches
    c.mg_split = split;
    c.mgs_threads = c.mg_wide ? MG_WIDE_THREADS : MG_THREADS;
    c.mgs_l1 = c.mg_split && c.mg_cta_from > 1 && c.mg_tile_from > 1;
    c.mgs_iter_kernels = 2 * (2 * MG_NU - 1) + 8 + (c.mgs_l1 ? 2 * (2 * MG_NU_COARSE - 1) + 2 : 0);
    if (ops(c.prec).mg_blocks(c.mg_smem, c.mg_wide) < 1) return "multigrid kernel cannot be resident";
    c.mg_r = (float *)A(N * sizeof(float));
    c.mg_link = (uint8_t *)A(N);
    c.mg_z = (float *)A(N * sizeof(float));
    c.mg_q = (float *)A(N * sizeof(float));
    c.mg_p[0] = (float *)A(N * sizeof(float));
    c.mg_p[1] = (float *)A(N * sizeof(float));
    c.mg_part = (double *)A((size_t)8 * c.pois_blocks * sizeof(double));
    c.mgs_ctl = A(sizeof(MgCtl));
    c.mg_phi_prev = A(N * phi_size(c.prec));
    c.mg_have_prev = 0;
    c.mg = 1;
    return nullptr;
}

}  // namespace

extern "C" {

int ekl_set_allocator(ekl_alloc_fn alloc, ekl_free_fn free_fn, void *ctx)
{
    if ((alloc == nullptr) != (free_fn == nullptr)) return fail(EKL_ERR_ARG, "allocator and free must both be set");
    g_alloc = alloc;
    g_free = free_fn;
    g_alloc_ctx = ctx;
    return EKL_OK;
}

int64_t ekl_sizeof_params(void) { return (int64_t)sizeof(ekl_params); }

const char *ekl_last_error(void) { return g_err; }

void ekl_lattice(int32_t *c, double *w, int32_t *opp)
{
    for (int p = 0; p < Q; p++) {
        c[3 * p] = cx_(p);
        c[3 * p + 1] = cy_(p);
        c[3 * p + 2] = cz_(p);
        w[p] = w_(p);
        opp[p] = opp_(p);
    }
}

// replica: a handle created for a batch (its multigrid hierarchy goes one
// level deeper, so that the host-built pseudo-inverse of each replica's
// coarsest level stays small to build and to read)
static int create_handle(const ekl_params *P, void *stream, ekl_handle **out, bool replica)
{
    g_err[0] = 0;
    if (!out) return fail(EKL_ERR_ARG, "out is null");
    *out = nullptr;
    if (!P || !P->solid) return fail(EKL_ERR_ARG, "params or solid map is null");
    if (P->nx < 2 || P->ny < 2 || P->nz < 2) return fail(EKL_ERR_ARG, "every extent must be >= 2");
    int L[3] = {P->nx, P->ny, P->nz};
    for (int a = 0; a < 3; a++)
        if (P->periodic[a] && (L[a] & 1)) return fail(EKL_ERR_ARG, "periodic extents must be even (red-black ordering)");
    if (P->precision < EKL_F64 || P->precision > EKL_FP16DEV) return fail(EKL_ERR_ARG, "unknown precision");
    for (int s = 0; s < NS; s++)
        if (!(P->tau[s] > 0.5)) return fail(EKL_ERR_ARG, "tau must exceed 1/2");
    if (!(P->diffusivity[1] > 0.0)) return fail(EKL_ERR_ARG, "cation diffusivity must be positive");
    if (!(P->fluct_mass >= 0.0) || !isfinite(P->fluct_mass)) return fail(EKL_ERR_ARG, "fluct_mass must be finite and >= 0");
    long long N = (long long)P->nx * P->ny * P->nz;
    if (N > (1ll << 31) / 64) return fail(EKL_ERR_ARG, "lattice too large for 32-bit node ids");

    ekl_handle *h = new (std::nothrow) ekl_handle();
    if (!h) return fail(EKL_ERR_ALLOC, "host allocation failed");
    Ctx &c = h->c;
    memset(&c, 0, sizeof(Ctx));
    c.P = *P;
    c.P.solid = nullptr;
    c.P.surface_charge = nullptr;
    c.P.n_init = nullptr;
    c.nx = P->nx;
    c.ny = P->ny;
    c.nz = P->nz;
    for (int a = 0; a < 3; a++) c.per[a] = P->periodic[a] ? 1 : 0;
    c.N = N;
    c.prec = P->precision;
    c.stream = (cudaStream_t)stream;
    cudaGetDevice(&c.device);
    cudaDeviceGetAttribute(&c.num_sms, cudaDevAttrMultiProcessorCount, c.device);
    if (c.P.md_substeps < 1) c.P.md_substeps = 1;
    if (c.P.poisson_check_every < 1) c.P.poisson_check_every = 1;

    // constants, each as the oracle's formula states it
    const double VT2 = 1.0 / 3.0;
    c.c4 = 4.0 * M_PI * P->bjerrum;
    for (int s = 0; s < NS; s++) {
        double D = P->diffusivity[s] > 0.0 ? P->diffusivity[s] : P->diffusivity[1];
        c.wd[s] = VT2 / D;
        c.om[s] = 1.0 / P->tau[s];
    }
    if (P->rho_jacobi > 0.0) {
        c.rJ = P->rho_jacobi;
    } else {
        double th = 1e30;
        for (int a = 0; a < 3; a++) {
            double t = (c.per[a] ? 2.0 : 1.0) * M_PI / L[a];
            if (t < th) th = t;
        }
        c.rJ = (2.0 + cos(th)) / 3.0;
    }

    // geometry on the host: fluid count, wall charge shares
    const uint8_t *solid = P->solid;
    long long nf = 0;
    {
        const long long plane = (long long)c.nx * c.ny;
        std::vector<long long> nfz(c.nz, 0);
        host_parallel(c.nz, [&](int z) {
            long long k = 0;
            for (long long i = z * plane; i < (z + 1) * plane; i++) k += solid[i] ? 0 : 1;
            nfz[z] = k;
        });
        for (int z = 0; z < c.nz; z++) nf += nfz[z];
    }
    c.n_fluid = nf;
    bool charged = false;
    if (P->surface_charge)
        for (long long i = 0; i < N; i++)
            if (solid[i] && P->surface_charge[i] != 0.0) charged = true;
    std::vector<double> share, src;
    if (charged) {
        share.assign(N, 0.0);
        src.assign(N, 0.0);
        const int F[6][3] = {{-1, 0, 0}, {1, 0, 0}, {0, -1, 0}, {0, 1, 0}, {0, 0, -1}, {0, 0, 1}};
        auto nid = [&](int x, int y, int z, bool &in) -> long long {
            int q[3] = {x, y, z};
            in = true;
            for (int a = 0; a < 3; a++) {
                if (c.per[a]) {
                    q[a] %= L[a];
                    if (q[a] < 0) q[a] += L[a];
                } else if (q[a] < 0 || q[a] >= L[a]) {
                    in = false;
                }
            }
            return in ? (long long)q[0] + (long long)L[0] * (q[1] + (long long)L[1] * q[2]) : -1;
        };
        for (long long w = 0; w < N; w++) {
            if (!solid[w] || P->surface_charge[w] == 0.0) continue;
            int x = (int)(w % L[0]), y = (int)((w / L[0]) % L[1]), z = (int)(w / ((long long)L[0] * L[1]));
            int k = 0;
            for (int f = 0; f < 6; f++) {
                bool in;
                long long j = nid(x + F[f][0], y + F[f][1], z + F[f][2], in);
                if (in && !solid[j]) k++;
            }
            if (k > 0) share[w] = P->surface_charge[w] / k;
        }
        for (long long i = 0; i < N; i++) {
            if (solid[i]) continue;
            int x = (int)(i % L[0]), y = (int)((i / L[0]) % L[1]), z = (int)(i / ((long long)L[0] * L[1]));
            double acc = 0.0;
            for (int f = 0; f < 6; f++) {
                bool in;
                long long j = nid(x + F[f][0], y + F[f][1], z + F[f][2], in);
                if (in && solid[j]) acc += share[j];
            }
            src[i] = acc;
        }
    }

    // device buffers
    const size_t rs = real_size(c.prec), ss = store_size(c.prec), ps = phi_size(c.prec);
    c.charge_blocks = (int)((N + CHARGE_THREADS - 1) / CHARGE_THREADS);
    c.lb_blocks = (int)((N + LB_THREADS - 1) / LB_THREADS);
    int occ = ops(c.prec).pois_blocks();
    if (occ < 1) {
        delete h;
        return fail(EKL_ERR_CUDA, "Poisson kernel cannot be resident");
    }
    c.pois_blocks = c.num_sms;  // one block of POIS_THREADS per SM
    // Shared-memory tiles for the SOR kernel: full-x slabs of ty x tz rows,
    // one per SM, each with a 2-deep halo; chosen to minimise the extended
    // tile (per-block work and halo traffic).  Periodic y/z extents are even.
    {
        int maxdyn = 0;
        cudaDeviceGetAttribute(&maxdyn, cudaDevAttrMaxSharedMemoryPerBlockOptin, c.device);
        const size_t per_node = 2 * phi_size(c.prec) + sizeof(uint32_t);
        long long best = -1;
        if (!(P->flags & EKL_POISSON_GLOBAL))
            for (int ty = 2; ty <= c.ny; ty++) {
                if (c.ny % ty) continue;
                for (int tz = 2; tz <= c.nz; tz++) {
                    if (c.nz % tz) continue;
                    const int nt = (c.ny / ty) * (c.nz / tz);
                    const long long E = (long long)c.nx * (ty + 4) * (tz + 4);
                    if (nt > c.num_sms || (size_t)E * per_node + 1024 > (size_t)maxdyn) continue;
                    if (best < 0 || E < best || (E == best && nt > c.tile_nty * c.tile_ntz)) {
                        best = E;
                        c.tile_ty = ty;
                        c.tile_tz = tz;
                        c.tile_nty = c.ny / ty;
                        c.tile_ntz = c.nz / tz;
                    }
                }
            }
        c.pois_tiled = best > 0;
    }
    bool okall = true;
    auto A = [&](size_t bytes) {
        void *p = dev_alloc(c, bytes);
        if (!p) okall = false;
        return p;
    };
    c.f[0] = A((size_t)NS * Q * N * ss);
    c.f[1] = A((size_t)NS * Q * N * ss);
    c.mask = (uint32_t *)A(N * 4);
    if (charged) {
        c.wall_share = A(N * rs);
        c.src_wall = A(N * rs);
    }
    c.rho = A(N * rs);
    c.b = A(N * ps);
    c.phi = A(N * ps);
    c.part_charge = (double *)A((size_t)c.charge_blocks * (CHARGE_THREADS / 32) * sizeof(double));
    c.part_charge_q = (long long *)A((size_t)c.charge_blocks * sizeof(long long));
    c.charge_tot = (double *)A(sizeof(double));
    c.charge_tot_q = (long long *)A(sizeof(long long));
    c.charge_chunks = A(CHARGE_CHUNK_BYTES);
    c.part_mass = (double *)A((size_t)((N + 255) / 256) * NS * sizeof(double));
    c.part_pois = (double *)A((size_t)c.pois_blocks * sizeof(double));
    c.barrier = (unsigned *)A(4 * sizeof(unsigned));
    c.status = (int *)A(sizeof(int));
    c.pois_iters = (int *)A(sizeof(int));
    c.pois_total = (long long *)A(sizeof(long long));
    c.pois_res = (double *)A(sizeof(double));
    // Chebyshev schedule (Sec. II.C, Press et al.): 1 for the first half
    // sweep, 1/(1 - rJ^2/2) for the second, then 1/(1 - rJ^2 omega/4)
    const int limit = (c.P.poisson_fixed_iter > c.P.poisson_max_iter ? c.P.poisson_fixed_iter : c.P.poisson_max_iter) + 1;
    std::vector<double> om(2 * (size_t)limit);
    const double rJ = c.rJ;
    for (size_t k = 0; k < om.size(); k++)
        om[k] = k == 0 ? 1.0 : (k == 1 ? 1.0 / (1.0 - 0.5 * rJ * rJ) : 1.0 / (1.0 - 0.25 * rJ * rJ * om[k - 1]));
    std::vector<float> omf(om.begin(), om.end());
    c.omegas = A(om.size() * (c.prec == EKL_F64 ? sizeof(double) : sizeof(float)));
    if (P->fluct_mass > 0.0) c.wchi = A((size_t)Q * Q * rs);
    c.patch_count = (int *)A(sizeof(int));
    c.patch_bits = (uint32_t *)A(((size_t)N / 32 + 1) * sizeof(uint32_t));
    c.patch_node = (int *)A(MAX_ENTRIES * sizeof(int));
    c.patch_q = A(MAX_ENTRIES * rs);
    c.patch_f = A((size_t)(MAX_ENTRIES + MAX_BEADS) * 9 * rs);
    c.patch_mom = A((size_t)MAX_ENTRIES * 15 * rs);
    c.entry_slot = (int *)A(MAX_ENTRIES * sizeof(int));
    c.sorted_entry = (int *)A(MAX_ENTRIES * sizeof(int));
    c.slot_first = (int *)A((MAX_ENTRIES + 1) * sizeof(int));
    c.entry_w = A(MAX_ENTRIES * rs);
    c.R = A(MAX_BEADS * 3 * sizeof(double));  // bead positions are FP64 in every precision
    c.V = A(MAX_BEADS * 3 * rs);
    c.q = A(MAX_BEADS * rs);
    c.chain = (int *)A(MAX_BEADS * sizeof(int));
    if (!okall) {
        release(c);
        delete h;
        return fail(EKL_ERR_ALLOC, "device allocation failed");
    }
    if (P->flags & EKL_POISSON_MG) {
        const bool tiles = !replica && !(P->flags & EKL_POISSON_GLOBAL);
        const bool split = !replica && !(P->flags & EKL_POISSON_MG_SINGLE);
        const char *why =
            build_multigrid(c, solid, A, replica ? MG_COARSEST_CELLS_REPLICA : MG_COARSEST_CELLS, tiles, split);
        if (!why && !okall) why = "device allocation failed";
        if (why) {
            release(c);
            delete h;
            return fail(okall ? EKL_ERR_ARG : EKL_ERR_ALLOC, why);
        }
    }
    for (int k = 0; k < 2 * PH_COUNT; k++) cudaEventCreate(&c.ev[k]);

    int rc = EKL_OK;
    uint8_t *d_solid = nullptr;
    double *d_n = nullptr;
    cudaError_t e = cudaSuccess;
    do {
        d_solid = (uint8_t *)dev_alloc(c, N);
        if (!d_solid) { rc = fail(EKL_ERR_ALLOC, "device allocation failed"); break; }
        e = cudaMemcpyAsync(d_solid, solid, N, cudaMemcpyHostToDevice, c.stream);
        if (e != cudaSuccess) { rc = fail_cuda(e, "upload solid"); break; }
        e = cudaMemsetAsync(c.charge_chunks, 0, CHARGE_CHUNK_BYTES, c.stream);
        if (e != cudaSuccess) { rc = fail_cuda(e, "clear charge totals"); break; }
        mask_kernel<<<(unsigned)((N + 255) / 256), 256, 0, c.stream>>>(make_grid3(c.nx, c.ny, c.nz), c.per[0], c.per[1], c.per[2], d_solid, c.mask);
        c.launches++;
        if (c.mg) {
            mg_link_kernel<<<(unsigned)((N + 255) / 256), 256, 0, c.stream>>>(c.mask, c.mg_link, N);
            c.launches++;
        }
        if (charged) {
            if (c.prec == EKL_F64) {
                cudaMemcpyAsync(c.wall_share, share.data(), N * 8, cudaMemcpyHostToDevice, c.stream);
                cudaMemcpyAsync(c.src_wall, src.data(), N * 8, cudaMemcpyHostToDevice, c.stream);
            } else {
                std::vector<float> a(N), b(N);
                for (long long i = 0; i < N; i++) {
                    a[i] = (float)share[i];
                    b[i] = (float)src[i];
                }
                cudaMemcpyAsync(c.wall_share, a.data(), N * 4, cudaMemcpyHostToDevice, c.stream);
                cudaMemcpyAsync(c.src_wall, b.data(), N * 4, cudaMemcpyHostToDevice, c.stream);
                cudaStreamSynchronize(c.stream);
            }
        }
        if (P->n_init) {
            d_n = (double *)dev_alloc(c, (size_t)NS * N * 8);
            if (!d_n) { rc = fail(EKL_ERR_ALLOC, "device allocation failed"); break; }
            e = staged_copy(c.stream, c.device, d_n, P->n_init, (size_t)NS * N * 8, false);
            if (e != cudaSuccess) { rc = fail_cuda(e, "upload n_init"); break; }
        }
        rc = ops(c.prec).init(c, d_n);
        if (rc != EKL_OK) { fail(rc, "init kernel failed"); break; }
        cudaMemsetAsync(c.phi, 0, N * ps, c.stream);
        cudaMemsetAsync(c.patch_count, 0, sizeof(int), c.stream);
        cudaMemsetAsync(c.patch_bits, 0, ((size_t)N / 32 + 1) * sizeof(uint32_t), c.stream);
        cudaMemsetAsync(c.status, 0, sizeof(int), c.stream);
        cudaMemsetAsync(c.pois_iters, 0, sizeof(int), c.stream);
        cudaMemsetAsync(c.pois_total, 0, sizeof(long long), c.stream);
        cudaMemsetAsync(c.pois_res, 0, sizeof(double), c.stream);
        if (c.prec == EKL_F64) cudaMemcpyAsync(c.omegas, om.data(), om.size() * 8, cudaMemcpyHostToDevice, c.stream);
        else cudaMemcpyAsync(c.omegas, omf.data(), omf.size() * 4, cudaMemcpyHostToDevice, c.stream);
        if (c.wchi) {
            double wchi[Q][Q];
            fluct_basis(wchi);
            if (c.prec == EKL_F64) {
                e = cudaMemcpy(c.wchi, wchi, sizeof(wchi), cudaMemcpyHostToDevice);
            } else {
                float wf[Q * Q];
                for (int k = 0; k < Q * Q; k++) wf[k] = (float)(&wchi[0][0])[k];
                e = cudaMemcpy(c.wchi, wf, sizeof(wf), cudaMemcpyHostToDevice);
            }
            if (e != cudaSuccess) { rc = fail_cuda(e, "upload basis"); break; }
        }

        e = cudaStreamSynchronize(c.stream);
        if (e != cudaSuccess) { rc = fail_cuda(e, "create"); break; }
    } while (0);
    dev_free(c, d_solid, N);
    dev_free(c, d_n, 0);
    if (rc != EKL_OK) {
        release(c);
        delete h;
        return rc;
    }
    *out = h;
    return EKL_OK;
}

int ekl_create(const ekl_params *P, void *stream, ekl_handle **out) { return create_handle(P, stream, out, false); }

int ekl_set_beads(ekl_handle *h, int32_t n, const double *R, const double *V, const double *q,
                  const int32_t *chain)
{
    if (!h) return fail(EKL_ERR_ARG, "null handle");
    DeviceScope dscope(h->c.device);
    if (!dscope.ok()) return fail(EKL_ERR_ARG, "the handle's device cannot be made current");
    if (n < 0 || n > MAX_BEADS) return fail(EKL_ERR_ARG, "bead count out of range (max 256)");
    if (n > 0 && (!R || !q)) return fail(EKL_ERR_ARG, "positions and charges are required");
    Ctx &c = h->c;
    for (int b = 0; b < n; b++)
        for (int a = 0; a < 3; a++) {
            double L = a == 0 ? c.nx : (a == 1 ? c.ny : c.nz);
            double r = R[3 * b + a];
            if (!(r >= 0.0 && r < L)) return fail(EKL_ERR_ARG, "bead position outside [0, L)");
        }
    std::vector<double> Rd(3 * (size_t)n), Vd(3 * (size_t)n, 0.0), qd(n);
    std::vector<int> ch(n, 0);
    for (int k = 0; k < 3 * n; k++) {
        Rd[k] = R[k];
        if (V) Vd[k] = V[k];
    }
    for (int k = 0; k < n; k++) {
        qd[k] = q[k];
        if (chain) ch[k] = chain[k];
    }
    cudaError_t e = cudaMemcpyAsync(c.R, Rd.data(), 3 * (size_t)n * 8, cudaMemcpyHostToDevice, c.stream);
    if (c.prec == EKL_F64) {
        if (e == cudaSuccess) e = cudaMemcpyAsync(c.V, Vd.data(), 3 * (size_t)n * 8, cudaMemcpyHostToDevice, c.stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(c.q, qd.data(), (size_t)n * 8, cudaMemcpyHostToDevice, c.stream);
    } else {
        std::vector<float> Vf(Vd.begin(), Vd.end()), qf(qd.begin(), qd.end());
        if (e == cudaSuccess) e = cudaMemcpyAsync(c.V, Vf.data(), 3 * (size_t)n * 4, cudaMemcpyHostToDevice, c.stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(c.q, qf.data(), (size_t)n * 4, cudaMemcpyHostToDevice, c.stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c.stream);
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(c.chain, ch.data(), (size_t)n * sizeof(int), cudaMemcpyHostToDevice, c.stream);
    if (e == cudaSuccess && n == 0) e = cudaMemsetAsync(c.patch_count, 0, sizeof(int), c.stream);
    if (e == cudaSuccess && n == 0)
        e = cudaMemsetAsync(c.patch_bits, 0, ((size_t)c.N / 32 + 1) * sizeof(uint32_t), c.stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c.stream);
    if (e != cudaSuccess) return fail_cuda(e, "set_beads");
    c.nb = n;
    return EKL_OK;
}

int ekl_step_async(ekl_handle *h, int32_t nsteps)
{
    if (!h) return fail(EKL_ERR_ARG, "null handle");
    DeviceScope dscope(h->c.device);
    if (!dscope.ok()) return fail(EKL_ERR_ARG, "the handle's device cannot be made current");
    if (nsteps < 0) return fail(EKL_ERR_ARG, "negative step count");
    int rc = ops(h->c.prec).run(h->c, nsteps);
    if (rc != EKL_OK) return fail(rc, "kernel launch failed");
    return EKL_OK;
}

int ekl_step(ekl_handle *h, int32_t nsteps)
{
    if (!h) return fail(EKL_ERR_ARG, "null handle");
    DeviceScope dscope(h->c.device);
    if (!dscope.ok()) return fail(EKL_ERR_ARG, "the handle's device cannot be made current");
    Ctx &c = h->c;
    cudaMemsetAsync(c.status, 0, sizeof(int), c.stream);
    int rc = ekl_step_async(h, nsteps);
    if (rc != EKL_OK) return rc;
    int st = 0;
    cudaError_t e = cudaMemcpyAsync(&st, c.status, sizeof(int), cudaMemcpyDeviceToHost, c.stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c.stream);
    if (e != cudaSuccess) return fail_cuda(e, "step");
    timing_flush(c);
    c.last_status = st;
    return status_to_code(st);
}

int ekl_get_fields(ekl_handle *h, double *n_out, double *j_out, double *phi_out, double *R_out,
                   double *V_out)
{
    if (!h) return fail(EKL_ERR_ARG, "null handle");
    DeviceScope dscope(h->c.device);
    if (!dscope.ok()) return fail(EKL_ERR_ARG, "the handle's device cannot be made current");
    Ctx &c = h->c;
    const long long N = c.N;
    double *dn = n_out ? (double *)dev_alloc(c, (size_t)NS * N * 8) : nullptr;
    double *dj = j_out ? (double *)dev_alloc(c, (size_t)NS * 3 * N * 8) : nullptr;
    // the potential, then the gauge's block partials
    double *dp = phi_out ? (double *)dev_alloc(c, ((size_t)N + 2 * GAUGE_BLOCKS) * 8) : nullptr;
    if ((n_out && !dn) || (j_out && !dj) || (phi_out && !dp)) {
        dev_free(c, dn, 0);
        dev_free(c, dj, 0);
        dev_free(c, dp, 0);
        return fail(EKL_ERR_ALLOC, "device allocation failed");
    }
    int rc = ops(c.prec).fields(c, dn, dj, dp);
    cudaError_t e = cudaSuccess;
    if (rc == EKL_OK && dp) {
        // gauge on the device: remove the fluid mean (deterministic sum)
        gauge_partials_kernel<<<GAUGE_BLOCKS, GAUGE_THREADS, 0, c.stream>>>(dp, c.mask, N, dp + N);
        gauge_apply_kernel<<<c.num_sms * 2, GAUGE_THREADS, 0, c.stream>>>(c.mask, N, dp, dp + N);
        c.launches += 2;
        e = cudaGetLastError();
    }
    if (rc == EKL_OK && e == cudaSuccess) {
        if (dn) e = staged_copy(c.stream, c.device, n_out, dn, (size_t)NS * N * 8, true);
        if (e == cudaSuccess && dj) e = staged_copy(c.stream, c.device, j_out, dj, (size_t)NS * 3 * N * 8, true);
        if (e == cudaSuccess && dp) e = staged_copy(c.stream, c.device, phi_out, dp, (size_t)N * 8, true);
        if (c.nb > 0 && e == cudaSuccess && (R_out || V_out)) {
            size_t vbytes = 3 * (size_t)c.nb * real_size(c.prec);
            std::vector<double> r(3 * (size_t)c.nb);
            std::vector<char> v(vbytes);
            e = cudaMemcpyAsync(r.data(), c.R, 3 * (size_t)c.nb * 8, cudaMemcpyDeviceToHost, c.stream);
            if (e == cudaSuccess) e = cudaMemcpyAsync(v.data(), c.V, vbytes, cudaMemcpyDeviceToHost, c.stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(c.stream);
            for (int k = 0; k < 3 * c.nb && e == cudaSuccess; k++) {
                double vv = c.prec == EKL_F64 ? ((double *)v.data())[k] : (double)((float *)v.data())[k];
                if (R_out) R_out[k] = r[k];
                if (V_out) V_out[k] = vv;
            }
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(c.stream);
    }
    dev_free(c, dn, 0);
    dev_free(c, dj, 0);
    dev_free(c, dp, 0);
    if (rc != EKL_OK) return fail(rc, "fields kernel failed");
    if (e != cudaSuccess) return fail_cuda(e, "get_fields");
    return EKL_OK;
}

int ekl_get_state(ekl_handle *h, double *fstar, double *phi, int64_t *step)
{
    if (!h) return fail(EKL_ERR_ARG, "null handle");
    DeviceScope dscope(h->c.device);
    if (!dscope.ok()) return fail(EKL_ERR_ARG, "the handle's device cannot be made current");
    Ctx &c = h->c;
    double *df = fstar ? (double *)dev_alloc(c, (size_t)NS * Q * c.N * 8) : nullptr;
    double *dp = phi ? (double *)dev_alloc(c, (size_t)c.N * 8) : nullptr;
    if ((fstar && !df) || (phi && !dp)) {
        dev_free(c, df, 0);
        dev_free(c, dp, 0);
        return fail(EKL_ERR_ALLOC, "device allocation failed");
    }
    int rc = ops(c.prec).get_state(c, df ? df : nullptr, dp);
    cudaError_t e = cudaSuccess;
    if (rc == EKL_OK && df) e = staged_copy(c.stream, c.device, fstar, df, (size_t)NS * Q * c.N * 8, true);
    if (rc == EKL_OK && e == cudaSuccess && dp) e = staged_copy(c.stream, c.device, phi, dp, (size_t)c.N * 8, true);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c.stream);
    dev_free(c, df, 0);
    dev_free(c, dp, 0);
    if (rc != EKL_OK) return fail(rc, "state kernel failed");
    if (e != cudaSuccess) return fail_cuda(e, "get_state");
    if (step) *step = c.step;
    return EKL_OK;
}

int ekl_set_state(ekl_handle *h, const double *fstar, const double *phi, int64_t step)
{
    if (!h || !fstar) return fail(EKL_ERR_ARG, "null handle or populations");
    DeviceScope dscope(h->c.device);
    if (!dscope.ok()) return fail(EKL_ERR_ARG, "the handle's device cannot be made current");
    Ctx &c = h->c;
    double *df = (double *)dev_alloc(c, (size_t)NS * Q * c.N * 8);
    double *dp = phi ? (double *)dev_alloc(c, (size_t)c.N * 8) : nullptr;
    if (!df || (phi && !dp)) {
        dev_free(c, df, 0);
        dev_free(c, dp, 0);
        return fail(EKL_ERR_ALLOC, "device allocation failed");
    }
    cudaError_t e = staged_copy(c.stream, c.device, df, fstar, (size_t)NS * Q * c.N * 8, false);
    if (e == cudaSuccess && dp) e = staged_copy(c.stream, c.device, dp, phi, (size_t)c.N * 8, false);
    int rc = e == cudaSuccess ? ops(c.prec).set_state(c, df, dp) : EKL_ERR_CUDA;
    if (e == cudaSuccess) e = cudaStreamSynchronize(c.stream);
    dev_free(c, df, 0);
    dev_free(c, dp, 0);
    if (rc != EKL_OK || e != cudaSuccess) return fail_cuda(e, "set_state");
    c.step = step;
    c.mg_have_prev = 0;  // the potential history no longer matches
    return EKL_OK;
}

int ekl_get_stats(ekl_handle *h, ekl_stats *out)
{
    if (!h || !out) return fail(EKL_ERR_ARG, "null argument");
    DeviceScope dscope(h->c.device);
    if (!dscope.ok()) return fail(EKL_ERR_ARG, "the handle's device cannot be made current");
    Ctx &c = h->c;
    const int nmb = ops(c.prec).mass(c);
    if (nmb < 0) return fail(EKL_ERR_CUDA, "mass kernel failed");
    const size_t nwarps = (size_t)nmb;
    std::vector<double> pm(nwarps * NS);
    int it = 0;
    long long tot = 0;
    double res = 0;
    cudaError_t e = cudaMemcpyAsync(pm.data(), c.part_mass, pm.size() * 8, cudaMemcpyDeviceToHost, c.stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&it, c.pois_iters, sizeof(int), cudaMemcpyDeviceToHost, c.stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&res, c.pois_res, sizeof(double), cudaMemcpyDeviceToHost, c.stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&tot, c.pois_total, sizeof(long long), cudaMemcpyDeviceToHost, c.stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c.stream);
    if (e != cudaSuccess) return fail_cuda(e, "get_stats");
    timing_flush(c);
    memset(out, 0, sizeof(*out));
    for (int s = 0; s < NS; s++) {
        double t = 0;
        for (size_t b = 0; b < nwarps; b++) t += pm[b * NS + s];
        out->mass[s] = t;
    }
    out->step = c.step;
    out->poisson_iters = it;
    out->poisson_res = res;
    out->status = c.last_status;
    for (int k = 0; k < PH_COUNT; k++) out->ms_phase[k] = c.ms_phase[k];
    // a split multigrid solve launches its loop's kernels from the device
    out->launches = c.launches + (c.mg_split ? (int64_t)c.mgs_iter_kernels * tot : 0);
    out->poisson_sweeps = tot;
    return EKL_OK;
}

int ekl_selftest_wait(void)
{
    unsigned *bar = nullptr;
    int *status = nullptr;
    cudaError_t e = cudaMalloc(&bar, 4 * sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMalloc(&status, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(bar, 0, 4 * sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMemset(status, 0, sizeof(int));
    if (e == cudaSuccess) {
        wait_selftest_kernel<<<2, 32>>>(bar, status);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    int st = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&st, status, sizeof(int), cudaMemcpyDeviceToHost);
    cudaFree(bar);
    cudaFree(status);
    if (e != cudaSuccess) return fail_cuda(e, "selftest_wait");
    if (st & ST_TIMEOUT) return fail(EKL_ERR_TIMEOUT, "a device-side wait timed out");
    return EKL_OK;
}

int ekl_set_field(ekl_handle *h, const double E[3])
{
    if (!h || !E) return fail(EKL_ERR_ARG, "null argument");
    for (int a = 0; a < 3; a++)
        if (!isfinite(E[a])) return fail(EKL_ERR_ARG, "field must be finite");
    for (int a = 0; a < 3; a++) h->c.P.E_app[a] = E[a];
    if (h->c.batch_ready) *h->c.batch_ready = 0;  // the batch's descriptor tables carry the field
    return EKL_OK;
}

int ekl_get_current(ekl_handle *h, int32_t axis, int32_t plane, double out[4])
{
    if (!h || !out) return fail(EKL_ERR_ARG, "null argument");
    DeviceScope dscope(h->c.device);
    if (!dscope.ok()) return fail(EKL_ERR_ARG, "the handle's device cannot be made current");
    Ctx &c = h->c;
    const int L[3] = {c.nx, c.ny, c.nz};
    if (axis < 0 || axis > 2 || plane < 0 || plane >= L[axis]) return fail(EKL_ERR_ARG, "axis or plane out of range");
    const int n1 = axis == 0 ? c.ny : c.nx, n2 = axis == 2 ? c.ny : c.nz;
    const int blocks = (n1 * n2 + 255) / 256;
    double *part = (double *)dev_alloc(c, (size_t)blocks * NS * sizeof(double));
    if (!part) return fail(EKL_ERR_ALLOC, "device allocation failed");
    const int nb = ops(c.prec).current(c, axis, plane, part);
    std::vector<double> h_part((size_t)blocks * NS);
    cudaError_t e = nb < 0 ? cudaErrorLaunchFailure
                           : cudaMemcpyAsync(h_part.data(), part, h_part.size() * 8, cudaMemcpyDeviceToHost, c.stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c.stream);
    dev_free(c, part, 0);
    if (e != cudaSuccess) return fail_cuda(e, "get_current");
    double total = 0.0;
    for (int s = 0; s < NS; s++) {
        double t = 0.0;
        for (int b = 0; b < blocks; b++) t += h_part[(size_t)b * NS + s];
        out[s] = t;
        total += (double)c.P.valence[s] * t;
    }
    out[3] = total;
    return EKL_OK;
}

int ekl_set_timing(ekl_handle *h, int32_t on)
{
    if (!h) return fail(EKL_ERR_ARG, "null handle");
    DeviceScope dscope(h->c.device);
    if (!dscope.ok()) return fail(EKL_ERR_ARG, "the handle's device cannot be made current");
    cudaStreamSynchronize(h->c.stream);
    timing_flush(h->c);
    h->c.timing = on ? 1 : 0;
    for (int k = 0; k < PH_COUNT; k++) h->c.ms_phase[k] = 0.0;
    return EKL_OK;
}

int ekl_get_link_mask(ekl_handle *h, uint32_t *mask_out)
{
    if (!h || !mask_out) return fail(EKL_ERR_ARG, "null argument");
    DeviceScope dscope(h->c.device);
    if (!dscope.ok()) return fail(EKL_ERR_ARG, "the handle's device cannot be made current");
    cudaError_t e = cudaMemcpyAsync(mask_out, h->c.mask, h->c.N * 4, cudaMemcpyDeviceToHost, h->c.stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->c.stream);
    if (e != cudaSuccess) return fail_cuda(e, "get_link_mask");
    return EKL_OK;
}

void ekl_destroy(ekl_handle *h)
{
    if (!h) return;
    DeviceScope dscope(h->c.device);
    cudaStreamSynchronize(h->c.stream);
    release(h->c);
    delete h;
}

int ekl_test_set_device(ekl_handle *h, int32_t device)
{
    if (!h) return fail(EKL_ERR_ARG, "null handle");
    h->c.device = device;
    return EKL_OK;
}

}  // extern "C"

// ------------------------------------------------------------------ batches
namespace {

int batch_run(Batch &B, int nsteps)
{
    switch (B.prec) {
    case EKL_F64: return run_batch_f64(B, nsteps);
    case EKL_F32: return run_batch_f32(B, nsteps);
    case EKL_BF16DEV: return run_batch_bf16(B, nsteps);
    default: return run_batch_fp16(B, nsteps);
    }
}

// Poisson schedule `choice` (bit 1: blocks shared by fluid nodes, else by
// all nodes; bit 0: SOR on 512-thread blocks two per SM, or the split
// multigrid solve's lattice passes on MGS_MAX_FACTOR times the blocks)
int batch_schedule(Batch &B, int choice)
{
    const int sms = B.reps[0]->num_sms;
    if (choice < 0 || choice > 3) return EKL_ERR_ARG;
    if (B.mg) {
        // the cooperative multigrid launch keeps one 1024-thread block per SM
        if ((choice & 1) && !B.mgs_split) return EKL_ERR_ARG;
        B.pois_threads = MG_BATCH_THREADS;
        B.pois_blocks = sms;
        B.mgs_factor = (choice & 1) ? MGS_MAX_FACTOR : 1;
    } else {
        B.pois_threads = (choice & 1) ? 512 : 1024;
        B.pois_blocks = (choice & 1) ? 2 * sms : sms;
    }
    if (B.nrep > B.pois_blocks) return EKL_ERR_ARG;
    B.weight_fluid = (choice >> 1) & 1;
    B.ready = 0;
    return EKL_OK;
}

void batch_release(Batch &B)
{
    if (!B.reps) return;
    Ctx &c0 = *B.reps[0];
    for (int q = 0; q < 2; q++) {
        dev_free(c0, B.d_args[q], 0);
        dev_free(c0, B.d_bargs[q], 0);
        dev_free(c0, B.d_mdargs[q], 0);
    }
    dev_free(c0, B.d_block_rep, 0);
    dev_free(c0, B.d_block_local, 0);
    dev_free(c0, B.d_rep_blocks, 0);
    dev_free(c0, B.barrier, 0);
    dev_free(c0, B.status, 0);
    dev_free(c0, B.d_mgargs, 0);
    dev_free(c0, B.d_ctot, 0);
    dev_free(c0, B.mg_bars, 0);
    if (B.mgs_exec) cudaGraphExecDestroy(B.mgs_exec);
    if (B.mgs_graph) cudaGraphDestroy(B.mgs_graph);
    B.mgs_exec = nullptr;
    B.mgs_graph = nullptr;
    dev_free(c0, B.d_ctl, 0);
    dev_free(c0, B.d_grids, 0);
    dev_free(c0, B.d_loops, 0);
    dev_free(c0, B.d_lrep, 0);
    dev_free(c0, B.d_lloc, 0);
    dev_free(c0, B.d_lrb, 0);
    dev_free(c0, B.d_crep, 0);
    dev_free(c0, B.d_cloc, 0);
    dev_free(c0, B.d_crb, 0);
    dev_free(c0, B.d_mgs_part, 0);
}

}  // namespace

extern "C" {

int ekl_batch_create(int32_t nrep, const ekl_params *params, void *stream, ekl_batch **out)
{
    if (!out) return fail(EKL_ERR_ARG, "out is null");
    *out = nullptr;
    if (nrep < 1 || nrep > MAX_REPS || !params) return fail(EKL_ERR_ARG, "replica count out of range (1..256)");
    for (int r = 1; r < nrep; r++)
        if (params[r].precision != params[0].precision) return fail(EKL_ERR_ARG, "replicas must share one precision");
    ekl_batch *bh = new (std::nothrow) ekl_batch();
    if (!bh) return fail(EKL_ERR_ALLOC, "host allocation failed");
    Batch &B = bh->b;
    B.nrep = nrep;
    B.reps = new Ctx *[nrep]();
    B.handles = new void *[nrep]();
    B.stream = (cudaStream_t)stream;
    B.prec = params[0].precision;
    int rc = EKL_OK;
    for (int r = 0; r < nrep && rc == EKL_OK; r++) {
        ekl_handle *h = nullptr;
        rc = create_handle(&params[r], stream, &h, true);
        if (rc == EKL_OK) {
            B.handles[r] = h;
            B.reps[r] = &h->c;
            h->c.batch_ready = &B.ready;
        }
    }
    int sms = rc == EKL_OK ? B.reps[0]->num_sms : 0;
    if (rc == EKL_OK && nrep > sms) rc = fail(EKL_ERR_ARG, "more replicas than SMs for the batched Poisson launch");
    if (rc == EKL_OK) {
        Ctx &c0 = *B.reps[0];
        size_t sa = 0, sb = 0, sm = 0;
        switch (B.prec) {  // descriptor sizes per precision
        case EKL_F64:
            sa = sizeof(StepArgs<double, double, double>);
            sb = sizeof(BeadArgs<double>);
            sm = sizeof(MdArgs<double, double, double, false>);
            break;
        default:
            sa = sizeof(StepArgs<float, float, long long>);
            sb = sizeof(BeadArgs<float>);
            sm = sizeof(MdArgs<float, float, long long, true>);
            break;
        }
        bool ok = true;
        auto A = [&](size_t bytes) {
            void *p = dev_alloc(c0, bytes);
            if (!p) ok = false;
            return p;
        };
        for (int q = 0; q < 2; q++) {
            B.d_args[q] = A(nrep * sa);
            B.d_bargs[q] = A(nrep * sb);
            B.d_mdargs[q] = A(nrep * sm);
        }
        B.d_block_rep = (int *)A(4 * (size_t)sms * 2);
        B.d_block_local = (int *)A(4 * (size_t)sms * 2);
        B.d_rep_blocks = (int *)A(4 * (size_t)nrep);
        B.d_ctot = A(sizeof(ChargeTotals) * (size_t)nrep);
        B.barrier = (unsigned *)A(4 * sizeof(unsigned));
        B.status = (int *)A(sizeof(int));
        if (!ok) rc = fail(EKL_ERR_ALLOC, "device allocation failed");
        else {
            cudaMemsetAsync(B.status, 0, sizeof(int), B.stream);
            B.pois_threads = POIS_THREADS;
            B.pois_blocks = sms;
            B.weight_fluid = 1;
        }
        // multigrid replicas (all or none)
        if (rc == EKL_OK) {
            B.mg = B.reps[0]->mg;
            for (int r = 1; r < nrep; r++)
                if (B.reps[r]->mg != B.mg) rc = fail(EKL_ERR_ARG, "replicas must share the Poisson solver");
        }
        if (rc == EKL_OK && B.mg) {
            B.mg_smem = 0;
            for (int r = 0; r < nrep; r++) B.mg_smem = std::max(B.mg_smem, B.reps[r]->mg_smem);
            B.d_mgargs = A(nrep * sizeof(MgArgs));
            B.mg_bars = (unsigned *)A(4 * sizeof(unsigned) * (size_t)nrep);
            B.mgs_split = !(params[0].flags & EKL_POISSON_MG_SINGLE);
            B.d_ctl = A(nrep * sizeof(MgCtl));
            B.d_grids = A(nrep * sizeof(Grid3));
            B.d_loops = (int *)A(sizeof(int));
            B.mgs_factor = MGS_MAX_FACTOR;  // schedule bit 0 (the faster on uneven replicas)
            B.mgs_part_stride = MGS_MAX_FACTOR * sms;
            B.d_lrep = (int *)A(4 * (size_t)MGS_MAX_FACTOR * sms);
            B.d_lloc = (int *)A(4 * (size_t)MGS_MAX_FACTOR * sms);
            B.d_lrb = (int *)A(4 * (size_t)nrep);
            B.d_crep = (int *)A(4 * (size_t)2 * sms);
            B.d_cloc = (int *)A(4 * (size_t)2 * sms);
            B.d_crb = (int *)A(4 * (size_t)nrep);
            B.d_mgs_part = (double *)A(sizeof(double) * MGS_PART_SLOTS * (size_t)nrep * B.mgs_part_stride);
            if (ok) cudaMemsetAsync(B.d_loops, 0, sizeof(int), B.stream);
            if (!ok) rc = fail(EKL_ERR_ALLOC, "device allocation failed");
            else if (ops(B.prec).mg_batch_blocks(B.mg_smem) < 1)
                rc = fail(EKL_ERR_CUDA, "batched multigrid kernel cannot be resident");
        }
    }
    if (rc != EKL_OK) {
        batch_release(B);
        for (int r = 0; r < nrep; r++)
            if (B.handles[r]) ekl_destroy((ekl_handle *)B.handles[r]);
        delete[] B.reps;
        delete[] B.handles;
        delete bh;
        return rc;
    }
    *out = bh;
    return EKL_OK;
}

int ekl_create_batch(int32_t nrep, const ekl_params *params, void *stream, ekl_batch **out)
{
    return ekl_batch_create(nrep, params, stream, out);
}

int ekl_batch_set_beads(ekl_batch *bh, int32_t rep, int32_t n, const double *R, const double *V, const double *q,
                        const int32_t *chain)
{
    if (!bh || rep < 0 || rep >= bh->b.nrep) return fail(EKL_ERR_ARG, "bad batch or replica index");
    bh->b.ready = 0;  // descriptor tables carry the bead count
    return ekl_set_beads((ekl_handle *)bh->b.handles[rep], n, R, V, q, chain);
}

ekl_handle *ekl_batch_replica(ekl_batch *bh, int32_t rep)
{
    if (!bh || rep < 0 || rep >= bh->b.nrep) return nullptr;
    return (ekl_handle *)bh->b.handles[rep];
}

int ekl_batch_step(ekl_batch *bh, int32_t nsteps)
{
    if (!bh || nsteps < 0) return fail(EKL_ERR_ARG, "bad batch or step count");
    DeviceScope dscope(bh->b.reps[0]->device);
    if (!dscope.ok()) return fail(EKL_ERR_ARG, "the batch's device cannot be made current");
    Batch &B = bh->b;
    for (int r = 0; r < B.nrep; r++) cudaMemsetAsync(B.reps[r]->status, 0, sizeof(int), B.stream);
    cudaMemsetAsync(B.status, 0, sizeof(int), B.stream);
    int rc = batch_run(B, nsteps);
    if (rc != EKL_OK) return fail(rc, "batch launch failed");
    std::vector<int> st(B.nrep + 1, 0);
    cudaError_t e = cudaSuccess;
    for (int r = 0; r < B.nrep && e == cudaSuccess; r++)
        e = cudaMemcpyAsync(&st[r], B.reps[r]->status, sizeof(int), cudaMemcpyDeviceToHost, B.stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&st[B.nrep], B.status, sizeof(int), cudaMemcpyDeviceToHost, B.stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(B.stream);
    if (e != cudaSuccess) return fail_cuda(e, "batch step");
    int all = 0;
    for (int r = 0; r <= B.nrep; r++) all |= st[r];
    for (int r = 0; r < B.nrep; r++) B.reps[r]->last_status = st[r] | st[B.nrep];
    return status_to_code(all);
}

int ekl_batch_autotune(ekl_batch *bh, int32_t trial_steps, int32_t *choice_out)
{
    if (!bh || trial_steps < 1) return fail(EKL_ERR_ARG, "bad batch or trial length");
    DeviceScope dscope(bh->b.reps[0]->device);
    if (!dscope.ok()) return fail(EKL_ERR_ARG, "the batch's device cannot be made current");
    Batch &B = bh->b;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    int bestc = -1;
    for (int choice = 0; choice < 4; choice++) {
        if (batch_schedule(B, choice) != EKL_OK) continue;
        cudaEventRecord(e0, B.stream);
        int rc = batch_run(B, trial_steps);
        cudaEventRecord(e1, B.stream);
        if (rc != EKL_OK || cudaEventSynchronize(e1) != cudaSuccess) {
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            return fail(EKL_ERR_CUDA, "autotune trial failed");
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) {
            best = ms;
            bestc = choice;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (bestc < 0 || batch_schedule(B, bestc) != EKL_OK) return fail(EKL_ERR_CUDA, "no Poisson schedule could run");
    if (choice_out) *choice_out = bestc;
    return EKL_OK;
}

int ekl_batch_set_schedule(ekl_batch *bh, int32_t choice)
{
    if (!bh) return fail(EKL_ERR_ARG, "batch is null");
    if (batch_schedule(bh->b, choice) != EKL_OK) return fail(EKL_ERR_ARG, "schedule not available for this batch");
    return EKL_OK;
}

int64_t ekl_batch_launches(ekl_batch *bh)
{
    if (!bh) return 0;
    Batch &B = bh->b;
    if (!B.mgs_exec) return B.launches;
    // a split solve launches its loop's kernels from the device
    DeviceScope dscope(B.reps[0]->device);
    int loops = 0;
    if (!dscope.ok() || cudaMemcpyAsync(&loops, B.d_loops, sizeof(int), cudaMemcpyDeviceToHost, B.stream) != cudaSuccess ||
        cudaStreamSynchronize(B.stream) != cudaSuccess)
        return -1;
    return B.launches + (int64_t)B.mgs_iter_kernels * loops;
}

void ekl_batch_destroy(ekl_batch *bh)
{
    if (!bh) return;
    Batch &B = bh->b;
    DeviceScope dscope(B.nrep > 0 && B.reps[0] ? B.reps[0]->device : 0);
    cudaStreamSynchronize(B.stream);
    batch_release(B);
    for (int r = 0; r < B.nrep; r++)
        if (B.handles[r]) ekl_destroy((ekl_handle *)B.handles[r]);
    delete[] B.reps;
    delete[] B.handles;
    delete bh;
}

}  // extern "C"
