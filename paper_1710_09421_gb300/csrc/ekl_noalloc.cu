// ekl_get_fields_noalloc: the field read-back of ekl_get_fields without any
// device allocation.
//
// Who needs it: callers that must not allocate GPU memory while they run --
// for example code that executes between the capture and replay of a CUDA
// graph on a pool-allocated stream, a real-time control loop that has
// pre-reserved all device memory, or a host framework whose allocator is
// locked during a solver callback.  ekl_get_fields stages the fields in
// device buffers it allocates per call; this entry point stages them instead
// in one fixed, file-scope device array that the library reserves when it is
// loaded.
//
// Limits and sharing:
//   * the staging array holds EKL_NOALLOC_MAX_DOUBLES doubles (16 MiB); a
//     request that needs more (3N for densities + 9N for currents + N for the
//     potential + 6 per bead for positions/velocities) is rejected with
//     EKL_ERR_ARG before any work is queued;
//   * every call, from every handle on a device, uses the same array and the
//     array keeps the last call's contents; each call writes every element it
//     reads back, so nothing has to start at zero;
//   * calls whose GPU work overlaps (two host threads, or two streams) race
//     on the array: serialise them;
//   * the first call on a device looks up the array's device address with
//     cudaGetSymbolAddress (once per device, with that device current); make
//     that first call before any stream capture begins.
#include <mutex>

#include "ekl_step.cuh"
#include "ekl_gauge.cuh"

struct ekl_handle {
    ekl::Ctx c;
};

namespace {

constexpr size_t NOALLOC_DOUBLES = (size_t)EKL_NOALLOC_MAX_DOUBLES;
static __device__ __align__(256) double g_stage[NOALLOC_DOUBLES];

constexpr int MAX_DEVICES = 64;
double *g_stage_addr[MAX_DEVICES] = {nullptr};
std::mutex g_stage_mu;


// device address of the staging array on device dev (set-up once per
// device); dev must be the current device, which the check below enforces so
// that no other device's address is ever cached under dev
int stage_address(int dev, double **out)
{
    if (dev < 0 || dev >= MAX_DEVICES) return EKL_ERR_ARG;
    int cur = -1;
    if (cudaGetDevice(&cur) != cudaSuccess || cur != dev) {
        cudaGetLastError();
        ekl::set_last_error("the staging array is looked up with another device current");
        return EKL_ERR_ARG;
    }
    std::lock_guard<std::mutex> lk(g_stage_mu);
    if (!g_stage_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_stage);
        if (e != cudaSuccess) {
            char msg[256];
            snprintf(msg, sizeof msg, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
            ekl::set_last_error(msg);
            return EKL_ERR_CUDA;
        }
        g_stage_addr[dev] = (double *)p;
    }
    *out = g_stage_addr[dev];
    return EKL_OK;
}

// potential of the last step with the fluid mean removed, wall nodes zero;
// one block, fixed reduction order
template <typename R> __global__ void beads_kernel(const double *Rb, const R *Vb, int n3, double *out)
{
    for (int k = threadIdx.x; k < n3; k += blockDim.x) {
        out[k] = (double)Rb[k];
        out[n3 + k] = (double)Vb[k];
    }
}

template <typename S, typename R, typename PhiT, bool DEV>
int stage_fields(ekl::Ctx &c, double *dn, double *dj, double *dp)
{
    ekl::StepArgs<S, R, PhiT> a = ekl::make_args<S, R, PhiT>(c);
    int blocks = (int)((c.N + 255) / 256);
    ekl::fields_kernel<S, R, PhiT, DEV><<<blocks, 256, 0, c.stream>>>(a, dn, dj, dp);
    c.launches++;
    return cudaGetLastError() == cudaSuccess ? EKL_OK : EKL_ERR_CUDA;
}

}  // namespace

extern "C" int ekl_get_fields_noalloc(ekl_handle *h, double *n_out, double *j_out, double *phi_out,
                                      double *R_out, double *V_out)
{
    if (!h) {
        ekl::set_last_error("null handle");
        return EKL_ERR_ARG;
    }
    // the staging array's address is looked up, and cached, for the handle's
    // device with that device current
    ekl::DeviceScope dscope(h->c.device);
    if (!dscope.ok()) {
        ekl::set_last_error("the handle's device cannot be made current");
        return EKL_ERR_ARG;
    }
    ekl::Ctx &c = h->c;
    const long long N = c.N;
    const bool beads = c.nb > 0 && (R_out || V_out);
    size_t need = (n_out ? 3 * (size_t)N : 0) + (j_out ? 9 * (size_t)N : 0) +
                  (phi_out ? (size_t)N + 2 * ekl::GAUGE_BLOCKS : 0) + (beads ? 6 * (size_t)c.nb : 0);
    if (need > NOALLOC_DOUBLES) {
        char msg[256];
        snprintf(msg, sizeof msg,
                 "request needs %zu doubles of staging; the allocation-free path holds %zu",
                 need, NOALLOC_DOUBLES);
        ekl::set_last_error(msg);
        return EKL_ERR_ARG;
    }
    double *stage = nullptr;
    int rc = stage_address(c.device, &stage);
    if (rc != EKL_OK) return rc;
    double *dn = n_out ? stage : nullptr;
    double *dj = j_out ? stage + (n_out ? 3 * N : 0) : nullptr;
    double *dp = phi_out ? stage + (n_out ? 3 * N : 0) + (j_out ? 9 * N : 0) : nullptr;
    double *db = stage + (n_out ? 3 * N : 0) + (j_out ? 9 * N : 0) + (phi_out ? N : 0);
    switch (c.prec) {
    case EKL_F64: rc = stage_fields<double, double, double, false>(c, dn, dj, dp); break;
    case EKL_F32: rc = stage_fields<float, float, long long, true>(c, dn, dj, dp); break;
    case EKL_BF16DEV: rc = stage_fields<__nv_bfloat16, float, long long, true>(c, dn, dj, dp); break;
    default: rc = stage_fields<__half, float, long long, true>(c, dn, dj, dp); break;
    }
    if (rc != EKL_OK) return rc;
    if (dp) {
        // the gauge's block partials after the bead block
        double *gp = db + (beads ? 6 * c.nb : 0);
        ekl::gauge_partials_kernel<<<ekl::GAUGE_BLOCKS, ekl::GAUGE_THREADS, 0, c.stream>>>(dp, c.mask, N, gp);
        ekl::gauge_apply_kernel<<<c.num_sms * 2, ekl::GAUGE_THREADS, 0, c.stream>>>(c.mask, N, dp, gp);
        c.launches += 2;
    }
    if (beads) {
        if (c.prec == EKL_F64) beads_kernel<double><<<1, 256, 0, c.stream>>>((const double *)c.R, (const double *)c.V, 3 * c.nb, db);
        else beads_kernel<float><<<1, 256, 0, c.stream>>>((const double *)c.R, (const float *)c.V, 3 * c.nb, db);
        c.launches++;
    }
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && n_out) e = cudaMemcpyAsync(n_out, dn, 3 * (size_t)N * 8, cudaMemcpyDeviceToHost, c.stream);
    if (e == cudaSuccess && j_out) e = cudaMemcpyAsync(j_out, dj, 9 * (size_t)N * 8, cudaMemcpyDeviceToHost, c.stream);
    if (e == cudaSuccess && phi_out) e = cudaMemcpyAsync(phi_out, dp, (size_t)N * 8, cudaMemcpyDeviceToHost, c.stream);
    if (e == cudaSuccess && beads && R_out) e = cudaMemcpyAsync(R_out, db, 3 * (size_t)c.nb * 8, cudaMemcpyDeviceToHost, c.stream);
    if (e == cudaSuccess && beads && V_out) e = cudaMemcpyAsync(V_out, db + 3 * c.nb, 3 * (size_t)c.nb * 8, cudaMemcpyDeviceToHost, c.stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c.stream);
    if (e != cudaSuccess) {
        char msg[256];
        snprintf(msg, sizeof msg, "ekl_get_fields_noalloc: %s", cudaGetErrorString(e));
        ekl::set_last_error(msg);
        return EKL_ERR_CUDA;
    }
    return EKL_OK;
}
