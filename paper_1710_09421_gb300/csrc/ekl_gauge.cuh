// Gauge of a read-out potential (ekl_get_fields, ekl_get_fields_noalloc).
#pragma once
#include "ekl_dev.cuh"

namespace ekl {

// Gauge of a read-out potential: phi minus its mean over the fluid nodes, 0 on
// walls.  The sum is deterministic: block b sums the contiguous chunk b of
// the nodes (thread-strided, then a fixed tree), and every block of the
// second kernel adds the GAUGE_BLOCKS partials in block order.
constexpr int GAUGE_BLOCKS = 256;
constexpr int GAUGE_THREADS = 1024;
static __global__ void __launch_bounds__(GAUGE_THREADS)
    gauge_partials_kernel(const double *__restrict__ phi, const uint32_t *__restrict__ mask, long long N,
                          double *__restrict__ part)
{
    __shared__ double sh[GAUGE_THREADS / 32];
    const long long chunk = (N + GAUGE_BLOCKS - 1) / GAUGE_BLOCKS;
    const long long i0 = blockIdx.x * chunk, i1 = i0 + chunk < N ? i0 + chunk : N;
    double s = 0.0, c = 0.0;
    for (long long i = i0 + threadIdx.x; i < i1; i += blockDim.x)
        if (!(mask[i] & SOLID_BIT)) {
            s += phi[i];
            c += 1.0;
        }
    s = block_sum(s, sh);
    c = block_sum(c, sh);
    if (threadIdx.x == 0) {
        part[blockIdx.x] = s;
        part[GAUGE_BLOCKS + blockIdx.x] = c;
    }
}
static __global__ void __launch_bounds__(GAUGE_THREADS)
    gauge_apply_kernel(const uint32_t *__restrict__ mask, long long N, double *__restrict__ phi,
                       const double *__restrict__ part)
{
    __shared__ double mean_s;
    if (threadIdx.x == 0) {
        double s = 0.0, c = 0.0;
        for (int b = 0; b < GAUGE_BLOCKS; b++) {
            s += part[b];
            c += part[GAUGE_BLOCKS + b];
        }
        mean_s = c > 0.0 ? s / c : 0.0;
    }
    __syncthreads();
    const double mean = mean_s;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x)
        phi[i] = (mask[i] & SOLID_BIT) ? 0.0 : phi[i] - mean;
}

}  // namespace ekl
