// Device-side building blocks shared by the kernels of the library:
// D3Q19 table, storage conversions, neighbour indexing, Philox-4x32-10,
// bounded grid barrier, warp reductions.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "ekl_ctx.h"

namespace ekl {

// D3Q19 velocity set (Sec. II.C): rest, +-x, +-y, +-z, then the xy, xz and
// yz diagonals, each velocity followed by its opposite.
__host__ __device__ constexpr int cx_(int p)
{
    constexpr int t[Q] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
    return t[p];
}
__host__ __device__ constexpr int cy_(int p)
{
    constexpr int t[Q] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1};
    return t[p];
}
__host__ __device__ constexpr int cz_(int p)
{
    constexpr int t[Q] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1};
    return t[p];
}
__host__ __device__ constexpr int opp_(int p) { return p == 0 ? 0 : ((p & 1) ? p + 1 : p - 1); }
// weights 1/3, 1/18 (|c| = 1), 1/36 (|c| = sqrt 2)
__host__ __device__ constexpr double w_(int p)
{
    return p == 0 ? 1.0 / 3.0 : (p <= 6 ? 1.0 / 18.0 : 1.0 / 36.0);
}

constexpr uint32_t SOLID_BIT = 0x80000000u;

// ---------------------------------------------------------------- storage
template <typename S> struct Store;
template <> struct Store<double> {
    __device__ static double ld(const double *p) { return __ldg(p); }
    __device__ static void st(double *p, double v) { *p = v; }
};
template <> struct Store<float> {
    __device__ static float ld(const float *p) { return __ldg(p); }
    __device__ static void st(float *p, float v) { *p = v; }
};
template <> struct Store<__nv_bfloat16> {
    __device__ static float ld(const __nv_bfloat16 *p) { return __bfloat162float(__ldg(p)); }
    __device__ static void st(__nv_bfloat16 *p, float v) { *p = __float2bfloat16_rn(v); }
};
// FP16 deviations are stored times 2^12: the ion deviations (about 1e-6 to
// 1e-4 at salt 0.01) would otherwise sit below FP16's normal range (6.1e-5)
// and lose bits as subnormals; scaled, deviations from 1.5e-8 to 16 are
// normal numbers.  The power of two makes the scaling exact.
constexpr float FP16_DEV_SCALE = 4096.0f;
template <> struct Store<__half> {
    __device__ static float ld(const __half *p) { return __half2float(__ldg(p)) * (1.0f / FP16_DEV_SCALE); }
    __device__ static void st(__half *p, float v) { *p = __float2half_rn(v * FP16_DEV_SCALE); }
};

// ---------------------------------------------------------------- indexing
struct Grid3 {
    int nx, ny, nz;
    long long N;
    // i / nx and r / ny for 0 <= i, r < 2^31 as (i * m) >> s: with
    // L = ceil(log2 d), s = 31 + L and m = ceil(2^s / d) (< 2^32), the error
    // i (m d - 2^s) / (d 2^s) stays below 1/d, so the floor is exact
    unsigned mx, my;
    int sx, sy;
};
inline void grid_divisor(int d, unsigned &m, int &s)
{
    int L = 0;
    while ((1ll << L) < (long long)d) L++;
    s = 31 + L;
    m = (unsigned)(((1ull << s) + (unsigned long long)d - 1) / (unsigned long long)d);
}
inline Grid3 make_grid3(int nx, int ny, int nz)
{
    Grid3 g{nx, ny, nz, (long long)nx * ny * nz, 0u, 0u, 0, 0};
    grid_divisor(nx, g.mx, g.sx);
    grid_divisor(ny, g.my, g.sy);
    return g;
}

// n / d for 0 <= n < 2^21 from inv = 1/d (rounded): (n + 1/2) / d lies at
// least 1/(2d) from an integer and the two roundings move it by less than
// 2^-23 (n + 1/2) / d, so truncation gives the floor
__device__ __forceinline__ int tdiv(int n, float inv) { return (int)(((float)n + 0.5f) * inv); }

// node coordinates; node ids fit 32 bits (lattices are capped at 2^31/64 nodes)
__device__ __forceinline__ void coords_of(const Grid3 &g, long long i64, int &x, int &y, int &z)
{
    const int i = (int)i64;
    const int r = (int)(((unsigned long long)(unsigned)i * g.mx) >> g.sx);
    x = i - r * g.nx;
    z = (int)(((unsigned long long)(unsigned)r * g.my) >> g.sy);
    y = r - z * g.ny;
}

// Neighbour offsets for the pull x - c_p: X[cx + 1] = {x+1, x, x-1}.  Indices
// wrap on every axis; on a closed axis the wrapped neighbour is never read
// because the link bit of that direction is set.
struct Nbr {
    int X[3];
    int Y[3];
    int Z[3];
    __device__ __forceinline__ int pull(int p) const { return X[cx_(p) + 1] + Y[cy_(p) + 1] + Z[cz_(p) + 1]; }
};

__device__ __forceinline__ Nbr make_nbr(const Grid3 &g, int x, int y, int z)
{
    Nbr n;
    const int xm = x == 0 ? g.nx - 1 : x - 1, xp = x == g.nx - 1 ? 0 : x + 1;
    const int ym = y == 0 ? g.ny - 1 : y - 1, yp = y == g.ny - 1 ? 0 : y + 1;
    const int zm = z == 0 ? g.nz - 1 : z - 1, zp = z == g.nz - 1 ? 0 : z + 1;
    const int sxy = g.nx * g.ny;
    n.X[0] = xp; n.X[1] = x; n.X[2] = xm;
    n.Y[0] = yp * g.nx; n.Y[1] = y * g.nx; n.Y[2] = ym * g.nx;
    n.Z[0] = zp * sxy; n.Z[1] = z * sxy; n.Z[2] = zm * sxy;
    return n;
}

// face neighbours (-x, +x, -y, +y, -z, +z) are the pulls of p = 1..6
__device__ __forceinline__ int face_idx(const Nbr &n, int f)
{
    // face f is the node x + e_f; pull p gives x - c_p: -x face = p1, +x = p2, ...
    return n.pull(f + 1);
}

// ---------------------------------------------------------------- Philox
// Philox-4x32-10 (Salmon et al., SC'11): ten rounds of two 32x32->64
// multiplies, key bumped by the Weyl increments between rounds.
__host__ __device__ inline void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; r++) {
        if (r > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
#ifdef __CUDA_ARCH__
        uint32_t lo0 = 0xD2511F53u * c[0], hi0 = __umulhi(0xD2511F53u, c[0]);
        uint32_t lo1 = 0xCD9E8D57u * c[2], hi1 = __umulhi(0xCD9E8D57u, c[2]);
#else
        uint64_t p0 = (uint64_t)0xD2511F53u * c[0], p1 = (uint64_t)0xCD9E8D57u * c[2];
        uint32_t lo0 = (uint32_t)p0, hi0 = (uint32_t)(p0 >> 32);
        uint32_t lo1 = (uint32_t)p1, hi1 = (uint32_t)(p1 >> 32);
#endif
        uint32_t n0 = hi1 ^ c[1] ^ k0;
        uint32_t n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0;
        c[1] = lo1;
        c[2] = n2;
        c[3] = lo0;
    }
}

// zero-mean unit-variance variate sqrt(3)(2U - 1), U = (x + 1/2) / 2^32
template <typename R> __device__ __forceinline__ R unit_variate(uint32_t x);
template <> __device__ __forceinline__ double unit_variate<double>(uint32_t x)
{
    double t = ((double)(2.0 * (double)x + 1.0) - 4294967296.0) * (1.0 / 4294967296.0);
    return 1.7320508075688772 * t;
}
// The same variate in FP32 arithmetic without a 64-bit conversion (GB300 runs
// those at the FP64 rate): (x - 2^31 + 1/2) 2^-31 = 2U - 1, the 32-bit
// conversion rounding to FP32.  Used by the reduced-precision paths.
__device__ __forceinline__ float unit_variate_f32(uint32_t x)
{
    const float t = __int2float_rn((int)(x ^ 0x80000000u)) * 4.656612873077393e-10f + 2.3283064365386963e-10f;
    return 1.7320508f * t;
}
template <> __device__ __forceinline__ float unit_variate<float>(uint32_t x)
{
    // exact: 2x + 1 - 2^32 is an odd integer below 2^33 in magnitude
    float t = (float)((int64_t)(2ull * x + 1ull) - 4294967296ll) * (1.0f / 4294967296.0f);
    return 1.7320508f * t;
}

// ---------------------------------------------------------------- sync
__device__ __forceinline__ unsigned ld_relaxed(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void red_release_add(unsigned *p, unsigned v)
{
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void fence_acq_rel_gpu() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }
__device__ __forceinline__ uint64_t globaltimer_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Grid-wide barrier of a cooperative launch with a bounded wait.  bar[0]
// counts arrivals monotonically within a launch (reset by the host before
// the launch); barrier number k (k = 1, 2, ...) is passed when the count
// reaches k * nblocks.  Arrival is a release reduction (it publishes the
// block's writes, ordered before it by __syncthreads); the wait polls with
// relaxed loads, one load per poll, and the fence after the last poll makes
// it an acquire.  A block that waits more than ~2 s raises ST_TIMEOUT and
// the abort word bar[2]; every waiter also leaves soon after the abort word
// is set (it is read every 64 polls).  Returns false on abort.
__device__ __forceinline__ bool grid_barrier(unsigned *bar, unsigned nblocks, unsigned &k, int *status)
{
    __shared__ int ok_s;
    __syncthreads();
    k++;
    if (threadIdx.x == 0) {
        int ok = 1;
        const unsigned target = k * nblocks;
        red_release_add(&bar[0], 1u);
        uint64_t t0 = 0;
        unsigned spins = 0;
        while ((int)(ld_relaxed(&bar[0]) - target) < 0) {
            if ((++spins & 63u) == 0) {
                if (ld_relaxed(&bar[2])) {
                    ok = 0;
                    break;
                }
                uint64_t t = globaltimer_ns();
                if (t0 == 0) t0 = t;
                else if (t - t0 > 2000000000ull) {
                    atomicOr(status, ST_TIMEOUT);
                    atomicExch(&bar[2], 1u);
                    ok = 0;
                    break;
                }
            }
        }
        fence_acq_rel_gpu();
        ok_s = ok;
    }
    __syncthreads();
    return ok_s != 0;
}

// ---------------------------------------------------------------- conversions
// GB300 runs FP64 (and 64-bit integer<->float conversions) at a small
// fraction of the FP32 rate, so per-node work avoids them.
// int64 -> float, round to nearest for |r| < 2^31, within one float ulp above.
__device__ __forceinline__ float ll_to_float(long long r)
{
    if (r == (long long)(int)r) return __int2float_rn((int)r);
    return fmaf(__int2float_rn((int)(r >> 32)), 4294967296.0f, __uint2float_rn((unsigned)r));
}
// float -> int64, round to nearest; exact split above 2^31 where d is a
// multiple of 256.
__device__ __forceinline__ long long float_to_ll(float d)
{
    if (fabsf(d) < 2147483520.0f) return (long long)__float2int_rn(d);
    float hi = floorf(d * 2.3283064365386963e-10f);  // d / 2^32
    float lo = d - hi * 4294967296.0f;               // exact, in [0, 2^32)
    return ((long long)__float2int_rn(hi) << 32) + (long long)__float2uint_rn(lo);
}

// ---------------------------------------------------------------- potential
// FP64 path: phi stored as double.  Reduced-precision paths: phi stored as a
// signed 64-bit fixed-point number with 40 fractional bits, so that the
// 7-point residual is computed exactly in integer arithmetic.
template <typename PhiT> struct PhiOps;
template <> struct PhiOps<double> {
    __device__ static double diff(double a, double b) { return a - b; }  // as real
};
template <> struct PhiOps<long long> {
    __device__ static float diff(long long a, long long b) { return ll_to_float(a - b) * (float)PHI_INV; }
};

// ---------------------------------------------------------------- reductions
// Warp sum of FP32 values carried as an unevaluated float pair (TwoSum at
// each level of a fixed xor tree): about 48 bits, FP32 pipe only; the result
// is returned as a double in every lane.
__device__ __forceinline__ void warp_sum_ff2(float v, float &hi, float &lo)
{
    hi = v;
    lo = 0.f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        float oh = __shfl_xor_sync(0xffffffffu, hi, o);
        float ol = __shfl_xor_sync(0xffffffffu, lo, o);
        float s = hi + oh;
        float bb = s - hi;
        float err = (hi - (s - bb)) + (oh - bb);
        hi = s;
        lo = lo + ol + err;
    }
}
__device__ __forceinline__ double warp_sum_ff(float v)
{
    float hi, lo;
    warp_sum_ff2(v, hi, lo);
    return (double)hi + (double)lo;
}
// same, converted to FP64 in lane 0 only (the value is meaningful there)
__device__ __forceinline__ double warp_sum_ff_lane0(float v)
{
    float hi, lo;
    warp_sum_ff2(v, hi, lo);
    double r = 0.0;
    if ((threadIdx.x & 31) == 0) r = (double)hi + (double)lo;
    return r;
}

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Deterministic block sum (fixed shuffle tree, fixed warp order); result valid
// in thread 0.  `sh` must hold blockDim.x / 32 doubles.
__device__ __forceinline__ double block_sum(double v, double *sh)
{
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0) {
        int nw = (blockDim.x + 31) >> 5;
        for (int k = 0; k < nw; k++) t += sh[k];
    }
    return t;
}

// Block sum of per-warp values already reduced within each warp (lane 0
// holds the warp's value); fixed warp order; result valid in thread 0.
__device__ __forceinline__ double block_sum_lanes0(double wv, double *sh)
{
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[wid] = wv;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0) {
        int nw = (blockDim.x + 31) >> 5;
        for (int k = 0; k < nw; k++) t += sh[k];
    }
    return t;
}

// Sum of n per-block partials, identical in every block: warp 0 reads them
// (lane l takes l, l+32, ...), reduces with a fixed shuffle tree and
// broadcasts through shared memory.  Every thread of the block must call it.
__device__ __forceinline__ double sum_partials(const double *p, int n, double *sh)
{
    __syncthreads();
    if (threadIdx.x < 32) {
        double v = 0.0;
        for (int k = threadIdx.x; k < n; k += 32) v += __ldcg(p + k);
        v = warp_sum(v);
        if (threadIdx.x == 0) sh[0] = v;
    }
    __syncthreads();
    return sh[0];
}

// The same for 64-bit integer partials (exact).
__device__ __forceinline__ long long sum_partials_ll(const long long *p, int n)
{
    __shared__ long long s_ll;
    __syncthreads();
    if (threadIdx.x < 32) {
        long long v = 0;
        for (int k = threadIdx.x; k < n; k += 32) v += __ldcg(p + k);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (threadIdx.x == 0) s_ll = v;
    }
    __syncthreads();
    return s_ll;
}

// A uniform number in [0, 1) fixed per node index (integer hash: multiply by
// the golden-ratio constant, then xor-shift / multiply mixing rounds)
__device__ __forceinline__ float node_uniform(long long i)
{
    uint32_t h = (uint32_t)i * 0x9E3779B1u;
    h ^= h >> 16;
    h *= 0x85EBCA6Bu;
    h ^= h >> 13;
    h *= 0xC2B2AE35u;
    h ^= h >> 16;
    return (float)(h >> 8) * (1.0f / 16777216.0f);
}

// Residual test of an iteration: warp 0 sums the block partials (fixed
// order), thread 0 compares sqrt(sum) with tol * bnorm and broadcasts the
// result; every thread of the block must call it.
__device__ __forceinline__ bool test_partials(const double *p, int n, double tolb, double *sh,
                                              int *flag, double &sum_out)
{
    __syncthreads();
    if (threadIdx.x < 32) {
        double v = 0.0;
        for (int k = threadIdx.x; k < n; k += 32) v += __ldcg(p + k);
        v = warp_sum(v);
        if (threadIdx.x == 0) {
            sh[0] = v;
            *flag = sqrt(v) <= tolb;
        }
    }
    __syncthreads();
    sum_out = sh[0];
    return *flag != 0;
}

// lower bound of `key` in sorted a[0..n)
__device__ __forceinline__ int lower_bound_i(const int *a, int n, long long key)
{
    int lo = 0, hi = n;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if ((long long)a[mid] < key) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

}  // namespace ekl
