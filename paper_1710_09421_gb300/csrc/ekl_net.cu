// Learned warm start for the Poisson solve: a 3D convolutional network
// (3^3 kernels, channels 2 -> 16 -> 16 -> 16 -> 1, ReLU between layers,
// linear output) mapping the step's change of the Poisson source and the
// previous potential to the change of the potential.  The solver then runs to
// its usual residual from the improved start, so only iterations are saved.
//
// Layout: activations node-major, 16 channels contiguous (NDHWC) in BF16;
// parameters as one FP32 vector, per layer W[co][ci][k] then b[co] with
// k = (dz+1)*9 + (dy+1)*3 + (dx+1); periodic wrap on periodic axes, zeros
// beyond closed ones.
//
// The two 16 -> 16 layers (about 93 % of the arithmetic) are implicit GEMMs
// on the tensor cores, K = 27 offsets x 16 input channels, BF16 operands,
// FP32 accumulation: by default on tcgen05 (128 nodes per block, the
// accumulator in tensor memory, operands staged in shared memory), or with
// the warp-level mma.sync m16n8k16 (16 nodes per warp); the data gradient of
// those layers is the same kernel with flipped offsets and transposed
// channels.  The 2 -> 16 and 16 -> 1 layers, the weight
// gradients (per-block partial sums reduced in a fixed order) and Adam run on
// the CUDA cores in FP32.
#include <cuda_bf16.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <vector>

#include <new>
#include <utility>

#include "ekl_kernels.cuh"

struct ekl_handle {
    ekl::Ctx c;
};

namespace {

using namespace ekl;

constexpr int C = 16;     // hidden channels
constexpr int K27 = 27;
constexpr int NT = 256;   // threads per block of the CUDA-core kernels
// parameter offsets
constexpr int OW1 = 0, OB1 = OW1 + 16 * 2 * 27, OW2 = OB1 + 16, OB2 = OW2 + 16 * 16 * 27,
              OW3 = OB2 + 16, OB3 = OW3 + 16 * 16 * 27, OW4 = OB3 + 16, OB4 = OW4 + 16 * 27,
              NPARAM = OB4 + 1;
static_assert(NPARAM == EKL_NET_PARAMS, "parameter count");

struct NetGrid {
    int nx, ny, nz;
    int per[3];
    int N;
};

// neighbour of node (x,y,z) at offset k; -1 beyond a closed face
__device__ __forceinline__ int nbr_off(const NetGrid &g, int x, int y, int z, int k)
{
    int dx = k % 3 - 1, dy = (k / 3) % 3 - 1, dz = k / 9 - 1;
    int X = x + dx, Y = y + dy, Z = z + dz;
    if (X < 0 || X >= g.nx) {
        if (!g.per[0]) return -1;
        X = X < 0 ? X + g.nx : X - g.nx;
    }
    if (Y < 0 || Y >= g.ny) {
        if (!g.per[1]) return -1;
        Y = Y < 0 ? Y + g.ny : Y - g.ny;
    }
    if (Z < 0 || Z >= g.nz) {
        if (!g.per[2]) return -1;
        Z = Z < 0 ? Z + g.nz : Z - g.nz;
    }
    return X + g.nx * (Y + g.ny * Z);
}

__device__ __forceinline__ void xyz_of(const NetGrid &g, int n, int &x, int &y, int &z)
{
    int r = n / g.nx;
    x = n - r * g.nx;
    z = r / g.ny;
    y = r - z * g.ny;
}

// ---------------------------------------------------------------- layer 1
// act1[n][co] = relu(b1[co] + sum_k sum_ci W1[co][ci][k] x[ci][n + off_k])
__global__ void __launch_bounds__(NT) l1_fwd(NetGrid g, const float *__restrict__ x, const float *__restrict__ w,
                                             __nv_bfloat16 *__restrict__ act)
{
    __shared__ float sw[16 * 2 * 27 + 16];
    for (int t = threadIdx.x; t < 16 * 2 * 27 + 16; t += blockDim.x) sw[t] = w[OW1 + t];
    __syncthreads();
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= g.N) return;
    int X, Y, Z;
    xyz_of(g, n, X, Y, Z);
    float acc[16];
    for (int c = 0; c < 16; c++) acc[c] = sw[16 * 54 + c];
    for (int k = 0; k < K27; k++) {
        const int j = nbr_off(g, X, Y, Z, k);
        if (j < 0) continue;
        const float x0 = x[j], x1 = x[g.N + j];
        for (int c = 0; c < 16; c++) acc[c] += sw[c * 54 + k] * x0 + sw[c * 54 + 27 + k] * x1;
    }
    for (int c = 0; c < 16; c += 2) {
        __nv_bfloat162 v = __floats2bfloat162_rn(fmaxf(acc[c], 0.f), fmaxf(acc[c + 1], 0.f));
        *(__nv_bfloat162 *)(act + (size_t)n * 16 + c) = v;
    }
}

// ---------------------------------------------------------------- 16 -> 16 on tensor cores
__device__ __forceinline__ void mma_bf16(float d[4], const uint32_t a[4], const uint32_t b[2])
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// out[n][co] = act?(bias[co] + sum_k sum_ci Wt[k][co][ci] in[n + off_k][ci]); flip = use -off_k.
// Wt is BF16 [27][16 co][16 ci] (ci contiguous).  One warp: 16 consecutive nodes.
template <bool RELU, bool OUT_F32>
__global__ void __launch_bounds__(256) conv16_mma(NetGrid g, const __nv_bfloat16 *__restrict__ in,
                                                  const __nv_bfloat16 *__restrict__ Wt,
                                                  const float *__restrict__ bias, int flip, void *out,
                                                  const __nv_bfloat16 *__restrict__ relu_mask_src)
{
    __shared__ uint32_t sW[27 * 16 * 8];  // [k][co][ci pair]
    for (int t = threadIdx.x; t < 27 * 16 * 8; t += blockDim.x) sW[t] = ((const uint32_t *)Wt)[t];
    __syncthreads();
    const int lane = threadIdx.x & 31, gid = lane >> 2, tig = lane & 3;
    const int warp_global = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int n0 = warp_global * 16;
    if (n0 >= g.N) return;
    const int na = n0 + gid, nb = n0 + gid + 8;
    int xa, ya, za, xb, yb, zb;
    xyz_of(g, na < g.N ? na : 0, xa, ya, za);
    xyz_of(g, nb < g.N ? nb : 0, xb, yb, zb);
    float d[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
    const uint32_t *in32 = (const uint32_t *)in;
    for (int k = 0; k < K27; k++) {
        const int kk = flip ? 26 - k : k;
        const int ja = na < g.N ? nbr_off(g, xa, ya, za, kk) : -1;
        const int jb = nb < g.N ? nbr_off(g, xb, yb, zb, kk) : -1;
        uint32_t a[4];
        a[0] = ja >= 0 ? in32[(size_t)ja * 8 + tig] : 0u;
        a[1] = jb >= 0 ? in32[(size_t)jb * 8 + tig] : 0u;
        a[2] = ja >= 0 ? in32[(size_t)ja * 8 + tig + 4] : 0u;
        a[3] = jb >= 0 ? in32[(size_t)jb * 8 + tig + 4] : 0u;
#pragma unroll
        for (int h = 0; h < 2; h++) {
            const int co = h * 8 + gid;
            uint32_t b[2] = {sW[(k * 16 + co) * 8 + tig], sW[(k * 16 + co) * 8 + tig + 4]};
            mma_bf16(d[h], a, b);
        }
    }
#pragma unroll
    for (int h = 0; h < 2; h++) {
        const int co = h * 8 + 2 * tig;
        float v[4] = {d[h][0], d[h][1], d[h][2], d[h][3]};
        if (bias) {
            v[0] += bias[co];
            v[1] += bias[co + 1];
            v[2] += bias[co];
            v[3] += bias[co + 1];
        }
        if (RELU)
            for (int q = 0; q < 4; q++) v[q] = fmaxf(v[q], 0.f);
        // gradient through the ReLU of the layer that produced `relu_mask_src`
        if (relu_mask_src) {
            if (na < g.N) {
                if (!(__bfloat162float(relu_mask_src[(size_t)na * 16 + co]) > 0.f)) v[0] = 0.f;
                if (!(__bfloat162float(relu_mask_src[(size_t)na * 16 + co + 1]) > 0.f)) v[1] = 0.f;
            }
            if (nb < g.N) {
                if (!(__bfloat162float(relu_mask_src[(size_t)nb * 16 + co]) > 0.f)) v[2] = 0.f;
                if (!(__bfloat162float(relu_mask_src[(size_t)nb * 16 + co + 1]) > 0.f)) v[3] = 0.f;
            }
        }
        if (OUT_F32) {
            float *o = (float *)out;
            if (na < g.N) { o[(size_t)na * 16 + co] = v[0]; o[(size_t)na * 16 + co + 1] = v[1]; }
            if (nb < g.N) { o[(size_t)nb * 16 + co] = v[2]; o[(size_t)nb * 16 + co + 1] = v[3]; }
        } else {
            __nv_bfloat16 *o = (__nv_bfloat16 *)out;
            if (na < g.N) *(__nv_bfloat162 *)(o + (size_t)na * 16 + co) = __floats2bfloat162_rn(v[0], v[1]);
            if (nb < g.N) *(__nv_bfloat162 *)(o + (size_t)nb * 16 + co) = __floats2bfloat162_rn(v[2], v[3]);
        }
    }
}

// ---------------------------------------------------------------- 16 -> 16 on tcgen05
// The same layer as an implicit GEMM on the fifth-generation tensor cores:
// a block takes 128 consecutive nodes (M = 128), N = 16 output channels, and
// K = 27 offsets x 16 input channels as 27 MMAs of K = 16 (one per offset),
// BF16 operands from shared memory, FP32 accumulation in tensor memory.
//   * A (per offset): the 16 input channels of each node's neighbour, 128 x 16
//     BF16, K-major without swizzle: core matrices of 8 rows x 16 bytes,
//     row-group g and K-half h at byte g * 256 + h * 128 (LBO = 128 between
//     the K-halves, SBO = 256 between row groups);
//   * B (per offset): W[co][ci], 16 x 16 BF16, the same layout;
//   * D: TMEM lanes 0..127 = nodes, columns 0..15 = output channels; warp w
//     reads lanes 32w..32w+31 back with tcgen05.ld (32x32b, 16 columns).
// One thread issues the 27 MMAs and commits them to an mbarrier; the wait is
// bounded (on giving up the block raises tc_status and skips the epilogue),
// and the block frees its tensor memory on every path.
constexpr int TC_M = 128;
constexpr int TC_A_BYTES = TC_M * 32;           // one offset's A tile
constexpr int TC_B_BYTES = 16 * 32;             // one offset's B tile
constexpr int TC_SMEM = K27 * (TC_A_BYTES + TC_B_BYTES) + 64;

__device__ int tc_status;  // nonzero after a bounded wait gave up

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: no swizzle, K-major core matrices
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}
// instruction descriptor: D FP32, A and B BF16, both K-major, N = 16, M = 128
constexpr uint32_t TC_IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((16u >> 3) << 17) | ((128u >> 4) << 24);

// byte offset of element (row, k) (k < 16) in a no-swizzle K-major tile
__device__ __forceinline__ int tc_off(int row, int k) { return (row >> 3) * 256 + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2; }

// wait (bounded, about a second at most) for phase 0 of the mbarrier
__device__ __forceinline__ uint32_t tc_wait(uint64_t *mbar)
{
    uint32_t done = 0;
    for (int it = 0; it < (1 << 20) && !done; it++) {
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(smem_u32(mbar)));
    }
    return done;
}

template <bool RELU>
__global__ void __launch_bounds__(TC_M) conv16_tc(NetGrid g, const __nv_bfloat16 *__restrict__ in,
                                                  const __nv_bfloat16 *__restrict__ Wt,
                                                  const float *__restrict__ bias, int flip,
                                                  __nv_bfloat16 *__restrict__ out,
                                                  const __nv_bfloat16 *__restrict__ relu_mask_src)
{
    extern __shared__ __align__(1024) uint8_t tc_sm[];
    uint8_t *sA = tc_sm;                              // [27][TC_A_BYTES]
    uint8_t *sB = tc_sm + K27 * TC_A_BYTES;           // [27][TC_B_BYTES]
    uint64_t *mbar = (uint64_t *)(sB + K27 * TC_B_BYTES);
    uint32_t *tmem_slot = (uint32_t *)(mbar + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int n = blockIdx.x * TC_M + tid;
    const bool valid = n < g.N;

    // tensor memory: 32 columns (the smallest allocation) for the 16 of D
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 32;\n" ::"r"(smem_u32(tmem_slot)));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(mbar)));
    }
    // operands: B tiles (weights of every offset), A tiles (this thread's
    // node's neighbour at every offset, zero beyond a closed face)
    for (int t = tid; t < K27 * 16 * 2; t += TC_M) {
        const int k = t >> 5, co = (t >> 1) & 15, h = t & 1;
        const uint4 v = *(const uint4 *)(Wt + ((size_t)k * 16 + co) * 16 + 8 * h);
        *(uint4 *)(sB + k * TC_B_BYTES + tc_off(co, 8 * h)) = v;
    }
    int X = 0, Y = 0, Z = 0;
    if (valid) xyz_of(g, n, X, Y, Z);
    for (int k = 0; k < K27; k++) {
        const int j = valid ? nbr_off(g, X, Y, Z, flip ? 26 - k : k) : -1;
        uint4 v0 = make_uint4(0u, 0u, 0u, 0u), v1 = v0;
        if (j >= 0) {
            const uint4 *src = (const uint4 *)(in + (size_t)j * 16);
            v0 = src[0];
            v1 = src[1];
        }
        *(uint4 *)(sA + k * TC_A_BYTES + tc_off(tid, 0)) = v0;
        *(uint4 *)(sA + k * TC_A_BYTES + tc_off(tid, 8)) = v1;
    }
    // make the generic-proxy writes visible to the tensor cores' async proxy
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t tmem = *tmem_slot;
    if (tid == 0) {
        const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sB);
        for (int k = 0; k < K27; k++) {
            const uint64_t ad = tc_desc(a0 + k * TC_A_BYTES, 128, 256);
            const uint64_t bd = tc_desc(b0 + k * TC_B_BYTES, 128, 256);
            const uint32_t acc = k > 0;
            asm volatile(
                "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                "l"(ad), "l"(bd), "r"(TC_IDESC), "r"(acc));
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
            smem_u32(mbar)));
    }
    // bounded wait for the MMAs (phase 0 of the mbarrier)
    uint32_t done = tc_wait(mbar);
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    if (!done) {
        // give up: raise the status, wait once more (bounded) for the MMAs
        // still in flight, then free the tensor memory below
        if (lane == 0) atomicExch(&tc_status, 1);
        done = tc_wait(mbar);
    } else {
        uint32_t d[16];
        const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16);
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
            "%14, %15}, [%16];\n"
            : "=r"(d[0]), "=r"(d[1]), "=r"(d[2]), "=r"(d[3]), "=r"(d[4]), "=r"(d[5]), "=r"(d[6]), "=r"(d[7]),
              "=r"(d[8]), "=r"(d[9]), "=r"(d[10]), "=r"(d[11]), "=r"(d[12]), "=r"(d[13]), "=r"(d[14]), "=r"(d[15])
            : "r"(taddr));
        asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
        if (valid) {
            float v[16];
#pragma unroll
            for (int co = 0; co < 16; co++) {
                v[co] = __uint_as_float(d[co]) + (bias ? bias[co] : 0.f);
                if (RELU) v[co] = fmaxf(v[co], 0.f);
                // gradient through the ReLU of the layer that produced relu_mask_src
                if (relu_mask_src && !(__bfloat162float(relu_mask_src[(size_t)n * 16 + co]) > 0.f)) v[co] = 0.f;
            }
            __nv_bfloat162 *o = (__nv_bfloat162 *)(out + (size_t)n * 16);
#pragma unroll
            for (int c = 0; c < 8; c++) o[c] = __floats2bfloat162_rn(v[2 * c], v[2 * c + 1]);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 32;\n" ::"r"(tmem));
}

// which kernel runs the 16 -> 16 layers: 1 = tcgen05 (default), 0 = mma.sync
int g_tensor_path = 1;

template <bool RELU>
void conv16(const NetGrid &g, const __nv_bfloat16 *in, const __nv_bfloat16 *Wt, const float *bias, int flip,
            __nv_bfloat16 *out, const __nv_bfloat16 *relu_mask_src, cudaStream_t s)
{
    if (g_tensor_path) {
        static bool attr = false;
        if (!attr) {
            cudaFuncSetAttribute(conv16_tc<RELU>, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM);
            attr = true;
        }
        conv16_tc<RELU><<<(g.N + TC_M - 1) / TC_M, TC_M, TC_SMEM, s>>>(g, in, Wt, bias, flip, out, relu_mask_src);
    } else {
        conv16_mma<RELU, false><<<(g.N + 127) / 128, 256, 0, s>>>(g, in, Wt, bias, flip, out, relu_mask_src);
    }
}

// BF16 B-operand tables of a 16->16 layer: forward Wt[k][co][ci] = W[co][ci][k];
// data gradient Wb[k][ci][co] = W[co][ci][k] (used with flipped offsets).
__global__ void prep_w16(const float *__restrict__ w, int ow, __nv_bfloat16 *__restrict__ Wf, __nv_bfloat16 *__restrict__ Wb)
{
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 27 * 16 * 16) return;
    int k = t / 256, r = t % 256, co = r / 16, ci = r % 16;
    float v = w[ow + (co * 16 + ci) * 27 + k];
    Wf[(k * 16 + co) * 16 + ci] = __float2bfloat16_rn(v);
    Wb[(k * 16 + ci) * 16 + co] = __float2bfloat16_rn(v);
}

// ---------------------------------------------------------------- layer 4
__global__ void __launch_bounds__(NT) l4_fwd(NetGrid g, const __nv_bfloat16 *__restrict__ act, const float *__restrict__ w,
                                             float *__restrict__ y)
{
    __shared__ float sw[16 * 27 + 1];
    for (int t = threadIdx.x; t < 16 * 27 + 1; t += blockDim.x) sw[t] = w[OW4 + t];
    __syncthreads();
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= g.N) return;
    int X, Y, Z;
    xyz_of(g, n, X, Y, Z);
    float acc = sw[16 * 27];
    for (int k = 0; k < K27; k++) {
        const int j = nbr_off(g, X, Y, Z, k);
        if (j < 0) continue;
        const __nv_bfloat162 *a = (const __nv_bfloat162 *)(act + (size_t)j * 16);
        for (int c = 0; c < 8; c++) {
            float2 v = __bfloat1622float2(a[c]);
            acc += sw[(2 * c) * 27 + k] * v.x + sw[(2 * c + 1) * 27 + k] * v.y;
        }
    }
    y[n] = acc;
}

// loss gradient g = 2 (y - t) / cnt on masked nodes; per-block loss partials
__global__ void __launch_bounds__(NT) loss_grad_k(int N, const float *y, const float *t, const uint8_t *mask, float inv_cnt,
                                                  float *g, double *part)
{
    __shared__ double sh[NT / 32];
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    float l = 0.f;
    if (n < N) {
        float d = (mask == nullptr || mask[n]) ? y[n] - t[n] : 0.f;
        g[n] = 2.f * d * inv_cnt;
        l = d * d;
    }
    double s = block_sum((double)l, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// d_act3[m][ci] = relu'(act3) * sum_k W4[ci][k] g[m - off_k]  (BF16 out)
__global__ void __launch_bounds__(NT) l4_bwd_data(NetGrid g, const float *__restrict__ gy, const float *__restrict__ w,
                                                  const __nv_bfloat16 *__restrict__ act3, __nv_bfloat16 *__restrict__ dz)
{
    __shared__ float sw[16 * 27];
    for (int t = threadIdx.x; t < 16 * 27; t += blockDim.x) sw[t] = w[OW4 + t];
    __syncthreads();
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= g.N) return;
    int X, Y, Z;
    xyz_of(g, m, X, Y, Z);
    float acc[16];
    for (int c = 0; c < 16; c++) acc[c] = 0.f;
    for (int k = 0; k < K27; k++) {
        const int j = nbr_off(g, X, Y, Z, 26 - k);  // m - off_k
        if (j < 0) continue;
        const float gv = gy[j];
        for (int c = 0; c < 16; c++) acc[c] += sw[c * 27 + k] * gv;
    }
    for (int c = 0; c < 16; c += 2) {
        float v0 = __bfloat162float(act3[(size_t)m * 16 + c]) > 0.f ? acc[c] : 0.f;
        float v1 = __bfloat162float(act3[(size_t)m * 16 + c + 1]) > 0.f ? acc[c + 1] : 0.f;
        *(__nv_bfloat162 *)(dz + (size_t)m * 16 + c) = __floats2bfloat162_rn(v0, v1);
    }
}

// ---------------------------------------------------------------- weight gradients
// Per-block partials of dW[co][ci][k] = sum_n dz[n][co] a[ci][n + off_k] and
// db[co] = sum_n dz[n][co], for CI input channels stored either as BF16
// node-major [n][16] (hidden) or FP32 channel-major [ci][N] (network input),
// CO output channels stored as BF16 [n][16] or FP32 [N] (CO = 1).
template <int CI, int CO>
__global__ void __launch_bounds__(NT) wgrad_partial(NetGrid g, const void *a_in, int a_bf16, const void *dz, int dz_bf16,
                                                    float *part)
{
    constexpr int NW = CO * CI * 27 + CO;
    constexpr int CH = 16;  // nodes per shared-memory chunk
    __shared__ float sa[CH][CI][27];
    __shared__ float sd[CH][CO];
    float acc[(NW + NT - 1) / NT];
    for (int q = 0; q < (NW + NT - 1) / NT; q++) acc[q] = 0.f;
    const int base = blockIdx.x * 512;
    for (int chunk = 0; chunk < 512; chunk += CH) {
        __syncthreads();
        for (int t = threadIdx.x; t < CH * CI * 27; t += blockDim.x) {
            int nn = t / (CI * 27), r = t % (CI * 27), ci = r / 27, k = r % 27;
            int n = base + chunk + nn;
            float v = 0.f;
            if (n < g.N) {
                int X, Y, Z;
                xyz_of(g, n, X, Y, Z);
                int j = nbr_off(g, X, Y, Z, k);
                if (j >= 0)
                    v = a_bf16 ? __bfloat162float(((const __nv_bfloat16 *)a_in)[(size_t)j * 16 + ci])
                               : ((const float *)a_in)[(size_t)ci * g.N + j];
            }
            sa[nn][ci][k] = v;
        }
        for (int t = threadIdx.x; t < CH * CO; t += blockDim.x) {
            int nn = t / CO, co = t % CO, n = base + chunk + nn;
            float v = 0.f;
            if (n < g.N)
                v = dz_bf16 ? __bfloat162float(((const __nv_bfloat16 *)dz)[(size_t)n * 16 + co])
                            : ((const float *)dz)[n];
            sd[nn][co] = v;
        }
        __syncthreads();
        for (int q = 0; q < (NW + NT - 1) / NT; q++) {
            int wi = q * NT + threadIdx.x;
            if (wi >= NW) break;
            float s = 0.f;
            if (wi < CO * CI * 27) {
                int co = wi / (CI * 27), r = wi % (CI * 27), ci = r / 27, k = r % 27;
                for (int nn = 0; nn < CH; nn++) s += sd[nn][co] * sa[nn][ci][k];
            } else {
                int co = wi - CO * CI * 27;
                for (int nn = 0; nn < CH; nn++) s += sd[nn][co];
            }
            acc[q] += s;
        }
    }
    for (int q = 0; q < (NW + NT - 1) / NT; q++) {
        int wi = q * NT + threadIdx.x;
        if (wi < NW) part[(size_t)blockIdx.x * NW + wi] = acc[q];
    }
}

// grad[o + i] += sum over blocks (fixed order) of part[b][i]
__global__ void reduce_partials(const float *part, int nblocks, int nw, float *grad, int o)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nw) return;
    float s = 0.f;
    for (int b = 0; b < nblocks; b++) s += part[(size_t)b * nw + i];
    grad[o + i] += s;
}

// Adam (Kingma & Ba) on the FP32 master parameters
__global__ void adam_k(int n, float *w, const float *g, float *m, float *v, float lr, float b1, float b2, float eps,
                       float c1, float c2)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float gi = g[i];
    m[i] = b1 * m[i] + (1.f - b1) * gi;
    v[i] = b2 * v[i] + (1.f - b2) * gi * gi;
    w[i] -= lr * (m[i] / c1) / (sqrtf(v[i] / c2) + eps);
}

// ---------------------------------------------------------------- host side
struct NetWork {
    NetGrid g;
    float *x = nullptr;         // [2][N]
    __nv_bfloat16 *a1 = nullptr, *a2 = nullptr, *a3 = nullptr, *dz = nullptr, *dz2 = nullptr;
    float *y = nullptr, *gy = nullptr;
    float *w = nullptr, *grad = nullptr;
    __nv_bfloat16 *W2f = nullptr, *W2b = nullptr, *W3f = nullptr, *W3b = nullptr;
    float *part = nullptr;
    double *lpart = nullptr;
    size_t part_floats = 0;
    int cap = 0;
};

int cuda_err(cudaError_t e) { return e == cudaSuccess ? EKL_OK : EKL_ERR_CUDA; }

int work_alloc(NetWork &W, int N)
{
    if (N <= W.cap) return EKL_OK;
    cudaFree(W.x); cudaFree(W.a1); cudaFree(W.a2); cudaFree(W.a3); cudaFree(W.dz); cudaFree(W.dz2);
    cudaFree(W.y); cudaFree(W.gy); cudaFree(W.part); cudaFree(W.lpart);
    const int nblk_w = (N + 511) / 512;
    W.part_floats = (size_t)nblk_w * (16 * 16 * 27 + 16);
    cudaError_t e = cudaMalloc(&W.x, 2 * (size_t)N * 4);
    if (e == cudaSuccess) e = cudaMalloc(&W.a1, (size_t)N * 32);
    if (e == cudaSuccess) e = cudaMalloc(&W.a2, (size_t)N * 32);
    if (e == cudaSuccess) e = cudaMalloc(&W.a3, (size_t)N * 32);
    if (e == cudaSuccess) e = cudaMalloc(&W.dz, (size_t)N * 32);
    if (e == cudaSuccess) e = cudaMalloc(&W.dz2, (size_t)N * 32);
    if (e == cudaSuccess) e = cudaMalloc(&W.y, (size_t)N * 4);
    if (e == cudaSuccess) e = cudaMalloc(&W.gy, (size_t)N * 4);
    if (e == cudaSuccess) e = cudaMalloc(&W.part, W.part_floats * 4);
    if (e == cudaSuccess) e = cudaMalloc(&W.lpart, ((N + NT - 1) / NT) * sizeof(double));
    if (!W.w) {
        if (e == cudaSuccess) e = cudaMalloc(&W.w, NPARAM * 4);
        if (e == cudaSuccess) e = cudaMalloc(&W.grad, NPARAM * 4);
        if (e == cudaSuccess) e = cudaMalloc(&W.W2f, 27 * 256 * 2);
        if (e == cudaSuccess) e = cudaMalloc(&W.W2b, 27 * 256 * 2);
        if (e == cudaSuccess) e = cudaMalloc(&W.W3f, 27 * 256 * 2);
        if (e == cudaSuccess) e = cudaMalloc(&W.W3b, 27 * 256 * 2);
    }
    if (e != cudaSuccess) return EKL_ERR_ALLOC;
    W.cap = N;
    return EKL_OK;
}

void work_free(NetWork &W)
{
    cudaFree(W.x); cudaFree(W.a1); cudaFree(W.a2); cudaFree(W.a3); cudaFree(W.dz); cudaFree(W.dz2);
    cudaFree(W.y); cudaFree(W.gy); cudaFree(W.part); cudaFree(W.lpart); cudaFree(W.w); cudaFree(W.grad);
    cudaFree(W.W2f); cudaFree(W.W2b); cudaFree(W.W3f); cudaFree(W.W3b);
    W = NetWork();
}

// forward pass on W.x with the parameters in W.w; output in W.y
void net_forward(NetWork &W, cudaStream_t s)
{
    const NetGrid &g = W.g;
    prep_w16<<<27, 256, 0, s>>>(W.w, OW2, W.W2f, W.W2b);
    prep_w16<<<27, 256, 0, s>>>(W.w, OW3, W.W3f, W.W3b);
    const int bn = (g.N + NT - 1) / NT;
    l1_fwd<<<bn, NT, 0, s>>>(g, W.x, W.w, W.a1);
    conv16<true>(g, W.a1, W.W2f, W.w + OB2, 0, W.a2, nullptr, s);
    conv16<true>(g, W.a2, W.W3f, W.w + OB3, 0, W.a3, nullptr, s);
    l4_fwd<<<bn, NT, 0, s>>>(g, W.a3, W.w, W.y);
}

// loss and gradient (W.grad) for target t and mask on W.x
int net_backward(NetWork &W, const float *d_t, const uint8_t *d_mask, float inv_cnt, double *loss, cudaStream_t s)
{
    const NetGrid &g = W.g;
    const int bn = (g.N + NT - 1) / NT;
    const int bw = (g.N + 511) / 512;
    loss_grad_k<<<bn, NT, 0, s>>>(g.N, W.y, d_t, d_mask, inv_cnt, W.gy, W.lpart);
    // layer 4
    wgrad_partial<16, 1><<<bw, NT, 0, s>>>(g, W.a3, 1, W.gy, 0, W.part);
    reduce_partials<<<(16 * 27 + 1 + 255) / 256, 256, 0, s>>>(W.part, bw, 16 * 27 + 1, W.grad, OW4);
    l4_bwd_data<<<bn, NT, 0, s>>>(g, W.gy, W.w, W.a3, W.dz);
    // layer 3: dz holds d z3 (through relu of a3)
    wgrad_partial<16, 16><<<bw, NT, 0, s>>>(g, W.a2, 1, W.dz, 1, W.part);
    reduce_partials<<<(16 * 16 * 27 + 16 + 255) / 256, 256, 0, s>>>(W.part, bw, 16 * 16 * 27 + 16, W.grad, OW3);
    conv16<false>(g, W.dz, W.W3b, nullptr, 1, W.dz2, W.a2, s);
    // layer 2
    wgrad_partial<16, 16><<<bw, NT, 0, s>>>(g, W.a1, 1, W.dz2, 1, W.part);
    reduce_partials<<<(16 * 16 * 27 + 16 + 255) / 256, 256, 0, s>>>(W.part, bw, 16 * 16 * 27 + 16, W.grad, OW2);
    conv16<false>(g, W.dz2, W.W2b, nullptr, 1, W.dz, W.a1, s);
    // layer 1
    wgrad_partial<2, 16><<<bw, NT, 0, s>>>(g, W.x, 0, W.dz, 1, W.part);
    reduce_partials<<<(16 * 2 * 27 + 16 + 255) / 256, 256, 0, s>>>(W.part, bw, 16 * 2 * 27 + 16, W.grad, OW1);
    if (loss) {
        std::vector<double> lp(bn);
        cudaError_t e = cudaMemcpyAsync(lp.data(), W.lpart, bn * sizeof(double), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return EKL_ERR_CUDA;
        double t = 0;
        for (int b = 0; b < bn; b++) t += lp[b];
        *loss = t * inv_cnt;
    }
    return cuda_err(cudaGetLastError());
}

NetGrid make_grid(const int32_t dims[3], const int32_t periodic[3])
{
    NetGrid g;
    g.nx = dims[0];
    g.ny = dims[1];
    g.nz = dims[2];
    for (int a = 0; a < 3; a++) g.per[a] = periodic ? (periodic[a] ? 1 : 0) : 0;
    g.N = g.nx * g.ny * g.nz;
    return g;
}

// ---------------------------------------------------------------- in-step warm start
struct WarmStart {
    NetWork W;               // on the lattice (level 0) or on cubes of 2^level nodes
    float s_db = 1.f, s_phi = 1.f, s_out = 1.f;
    int enabled = 0;
    int have_prev = 0;
    int level = 0;
    NetGrid fine;            // the lattice
    float *bprev = nullptr, *bcur = nullptr, *phiprev = nullptr;
    float *dbf = nullptr, *phf = nullptr;  // level > 0: the lattice's inputs before restriction
    double *mean = nullptr;
    int collect = 0, crop = 0, ncrops = 0;
    float *crops = nullptr;  // [cap][3][crop^3]: dB, phi_prev, dphi
    long long cap = 0, used = 0;
    uint64_t seed = 0;
};

__global__ void mean_k(const double *part, int n, double nfl, double *mean)
{
    __shared__ double sh[32];
    double v = 0.0;
    for (int k = threadIdx.x; k < n; k += blockDim.x) v += part[k];
    double t = block_sum(v, sh);
    if (threadIdx.x == 0) *mean = nfl > 0 ? t / nfl : 0.0;
}

// network inputs on the lattice: x0 = s_db (b(t) - b(t-1)), x1 = s_phi phi(t-1);
// b = 4 pi l_B (rho - mean)
template <typename R, typename PhiT>
__global__ void ws_inputs(int N, const uint32_t *mask, const R *rho, const double *mean, double c4, const PhiT *phi,
                          const float *bprev, int have_prev, float s_db, float s_phi, float *x0, float *x1,
                          float *bcur, float *phiprev)
{
    int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const bool solid = mask[n] & SOLID_BIT;
    float b = solid ? 0.f : (float)(c4 * ((double)rho[n] - *mean));
    float p;
    if constexpr (((PhiT)0.5) != 0) p = (float)phi[n];
    else p = ll_to_float(phi[n]) * (float)PHI_INV;
    if (solid) p = 0.f;
    bcur[n] = b;
    if (phiprev) phiprev[n] = p;
    x0[n] = solid ? 0.f : s_db * (b - (have_prev ? bprev[n] : b));
    x1[n] = s_phi * p;
}

// The network on a coarse level: cell (X, Y, Z) of level L covers the cube
// of 2^L nodes starting at 2^L (X, Y, Z).  Inputs: x0 = s_db times the sum of
// the change of the source over the cube (the source a coarse Poisson
// operator sees), x1 = s_phi times the mean of phi(t-1) over its fluid nodes.
__global__ void ws_restrict(NetGrid f, NetGrid c, int L, const uint32_t *mask, const float *db, const float *ph,
                            float s_db, float s_phi, float *x)
{
    const int I = blockIdx.x * blockDim.x + threadIdx.x;
    if (I >= c.N) return;
    int X, Y, Z;
    xyz_of(c, I, X, Y, Z);
    const int B = 1 << L;
    double sd = 0.0, sp = 0.0;
    int cnt = 0;
    for (int dz = 0; dz < B; dz++)
        for (int dy = 0; dy < B; dy++)
            for (int dx = 0; dx < B; dx++) {
                const int n = (X * B + dx) + f.nx * ((Y * B + dy) + f.ny * (Z * B + dz));
                if (mask[n] & SOLID_BIT) continue;
                sd += (double)db[n];
                sp += (double)ph[n];
                cnt++;
            }
    x[I] = (float)(s_db * sd);
    x[c.N + I] = cnt ? (float)(s_phi * (sp / cnt)) : 0.f;
}

// mean over the fluid nodes of each cube of phi(t) - phi(t-1): the training
// target of the coarse network
template <typename PhiT>
__global__ void ws_coarse_target(NetGrid f, NetGrid c, int L, const uint32_t *mask, const PhiT *phi,
                                 const float *phiprev, float *out)
{
    const int I = blockIdx.x * blockDim.x + threadIdx.x;
    if (I >= c.N) return;
    int X, Y, Z;
    xyz_of(c, I, X, Y, Z);
    const int B = 1 << L;
    double s = 0.0;
    int cnt = 0;
    for (int dz = 0; dz < B; dz++)
        for (int dy = 0; dy < B; dy++)
            for (int dx = 0; dx < B; dx++) {
                const int n = (X * B + dx) + f.nx * ((Y * B + dy) + f.ny * (Z * B + dz));
                if (mask[n] & SOLID_BIT) continue;
                float pn;
                if constexpr (((PhiT)0.5) != 0) pn = (float)phi[n];
                else pn = ll_to_float(phi[n]) * (float)PHI_INV;
                s += (double)(pn - phiprev[n]);
                cnt++;
            }
    out[I] = cnt ? (float)(s / cnt) : 0.f;
}

// phi += s_out y(cube of the node) on the fluid nodes (piecewise-constant
// prolongation of the coarse network's output)
template <typename PhiT>
__global__ void ws_apply_coarse(NetGrid f, NetGrid c, int L, const uint32_t *mask, const float *y, float s_out,
                                PhiT *phi)
{
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= f.N || (mask[n] & SOLID_BIT)) return;
    int x, yy, z;
    xyz_of(f, n, x, yy, z);
    const float d = s_out * y[(x >> L) + c.nx * ((yy >> L) + c.ny * (z >> L))];
    if constexpr (((PhiT)0.5) != 0) phi[n] += (double)d;
    else phi[n] += float_to_ll(d * (float)PHI_SCALE);
}

template <typename PhiT>
__global__ void ws_apply(int N, const uint32_t *mask, const float *y, float s_out, PhiT *phi)
{
    int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N || (mask[n] & SOLID_BIT)) return;
    const float d = s_out * y[n];
    if constexpr (((PhiT)0.5) != 0) phi[n] += (double)d;
    else phi[n] += float_to_ll(d * (float)PHI_SCALE);
}

// training crops centred on beads (seeded jitter): inputs and the change of
// the converged potential
template <typename PhiT>
__global__ void ws_crops(NetGrid g, const float *x, const float *phiprev, const PhiT *phi, const double *Rb,
                         int nb, int crop, int ncrops, long long step, uint64_t seed, float *out)
{
    const int j = blockIdx.x;
    const int c3 = crop * crop * crop;
    const int b = (int)((step * ncrops + j) % nb);
    uint32_t ctr[4] = {(uint32_t)j, 3u << 24, (uint32_t)step, (uint32_t)((uint64_t)step >> 32)};
    philox4x32_10(ctr, (uint32_t)seed, (uint32_t)(seed >> 32));
    int o[3];
    for (int a = 0; a < 3; a++) {
        int jit = (int)(ctr[a] % 5u) - 2;
        o[a] = (int)floor(Rb[3 * b + a]) + jit - crop / 2;
    }
    for (int t = threadIdx.x; t < c3; t += blockDim.x) {
        int cx = t % crop, cy = (t / crop) % crop, cz = t / (crop * crop);
        int q[3] = {o[0] + cx, o[1] + cy, o[2] + cz};
        const int dims[3] = {g.nx, g.ny, g.nz};
        bool in = true;
        for (int a = 0; a < 3; a++) {
            if (q[a] < 0 || q[a] >= dims[a]) {
                if (g.per[a]) q[a] = ((q[a] % dims[a]) + dims[a]) % dims[a];
                else in = false;
            }
        }
        float v0 = 0.f, v1 = 0.f, v2 = 0.f;
        if (in) {
            int n = q[0] + g.nx * (q[1] + g.ny * q[2]);
            v0 = x[n];
            v1 = x[g.N + n];
            float pn;
            if constexpr (((PhiT)0.5) != 0) pn = (float)phi[n];
            else pn = ll_to_float(phi[n]) * (float)PHI_INV;
            v2 = (v1 == 0.f && phiprev[n] == 0.f) ? 0.f : pn - phiprev[n];
        }
        float *dst = out + (size_t)j * 3 * c3;
        dst[t] = v0;
        dst[c3 + t] = v1;
        dst[2 * c3 + t] = v2;
    }
}

}  // namespace

namespace ekl {

int warmstart_before_poisson(Ctx &c)
{
    WarmStart &ws = *(WarmStart *)c.net;
    const int N = (int)c.N;
    mean_k<<<1, 1024, 0, c.stream>>>(c.part_charge, c.charge_blocks, (double)c.n_fluid, ws.mean);
    const int bn = (N + 255) / 256;
    const int have = ws.have_prev;
    const int L = ws.level;
    // level 0: the inputs go straight to the network; level > 0: unscaled
    // into the lattice buffers, then restricted (and scaled) per cube
    float *x0 = L ? ws.dbf : ws.W.x, *x1 = L ? ws.phf : ws.W.x + N;
    const float sdb = L ? 1.f : ws.s_db, sph = L ? 1.f : ws.s_phi;
    if (c.prec == EKL_F64)
        ws_inputs<double, double><<<bn, 256, 0, c.stream>>>(N, c.mask, (const double *)c.rho, ws.mean, c.c4,
                                                           (const double *)c.phi, ws.bprev, have, sdb, sph, x0, x1,
                                                           ws.bcur, ws.collect ? ws.phiprev : nullptr);
    else
        ws_inputs<float, long long><<<bn, 256, 0, c.stream>>>(N, c.mask, (const float *)c.rho, ws.mean, c.c4,
                                                             (const long long *)c.phi, ws.bprev, have, sdb, sph, x0,
                                                             x1, ws.bcur, ws.collect ? ws.phiprev : nullptr);
    c.launches += 2;
    if (L) {
        ws_restrict<<<(ws.W.g.N + 255) / 256, 256, 0, c.stream>>>(ws.fine, ws.W.g, L, c.mask, ws.dbf, ws.phf,
                                                                  ws.s_db, ws.s_phi, ws.W.x);
        c.launches++;
    }
    if (ws.enabled && have) {
        net_forward(ws.W, c.stream);
        if (L) {
            if (c.prec == EKL_F64)
                ws_apply_coarse<double><<<bn, 256, 0, c.stream>>>(ws.fine, ws.W.g, L, c.mask, ws.W.y, ws.s_out,
                                                                  (double *)c.phi);
            else
                ws_apply_coarse<long long><<<bn, 256, 0, c.stream>>>(ws.fine, ws.W.g, L, c.mask, ws.W.y, ws.s_out,
                                                                     (long long *)c.phi);
        } else {
            if (c.prec == EKL_F64) ws_apply<double><<<bn, 256, 0, c.stream>>>(N, c.mask, ws.W.y, ws.s_out, (double *)c.phi);
            else ws_apply<long long><<<bn, 256, 0, c.stream>>>(N, c.mask, ws.W.y, ws.s_out, (long long *)c.phi);
        }
        c.launches += 7;
    }
    std::swap(ws.bprev, ws.bcur);
    ws.have_prev = 1;
    return cudaGetLastError() == cudaSuccess ? EKL_OK : EKL_ERR_CUDA;
}

int warmstart_after_poisson(Ctx &c)
{
    WarmStart &ws = *(WarmStart *)c.net;
    if (ws.collect && ws.level && ws.used < ws.cap) {
        // one sample per step: the whole coarse grid (inputs as fed, target)
        const size_t NL = (size_t)ws.W.g.N;
        float *dst = ws.crops + (size_t)ws.used * 3 * NL;
        cudaMemcpyAsync(dst, ws.W.x, 2 * NL * 4, cudaMemcpyDeviceToDevice, c.stream);
        if (c.prec == EKL_F64)
            ws_coarse_target<double><<<(ws.W.g.N + 255) / 256, 256, 0, c.stream>>>(
                ws.fine, ws.W.g, ws.level, c.mask, (const double *)c.phi, ws.phiprev, dst + 2 * NL);
        else
            ws_coarse_target<long long><<<(ws.W.g.N + 255) / 256, 256, 0, c.stream>>>(
                ws.fine, ws.W.g, ws.level, c.mask, (const long long *)c.phi, ws.phiprev, dst + 2 * NL);
        c.launches++;
        ws.used++;
        return cudaGetLastError() == cudaSuccess ? EKL_OK : EKL_ERR_CUDA;
    }
    if (!ws.collect || ws.level || c.nb == 0 || ws.used + ws.ncrops > ws.cap) return EKL_OK;
    const size_t c3 = (size_t)ws.crop * ws.crop * ws.crop;
    float *dst = ws.crops + (size_t)ws.used * 3 * c3;
    if (c.prec == EKL_F64)
        ws_crops<double><<<ws.ncrops, 256, 0, c.stream>>>(ws.W.g, ws.W.x, ws.phiprev, (const double *)c.phi,
                                                         (const double *)c.R, c.nb, ws.crop, ws.ncrops, c.step,
                                                         ws.seed, dst);
    else
        ws_crops<long long><<<ws.ncrops, 256, 0, c.stream>>>(ws.W.g, ws.W.x, ws.phiprev, (const long long *)c.phi,
                                                            (const double *)c.R, c.nb, ws.crop, ws.ncrops, c.step,
                                                            ws.seed, dst);
    c.launches++;
    ws.used += ws.ncrops;
    return cudaGetLastError() == cudaSuccess ? EKL_OK : EKL_ERR_CUDA;
}

void warmstart_free(Ctx &c)
{
    if (!c.net) return;
    WarmStart *ws = (WarmStart *)c.net;
    work_free(ws->W);
    cudaFree(ws->bprev);
    cudaFree(ws->bcur);
    cudaFree(ws->phiprev);
    cudaFree(ws->dbf);
    cudaFree(ws->phf);
    cudaFree(ws->mean);
    cudaFree(ws->crops);
    delete ws;
    c.net = nullptr;
}

// the warm start's state on the network level `level` (recreated when the
// level changes; the parameters are installed afterwards)
static int warmstart_ensure(Ctx &c, int level = -1)
{
    if (c.net && (level < 0 || ((WarmStart *)c.net)->level == level)) return EKL_OK;
    if (c.net) warmstart_free(c);
    if (level < 0) level = 0;
    WarmStart *ws = new (std::nothrow) WarmStart();
    if (!ws) return EKL_ERR_ALLOC;
    const int32_t dims[3] = {c.nx, c.ny, c.nz};
    ws->fine = make_grid(dims, c.per);
    ws->level = level;
    const int32_t cdims[3] = {c.nx >> level, c.ny >> level, c.nz >> level};
    ws->W.g = make_grid(cdims, c.per);
    const int N = (int)c.N;
    int rc = work_alloc(ws->W, ws->W.g.N);
    cudaError_t e = rc == EKL_OK ? cudaSuccess : cudaErrorMemoryAllocation;
    if (e == cudaSuccess) e = cudaMalloc(&ws->bprev, (size_t)N * 4);
    if (e == cudaSuccess) e = cudaMalloc(&ws->bcur, (size_t)N * 4);
    if (e == cudaSuccess) e = cudaMalloc(&ws->phiprev, (size_t)N * 4);
    if (e == cudaSuccess && level) e = cudaMalloc(&ws->dbf, (size_t)N * 4);
    if (e == cudaSuccess && level) e = cudaMalloc(&ws->phf, (size_t)N * 4);
    if (e == cudaSuccess) e = cudaMalloc(&ws->mean, sizeof(double));
    c.net = ws;
    if (e != cudaSuccess) {
        warmstart_free(c);
        return EKL_ERR_ALLOC;
    }
    return EKL_OK;
}

}  // namespace ekl

// EKL_ERR_TIMEOUT when a tensor-core block gave up waiting for its MMAs
// (the flag is cleared on reading)
static int tc_check()
{
    int st = 0;
    if (cudaMemcpyFromSymbol(&st, tc_status, sizeof(int)) != cudaSuccess) return EKL_ERR_CUDA;
    if (!st) return EKL_OK;
    const int zero = 0;
    cudaMemcpyToSymbol(tc_status, &zero, sizeof(int));
    return EKL_ERR_TIMEOUT;
}

extern "C" {

int ekl_net_tensor_path(int32_t path)
{
    const int prev = g_tensor_path;
    if (path == 0 || path == 1) g_tensor_path = path;
    return prev;
}

int ekl_net_eval(const int32_t dims[3], const int32_t periodic[3], const float *x, const float *w, float *y)
{
    if (!dims || !x || !w || !y || dims[0] < 1 || dims[1] < 1 || dims[2] < 1) return EKL_ERR_ARG;
    NetWork W;
    W.g = make_grid(dims, periodic);
    int rc = work_alloc(W, W.g.N);
    if (rc != EKL_OK) { work_free(W); return rc; }
    cudaError_t e = cudaMemcpy(W.x, x, 2 * (size_t)W.g.N * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(W.w, w, NPARAM * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        net_forward(W, 0);
        e = cudaMemcpy(y, W.y, (size_t)W.g.N * 4, cudaMemcpyDeviceToHost);
    }
    work_free(W);
    if (e == cudaSuccess) return tc_check();
    return cuda_err(e);
}

int ekl_net_loss_grad(const int32_t dims[3], const int32_t periodic[3], const float *x, const float *target,
                      const uint8_t *mask, const float *w, double *loss, float *grad)
{
    if (!dims || !x || !target || !w || !grad) return EKL_ERR_ARG;
    NetWork W;
    W.g = make_grid(dims, periodic);
    const int N = W.g.N;
    int rc = work_alloc(W, N);
    if (rc != EKL_OK) { work_free(W); return rc; }
    float *dt = nullptr;
    uint8_t *dm = nullptr;
    long long cnt = N;
    if (mask) {
        cnt = 0;
        for (int i = 0; i < N; i++) cnt += mask[i] ? 1 : 0;
    }
    cudaError_t e = cudaMalloc(&dt, (size_t)N * 4);
    if (e == cudaSuccess && mask) e = cudaMalloc(&dm, N);
    if (e == cudaSuccess) e = cudaMemcpy(W.x, x, 2 * (size_t)N * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(W.w, w, NPARAM * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dt, target, (size_t)N * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && mask) e = cudaMemcpy(dm, mask, N, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(W.grad, 0, NPARAM * 4);
    if (e == cudaSuccess) {
        net_forward(W, 0);
        rc = net_backward(W, dt, dm, 1.f / (float)(cnt > 0 ? cnt : 1), loss, 0);
        if (rc == EKL_OK) e = cudaMemcpy(grad, W.grad, NPARAM * 4, cudaMemcpyDeviceToHost);
    }
    cudaFree(dt);
    cudaFree(dm);
    work_free(W);
    if (rc != EKL_OK) return rc;
    if (e == cudaSuccess) return tc_check();
    return cuda_err(e);
}

int ekl_net_train_grid(int32_t nsamples, const int32_t dims[3], const int32_t periodic[3], const float *x,
                       const float *target, const uint8_t *mask, float *w, int32_t iters, int32_t batch, float lr,
                       uint64_t seed, float *loss_out)
{
    if (nsamples < 1 || !dims || !x || !target || !w || iters < 0 || batch < 1) return EKL_ERR_ARG;
    NetWork W;
    W.g = make_grid(dims, periodic);
    const int N = W.g.N;
    int rc = work_alloc(W, N);
    if (rc != EKL_OK) { work_free(W); return rc; }
    float *dx = nullptr, *dt = nullptr, *m1 = nullptr, *m2 = nullptr;
    uint8_t *dm = nullptr;
    long long cnt = N;
    if (mask) {
        cnt = 0;
        for (int i = 0; i < N; i++) cnt += mask[i] ? 1 : 0;
    }
    cudaError_t e = cudaMalloc(&dx, (size_t)nsamples * 2 * N * 4);
    if (e == cudaSuccess) e = cudaMalloc(&dt, (size_t)nsamples * N * 4);
    if (e == cudaSuccess) e = cudaMalloc(&m1, NPARAM * 4);
    if (e == cudaSuccess) e = cudaMalloc(&m2, NPARAM * 4);
    if (e == cudaSuccess && mask) e = cudaMalloc(&dm, N);
    if (e == cudaSuccess) e = cudaMemcpy(dx, x, (size_t)nsamples * 2 * N * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dt, target, (size_t)nsamples * N * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && mask) e = cudaMemcpy(dm, mask, N, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(W.w, w, NPARAM * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(m1, 0, NPARAM * 4);
    if (e == cudaSuccess) e = cudaMemset(m2, 0, NPARAM * 4);
    // seeded sample order (splitmix64)
    uint64_t st = seed;
    auto next = [&]() {
        st += 0x9E3779B97F4A7C15ull;
        uint64_t z = st;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    };
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    for (int it = 0; it < iters && e == cudaSuccess && rc == EKL_OK; it++) {
        cudaMemsetAsync(W.grad, 0, NPARAM * 4, 0);
        double lsum = 0.0;
        for (int bidx = 0; bidx < batch; bidx++) {
            const int smp = (int)(next() % (uint64_t)nsamples);
            e = cudaMemcpyAsync(W.x, dx + (size_t)smp * 2 * N, 2 * (size_t)N * 4, cudaMemcpyDeviceToDevice, 0);
            if (e != cudaSuccess) break;
            net_forward(W, 0);
            double l = 0.0;
            rc = net_backward(W, dt + (size_t)smp * N, dm, 1.f / (float)(cnt * batch), &l, 0);
            lsum += l * batch;
            if (rc != EKL_OK) break;
        }
        const float c1 = 1.f - powf(b1, (float)(it + 1)), c2 = 1.f - powf(b2, (float)(it + 1));
        adam_k<<<(NPARAM + 255) / 256, 256>>>(NPARAM, W.w, W.grad, m1, m2, lr, b1, b2, eps, c1, c2);
        if (loss_out) loss_out[it] = (float)(lsum / batch);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && rc == EKL_OK) e = cudaMemcpy(w, W.w, NPARAM * 4, cudaMemcpyDeviceToHost);
    cudaFree(dx); cudaFree(dt); cudaFree(m1); cudaFree(m2); cudaFree(dm);
    work_free(W);
    if (rc != EKL_OK) return rc;
    if (e == cudaSuccess) return tc_check();
    return cuda_err(e);
}

int ekl_net_train(int32_t nsamples, const int32_t dims[3], const float *x, const float *target,
                  const uint8_t *mask, float *w, int32_t iters, int32_t batch, float lr, uint64_t seed,
                  float *loss_out)
{
    const int32_t closed[3] = {0, 0, 0};
    return ekl_net_train_grid(nsamples, dims, closed, x, target, mask, w, iters, batch, lr, seed, loss_out);
}

}  // extern "C"

extern "C" {

int ekl_warmstart_level(ekl_handle *h, int32_t level)
{
    if (!h || level < 0 || level > 4) return EKL_ERR_ARG;
    ekl::DeviceScope dscope(h->c.device);
    if (!dscope.ok()) {
        ekl::set_last_error("the handle's device cannot be made current");
        return EKL_ERR_ARG;
    }
    ekl::Ctx &c = h->c;
    const int B = 1 << level;
    if (c.nx % B || c.ny % B || c.nz % B) {
        ekl::set_last_error("every extent must be a multiple of 2^level");
        return EKL_ERR_ARG;
    }
    return ekl::warmstart_ensure(c, level);
}

int ekl_set_warmstart(ekl_handle *h, const float *w, const float scales[3])
{
    if (!h) return EKL_ERR_ARG;
    ekl::DeviceScope dscope(h->c.device);
    if (!dscope.ok()) {
        ekl::set_last_error("the handle's device cannot be made current");
        return EKL_ERR_ARG;
    }
    ekl::Ctx &c = h->c;
    if (!w) {
        if (c.net) ((WarmStart *)c.net)->enabled = 0;
        return EKL_OK;
    }
    int rc = ekl::warmstart_ensure(c);
    if (rc != EKL_OK) return rc;
    WarmStart &ws = *(WarmStart *)c.net;
    if (cudaMemcpy(ws.W.w, w, NPARAM * 4, cudaMemcpyHostToDevice) != cudaSuccess) return EKL_ERR_CUDA;
    if (scales) {
        ws.s_db = scales[0];
        ws.s_phi = scales[1];
        ws.s_out = scales[2];
    }
    ws.enabled = 1;
    return EKL_OK;
}

int ekl_warmstart_collect(ekl_handle *h, int32_t nsteps, int32_t crop, int32_t ncrops, uint64_t seed, float *out,
                          int64_t *n_out)
{
    if (!h || nsteps < 1 || ncrops < 1 || !out) return EKL_ERR_ARG;
    ekl::DeviceScope dscope(h->c.device);
    if (!dscope.ok()) {
        ekl::set_last_error("the handle's device cannot be made current");
        return EKL_ERR_ARG;
    }
    ekl::Ctx &c = h->c;
    int rc = ekl::warmstart_ensure(c);
    if (rc != EKL_OK) return rc;
    WarmStart &ws = *(WarmStart *)c.net;
    if (!ws.level && (c.nb == 0 || crop < 4)) return EKL_ERR_ARG;  // bead-centred crops
    const int en = ws.enabled;
    const float s0 = ws.s_db, s1 = ws.s_phi, s2 = ws.s_out;
    ws.enabled = 0;
    ws.s_db = ws.s_phi = ws.s_out = 1.f;
    ws.collect = 1;
    ws.crop = crop;
    ws.ncrops = ncrops;
    ws.seed = seed;
    // level > 0: one sample per step, the whole coarse grid
    ws.cap = ws.level ? (long long)nsteps : (long long)nsteps * ncrops;
    ws.used = 0;
    const size_t c3 = ws.level ? (size_t)ws.W.g.N : (size_t)crop * crop * crop;
    if (cudaMalloc(&ws.crops, (size_t)ws.cap * 3 * c3 * 4) != cudaSuccess) {
        ws.collect = 0;
        return EKL_ERR_ALLOC;
    }
    rc = ekl_step(h, nsteps);
    if (rc >= 0) {
        if (cudaMemcpy(out, ws.crops, (size_t)ws.used * 3 * c3 * 4, cudaMemcpyDeviceToHost) != cudaSuccess)
            rc = EKL_ERR_CUDA;
        if (n_out) *n_out = ws.used;
    }
    cudaFree(ws.crops);
    ws.crops = nullptr;
    ws.collect = 0;
    ws.enabled = en;
    ws.s_db = s0;
    ws.s_phi = s1;
    ws.s_out = s2;
    return rc;
}

}  // extern "C"
