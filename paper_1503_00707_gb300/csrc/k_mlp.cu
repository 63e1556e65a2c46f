// The learned collision operator's network: 64 -> 256 -> 256 -> 256 -> 64 with
// SiLU hidden activations, BF16 weights and activations, FP32 accumulation,
// run and trained on the 5th-generation tensor cores.
//
// Every contraction is one kernel, C[M x N] = A[M x K] . B[N x K]^T with both
// operands BF16 and K contiguous in global memory: a CTA owns 128 rows of C,
// stages 64-wide K chunks of A and B into shared memory in the 128-byte
// swizzled K-major layout (two stages), one thread issues tcgen05.mma
// (M = 128, N <= 256, K = 16 per instruction) into a tensor-memory
// accumulator, and the four warps read their 32 rows back with tcgen05.ld
// for a fused epilogue (bias, SiLU, BF16 rounding, transposed copies).
// Forward, backward (weight gradients as C = dZ^T-by-activation products)
// and the Adam update all run on the device.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "../../include/dvm.h"
#include "async.cuh"
#include "kernels.hpp"
#include "mlp.hpp"
#include "tc.cuh"

namespace dvm {

void count_launch();

namespace {

constexpr int GT = 128;             // threads per GEMM CTA
constexpr uint32_t STAGE_A = 16384; // 128 rows x 128 bytes

struct GemmArgs {
    const __nv_bfloat16 *A;
    int64_t lda;
    const __nv_bfloat16 *B;
    int64_t ldb;
    int64_t M;
    int N;
    int64_t K;              // multiple of 64
    const float *bias;      // [N] or null
    float *Cf;              // FP32 output (pre-activation), [M][ldc], or null
    int64_t ldc;
    __nv_bfloat16 *H;       // BF16 output (activation), [M][ldh], or null
    int64_t ldh;
    __nv_bfloat16 *HT;      // BF16 transposed output, [N][ldt], or null
    int64_t ldt;
    int act;                // 0 none, 1 SiLU
    int *status;
    int vec;                // set by gemm(): Cf and H rows take 16-byte vector stores
};

__device__ inline float silu(float x) { return x / (1.0f + __expf(-x)); }

__global__ void __launch_bounds__(GT) k_gemm(const GemmArgs g)
{
    extern __shared__ unsigned char sraw[];
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ uint32_t tmem_slot;
    __shared__ int abort_flag;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // operand tiles must start on 1024-byte boundaries (swizzle atoms)
    const uint32_t raw = smem_u32(sraw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    unsigned char *sbase = sraw + (base - raw);
    const uint32_t stage_b = (uint32_t)g.N * 128u;
    const uint32_t stage = STAGE_A + stage_b;
    const int64_t m0 = (int64_t)blockIdx.x * 128;
    const uint32_t ncols = g.N <= 32 ? 32u : g.N <= 64 ? 64u : g.N <= 128 ? 128u : 256u;
    const uint32_t idesc = idesc_bf16(128, g.N);

    if (warp == 0) tmem_alloc(&tmem_slot, ncols);
    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        abort_flag = 0;
        mbar_fence_init();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;
    const int64_t nk = g.K / 64;

    for (int64_t kc = 0; kc < nk; kc++) {
        const int s = (int)(kc & 1);
        // the MMAs of chunk kc-2 read this stage
        if (kc >= 2 && !mbar_wait(&bar[s], (uint32_t)((kc - 2) >> 1) & 1u)) abort_flag = 1;
        __syncthreads();
        if (abort_flag) break;
        unsigned char *sa = sbase + (size_t)s * stage;
        unsigned char *sb = sa + STAGE_A;
        for (int i = tid; i < 128 * 8; i += GT) {
            const int r = i >> 3, c = i & 7;
            const int64_t row = m0 + r;
            uint4 v = make_uint4(0, 0, 0, 0);
            if (row < g.M) v = *reinterpret_cast<const uint4 *>(g.A + row * g.lda + kc * 64 + c * 8);
            *reinterpret_cast<uint4 *>(sa + sw128_offset(r, c)) = v;
        }
        for (int i = tid; i < g.N * 8; i += GT) {
            const int r = i >> 3, c = i & 7;
            const uint4 v = *reinterpret_cast<const uint4 *>(g.B + (int64_t)r * g.ldb + kc * 64 + c * 8);
            *reinterpret_cast<uint4 *>(sb + sw128_offset(r, c)) = v;
        }
        fence_proxy_async();
        __syncthreads();
        if (tid == 0) {
            tc_fence_after();
            const uint32_t a_addr = base + (uint32_t)s * stage, b_addr = a_addr + STAGE_A;
#pragma unroll
            for (int ks = 0; ks < 4; ks++)
                tc_mma_bf16(tmem, sw128_desc(a_addr + ks * 32), sw128_desc(b_addr + ks * 32), idesc,
                            kc > 0 || ks > 0);
            tc_commit(&bar[s]);
        }
    }
    if (!abort_flag && nk > 0) {
        const int64_t last = nk - 1;
        if (!mbar_wait(&bar[last & 1], (uint32_t)(last >> 1) & 1u)) abort_flag = 1;
    }
    tc_fence_after();
    __syncthreads();
    if (!abort_flag) {
        const int64_t row = m0 + 32 * warp + lane;
        for (int col = 0; col < g.N; col += 16) {
            float v[16];
            tmem_ld16(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)col, v);
            if (row < g.M && g.vec) {
                // the thread's 16 values of its row: contiguous in Cf and H,
                // so each goes out as 16-byte stores (a column of HT, across
                // the warp's rows, is contiguous as it is)
                float z[16];
                uint32_t hp[8];
#pragma unroll
                for (int j = 0; j < 16; j++) z[j] = v[j] + (g.bias ? g.bias[col + j] : 0.0f);
#pragma unroll
                for (int j = 0; j < 16; j += 2) {
                    const float h0 = g.act ? silu(z[j]) : z[j], h1 = g.act ? silu(z[j + 1]) : z[j + 1];
                    const __nv_bfloat162 p2 = __floats2bfloat162_rn(h0, h1);
                    hp[j / 2] = *reinterpret_cast<const uint32_t *>(&p2);
                    if (g.HT) {
                        g.HT[(int64_t)(col + j) * g.ldt + row] = p2.x;
                        g.HT[(int64_t)(col + j + 1) * g.ldt + row] = p2.y;
                    }
                }
                if (g.Cf) {
                    float4 *d = reinterpret_cast<float4 *>(g.Cf + row * g.ldc + col);
#pragma unroll
                    for (int q = 0; q < 4; q++) d[q] = make_float4(z[4 * q], z[4 * q + 1], z[4 * q + 2], z[4 * q + 3]);
                }
                if (g.H) {
                    uint4 *d = reinterpret_cast<uint4 *>(g.H + row * g.ldh + col);
                    d[0] = make_uint4(hp[0], hp[1], hp[2], hp[3]);
                    d[1] = make_uint4(hp[4], hp[5], hp[6], hp[7]);
                }
            } else if (row < g.M) {
#pragma unroll
                for (int j = 0; j < 16; j++) {
                    float z = v[j] + (g.bias ? g.bias[col + j] : 0.0f);
                    if (g.Cf) g.Cf[row * g.ldc + col + j] = z;
                    const float h = g.act ? silu(z) : z;
                    const __nv_bfloat16 hb = __float2bfloat16_rn(h);
                    if (g.H) g.H[row * g.ldh + col + j] = hb;
                    if (g.HT) g.HT[(int64_t)(col + j) * g.ldt + row] = hb;
                }
            }
        }
    } else if (tid == 0) {
        atomicOr(g.status, ST_TIMEOUT);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, ncols);
}

int gemm(const GemmArgs &g0, cudaStream_t s)
{
    GemmArgs g = g0;
    if (g.M <= 0) return DVM_OK;
    g.vec = (reinterpret_cast<uintptr_t>(g.Cf) % 16 == 0 && g.ldc % 4 == 0 &&
             reinterpret_cast<uintptr_t>(g.H) % 16 == 0 && g.ldh % 8 == 0) ? 1 : 0;
    if (g.K % 64 || g.N % 16 || g.N < 16 || g.N > 256) return DVM_EINVAL;
    const size_t dyn = 2 * (size_t)(STAGE_A + (uint32_t)g.N * 128u) + 1024;
    static bool configured = false;
    if (!configured) {
        if (cudaFuncSetAttribute(k_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, 2 * (16384 + 32768) + 1024) !=
            cudaSuccess)
            return DVM_ECUDA;
        configured = true;
    }
    k_gemm<<<(unsigned)((g.M + 127) / 128), GT, dyn, s>>>(g);
    count_launch();
    return cudaGetLastError() == cudaSuccess ? DVM_OK : DVM_ECUDA;
}

// ---- elementwise kernels ------------------------------------------------------
__global__ void k_to_bf16(const float *x, __nv_bfloat16 *y, __nv_bfloat16 *yt, int64_t n, int cols, int64_t ldt)
{
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n * cols; q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = q / cols;
        const int c = (int)(q - r * cols);
        const __nv_bfloat16 b = __float2bfloat16_rn(x[q]);
        if (y) y[q] = b;
        if (yt) yt[(int64_t)c * ldt + r] = b;
    }
}

// dO = 2 (O - T) / (n * 64), accumulate the squared error
__global__ void k_out_grad(const float *O, const float *T, int64_t n, __nv_bfloat16 *dO, __nv_bfloat16 *dOt,
                           int64_t ldt, float *dOf, double *loss)
{
    __shared__ double red[8];
    double acc = 0.0;
    const float scale = 2.0f / ((float)n * 64.0f);
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n * 64; q += (int64_t)gridDim.x * blockDim.x) {
        const float r = O[q] - T[q];
        acc += (double)r * r;
        const float d = scale * r;
        dOf[q] = d;
        const __nv_bfloat16 b = __float2bfloat16_rn(d);
        dO[q] = b;
        dOt[(q & 63) * ldt + (q >> 6)] = b;
    }
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) s += red[w];
        atomicAdd(loss, s);
    }
}

// dZ = dH * silu'(Z), stored BF16 row-major and transposed
__global__ void k_silu_grad(const float *dH, const float *Z, int64_t n, int cols, __nv_bfloat16 *dZ,
                            __nv_bfloat16 *dZt, int64_t ldt, float *dZf)
{
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n * cols; q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = q / cols;
        const int c = (int)(q - r * cols);
        const float z = Z[q];
        const float sg = 1.0f / (1.0f + __expf(-z));
        const float d = dH[q] * sg * (1.0f + z * (1.0f - sg));
        dZf[q] = d;
        const __nv_bfloat16 b = __float2bfloat16_rn(d);
        dZ[q] = b;
        dZt[(int64_t)c * ldt + r] = b;
    }
}

// column sums of a [n][cols] FP32 matrix into out[cols] (bias gradients)
__global__ void k_colsum(const float *x, int64_t n, int cols, float *out)
{
    const int c = blockIdx.x;
    float s = 0.0f;
    for (int64_t r = threadIdx.x; r < n; r += blockDim.x) s += x[r * cols + c];
    for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
    __shared__ float red[8];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.0f;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) t += red[w];
        out[c] = t;
    }
}

// FP32 master weights -> BF16 W[out][in] and W^T[in][out]; biases stay FP32
__global__ void k_cast_weights(const float *w, int rows, int cols, __nv_bfloat16 *W, __nv_bfloat16 *WT)
{
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < rows * cols; q += gridDim.x * blockDim.x) {
        const int r = q / cols, c = q - r * cols;
        const __nv_bfloat16 b = __float2bfloat16_rn(w[q]);
        W[q] = b;
        WT[c * rows + r] = b;
    }
}

// Adam (Kingma & Ba) on the flat FP32 parameter vector
__global__ void k_adam(float *w, float *m, float *v, const float *g, int64_t n, float lr, float b1, float b2,
                       float eps, float c1, float c2)
{
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
        const float gq = g[q];
        const float mq = b1 * m[q] + (1.0f - b1) * gq;
        const float vq = b2 * v[q] + (1.0f - b2) * gq * gq;
        m[q] = mq;
        v[q] = vq;
        w[q] -= lr * (mq / c1) / (sqrtf(vq / c2) + eps);
    }
}

// weight gradient of layer l, computed as gW^T for the 64-row layer
__global__ void k_transpose_f32(const float *x, int rows, int cols, float *y)
{
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < rows * cols; q += gridDim.x * blockDim.x) {
        const int r = q / cols, c = q - r * cols;
        y[c * rows + r] = x[q];
    }
}

unsigned blocks(int64_t n) { return (unsigned)std::min<int64_t>(std::max<int64_t>((n + 255) / 256, 1), 152 * 16); }

}  // namespace

// ---------------------------------------------------------------- MLP object
static const int L_IN[4] = {64, 256, 256, 256};
static const int L_OUT[4] = {256, 256, 256, 64};

static size_t param_offset(int l)
{
    size_t off = 0;
    for (int k = 0; k < l; k++) off += (size_t)L_IN[k] * L_OUT[k] + L_OUT[k];
    return off;
}

int mlp_init(Mlp &m, const DevAllocF &alloc)
{
    if (m.ready) return DVM_OK;
    const size_t n = MLP_NPARAM;
    m.w = static_cast<float *>(alloc(n * 4));
    m.m = static_cast<float *>(alloc(n * 4));
    m.v = static_cast<float *>(alloc(n * 4));
    m.g = static_cast<float *>(alloc(n * 4));
    m.loss = static_cast<double *>(alloc(8));
    for (int l = 0; l < 4; l++) {
        m.W[l] = static_cast<__nv_bfloat16 *>(alloc((size_t)L_IN[l] * L_OUT[l] * 2));
        m.WT[l] = static_cast<__nv_bfloat16 *>(alloc((size_t)L_IN[l] * L_OUT[l] * 2));
    }
    if (!m.w || !m.m || !m.v || !m.g || !m.loss) return DVM_ENOMEM;
    for (int l = 0; l < 4; l++)
        if (!m.W[l] || !m.WT[l]) return DVM_ENOMEM;
    cudaMemset(m.m, 0, n * 4);
    cudaMemset(m.v, 0, n * 4);
    m.steps = 0;
    m.ready = true;
    return cudaGetLastError() == cudaSuccess ? DVM_OK : DVM_ECUDA;
}

void mlp_free(Mlp &m, const DevFreeF &dfree)
{
    void *ps[] = {m.w, m.m, m.v, m.g, m.loss};
    for (void *p : ps)
        if (p) dfree(p);
    for (int l = 0; l < 4; l++) {
        if (m.W[l]) dfree(m.W[l]);
        if (m.WT[l]) dfree(m.WT[l]);
    }
    for (int l = 0; l < 4; l++) m.W[l] = m.WT[l] = nullptr;
    m.w = m.m = m.v = m.g = nullptr;
    m.loss = nullptr;
    m.ready = false;
    for (auto &b : m.work) b.reset(dfree);
}

int mlp_cast(Mlp &m, cudaStream_t s)
{
    for (int l = 0; l < 4; l++) {
        k_cast_weights<<<blocks((int64_t)L_IN[l] * L_OUT[l]), 256, 0, s>>>(m.w + param_offset(l), L_OUT[l], L_IN[l],
                                                                            m.W[l], m.WT[l]);
        count_launch();
    }
    return cudaGetLastError() == cudaSuccess ? DVM_OK : DVM_ECUDA;
}

const float *mlp_bias(const Mlp &m, int l) { return m.w + param_offset(l) + (size_t)L_IN[l] * L_OUT[l]; }

// working buffers for a batch of n rows (n padded to a multiple of 64)
int mlp_reserve(Mlp &m, int64_t n, const DevAllocF &alloc, const DevFreeF &dfree)
{
    const int64_t np = (n + 63) / 64 * 64;
    if (np <= m.cap) return DVM_OK;
    for (auto &b : m.work) b.reset(dfree);
    m.cap = 0;
    // X, Xt, Z1-3 (f32), H1-3, H1t-3t, O (f32), T (f32), dO, dOt, dOf, dH (f32), dZ, dZt, dZf
    const size_t sz[] = {(size_t)np * 64 * 2, (size_t)np * 64 * 2,       // X, Xt
                         (size_t)np * 256 * 4 * 3,                           // Z1..Z3
                         (size_t)np * 256 * 2 * 3, (size_t)np * 256 * 2 * 3, // H, Ht
                         (size_t)np * 64 * 4, (size_t)np * 64 * 4,           // O, T
                         (size_t)np * 64 * 2, (size_t)np * 64 * 2, (size_t)np * 64 * 4,  // dO, dOt, dOf
                         (size_t)np * 256 * 4,                               // dH
                         (size_t)np * 256 * 2, (size_t)np * 256 * 2, (size_t)np * 256 * 4};  // dZ, dZt, dZf
    static_assert(sizeof(sz) / sizeof(sz[0]) == MLP_NWORK, "work buffer count");
    for (int i = 0; i < MLP_NWORK; i++) {
        m.work[i].p = alloc(sz[i]);
        m.work[i].bytes = sz[i];
        if (!m.work[i].p) return DVM_ENOMEM;
        cudaMemset(m.work[i].p, 0, sz[i]);
    }
    m.cap = np;
    return DVM_OK;
}

// forward on rows X (BF16 [n][64] in work X); with train = true also keeps
// pre-activations, activations and their transposes for the backward pass
static int forward(Mlp &m, int64_t n, bool train, int *status, cudaStream_t s)
{
    const int64_t np = m.cap;
    auto *X = static_cast<__nv_bfloat16 *>(m.work[W_X].p);
    auto *Z = static_cast<float *>(m.work[W_Z].p);
    auto *H = static_cast<__nv_bfloat16 *>(m.work[W_H].p);
    auto *Ht = static_cast<__nv_bfloat16 *>(m.work[W_HT].p);
    auto *O = static_cast<float *>(m.work[W_O].p);
    const __nv_bfloat16 *in = X;
    int64_t ld_in = 64;
    for (int l = 0; l < 4; l++) {
        GemmArgs g{};
        g.A = in;
        g.lda = ld_in;
        g.B = m.W[l];
        g.ldb = L_IN[l];
        g.M = n;
        g.N = L_OUT[l];
        g.K = L_IN[l];
        g.bias = mlp_bias(m, l);
        g.status = status;
        if (l < 3) {
            g.act = 1;
            g.Cf = train ? Z + (size_t)l * np * 256 : nullptr;
            g.ldc = 256;
            g.H = H + (size_t)l * np * 256;
            g.ldh = 256;
            g.HT = train ? Ht + (size_t)l * np * 256 : nullptr;
            g.ldt = np;
            in = g.H;
            ld_in = 256;
        } else {
            g.act = 0;
            g.Cf = O;
            g.ldc = 64;
        }
        int rc = gemm(g, s);
        if (rc) return rc;
    }
    return DVM_OK;
}

int mlp_forward(Mlp &m, const float *x_dev, int64_t n, float *y_dev, int *status, cudaStream_t s)
{
    if (n > m.cap) return DVM_EINVAL;
    k_to_bf16<<<blocks(n * 64), 256, 0, s>>>(x_dev, static_cast<__nv_bfloat16 *>(m.work[W_X].p), nullptr, n, 64, 0);
    count_launch();
    int rc = forward(m, n, false, status, s);
    if (rc) return rc;
    return cudaMemcpyAsync(y_dev, m.work[W_O].p, (size_t)n * 64 * 4, cudaMemcpyDeviceToDevice, s) == cudaSuccess
               ? DVM_OK
               : DVM_ECUDA;
}

// loss and gradient (m.g) for rows x_dev / targets t_dev (FP32 [n][64])
int mlp_grad(Mlp &m, const float *x_dev, const float *t_dev, int64_t n, int *status, cudaStream_t s)
{
    if (n > m.cap) return DVM_EINVAL;
    const int64_t np = m.cap;
    auto *X = static_cast<__nv_bfloat16 *>(m.work[W_X].p);
    auto *Xt = static_cast<__nv_bfloat16 *>(m.work[W_XT].p);
    auto *Z = static_cast<float *>(m.work[W_Z].p);
    auto *H = static_cast<__nv_bfloat16 *>(m.work[W_H].p);
    auto *Ht = static_cast<__nv_bfloat16 *>(m.work[W_HT].p);
    auto *O = static_cast<float *>(m.work[W_O].p);
    auto *dO = static_cast<__nv_bfloat16 *>(m.work[W_DO].p);
    auto *dOt = static_cast<__nv_bfloat16 *>(m.work[W_DOT].p);
    auto *dOf = static_cast<float *>(m.work[W_DOF].p);
    auto *dH = static_cast<float *>(m.work[W_DH].p);
    auto *dZ = static_cast<__nv_bfloat16 *>(m.work[W_DZ].p);
    auto *dZt = static_cast<__nv_bfloat16 *>(m.work[W_DZT].p);
    auto *dZf = static_cast<float *>(m.work[W_DZF].p);
    // the weight gradients sum over K = n rounded up to 64: the transposed
    // operands must hold zeros past row n
    const int64_t nk = (n + 63) / 64 * 64;
    cudaMemsetAsync(Xt, 0, m.work[W_XT].bytes, s);
    cudaMemsetAsync(Ht, 0, m.work[W_HT].bytes, s);
    cudaMemsetAsync(dOt, 0, m.work[W_DOT].bytes, s);
    cudaMemsetAsync(dZt, 0, m.work[W_DZT].bytes, s);
    k_to_bf16<<<blocks(n * 64), 256, 0, s>>>(x_dev, X, Xt, n, 64, np);
    count_launch();
    int rc = forward(m, n, true, status, s);
    if (rc) return rc;
    cudaMemsetAsync(m.loss, 0, 8, s);
    k_out_grad<<<blocks(n * 64), 256, 0, s>>>(O, t_dev, n, dO, dOt, np, dOf, m.loss);
    count_launch();
    // layer 4: gW4^T[in][out] = H3^T . dO ; gb4 = colsum dO ; dH3 = dO . W4
    {
        GemmArgs g{};
        g.A = Ht + (size_t)2 * np * 256; g.lda = np;
        g.B = dOt; g.ldb = np;
        g.M = 256; g.N = 64; g.K = nk;
        g.Cf = dH; g.ldc = 64;  // scratch for gW4^T
        g.status = status;
        if ((rc = gemm(g, s))) return rc;
        k_transpose_f32<<<blocks(256 * 64), 256, 0, s>>>(dH, 256, 64, m.g + param_offset(3));
        count_launch();
        k_colsum<<<64, 256, 0, s>>>(dOf, n, 64, m.g + param_offset(3) + 256 * 64);
        count_launch();
        GemmArgs h{};
        h.A = dO; h.lda = 64;
        h.B = m.WT[3]; h.ldb = 64;
        h.M = n; h.N = 256; h.K = 64;
        h.Cf = dH; h.ldc = 256;
        h.status = status;
        if ((rc = gemm(h, s))) return rc;
    }
    for (int l = 2; l >= 0; l--) {
        // dZ_l = dH_l * silu'(Z_l)
        k_silu_grad<<<blocks(n * 256), 256, 0, s>>>(dH, Z + (size_t)l * np * 256, n, 256, dZ, dZt, np, dZf);
        count_launch();
        // gW_l[out][in] = dZ^T . (input of layer l)
        GemmArgs g{};
        g.A = dZt; g.lda = np;
        g.B = l > 0 ? Ht + (size_t)(l - 1) * np * 256 : Xt; g.ldb = np;
        g.M = 256; g.N = L_IN[l]; g.K = nk;
        g.Cf = m.g + param_offset(l); g.ldc = L_IN[l];
        g.status = status;
        if ((rc = gemm(g, s))) return rc;
        k_colsum<<<256, 256, 0, s>>>(dZf, n, 256, m.g + param_offset(l) + (size_t)L_IN[l] * 256);
        count_launch();
        if (l > 0) {
            // dH_{l-1} = dZ_l . W_l
            GemmArgs h{};
            h.A = dZ; h.lda = 256;
            h.B = m.WT[l]; h.ldb = 256;
            h.M = n; h.N = 256; h.K = 256;
            h.Cf = dH; h.ldc = 256;
            h.status = status;
            if ((rc = gemm(h, s))) return rc;
        }
    }
    (void)H;
    return cudaGetLastError() == cudaSuccess ? DVM_OK : DVM_ECUDA;
}

int mlp_adam(Mlp &m, double lr, cudaStream_t s)
{
    m.steps++;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.0f - powf(b1, (float)m.steps), c2 = 1.0f - powf(b2, (float)m.steps);
    k_adam<<<blocks(MLP_NPARAM), 256, 0, s>>>(m.w, m.m, m.v, m.g, MLP_NPARAM, (float)lr, b1, b2, 1e-8f, c1, c2);
    count_launch();
    return mlp_cast(m, s);
}

}  // namespace dvm
