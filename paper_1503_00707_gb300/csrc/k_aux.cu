// Auxiliary kernels outside the timed step: Maxwellian initialisation,
// moments of the stored f, and precision conversions for host transfers.
#include <algorithm>
#include <cmath>

#include "../../include/dvm.h"
#include "common.cuh"
#include "kernels.hpp"

namespace dvm {

void count_launch();

namespace {

template <typename TS> __device__ inline TS from_double(double v);
template <> __device__ inline double from_double<double>(double v) { return v; }
template <> __device__ inline float from_double<float>(double v) { return (float)v; }
template <> __device__ inline __nv_bfloat16 from_double<__nv_bfloat16>(double v) { return __double2bfloat16(v); }

template <typename TS> __device__ inline double to_double(TS v);
template <> __device__ inline double to_double<double>(double v) { return v; }
template <> __device__ inline double to_double<float>(float v) { return (double)v; }
template <> __device__ inline double to_double<__nv_bfloat16>(__nv_bfloat16 v) { return (double)__bfloat162float(v); }

// M(rho, u, T; xi) = rho (2 pi T)^(-3/2) exp(-|xi - u|^2 / (2T)), FP64
template <typename TS>
__global__ void k_init(TS *f, int64_t ncells, int nv, int nmix, const double *w, const double *rho,
                       const double *u, const double *T, const double *xi)
{
    const int64_t total = ncells * (int64_t)nv;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = q / nv;
        const int v = (int)(q - c * nv);
        double s = 0.0;
        for (int m = 0; m < nmix; m++) {
            const int64_t k = c * nmix + m;
            double d2 = 0.0;
            for (int d = 0; d < 3; d++) {
                const double t = xi[3 * v + d] - u[3 * k + d];
                d2 += t * t;
            }
            const double tp = 2.0 * 3.14159265358979323846 * T[k];
            s += w[k] * rho[k] / (tp * sqrt(tp)) * exp(-d2 / (2.0 * T[k]));
        }
        f[q] = from_double<TS>(s);
    }
}

template <typename TS>
__global__ void k_moments(const TS *f, int64_t ncells, int nv, const double *xi, double dV, double *out)
{
    __shared__ double red[5][32];
    const int64_t c = blockIdx.x;
    double s[5] = {0, 0, 0, 0, 0};
    for (int v = threadIdx.x; v < nv; v += blockDim.x) {
        const double fv = to_double<TS>(f[c * nv + v]);
        const double x = xi[3 * v], y = xi[3 * v + 1], z = xi[3 * v + 2];
        s[0] += fv;
        s[1] += x * fv;
        s[2] += y * fv;
        s[3] += z * fv;
        s[4] += (x * x + y * y + z * z) * fv;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int k = 0; k < 5; k++) {
        s[k] = warp_allsum(s[k]);
        if (lane == 0) red[k][warp] = s[k];
    }
    __syncthreads();
    if (warp == 0) {
        const int nw = blockDim.x >> 5;
        for (int k = 0; k < 5; k++) s[k] = warp_allsum(lane < nw ? red[k][lane] : 0.0);
        if (lane == 0) {
            const double s0 = s[0];
            const double ux = s[1] / s0, uy = s[2] / s0, uz = s[3] / s0;
            double *o = out + c * 5;
            o[0] = s0 * dV;
            o[1] = ux; o[2] = uy; o[3] = uz;
            o[4] = (s[4] / s0 - (ux * ux + uy * uy + uz * uz)) / 3.0;
        }
    }
}

template <typename TS>
__global__ void k_to_f64(const TS *src, double *dst, int64_t n)
{
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x)
        dst[q] = to_double<TS>(src[q]);
}

template <typename TS>
__global__ void k_from_f64(const double *src, TS *dst, int64_t n)
{
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x)
        dst[q] = from_double<TS>(src[q]);
}

inline unsigned blocks_for(int64_t n, int threads)
{
    int64_t b = (n + threads - 1) / threads;
    if (b > 152 * 64) b = 152 * 64;
    if (b < 1) b = 1;
    return (unsigned)b;
}

int last_status()
{
    count_launch();
    return cudaGetLastError() == cudaSuccess ? DVM_OK : DVM_ECUDA;
}

// Row copies between buffers: entry r of rows is {destination buffer, row,
// source buffer, row}; rows are row_bytes long (a multiple of 16).
__global__ void k_copy_rows(void *const *bufs, const int64_t *rows, int64_t n, int64_t row_bytes)
{
    const int64_t n16 = row_bytes / 16;
    for (int64_t r = blockIdx.x; r < n; r += gridDim.x) {
        const int64_t *e = rows + 4 * r;
        const uint4 *src = reinterpret_cast<const uint4 *>(static_cast<const char *>(bufs[e[2]]) + e[3] * row_bytes);
        uint4 *dst = reinterpret_cast<uint4 *>(static_cast<char *>(bufs[e[0]]) + e[1] * row_bytes);
        for (int64_t i = threadIdx.x; i < n16; i += blockDim.x) dst[i] = src[i];
    }
}

// Halo pack and unpack: dst row r = src row idx[r] (gather), or dst row
// idx[r] = src row r (scatter); rows are row_bytes long (a multiple of 16).
template <bool GATHER>
__global__ void k_rows_indexed(char *dst, const char *src, const int64_t *idx, int64_t n, int64_t row_bytes)
{
    const int64_t n16 = row_bytes / 16;
    for (int64_t r = blockIdx.x; r < n; r += gridDim.x) {
        const int64_t rd = GATHER ? r : idx[r], rs = GATHER ? idx[r] : r;
        const uint4 *a = reinterpret_cast<const uint4 *>(src + rs * row_bytes);
        uint4 *b = reinterpret_cast<uint4 *>(dst + rd * row_bytes);
        for (int64_t i = threadIdx.x; i < n16; i += blockDim.x) b[i] = a[i];
    }
}

// Row means: destination row r of dst is the mean of source rows
// idx[start[r] .. start[r+1]) of src (nv values each, storage precision;
// the sum in FP64 for FP64 storage, FP32 otherwise).
template <typename T, typename A>
__global__ void k_mean_rows(T *dst, const T *src, const int64_t *start, const int64_t *idx, int64_t nrows, int nv)
{
    for (int64_t r = blockIdx.x; r < nrows; r += gridDim.x) {
        const int64_t b = start[r], e = start[r + 1];
        const A inv = A(1) / A(e - b);
        for (int v = threadIdx.x; v < nv; v += blockDim.x) {
            A acc = A(0);
            for (int64_t k = b; k < e; k++) acc += (A)src[idx[k] * nv + v];
            dst[r * nv + v] = (T)(acc * inv);
        }
    }
}

}  // namespace

int launch_mean_rows(int prec, void *dst, const void *src, const int64_t *start, const int64_t *idx, int64_t nrows,
                     int nv, cudaStream_t s)
{
    if (nrows <= 0) return DVM_OK;
    const unsigned grid = (unsigned)std::min<int64_t>(nrows, 1 << 16);
    switch (prec) {
    case DVM_F64: k_mean_rows<double, double><<<grid, 256, 0, s>>>((double *)dst, (const double *)src, start, idx, nrows, nv); break;
    case DVM_F32: k_mean_rows<float, float><<<grid, 256, 0, s>>>((float *)dst, (const float *)src, start, idx, nrows, nv); break;
    case DVM_BF16:
        k_mean_rows<__nv_bfloat16, float><<<grid, 256, 0, s>>>((__nv_bfloat16 *)dst, (const __nv_bfloat16 *)src, start,
                                                               idx, nrows, nv);
        break;
    default: return DVM_EINVAL;
    }
    count_launch();
    return cudaGetLastError() == cudaSuccess ? DVM_OK : DVM_ECUDA;
}

int launch_copy_rows(void *const *bufs, const int64_t *rows, int64_t n, int64_t row_bytes, cudaStream_t s)
{
    if (n <= 0) return DVM_OK;
    if (row_bytes % 16 != 0) return DVM_EINVAL;
    const unsigned grid = (unsigned)std::min<int64_t>(n, 1 << 16);
    k_copy_rows<<<grid, 256, 0, s>>>(bufs, rows, n, row_bytes);
    count_launch();
    return cudaGetLastError() == cudaSuccess ? DVM_OK : DVM_ECUDA;
}

int launch_rows_indexed(bool gather, void *dst, const void *src, const int64_t *idx, int64_t n, int64_t row_bytes,
                        cudaStream_t s)
{
    if (n <= 0) return DVM_OK;
    if (row_bytes % 16 != 0) return DVM_EINVAL;
    const unsigned grid = (unsigned)std::min<int64_t>(n, 1 << 16);
    if (gather)
        k_rows_indexed<true><<<grid, 256, 0, s>>>(static_cast<char *>(dst), static_cast<const char *>(src), idx, n,
                                                  row_bytes);
    else
        k_rows_indexed<false><<<grid, 256, 0, s>>>(static_cast<char *>(dst), static_cast<const char *>(src), idx, n,
                                                   row_bytes);
    count_launch();
    return cudaGetLastError() == cudaSuccess ? DVM_OK : DVM_ECUDA;
}

int launch_init_maxwellian(int prec, void *f, int64_t ncells, int nv, int nmix, const double *w,
                           const double *rho, const double *u, const double *T, const double *xi,
                           cudaStream_t s)
{
    const int64_t n = ncells * (int64_t)nv;
    const unsigned b = blocks_for(n, 256);
    switch (prec) {
    case DVM_F64: k_init<double><<<b, 256, 0, s>>>((double *)f, ncells, nv, nmix, w, rho, u, T, xi); break;
    case DVM_F32: k_init<float><<<b, 256, 0, s>>>((float *)f, ncells, nv, nmix, w, rho, u, T, xi); break;
    case DVM_BF16: k_init<__nv_bfloat16><<<b, 256, 0, s>>>((__nv_bfloat16 *)f, ncells, nv, nmix, w, rho, u, T, xi); break;
    default: return DVM_EINVAL;
    }
    return last_status();
}

int launch_moments(int prec, const void *f, int64_t ncells, int nv, const double *xi, double dV,
                   double *out, cudaStream_t s)
{
    if (ncells <= 0) return DVM_OK;
    const dim3 grid((unsigned)ncells);
    switch (prec) {
    case DVM_F64: k_moments<double><<<grid, 256, 0, s>>>((const double *)f, ncells, nv, xi, dV, out); break;
    case DVM_F32: k_moments<float><<<grid, 256, 0, s>>>((const float *)f, ncells, nv, xi, dV, out); break;
    case DVM_BF16: k_moments<__nv_bfloat16><<<grid, 256, 0, s>>>((const __nv_bfloat16 *)f, ncells, nv, xi, dV, out); break;
    default: return DVM_EINVAL;
    }
    return last_status();
}

int launch_to_f64(int prec, const void *src, double *dst, int64_t n, cudaStream_t s)
{
    const unsigned b = blocks_for(n, 256);
    switch (prec) {
    case DVM_F64: k_to_f64<double><<<b, 256, 0, s>>>((const double *)src, dst, n); break;
    case DVM_F32: k_to_f64<float><<<b, 256, 0, s>>>((const float *)src, dst, n); break;
    case DVM_BF16: k_to_f64<__nv_bfloat16><<<b, 256, 0, s>>>((const __nv_bfloat16 *)src, dst, n); break;
    default: return DVM_EINVAL;
    }
    return last_status();
}

int launch_from_f64(int prec, const double *src, void *dst, int64_t n, cudaStream_t s)
{
    const unsigned b = blocks_for(n, 256);
    switch (prec) {
    case DVM_F64: k_from_f64<double><<<b, 256, 0, s>>>(src, (double *)dst, n); break;
    case DVM_F32: k_from_f64<float><<<b, 256, 0, s>>>(src, (float *)dst, n); break;
    case DVM_BF16: k_from_f64<__nv_bfloat16><<<b, 256, 0, s>>>(src, (__nv_bfloat16 *)dst, n); break;
    default: return DVM_EINVAL;
    }
    return last_status();
}

}  // namespace dvm
