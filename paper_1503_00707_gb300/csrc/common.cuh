// Device helpers shared by the step kernels: vectorised storage access,
// double-float accumulation and warp reductions.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cstdint>

namespace dvm {

// ---------------------------------------------------------------- storage
// One "quad" is the unit a thread loads: 16 bytes of FP32 (4 values) or FP64
// (2 values), or 8 bytes of BF16 (4 values).  Loads go through the read-only
// path; stores stream (evict-first) so that L2 keeps the upwind neighbours.
template <typename TS> struct Store;

template <> struct Store<double> {
    static constexpr int VEC = 2;
    using TC = double;
    __device__ static inline void load(const double *p, double v[2])
    {
        const double2 t = __ldg(reinterpret_cast<const double2 *>(p));
        v[0] = t.x; v[1] = t.y;
    }
    __device__ static inline void store(double *p, const double v[2])
    {
        __stcs(reinterpret_cast<double2 *>(p), make_double2(v[0], v[1]));
    }
    __device__ static inline void load_shared(const double *p, double v[2])
    {
        const double2 t = *reinterpret_cast<const double2 *>(p);
        v[0] = t.x; v[1] = t.y;
    }
};

template <> struct Store<float> {
    static constexpr int VEC = 4;
    using TC = float;
    __device__ static inline void load(const float *p, float v[4])
    {
        const float4 t = __ldg(reinterpret_cast<const float4 *>(p));
        v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
    }
    __device__ static inline void store(float *p, const float v[4])
    {
        __stcs(reinterpret_cast<float4 *>(p), make_float4(v[0], v[1], v[2], v[3]));
    }
    __device__ static inline void load_shared(const float *p, float v[4])
    {
        const float4 t = *reinterpret_cast<const float4 *>(p);
        v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
    }
};

template <> struct Store<__nv_bfloat16> {
    static constexpr int VEC = 4;
    using TC = float;
    __device__ static inline void load(const __nv_bfloat16 *p, float v[4])
    {
        const uint2 raw = __ldg(reinterpret_cast<const uint2 *>(p));
        __nv_bfloat162 a = *reinterpret_cast<const __nv_bfloat162 *>(&raw.x);
        __nv_bfloat162 b = *reinterpret_cast<const __nv_bfloat162 *>(&raw.y);
        const float2 fa = __bfloat1622float2(a), fb = __bfloat1622float2(b);
        v[0] = fa.x; v[1] = fa.y; v[2] = fb.x; v[3] = fb.y;
    }
    __device__ static inline void store(__nv_bfloat16 *p, const float v[4])
    {
        __nv_bfloat162 a = __floats2bfloat162_rn(v[0], v[1]);
        __nv_bfloat162 b = __floats2bfloat162_rn(v[2], v[3]);
        uint2 raw;
        raw.x = *reinterpret_cast<const uint32_t *>(&a);
        raw.y = *reinterpret_cast<const uint32_t *>(&b);
        __stcs(reinterpret_cast<uint2 *>(p), raw);
    }
    __device__ static inline void load_shared(const __nv_bfloat16 *p, float v[4])
    {
        const uint2 raw = *reinterpret_cast<const uint2 *>(p);
        __nv_bfloat162 a = *reinterpret_cast<const __nv_bfloat162 *>(&raw.x);
        __nv_bfloat162 b = *reinterpret_cast<const __nv_bfloat162 *>(&raw.y);
        const float2 fa = __bfloat1622float2(a), fb = __bfloat1622float2(b);
        v[0] = fa.x; v[1] = fa.y; v[2] = fb.x; v[3] = fb.y;
    }
};

// ---------------------------------------------------------------- double-float
// An unevaluated sum hi + lo of two FP32 numbers (Dekker/Knuth).  Addition
// uses the branch-free TwoSum; a product of two floats is split exactly with
// one FMA.  About 48 significant bits, enough for FP64-class moment sums
// without FP64 arithmetic per element.
struct FF {
    float hi, lo;
};

__device__ inline FF ff_make(float a) { return {a, 0.0f}; }

__device__ inline FF ff_add(FF a, FF b)
{
    const float s = a.hi + b.hi;
    const float bb = s - a.hi;
    float e = (a.hi - (s - bb)) + (b.hi - bb);
    e += a.lo;
    e += b.lo;
    const float h = s + e;
    return {h, e - (h - s)};
}

__device__ inline FF ff_prod(float a, float b)
{
    const float p = a * b;
    return {p, fmaf(a, b, -p)};
}

__device__ inline double ff_to_double(FF a) { return (double)a.hi + (double)a.lo; }

template <typename TC> struct Red;

template <> struct Red<float> {
    using T = FF;
    __device__ static inline T zero() { return {0.0f, 0.0f}; }
    __device__ static inline T from(float a) { return ff_make(a); }
    __device__ static inline T mul(float a, float b) { return ff_prod(a, b); }
    __device__ static inline T add(T a, T b) { return ff_add(a, b); }
    __device__ static inline T shfl_down(T a, int off)
    {
        return {__shfl_down_sync(0xffffffffu, a.hi, off), __shfl_down_sync(0xffffffffu, a.lo, off)};
    }
    __device__ static inline double to_double(T a) { return ff_to_double(a); }
};

template <> struct Red<double> {
    using T = double;
    __device__ static inline T zero() { return 0.0; }
    __device__ static inline T from(double a) { return a; }
    __device__ static inline T mul(double a, double b) { return a * b; }
    __device__ static inline T add(T a, T b) { return a + b; }
    __device__ static inline T shfl_down(T a, int off) { return __shfl_down_sync(0xffffffffu, a, off); }
    __device__ static inline double to_double(T a) { return a; }
};

__device__ inline double warp_allsum(double v)
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

// Solve A x = b for a symmetric positive definite 5x5 A (the moment systems
// sum_i phi_r phi_s w_i with positive weights w_i) by an LDL^T factorisation.
// Every index is a compile-time constant, so the whole solve stays in
// registers (no local memory).  Returns false if a pivot is not positive or
// a result is not finite.
template <typename T>
__device__ inline bool solve5(const T A[25], const T b[5], T x[5])
{
    T L[5][5], D[5];
#pragma unroll
    for (int j = 0; j < 5; j++) {
        T d = A[j * 5 + j];
#pragma unroll
        for (int k = 0; k < j; k++) d -= L[j][k] * L[j][k] * D[k];
        if (!(d > (T)0) || !isfinite(d)) return false;
        D[j] = d;
        const T inv = (T)1 / d;
#pragma unroll
        for (int i = j + 1; i < 5; i++) {
            T s = A[i * 5 + j];
#pragma unroll
            for (int k = 0; k < j; k++) s -= L[i][k] * L[j][k] * D[k];
            L[i][j] = s * inv;
        }
    }
    T y[5];
#pragma unroll
    for (int i = 0; i < 5; i++) {
        T s = b[i];
#pragma unroll
        for (int k = 0; k < i; k++) s -= L[i][k] * y[k];
        y[i] = s;
    }
#pragma unroll
    for (int i = 4; i >= 0; i--) {
        T s = y[i] / D[i];
#pragma unroll
        for (int k = i + 1; k < 5; k++) s -= L[k][i] * x[k];
        x[i] = s;
        if (!isfinite(s)) return false;
    }
    return true;
}

// The same LDL^T solve with one reciprocal per pivot in place of the ten
// divisions (FP32: correctly rounded reciprocal, so each quotient carries one
// more rounding than a division would).
__device__ inline float rcp_rn(float d) { return __frcp_rn(d); }
__device__ inline double rcp_rn(double d) { return 1.0 / d; }

template <typename T>
__device__ inline bool solve5_rcp(const T A[25], const T b[5], T x[5])
{
    T L[5][5], D[5], Di[5];
#pragma unroll
    for (int j = 0; j < 5; j++) {
        T d = A[j * 5 + j];
#pragma unroll
        for (int k = 0; k < j; k++) d -= L[j][k] * L[j][k] * D[k];
        if (!(d > (T)0) || !isfinite(d)) return false;
        D[j] = d;
        Di[j] = rcp_rn(d);
#pragma unroll
        for (int i = j + 1; i < 5; i++) {
            T s = A[i * 5 + j];
#pragma unroll
            for (int k = 0; k < j; k++) s -= L[i][k] * L[j][k] * D[k];
            L[i][j] = s * Di[j];
        }
    }
    T y[5];
#pragma unroll
    for (int i = 0; i < 5; i++) {
        T s = b[i];
#pragma unroll
        for (int k = 0; k < i; k++) s -= L[i][k] * y[k];
        y[i] = s;
    }
#pragma unroll
    for (int i = 4; i >= 0; i--) {
        T s = y[i] * Di[i];
#pragma unroll
        for (int k = i + 1; k < 5; k++) s -= L[k][i] * x[k];
        x[i] = s;
        if (!isfinite(s)) return false;
    }
    return true;
}

// LDL^T factor of a symmetric positive definite 5x5 matrix (unit lower L,
// reciprocal pivots Di); false if a pivot is not positive and finite.
template <typename T> __device__ inline bool ldl5(const T A[25], T L[5][5], T Di[5])
{
    T D[5];
#pragma unroll
    for (int j = 0; j < 5; j++) {
        T d = A[j * 5 + j];
#pragma unroll
        for (int k = 0; k < j; k++) d -= L[j][k] * L[j][k] * D[k];
        if (!(d > (T)0) || !isfinite(d)) return false;
        D[j] = d;
        Di[j] = rcp_rn(d);
#pragma unroll
        for (int i = j + 1; i < 5; i++) {
            T s = A[i * 5 + j];
#pragma unroll
            for (int k = 0; k < j; k++) s -= L[i][k] * L[j][k] * D[k];
            L[i][j] = s * Di[j];
        }
    }
    return true;
}

template <typename T> __device__ inline void ldl5_solve(const T L[5][5], const T Di[5], const T b[5], T x[5])
{
    T y[5];
#pragma unroll
    for (int i = 0; i < 5; i++) {
        T s = b[i];
#pragma unroll
        for (int k = 0; k < i; k++) s -= L[i][k] * y[k];
        y[i] = s;
    }
#pragma unroll
    for (int i = 4; i >= 0; i--) {
        T s = y[i] * Di[i];
#pragma unroll
        for (int k = i + 1; k < 5; k++) s -= L[k][i] * x[k];
        x[i] = s;
    }
}

}  // namespace dvm

namespace dvm {

// ---------------------------------------------------------------- double-float numbers
// Arithmetic on unevaluated pairs hi + lo of FP32 values (Dekker 1971, with
// FMA-based exact products): about 48 significant bits on the FP32 pipe,
// used for the per-cell reductions and scalars where FP64 (1/64 of the FP32
// rate on this GPU) would serialise the cell.
struct ffn {
    float hi, lo;
};

__device__ inline ffn ffn_norm(float s, float e)
{
    const float h = s + e;
    return {h, e - (h - s)};
}

__device__ inline ffn operator+(ffn a, ffn b)
{
    const FF r = ff_add({a.hi, a.lo}, {b.hi, b.lo});
    return {r.hi, r.lo};
}
__device__ inline ffn operator-(ffn a) { return {-a.hi, -a.lo}; }
__device__ inline ffn operator-(ffn a, ffn b) { return a + (-b); }
__device__ inline ffn operator*(ffn a, ffn b)
{
    const float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    return ffn_norm(p, e);
}
__device__ inline ffn operator*(ffn a, float b)
{
    const float p = a.hi * b;
    float e = fmaf(a.hi, b, -p);
    e = fmaf(a.lo, b, e);
    return ffn_norm(p, e);
}
__device__ inline ffn operator/(ffn a, ffn b)
{
    const float q1 = a.hi / b.hi;
    const ffn r1 = a - b * q1;
    const float q2 = r1.hi / b.hi;
    const ffn r2 = r1 - b * q2;
    const float q3 = r2.hi / b.hi;
    return ffn_norm(q1, q2) + ffn{q3, 0.0f};
}

template <typename TC> struct Num;

template <> struct Num<float> {
    using X = ffn;
    __device__ static inline X make(float v) { return {v, 0.0f}; }
    __device__ static inline X from_double_host_split(float hi, float lo) { return {hi, lo}; }
    __device__ static inline float tc(X v) { return v.hi + v.lo; }
    __device__ static inline float f(X v) { return v.hi + v.lo; }
    __device__ static inline bool finite_pos(X v) { return isfinite(v.hi) && v.hi > 0.0f; }
    __device__ static inline X shfl_xor(X v, int m)
    {
        return {__shfl_xor_sync(0xffffffffu, v.hi, m), __shfl_xor_sync(0xffffffffu, v.lo, m)};
    }
    __device__ static inline X shfl(X v, int src)
    {
        return {__shfl_sync(0xffffffffu, v.hi, src), __shfl_sync(0xffffffffu, v.lo, src)};
    }
    // 1/v: FP32 reciprocal refined by one Newton step in double-float
    __device__ static inline X recip(X v)
    {
        const float y = __frcp_rn(v.hi);
        const ffn e = ffn{1.0f, 0.0f} - v * y;
        return ffn_norm(y, y * e.hi);
    }
    // 1/sqrt(v): FP32 estimate refined by one Newton step in double-float
    __device__ static inline X rsqrt(X v)
    {
        const float y = rsqrtf(v.hi);
        const ffn e = ffn{1.0f, 0.0f} - v * y * y;
        return ffn_norm(y, 0.5f * y * e.hi);
    }
};

template <> struct Num<double> {
    using X = double;
    __device__ static inline X make(double v) { return v; }
    __device__ static inline X from_double_host_split(float hi, float lo) { return (double)hi + (double)lo; }
    __device__ static inline double tc(X v) { return v; }
    __device__ static inline float f(X v) { return (float)v; }
    __device__ static inline bool finite_pos(X v) { return isfinite(v) && v > 0.0; }
    __device__ static inline X shfl_xor(X v, int m) { return __shfl_xor_sync(0xffffffffu, v, m); }
    __device__ static inline X shfl(X v, int src) { return __shfl_sync(0xffffffffu, v, src); }
    __device__ static inline X recip(X v) { return 1.0 / v; }
    __device__ static inline X rsqrt(X v) { return 1.0 / sqrt(v); }
};

}  // namespace dvm
