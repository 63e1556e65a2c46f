// Fused DVM step: upwind transport (Eq. 2) -> moments of f* -> conservative
// BGK relaxation, with f* held on chip between the phases.
//
// Layout (paper Sec. 3.1 steps 1-3): f[cell][group][position], 8 sign groups
// per cell.  A compute thread owns the same "quad" of positions (4 FP32/BF16
// or 2 FP64 values along z) in all 8 groups, and the stencil of Eq. 2 is
// warp-uniform, since it depends on the group only through the signs of the
// velocity components (Sec. 3.1).
//
// Persistent CTAs take the Morton-ordered cells from a global counter, so
// the cells in flight on the whole GPU form one contiguous Morton window and
// upwind neighbours are served from L2 (a fixed assignment, cells b, b + G,
// ... for CTA b, lets the CTAs drift apart and measured 1.6x slower).
// A CTA's iterations alternate between two parities, one per solver warp,
// and each parity's cells are taken in program order: once a slot of a
// parity comes back empty, every later slot of that parity is empty.  The
// other parity may still hold a cell, so every warp tracks the two parities
// separately (see the loops below); no barrier is used for an empty slot.
//
// Compute warps, iteration j:
//   phase 1  f*_i = (1 - dt invh sum_d |xi_d,i|) f_i + sum_d dt |xi_d,i| sum_k
//            w_k src_k,i for cell j on packed FP32 pairs, into registers.  The
//            inputs of each sign group (the cell's own values and the first
//            upwind source of each axis, Sec. 3.1 step 4) come from a 4-stage
//            shared-memory ring that every thread fills for its own
//            positions with cp.async, four groups ahead; further sources
//            behind coarse-fine faces come from L2.  Per-thread FP32 partials
//            of the seven sums sum f, sum j_d f, sum j_d^2 f (xi_d = (h_d/2)
//            j_d, j_d odd) are reduced per warp.
//   phase 3  the collision of cell j - 2, whose f* waits in one of two
//            shared tiles, straight to HBM; then f* of cell j takes its tile.
// Two solver warps take the even and the odd cells: phase 2 of cell j
// (double-float sum of the warp partials -> rho, u, T; the discrete
// Maxwellian's moments in the centred basis phi = (1, c, |c|^2 - 3),
// c = (xi - u)/sqrt(T), as products of 1D sums; the five coefficients d of
// M~ = M (1 + d.phi) (the correction form of Eq. 6) that make M~ carry the
// moments of f*; per-axis tables g = exp(-c^2/2), P = d_axis c + d4 c^2)
// runs while the compute warps transport cells j + 1 and j + 2.  Solver warps
// also fetch the cells' stencils, four iterations ahead.
//
// Phase 3: f^{n+1} = (1 - nu dt) f* + nu dt M~ with M~ = rho (2 pi T)^(-3/2)
//   gx gy gz (1 + d0 - 3 d4 + Px + Py + Pz), nu = sqrt(8/pi) rho sqrt(T)/Kn.
//
// Compute and solver warps meet on named barriers, "partials of cell j
// ready" and "coefficients of cell j ready", each with four instances used
// in turn, which makes every reuse of a barrier ordered after its previous
// completion.  Both sides use the barriers of slot j only if slot j holds a
// cell, which both read from the same slot record; no warp waits on a flag.
#include <algorithm>
#include <atomic>
#include <cmath>

#include "../../include/dvm.h"
#include "async.cuh"
#include "common.cuh"
#include "kernels.hpp"
#include "mesh.hpp"

namespace dvm {

static std::atomic<int64_t> g_launches{0};
int64_t launches_issued() { return g_launches.load(); }
void count_launch() { g_launches.fetch_add(1); }

namespace {

constexpr int MAXCW = 14;     // compute warps per CTA (at most)
constexpr int NAX = 32;       // velocity nodes per axis supported
constexpr int MAXT = MAXCW * 32 + 64;
constexpr int NST = 4;        // ring stages (one sign group of one cell each)
constexpr int NSS = 4;        // solver result slots (cell j in slot j % NSS)
constexpr int NSL = 8;        // ring of per-cell stencil slots (dispatched four iterations ahead)

template <typename TC> __device__ inline TC tc_exp(TC x);
template <> __device__ inline float tc_exp<float>(float x) { return expf(x); }
template <> __device__ inline double tc_exp<double>(double x) { return exp(x); }

// ---------------------------------------------------------------- quads
// The values one thread handles per group: four FP32 values as two packed
// pairs (FFMA2/FADD2/FMUL2, two lanes per instruction), or two FP64 values.
template <typename TC> struct QV;
template <> struct QV<float> { float2 a, b; };
template <> struct QV<double> { double a, b; };

__device__ inline QV<float> q_splat(float s) { return {make_float2(s, s), make_float2(s, s)}; }
__device__ inline QV<double> q_splat(double s) { return {s, s}; }
__device__ inline QV<float> q_fma(QV<float> x, QV<float> y, QV<float> z)
{
    return {__ffma2_rn(x.a, y.a, z.a), __ffma2_rn(x.b, y.b, z.b)};
}
__device__ inline QV<double> q_fma(QV<double> x, QV<double> y, QV<double> z)
{
    return {fma(x.a, y.a, z.a), fma(x.b, y.b, z.b)};
}
__device__ inline QV<float> q_mul(QV<float> x, QV<float> y) { return {__fmul2_rn(x.a, y.a), __fmul2_rn(x.b, y.b)}; }
__device__ inline QV<double> q_mul(QV<double> x, QV<double> y) { return {x.a * y.a, x.b * y.b}; }
__device__ inline QV<float> q_add(QV<float> x, QV<float> y) { return {__fadd2_rn(x.a, y.a), __fadd2_rn(x.b, y.b)}; }
__device__ inline QV<double> q_add(QV<double> x, QV<double> y) { return {x.a + y.a, x.b + y.b}; }
__device__ inline QV<float> q_neg(QV<float> x) { return {make_float2(-x.a.x, -x.a.y), make_float2(-x.b.x, -x.b.y)}; }
__device__ inline QV<double> q_neg(QV<double> x) { return {-x.a, -x.b}; }
__device__ inline float q_sum(QV<float> x)
{
    const float2 t = __fadd2_rn(x.a, x.b);
    return t.x + t.y;
}
__device__ inline double q_sum(QV<double> x) { return x.a + x.b; }
__device__ inline QV<float> q_make(const float v[4]) { return {make_float2(v[0], v[1]), make_float2(v[2], v[3])}; }
__device__ inline QV<double> q_make(const double v[2]) { return {v[0], v[1]}; }

// storage <-> quads
template <typename TS> struct QIO;
template <> struct QIO<float> {
    __device__ static inline QV<float> ldg(const float *p)
    {
        const float4 t = __ldg(reinterpret_cast<const float4 *>(p));
        return {make_float2(t.x, t.y), make_float2(t.z, t.w)};
    }
    __device__ static inline QV<float> lds(const float *p)
    {
        const float4 t = *reinterpret_cast<const float4 *>(p);
        return {make_float2(t.x, t.y), make_float2(t.z, t.w)};
    }
    __device__ static inline void stg(float *p, QV<float> q)
    {
        __stcs(reinterpret_cast<float4 *>(p), make_float4(q.a.x, q.a.y, q.b.x, q.b.y));
    }
    __device__ static inline void sts(float *p, QV<float> q)
    {
        *reinterpret_cast<float4 *>(p) = make_float4(q.a.x, q.a.y, q.b.x, q.b.y);
    }
};
template <> struct QIO<double> {
    __device__ static inline QV<double> ldg(const double *p)
    {
        const double2 t = __ldg(reinterpret_cast<const double2 *>(p));
        return {t.x, t.y};
    }
    __device__ static inline QV<double> lds(const double *p)
    {
        const double2 t = *reinterpret_cast<const double2 *>(p);
        return {t.x, t.y};
    }
    __device__ static inline void stg(double *p, QV<double> q)
    {
        __stcs(reinterpret_cast<double2 *>(p), make_double2(q.a, q.b));
    }
    __device__ static inline void sts(double *p, QV<double> q) { *reinterpret_cast<double2 *>(p) = make_double2(q.a, q.b); }
};
template <> struct QIO<__nv_bfloat16> {
    __device__ static inline QV<float> cvt(uint2 raw)
    {
        const float2 fa = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&raw.x));
        const float2 fb = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&raw.y));
        return {fa, fb};
    }
    __device__ static inline QV<float> ldg(const __nv_bfloat16 *p) { return cvt(__ldg(reinterpret_cast<const uint2 *>(p))); }
    __device__ static inline QV<float> lds(const __nv_bfloat16 *p) { return cvt(*reinterpret_cast<const uint2 *>(p)); }
    __device__ static inline uint2 pack(QV<float> q)
    {
        const __nv_bfloat162 a = __floats2bfloat162_rn(q.a.x, q.a.y), b = __floats2bfloat162_rn(q.b.x, q.b.y);
        uint2 raw;
        raw.x = *reinterpret_cast<const uint32_t *>(&a);
        raw.y = *reinterpret_cast<const uint32_t *>(&b);
        return raw;
    }
    __device__ static inline void stg(__nv_bfloat16 *p, QV<float> q) { __stcs(reinterpret_cast<uint2 *>(p), pack(q)); }
    __device__ static inline void sts(__nv_bfloat16 *p, QV<float> q) { *reinterpret_cast<uint2 *>(p) = pack(q); }
};

// list of the upwind sources that group o uses along axis d: the minus-side
// list 2d for a positive velocity component, the plus-side list 2d+1 otherwise
__host__ __device__ constexpr int list_of(int o, int d) { return 2 * d + (((o >> (2 - d)) & 1) ? 0 : 1); }
template <int DIM> __host__ __device__ constexpr int lists_of(int o)
{
    return (1 << list_of(o, 0)) | (1 << list_of(o, 1)) | (DIM == 3 ? (1 << list_of(o, 2)) : 0);
}

// coefficient slots written by the solver warp for phase 3:
// f^{n+1} = (1 - nu dt) f* + KN gx gy gz (C0 + Px + Py + Pz)
enum { CF_KN = 0, CF_C0, CF_OMN, CF_DX, CF_DY, CF_DZ, CF_D4, CF_D0, CF_N };

// per-axis factors of the corrected Maxwellian: g = exp(-c^2/2) and
// P = d_axis c + d4 c^2, c = (xi - u)/sqrt(T)
template <typename TC> struct TabE {
    TC g, p;
};

// One cell's stencil, as the dispatching solver warp hands it to the
// compute warps three iterations ahead.
template <typename TC> struct CellSlot {
    long long cell;      // -1: no cell left
    int32_t sidx[6];     // chunk index (cell * 8 + group, in units of P) of each list's first
                         // source for group 0, wall flip folded in
    int32_t src[24];     // per list (axis x side) up to 4 sources: cell | group flip << 28
    TC w[24];            // A_k / V_j
    int cnt[6];
    int xmask;           // lists with more than one source
    TC invh;
};

template <typename TC> struct StepSmem {
    using X = typename Num<TC>::X;
    CellSlot<TC> slot[NSL];
    X red[NSS][MAXCW][7];  // per compute warp: the seven moment partials of a cell
    long long cellp[NSS];  // cell of the partials in red (-1: none)
    TabE<TC> tab[NSS][3][NAX];
    TC coef[NSS][CF_N];
    typename Num<TC>::X mom[NSS][5];  // rho, u, T of the cell
    int ok[NSS];
    TC xin[3][NAX];   // velocity node values per axis, in index order
    long long next0[2];  // the cells of slots 4 and 5, taken by warp 0
    // the final solve of each solver warp: 1D sums, matrix entries,
    // right-hand side, solution and residual
    X g1d[2][3][5];
    X sys[2][15];
    X rhs[2][5], dsol[2][5], resid[2][5];
    // c_terms in shared memory: each lane of the matrix assembly reads its own
    // entry, which a constant-memory load would serialise
    int32_t terms[15][10];
};

template <typename TC> struct Consts {
    using N = Num<TC>;
    using X = typename N::X;
    X dV, hh[3], hh2[3], third, c15, one;
    TC nu0;  // sqrt(8/pi) dt / Kn: nu dt = nu0 rho sqrt(T)
};

template <typename TC>
__device__ inline typename Num<TC>::X split(double v)
{
    if constexpr (sizeof(TC) == 8) {
        return v;
    } else {
        const float hi = (float)v;
        return ffn{hi, (float)(v - (double)hi)};
    }
}

__device__ inline void bar_sync_n(int id, int n) { asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory"); }
__device__ inline void bar_arrive_n(int id, int n) { asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(n) : "memory"); }

// named barriers: BAR_P + j % 4 "partials of cell j ready",
// BAR_C + j % 4 "coefficients of cell j ready"
constexpr int BAR_P = 1, BAR_C = 5;

template <typename TS, int DIM> constexpr size_t stage_bytes(int P) { return (size_t)(1 + DIM) * P * sizeof(TS); }
// dynamic shared memory: the ring and the two f* tiles
template <typename TS, int DIM> constexpr size_t step_dyn_bytes(int P) { return NST * stage_bytes<TS, DIM>(P) + (size_t)2 * 8 * P * sizeof(TS); }

// the 16- or 8-byte piece of one thread
template <typename TS> __device__ inline void cp_piece(TS *dst, const TS *src, uint32_t dep)
{
    if constexpr (sizeof(TS) == 2) cp_async8(dst, src, dep);
    else cp_async16(dst, src, dep);
}

// Warp totals of seven per-lane sums by reduce-scatter: each butterfly level
// sends only the half of the sums that the partner keeps, so that three
// levels leave lane l with the sum (l >> 2) over the eight lanes that differ
// from it in bits 2-4, and two full levels finish it.  9 shuffles instead of
// 35.  Returns, in lane l, the warp total of sum l >> 2 (l < 28).
template <typename TC> __device__ inline TC warp_reduce7(const TC (&m)[7], int lane)
{
    TC a[4], b[2];
    const bool h4 = lane & 16, h3 = lane & 8, h2 = lane & 4;
#pragma unroll
    for (int i = 0; i < 4; i++) {
        const TC lo = m[i], hi = i < 3 ? m[4 + i] : (TC)0;
        a[i] = (h4 ? hi : lo) + __shfl_xor_sync(0xffffffffu, h4 ? lo : hi, 16);
    }
#pragma unroll
    for (int i = 0; i < 2; i++)
        b[i] = (h3 ? a[2 + i] : a[i]) + __shfl_xor_sync(0xffffffffu, h3 ? a[i] : a[2 + i], 8);
    TC c = (h2 ? b[1] : b[0]) + __shfl_xor_sync(0xffffffffu, h2 ? b[0] : b[1], 4);
    c += __shfl_xor_sync(0xffffffffu, c, 2);
    c += __shfl_xor_sync(0xffffffffu, c, 1);
    return c;
}

// ---------------------------------------------------------------- exact moment partials
// Error-free product (Dekker 1971): a b = p + e exactly, e recovered with one
// FMA.
__device__ inline ffn two_prod(float a, float b)
{
    const float p = a * b;
    return {p, fmaf(a, b, -p)};
}

__device__ inline float2 f2_add(float2 a, float2 b) { return __fadd2_rn(a, b); }
// b - a, rounded once
__device__ inline float2 f2_sub(float2 b, float2 a) { return __ffma2_rn(a, make_float2(-1.0f, -1.0f), b); }

// Signed sums over the eight sign groups, per position (packed pairs):
// S = sum_o x_o and X, Y, Z = sum_o s_d(o) x_o with s_d = +1 in the groups of
// positive xi_d (group o = 4[xi_x > 0] + 2[xi_y > 0] + [xi_z > 0]).
__device__ inline void group_sums(const float2 (&x)[8], float2 &S, float2 &X, float2 &Y, float2 &Z)
{
    float2 pz[4], mz[4];
#pragma unroll
    for (int k = 0; k < 4; k++) {
        pz[k] = f2_add(x[2 * k], x[2 * k + 1]);
        mz[k] = f2_sub(x[2 * k + 1], x[2 * k]);
    }
    Z = f2_add(f2_add(mz[0], mz[1]), f2_add(mz[2], mz[3]));
    const float2 pp0 = f2_add(pz[0], pz[1]), pm0 = f2_sub(pz[1], pz[0]);
    const float2 pp1 = f2_add(pz[2], pz[3]), pm1 = f2_sub(pz[3], pz[2]);
    Y = f2_add(pm0, pm1);
    S = f2_add(pp0, pp1);
    X = f2_sub(pp1, pp0);
}

// The seven moment partials of one thread's 32 values of f* (8 groups x 4
// consecutive z positions, node indices jx, jy, jz0 + 2e as odd integers,
// xi_d = (h_d/2) s_d j_d):
//   sum f, jx sum s_x f, jy sum s_y f, sum s_z jz f, jx^2 sum f, jy^2 sum f,
//   sum jz^2 f
// as double-float numbers, exact to about 2^-38 of the thread's sum |f|.
// Each value is split x = q + r against sigma = 2^k >= 16 sum |x| (the
// extraction of Rump, Ogita and Oishi, 2008): q = fl(fl(sigma + x) - sigma)
// and r = x - q are exact, q is a multiple of 2^(k-24) and |r| <= 2^(k-24).
// Every signed sum of the q's with integer weights of total size below 16
// then stays a multiple of 2^(k-24) below 2^k, hence exact in FP32; the
// weights jz = jz0 + 2e enter through
//   sum_e jz_e Z_e = jz0 sum Z + 2 (Z_1 + 2 Z_2 + 3 Z_3),
//   sum_e jz_e^2 S_e = jz0^2 sum S + 4 jz0 (S_1 + 2 S_2 + 3 S_3) + 4 (S_1 + 4 S_2 + 9 S_3)
// and exact products; the r's, 2^-19 of sum |x| at most, are summed in FP32.
__device__ inline void thread_moments(const QV<float> (&cur)[8], float jx, float jy, float jz0, ffn (&m)[7])
{
    float2 B2 = make_float2(0.0f, 0.0f);
#pragma unroll
    for (int o = 0; o < 8; o++) {
        B2 = f2_add(B2, make_float2(fabsf(cur[o].a.x), fabsf(cur[o].a.y)));
        B2 = f2_add(B2, make_float2(fabsf(cur[o].b.x), fabsf(cur[o].b.y)));
    }
    const float B = B2.x + B2.y;
    // B < 2^(ex - 126): sigma = 2^(ex - 122) >= 16 B (B finite)
    const int ex = min((__float_as_int(B) >> 23) & 0xff, 249);
    const float sg = __int_as_float((ex + 5) << 23);
    const float2 s2 = make_float2(sg, sg);
    float2 qa[8], qb[8], ra[8], rb[8];
#pragma unroll
    for (int o = 0; o < 8; o++) {
        qa[o] = f2_sub(f2_add(cur[o].a, s2), s2);
        qb[o] = f2_sub(f2_add(cur[o].b, s2), s2);
        ra[o] = f2_sub(cur[o].a, qa[o]);
        rb[o] = f2_sub(cur[o].b, qb[o]);
    }
    // exact parts: per position e = 0..3 (pairs a = (0, 1), b = (2, 3))
    float2 Sa, Xa, Ya, Za, Sb, Xb, Yb, Zb;
    group_sums(qa, Sa, Xa, Ya, Za);
    group_sums(qb, Sb, Xb, Yb, Zb);
    const float2 Sab = f2_add(Sa, Sb), Xab = f2_add(Xa, Xb), Yab = f2_add(Ya, Yb), Zab = f2_add(Za, Zb);
    const float Sq = Sab.x + Sab.y;
    const float Xq = Xab.x + Xab.y;
    const float Yq = Yab.x + Yab.y;
    const float Zq = Zab.x + Zab.y;
    const float Az = (Za.y + (Zb.x + Zb.x)) + 3.0f * Zb.y;
    const float A1 = (Sa.y + (Sb.x + Sb.x)) + 3.0f * Sb.y;
    const float A2 = (Sa.y + 4.0f * Sb.x) + 9.0f * Sb.y;
    // rounding parts, in FP32
    group_sums(ra, Sa, Xa, Ya, Za);
    group_sums(rb, Sb, Xb, Yb, Zb);
    const float Sr = (Sa.x + Sa.y) + (Sb.x + Sb.y);
    const float Xr = (Xa.x + Xa.y) + (Xb.x + Xb.y);
    const float Yr = (Ya.x + Ya.y) + (Yb.x + Yb.y);
    const float Zr = (Za.x + Za.y) + (Zb.x + Zb.y);
    const float Azr = (Za.y + 2.0f * Zb.x) + 3.0f * Zb.y;
    const float A1r = (Sa.y + 2.0f * Sb.x) + 3.0f * Sb.y;
    const float A2r = (Sa.y + 4.0f * Sb.x) + 9.0f * Sb.y;
    const float jx2 = jx * jx, jy2 = jy * jy, jz2 = jz0 * jz0, jz4 = 4.0f * jz0;
    ffn t[7];
    t[0] = ffn{Sq, 0.0f};
    t[1] = two_prod(jx, Xq);
    t[2] = two_prod(jy, Yq);
    t[3] = two_prod(jz0, Zq) + ffn{2.0f * Az, 0.0f};
    t[4] = two_prod(jx2, Sq);
    t[5] = two_prod(jy2, Sq);
    t[6] = (two_prod(jz2, Sq) + two_prod(jz4, A1)) + ffn{4.0f * A2, 0.0f};
    const float r[7] = {Sr, jx * Xr, jy * Yr, fmaf(jz0, Zr, 2.0f * Azr), jx2 * Sr, jy2 * Sr,
                        fmaf(jz2, Sr, fmaf(jz4, A1r, 4.0f * A2r))};
#pragma unroll
    for (int k = 0; k < 7; k++) m[k] = ffn{t[k].hi, t[k].lo + r[k]};  // normalised by the first add of the reduction
}

// warp_reduce7 on double-float numbers (the same reduce-scatter): returns,
// in lane l, the warp total of sum l >> 2 (l < 28)
__device__ inline ffn warp_reduce7_df(const ffn (&m)[7], int lane)
{
    auto sx = [](ffn v, int k) -> ffn {
        return {__shfl_xor_sync(0xffffffffu, v.hi, k), __shfl_xor_sync(0xffffffffu, v.lo, k)};
    };
    // a + b with one error-free transformation of the high parts and the
    // low parts added: left unnormalised until the last add, which
    // normalises
    auto add = [](ffn a, ffn b) -> ffn {
        const float t = a.hi + b.hi;
        const float bb = t - a.hi;
        return {t, ((a.hi - (t - bb)) + (b.hi - bb)) + (a.lo + b.lo)};
    };
    ffn a[4], b[2];
    const bool h4 = lane & 16, h3 = lane & 8, h2 = lane & 4;
#pragma unroll
    for (int i = 0; i < 4; i++) {
        const ffn lo = m[i], hi = i < 3 ? m[4 + i] : ffn{0.0f, 0.0f};
        a[i] = add(h4 ? hi : lo, sx(h4 ? lo : hi, 16));
    }
#pragma unroll
    for (int i = 0; i < 2; i++) b[i] = add(h3 ? a[2 + i] : a[i], sx(h3 ? a[i] : a[2 + i], 8));
    ffn c = add(h2 ? b[1] : b[0], sx(h2 ? b[0] : b[1], 4));
    c = add(c, sx(c, 2));
    c = c + sx(c, 1);
    return c;
}

template <typename T> __device__ inline uint32_t dep_of(const QV<T> &q)
{
    if constexpr (sizeof(T) == 8) return (uint32_t)__double2loint(q.a);
    else return __float_as_uint(q.a.x);
}

// ---------------------------------------------------------------- solver
// The 15 distinct entries (r <= s) of the moment matrix of the target in the
// centred basis phi = (1, c_x, c_y, c_z, |c|^2 - 3):
//   A_rs = K dV sum_i phi_r phi_s g_x g_y g_z = K dV sum_t coef_t Gx[a_t] Gy[b_t] Gz[c_t],
// G_d[k] = sum_n g_d(n) c_d(n)^k the 1D sums of axis d.  Each term is packed
// as coef (signed byte) | a << 8 | b << 12 | c << 16; coef 0 pads.  Entry 14,
// (|c|^2 - 3)^2, has ten terms and is split over two lanes.
#define DVM_T(cf, a, b, c) ((int32_t)((cf) & 0xff) | ((a) << 8) | ((b) << 12) | ((c) << 16))
__constant__ int32_t c_terms[15][10] = {
    {DVM_T(1, 0, 0, 0)},
    {DVM_T(1, 1, 0, 0)},
    {DVM_T(1, 0, 1, 0)},
    {DVM_T(1, 0, 0, 1)},
    {DVM_T(1, 2, 0, 0), DVM_T(1, 0, 2, 0), DVM_T(1, 0, 0, 2), DVM_T(-3, 0, 0, 0)},
    {DVM_T(1, 2, 0, 0)},
    {DVM_T(1, 1, 1, 0)},
    {DVM_T(1, 1, 0, 1)},
    {DVM_T(1, 3, 0, 0), DVM_T(1, 1, 2, 0), DVM_T(1, 1, 0, 2), DVM_T(-3, 1, 0, 0)},
    {DVM_T(1, 0, 2, 0)},
    {DVM_T(1, 0, 1, 1)},
    {DVM_T(1, 2, 1, 0), DVM_T(1, 0, 3, 0), DVM_T(1, 0, 1, 2), DVM_T(-3, 0, 1, 0)},
    {DVM_T(1, 0, 0, 2)},
    {DVM_T(1, 2, 0, 1), DVM_T(1, 0, 2, 1), DVM_T(1, 0, 0, 3), DVM_T(-3, 0, 0, 1)},
    {DVM_T(1, 4, 0, 0), DVM_T(1, 0, 4, 0), DVM_T(1, 0, 0, 4), DVM_T(2, 2, 2, 0), DVM_T(2, 2, 0, 2),
     DVM_T(2, 0, 2, 2), DVM_T(-6, 2, 0, 0), DVM_T(-6, 0, 2, 0), DVM_T(-6, 0, 0, 2), DVM_T(9, 0, 0, 0)},
};
#undef DVM_T

// index of entry (r, s) among the 15 distinct ones
__device__ inline int sym_e(int r, int s)
{
    const int a = r < s ? r : s, c = r < s ? s : r;
    return a * 5 - (a * (a - 1)) / 2 + (c - a);
}

// a double-float pair (hi, lo) of a compute-precision-class number
__device__ inline float2 to_pair(ffn v) { return make_float2(v.hi, v.lo); }
__device__ inline float2 to_pair(double v)
{
    const float hi = (float)v;
    return make_float2(hi, (float)(v - (double)hi));
}

// Phase 2 of one cell on one warp (parity par): moments of f* from the
// compute warps' partials, the coefficients of the target and its per-axis
// tables into slot b.  Returns the status flags of the cell.  The code is
// kept compact (rolled loops) because it runs once per cell between the
// compute warps' instruction streams: straight-line code of this length would
// be fetched from beyond the instruction cache every time.
//
// Precision (FP32/BF16 storage): the moment sums arrive in double-float; the
// target's 1D sums, the 5x5 system of Eq. 6's correction and its solution are
// formed in double-float (an FP32 LDL^T factor refined once against a
// double-float residual), so that the collision term nu (M~ - f*) defined by
// the per-axis tables g and the double-float coefficients carries the moments
// of f* to double-float accuracy.  Its residual sum_i phi_r (M~ - f*)_i dV in
// the centred basis goes to res_phi as double-float pairs (no FP64
// instruction on this warp: FP64 runs at a small fraction of the FP32 rate
// here and measured 8 ms per step on the Mach-5 workload).  The FP32 evaluation of M~ at each
// node (and the FP32 copy of the coefficients it uses) rounds like the FP32
// store that follows it.
template <typename TC, int COLL>
__device__ inline int solve_cell(const StepParams &p, StepSmem<TC> &sm, const Consts<TC> &K, int b, int ncw,
                                 long long cell, int par)
{
    using N = Num<TC>;
    using X = typename N::X;
    const int lane = threadIdx.x & 31;
    // the seven sums: lane 4k + q adds the partials of warps q, q + 4, ...
    // of sum k, then the four lanes of each sum combine
    X acc = N::make((TC)0);
    {
        const int k = lane >> 2;
        if (k < 7) {
#pragma unroll 1
            for (int w = lane & 3; w < ncw; w += 4) acc = acc + sm.red[b][w][k];
        }
        acc = acc + N::shfl_xor(acc, 1);
        acc = acc + N::shfl_xor(acc, 2);
    }
    X Ssum[7];
#pragma unroll
    for (int k = 0; k < 7; k++) Ssum[k] = N::shfl(acc, 4 * k);
    const X s0 = Ssum[0];
    const X rho = s0 * K.dV;
    const X inv = N::recip(s0);
    const X ux = Ssum[1] * inv * K.hh[0];
    const X uy = Ssum[2] * inv * K.hh[1];
    const X uz = Ssum[3] * inv * K.hh[2];
    const X e2 = (Ssum[4] * K.hh2[0] + Ssum[5] * K.hh2[1] + Ssum[6] * K.hh2[2]) * inv;
    const X T = (e2 - (ux * ux + uy * uy + uz * uz)) * K.third;
    int flags = 0;
    if (!N::finite_pos(s0) || !N::finite_pos(T) || !isfinite(N::f(ux) + N::f(uy) + N::f(uz))) flags |= ST_NONPOS;
    // lane 0's verdict for the whole warp (the lanes' double-float sums may
    // differ in their last bits)
    flags = __shfl_sync(0xffffffffu, flags, 0);
    auto dbl = [](X v) -> double {
        if constexpr (sizeof(TC) == 4) return (double)v.hi + (double)v.lo;
        else return v;
    };
    // BGK: the target is the Maxwellian times the correction polynomial
    // 1 + d.phi, phi = (1, c, |c|^2 - 3), of Eq. 6's form.  Entropic BGK: the
    // target is exp(-|c|^2/2 + e.phi) (1 + d.phi); Newton steps on e (the
    // same solve, made at the current target) run in the compute precision
    // until the step is below ENT_TOL, and the last solve, below, gives the
    // polynomial d that closes the moments (O(d^2) from the exponential).
    constexpr bool ENT = COLL == DVM_COLL_BGK_ENTROPIC;
    constexpr int NIT = ENT ? 8 : 1;
    const TC ENT_TOL = sizeof(TC) == 8 ? (TC)1e-9 : (TC)1e-5;
    const int ax = lane >> 3, sub = lane & 7;
    const int nax = ax < 3 ? p.n[ax] : 0;
    if ((COLL == DVM_COLL_BGK || ENT) && flags == 0) {
        const TC uT[3] = {N::tc(ux), N::tc(uy), N::tc(uz)};
        const X isT = N::rsqrt(T);
        const TC isTt = N::tc(isT);
        const X Kc = rho * K.c15 * isT * isT * isT;  // rho (2 pi T)^(-3/2)
        const TC ud = ax == 0 ? uT[0] : (ax == 1 ? uT[1] : uT[2]);
        TC e[5] = {0, 0, 0, 0, 0};  // entropic: the accumulated e (every lane)
        if constexpr (ENT) {
            TC Kpt = N::tc(Kc);
#pragma unroll 1
            for (int it = 0; it < NIT; it++) {
                const TC ea = ax == 0 ? e[1] : (ax == 1 ? e[2] : e[3]), e4 = e[4];
                // 1D sums of g c^k, k = 0..4 (k = 0, 2 in double-float), with
                // c = (xi - u)/sqrt(T), g = exp(-c^2/2 + e_axis c + e4 c^2):
                // lanes 8d .. 8d + 7 take axis d, lane 8d + s the nodes s,
                // s + 8, ...; the eight lanes of an axis then combine
                X A0 = N::make((TC)0), A2 = N::make((TC)0);
                TC A1 = 0, A3 = 0, A4 = 0;
#pragma unroll 1
                for (int i = sub; i < nax; i += 8) {
                    const TC c = (sm.xin[ax][i] - ud) * isTt;
                    const TC g = tc_exp<TC>((TC)-0.5 * c * c + c * (ea + e4 * c));
                    const TC gc = g * c;
                    A0 = A0 + N::make(g);
                    A2 = A2 + N::make(gc) * c;
                    A1 += gc;
                    A3 += gc * c * c;
                    A4 += gc * c * c * c;
                }
#pragma unroll
                for (int m = 4; m > 0; m >>= 1) {
                    A0 = A0 + N::shfl_xor(A0, m);
                    A2 = A2 + N::shfl_xor(A2, m);
                    A1 += __shfl_xor_sync(0xffffffffu, A1, m);
                    A3 += __shfl_xor_sync(0xffffffffu, A3, m);
                    A4 += __shfl_xor_sync(0xffffffffu, A4, m);
                }
                X G0[3], G2[3];
                TC G1[3], G3[3], G4[3];
#pragma unroll
                for (int d = 0; d < 3; d++) {
                    G0[d] = N::shfl(A0, 8 * d);
                    G2[d] = N::shfl(A2, 8 * d);
                    G1[d] = __shfl_sync(0xffffffffu, A1, 8 * d);
                    G3[d] = __shfl_sync(0xffffffffu, A3, 8 * d);
                    G4[d] = __shfl_sync(0xffffffffu, A4, 8 * d);
                }
                const X KdV = N::make(Kpt) * K.dV;
                int done = 1;
                if (lane == 0) {
                    const X P0 = G0[0] * G0[1] * G0[2];
                    const X Q2 = G2[0] * G0[1] * G0[2] + G0[0] * G2[1] * G0[2] + G0[0] * G0[1] * G2[2];
                    const TC k = N::tc(KdV);
                    TC g0[3], g2[3];
#pragma unroll
                    for (int d = 0; d < 3; d++) { g0[d] = N::tc(G0[d]); g2[d] = N::tc(G2[d]); }
                    const TC p0v = g0[0] * g0[1] * g0[2];
                    TC A[25], rhs[5], dd[5];
                    A[0] = N::tc(KdV * P0);
                    A[1] = k * G1[0] * g0[1] * g0[2];
                    A[2] = k * g0[0] * G1[1] * g0[2];
                    A[3] = k * g0[0] * g0[1] * G1[2];
                    A[4] = N::tc(KdV * (Q2 - P0 - P0 - P0));
                    A[6] = k * g2[0] * g0[1] * g0[2];
                    A[7] = k * G1[0] * G1[1] * g0[2];
                    A[8] = k * G1[0] * g0[1] * G1[2];
                    A[9] = k * (G3[0] * g0[1] * g0[2] + G1[0] * g2[1] * g0[2] + G1[0] * g0[1] * g2[2] -
                                (TC)3 * G1[0] * g0[1] * g0[2]);
                    A[12] = k * g0[0] * g2[1] * g0[2];
                    A[13] = k * g0[0] * G1[1] * G1[2];
                    A[14] = k * (g2[0] * G1[1] * g0[2] + g0[0] * G3[1] * g0[2] + g0[0] * G1[1] * g2[2] -
                                 (TC)3 * g0[0] * G1[1] * g0[2]);
                    A[18] = k * g0[0] * g0[1] * g2[2];
                    A[19] = k * (g2[0] * g0[1] * G1[2] + g0[0] * g2[1] * G1[2] + g0[0] * g0[1] * G3[2] -
                                 (TC)3 * g0[0] * g0[1] * G1[2]);
                    const TC s2 = g2[0] * g0[1] * g0[2] + g0[0] * g2[1] * g0[2] + g0[0] * g0[1] * g2[2];
                    A[24] = k * (G4[0] * g0[1] * g0[2] + g0[0] * G4[1] * g0[2] + g0[0] * g0[1] * G4[2] +
                                 (TC)2 * (g2[0] * g2[1] * g0[2] + g2[0] * g0[1] * g2[2] + g0[0] * g2[1] * g2[2]) -
                                 (TC)6 * s2 + (TC)9 * p0v);
#pragma unroll
                    for (int r = 0; r < 5; r++)
#pragma unroll
                        for (int c2 = 0; c2 < r; c2++) A[r * 5 + c2] = A[c2 * 5 + r];
                    rhs[0] = N::tc(rho - KdV * P0);
                    rhs[1] = -A[1];
                    rhs[2] = -A[2];
                    rhs[3] = -A[3];
                    rhs[4] = -A[4];
                    const bool okk = solve5_rcp<TC>(A, rhs, dd);
                    bool conv = okk;
#pragma unroll
                    for (int r = 0; r < 5; r++) {
                        if (!okk) dd[r] = 0;
                        conv = conv && fabs(dd[r]) < ENT_TOL;  // false on NaN
                        sm.coef[b][r == 0 ? CF_D0 : CF_DX + r - 1] = dd[r];
                    }
                    if (!okk) flags |= ST_SINGULAR;
                    done = conv || !okk;
                }
                __syncwarp();
                e[0] += sm.coef[b][CF_D0];
                e[1] += sm.coef[b][CF_DX];
                e[2] += sm.coef[b][CF_DY];
                e[3] += sm.coef[b][CF_DZ];
                e[4] += sm.coef[b][CF_D4];
                Kpt = N::tc(Kc) * tc_exp<TC>(e[0] - (TC)3 * e[4]);
                __syncwarp();
                if (__shfl_sync(0xffffffffu, done, 0)) break;
            }
        }
        // ---- the final solve, in X arithmetic (double-float for FP32 storage)
        // K of the target: rho (2 pi T)^(-3/2) (entropic: times exp(e0 - 3 e4))
        const X Kx = ENT ? Kc * tc_exp<TC>(e[0] - (TC)3 * e[4]) : Kc;
        const X KdV = Kx * K.dV;
        {
            // 1D sums G_d[k] = sum_n g_d(n) c_d(n)^k, k = 0..4, with the node
            // xi = (h_d/2) J, J = 2n + 1 - n_d (exact), c = (xi - u)/sqrt(T) in
            // X, g from c rounded to TC (the table value the collision uses)
            X G[5];
#pragma unroll
            for (int k = 0; k < 5; k++) G[k] = N::make((TC)0);
            if (ax < 3) {
                const X uX = ax == 0 ? ux : (ax == 1 ? uy : uz);
                const TC ea = ENT ? (ax == 0 ? e[1] : (ax == 1 ? e[2] : e[3])) : (TC)0, e4 = ENT ? e[4] : (TC)0;
#pragma unroll 1
                for (int i = sub; i < nax; i += 8) {
                    const X c = (K.hh[ax] * (TC)(2 * i + 1 - nax) - uX) * isT;
                    const TC cf = N::tc(c);
                    TC ex = (TC)-0.5 * cf * cf;
                    if constexpr (ENT) ex += cf * (ea + e4 * cf);
                    const TC g = tc_exp<TC>(ex);
                    sm.tab[b][ax][i] = TabE<TC>{g, cf};  // p holds c until the solve is done
                    const X c2 = c * c;
                    G[0] = G[0] + N::make(g);
                    G[1] = G[1] + c * g;
                    G[2] = G[2] + c2 * g;
                    G[3] = G[3] + (c2 * c) * g;
                    G[4] = G[4] + (c2 * c2) * g;
                }
            }
#pragma unroll
            for (int m = 4; m > 0; m >>= 1)
#pragma unroll
                for (int k = 0; k < 5; k++) G[k] = G[k] + N::shfl_xor(G[k], m);
            if (sub == 0 && ax < 3)
#pragma unroll
                for (int k = 0; k < 5; k++) sm.g1d[par][ax][k] = G[k];
        }
        __syncwarp();
        {
            // the 15 entries on lanes 0..15 (entry 14 on lanes 14 and 15)
            X a = N::make((TC)0);
            if (lane < 16) {
                const int en = lane < 15 ? lane : 14, t0 = lane == 15 ? 5 : 0;
#pragma unroll 1
                for (int t = t0; t < t0 + 5; t++) {
                    const int32_t w = sm.terms[en][t];
                    const int cf = (int)(int8_t)(w & 0xff);
                    if (cf != 0) {
                        const X pr = sm.g1d[par][0][(w >> 8) & 15] * sm.g1d[par][1][(w >> 12) & 15] *
                                     sm.g1d[par][2][(w >> 16) & 15];
                        a = a + pr * (TC)cf;
                    }
                }
            }
            const X other = N::shfl(a, 15);
            if (lane == 14) a = a + other;
            if (lane < 15) sm.sys[par][lane] = a * KdV;
        }
        __syncwarp();
        // right-hand side: the moments of f* in phi are (rho, 0, 0, 0, 0) by
        // the definition of u and T, less those of the uncorrected target
        // (row 0 of the matrix); the TC factor of lane 0, then one refinement
        // against the X residual rhs - A d computed one row per lane (the
        // FP32 factor solves to ~1e-6 relative, one refinement to ~1e-12, and
        // the residual written below measures what is left)
        TC Lf[5][5], Dif[5];
        int fok = 1;
        if (lane == 0) {
            TC Af[25], r[5], dl[5];
#pragma unroll
            for (int r2 = 0; r2 < 5; r2++)
#pragma unroll
                for (int c2 = 0; c2 < 5; c2++) Af[r2 * 5 + c2] = N::tc(sm.sys[par][sym_e(r2, c2)]);
            sm.rhs[par][0] = rho - sm.sys[par][0];
#pragma unroll
            for (int r2 = 1; r2 < 5; r2++) sm.rhs[par][r2] = -sm.sys[par][r2];
            fok = ldl5<TC>(Af, Lf, Dif) ? 1 : 0;
#pragma unroll
            for (int r2 = 0; r2 < 5; r2++) r[r2] = N::tc(sm.rhs[par][r2]);
            if (fok) ldl5_solve<TC>(Lf, Dif, r, dl);
            else flags |= ST_SINGULAR;
#pragma unroll
            for (int r2 = 0; r2 < 5; r2++) sm.dsol[par][r2] = N::make(fok ? dl[r2] : (TC)0);
        }
        __syncwarp();
        fok = __shfl_sync(0xffffffffu, fok, 0);
#pragma unroll 1
        for (int it = 1; it < 3; it++) {
            if (lane < 5) {
                X s = sm.rhs[par][lane];
#pragma unroll
                for (int c2 = 0; c2 < 5; c2++) s = s - sm.sys[par][sym_e(lane, c2)] * sm.dsol[par][c2];
                sm.resid[par][lane] = s;
                // the last round: sum_i phi_r (M~ - f*)_i dV = A d - rhs, as a
                // double-float pair (the host takes it to psi and multiplies
                // by nu, in FP64)
                if (it == 2 && p.res_phi) p.res_phi[cell * 5 + lane] = fok ? to_pair(-s) : make_float2(0.0f, 0.0f);
            }
            __syncwarp();
            if (it == 2) break;
            if (lane == 0 && fok) {
                TC r[5], dl[5];
#pragma unroll
                for (int r2 = 0; r2 < 5; r2++) r[r2] = N::tc(sm.resid[par][r2]);
                ldl5_solve<TC>(Lf, Dif, r, dl);
#pragma unroll
                for (int r2 = 0; r2 < 5; r2++) sm.dsol[par][r2] = sm.dsol[par][r2] + N::make(dl[r2]);
            }
            __syncwarp();
        }
        TC *cf = sm.coef[b];
        if (lane == 0) {
            const X d0 = sm.dsol[par][0], d4 = sm.dsol[par][4];
            cf[CF_D0] = N::tc(d0);
            cf[CF_DX] = N::tc(sm.dsol[par][1]);
            cf[CF_DY] = N::tc(sm.dsol[par][2]);
            cf[CF_DZ] = N::tc(sm.dsol[par][3]);
            cf[CF_D4] = N::tc(d4);
            cf[CF_C0] = N::tc(N::make((TC)1) + d0 - d4 * (TC)3);
            const TC nudt = K.nu0 * N::tc(rho) * sqrt(N::tc(T));
            if (nudt > (TC)1) flags |= ST_NUDT;
            cf[CF_KN] = nudt * N::tc(Kx);
            cf[CF_OMN] = (TC)1 - nudt;
        }
        __syncwarp();
        // per-axis factors of the target, each lane for its nodes:
        // g (stored above) and P = c (d_axis + d4 c)
        const TC d4 = cf[CF_D4];
        if (ax < 3) {
            const TC da = cf[CF_DX + ax];
#pragma unroll 1
            for (int i = sub; i < nax; i += 8) {
                const TC c = sm.tab[b][ax][i].p;
                sm.tab[b][ax][i].p = c * (da + d4 * c);
            }
        }
    } else if (lane < 5 && p.res_phi) {
        p.res_phi[cell * 5 + lane] = make_float2(0.0f, 0.0f);
    }
    if (lane == 0) {
        sm.mom[b][0] = rho;
        sm.mom[b][1] = ux;
        sm.mom[b][2] = uy;
        sm.mom[b][3] = uz;
        sm.mom[b][4] = T;
    }
    return __shfl_sync(0xffffffffu, flags, 0);
}

// PC: the group size P as a compile-time constant (0: read it from p), so
// that every group offset of the unrolled loops is an immediate.
template <typename TS, int DIM, int COLL, int PC>
__global__ void __launch_bounds__(MAXT, 1) k_step(const StepParams p)
{
    using S = Store<TS>;
    using IO = QIO<TS>;
    using TC = typename S::TC;
    using Q4 = QV<TC>;
    constexpr int VEC = S::VEC;

    const int P = PC ? PC : p.P;  // velocity nodes per sign group
    const int NV = 8 * P;
    __shared__ StepSmem<TC> sm;
    __shared__ Consts<TC> K;
    extern __shared__ __align__(128) unsigned char dsm[];
    TS *ring = reinterpret_cast<TS *>(dsm);       // [NST][1 + DIM][P]
    TS *tiles = ring + (size_t)NST * (1 + DIM) * P;  // [2][nv]: f* of cells j - 1 and j - 2

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // warps 0 and 1 solve (the lowest warp numbers, so that a scheduler that
    // favours older warps gives the serial per-cell work precedence); warps
    // 2 .. ncw + 1 compute, thread ctid of them
    const int ncw = (blockDim.x >> 5) - 2;
    const int cw = warp - 2, ctid = tid - 64;
    const int nbar = (ncw + 1) * 32;        // threads on each named barrier
    const int Q = P / VEC;
    const TS *__restrict__ fin = static_cast<const TS *>(p.f_in);
    TS *__restrict__ fout = static_cast<TS *>(p.f_out);

    // cell dispatch (one warp): a cell index from the global counter (-1
    // once it has run out), its stencil fetched into registers, then stored
    // into a slot; split so that a solver overlaps the counter's round trip
    // and the loads with its own work.
    // raw loaded values only: anything computed from them waits for the
    // loads, so it is left to store(), after the solve
    struct Sten {
        long long cell;
        int32_t src, first;
        TC w;
        int cnt;
        TC invh;
    };
    auto take_issue = [&]() -> unsigned long long { return lane == 0 ? atomicAdd(p.counter, 1ull) : 0ull; };
    auto take_finish = [&](unsigned long long c) -> long long {
        c = __shfl_sync(0xffffffffu, c, 0);
        return c < (unsigned long long)p.ncells ? (long long)c : -1;
    };
    auto take = [&]() -> long long { return take_finish(take_issue()); };
    auto fetch = [&](long long cell) {
        Sten t{cell, 0, 0, (TC)0, 0, (TC)0};
        if (cell >= 0) {
            if (lane < 24) {
                t.src = p.st_src[cell * 24 + lane];
                t.w = static_cast<const TC *>(p.st_w)[cell * 24 + lane];
            }
            if (lane < 6) {
                t.cnt = p.st_cnt[cell * 8 + lane];
                t.first = p.st_src[cell * 24 + lane * 4];
            }
            if (lane == 0) t.invh = static_cast<const TC *>(p.inv_h)[cell];
        }
        return t;
    };
    auto store = [&](const Sten &t, int k) {
        CellSlot<TC> &sl = sm.slot[k % NSL];
        if (t.cell >= 0) {
            if (lane < 24) {
                sl.src[lane] = t.src;
                sl.w[lane] = t.w;
            }
            if (lane < 6) {
                sl.cnt[lane] = t.cnt;
                // group o reads source group o ^ flip = o -/+ flip for the minus/plus list
                const int32_t flip = t.first >> 28;
                sl.sidx[lane] = (t.first & 0x0fffffff) * 8 + ((lane & 1) ? flip : -flip);
            }
            const unsigned xm = __ballot_sync(0xffffffffu, lane < 6 && t.cnt > 1);
            if (lane == 0) {
                sl.xmask = (int)xm;
                sl.invh = t.invh;
            }
        }
        if (lane == 0) sl.cell = t.cell;
    };

    if (warp == 0) {
        // the cells of slots 0..5 in slot order (so that each parity's takes
        // come in its slot order) and the stencils of slots 0..3; the solver
        // warps fetch those of slot j + 4 while they solve cell j
        for (int k = 0; k < 4; k++) store(fetch(take()), k);
        for (int i = lane; i < 150; i += 32) (&sm.terms[0][0])[i] = (&c_terms[0][0])[i];
        {
            const long long n4 = take();
            const long long n5 = take();
            if (lane == 0) {
                sm.next0[0] = n4;
                sm.next0[1] = n5;
            }
        }
#pragma unroll
        for (int d = 0; d < 3; d++) {
            const int hd = p.half[d];
            if (lane < p.n[d]) {
                const int mm = lane < hd ? hd - 1 - lane : lane - hd;
                TC xi;
                if constexpr (sizeof(TC) == 8) xi = p.amag[d * 32 + mm];
                else xi = p.amag_f[d * 32 + mm];
                sm.xin[d][lane] = lane < hd ? -xi : xi;
            }
        }
        if (lane == 0) {
            K.dV = split<TC>(p.dV);
            for (int d = 0; d < 3; d++) {
                K.hh[d] = split<TC>(0.5 * p.hv[d]);
                K.hh2[d] = split<TC>(0.25 * p.hv[d] * p.hv[d]);
            }
            K.third = split<TC>(1.0 / 3.0);
            K.c15 = split<TC>(0.06349363593424097);  // (2 pi)^(-3/2)
            K.one = split<TC>(1.0);
            K.nu0 = (TC)(1.5957691216057308 * p.dt / p.kn);
        }
    }
    __syncthreads();

    if (warp < 2) {
        // ================= solver warps: warp b takes the cells j = b mod 2
        // It stops at its first empty slot: every later slot of its parity
        // is empty too.  The slot records of its parity are written by this
        // warp (or by warp 0 before the CTA barrier), so the test is local.
        const int par = warp;
        long long next_cell = sm.next0[par];  // the cell of slot par + 4
        for (int j = par;; j += 2) {
            if (sm.slot[j % NSL].cell < 0) break;
            const int q = j % NSS;
            bar_sync_n(BAR_P + q, nbar);
            const long long cell = sm.cellp[q];
            // the stencil of slot j + 4 and the cell of slot j + 6: their
            // loads and the counter's round trip are in flight during the solve
            const Sten nst = fetch(next_cell);
            const unsigned long long nc = take_issue();
            const int flags = solve_cell<TC, COLL>(p, sm, K, q, ncw, cell, par);
            store(nst, j + 4);
            next_cell = take_finish(nc);
            if (lane == 0) {
                if (flags) atomicOr(p.status, flags);
                sm.ok[q] = (COLL == DVM_COLL_BGK || COLL == DVM_COLL_BGK_ENTROPIC) &&
                           (flags & (ST_NONPOS | ST_SINGULAR)) == 0;
            }
            bar_arrive_n(BAR_C + q, nbar);
        }
        return;
    }

    // ================= compute warps
    const bool active = ctid < Q;
    const int p0 = active ? ctid * VEC : 0;
    int mpk;  // the thread's node indices (each < 32) packed into one register
    TC dax, day;
    Q4 daz;   // dt |xi_d| per axis (the self coefficient is 1 - invh * their sum)
    {
        const int hz = p.half[2], hyy = p.half[1];
        const int mz0 = p0 % hz, my = (p0 / hz) % hyy, mx = p0 / (hz * hyy);
        mpk = mx | (my << 8) | (mz0 << 16);
        const TC dt = (TC)p.dt;
        TC t[VEC];
        if constexpr (sizeof(TC) == 8) {
            dax = dt * p.amag[mx];
            day = dt * p.amag[32 + my];
#pragma unroll
            for (int e = 0; e < VEC; e++) t[e] = DIM == 3 ? dt * p.amag[64 + mz0 + e] : (TC)0;
        } else {
            dax = dt * p.amag_f[mx];
            day = dt * p.amag_f[32 + my];
#pragma unroll
            for (int e = 0; e < VEC; e++) t[e] = DIM == 3 ? dt * p.amag_f[64 + mz0 + e] : (TC)0;
        }
        daz = q_make(t);
    }

    // The chunk indices (units of P values) of the cell whose groups are
    // being copied: its own group 0 and the first source of each list
    // (group o adds o).  Each thread reads back only the pieces it copied.
    const TS *fin_p0 = fin + p0;
    int idx_own = 0, idx_l[2 * DIM];
    // bit b set: parity b has met an empty slot, so every later slot of that
    // parity is empty (its solver warp has stopped writing slot records)
    int ended = 0;
    auto slot_cell = [&](int k) -> long long { return ((ended >> (k & 1)) & 1) ? -1 : sm.slot[k % NSL].cell; };
    auto point = [&](int k) -> bool {
        const CellSlot<TC> &sl = sm.slot[k % NSL];
        const long long c = slot_cell(k);
#pragma unroll
        for (int L = 0; L < 2 * DIM; L++) idx_l[L] = sl.sidx[L];
        idx_own = (int)c * 8;
        return c >= 0 && active;
    };
    // group o of the pointed cell into stage st; dep orders the previous
    // reads of the stage before the copy
    auto copy_group = [&](bool on, int o, int st, uint32_t dep) {
        if (on) {
            TS *d = ring + (size_t)st * (1 + DIM) * P + p0;
            cp_piece(d, fin_p0 + (size_t)(uint32_t)(idx_own + o) * P, dep);
#pragma unroll
            for (int a = 0; a < DIM; a++)
                cp_piece(d + (1 + a) * P, fin_p0 + (size_t)(uint32_t)(idx_l[list_of(o, a)] + o) * P, dep);
        }
        cp_async_commit();
    };
    {
        const bool on = point(0);
#pragma unroll
        for (int o = 0; o < NST; o++) copy_group(on, o, o, 0u);
    }

    Q4 cur[8];   // f* of cell j
    long long cprev1 = -1, cprev2 = -1;  // the cells of slots j - 1 and j - 2
    for (int j = 0;; j++) {
        const int q = j % NSS;
        const CellSlot<TC> &sl = sm.slot[j % NSL];
        const long long cell = slot_cell(j);
        if (cell < 0) ended |= 1 << (j & 1);
        const bool valid = cell >= 0;
        {
            // ================= phase 1: transport of cell j (an empty slot
            // runs only the copy ring, which brings in the next cell)
            bool on = point(j);  // groups 4..7 of this cell are copied first
            // the next cell's own values (an HBM stream) are prefetched into L2
            // one cell ahead, so that their copies four groups later hit L2
            const long long nxt = slot_cell(j + 1);
            const TS *pf = fin_p0 + (size_t)(nxt < 0 ? 0 : nxt) * NV;
            const TC invh = sl.invh;
            const Q4 cs = q_fma(q_splat(-invh), q_add(q_splat(dax + day), daz), q_splat((TC)1));
            TC aw[4], wz[2];
#pragma unroll
            for (int L = 0; L < 4; L++) aw[L] = (L < 2 ? dax : day) * sl.w[L * 4];
            wz[0] = sl.w[16];
            wz[1] = sl.w[20];
            const Q4 dz0 = q_mul(daz, q_splat(wz[0])), dz1 = q_mul(daz, q_splat(wz[1]));
            const int xm = sl.xmask;
#pragma unroll
            for (int o = 0; o < 8; o++) {
                // this thread's pieces of group o have landed when at most
                // NST - 1 younger copy groups are pending
                cp_async_wait<NST - 1>();
                Q4 fs = q_splat((TC)0);
                if (valid && active) {
                    const TS *st = ring + (size_t)(o % NST) * (1 + DIM) * P + p0;
                    fs = q_mul(cs, IO::lds(st));
#pragma unroll
                    for (int d = 0; d < DIM; d++) {
                        const int L = list_of(o, d);
                        const Q4 w = d < 2 ? q_splat(aw[L]) : (L == 4 ? dz0 : dz1);
                        fs = q_fma(w, IO::lds(st + (1 + d) * P), fs);
                    }
                    if (xm & lists_of<DIM>(o)) {
                        // further sources: the fine neighbours behind a coarse face
#pragma unroll 1
                        for (int d = 0; d < DIM; d++) {
                            const int L = list_of(o, d);
                            const Q4 da = d == 0 ? q_splat(dax) : (d == 1 ? q_splat(day) : daz);
                            for (int k = 1; k < sl.cnt[L]; k++) {
                                const int32_t src = sl.src[L * 4 + k];
                                const Q4 v = IO::ldg(fin + (int64_t)(src & 0x0fffffff) * NV +
                                                     (o ^ (src >> 28)) * P + p0);
                                fs = q_fma(q_mul(da, q_splat(sl.w[L * 4 + k])), v, fs);
                            }
                        }
                    }
                }
                cur[o] = fs;
                if (active && nxt >= 0) prefetch_l2(pf + o * P);
                // refill the stage, NST groups ahead: groups 4..7 of this cell,
                // then groups 0..3 of the next one
                if (o == NST) on = point(j + 1);
                copy_group(on, (o + NST) & 7, o % NST, dep_of(fs));
            }
        }
        if (valid) {
            // the seven integer-weighted partial sums of this thread:
            // sum f, sum s_x j_x f, sum s_y j_y f, sum s_z j_z f, sum j_x^2 f,
            // sum j_y^2 f, sum j_z^2 f  (xi_d = (h_d/2) s_d j_d, j_d odd)
            const int kx = mpk & 0xff, ky = (mpk >> 8) & 0xff, kz = mpk >> 16;
            if constexpr (sizeof(TC) == 4) {
                ffn m[7];
                thread_moments(cur, (float)(2 * kx + 1), (float)(2 * ky + 1), (float)(2 * kz + 1), m);
                const ffn tot = warp_reduce7_df(m, lane);
                if ((lane & 3) == 0 && lane < 28) sm.red[q][cw][lane >> 2] = tot;
            } else {
                Q4 T0 = q_splat((TC)0), Tz = q_splat((TC)0);
                TC Sx = 0, Sy = 0;
#pragma unroll
                for (int o = 0; o < 8; o++) {
                    T0 = q_add(T0, cur[o]);
                    Tz = q_add(Tz, (o & 1) ? cur[o] : q_neg(cur[o]));
                    const TC qs = q_sum(cur[o]);
                    Sx += (o & 4) ? qs : -qs;
                    Sy += (o & 2) ? qs : -qs;
                }
                const TC jx = (TC)(2 * kx + 1), jy = (TC)(2 * ky + 1);
                TC jz[VEC], jz2[VEC];
#pragma unroll
                for (int e = 0; e < VEC; e++) {
                    jz[e] = (TC)(2 * (kz + e) + 1);
                    jz2[e] = jz[e] * jz[e];
                }
                TC m[7];
                m[0] = q_sum(T0);
                m[1] = jx * Sx;
                m[2] = jy * Sy;
                m[3] = q_sum(q_mul(q_make(jz), Tz));
                m[4] = jx * jx * m[0];
                m[5] = jy * jy * m[0];
                m[6] = q_sum(q_mul(q_make(jz2), T0));
                const TC tot = warp_reduce7<TC>(m, lane);
                if ((lane & 3) == 0 && lane < 28) sm.red[q][cw][lane >> 2] = tot;
            }
            if (ctid == 0) sm.cellp[q] = cell;
            bar_arrive_n(BAR_P + q, nbar);
        }

        TS *tile = tiles + (size_t)(j & 1) * NV + p0;  // f* of cell j - 2, then of cell j
        if (cprev2 >= 0) {
            // ================= phase 3: collision of cell j - 2
            const int q2 = (j - 2) % NSS;
            bar_sync_n(BAR_C + q2, nbar);
            const long long pc = cprev2;
            if (cw == 0 && lane < 5) {
                // the moments of f* in FP64, one per lane
                const typename Num<TC>::X v = sm.mom[q2][lane];
                if constexpr (sizeof(TC) == 4) p.mom_out[pc * 5 + lane] = (double)v.hi + (double)v.lo;
                else p.mom_out[pc * 5 + lane] = (double)v;
            }
            if (active) {
                TS *dst = fout + pc * (int64_t)NV + p0;
                if (sm.ok[q2]) {
                    const int mx = mpk & 0xff, my = (mpk >> 8) & 0xff, mz0 = mpk >> 16;
                    const int hz = p.half[2], hyy = p.half[1], hxx = p.half[0];
                    const TabE<TC> *tx = sm.tab[q2][0], *ty = sm.tab[q2][1], *tz = sm.tab[q2][2];
                    const TC KN = sm.coef[q2][CF_KN], C0 = sm.coef[q2][CF_C0];
                    const Q4 omn = q_splat(sm.coef[q2][CF_OMN]);
                    // the x-y factors of the four x-y sign pairs (the same for
                    // both z signs), then per z sign the z factors gz and gz Pz
                    // of the thread's nodes
                    TC Axy[4], Bxy[4];
#pragma unroll
                    for (int sxy = 0; sxy < 4; sxy++) {
                        const TabE<TC> a = tx[(sxy & 2) ? hxx + mx : hxx - 1 - mx];
                        const TabE<TC> c = ty[(sxy & 1) ? hyy + my : hyy - 1 - my];
                        Bxy[sxy] = KN * a.g * c.g;
                        Axy[sxy] = Bxy[sxy] * (C0 + a.p + c.p);
                    }
#pragma unroll
                    for (int pz = 0; pz < 2; pz++) {
                        TC g[VEC], gp[VEC];
#pragma unroll
                        for (int e = 0; e < VEC; e++) {
                            const TabE<TC> t = tz[pz ? hz + mz0 + e : hz - 1 - mz0 - e];
                            g[e] = t.g;
                            gp[e] = t.g * t.p;
                        }
                        const Q4 Z1 = q_make(g), Z2 = q_make(gp);
#pragma unroll
                        for (int sxy = 0; sxy < 4; sxy++) {
                            const TC B = Bxy[sxy];
                            const TC A = Axy[sxy];
                            const int o = 2 * sxy + pz;
                            const Q4 mt = q_fma(q_splat(A), Z1, q_mul(q_splat(B), Z2));
                            IO::stg(dst + o * P, q_fma(omn, IO::lds(tile + o * P), mt));
                        }
                    }
                } else {
#pragma unroll
                    for (int o = 0; o < 8; o++) IO::stg(dst + o * P, IO::lds(tile + o * P));
                }
            }
        }
        // f* of cell j waits in the tile the collision just read (each thread
        // rewrites only its own positions)
        if (valid && active) {
#pragma unroll
            for (int o = 0; o < 8; o++) IO::sts(tile + o * P, cur[o]);
        }
        cprev2 = cprev1;
        cprev1 = cell;
        // done once both parities have run out and no collision is pending
        if (ended == 3 && cprev1 < 0 && cprev2 < 0) break;
    }
    cp_async_wait_all();
}

template <typename TS, int DIM, int COLL, int PC>
int launch_kernel(const StepParams &p, int ncw)
{
    auto kern = k_step<TS, DIM, COLL, PC>;
    const int threads = (ncw + 2) * 32;
    const size_t dyn = step_dyn_bytes<TS, DIM>(p.P);
    cudaFuncAttributes fa{};
    if (cudaFuncGetAttributes(&fa, kern) != cudaSuccess) return DVM_ECUDA;
    int dev = 0, optin = 0, nsm = 0, occ = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (fa.sharedSizeBytes + dyn > (size_t)optin) return DVM_ENOTIMPL;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn) != cudaSuccess)
        return DVM_ECUDA;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, threads, dyn) != cudaSuccess || occ < 1)
        return DVM_ENOTIMPL;
    const int64_t grid = std::min<int64_t>(p.ncells, (int64_t)nsm * occ);
    kern<<<(unsigned)grid, threads, dyn, p.stream>>>(p);
    count_launch();
    return cudaGetLastError() == cudaSuccess ? DVM_OK : DVM_ECUDA;
}

// compile-time group sizes for the 24^3 and 16^3 grids of 3D FP32/BF16 runs
// (BGK, entropic BGK and transport alone)
template <typename TS, int DIM, int COLL>
int launch_sized(const StepParams &p, int ncw)
{
    if constexpr (DIM == 3 && sizeof(TS) <= 4) {
        if (p.P == 1728) return launch_kernel<TS, DIM, COLL, 1728>(p, ncw);
        if (p.P == 512) return launch_kernel<TS, DIM, COLL, 512>(p, ncw);
    }
    return launch_kernel<TS, DIM, COLL, 0>(p, ncw);
}

template <typename TS, int DIM>
int launch_typed(const StepParams &p)
{
    const int vec = Store<TS>::VEC;
    if (p.P % vec != 0 || p.half[2] % vec != 0) return DVM_EINVAL;
    for (int d = 0; d < 3; d++)
        if (p.n[d] > NAX) return DVM_ENOTIMPL;
    const int Q = p.P / vec;
    const int ncw = (Q + 31) / 32;
    if (ncw > MAXCW) return DVM_ENOTIMPL;
    if (p.coll == DVM_COLL_BGK) return launch_sized<TS, DIM, DVM_COLL_BGK>(p, ncw);
    if (p.coll == DVM_COLL_BGK_ENTROPIC) return launch_sized<TS, DIM, DVM_COLL_BGK_ENTROPIC>(p, ncw);
    return launch_sized<TS, DIM, DVM_COLL_NONE>(p, ncw);
}

}  // namespace

int launch_step(const StepParams &p)
{
    if (p.ncells <= 0) return DVM_OK;
    if (p.coll != DVM_COLL_NONE && p.coll != DVM_COLL_BGK && p.coll != DVM_COLL_BGK_ENTROPIC) return DVM_ENOTIMPL;
    switch (p.prec) {
    case DVM_F64: return p.dim == 3 ? launch_typed<double, 3>(p) : launch_typed<double, 2>(p);
    case DVM_F32: return p.dim == 3 ? launch_typed<float, 3>(p) : launch_typed<float, 2>(p);
    case DVM_BF16: return p.dim == 3 ? launch_typed<__nv_bfloat16, 3>(p) : launch_typed<__nv_bfloat16, 2>(p);
    default: return DVM_EINVAL;
    }
}

}  // namespace dvm
