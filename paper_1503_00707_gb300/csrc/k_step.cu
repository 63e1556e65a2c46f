// Fused DVM step: upwind transport (Eq. 2) -> moments of f* -> conservative
// BGK relaxation, with f* held on chip between the phases.
//
// Layout (paper Sec. 3.1 steps 1-3): f[cell][group][position], 8 sign groups
// per cell.  A compute thread owns the same "quad" of positions (4 FP32/BF16
// or 2 FP64 values along z) in all 8 groups: every warp reads 32 consecutive
// quads of one group (coalesced 16-byte loads) and the stencil of Eq. 2 is
// warp-uniform, since it depends on the group only through the signs of the
// velocity components (Sec. 3.1).
//
// Persistent CTAs take the Morton-ordered cells from a global counter, so
// the cells in flight on the whole GPU form one contiguous Morton window and
// upwind neighbours are served from L2 (a fixed round-robin assignment lets
// the CTAs drift apart over thousands of cells and spreads the window far
// beyond L2).  Each CTA has NCW compute warps and two solver warps that take
// alternate cells, so a cell's solve spans two pipeline iterations; one
// barrier per iteration:
//
//   iteration i, compute warps:  phase 1 of c_i              | barrier | phase 3 of c_{i-2}
//   iteration i, solver warp A:  first half of phase 2, c_{i-1}  |
//   iteration i, solver warp B:  second half of phase 2, c_{i-2};  |  bulk copy of c_{i+1}
//                                stencil of c_{i+1}              |
//
// A cell's own f arrives as one bulk copy (cp.async.bulk, completion on an
// mbarrier) into one of four shared tiles, issued one iteration ahead; phase
// 1 reads it from shared memory and writes f* over it in place, where it
// waits for phase 3.  Only the upwind neighbours are read through L2.  Waits
// on the tiles are bounded and report DVM_ETIMEOUT instead of hanging.
//
// Phase 1: f*_i = (1 - dt invh sum_d |xi_d,i|) f_i + sum_d dt |xi_d,i| sum_k
//   w_k src_k,i (Eq. 2 with the per-cell coefficients folded once), on packed
//   FP32 pairs; per-thread FP32 partials of the seven sums sum f, sum j_d f,
//   sum j_d^2 f (xi_d = (h_d/2) j_d with j_d an odd integer), reduced per
//   warp.
// Phase 2, first half: double-float sum of the warp partials -> rho, u, T;
//   the discrete Maxwellian factorises over the tensor grid, so its moments
//   in the centred basis phi = (1, c, |c|^2 - 3), c = (xi - u)/sqrt(T), are
//   products of 1D sums, formed here.  Second half: the five coefficients d
//   of M~ = M (1 + d.phi) (the correction form of Eq. 6) that make M~ carry
//   the moments of f* (defects of M's own moments in double-float, LDL^T
//   solve), and per-axis tables g = exp(-c^2/2), P = d_axis c + d4 c^2.
// Phase 3: f^{n+1} = (1 - nu dt) f* + nu dt M~ with M~ = rho (2 pi T)^(-3/2)
//   gx gy gz (1 + d0 - 3 d4 + Px + Py + Pz), nu = sqrt(8/pi) rho sqrt(T)/Kn.
// BF16 storage keeps f* in the tile rounded to BF16.
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
constexpr int NTILE = 4;      // shared tiles holding cells' own f
constexpr int NCQ = 8;        // ring of cell indices (taken three iterations ahead)

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
enum { CF_KN = 0, CF_C0, CF_OMN, CF_DX, CF_DY, CF_DZ, CF_D4, CF_N };

// per-axis factors of the corrected Maxwellian: g = exp(-c^2/2) and
// P = d_axis c + d4 c^2, c = (xi - u)/sqrt(T)
template <typename TC> struct TabE {
    TC g, p;
};

template <typename TC> struct StepSmem {
    int32_t src[2][24];
    TC w[2][24];
    int cnt[2][8];
    long long soff[2][6];  // element offset of each list's first source, wall flip folded in
    int xmask[2];          // lists with more than one source
    TC invh[2];
    TC red[2][MAXCW][7];
    TabE<TC> tab[2][3][NAX];
    TC coef[2][CF_N];
    int ok[2];
};

template <typename TC> struct Consts {
    using N = Num<TC>;
    using X = typename N::X;
    X dV, hh[3], hh2[3], third, c15, one;
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

template <typename TS> constexpr size_t step_dyn_smem(int nv) { return (size_t)NTILE * nv * sizeof(TS); }

// Solver state of one cell between its two halves, in shared memory (one
// slot per solver warp) so that it does not occupy registers across the
// loop: moments, the Maxwellian's prefactor and per-axis sums, and for node
// i of each axis c_i and exp(-c_i^2/2).
template <typename TC> struct Half {
    using X = typename Num<TC>::X;
    X rho, ux, uy, uz, T, Kc, KdV;
    X G0[3], G2[3];
    TC G1[3], G3[3], G4[3];
    TC cl[3][NAX], gl[3][NAX];
    int flags;
};

template <typename TS, int DIM, int COLL>
__global__ void __launch_bounds__(MAXT, 1) k_step(const StepParams p)
{
    using S = Store<TS>;
    using IO = QIO<TS>;
    using TC = typename S::TC;
    using N = Num<TC>;
    using X = typename N::X;
    using Q4 = QV<TC>;
    constexpr int VEC = S::VEC;

    __shared__ StepSmem<TC> sm;
    __shared__ __align__(8) uint64_t bar[NTILE];
    __shared__ int abort_flag;
    __shared__ int64_t cellq[NCQ];  // cell of pipeline iteration j at j % NCQ (-1: none left)
    extern __shared__ __align__(128) unsigned char dsm[];
    TS *tiles = reinterpret_cast<TS *>(dsm);  // [NTILE][nv]: own f of cell j, then its f*, at j % NTILE
    auto tile_of = [&](int64_t j) { return tiles + (size_t)(j % NTILE) * p.nv; };

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int ncw = (blockDim.x >> 5) - 2;  // compute warps; the last two warps solve
    const bool solver = warp >= ncw;
    const int Q = p.P / VEC;

    // ---- stencil of one cell (solver warps): fetched into registers early,
    // stored to a shared slot later so that its latency overlaps
    struct Sten {
        int32_t src;
        TC w;
        int cnt;
        TC invh;
    };
    auto fetch_stencil = [&](int64_t cell) {
        Sten s{0, (TC)0, 0, (TC)0};
        if (cell >= 0) {
            if (lane < 24) {
                s.src = p.st_src[cell * 24 + lane];
                s.w = static_cast<const TC *>(p.st_w)[cell * 24 + lane];
            }
            if (lane < 6) s.cnt = p.st_cnt[cell * 8 + lane];
            if (lane == 0) s.invh = static_cast<const TC *>(p.inv_h)[cell];
        }
        return s;
    };
    auto store_stencil = [&](const Sten &s, int slot) {
        if (lane < 24) {
            sm.src[slot][lane] = s.src;
            sm.w[slot][lane] = s.w;
        }
        if (lane < 6) sm.cnt[slot][lane] = s.cnt;
        const int32_t first = __shfl_sync(0xffffffffu, s.src, (lane & 7) * 4);
        if (lane < 6) {
            // group o reads source group o ^ flip = o -/+ flip for the minus/plus list
            const long long flip = first >> 28;
            sm.soff[slot][lane] = (long long)(first & 0x0fffffff) * p.nv + ((lane & 1) ? flip : -flip) * p.P;
        }
        const unsigned xm = __ballot_sync(0xffffffffu, lane < 6 && s.cnt > 1);
        if (lane == 0) {
            sm.xmask[slot] = (int)xm;
            sm.invh[slot] = s.invh;
        }
    };
    const uint32_t tile_bytes = (uint32_t)p.nv * (uint32_t)sizeof(TS);
    const TS *__restrict__ fin = static_cast<const TS *>(p.f_in);
    TS *__restrict__ fout = static_cast<TS *>(p.f_out);
    // lane 0 of the first solver warp: bulk copy of the own f of iteration j
    auto issue_copy = [&](int64_t j) {
        const int64_t cell = cellq[j % NCQ];
        if (cell < 0) return;
        const int t = (int)(j % NTILE);
        mbar_expect_tx(&bar[t], tile_bytes);
        bulk_g2s(tiles + (size_t)t * p.nv, fin + cell * (int64_t)p.nv, tile_bytes, &bar[t]);
    };
    auto take = [&](int64_t c) -> int64_t { return c < p.ncells ? c : -1; };
    // next cell index from the global counter, fetched one iteration before
    // it is recorded (lane 0 of the first solver warp)
    int64_t pending = 0;
    if (tid == 0) {
        for (int t = 0; t < NTILE; t++) mbar_init(&bar[t], 1);
        abort_flag = 0;
        mbar_fence_init();
    }
    __syncthreads();
    if (warp == ncw && lane == 0) {
        // cells of iterations 0..2; the own f of iteration 0
        for (int j = 0; j < 3; j++) cellq[j] = take((int64_t)atomicAdd(p.counter, 1ull));
        pending = (int64_t)atomicAdd(p.counter, 1ull);
        issue_copy(0);
    }
    __syncwarp();
    if (warp == ncw) store_stencil(fetch_stencil(cellq[0]), 0);

    // ---- per-thread position (compute warps)
    const bool active = !solver && tid < Q;
    const int hz = p.half[2], hyy = p.half[1], hxx = p.half[0];
    const int p0 = active ? tid * VEC : 0;
    const int mz0 = p0 % hz, my = (p0 / hz) % hyy, mx = p0 / (hz * hyy);
    TC ax, ay, azv[VEC];
    if constexpr (sizeof(TC) == 8) {
        ax = p.amag[mx];
        ay = p.amag[32 + my];
#pragma unroll
        for (int e = 0; e < VEC; e++) azv[e] = p.amag[64 + mz0 + e];
    } else {
        ax = p.amag_f[mx];
        ay = p.amag_f[32 + my];
#pragma unroll
        for (int e = 0; e < VEC; e++) azv[e] = p.amag_f[64 + mz0 + e];
    }
    const TC jx = (TC)(2 * mx + 1), jy = (TC)(2 * my + 1);
    const TC dt = (TC)p.dt;
    // dt |xi_d| per axis and their sum (the self coefficient is 1 - invh * sum)
    const TC dax = dt * ax, day = dt * ay;
    Q4 daz, dsum;
    {
        TC t[VEC], s[VEC];
#pragma unroll
        for (int e = 0; e < VEC; e++) {
            t[e] = dt * azv[e];
            s[e] = DIM == 3 ? dax + day + t[e] : dax + day;
        }
        daz = q_make(t);
        dsum = q_make(s);
    }
    // solver lanes: the velocity of node `lane` of each axis
    TC xil[3] = {0, 0, 0};
    if (solver) {
#pragma unroll
        for (int d = 0; d < 3; d++) {
            const int hd = p.half[d];
            if (lane < p.n[d]) {
                const int mm = lane < hd ? hd - 1 - lane : lane - hd;
                TC xi;
                if constexpr (sizeof(TC) == 8) xi = p.amag[d * 32 + mm];
                else xi = p.amag_f[d * 32 + mm];
                xil[d] = lane < hd ? -xi : xi;
            }
        }
    }

    // ---- solver constants, split once into shared memory
    __shared__ Consts<TC> K;
    if (warp == ncw && lane == 0) {
        K.dV = split<TC>(p.dV);
        for (int d = 0; d < 3; d++) {
            K.hh[d] = split<TC>(0.5 * p.hv[d]);
            K.hh2[d] = split<TC>(0.25 * p.hv[d] * p.hv[d]);
        }
        K.third = split<TC>(1.0 / 3.0);
        K.c15 = split<TC>(0.06349363593424097);  // (2 pi)^(-3/2)
        K.one = split<TC>(1.0);
    }
    __syncthreads();

    __shared__ Half<TC> halves[2];
    for (int64_t it = 0;; it++) {
        const int64_t cell = cellq[it % NCQ];                              // c_i
        const int64_t prev = it >= 1 ? cellq[(it - 1) % NCQ] : -1;         // c_{i-1}: first half
        const int64_t prev2 = it >= 2 ? cellq[(it - 2) % NCQ] : -1;        // c_{i-2}: second half, phase 3
        if (cell < 0 && prev < 0 && prev2 < 0) break;
        const int b = (int)(it & 1), bp = b ^ 1;

        if (!solver) {
            // ================= phase 1: transport of c_i into its tile
            if (cell >= 0) {
                // per-cell coefficients: f* = cs f + sum_d aw_L src_L
                const TC invh = sm.invh[b];
                const Q4 cs = q_fma(q_splat(-invh), dsum, q_splat((TC)1));
                TC aw[4];
                Q4 awz[2];
#pragma unroll
                for (int L = 0; L < 4; L++) aw[L] = (L < 2 ? dax : day) * sm.w[b][L * 4];
                if constexpr (DIM == 3) {
                    awz[0] = q_mul(daz, q_splat(sm.w[b][16]));
                    awz[1] = q_mul(daz, q_splat(sm.w[b][20]));
                }
                const TS *base[2 * DIM];
#pragma unroll
                for (int L = 0; L < 2 * DIM; L++) base[L] = fin + sm.soff[b][L] + p0;
                const int xm = sm.xmask[b];
                // first upwind source of every axis for group o: these loads do
                // not depend on the tile, so two groups are in flight before
                // the tile is awaited and one more is issued per group
                auto load_first = [&](int o, Q4 (&nb)[3]) {
#pragma unroll
                    for (int d = 0; d < DIM; d++) nb[d] = IO::ldg(base[list_of(o, d)] + o * p.P);
                };
                Q4 nbA[3], nbB[3];
                Q4 T0 = q_splat((TC)0), Tz = q_splat((TC)0);
                TC Sx = 0, Sy = 0;
                if (active) {
                    load_first(0, nbA);
                    load_first(1, nbB);
                }
                if (!mbar_wait(&bar[it % NTILE], (uint32_t)(it / NTILE) & 1u)) abort_flag = 1;
                if (active) {
                    TS *own = tile_of(it);
#pragma unroll
                    for (int o = 0; o < 8; o++) {
                        Q4 (&cur)[3] = (o & 1) ? nbB : nbA;
                        const int off = o * p.P + p0;
                        Q4 fs = q_mul(cs, IO::lds(own + off));
#pragma unroll
                        for (int d = 0; d < DIM; d++) {
                            const int L = list_of(o, d);
                            const Q4 w = d < 2 ? q_splat(aw[L]) : awz[L - 4];
                            fs = q_fma(w, cur[d], fs);
                        }
                        if (xm & lists_of<DIM>(o)) {
                            // further sources: the fine neighbours behind a coarse face
#pragma unroll 1
                            for (int d = 0; d < DIM; d++) {
                                const int L = list_of(o, d);
                                const Q4 da = d == 0 ? q_splat(dax) : (d == 1 ? q_splat(day) : daz);
                                for (int q = 1; q < sm.cnt[b][L]; q++) {
                                    const int32_t src = sm.src[b][L * 4 + q];
                                    const Q4 v = IO::ldg(fin + (int64_t)(src & 0x0fffffff) * p.nv +
                                                         (o ^ (src >> 28)) * p.P + p0);
                                    fs = q_fma(q_mul(da, q_splat(sm.w[b][L * 4 + q])), v, fs);
                                }
                            }
                        }
                        if (o + 2 < 8) load_first(o + 2, cur);
                        IO::sts(own + off, fs);
                        T0 = q_add(T0, fs);
                        Tz = q_add(Tz, (o & 1) ? fs : q_neg(fs));
                        const TC qs = q_sum(fs);
                        Sx += (o & 4) ? qs : -qs;
                        Sy += (o & 2) ? qs : -qs;
                    }
                }
                // seven integer-weighted partial sums of this thread:
                // sum f, sum s_x j_x f, sum s_y j_y f, sum s_z j_z f, sum j_x^2 f,
                // sum j_y^2 f, sum j_z^2 f  (xi_d = (h_d/2) s_d j_d, j_d odd)
                TC jz[VEC], jz2[VEC];
#pragma unroll
                for (int e = 0; e < VEC; e++) {
                    jz[e] = (TC)(2 * (mz0 + e) + 1);
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
#pragma unroll
                for (int k = 0; k < 7; k++) {
#pragma unroll
                    for (int off = 16; off > 0; off >>= 1) m[k] += __shfl_down_sync(0xffffffffu, m[k], off);
                    if (lane == 0) sm.red[b][warp][k] = m[k];
                }
            }
        } else if (warp - ncw == (int)(it & 1)) {
            // ================= solver, second half of c_{i-2} (this warp took
            // its first half in the previous iteration), and the stencil of
            // c_{i+1}
            const Sten nst = fetch_stencil(cellq[(it + 1) % NCQ]);
            const Half<TC> &hf = halves[warp - ncw];
            if (prev2 >= 0) {
                int flags = hf.flags;
                if (COLL == DVM_COLL_BGK && flags == 0) {
                    if (lane == 0) {
                        // moments of M in the centred basis; defects in double-float
                        const X P0 = hf.G0[0] * hf.G0[1] * hf.G0[2];
                        const X Q2 = hf.G2[0] * hf.G0[1] * hf.G0[2] + hf.G0[0] * hf.G2[1] * hf.G0[2] +
                                     hf.G0[0] * hf.G0[1] * hf.G2[2];
                        const TC r0 = N::tc(hf.rho - hf.KdV * P0);
                        const TC b04 = N::tc(hf.KdV * (Q2 - P0 - P0 - P0));
                        const TC k = N::tc(hf.KdV);
                        const TC *G1 = hf.G1, *G3 = hf.G3, *G4 = hf.G4;
                        TC g0[3], g2[3];
#pragma unroll
                        for (int d = 0; d < 3; d++) { g0[d] = N::tc(hf.G0[d]); g2[d] = N::tc(hf.G2[d]); }
                        const TC p0v = g0[0] * g0[1] * g0[2];
                        TC A[25], rhs[5], dd[5];
                        A[0] = N::tc(hf.KdV * P0);
                        A[1] = k * G1[0] * g0[1] * g0[2];
                        A[2] = k * g0[0] * G1[1] * g0[2];
                        A[3] = k * g0[0] * g0[1] * G1[2];
                        A[4] = b04;
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
                        rhs[0] = r0;
                        rhs[1] = -A[1];
                        rhs[2] = -A[2];
                        rhs[3] = -A[3];
                        rhs[4] = -b04;
                        if (!solve5<TC>(A, rhs, dd)) flags |= ST_SINGULAR;
                        const TC rhot = N::tc(hf.rho), Tt = N::tc(hf.T);
                        const TC nudt = (TC)(1.5957691216057308 * p.dt / p.kn) * rhot * sqrt(Tt);
                        if (nudt > (TC)1) flags |= ST_NUDT;
                        TC *cf = sm.coef[b];
                        cf[CF_KN] = nudt * N::tc(hf.Kc);
                        cf[CF_C0] = (TC)1 + dd[0] - (TC)3 * dd[4];
                        cf[CF_OMN] = (TC)1 - nudt;
                        cf[CF_DX] = dd[1];
                        cf[CF_DY] = dd[2];
                        cf[CF_DZ] = dd[3];
                        cf[CF_D4] = dd[4];
                    }
                    __syncwarp();
                    // per-axis factors of the corrected Maxwellian
                    const TC d4 = sm.coef[b][CF_D4];
#pragma unroll
                    for (int d = 0; d < 3; d++)
                        if (lane < p.n[d])
                            sm.tab[b][d][lane] =
                                TabE<TC>{hf.gl[d][lane], hf.cl[d][lane] * (sm.coef[b][CF_DX + d] + d4 * hf.cl[d][lane])};
                }
                if (lane == 0) {
                    double *mo = p.mom_out + prev2 * 5;
                    if constexpr (sizeof(TC) == 4) {
                        mo[0] = (double)hf.rho.hi + (double)hf.rho.lo;
                        mo[1] = (double)hf.ux.hi + (double)hf.ux.lo;
                        mo[2] = (double)hf.uy.hi + (double)hf.uy.lo;
                        mo[3] = (double)hf.uz.hi + (double)hf.uz.lo;
                        mo[4] = (double)hf.T.hi + (double)hf.T.lo;
                    } else {
                        mo[0] = (double)hf.rho;
                        mo[1] = (double)hf.ux; mo[2] = (double)hf.uy; mo[3] = (double)hf.uz;
                        mo[4] = (double)hf.T;
                    }
                    if (flags) atomicOr(p.status, flags);
                    sm.ok[b] = COLL == DVM_COLL_BGK && (flags & (ST_NONPOS | ST_SINGULAR)) == 0;
                }
            }
            // the stencil of c_{i+1} into the slot phase 1 of c_{i-1} has released
            store_stencil(nst, bp);
        } else {
            // ================= solver, first half of c_{i-1}: moments, the
            // Maxwellian's per-axis sums
            Half<TC> &hf = halves[warp - ncw];
            if (prev >= 0) {
                X Ssum[7];
#pragma unroll
                for (int k = 0; k < 7; k++) {
                    Ssum[k] = N::make(lane < ncw ? sm.red[bp][lane][k] : (TC)0);
#pragma unroll
                    for (int m = 16; m > 0; m >>= 1) Ssum[k] = Ssum[k] + N::shfl_xor(Ssum[k], m);
                }
                const X s0 = Ssum[0];
                const X rho = s0 * K.dV;
                const X inv = K.one / s0;
                const X ux = Ssum[1] * inv * K.hh[0];
                const X uy = Ssum[2] * inv * K.hh[1];
                const X uz = Ssum[3] * inv * K.hh[2];
                const X e2 = (Ssum[4] * K.hh2[0] + Ssum[5] * K.hh2[1] + Ssum[6] * K.hh2[2]) * inv;
                const X T = (e2 - (ux * ux + uy * uy + uz * uz)) * K.third;
                int flags = 0;
                if (!N::finite_pos(s0) || !N::finite_pos(T) || !isfinite(N::f(ux) + N::f(uy) + N::f(uz)))
                    flags |= ST_NONPOS;
                // lane 0's verdict for the whole warp (the lanes' double-float
                // sums may differ in their last bits)
                flags = __shfl_sync(0xffffffffu, flags, 0);
                if (lane == 0) {
                    hf.rho = rho; hf.ux = ux; hf.uy = uy; hf.uz = uz; hf.T = T;
                    hf.flags = flags;
                }
                if (COLL == DVM_COLL_BGK && flags == 0) {
                    const TC uT[3] = {N::tc(ux), N::tc(uy), N::tc(uz)};
                    const X isT = N::rsqrt(T);
                    const TC isTt = N::tc(isT);
                    const X Kc = rho * K.c15 * isT * isT * isT;  // rho (2 pi T)^(-3/2)
                    X G0[3], G2[3];
                    TC G1[3], G3[3], G4[3];
#pragma unroll
                    for (int d = 0; d < 3; d++) {
                        G0[d] = N::make((TC)0); G2[d] = N::make((TC)0);
                        G1[d] = 0; G3[d] = 0; G4[d] = 0;
                        if (lane < p.n[d]) {
                            const TC c = (xil[d] - uT[d]) * isTt;
                            const TC g = tc_exp<TC>((TC)-0.5 * c * c);
                            hf.cl[d][lane] = c;
                            hf.gl[d][lane] = g;
                            G0[d] = N::make(g);
                            G2[d] = N::make(g) * c * c;
                            G1[d] = g * c;
                            G3[d] = G1[d] * c * c;
                            G4[d] = G3[d] * c;
                        }
#pragma unroll
                        for (int m = 16; m > 0; m >>= 1) {
                            G0[d] = G0[d] + N::shfl_xor(G0[d], m);
                            G2[d] = G2[d] + N::shfl_xor(G2[d], m);
                            G1[d] += __shfl_xor_sync(0xffffffffu, G1[d], m);
                            G3[d] += __shfl_xor_sync(0xffffffffu, G3[d], m);
                            G4[d] += __shfl_xor_sync(0xffffffffu, G4[d], m);
                        }
                    }
                    if (lane == 0) {
                        hf.Kc = Kc;
                        hf.KdV = Kc * K.dV;
#pragma unroll
                        for (int d = 0; d < 3; d++) {
                            hf.G0[d] = G0[d]; hf.G2[d] = G2[d];
                            hf.G1[d] = G1[d]; hf.G3[d] = G3[d]; hf.G4[d] = G4[d];
                        }
                    }
                }
            }
        }
        __syncthreads();
        if (abort_flag) {
            // a tile never arrived: report it, give the copy in flight (the
            // own f of c_i) a bounded time to land, stop
            if (warp == ncw && lane == 0) {
                atomicOr(p.status, ST_TIMEOUT);
                if (cell >= 0) mbar_wait(&bar[it % NTILE], (uint32_t)(it / NTILE) & 1u);
            }
            return;
        }
        if (warp == ncw && lane == 0) {
            // the tile of c_{i-3} was drained by phase 3 of the previous
            // iteration: the own f of c_{i+1} goes there; c_{i+3} is recorded
            issue_copy(it + 1);
            cellq[(it + 3) % NCQ] = take(pending);
            pending = (int64_t)atomicAdd(p.counter, 1ull);
        }

        // ================= phase 3 (compute warps): collision of c_{i-2}
        if (!solver && prev2 >= 0 && active) {
            TS *dst = fout + prev2 * (int64_t)p.nv + p0;
            const TS *src = tile_of(it - 2) + p0;
            if (sm.ok[b]) {
                const TabE<TC> *tx = sm.tab[b][0], *ty = sm.tab[b][1], *tz = sm.tab[b][2];
                const TC KN = sm.coef[b][CF_KN], C0 = sm.coef[b][CF_C0];
                const Q4 omn = q_splat(sm.coef[b][CF_OMN]);
                // z factors of the thread's nodes for both signs: gz and gz Pz
                Q4 Z1[2], Z2[2];
#pragma unroll
                for (int pz = 0; pz < 2; pz++) {
                    TC g[VEC], gp[VEC];
#pragma unroll
                    for (int e = 0; e < VEC; e++) {
                        const TabE<TC> t = tz[pz ? hz + mz0 + e : hz - 1 - mz0 - e];
                        g[e] = t.g;
                        gp[e] = t.g * t.p;
                    }
                    Z1[pz] = q_make(g);
                    Z2[pz] = q_make(gp);
                }
                // x-y factors for the four sign pairs
                TC Axy[4], Bxy[4];
#pragma unroll
                for (int s = 0; s < 4; s++) {
                    const TabE<TC> a = tx[(s & 2) ? hxx + mx : hxx - 1 - mx];
                    const TabE<TC> c = ty[(s & 1) ? hyy + my : hyy - 1 - my];
                    Bxy[s] = KN * a.g * c.g;
                    Axy[s] = Bxy[s] * (C0 + a.p + c.p);
                }
#pragma unroll
                for (int o = 0; o < 8; o++) {
                    const int off = o * p.P;
                    const Q4 fs = IO::lds(src + off);
                    const Q4 mt = q_fma(q_splat(Axy[o >> 1]), Z1[o & 1], q_mul(q_splat(Bxy[o >> 1]), Z2[o & 1]));
                    IO::stg(dst + off, q_fma(omn, fs, mt));
                }
            } else {
#pragma unroll
                for (int o = 0; o < 8; o++) IO::stg(dst + o * p.P, IO::lds(src + o * p.P));
            }
        }
        // order this thread's generic accesses to the tiles before the bulk
        // copies that will refill them
        if (!solver) fence_proxy_async();
    }
}

template <typename TS, int DIM, int COLL>
int launch_kernel(const StepParams &p, int ncw)
{
    auto kern = k_step<TS, DIM, COLL>;
    const int threads = (ncw + 2) * 32;
    const size_t dyn = step_dyn_smem<TS>(p.nv);
    cudaFuncAttributes fa{};
    if (cudaFuncGetAttributes(&fa, kern) != cudaSuccess) return DVM_ECUDA;
    int dev0 = 0, optin = 0;
    cudaGetDevice(&dev0);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev0);
    if (fa.sharedSizeBytes + dyn > (size_t)optin) return DVM_ENOTIMPL;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn) != cudaSuccess)
        return DVM_ECUDA;
    int dev = 0, nsm = 0, occ = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, threads, dyn) != cudaSuccess || occ < 1)
        return DVM_ENOTIMPL;
    const int64_t grid = std::min<int64_t>(p.ncells, (int64_t)nsm * occ);
    kern<<<(unsigned)grid, threads, dyn, p.stream>>>(p);
    count_launch();
    return cudaGetLastError() == cudaSuccess ? DVM_OK : DVM_ECUDA;
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
    if (p.coll == DVM_COLL_BGK) return launch_kernel<TS, DIM, DVM_COLL_BGK>(p, ncw);
    return launch_kernel<TS, DIM, DVM_COLL_NONE>(p, ncw);
}

}  // namespace

int launch_step(const StepParams &p)
{
    if (p.ncells <= 0) return DVM_OK;
    if (p.coll != DVM_COLL_NONE && p.coll != DVM_COLL_BGK) return DVM_ENOTIMPL;
    switch (p.prec) {
    case DVM_F64: return p.dim == 3 ? launch_typed<double, 3>(p) : launch_typed<double, 2>(p);
    case DVM_F32: return p.dim == 3 ? launch_typed<float, 3>(p) : launch_typed<float, 2>(p);
    case DVM_BF16: return p.dim == 3 ? launch_typed<__nv_bfloat16, 3>(p) : launch_typed<__nv_bfloat16, 2>(p);
    default: return DVM_EINVAL;
    }
}

}  // namespace dvm
