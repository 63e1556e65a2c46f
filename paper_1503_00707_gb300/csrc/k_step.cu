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
// Persistent CTAs take the Morton-ordered cells from a global counter, two
// cells ahead of their pipeline, so the cells in flight on the whole GPU form
// one contiguous Morton window and upwind neighbours are served from L2 (a
// fixed round-robin assignment lets the CTAs drift apart over thousands of
// cells and spreads the window far beyond L2).  Each CTA has NCW compute warps and one solver warp and
// overlaps cells in a pipeline with one barrier per cell:
//
//   iteration i, compute warps:  phase 1 of cell c_i        | barrier | phase 3 of c_{i-1}
//   iteration i, solver warp:    phase 2 of c_{i-1},        | barrier | bulk copy of c_{i+2}
//                                prefetch stencil of c_{i+1}
//
// A cell's own f arrives as one bulk copy (cp.async.bulk, completion on an
// mbarrier) into one of four shared tiles, issued two cells ahead; phase 1
// reads it from shared memory and writes f* over it in place (FP32/FP64
// storage; BF16 storage keeps f* in a separate FP32 buffer).  Only the upwind
// neighbours are read through L2.  Waits on the tiles are bounded and report
// DVM_ETIMEOUT instead of hanging.
//
// Phase 1: f*_i = f_i - dt sum_d |xi_d,i| (f_i / h - sum_k w_k src_k,i) into a
//   shared buffer; per-thread FP32 partials of the seven sums sum f,
//   sum j_d f, sum j_d^2 f (xi_d = (h_d/2) j_d with j_d an odd integer),
//   reduced per warp.
// Phase 2 (solver warp): double-float sum of the warp partials -> rho, u, T;
//   the discrete Maxwellian factorises over the tensor grid, so its moments
//   in the centred basis phi = (1, c, |c|^2 - 3), c = (xi - u)/sqrt(T), are
//   products of 1D sums; the five coefficients d of M~ = M (1 + d.phi) (the
//   correction form of Eq. 6) make M~ carry the moments of f*.  The defects
//   of M's own moments (the right-hand side) are formed in double-float.
// Phase 3: f^{n+1} = f* + nu dt (M~ - f*), nu = sqrt(8/pi) rho sqrt(T) / Kn.
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
constexpr int MAXT = MAXCW * 32 + 32;
constexpr int NTILE = 4;      // shared tiles holding cells' own f

template <typename TC> __device__ inline TC tc_exp(TC x);
template <> __device__ inline float tc_exp<float>(float x) { return expf(x); }
template <> __device__ inline double tc_exp<double>(double x) { return exp(x); }

// coefficient slots written by the solver warp for phase 3
enum { CF_PRE = 0, CF_UX, CF_UY, CF_UZ, CF_IST, CF_D0, CF_DX, CF_DY, CF_DZ, CF_D4, CF_NUDT, CF_N };

template <typename TC> struct StepSmem {
    int32_t src[2][24];
    TC w[2][24];
    int cnt[2][8];
    TC invh[2];
    TC red[2][MAXCW][7];
    TC g[2][3][NAX];
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

template <typename TS> constexpr size_t step_dyn_smem(int nv)
{
    using TC = typename Store<TS>::TC;
    return sizeof(TS) == sizeof(TC) ? (size_t)NTILE * nv * sizeof(TS)
                                    : (size_t)NTILE * nv * sizeof(TS) + 2 * (size_t)nv * sizeof(TC);
}

template <typename TS, int DIM, int COLL>
__global__ void __launch_bounds__(MAXT, 1) k_step(const StepParams p)
{
    using S = Store<TS>;
    using TC = typename S::TC;
    using N = Num<TC>;
    using X = typename N::X;
    constexpr int VEC = S::VEC;

    constexpr bool INPLACE = sizeof(TS) == sizeof(TC);
    __shared__ StepSmem<TC> sm;
    __shared__ __align__(8) uint64_t bar[NTILE];
    __shared__ int abort_flag;
    __shared__ int64_t cellq[NTILE];  // cell of pipeline iteration i at i % NTILE (-1: none left)
    extern __shared__ __align__(128) unsigned char dsm[];
    TS *tiles = reinterpret_cast<TS *>(dsm);  // [NTILE][nv] own f of upcoming cells
    TC *fsep = reinterpret_cast<TC *>(dsm + (size_t)NTILE * p.nv * sizeof(TS));  // [2][nv] (BF16 storage)
    // f* of pipeline iteration i
    auto fstar = [&](int64_t i) -> TC * {
        if constexpr (INPLACE) return reinterpret_cast<TC *>(tiles + (size_t)(i % NTILE) * p.nv);
        else return fsep + (size_t)(i & 1) * p.nv;
    };

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int ncw = (blockDim.x >> 5) - 1;  // compute warps; the last warp solves
    const bool solver = warp == ncw;
    const int Q = p.P / VEC;

    // ---- stencil prefetch (solver warp): cell -> slot
    auto load_stencil = [&](int64_t cell, int slot) {
        if (lane < 24) {
            sm.src[slot][lane] = p.st_src[cell * 24 + lane];
            sm.w[slot][lane] = static_cast<const TC *>(p.st_w)[cell * 24 + lane];
        }
        if (lane < 6) sm.cnt[slot][lane] = p.st_cnt[cell * 8 + lane];
        if (lane == 0) sm.invh[slot] = static_cast<const TC *>(p.inv_h)[cell];
    };
    const uint32_t tile_bytes = (uint32_t)p.nv * (uint32_t)sizeof(TS);
    const TS *__restrict__ fin_all = static_cast<const TS *>(p.f_in);
    // solver lane 0: take the next cell for pipeline iteration i and start the
    // bulk copy of its own f into tile i % NTILE
    auto issue = [&](int64_t i) {
        const int t = (int)(i % NTILE);
        const int64_t cell = (int64_t)atomicAdd(p.counter, 1ull);
        if (cell >= p.ncells) {
            cellq[t] = -1;
            return;
        }
        cellq[t] = cell;
        mbar_expect_tx(&bar[t], tile_bytes);
        bulk_g2s(tiles + (size_t)t * p.nv, fin_all + cell * (int64_t)p.nv, tile_bytes, &bar[t]);
    };
    if (tid == 0) {
        for (int t = 0; t < NTILE; t++) mbar_init(&bar[t], 1);
        abort_flag = 0;
        mbar_fence_init();
    }
    __syncthreads();
    if (solver) {
        if (lane == 0) {
            issue(0);
            issue(1);
        }
        __syncwarp();
        if (cellq[0] >= 0) load_stencil(cellq[0], 0);
    }

    // ---- per-thread position (compute warps)
    const bool active = !solver && tid < Q;
    const int hz = p.half[2], hyy = p.half[1], hxx = p.half[0];
    const int p0 = active ? tid * VEC : 0;
    const int mz0 = p0 % hz, my = (p0 / hz) % hyy, mx = p0 / (hz * hyy);
    TC ax, ay, az[VEC];
    if constexpr (sizeof(TC) == 8) {
        ax = p.amag[mx];
        ay = p.amag[32 + my];
#pragma unroll
        for (int e = 0; e < VEC; e++) az[e] = p.amag[64 + mz0 + e];
    } else {
        ax = p.amag_f[mx];
        ay = p.amag_f[32 + my];
#pragma unroll
        for (int e = 0; e < VEC; e++) az[e] = p.amag_f[64 + mz0 + e];
    }
    const TC jx = (TC)(2 * mx + 1), jy = (TC)(2 * my + 1);
    const TS *__restrict__ fin = static_cast<const TS *>(p.f_in);
    TS *__restrict__ fout = static_cast<TS *>(p.f_out);
    const TC dt = (TC)p.dt;

    // ---- solver constants, split once into shared memory
    __shared__ Consts<TC> K;
    if (solver && lane == 0) {
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

    for (int64_t it = 0;; it++) {
        const int b = (int)(it & 1), bp = b ^ 1;
        const int64_t cell = cellq[it % NTILE];                          // c_i, or -1
        const int64_t prev = it >= 1 ? cellq[(it - 1) % NTILE] : -1;     // c_{i-1}, or -1
        if (cell < 0 && prev < 0) break;

        if (!solver) {
            // ================= phase 1: transport of c_i into its tile
            if (cell >= 0) {
                // per-thread partials: sum f, sum s_x f, sum s_y f, sum j_z s_z f, sum j_z^2 f
                TC a0 = 0, ax1 = 0, ay1 = 0, az1 = 0, az2 = 0;
                const int tl = (int)(it % NTILE);
                // first upwind source of every axis for group o: these loads do
                // not depend on the tile, so two groups are in flight before
                // the tile is awaited and one more is issued per group
                auto load_first = [&](int o, TC (&nb)[3][VEC]) {
#pragma unroll
                    for (int d = 0; d < DIM; d++) {
                        const int list = 2 * d + (((o >> (2 - d)) & 1) ? 0 : 1);
                        const int32_t src = sm.src[b][list * 4];
                        S::load(fin + (int64_t)(src & 0x0fffffff) * p.nv + (o ^ (src >> 28)) * p.P + p0, nb[d]);
                    }
                };
                TC nbA[3][VEC], nbB[3][VEC];
                if (active) {
                    load_first(0, nbA);
                    load_first(1, nbB);
                }
                if (!mbar_wait(&bar[tl], (uint32_t)(it / NTILE) & 1u)) abort_flag = 1;
                if (active) {
                    const TC invh = sm.invh[b];
                    const TS *own = tiles + (size_t)tl * p.nv;
                    TC *bb = fstar(it);
#pragma unroll
                    for (int o = 0; o < 8; o++) {
                        TC (&cur)[3][VEC] = (o & 1) ? nbB : nbA;
                        const int off = o * p.P + p0;
                        TC self[VEC], acc[VEC];
                        S::load_shared(own + off, self);
#pragma unroll
                        for (int e = 0; e < VEC; e++) acc[e] = 0;
#pragma unroll
                        for (int d = 0; d < DIM; d++) {
                            const int list = 2 * d + (((o >> (2 - d)) & 1) ? 0 : 1);
                            TC sd[VEC];
                            const TC w0 = sm.w[b][list * 4];
#pragma unroll
                            for (int e = 0; e < VEC; e++) sd[e] = w0 * cur[d][e];
                            // further sources: the fine neighbours behind a coarse face
                            const int cnt = sm.cnt[b][list];
                            for (int q = 1; q < cnt; q++) {
                                const int32_t src = sm.src[b][list * 4 + q];
                                const TC w = sm.w[b][list * 4 + q];
                                TC v[VEC];
                                S::load(fin + (int64_t)(src & 0x0fffffff) * p.nv + (o ^ (src >> 28)) * p.P + p0, v);
#pragma unroll
                                for (int e = 0; e < VEC; e++) sd[e] = fma(w, v[e], sd[e]);
                            }
#pragma unroll
                            for (int e = 0; e < VEC; e++) {
                                const TC a = d == 0 ? ax : (d == 1 ? ay : az[e]);
                                acc[e] = fma(a, fma(self[e], invh, -sd[e]), acc[e]);
                            }
                        }
                        if (o + 2 < 8) load_first(o + 2, cur);
                        TC fs[VEC], r0 = 0, r1 = 0, r2 = 0;
#pragma unroll
                        for (int e = 0; e < VEC; e++) {
                            fs[e] = fma(-dt, acc[e], self[e]);
                            const TC jz = (TC)(2 * (mz0 + e) + 1);
                            r0 += fs[e];
                            r1 = fma(jz, fs[e], r1);
                            r2 = fma(jz * jz, fs[e], r2);
                        }
                        a0 += r0;
                        ax1 += (o & 4) ? r0 : -r0;
                        ay1 += (o & 2) ? r0 : -r0;
                        az1 += (o & 1) ? r1 : -r1;
                        az2 += r2;
                        if constexpr (VEC == 4)
                            *reinterpret_cast<float4 *>(bb + off) = make_float4(fs[0], fs[1], fs[2], fs[3]);
                        else
                            *reinterpret_cast<double2 *>(bb + off) = make_double2(fs[0], fs[1]);
                    }
                }
                // seven integer-weighted partial sums of this thread
                TC m[7];
                m[0] = a0;
                m[1] = jx * ax1;
                m[2] = jy * ay1;
                m[3] = az1;
                m[4] = jx * jx * a0;
                m[5] = jy * jy * a0;
                m[6] = az2;
#pragma unroll
                for (int k = 0; k < 7; k++) {
#pragma unroll
                    for (int off = 16; off > 0; off >>= 1) m[k] += __shfl_down_sync(0xffffffffu, m[k], off);
                    if (lane == 0) sm.red[b][warp][k] = m[k];
                }
            }
        } else {
            // ================= phase 2 (solver warp): cell c_{i-1}
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
                const TC uT[3] = {N::tc(ux), N::tc(uy), N::tc(uz)};
                if (COLL == DVM_COLL_BGK && flags == 0) {
                    const X isT = N::rsqrt(T);
                    const TC isTt = N::tc(isT);
                    const X Kc = rho * K.c15 * isT * isT * isT;  // rho (2 pi T)^(-3/2)
                    const X KdV = Kc * K.dV;
                    X G0[3], G2[3];
                    TC G1[3], G3[3], G4[3];
#pragma unroll
                    for (int d = 0; d < 3; d++) {
                        G0[d] = N::make((TC)0); G2[d] = N::make((TC)0);
                        G1[d] = 0; G3[d] = 0; G4[d] = 0;
                        const int hd = p.half[d];
                        if (lane < p.n[d]) {
                            const int mm = lane < hd ? hd - 1 - lane : lane - hd;
                            TC xi;
                            if constexpr (sizeof(TC) == 8) xi = p.amag[d * 32 + mm];
                            else xi = p.amag_f[d * 32 + mm];
                            if (lane < hd) xi = -xi;
                            const TC c = (xi - uT[d]) * isTt;
                            const TC g = tc_exp<TC>((TC)-0.5 * c * c);
                            sm.g[bp][d][lane] = g;
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
                        // moments of M in the centred basis; defects in double-float
                        const X P0 = G0[0] * G0[1] * G0[2];
                        const X Q2 = G2[0] * G0[1] * G0[2] + G0[0] * G2[1] * G0[2] + G0[0] * G0[1] * G2[2];
                        const TC r0 = N::tc(rho - KdV * P0);
                        const TC b04 = N::tc(KdV * (Q2 - P0 - P0 - P0));
                        const TC k = N::tc(KdV);
                        TC g0[3], g2[3];
                        for (int d = 0; d < 3; d++) { g0[d] = N::tc(G0[d]); g2[d] = N::tc(G2[d]); }
                        const TC p0v = g0[0] * g0[1] * g0[2];
                        TC A[25], rhs[5], dd[5];
                        A[0] = N::tc(KdV * P0);
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
                        const TC rhot = N::tc(rho), Tt = N::tc(T);
                        const TC nudt = (TC)(1.5957691216057308 * p.dt / p.kn) * rhot * sqrt(Tt);
                        if (nudt > (TC)1) flags |= ST_NUDT;
                        TC *cf = sm.coef[bp];
                        cf[CF_PRE] = N::tc(Kc);
                        cf[CF_UX] = uT[0]; cf[CF_UY] = uT[1]; cf[CF_UZ] = uT[2];
                        cf[CF_IST] = isTt;
                        cf[CF_D0] = dd[0]; cf[CF_DX] = dd[1]; cf[CF_DY] = dd[2]; cf[CF_DZ] = dd[3];
                        cf[CF_D4] = dd[4];
                        cf[CF_NUDT] = nudt;
                    }
                }
                if (lane == 0) {
                    double *mo = p.mom_out + prev * 5;
                    mo[0] = (double)N::tc(rho);
                    mo[1] = (double)N::tc(ux); mo[2] = (double)N::tc(uy); mo[3] = (double)N::tc(uz);
                    mo[4] = (double)N::tc(T);
                    if constexpr (sizeof(TC) == 4) {
                        mo[0] = (double)rho.hi + (double)rho.lo;
                        mo[1] = (double)ux.hi + (double)ux.lo;
                        mo[2] = (double)uy.hi + (double)uy.lo;
                        mo[3] = (double)uz.hi + (double)uz.lo;
                        mo[4] = (double)T.hi + (double)T.lo;
                    }
                    if (flags) atomicOr(p.status, flags);
                    sm.ok[bp] = COLL == DVM_COLL_BGK && (flags & (ST_NONPOS | ST_SINGULAR)) == 0;
                }
            }
            // prefetch the stencil of c_{i+1} (its cell was taken by lane 0 two
            // iterations ago)
            __syncwarp();
            const int64_t next = cellq[(it + 1) % NTILE];
            if (next >= 0) load_stencil(next, bp);
        }
        __syncthreads();
        if (abort_flag) {
            // a tile never arrived: report it, give the copies in flight
            // (cells it and it+1 at most) a bounded time to land, stop
            if (solver && lane == 0) {
                atomicOr(p.status, ST_TIMEOUT);
                for (int64_t i = it; i <= it + 1; i++)
                    if (cellq[i % NTILE] >= 0) mbar_wait(&bar[i % NTILE], (uint32_t)(i / NTILE) & 1u);
            }
            return;
        }
        // the tile of c_{i-2} was drained by phase 3 of the previous iteration
        if (solver && lane == 0) issue(it + 2);

        // ================= phase 3 (compute warps): collision of c_{i-1}
        if (!solver && prev >= 0 && active) {
            const int64_t cbase = prev * (int64_t)p.nv;
            const TC *bb = fstar(it - 1);
            const bool collide = sm.ok[bp];
            const TC *cf = sm.coef[bp];
            const TC pre = cf[CF_PRE], ux = cf[CF_UX], uy = cf[CF_UY], uz = cf[CF_UZ], ist = cf[CF_IST];
            const TC d0 = cf[CF_D0], dx = cf[CF_DX], dy = cf[CF_DY], dz = cf[CF_DZ], d4 = cf[CF_D4];
            const TC nudt = cf[CF_NUDT];
#pragma unroll
            for (int o = 0; o < 8; o++) {
                const int off = o * p.P + p0;
                TC fs[VEC], out[VEC];
                if constexpr (VEC == 4) {
                    const float4 t = *reinterpret_cast<const float4 *>(bb + off);
                    fs[0] = t.x; fs[1] = t.y; fs[2] = t.z; fs[3] = t.w;
                } else {
                    const double2 t = *reinterpret_cast<const double2 *>(bb + off);
                    fs[0] = t.x; fs[1] = t.y;
                }
                if (collide) {
                    const bool px = o & 4, py = o & 2, pz = o & 1;
                    const TC cx = ((px ? ax : -ax) - ux) * ist, cy = ((py ? ay : -ay) - uy) * ist;
                    const int kx = px ? hxx + mx : hxx - 1 - mx;
                    const int ky = py ? hyy + my : hyy - 1 - my;
                    const TC cxy = pre * sm.g[bp][0][kx] * sm.g[bp][1][ky];
                    const TC pxy = (TC)1 + d0 + dx * cx + dy * cy + d4 * (cx * cx + cy * cy - (TC)3);
#pragma unroll
                    for (int e = 0; e < VEC; e++) {
                        const TC cz = ((pz ? az[e] : -az[e]) - uz) * ist;
                        const int kz = pz ? hz + mz0 + e : hz - 1 - mz0 - e;
                        const TC mt = cxy * sm.g[bp][2][kz] * (pxy + dz * cz + d4 * cz * cz);
                        out[e] = fma(nudt, mt - fs[e], fs[e]);
                    }
                } else {
#pragma unroll
                    for (int e = 0; e < VEC; e++) out[e] = fs[e];
                }
                S::store(fout + cbase + off, out);
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
    const int threads = (ncw + 1) * 32;
    const size_t dyn = step_dyn_smem<TS>(p.nv);
    if (dyn > 220 * 1024) return DVM_ENOTIMPL;
    static bool configured = false;
    if (!configured) {
        if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024) != cudaSuccess)
            return DVM_ECUDA;
        configured = true;
    }
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
