// Fused DVM step: upwind transport (Eq. 2) -> moments of f* -> conservative
// BGK relaxation, one CTA per cell, f* kept in registers between the phases.
//
// Layout (paper Sec. 3.1 steps 1-3): f[cell][group][position], 8 sign groups
// per cell.  Thread t of a cell owns the same "quad" of positions (4 FP32 /
// BF16 or 2 FP64 values along z) in all 8 groups, so every warp reads 32
// consecutive quads of one group (coalesced 16-byte loads) and the stencil
// of Eq. 2 is uniform across the warp: it depends on the group only through
// the signs of the velocity components (Sec. 3.1).
//
// Phase 1: f*_i = f_i - dt sum_d |xi_d,i| (f_i / h - sum_k w_k src_k,i) with
//   the upwind sources of the cell's side facing the incoming velocity.
// Phase 2: the seven sums sum f, sum j_d f, sum j_d^2 f (j_d the odd integer
//   with xi_d = (h_d/2) j_d) in FP32 per thread, double-float across threads,
//   FP64 at the end -> rho, u, T.
// Phase 3 (warp 0): the discrete Maxwellian factorises over the tensor grid,
//   so the 5x5 moment matrix sum psi_r psi_s M dV comes from 1D sums of the
//   per-axis factors (FP64); Gauss with pivoting gives d of the correction
//   polynomial (the Eq. 6 form) that makes M~ = M (1 + d.psi) carry the
//   moments of f*.
// Phase 4: f^{n+1} = f* + nu dt (M~ - f*), nu = sqrt(8/pi) rho sqrt(T) / Kn.
#include <atomic>
#include <cmath>

#include "../../include/dvm.h"
#include "common.cuh"
#include "kernels.hpp"
#include "mesh.hpp"

namespace dvm {

static std::atomic<int64_t> g_launches{0};
int64_t launches_issued() { return g_launches.load(); }
void count_launch() { g_launches.fetch_add(1); }

namespace {

constexpr int MAXT = 512;
constexpr int NAX = 64;  // nodes per velocity axis supported

template <typename TC> __device__ inline TC tc_exp(TC x);
template <> __device__ inline float tc_exp<float>(float x) { return expf(x); }
template <> __device__ inline double tc_exp<double>(double x) { return exp(x); }

template <typename TS, int DIM, int COLL>
__global__ void __launch_bounds__(MAXT, 2) k_step(const StepParams p)
{
    using S = Store<TS>;
    using TC = typename S::TC;
    using R = Red<TC>;
    using RT = typename R::T;
    constexpr int VEC = S::VEC;

    __shared__ int32_t s_src[24];
    __shared__ TC s_w[24];
    __shared__ int s_cnt[6];
    __shared__ TC s_g[3][NAX];
    __shared__ RT s_red[MAXT / 32][7];
    __shared__ TC s_coef[7];
    __shared__ int s_ok;

    const int64_t cell = blockIdx.x;
    const int t = threadIdx.x;
    const int Q = p.P / VEC;
    const bool active = t < Q;
    if (t < 24) {
        s_src[t] = p.st_src[cell * 24 + t];
        s_w[t] = static_cast<const TC *>(p.st_w)[cell * 24 + t];
    }
    if (t < 6) s_cnt[t] = p.st_cnt[cell * 8 + t];
    const TC invh = static_cast<const TC *>(p.inv_h)[cell];
    __syncthreads();

    const int hz = p.half[2], hy = p.half[1];
    const int p0 = active ? t * VEC : 0;
    const int mz0 = p0 % hz, my = (p0 / hz) % hy, mx = p0 / (hz * hy);
    TC ax, ay, az[VEC], jz[VEC];
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
#pragma unroll
    for (int e = 0; e < VEC; e++) jz[e] = (TC)(2 * (mz0 + e) + 1);
    const TC jx = (TC)(2 * mx + 1), jy = (TC)(2 * my + 1);

    const TS *__restrict__ fin = static_cast<const TS *>(p.f_in);
    TS *__restrict__ fout = static_cast<TS *>(p.f_out);
    const TC *__restrict__ finf = static_cast<const TC *>(p.finf);
    const int64_t cbase = cell * (int64_t)p.nv;
    const TC dt = (TC)p.dt;

    TC fs[8][VEC];
    TC aS0 = 0, aX = 0, aY = 0, aZ1 = 0, aZ2 = 0;
#pragma unroll
    for (int o = 0; o < 8; o++) {
        const int off = o * p.P + p0;
        TC self[VEC];
#pragma unroll
        for (int e = 0; e < VEC; e++) self[e] = 0;
        TC acc[VEC];
#pragma unroll
        for (int e = 0; e < VEC; e++) acc[e] = 0;
        if (active) {
            S::load(fin + cbase + off, self);
#pragma unroll
            for (int d = 0; d < DIM; d++) {
                const int pos = (o >> (2 - d)) & 1;
                const int list = 2 * d + (pos ? 0 : 1);
                TC sd[VEC];
#pragma unroll
                for (int e = 0; e < VEC; e++) sd[e] = 0;
                const int cnt = s_cnt[list];
                for (int q = 0; q < cnt; q++) {
                    const int32_t src = s_src[list * 4 + q];
                    const TC w = s_w[list * 4 + q];
                    TC v[VEC];
                    if (src >= 0) {
                        S::load(fin + (int64_t)src * p.nv + off, v);
                    } else if (src == SRC_INFLOW) {
#pragma unroll
                        for (int e = 0; e < VEC; e++) v[e] = finf[off + e];
                    } else if (src == SRC_OUTFLOW) {
#pragma unroll
                        for (int e = 0; e < VEC; e++) v[e] = self[e];
                    } else {
                        S::load(fin + cbase + (o ^ (4 >> d)) * p.P + p0, v);
                    }
#pragma unroll
                    for (int e = 0; e < VEC; e++) sd[e] = fma(w, v[e], sd[e]);
                }
#pragma unroll
                for (int e = 0; e < VEC; e++) {
                    const TC a = d == 0 ? ax : (d == 1 ? ay : az[e]);
                    acc[e] = fma(a, fma(self[e], invh, -sd[e]), acc[e]);
                }
            }
        }
        TC r0 = 0, r1 = 0, r2 = 0;
#pragma unroll
        for (int e = 0; e < VEC; e++) {
            fs[o][e] = fma(-dt, acc[e], self[e]);
            r0 += fs[o][e];
            r1 = fma(jz[e], fs[o][e], r1);
            r2 = fma(jz[e] * jz[e], fs[o][e], r2);
        }
        aS0 += r0;
        aX += (o & 4) ? r0 : -r0;
        aY += (o & 2) ? r0 : -r0;
        aZ1 += (o & 1) ? r1 : -r1;
        aZ2 += r2;
    }

    // ---- block reduction of the seven integer-weighted sums
    RT m[7];
    m[0] = R::from(aS0);
    m[1] = R::mul(jx, aX);
    m[2] = R::mul(jy, aY);
    m[3] = R::from(aZ1);
    m[4] = R::mul(jx * jx, aS0);
    m[5] = R::mul(jy * jy, aS0);
    m[6] = R::from(aZ2);
    const int lane = t & 31, warp = t >> 5, nwarps = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int k = 0; k < 7; k++)
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) m[k] = R::add(m[k], R::shfl_down(m[k], off));
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < 7; k++) s_red[warp][k] = m[k];
    __syncthreads();

    if (warp == 0) {
        double Ssum[7];
#pragma unroll
        for (int k = 0; k < 7; k++) {
            RT v = lane < nwarps ? s_red[lane][k] : R::zero();
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) v = R::add(v, R::shfl_down(v, off));
            Ssum[k] = __shfl_sync(0xffffffffu, R::to_double(v), 0);
        }
        const double hx2 = 0.5 * p.hv[0], hy2 = 0.5 * p.hv[1], hz2 = 0.5 * p.hv[2];
        const double s0 = Ssum[0];
        const double rho = p.dV * s0;
        const double ux = hx2 * Ssum[1] / s0, uy = hy2 * Ssum[2] / s0, uz = hz2 * Ssum[3] / s0;
        const double e2 = (hx2 * hx2 * Ssum[4] + hy2 * hy2 * Ssum[5] + hz2 * hz2 * Ssum[6]) / s0;
        const double T = (e2 - (ux * ux + uy * uy + uz * uz)) / 3.0;
        int flags = 0;
        if (!(s0 > 0.0) || !(T > 0.0) || !isfinite(T) || !isfinite(ux + uy + uz)) flags |= ST_NONPOS;
        if (COLL == DVM_COLL_BGK && flags == 0) {
            const double u[3] = {ux, uy, uz};
            double m1[3][5];
#pragma unroll
            for (int d = 0; d < 3; d++)
#pragma unroll
                for (int q = 0; q < 5; q++) m1[d][q] = 0.0;
#pragma unroll
            for (int d = 0; d < 3; d++) {
                const int nd = p.n[d], hd = p.half[d];
                for (int l = lane; l < nd; l += 32) {
                    const int mm = l < hd ? hd - 1 - l : l - hd;
                    const double mag = p.amag[d * 32 + mm];
                    const double xi = l < hd ? -mag : mag;
                    const double arg = -(xi - u[d]) * (xi - u[d]) / (2.0 * T);
                    const TC g = tc_exp<TC>((TC)arg);
                    s_g[d][l] = g;
                    double pw = (double)g;
                    m1[d][0] += pw; pw *= xi;
                    m1[d][1] += pw; pw *= xi;
                    m1[d][2] += pw; pw *= xi;
                    m1[d][3] += pw; pw *= xi;
                    m1[d][4] += pw;
                }
            }
#pragma unroll
            for (int d = 0; d < 3; d++)
#pragma unroll
                for (int q = 0; q < 5; q++) m1[d][q] = warp_allsum(m1[d][q]);
            if (lane == 0) {
                const double twopiT = 2.0 * 3.14159265358979323846 * T;
                const double cn = rho / (twopiT * sqrt(twopiT));
                const double G = cn * p.dV;
                auto E = [&](int a, int b, int c) { return G * m1[0][a] * m1[1][b] * m1[2][c]; };
                double A[25], rhs[5], dd[5];
                A[0] = E(0, 0, 0);
                A[1] = E(1, 0, 0); A[2] = E(0, 1, 0); A[3] = E(0, 0, 1);
                A[4] = E(2, 0, 0) + E(0, 2, 0) + E(0, 0, 2);
                A[6] = E(2, 0, 0); A[7] = E(1, 1, 0); A[8] = E(1, 0, 1);
                A[9] = E(3, 0, 0) + E(1, 2, 0) + E(1, 0, 2);
                A[12] = E(0, 2, 0); A[13] = E(0, 1, 1);
                A[14] = E(2, 1, 0) + E(0, 3, 0) + E(0, 1, 2);
                A[18] = E(0, 0, 2);
                A[19] = E(2, 0, 1) + E(0, 2, 1) + E(0, 0, 3);
                A[24] = E(4, 0, 0) + E(0, 4, 0) + E(0, 0, 4) +
                        2.0 * (E(2, 2, 0) + E(2, 0, 2) + E(0, 2, 2));
                for (int r = 0; r < 5; r++)
                    for (int c = 0; c < r; c++) A[r * 5 + c] = A[c * 5 + r];
                const double F[5] = {rho, rho * ux, rho * uy, rho * uz,
                                     p.dV * (hx2 * hx2 * Ssum[4] + hy2 * hy2 * Ssum[5] + hz2 * hz2 * Ssum[6])};
                for (int r = 0; r < 5; r++) rhs[r] = F[r] - A[r * 5];
                if (!solve5(A, rhs, dd)) flags |= ST_SINGULAR;
                const double nudt = sqrt(8.0 / 3.14159265358979323846) * rho * sqrt(T) / p.kn * p.dt;
                if (nudt > 1.0) flags |= ST_NUDT;
                s_coef[0] = (TC)cn;
                for (int q = 0; q < 5; q++) s_coef[1 + q] = (TC)dd[q];
                s_coef[6] = (TC)nudt;
            }
        }
        if (lane == 0) {
            double *mo = p.mom_out + cell * 5;
            mo[0] = rho; mo[1] = ux; mo[2] = uy; mo[3] = uz; mo[4] = T;
            if (flags) atomicOr(p.status, flags);
            s_ok = (flags & (ST_NONPOS | ST_SINGULAR)) == 0;
        }
    }
    __syncthreads();

    if (!active) return;
    const bool collide = COLL == DVM_COLL_BGK && s_ok;
    TC cn = 0, d0 = 0, dxx = 0, dyy = 0, dzz = 0, d2 = 0, nudt = 0;
    if (collide) {
        cn = s_coef[0]; d0 = s_coef[1]; dxx = s_coef[2]; dyy = s_coef[3]; dzz = s_coef[4];
        d2 = s_coef[5]; nudt = s_coef[6];
    }
    const int hx = p.half[0], hyy = p.half[1], hzz = p.half[2];
#pragma unroll
    for (int o = 0; o < 8; o++) {
        const int off = o * p.P + p0;
        TC out[VEC];
        if (collide) {
            const bool px = o & 4, py = o & 2, pz = o & 1;
            const TC xx = px ? ax : -ax, yy = py ? ay : -ay;
            const int kx = px ? hx + mx : hx - 1 - mx;
            const int ky = py ? hyy + my : hyy - 1 - my;
            const TC cxy = cn * s_g[0][kx] * s_g[1][ky];
            const TC pxy = (TC)1 + d0 + dxx * xx + dyy * yy + d2 * (xx * xx + yy * yy);
#pragma unroll
            for (int e = 0; e < VEC; e++) {
                const TC zz = pz ? az[e] : -az[e];
                const int kz = pz ? hzz + mz0 + e : hzz - 1 - mz0 - e;
                const TC mt = cxy * s_g[2][kz] * (pxy + dzz * zz + d2 * zz * zz);
                out[e] = fma(nudt, mt - fs[o][e], fs[o][e]);
            }
        } else {
#pragma unroll
            for (int e = 0; e < VEC; e++) out[e] = fs[o][e];
        }
        S::store(fout + cbase + off, out);
    }
}

template <typename TS, int DIM>
int launch_typed(const StepParams &p)
{
    const int vec = Store<TS>::VEC;
    if (p.P % vec != 0 || p.half[2] % vec != 0) return DVM_EINVAL;
    const int Q = p.P / vec;
    if (Q > MAXT) return DVM_ENOTIMPL;
    for (int d = 0; d < 3; d++)
        if (p.n[d] > NAX) return DVM_ENOTIMPL;
    const int threads = (Q + 31) / 32 * 32;
    const dim3 grid((unsigned)p.ncells);
    if (p.coll == DVM_COLL_BGK)
        k_step<TS, DIM, DVM_COLL_BGK><<<grid, threads, 0, p.stream>>>(p);
    else
        k_step<TS, DIM, DVM_COLL_NONE><<<grid, threads, 0, p.stream>>>(p);
    count_launch();
    return cudaGetLastError() == cudaSuccess ? DVM_OK : DVM_ECUDA;
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
