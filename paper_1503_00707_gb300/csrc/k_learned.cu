// Learned collision operator (not in the paper: the network, its gating by
// the local Knudsen number and its checks).  Per cell:
//
//   k_kn      local Knudsen number Kn_loc = (Kn/rho) max(|grad rho|/rho,
//             |grad T|/T, |grad u|/sqrt(T)), gradients by weighted least
//             squares over the face neighbours (coefficients precomputed on
//             the host from the geometry);
//   k_proj    a_m = sum_i f_i H_m(c_i) dV / rho (mode 0) or
//             o_m = sum_i I_i H_m(c_i) dV / (rho^2 sqrt(T)) (mode 1), the
//             projection on the 64 tensor Hermite modes H_m = He_a He_b He_c
//             (orthonormal probabilists' Hermite, a, b, c < 4) in the
//             Maxwellian-normalised velocity c = (xi - u)/sqrt(T);
//             Mode 0 also gives the projection of the cell's own discrete
//             Maxwellian M(rho, u, T), whose network output is subtracted
//             below so that the learned term vanishes at equilibrium;
//   k_lapply  Q_i = M_i (rho sqrt(T) sum_m o_m H_m(c_i) - d.phi_i), with the
//             five coefficients d of the centred basis phi = (1, c, |c|^2 - 3)
//             chosen so that Q carries no mass, momentum or energy (the
//             correction form of Eq. 6 applied to the reconstructed term);
//             the cell keeps f + dt/Kn Q only if sum Q ln f <= 1e-5 sum |Q|
//             (entropy production non-positive within rounding) and the 5x5
//             solve is exact to its residual, else it joins the
//             list of cells left to the hard-sphere operator.
//
// Velocity nodes come in the step kernel's group layout: node (ix, iy, iz)
// of group o = 4 sx + 2 sy + sz sits at o P + (mx Hy + my) Hz + mz, with
// ix = Hx + mx for sx = 1 and Hx - 1 - mx for sx = 0.  The Hermite modes,
// the Maxwellian and the moment basis all factorise over the axes, so the
// projection and the reconstruction are separable contractions on per-axis
// tables in shared memory, and the moment system is built from per-axis
// sums.  A cell's f arrives in shared memory as one bulk copy; the updated
// f leaves it the same way.
#include <cuda_runtime.h>

#include <cmath>

#include "../../include/dvm.h"
#include "async.cuh"
#include "common.cuh"
#include "kernels.hpp"
#include "learned.hpp"

namespace dvm {

void count_launch();

namespace {

constexpr int PT = 128;   // threads of k_proj
constexpr int AT = 256;   // threads of k_lapply
constexpr int MAXN = 32;  // velocity nodes per axis

constexpr float RS2 = 0.70710678118654752f;  // 1/sqrt(2)
constexpr float RS6 = 0.40824829046386302f;  // 1/sqrt(6)

// ---------------------------------------------------------------- local Kn
__global__ void k_kn(const double *__restrict__ mom, const int32_t *__restrict__ start,
                     const int32_t *__restrict__ nb, const double *__restrict__ coef, int64_t ncells, double kn,
                     double *__restrict__ knl)
{
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncells) return;
    const double *m = mom + c * 5;
    const double q[5] = {m[0], m[4], m[1], m[2], m[3]};  // rho, T, u
    double g[5][3] = {};
    for (int e = start[c]; e < start[c + 1]; e++) {
        const double *mn = mom + (int64_t)nb[e] * 5;
        const double dq[5] = {mn[0] - q[0], mn[4] - q[1], mn[1] - q[2], mn[2] - q[3], mn[3] - q[4]};
        const double w0 = coef[3 * (int64_t)e], w1 = coef[3 * (int64_t)e + 1], w2 = coef[3 * (int64_t)e + 2];
#pragma unroll
        for (int k = 0; k < 5; k++) {
            g[k][0] = fma(w0, dq[k], g[k][0]);
            g[k][1] = fma(w1, dq[k], g[k][1]);
            g[k][2] = fma(w2, dq[k], g[k][2]);
        }
    }
    double gr = 0, gT = 0, gu = 0;
#pragma unroll
    for (int d = 0; d < 3; d++) {
        gr += g[0][d] * g[0][d];
        gT += g[1][d] * g[1][d];
        gu += g[2][d] * g[2][d] + g[3][d] * g[3][d] + g[4][d] * g[4][d];
    }
    double mm = sqrt(gr) / q[0];
    const double t1 = sqrt(gT) / q[1], t2 = sqrt(gu) / sqrt(q[1]);
    if (t1 > mm) mm = t1;
    if (t2 > mm) mm = t2;
    knl[c] = kn / q[0] * mm;
}

// ---------------------------------------------------------------- helpers
// per-axis tables: H[d][i] = (He_1, He_2, He_3, exp(-c^2/2)) and G[d][i] = c
// at node i of axis d, c = (xi - u_d) / sqrt(T)
__device__ inline void axis_tables(const double *amag, int3 n, const float u[3], float ist, float4 (*H)[MAXN],
                                   float (*G)[MAXN], int tid, int nthreads)
{
    const int tot = n.x + n.y + n.z;
    for (int k = tid; k < tot; k += nthreads) {
        const int d = k < n.x ? 0 : (k < n.x + n.y ? 1 : 2);
        const int i = k - (d == 0 ? 0 : (d == 1 ? n.x : n.x + n.y));
        const int nd = d == 0 ? n.x : (d == 1 ? n.y : n.z);
        const int hd = nd / 2;
        float xi = (float)amag[d * 32 + (i < hd ? hd - 1 - i : i - hd)];
        if (i < hd) xi = -xi;
        const float c = (xi - u[d]) * ist;
        const float c2 = c * c;
        H[d][i] = make_float4(c, (c2 - 1.0f) * RS2, (c2 - 3.0f) * c * RS6, expf(-0.5f * c2));
        if (G) G[d][i] = c;
    }
}

// Sum of v[0..63] over the warp, scattered: lane l ends with the sums of
// entries 2l and 2l+1 in v[0] and v[1] (62 shuffles instead of 320).
__device__ inline void warp_reduce_scatter64(float (&v)[64], int lane)
{
#pragma unroll
    for (int s = 0; s < 5; s++) {
        const int off = 16 >> s, half = 32 >> s;
        const bool up = lane & off;
#pragma unroll
        for (int i = 0; i < half; i++) {
            const float send = up ? v[i] : v[half + i];
            const float keep = up ? v[half + i] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, off);
        }
    }
}

// Bounded wait for a CTA's single tile copy; on failure every thread learns
// it through *abort and thread 0 gives the copy one more bounded wait.
__device__ inline bool tile_arrived(uint64_t *bar, int *abort, int *status)
{
    if (!mbar_wait(bar, 0)) *abort = 1;
    __syncthreads();
    if (*abort) {
        if (threadIdx.x == 0) {
            atomicOr(status, ST_TIMEOUT);
            mbar_wait(bar, 0);
        }
        return false;
    }
    return true;
}

// The 15 distinct entries (r <= s) of the moment matrix of the target in the
// centred basis phi = (1, c_x, c_y, c_z, |c|^2 - 3) as sums of products of the
// per-axis sums X[a] Y[b] Z[c] (E_k of axis d): each term packed as
// coef (signed byte) | a << 8 | b << 12 | c << 16; coef 0 pads.
#define DVM_LT(cf, a, b, c) ((int32_t)((cf) & 0xff) | ((a) << 8) | ((b) << 12) | ((c) << 16))
__device__ const int32_t lt_terms[15][10] = {
    {DVM_LT(1, 0, 0, 0)},
    {DVM_LT(1, 1, 0, 0)},
    {DVM_LT(1, 0, 1, 0)},
    {DVM_LT(1, 0, 0, 1)},
    {DVM_LT(1, 2, 0, 0), DVM_LT(1, 0, 2, 0), DVM_LT(1, 0, 0, 2), DVM_LT(-3, 0, 0, 0)},
    {DVM_LT(1, 2, 0, 0)},
    {DVM_LT(1, 1, 1, 0)},
    {DVM_LT(1, 1, 0, 1)},
    {DVM_LT(1, 3, 0, 0), DVM_LT(1, 1, 2, 0), DVM_LT(1, 1, 0, 2), DVM_LT(-3, 1, 0, 0)},
    {DVM_LT(1, 0, 2, 0)},
    {DVM_LT(1, 0, 1, 1)},
    {DVM_LT(1, 2, 1, 0), DVM_LT(1, 0, 3, 0), DVM_LT(1, 0, 1, 2), DVM_LT(-3, 0, 1, 0)},
    {DVM_LT(1, 0, 0, 2)},
    {DVM_LT(1, 2, 0, 1), DVM_LT(1, 0, 2, 1), DVM_LT(1, 0, 0, 3), DVM_LT(-3, 0, 0, 1)},
    {DVM_LT(1, 4, 0, 0), DVM_LT(1, 0, 4, 0), DVM_LT(1, 0, 0, 4), DVM_LT(2, 2, 2, 0), DVM_LT(2, 2, 0, 2),
     DVM_LT(2, 0, 2, 2), DVM_LT(-6, 2, 0, 0), DVM_LT(-6, 0, 2, 0), DVM_LT(-6, 0, 0, 2), DVM_LT(9, 0, 0, 0)},
};
#undef DVM_LT

// ---------------------------------------------------------------- projection
template <int MODE>
__global__ void __launch_bounds__(PT) k_proj(const float *__restrict__ f, const double *__restrict__ mom,
                                             const double *__restrict__ amag, int3 n, double dV,
                                             const int32_t *__restrict__ list, const int *__restrict__ count,
                                             float *__restrict__ out, float *__restrict__ out_eq, int *status)
{
    extern __shared__ __align__(128) float tile[];  // [nv]
    __shared__ float4 H[3][MAXN];
    __shared__ float red[PT / 32][64];
    __shared__ float gsum[3][4];
    __shared__ __align__(8) uint64_t bar;
    __shared__ int abort_flag;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (list && (int64_t)blockIdx.x >= (int64_t)*count) return;
    const int64_t row = blockIdx.x;
    const int64_t cell = list ? (int64_t)list[row] : row;
    const int nv = n.x * n.y * n.z;
    const uint32_t bytes = (uint32_t)nv * 4u;
    if (tid == 0) {
        mbar_init(&bar, 1);
        abort_flag = 0;
        mbar_fence_init();
    }
    __syncthreads();
    if (tid == 0) {
        mbar_expect_tx(&bar, bytes);
        bulk_g2s(tile, f + cell * nv, bytes, &bar);
    }
    const double *mo = mom + cell * 5;
    const double rho = mo[0], T = mo[4];
    const float u[3] = {(float)mo[1], (float)mo[2], (float)mo[3]};
    // the FP64 scalars once, for the CTA: 1/sqrt(T), the output scale and the
    // Maxwellian's prefactor dV (2 pi T)^(-3/2)
    __shared__ float ist_s;
    __shared__ double scale_s, pre_s;
    if (tid == 0) {
        const double sqT = sqrt(T);
        ist_s = T > 0.0 ? (float)(1.0 / sqT) : 0.0f;
        scale_s = MODE == 0 ? dV / rho : dV / (rho * rho * sqT);
        pre_s = dV * 0.06349363593424097 / (T * sqT);
    }
    __syncthreads();
    const float ist = ist_s;
    axis_tables(amag, n, u, ist, H, nullptr, tid, PT);
    if (!tile_arrived(&bar, &abort_flag, status)) return;  // includes a barrier
    if (out_eq && tid < 12) {
        // per-axis sums sum_i exp(-c_i^2/2) He_a(c_i) for the projection of the
        // cell's own discrete Maxwellian
        const int d = tid >> 2, a = tid & 3;
        const int nd = d == 0 ? n.x : (d == 1 ? n.y : n.z);
        float sacc = 0.0f;
        for (int i = 0; i < nd; i++) {
            const float4 h = H[d][i];
            sacc = fmaf(h.w, a == 0 ? 1.0f : (a == 1 ? h.x : (a == 2 ? h.y : h.z)), sacc);
        }
        gsum[d][a] = sacc;
    }

    float acc[64];
#pragma unroll
    for (int k = 0; k < 64; k++) acc[k] = 0.0f;
    const int Hx = n.x / 2, Hy = n.y / 2, Hz = n.z / 2, P = Hx * Hy * Hz;
    for (int pp = tid; pp < n.x * n.y; pp += PT) {
        const int ix = pp / n.y, iy = pp - ix * n.y;
        const int sx = ix >= Hx, sy = iy >= Hy;
        const int mx = sx ? ix - Hx : Hx - 1 - ix, my = sy ? iy - Hy : Hy - 1 - iy;
        // contraction over z: t_c = sum_iz f He_c(iz)
        float t0 = 0.0f, t1 = 0.0f, t2 = 0.0f, t3 = 0.0f;
#pragma unroll
        for (int sz = 0; sz < 2; sz++) {
            const float *hp = tile + (4 * sx + 2 * sy + sz) * P + (mx * Hy + my) * Hz;
            for (int mz = 0; mz < Hz; mz += 4) {
                const float4 v4 = *reinterpret_cast<const float4 *>(hp + mz);
                const float vv[4] = {v4.x, v4.y, v4.z, v4.w};
#pragma unroll
                for (int e = 0; e < 4; e++) {
                    const float4 h = H[2][sz ? Hz + mz + e : Hz - 1 - mz - e];
                    t0 += vv[e];
                    t1 = fmaf(vv[e], h.x, t1);
                    t2 = fmaf(vv[e], h.y, t2);
                    t3 = fmaf(vv[e], h.z, t3);
                }
            }
        }
        const float4 hx = H[0][ix], hy = H[1][iy];
        const float wx[4] = {1.0f, hx.x, hx.y, hx.z}, wy[4] = {1.0f, hy.x, hy.y, hy.z};
        const float tz[4] = {t0, t1, t2, t3};
#pragma unroll
        for (int a = 0; a < 4; a++)
#pragma unroll
            for (int b = 0; b < 4; b++) {
                const float w = wx[a] * wy[b];
#pragma unroll
                for (int c = 0; c < 4; c++) acc[16 * a + 4 * b + c] = fmaf(w, tz[c], acc[16 * a + 4 * b + c]);
            }
    }
    warp_reduce_scatter64(acc, lane);
    red[warp][2 * lane] = acc[0];
    red[warp][2 * lane + 1] = acc[1];
    __syncthreads();
    if (tid < 64) {
        float s = 0.0f;
#pragma unroll
        for (int w = 0; w < PT / 32; w++) s += red[w][tid];
        out[row * 64 + tid] = (float)((double)s * scale_s);
        if (out_eq) {
            // a of M(rho, u, T) sampled at the nodes: dV (2 pi T)^(-3/2) times
            // the product of per-axis sums
            out_eq[row * 64 + tid] = (float)(pre_s * (double)gsum[0][tid >> 4] * (double)gsum[1][(tid >> 2) & 3] *
                                             (double)gsum[2][tid & 3]);
        }
    }
}

// ---------------------------------------------------------------- apply
__global__ void __launch_bounds__(AT) k_lapply(float *__restrict__ f, const double *__restrict__ mom,
                                               const float *__restrict__ o, const float *__restrict__ o_eq,
                                               const double *__restrict__ knl,
                                               double thr, const double *__restrict__ amag, int3 n, float dtkn,
                                               int32_t *__restrict__ used, int32_t *__restrict__ list,
                                               int *__restrict__ count, float *__restrict__ q_out, double dV,
                                               double *__restrict__ res, int *status)
{
    extern __shared__ __align__(128) float dsm[];
    __shared__ float4 H[3][MAXN];
    __shared__ float G[3][MAXN];
    __shared__ float S1[16][MAXN];
    __shared__ float4 ZT[MAXN];  // (exp(-cz^2/2), d3 cz + d4 cz^2, cz^2/2, 0)
    __shared__ float os[64];
    __shared__ double sums[3][14];
    __shared__ double rred[2][5];
    __shared__ double cc[5];
    __shared__ double ered[AT / 32], qred[AT / 32];
    __shared__ int good;
    __shared__ __align__(8) uint64_t bar;
    __shared__ int abort_flag;
    __shared__ double pro_d[2];  // sqrt(T), Mc
    __shared__ float pro_f[4];   // 1/sqrt(T), Mc, ln Mc, rho sqrt(T)

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t cell = blockIdx.x;
    if (!(knl[cell] < thr)) {
        // above the Knudsen threshold (or undefined): the plain operator
        if (tid == 0) {
            used[cell] = 0;
            list[atomicAdd(count, 1)] = (int32_t)cell;
        }
        return;
    }
    const int nv = n.x * n.y * n.z;
    const uint32_t bytes = (uint32_t)nv * 4u;
    float *tile = dsm;                                             // [nv]
    float4 *S2 = reinterpret_cast<float4 *>(dsm + nv);            // [ny][nz]: modes a = 0..3
    if (tid == 0) {
        mbar_init(&bar, 1);
        abort_flag = 0;
        mbar_fence_init();
    }
    __syncthreads();
    const double *mo = mom + cell * 5;
    const double rho = mo[0], T = mo[4];
    const bool valid = rho > 0.0 && T > 0.0 && isfinite(rho) && isfinite(T);
    if (tid == 0) {
        mbar_expect_tx(&bar, bytes);
        bulk_g2s(tile, f + cell * nv, bytes, &bar);
        // the FP64 scalars of the cell, once (FP64 runs at a small fraction
        // of the FP32 rate on this GPU)
        const double sq0 = valid ? sqrt(T) : 1.0;
        const double Mc0 = valid ? rho * 0.06349363593424097 / (T * sq0) : 1.0;  // rho (2 pi T)^(-3/2)
        pro_d[0] = sq0;
        pro_d[1] = Mc0;
        pro_f[0] = (float)(1.0 / sq0);
        pro_f[1] = (float)Mc0;
        pro_f[2] = (float)log(Mc0);
        pro_f[3] = (float)(rho * sq0);
    }
    if (tid < 64) os[tid] = o[cell * 64 + tid] - (o_eq ? o_eq[cell * 64 + tid] : 0.0f);
    __syncthreads();
    const double sq = pro_d[0], Mc = pro_d[1];
    const float u[3] = {(float)mo[1], (float)mo[2], (float)mo[3]};
    const float ist = pro_f[0], Mcf = pro_f[1], lnMc = pro_f[2], rsq = pro_f[3];
    axis_tables(amag, n, u, ist, H, G, tid, AT);
    __syncthreads();
    const int nz = n.z;
    // per-axis sums: E_k = sum e c^k (k < 5), G_ak = sum e He_a c^k (a = 1..3,
    // k < 3), in double-float over the FP32 table values (products of FP32
    // numbers split exactly by FMA; FP64 would run on this GPU's narrow FP64
    // pipe): the term these tables define then has its moments, and the
    // correction below closes them, to double-float rounding
    if (tid < 42) {
        const int d = tid / 14, k = tid % 14;
        const int nd = d == 0 ? n.x : (d == 1 ? n.y : n.z);
        ffn s{0.0f, 0.0f};
        for (int i = 0; i < nd; i++) {
            const float4 h = H[d][i];
            const float c = G[d][i];
            int pw;
            float w0;
            if (k < 5) {
                w0 = h.w;
                pw = k;
            } else {
                const int a = (k - 5) / 3;
                w0 = a == 0 ? h.x : (a == 1 ? h.y : h.z);
                pw = (k - 5) % 3;
            }
            // t = e (or e He_a) times c^pw, as a double-float product
            const float p0 = k < 5 ? w0 : h.w * w0;
            ffn t{p0, k < 5 ? 0.0f : fmaf(h.w, w0, -p0)};
            for (int q = 0; q < pw; q++) t = t * c;
            s = s + t;
        }
        sums[d][k] = (double)s.hi + (double)s.lo;
    }
    // S1[4a+b][iz] = sum_c o_abc He_c(iz)
    for (int idx = tid; idx < 16 * nz; idx += AT) {
        const int ab = idx / nz, iz = idx - ab * nz;
        const float4 h = H[2][iz];
        const float *om = os + 4 * ab;
        S1[ab][iz] = om[0] + om[1] * h.x + om[2] * h.y + om[3] * h.z;
    }
    __syncthreads();
    // S2[iy][iz][a] = sum_b S1[4a+b][iz] He_b(iy)
    for (int idx = tid; idx < n.y * nz; idx += AT) {
        const int iy = idx / nz, iz = idx - iy * nz;
        const float4 h = H[1][iy];
        float r[4];
#pragma unroll
        for (int a = 0; a < 4; a++)
            r[a] = S1[4 * a][iz] + S1[4 * a + 1][iz] * h.x + S1[4 * a + 2][iz] * h.y + S1[4 * a + 3][iz] * h.z;
        S2[idx] = make_float4(r[0], r[1], r[2], r[3]);
    }
    // moments of the reconstructed term: sum_m o_m R_r(m), R_r = sum e H_m phi_r
    if (tid < 64) {
        const int a = tid >> 4, b = (tid >> 2) & 3, c = tid & 3;
        double gx[3], gy[3], gz[3];
#pragma unroll
        for (int k = 0; k < 3; k++) {
            gx[k] = a == 0 ? sums[0][k] : sums[0][5 + 3 * (a - 1) + k];
            gy[k] = b == 0 ? sums[1][k] : sums[1][5 + 3 * (b - 1) + k];
            gz[k] = c == 0 ? sums[2][k] : sums[2][5 + 3 * (c - 1) + k];
        }
        const double w = os[tid];
        double r[5];
        r[0] = gx[0] * gy[0] * gz[0];
        r[1] = gx[1] * gy[0] * gz[0];
        r[2] = gx[0] * gy[1] * gz[0];
        r[3] = gx[0] * gy[0] * gz[1];
        r[4] = gx[2] * gy[0] * gz[0] + gx[0] * gy[2] * gz[0] + gx[0] * gy[0] * gz[2] - 3.0 * r[0];
#pragma unroll
        for (int k = 0; k < 5; k++) {
            r[k] *= w;
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) r[k] += __shfl_xor_sync(0xffffffffu, r[k], off);
        }
        if (lane == 0)
#pragma unroll
            for (int k = 0; k < 5; k++) rred[warp][k] = r[k];
    }
    __syncthreads();
    if (warp == 0) {
        // The moment system over dV Mc, A_rs = sum e phi_r phi_s, from the
        // per-axis sums: entry r <= s on lane sym(r, s) as a sum of products
        // X[a] Y[b] Z[c] with integer coefficients (lt_terms), then the 5x5
        // solve: an FP32 LDL^T factor on lane 0 refined twice against FP64
        // residuals computed one row per lane (the system is symmetric
        // positive definite and well conditioned), its FP64 residual checked
        // against 1e-12 of its scale.  FP64 stays on few instructions: this
        // GPU's FP64 pipe takes about 32 cycles per warp instruction.
        double ae = 0.0;
        if (lane < 15) {
#pragma unroll 1
            for (int t = 0; t < 10; t++) {
                const int32_t w = lt_terms[lane][t];
                const int cf = (int)(int8_t)(w & 0xff);
                if (cf != 0)
                    ae = fma((double)cf, sums[0][(w >> 8) & 15] * sums[1][(w >> 12) & 15] * sums[2][(w >> 16) & 15],
                             ae);
            }
        }
        auto sym = [](int r, int q) {
            const int lo = r < q ? r : q, hi = r < q ? q : r;
            return lo * 5 - (lo * (lo - 1)) / 2 + (hi - lo);
        };
        const int rv = lane < 5 ? lane : 0;
        double Arow[5];  // row rv of A
#pragma unroll
        for (int q = 0; q < 5; q++) Arow[q] = __shfl_sync(0xffffffffu, ae, sym(rv, q));
        const double b0 = (double)rsq * (rred[0][rv] + rred[1][rv]);
        // the FP32 factor on lane 0
        float Af[25];
#pragma unroll
        for (int e = 0; e < 25; e++) Af[e] = (float)__shfl_sync(0xffffffffu, ae, sym(e / 5, e % 5));
        float Lf[5][5], Dif[5];
        bool ok = valid;
        if (lane == 0) ok = ok && ldl5<float>(Af, Lf, Dif);
        ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
        double x[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
        double rres = b0;  // b - A x on lane r
        for (int it = 0; it < 3 && ok; it++) {
            float rf[5], dl[5] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
            for (int q = 0; q < 5; q++) rf[q] = (float)__shfl_sync(0xffffffffu, rres, q);
            if (lane == 0) ldl5_solve<float>(Lf, Dif, rf, dl);
#pragma unroll
            for (int q = 0; q < 5; q++) x[q] += (double)__shfl_sync(0xffffffffu, dl[q], 0);
            rres = b0;
#pragma unroll
            for (int q = 0; q < 5; q++) rres = fma(-Arow[q], x[q], rres);
        }
        bool fin = ok;
#pragma unroll
        for (int q = 0; q < 5; q++) fin = fin && isfinite(x[q]);
        if (fin) {
            // |A x - b| against max_r (|b_r| + sum_s |A_rs x_s|)
            double t = fabs(b0);
#pragma unroll
            for (int q = 0; q < 5; q++) t += fabs(Arow[q] * x[q]);
            double rn = lane < 5 ? fabs(rres) : 0.0, sc = lane < 5 ? t : 0.0;
#pragma unroll
            for (int off = 4; off > 0; off >>= 1) {
                rn = fmax(rn, __shfl_xor_sync(0xffffffffu, rn, off));
                sc = fmax(sc, __shfl_xor_sync(0xffffffffu, sc, off));
            }
            rn = __shfl_sync(0xffffffffu, rn, 0);
            sc = __shfl_sync(0xffffffffu, sc, 0);
            fin = rn <= 1e-12 * sc;
        }
        if (fin && res) {
            // sum_i phi_r Q_i dV = dV Mc (rhs - A d), taken to psi = (1, xi,
            // |xi|^2) with xi = sqrt(T) c + u
            double rvv[5];
#pragma unroll
            for (int q = 0; q < 5; q++) rvv[q] = __shfl_sync(0xffffffffu, rres, q);
            if (lane < 5) {
                const double k = dV * Mc, uu[3] = {mo[1], mo[2], mo[3]};
                double o5;
                if (lane == 0) o5 = k * rvv[0];
                else if (lane < 4) o5 = k * (sq * rvv[lane] + uu[lane - 1] * rvv[0]);
                else {
                    const double dot = uu[0] * rvv[1] + uu[1] * rvv[2] + uu[2] * rvv[3];
                    o5 = k * (T * (rvv[4] + 3.0 * rvv[0]) + 2.0 * sq * dot +
                              (uu[0] * uu[0] + uu[1] * uu[1] + uu[2] * uu[2]) * rvv[0]);
                }
                res[cell * 5 + lane] = o5;
            }
        }
        if (lane < 5) cc[lane] = fin ? x[lane] : 0.0;
        if (lane == 0) good = fin ? 1 : 0;
    }
    __syncthreads();
    const float d0 = (float)cc[0], d1 = (float)cc[1], d2 = (float)cc[2], d3 = (float)cc[3], d4 = (float)cc[4];
    for (int iz = tid; iz < nz; iz += AT) {
        const float c = G[2][iz];
        ZT[iz] = make_float4(H[2][iz].w, c * (d3 + d4 * c), 0.5f * c * c, 0.0f);
    }
    if (!tile_arrived(&bar, &abort_flag, status)) return;  // includes a barrier

    const int Hx = n.x / 2, Hy = n.y / 2, Hz = nz / 2, P = Hx * Hy * Hz;
    // Q at node (pencil constants, mz + e): M (rho sqrt(T) s - d.phi)
    auto pencil = [&](int pp, auto &&visit) {
        const int ix = pp / n.y, iy = pp - ix * n.y;
        const int sx = ix >= Hx, sy = iy >= Hy;
        const int mx = sx ? ix - Hx : Hx - 1 - ix, my = sy ? iy - Hy : Hy - 1 - iy;
        const float4 hx = H[0][ix], hy = H[1][iy];
        const float gx = G[0][ix], gy = G[1][iy];
        const float w0 = rsq, w1 = rsq * hx.x, w2 = rsq * hx.y, w3 = rsq * hx.z;
        const float K0 = d0 + d1 * gx + d2 * gy + d4 * (gx * gx + gy * gy - 3.0f);
        const float Pxy = Mcf * hx.w * hy.w;
        const float Lxy = lnMc - 0.5f * (gx * gx + gy * gy);
        const float4 *s2row = S2 + iy * nz;
#pragma unroll
        for (int sz = 0; sz < 2; sz++) {
            const int base = (4 * sx + 2 * sy + sz) * P + (mx * Hy + my) * Hz;
            for (int mz = 0; mz < Hz; mz += 4) {
                float4 *fp = reinterpret_cast<float4 *>(tile + base + mz);
                float fv[4] = {fp->x, fp->y, fp->z, fp->w};
                float Q[4], lnM[4];
#pragma unroll
                for (int e = 0; e < 4; e++) {
                    const int iz = sz ? Hz + mz + e : Hz - 1 - mz - e;
                    const float4 s = s2row[iz];
                    const float4 z = ZT[iz];
                    const float sv = fmaf(w3, s.w, fmaf(w2, s.z, fmaf(w1, s.y, w0 * s.x)));
                    Q[e] = Pxy * z.x * (sv - K0 - z.y);
                    lnM[e] = Lxy - z.z;
                }
                visit(fp, fv, Q, lnM, base + mz);
            }
        }
    };
    float ent = 0.0f, qabs = 0.0f;
    if (good) {
        for (int pp = tid; pp < n.x * n.y; pp += AT)
            pencil(pp, [&](float4 *, const float (&fv)[4], const float (&Q)[4], const float (&lnM)[4], int) {
#pragma unroll
                for (int e = 0; e < 4; e++) {
                    const float x = fv[e];
                    // ln f, with ln(1e-300) standing in for f <= 0
                    const float lf = x >= 1.17549435e-38f ? __logf(x) : (x > 0.0f ? logf(x) : -690.77552789821f);
                    ent = fmaf(Q[e], lf - lnM[e], ent);
                    qabs += fabsf(Q[e]);
                }
            });
    }
    // warp sums in FP32 (their rounding is far below the gate's 1e-5), the
    // eight warp totals in FP64
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        ent += __shfl_xor_sync(0xffffffffu, ent, off);
        qabs += __shfl_xor_sync(0xffffffffu, qabs, off);
    }
    if (lane == 0) {
        ered[warp] = (double)ent;
        qred[warp] = (double)qabs;
    }
    __syncthreads();
    if (tid == 0) {
        double s = 0.0, sa = 0.0;
        for (int w = 0; w < AT / 32; w++) {
            s += ered[w];
            sa += qred[w];
        }
        // entropy production non-positive within the rounding of its FP32
        // evaluation (an equilibrium cell, where it is zero up to rounding,
        // passes)
        good = good && isfinite(s) && s <= 1e-5 * sa;
    }
    __syncthreads();
    if (!good) {
        if (tid == 0) {
            used[cell] = 0;
            list[atomicAdd(count, 1)] = (int32_t)cell;
        }
        return;
    }
    float *qc = q_out ? q_out + cell * nv : nullptr;
    for (int pp = tid; pp < n.x * n.y; pp += AT)
        pencil(pp, [&](float4 *fp, const float (&fv)[4], const float (&Q)[4], const float (&)[4], int v) {
            *fp = make_float4(fmaf(dtkn, Q[0], fv[0]), fmaf(dtkn, Q[1], fv[1]), fmaf(dtkn, Q[2], fv[2]),
                              fmaf(dtkn, Q[3], fv[3]));
            if (qc) *reinterpret_cast<float4 *>(qc + v) = make_float4(Q[0], Q[1], Q[2], Q[3]);
        });
    fence_proxy_async();
    __syncthreads();
    if (tid == 0) {
        used[cell] = 1;
        bulk_s2g(f + cell * nv, tile, bytes);
        bulk_commit();
        bulk_wait_read_all();
    }
}

bool grid_ok(const int n[3])
{
    for (int d = 0; d < 3; d++)
        if (n[d] > MAXN || n[d] < 2 || n[d] % 2) return false;
    return (n[2] / 2) % 4 == 0;
}

}  // namespace

bool learned_grid_supported(const int n[3]) { return grid_ok(n); }

int launch_kn_local(const double *mom, const int32_t *start, const int32_t *nb, const double *coef, int64_t ncells,
                    double kn, double *knl, cudaStream_t s)
{
    if (ncells <= 0) return DVM_OK;
    k_kn<<<(unsigned)((ncells + 255) / 256), 256, 0, s>>>(mom, start, nb, coef, ncells, kn, knl);
    count_launch();
    return cudaGetLastError() == cudaSuccess ? DVM_OK : DVM_ECUDA;
}

int launch_hermite_project(const float *f, const double *mom, const double *amag, int64_t rows, const int n[3],
                           double dV, int mode, const int32_t *list, const int *count, float *out, float *out_eq,
                           int *status, cudaStream_t s)
{
    if (!grid_ok(n)) return DVM_ENOTIMPL;
    if (rows <= 0) return DVM_OK;
    const size_t dyn = (size_t)n[0] * n[1] * n[2] * sizeof(float);
    if (dyn > 200 * 1024) return DVM_ENOTIMPL;
    const int3 nn = make_int3(n[0], n[1], n[2]);
    auto kern = mode == 0 ? k_proj<0> : k_proj<1>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024) != cudaSuccess)
        return DVM_ECUDA;
    kern<<<(unsigned)rows, PT, dyn, s>>>(f, mom, amag, nn, dV, list, count, out, mode == 0 ? out_eq : nullptr, status);
    count_launch();
    return cudaGetLastError() == cudaSuccess ? DVM_OK : DVM_ECUDA;
}

int launch_learned_apply(float *f, const double *mom, const float *o, const float *o_eq, const double *knl, double thr,
                         const double *amag, int64_t ncells, const int n[3], double dtkn, int32_t *used,
                         int32_t *list, int *count, float *q_out, double dV, double *res, int *status, cudaStream_t s)
{
    if (!grid_ok(n)) return DVM_ENOTIMPL;
    if (ncells <= 0) return DVM_OK;
    const size_t dyn = (size_t)n[0] * n[1] * n[2] * sizeof(float) + (size_t)n[1] * n[2] * sizeof(float4);
    if (dyn > 200 * 1024) return DVM_ENOTIMPL;
    if (cudaFuncSetAttribute(k_lapply, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024) != cudaSuccess)
        return DVM_ECUDA;
    k_lapply<<<(unsigned)ncells, AT, dyn, s>>>(f, mom, o, o_eq, knl, thr, amag, make_int3(n[0], n[1], n[2]), (float)dtkn,
                                                used, list, count, q_out, dV, res, status);
    count_launch();
    return cudaGetLastError() == cudaSuccess ? DVM_OK : DVM_ECUDA;
}

}  // namespace dvm
