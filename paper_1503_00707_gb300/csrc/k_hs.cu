// Hard-sphere discrete collision integral (paper Sec. 3.2, Eqs. 3-6).
//
// The trial table (gamma, l, m, b for every node i and trial k) is the same
// for all cells (Sec. 3.2), and each trial needs three random gathers from a
// cell's f.  The paper's kernel keeps one node's table in shared memory and
// gathers f across cells from a velocity-major copy; here the roles are
// swapped to keep every gather on chip:
//
//  k_hs_bc   table-stationary: a CTA holds the trials of 64 nodes (256
//            threads) or, on grids of more than 6144 nodes, 128 nodes (512
//            threads) in registers (32 per thread) and streams cells through a
//            double-buffered shared-memory tile, each tile a single bulk
//            copy (cp.async.bulk, completion on an mbarrier).  It writes
//            B_i = sum_k b f_gamma (Eq. 4) and C_i = sum_k c f_l f_m (Eq. 5)
//            for its nodes to a per-cell scratch array.
//  k_hs_corr per cell: the five coefficients of P (Eq. 6) from the moment
//            system, its sums formed exactly in an integer basis and
//            carried in double-float, solved in FP64 in the centred basis
//            (1, c, |c|^2 - 3), c = (xi - u)/sqrt(T), and refined against
//            the exact sums; then I = -f P B + C and f <- f + dt/Kn I in
//            place.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <mutex>

#include "../../include/dvm.h"
#include "async.cuh"
#include "common.cuh"
#include "hs.hpp"

namespace dvm {

void count_launch();

namespace {

constexpr int HE = 32;    // trials held per thread
constexpr int CT = 256;   // threads per CTA of k_hs_corr

// HT threads per CTA (256 or 512; at most 128 registers a thread either way)
template <int HT>
__global__ void __launch_bounds__(HT, 512 / HT)
    k_hs_bc(const float *__restrict__ fs, float2 *__restrict__ bc, int64_t ncells, int nv, int M,
            const uint2 *__restrict__ idx, const float *__restrict__ bw, int64_t cells_per_cta,
            const int32_t *__restrict__ list, const int *__restrict__ count, int *status)
{
    extern __shared__ __align__(128) float tile[];  // [2][nv]
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ int abort_flag;

    const int tid = threadIdx.x;
    const int tpn = M / HE;  // threads per node (power of two, <= 32)
    const int npc = HT / tpn;
    const int node = blockIdx.x * npc + tid / tpn;
    const bool valid = node < nv;
    const int64_t e0 = (int64_t)(valid ? node : 0) * M + (tid % tpn) * HE;
    uint32_t w0[HE], w1[HE];
    float b[HE];
#pragma unroll
    for (int e = 0; e < HE; e++) {
        const uint2 t = idx[e0 + e];
        w0[e] = t.x;
        w1[e] = t.y;
        b[e] = valid ? bw[e0 + e] : 0.0f;
    }
    // rows c0..c1-1 of this CTA: cells, or entries of the cell list
    int64_t nrows = ncells, per = cells_per_cta;
    if (list) {
        nrows = *count;
        per = (nrows + gridDim.y - 1) / gridDim.y;
    }
    const int64_t c0 = (int64_t)blockIdx.y * per;
    const int64_t c1 = c0 + per < nrows ? c0 + per : nrows;
    auto src = [&](int64_t r) { return fs + (list ? (int64_t)list[r] : r) * nv; };
    const uint32_t bytes = (uint32_t)nv * 4u;
    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        abort_flag = 0;
        mbar_fence_init();
    }
    __syncthreads();
    // copies issued into / completions seen on each buffer (uniform over the CTA)
    int issued[2] = {0, 0}, done[2] = {0, 0};
    if (c0 < c1) {
        if (tid == 0) {
            mbar_expect_tx(&bar[0], bytes);
            bulk_g2s(tile, src(c0), bytes, &bar[0]);
        }
        issued[0]++;
    }
    for (int64_t c = c0; c < c1; c++) {
        const int j = (int)(c - c0), s = j & 1;
        if (c + 1 < c1) {
            // buffer s^1 was last read in the previous iteration, which ended
            // with a barrier
            if (tid == 0) {
                mbar_expect_tx(&bar[s ^ 1], bytes);
                bulk_g2s(tile + (size_t)(s ^ 1) * nv, src(c + 1), bytes, &bar[s ^ 1]);
            }
            issued[s ^ 1]++;
        }
        if (mbar_wait(&bar[s], (uint32_t)done[s] & 1u)) done[s]++;
        else abort_flag = 1;
        const float *t = tile + (size_t)s * nv;
        float B = 0.0f, C = 0.0f;
#pragma unroll
        for (int e = 0; e < HE; e++) {
            const float fg = t[w0[e] & 0xffffu];
            const float fl = t[w0[e] >> 16];
            const float fm = t[w1[e]];
            B = fmaf(b[e], fg, B);
            C = fmaf(b[e], fl * fm, C);
        }
        for (int m = 1; m < tpn; m <<= 1) {
            B += __shfl_xor_sync(0xffffffffu, B, m);
            C += __shfl_xor_sync(0xffffffffu, C, m);
        }
        if (valid && tid % tpn == 0) bc[c * nv + node] = make_float2(B, C);
        __syncthreads();
        if (abort_flag) {
            // a tile never arrived: report, give the copies in flight a bounded
            // time to land, and stop
            if (tid == 0) {
                atomicOr(status, ST_TIMEOUT);
                for (int q = 0; q < 2; q++)
                    while (done[q] < issued[q] && mbar_wait(&bar[q], (uint32_t)done[q] & 1u)) done[q]++;
            }
            return;
        }
    }
}

// Sum2 accumulation (Ogita, Rump and Oishi, 2005) of exact products:
// s + e carries the running sum to about twice the FP32 precision.
struct Acc2 {
    float s, e;
};
// a += (x + xl) k, with x k split exactly (FMA) and xl k a small correction
__device__ inline void acc2_prod(Acc2 &a, float x, float xl, float k)
{
    const float p = x * k;
    const float pe = fmaf(x, k, -p);
    const float s = a.s + p;
    const float bb = s - a.s;
    const float se = (a.s - (s - bb)) + (p - bb);
    a.s = s;
    a.e += se + fmaf(xl, k, pe);
}

constexpr int NSUM = 20;  // 15 distinct entries of the moment matrix, 5 gain moments

// k_hs_corr: one CTA per cell.  The correction polynomial of Eq. 6,
// P = 1 + d.phi, phi = (1, c, |c|^2 - 3), c = (xi - u)/sqrt(T), makes
// I = C - f P B conserve mass, momentum and energy.  The system is formed
// exactly: with xi_d = (h/2) j_d (j_d odd integers, the same h on every
// axis) the integer basis psi^ = (1, j_x, j_y, j_z, |j|^2) spans the same
// polynomials, so the 15 sums A^_rs = sum_i psi^_r psi^_s f_i B_i and the 5
// sums c^_r = sum_i psi^_r C_i have integer weights below 2^24 and products
// split exactly (FMA); Sum2 carries them to double-float, and one thread
// solves A^ e = c^, e = (1, 0, 0, 0, 0) + L^T d (L the map psi^ -> phi), in
// FP64: the factor of L A^ L^T (well conditioned), refined twice against the
// residual of the exact sums.  That residual, sum_i psi_r I_i dV with
// psi = (1, xi, |xi|^2), goes to res (may be null).  Then I_i is evaluated
// in FP32 with the FP32 copy of d and f <- f + dt/Kn I (or I to q_out).
// three CTAs per SM (80 registers): other cells' sums overlap one CTA's
// serial solve (C4: 7.56 -> 7.29 ms per step; two or four CTAs were slower on
// one of the 16^3 and 24^3 grids)
__global__ void __launch_bounds__(CT, 3)
    k_hs_corr(float *__restrict__ f, const float2 *__restrict__ bc, const float *__restrict__ xi3,
              const uint32_t *__restrict__ jpk, double hh, double dV, const double *__restrict__ mom, int nv,
              int3 half, float dtkn, const int32_t *__restrict__ list, const int *__restrict__ count,
              float *__restrict__ q_out, double *__restrict__ res, int *status)
{
    __shared__ ffn part[NSUM][CT];
    __shared__ double S[NSUM];
    __shared__ float sd[5];
    // row blockIdx.x of B and C belongs to this cell (an entry of the list, if any)
    const int64_t row = blockIdx.x;
    if (list && row >= (int64_t)*count) return;
    const int64_t cell = list ? (int64_t)list[row] : row;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const double *mo = mom + cell * 5;
    const double rho = mo[0], Td = mo[4];
    if (!(rho > 0.0) || !(Td > 0.0) || !isfinite(rho + Td + mo[1] + mo[2] + mo[3])) {
        // no correction exists: report, leave f as it is
        if (tid == 0) {
            atomicOr(status, ST_NONPOS);
            if (res)
                for (int r = 0; r < 5; r++) res[cell * 5 + r] = 0.0;
        }
        return;
    }
    float *fc = f + cell * (int64_t)nv;
    const float2 *bcc = bc + row * (int64_t)nv;
    // The sums over the nodes, pencil by pencil: a pencil is the line of nodes
    // along z at fixed (x, y) node indices, both z signs (sign groups 2 o_xy
    // and 2 o_xy + 1, positions pos .. pos + hz - 1 in each).  Along a pencil
    // j_x = a and j_y = b are fixed, so with W_k = sum f B j_z^k (k <= 4) and
    // C_k = sum C j_z^k (k <= 2), s2 = a^2 + b^2, every sum of the system is a
    // combination of the pencil sums with integer coefficients, e.g.
    //   sum f B |j|^2 = s2 W_0 + W_2,  sum f B |j|^4 = s2^2 W_0 + 2 s2 W_2 + W_4.
    // Products by integers below 2^24 split exactly (FMA), so the sums stay
    // Sum2-exact, at 8 accumulations per node and 27 per pencil instead of
    // 20 per node.  The entries are numbered as the upper triangle of the 5x5
    // matrix over (1, j_x, j_y, j_z, |j|^2), then the 5 right-hand sums.
    Acc2 acc[NSUM];
#pragma unroll
    for (int k = 0; k < NSUM; k++) acc[k] = Acc2{0.0f, 0.0f};
    const int hxy = half.x * half.y, P = hxy * half.z, npen = 4 * hxy;
    for (int pen = tid; pen < npen; pen += CT) {
        const int oxy = pen / hxy, pos = (pen - oxy * hxy) * half.z;
        const uint32_t jp0 = jpk[2 * oxy * P + pos];
        const float a = (float)((int)(jp0 & 0xffu) - 64), b = (float)((int)((jp0 >> 8) & 0xffu) - 64);
        Acc2 W[5], Cs[3];
#pragma unroll
        for (int k = 0; k < 5; k++) W[k] = Acc2{0.0f, 0.0f};
#pragma unroll
        for (int k = 0; k < 3; k++) Cs[k] = Acc2{0.0f, 0.0f};
#pragma unroll
        for (int oz = 0; oz < 2; oz++) {
            const int v0 = (2 * oxy + oz) * P + pos;
            for (int m = 0; m < half.z; m++) {
                const int v = v0 + m;
                const float fv = fc[v];
                const float2 q = bcc[v];
                const float jz = (float)((int)((jpk[v] >> 16) & 0xffu) - 64);
                const float jz2 = jz * jz;
                const float w = fv * q.x, wl = fmaf(fv, q.x, -w);  // f B = w + wl exactly
                acc2_prod(W[0], w, wl, 1.0f);
                acc2_prod(W[1], w, wl, jz);
                acc2_prod(W[2], w, wl, jz2);
                acc2_prod(W[3], w, wl, jz2 * jz);
                acc2_prod(W[4], w, wl, jz2 * jz2);
                acc2_prod(Cs[0], q.y, 0.0f, 1.0f);
                acc2_prod(Cs[1], q.y, 0.0f, jz);
                acc2_prod(Cs[2], q.y, 0.0f, jz2);
            }
        }
        const float s2 = a * a + b * b;
        auto put = [&](int k, const Acc2 &x, float coef) { acc2_prod(acc[k], x.s, x.e, coef); };
        put(0, W[0], 1.0f);                                         // (1, 1)
        put(1, W[0], a);                                            // (1, j_x)
        put(2, W[0], b);                                            // (1, j_y)
        put(3, W[1], 1.0f);                                         // (1, j_z)
        put(4, W[0], s2); put(4, W[2], 1.0f);                       // (1, |j|^2)
        put(5, W[0], a * a);                                        // (j_x, j_x)
        put(6, W[0], a * b);                                        // (j_x, j_y)
        put(7, W[1], a);                                            // (j_x, j_z)
        put(8, W[0], a * s2); put(8, W[2], a);                      // (j_x, |j|^2)
        put(9, W[0], b * b);                                        // (j_y, j_y)
        put(10, W[1], b);                                           // (j_y, j_z)
        put(11, W[0], b * s2); put(11, W[2], b);                    // (j_y, |j|^2)
        put(12, W[2], 1.0f);                                        // (j_z, j_z)
        put(13, W[1], s2); put(13, W[3], 1.0f);                     // (j_z, |j|^2)
        put(14, W[0], s2 * s2); put(14, W[2], 2.0f * s2); put(14, W[4], 1.0f);  // (|j|^2, |j|^2)
        put(15, Cs[0], 1.0f);
        put(16, Cs[0], a);
        put(17, Cs[0], b);
        put(18, Cs[1], 1.0f);
        put(19, Cs[0], s2); put(19, Cs[2], 1.0f);
    }
#pragma unroll
    for (int k = 0; k < NSUM; k++) {
        const float s = acc[k].s + acc[k].e;
        const float bb = s - acc[k].s;
        part[k][tid] = ffn{s, (acc[k].s - (s - bb)) + (acc[k].e - bb)};
    }
    __syncthreads();
    // warp w adds sums w, w + 8, w + 16 over the CTA in double-float
    for (int k = warp; k < NSUM; k += CT / 32) {
        ffn a = part[k][lane];
#pragma unroll
        for (int t = lane + 32; t < CT; t += 32) a = a + part[k][t];
#pragma unroll
        for (int m = 16; m > 0; m >>= 1)
            a = a + ffn{__shfl_xor_sync(0xffffffffu, a.hi, m), __shfl_xor_sync(0xffffffffu, a.lo, m)};
        if (lane == 0) S[k] = (double)a.hi + (double)a.lo;
    }
    __syncthreads();
    if (warp == 0) {
        // The 5x5 solve on the lanes of warp 0, in FP64.  phi = L psi^ with
        //   phi_0 = 1, phi_d = be_d + al j_d, phi_4 = |be|^2 - 3 + 2 al be.j + al^2 |j|^2,
        // al = (h/2)/sqrt(T), be = -u/sqrt(T); the system A^ e = c^ with
        // e = (1, 0, 0, 0, 0) + L^T d is factored through the well-conditioned
        // centred-basis matrix L A^ L^T (an LDL^T on lane 0) and refined twice
        // against the residual of the exact sums.  Lane 5 r + s holds entry
        // (r, s) of the 5x5 products; lanes 0..4 hold the vectors.
        const double isT = 1.0 / sqrt(Td), al = hh * isT;
        const double be0 = -mo[1] * isT, be1 = -mo[2] * isT, be2 = -mo[3] * isT;
        auto Lm = [&](int r, int k) -> double {
            if (r == 0) return k == 0 ? 1.0 : 0.0;
            if (r < 4) {
                const double b = r == 1 ? be0 : (r == 2 ? be1 : be2);
                return k == 0 ? b : (k == r ? al : 0.0);
            }
            if (k == 0) return be0 * be0 + be1 * be1 + be2 * be2 - 3.0;
            if (k < 4) return 2.0 * al * (k == 1 ? be0 : (k == 2 ? be1 : be2));
            return al * al;
        };
        // entry (r, s) of A^ (index of the upper-triangle sum)
        auto Aj = [&](int r, int q) -> double {
            const int lo = r < q ? r : q, hi = r < q ? q : r;
            return S[lo * 5 - (lo * (lo - 1)) / 2 + (hi - lo)];
        };
        auto bcast = [](double v, int src) -> double { return __shfl_sync(0xffffffffu, v, src); };
        const int r5 = lane < 25 ? lane / 5 : 0, s5 = lane < 25 ? lane % 5 : 0;
        // T1 = L A^ (lane 5 r + s), then Ap = T1 L^T
        double t1 = 0.0;
#pragma unroll
        for (int k = 0; k < 5; k++) t1 = fma(Lm(r5, k), Aj(k, s5), t1);
        double ap = 0.0;
#pragma unroll
        for (int k = 0; k < 5; k++) ap = fma(bcast(t1, r5 * 5 + k), Lm(s5, k), ap);
        double Ap[25];
#pragma unroll
        for (int k = 0; k < 25; k++) Ap[k] = bcast(ap, k);
        double Lf[5][5], Di[5];
        bool ok = true;
        if (lane == 0) ok = ldl5<double>(Ap, Lf, Di);
        ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
        // lane r < 5: d_r; every lane: the whole d after each broadcast
        double d[5] = {0.0, 0.0, 0.0, 0.0, 0.0}, R = 0.0;
        const int rv = lane < 5 ? lane : 0;
        for (int it = 0; it < 3; it++) {
            // e_s = (s == 0) + sum_k L_ks d_k on lane s, then R_r = c^_r - sum_s A^_rs e_s
            double e = rv == 0 ? 1.0 : 0.0;
#pragma unroll
            for (int k = 0; k < 5; k++) e = fma(Lm(k, rv), d[k], e);
            double ev[5];
#pragma unroll
            for (int k = 0; k < 5; k++) ev[k] = bcast(e, k);
            R = S[15 + rv];
#pragma unroll
            for (int q = 0; q < 5; q++) R = fma(-Aj(rv, q), ev[q], R);
            if (it == 2 || !ok) break;
            // LR = L R on lane r, then the LDL^T solve on lane 0
            double Rv[5];
#pragma unroll
            for (int k = 0; k < 5; k++) Rv[k] = bcast(R, k);
            double lr = 0.0;
#pragma unroll
            for (int k = 0; k < 5; k++) lr = fma(Lm(rv, k), Rv[k], lr);
            double LR[5], dl[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
#pragma unroll
            for (int k = 0; k < 5; k++) LR[k] = bcast(lr, k);
            if (lane == 0) ldl5_solve<double>(Lf, Di, LR, dl);
#pragma unroll
            for (int k = 0; k < 5; k++) d[k] += bcast(dl[k], 0);
        }
        bool fin = ok;
#pragma unroll
        for (int k = 0; k < 5; k++) fin = fin && isfinite(d[k]);
        if (lane == 0 && !fin) atomicOr(status, ST_SINGULAR);
        if (lane < 5) {
            sd[lane] = fin ? (float)d[lane] : 0.0f;
            if (res) {
                const double sc = lane == 0 ? dV : (lane < 4 ? dV * hh : dV * hh * hh);
                res[cell * 5 + lane] = fin ? sc * R : 0.0;
            }
        }
    }
    __syncthreads();
    const float ux = (float)mo[1], uy = (float)mo[2], uz = (float)mo[3];
    const float ist = rsqrtf((float)Td);
    const float d0 = sd[0], dx = sd[1], dy = sd[2], dz = sd[3], d4 = sd[4];
    float worst = 0.0f;
    for (int v = tid; v < nv; v += CT) {
        const float fv = fc[v];
        const float2 q = bcc[v];
        const float cx = (xi3[v] - ux) * ist, cy = (xi3[nv + v] - uy) * ist, cz = (xi3[2 * nv + v] - uz) * ist;
        const float P = 1.0f + d0 + dx * cx + dy * cy + dz * cz + d4 * (cx * cx + cy * cy + cz * cz - 3.0f);
        const float loss = P * q.x;
        worst = fmaxf(worst, dtkn * loss);
        if (q_out) q_out[cell * (int64_t)nv + v] = q.y - fv * loss;  // the term I alone, f kept
        else fc[v] = fmaf(dtkn, q.y - fv * loss, fv);
    }
    if (worst > 1.0f) atomicOr(status, ST_NUDT);
}

}  // namespace

bool hs_trials_supported(int trials)
{
    if (trials < HE || trials % HE) return false;
    const int tpn = trials / HE;
    return tpn <= 32 && (tpn & (tpn - 1)) == 0;
}

int hs_prepare(HsTables &t, int64_t ncells, const DevAlloc &alloc, const DevFree &dfree)
{
    if (!t.ready) return DVM_ESTATE;
    if (t.d_bc && t.bc_cells == ncells) return DVM_OK;
    if (t.d_bc) dfree(t.d_bc);
    t.d_bc = static_cast<float *>(alloc((size_t)ncells * t.nv * 2 * sizeof(float)));
    t.bc_cells = t.d_bc ? ncells : 0;
    return t.d_bc ? DVM_OK : DVM_ENOMEM;
}

// Cell splits of the k_hs_bc grid (node chunks x cell ranges): at least two
// waves of resident CTAs, and a total that fills its last wave as far as
// possible.  Every CTA streams the same number of cells, so a last wave that
// is only partly full leaves the rest of the GPU idle for a whole CTA's time
// (64 chunks x 10 ranges on 304 resident CTAs ran as 304 + 304 + 32).
static int64_t hs_splits(int chunks, int slots, int64_t ncells)
{
    const int64_t s0 = std::max<int64_t>(1, (2 * (int64_t)slots + chunks - 1) / chunks);
    int64_t best = s0;
    double best_eff = -1.0;
    for (int64_t sp = s0; sp <= 4 * s0; sp++) {
        const int64_t per = (ncells + sp - 1) / sp, used = (ncells + per - 1) / per;
        const int64_t total = (int64_t)chunks * used, waves = (total + slots - 1) / slots;
        const double eff = (double)total / (double)(waves * slots);
        if (eff > best_eff + 1e-9) {
            best_eff = eff;
            best = sp;
        }
    }
    return std::max<int64_t>(1, std::min<int64_t>(best, ncells));
}

// The launch shape of k_hs_bc for nv nodes and ncells rows.  Each CTA streams
// the whole f of every cell of its range through shared memory for the trials
// of its nodes, so the tile is worth 3 M npc / nv gathers per loaded value:
// 1.8 at 24^3 with 64 nodes per CTA, 3.6 with 128.  Grids of more than 6144
// nodes take 512 threads (128 nodes), the others 256 (measured: 24^3, 543.9 ->
// 389.8 ms per step on the 253k-cell flow; 16^3 is 1.5% faster with 256).
// Every check that can refuse the launch is made here, before anything is
// queued.
struct BcLaunch {
    int threads = 0;
    dim3 grid;
    size_t dyn = 0;
    int64_t per = 0;  // rows per CTA
};

static int bc_plan(const HsTables &t, int nv, int64_t ncells, BcLaunch &L)
{
    const int ht = nv > 6144 ? 512 : 256;
    const int tpn = t.trials / HE, npc = ht / tpn;
    const int chunks = (nv + npc - 1) / npc;
    const size_t dyn = 2 * (size_t)nv * sizeof(float);
    if (dyn > 200 * 1024) return DVM_ENOTIMPL;
    auto kern = ht == 512 ? k_hs_bc<512> : k_hs_bc<256>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024) != cudaSuccess)
        return DVM_ECUDA;
    int dev = 0, nsm = 0, occ = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, ht, dyn) != cudaSuccess || occ < 1)
        return DVM_ENOTIMPL;
    int64_t splits = hs_splits(chunks, nsm * occ, ncells);
    L.per = (ncells + splits - 1) / splits;
    splits = (ncells + L.per - 1) / L.per;
    L.threads = ht;
    L.grid = dim3((unsigned)chunks, (unsigned)splits);
    L.dyn = dyn;
    return DVM_OK;
}

static int bc_launch(const BcLaunch &L, const HsTables &t, const float *f, float2 *bc, int64_t ncells, int nv,
                     const int32_t *list, const int *count, cudaStream_t s, int *status)
{
    const uint2 *idx = static_cast<const uint2 *>(t.d_idx);
    if (L.threads == 512)
        k_hs_bc<512><<<L.grid, 512, L.dyn, s>>>(f, bc, ncells, nv, t.trials, idx, t.d_b, L.per, list, count, status);
    else
        k_hs_bc<256><<<L.grid, 256, L.dyn, s>>>(f, bc, ncells, nv, t.trials, idx, t.d_b, L.per, list, count, status);
    count_launch();
    return cudaGetLastError() == cudaSuccess ? DVM_OK : DVM_ECUDA;
}

int launch_hs_collide(HsTables &t, const StepParams &p, void *f, double kn, double dt)
{
    if (p.prec != DVM_F32) return DVM_ENOTIMPL;
    if (!t.ready || t.nv != p.nv || !t.d_bc) return DVM_ESTATE;
    BcLaunch L;
    int rc = bc_plan(t, p.nv, p.ncells, L);
    if (!rc)
        rc = bc_launch(L, t, static_cast<const float *>(f), reinterpret_cast<float2 *>(t.d_bc), p.ncells, p.nv,
                       nullptr, nullptr, p.stream, p.status);
    if (rc) return rc;
    k_hs_corr<<<(unsigned)p.ncells, CT, 0, p.stream>>>(static_cast<float *>(f),
                                                      reinterpret_cast<const float2 *>(t.d_bc), t.d_xi, t.d_jpk,
                                                      t.hh, p.dV, p.mom_out, p.nv,
                                                      make_int3(t.half[0], t.half[1], t.half[2]), (float)(dt / kn),
                                                      nullptr, nullptr, nullptr, p.res_out, p.status);
    count_launch();
    return cudaGetLastError() == cudaSuccess ? DVM_OK : DVM_ECUDA;
}

// The update on the cells of a device list only (*count entries, at most
// p.ncells), or, with q_out, the term I of every cell without the update.
int launch_hs_general(HsTables &t, const StepParams &p, float *f, const int32_t *list, const int *count,
                      float *q_out, double kn, double dt)
{
    if (p.prec != DVM_F32) return DVM_ENOTIMPL;
    if (!t.ready || t.nv != p.nv || !t.d_bc || t.bc_cells < p.ncells) return DVM_ESTATE;
    if (p.ncells <= 0) return DVM_OK;
    BcLaunch L;
    int rc = bc_plan(t, p.nv, p.ncells, L);
    if (!rc)
        rc = bc_launch(L, t, f, reinterpret_cast<float2 *>(t.d_bc), p.ncells, p.nv, list, count, p.stream,
                       p.status);
    if (rc) return rc;
    k_hs_corr<<<(unsigned)p.ncells, CT, 0, p.stream>>>(f, reinterpret_cast<const float2 *>(t.d_bc), t.d_xi,
                                                      t.d_jpk, t.hh, p.dV, p.mom_out, p.nv,
                                                      make_int3(t.half[0], t.half[1], t.half[2]),
                                                      q_out ? 0.0f : (float)(dt / kn), list, count, q_out,
                                                      q_out ? nullptr : p.res_out, p.status);
    count_launch();
    return cudaGetLastError() == cudaSuccess ? DVM_OK : DVM_ECUDA;
}

// ---------------------------------------------------------------- allocation-free variant
namespace {

// Fixed scratch for dvm_hs_collide_noalloc.  It is part of the library's
// device image, so every GPU that loads the library holds it until the
// process exits; all calls share it.
constexpr size_t NOALLOC_BYTES = (size_t)DVM_HS_NOALLOC_SCRATCH_BYTES;
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];

std::mutex g_noalloc_mu;
struct NoallocSlot {
    void *ctx = nullptr;  // the context the address belongs to
    void *ptr = nullptr;
};
NoallocSlot g_noalloc[256];

// The calling thread's current context (a CUcontext), through the driver
// entry point that the runtime hands out; null if it cannot be had.  Called
// with g_noalloc_mu held.
void *current_context()
{
    using Fn = int (*)(void **);
    static Fn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<Fn>(f);
        else
            cudaGetLastError();
    }
    void *ctx = nullptr;
    if (!fn || fn(&ctx) != 0) return nullptr;
    return ctx;
}

// Device address of the fixed scratch on the current device.  In host code
// g_noalloc_scratch names a host-side stand-in, so the address is looked up
// with the device current: once per device, and again if the device's
// context has been re-created since (after cudaDeviceReset the old address
// is stale).
int noalloc_scratch(void **ptr)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) {
        cudaGetLastError();
        return DVM_ECUDA;
    }
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    NoallocSlot &slot = g_noalloc[dev];
    void *ctx = current_context();
    if (!slot.ptr || !ctx || slot.ctx != ctx) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return DVM_ECUDA;
        }
        slot.ptr = p;
        slot.ctx = current_context();  // the lookup has made the context current
    }
    *ptr = slot.ptr;
    return DVM_OK;
}

}  // namespace

int launch_hs_collide_noalloc(HsTables &t, const StepParams &p, float *f, const double *xi, double dV,
                              double kn, double dt)
{
    if (p.prec != DVM_F32) return DVM_ENOTIMPL;
    if (!t.ready || t.nv != p.nv) return DVM_ESTATE;
    const size_t need_bc = (size_t)p.ncells * p.nv * 2 * sizeof(float);
    if (need_bc + (size_t)p.ncells * 5 * sizeof(double) > NOALLOC_BYTES) return DVM_EINVAL;
    // every check comes before the first launch, so that a refusal queues no work
    BcLaunch L;
    int rc = bc_plan(t, p.nv, p.ncells, L);
    if (rc) return rc;
    void *base = nullptr;
    rc = noalloc_scratch(&base);
    if (rc) return rc;
    float *bc = static_cast<float *>(base);
    double *mom = reinterpret_cast<double *>(static_cast<unsigned char *>(base) + need_bc);
    rc = launch_moments(DVM_F32, f, p.ncells, p.nv, xi, dV, mom, p.stream);
    if (rc) return rc;
    rc = bc_launch(L, t, f, reinterpret_cast<float2 *>(bc), p.ncells, p.nv, nullptr, nullptr, p.stream, p.status);
    if (rc) return rc;
    k_hs_corr<<<(unsigned)p.ncells, CT, 0, p.stream>>>(f, reinterpret_cast<const float2 *>(bc), t.d_xi, t.d_jpk,
                                                      t.hh, dV, mom, p.nv, make_int3(t.half[0], t.half[1], t.half[2]),
                                                      (float)(dt / kn), nullptr, nullptr, nullptr, nullptr, p.status);
    count_launch();
    return cudaGetLastError() == cudaSuccess ? DVM_OK : DVM_ECUDA;
}

}  // namespace dvm
