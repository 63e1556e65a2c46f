// Lattice Boltzmann step on the tree (paper Sec. 4): finite-volume upwind
// transport of Eq. 2 on the lattice velocities, then the lattice BGK
// relaxation towards the second-order equilibrium, fused in one pass over f.
//
// Layout: f is [q][ld] (structure of arrays: velocity i of every cell is one
// contiguous row; column ncells holds the inflow ghost), so one thread per
// cell reads and writes each of its q values with fully coalesced warp
// accesses.  The upwind codes are [2 dim][ncells], also coalesced.  Upwind
// neighbours are gathered from the same rows: cells near in Morton order
// are near in the rows, so the gathers hit L1/L2.
#include <cuda_runtime.h>

#include <type_traits>

#include "../../include/dvm.h"
#include "lbm.hpp"

namespace dvm {

void count_launch();

namespace {

// The velocity set as compile-time tables (same rule as lbm_lattice: order
// by |c|^2, then lexicographic in (c_x, c_y, c_z)).
struct LatTab {
    int q = 0;
    int c[27][3] = {};
    int r2[27] = {};
    int mirror[27][3] = {};  // index of the velocity with component d negated
};

__host__ __device__ constexpr LatTab make_tab(int Q)
{
    LatTab t{};
    for (int r2 = 0; r2 <= 3; r2++)
        for (int x = -1; x <= 1; x++)
            for (int y = -1; y <= 1; y++)
                for (int z = -1; z <= 1; z++) {
                    if (x * x + y * y + z * z != r2) continue;
                    if (Q == 9 && z != 0) continue;
                    if (Q == 19 && r2 == 3) continue;
                    t.c[t.q][0] = x;
                    t.c[t.q][1] = y;
                    t.c[t.q][2] = z;
                    t.r2[t.q] = r2;
                    t.q++;
                }
    for (int i = 0; i < t.q; i++)
        for (int d = 0; d < 3; d++)
            for (int j = 0; j < t.q; j++) {
                bool same = true;
                for (int e = 0; e < 3; e++)
                    same = same && t.c[j][e] == (e == d ? -t.c[i][e] : t.c[i][e]);
                if (same) t.mirror[i][d] = j;
            }
    return t;
}

template <int Q> struct Lat {
    static constexpr LatTab t = make_tab(Q);
};

// every mirror exists, is an involution and negates exactly one component
__host__ __device__ constexpr bool tab_ok(int Q)
{
    const LatTab t = make_tab(Q);
    if (t.q != Q) return false;
    for (int i = 0; i < t.q; i++)
        for (int d = 0; d < 3; d++) {
            const int j = t.mirror[i][d];
            if (t.mirror[j][d] != i) return false;
            for (int e = 0; e < 3; e++)
                if (t.c[j][e] != (e == d ? -t.c[i][e] : t.c[i][e])) return false;
        }
    return true;
}
static_assert(tab_ok(9) && tab_ok(19) && tab_ok(27), "lattice tables");

// weight of |c|^2 class r2, exact quotients of small integers
template <typename T, int Q> __device__ constexpr T lat_w(int r2)
{
    if (Q == 9) return r2 == 0 ? T(4) / T(9) : r2 == 1 ? T(1) / T(9) : T(1) / T(36);
    if (Q == 19) return r2 == 0 ? T(1) / T(3) : r2 == 1 ? T(1) / T(18) : T(1) / T(36);
    return r2 == 0 ? T(8) / T(27) : r2 == 1 ? T(2) / T(27) : r2 == 2 ? T(1) / T(54) : T(1) / T(216);
}

// compile-time loop over velocities
template <int I, int Q> struct ForV {
    template <typename F> __device__ __forceinline__ static void run(F &&f)
    {
        f(std::integral_constant<int, I>{});
        ForV<I + 1, Q>::run(f);
    }
};
template <int Q> struct ForV<Q, Q> {
    template <typename F> __device__ __forceinline__ static void run(F &&) {}
};

// the side list (2d + s) whose sources velocity i takes along axis d: the
// minus side for c_d > 0, the plus side for c_d < 0
template <int Q> __host__ __device__ constexpr int side_of(int i, int d)
{
    return Lat<Q>::t.c[i][d] > 0 ? 2 * d : 2 * d + 1;
}

// compile-time loop over the 2 dim sides
template <int K, int NS> struct ForS {
    template <typename F> __device__ __forceinline__ static void run(F &&f)
    {
        f(std::integral_constant<int, K>{});
        ForS<K + 1, NS>::run(f);
    }
};
template <int NS> struct ForS<NS, NS> {
    template <typename F> __device__ __forceinline__ static void run(F &&) {}
};

// g_i += w f_e for every velocity i that takes side K, f_e the source's
// value of velocity i (or of its mirror along the side's axis for a wall)
template <typename T, int Q, int K>
__device__ __forceinline__ void add_side(T (&g)[Q], const T *__restrict__ fin, int64_t ld, int64_t src, bool wall,
                                         T w)
{
    constexpr int d = K / 2;
    ForV<0, Q>::run([&](auto II) {
        constexpr int i = decltype(II)::value;
        if constexpr (Lat<Q>::t.c[i][d] != 0 && side_of<Q>(i, d) == K) {
            constexpr int jm = Lat<Q>::t.mirror[i][d];
            g[i] += w * __ldg(fin + (int64_t)(wall ? jm : i) * ld + src);
        }
    });
}

// Fused step.  Every side's first source is decoded once (a side with
// several finer sources starts from its first overflow entry), and all
// first-source gathers are issued without branches, so a thread keeps its
// gathers in flight together; the remaining entries of sides with 2 or 4
// finer sources are added in a second pass that few threads take.
// CTAs of 256 threads per SM that the register budget is sized for: more
// registers keep more of a thread's gathers in flight, more CTAs hide more
// latency
__host__ __device__ constexpr int lbm_min_blocks(int Q, int tsize)
{
    return tsize == 8 ? 2 : Q == 27 ? 3 : Q == 19 ? 4 : 4;
}

template <typename T, int DIM, int Q>
__global__ void __launch_bounds__(256, lbm_min_blocks(Q, sizeof(T))) k_lbm(const LbmParams p)
{
    const int64_t cell = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (cell >= p.ncells) return;
    const T *__restrict__ fin = static_cast<const T *>(p.f_in);
    T *__restrict__ fout = static_cast<T *>(p.f_out);
    const int64_t ld = p.ld, nc = p.ncells;
    constexpr int NS = 2 * DIM;
    uint32_t code[NS];
#pragma unroll
    for (int k = 0; k < NS; k++) code[k] = __ldg(p.codes + (int64_t)k * nc + cell);
    // dt / h and dt / (2^(dim-1) h), h = 2^-level
    const T dth = T(p.dt) * T(1ull << __ldg(p.lev + cell));
    const T dtq = dth * (T(1) / T(1 << (DIM - 1)));
    // f_i (1 - dt n_i / h), n_i the number of non-zero components of c_i
    T g[Q];
    ForV<0, Q>::run([&](auto II) {
        constexpr int i = decltype(II)::value;
        constexpr int cx = Lat<Q>::t.c[i][0], cy = Lat<Q>::t.c[i][1], cz = Lat<Q>::t.c[i][2];
        constexpr int na = (cx != 0) + (cy != 0) + (DIM == 3 && cz != 0);
        const T v = __ldg(fin + (int64_t)i * ld + cell);
        g[i] = v - dth * T(na) * v;
    });
    // transport, Eq. 2: add dt m_e f_e / (2^(dim-1) h) over each upwind
    // side's sources, first sources for all sides at once
    bool any_ovf = false;
    ForS<0, NS>::run([&](auto KK) {
        constexpr int k = decltype(KK)::value;
        uint32_t e = code[k];
        if (e & LBM_OVF) {
            any_ovf = true;
            e = __ldg(p.ovf + (e & LBM_CELL));
        }
        add_side<T, Q, k>(g, fin, ld, e & LBM_CELL, (e & LBM_WALL) != 0,
                          dtq * T((int)((e >> LBM_M_SHIFT) & 3u) + 1));
    });
    if (any_ovf) {
        ForS<0, NS>::run([&](auto KK) {
            constexpr int k = decltype(KK)::value;
            if (code[k] & LBM_OVF) {
                const uint32_t base = code[k] & LBM_CELL;
                const int n = (int)((code[k] >> LBM_M_SHIFT) & 3u) + 1;
                for (int j = 1; j < n; j++) {
                    const uint32_t e = __ldg(p.ovf + base + j);
                    add_side<T, Q, k>(g, fin, ld, e & LBM_CELL, (e & LBM_WALL) != 0,
                                      dtq * T((int)((e >> LBM_M_SHIFT) & 3u) + 1));
                }
            }
        });
    }
    // moments of f*
    T rho = T(0), jx = T(0), jy = T(0), jz = T(0);
    ForV<0, Q>::run([&](auto II) {
        constexpr int i = decltype(II)::value;
        constexpr int cx = Lat<Q>::t.c[i][0], cy = Lat<Q>::t.c[i][1], cz = Lat<Q>::t.c[i][2];
        rho += g[i];
        if constexpr (cx > 0) jx += g[i];
        if constexpr (cx < 0) jx -= g[i];
        if constexpr (cy > 0) jy += g[i];
        if constexpr (cy < 0) jy -= g[i];
        if constexpr (cz > 0) jz += g[i];
        if constexpr (cz < 0) jz -= g[i];
    });
    const T irho = T(1) / rho;
    const T ux = jx * irho, uy = jy * irho, uz = jz * irho;
    if (!(rho > T(0)) || !isfinite(ux + uy + uz)) atomicOr(p.status, 1);
    const T om = T(p.omega);
    const T q0 = T(1) - T(1.5) * (ux * ux + uy * uy + uz * uz);
    // BGK towards feq_i = w_i rho (1 + 3 c.u + 4.5 (c.u)^2 - 1.5 |u|^2)
    ForV<0, Q>::run([&](auto II) {
        constexpr int i = decltype(II)::value;
        constexpr int cx = Lat<Q>::t.c[i][0], cy = Lat<Q>::t.c[i][1], cz = Lat<Q>::t.c[i][2];
        constexpr int r2 = Lat<Q>::t.r2[i];
        const T cu = T(cx) * ux + T(cy) * uy + T(cz) * uz;
        const T feq = lat_w<T, Q>(r2) * rho * (q0 + cu * (T(3) + T(4.5) * cu));
        fout[(int64_t)i * ld + cell] = g[i] - om * (g[i] - feq);
    });
}

template <typename T, int Q>
__global__ void __launch_bounds__(256) k_lbm_moments(const T *__restrict__ f, int64_t ncells, int64_t ld,
                                                     double *__restrict__ out)
{
    const int64_t cell = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (cell >= ncells) return;
    double rho = 0, j[3] = {0, 0, 0};
    ForV<0, Q>::run([&](auto II) {
        constexpr int i = decltype(II)::value;
        constexpr int cx = Lat<Q>::t.c[i][0], cy = Lat<Q>::t.c[i][1], cz = Lat<Q>::t.c[i][2];
        const double v = (double)f[(int64_t)i * ld + cell];
        rho += v;
        j[0] += cx * v;
        j[1] += cy * v;
        j[2] += cz * v;
    });
    out[cell * 4] = rho;
    for (int d = 0; d < 3; d++) out[cell * 4 + 1 + d] = j[d] / rho;
}

template <typename T, int DIM, int Q> int launch_t(const LbmParams &p)
{
    const int64_t blocks = (p.ncells + 255) / 256;
    k_lbm<T, DIM, Q><<<(unsigned)blocks, 256, 0, p.stream>>>(p);
    count_launch();
    return cudaGetLastError() == cudaSuccess ? DVM_OK : DVM_ECUDA;
}

template <typename T> int launch_prec(const LbmParams &p)
{
    if (p.dim == 2 && p.q == 9) return launch_t<T, 2, 9>(p);
    if (p.dim == 3 && p.q == 19) return launch_t<T, 3, 19>(p);
    if (p.dim == 3 && p.q == 27) return launch_t<T, 3, 27>(p);
    return DVM_EINVAL;
}

template <typename T>
int launch_mom_t(int q, const void *f, int64_t ncells, int64_t ld, double *out, cudaStream_t s)
{
    const unsigned blocks = (unsigned)((ncells + 255) / 256);
    const T *ft = static_cast<const T *>(f);
    if (q == 9) k_lbm_moments<T, 9><<<blocks, 256, 0, s>>>(ft, ncells, ld, out);
    else if (q == 19) k_lbm_moments<T, 19><<<blocks, 256, 0, s>>>(ft, ncells, ld, out);
    else if (q == 27) k_lbm_moments<T, 27><<<blocks, 256, 0, s>>>(ft, ncells, ld, out);
    else return DVM_EINVAL;
    count_launch();
    return cudaGetLastError() == cudaSuccess ? DVM_OK : DVM_ECUDA;
}

}  // namespace

int launch_lbm(const LbmParams &p)
{
    if (p.ncells <= 0) return DVM_OK;
    if (p.prec == DVM_F64) return launch_prec<double>(p);
    if (p.prec == DVM_F32) return launch_prec<float>(p);
    return DVM_ENOTIMPL;
}

int launch_lbm_moments(int prec, int q, const void *f, int64_t ncells, int64_t ld, double *out, cudaStream_t s)
{
    if (ncells <= 0) return DVM_OK;
    if (prec == DVM_F64) return launch_mom_t<double>(q, f, ncells, ld, out, s);
    if (prec == DVM_F32) return launch_mom_t<float>(q, f, ncells, ld, out, s);
    return DVM_ENOTIMPL;
}

}  // namespace dvm
