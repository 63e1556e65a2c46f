// Host construction of the hard-sphere trial tables for Eqs. 3-5.
//
// For node i and trial k (stream index s = i*M + k, SplitMix64 draws 3s,
// 3s+1, 3s+2): the partner gamma is uniform over the Nv nodes; the unit
// vector omega has z = 2u - 1 and azimuth 2 pi u'.  The lattice variant (the
// Korobov-grid quadrature the paper cites for the collision integral, Ref.
// [5]) takes the five coordinates of point k of a rank-1 lattice with
// generator (1, a, a^2, a^3, a^4) mod M, shifted per node by SplitMix64
// draws 5i .. 5i+4 modulo 1: the partner is the node whose axis indices are
// floor(u_d n_d), and omega comes from the last two coordinates.  The post-collision pair
// xi' = c + |g| omega / 2, xi'_* = c - |g| omega / 2 around the pair's mean c
// is snapped to the nearest nodes l, m (round half away from zero); a trial
// whose l or m falls off the grid contributes nothing.  The weights
// b = c = Nv dV |g| / (sqrt(2) M) are the Monte-Carlo weights of the
// hard-sphere integral (1/(4 sqrt(2) pi)) int int (f'f'_* - f f_*)|g| dOmega
// dxi_*, normalised so that a unit Maxwellian has mean collision frequency
// sqrt(8/pi) (mean free path Kn).
#include "hs.hpp"

#include <algorithm>
#include <atomic>
#include <climits>
#include <cmath>
#include <cstring>
#include <thread>

#include "../../include/dvm.h"

namespace dvm {

uint64_t splitmix64_at(uint64_t seed, uint64_t n)
{
    uint64_t x = seed + (n + 1) * 0x9E3779B97F4A7C15ull;
    x ^= x >> 30;
    x *= 0xBF58476D1CE4E5B9ull;
    x ^= x >> 27;
    x *= 0x94D049BB133111EBull;
    x ^= x >> 31;
    return x;
}

static double uniform01(uint64_t seed, uint64_t n)
{
    return std::ldexp((double)(splitmix64_at(seed, n) >> 11), -53);
}

int64_t korobov_multiplier(int64_t M)
{
    // the odd a whose lattice has the largest smallest torus distance between
    // points (integer squared distances in units of 1/M^2), smallest a on ties
    int64_t best = 1, best_sep = -1;
    for (int64_t a = 1; a < M; a += 2) {
        int64_t gen[5] = {1, 0, 0, 0, 0};
        for (int j = 1; j < 5; j++) gen[j] = gen[j - 1] * a % M;
        int64_t sep = INT64_MAX;
        for (int64_t k = 1; k < M && sep > best_sep; k++) {
            int64_t s2 = 0;
            for (int j = 0; j < 5; j++) {
                const int64_t r = k * gen[j] % M;
                const int64_t t = std::min(r, M - r);
                s2 += t * t;
            }
            sep = std::min(sep, s2);
        }
        if (sep > best_sep) {
            best_sep = sep;
            best = a;
        }
    }
    return best;
}

// Device order of the trials.  The collision kernel gives each node's
// trials to trials/32 lanes (lane t of the node takes trials 32 t .. 32 t + 31,
// one per slot) and a warp covers 32 / (trials/32) consecutive nodes; at each
// slot its lanes gather f at three node indices (gamma, l, m) from a
// shared-memory tile, and every distinct index in the same bank (index mod 32)
// costs one more shared-memory wavefront.  The sums B and C over a node's
// trials do not depend on their order, so the order is chosen per warp to
// keep those wavefronts few:
//   1. greedily, slot by slot: each lane takes, from its node's remaining
//      trials, the one that adds the fewest distinct indices to banks already
//      in use at this slot (over the three gathers);
//   2. then by local search: swaps of two trials of one node between two
//      slots, kept when they lower the slots' wavefronts (the largest count
//      of distinct indices in a bank, summed over the three gathers) or keep
//      them and spread the indices more evenly over the banks.  Each warp's
//      search draws from its own seeded stream, so the order does not depend
//      on the host threads that run the warps in parallel.
// On the 16^3 and 24^3 grids with 128 trials the mean wavefronts per gather
// go from 3.0 (seeded order) to 1.85 (greedy) to about 1.55.
//
// About 40% of the trials carry no weight (b = 0: post-collision velocities
// off the grid, or gamma = i).  Within a warp they are placed last: the
// weighted trials of every node fill the first R slots of its lanes, R =
// ceil(largest weighted count of the warp's nodes / lanes per node).  The
// zero-weight trials that fill a node's share of those R slots (fillers)
// gather at addresses another lane of the slot already loads, so they cost
// no wavefront, and the slots from R on gather at the warp's own consecutive
// nodes, one wavefront each.  Mean wavefronts per gather over all 32 slots:
// about 1.35 (16^3 and 24^3, 128 trials), against 1.55 with the zero-weight
// trials placed like the others (the kernel still runs every slot: stopping
// each warp after its R slots measured slower).
namespace {

struct BankSlot {
    // per gather and bank: the distinct indices of the slot and how many
    // lanes take each
    int cnt[3][32];
    int addr[3][32][32];
    int mult[3][32][32];
    void clear()
    {
        for (int g = 0; g < 3; g++)
            for (int k = 0; k < 32; k++) cnt[g][k] = 0;
    }
    void add(const int a3[3], int sgn)
    {
        for (int g = 0; g < 3; g++) {
            const int a = a3[g], bk = a & 31;
            int pos = -1;
            for (int q = 0; q < cnt[g][bk]; q++)
                if (addr[g][bk][q] == a) pos = q;
            if (sgn > 0) {
                if (pos < 0) {
                    pos = cnt[g][bk]++;
                    addr[g][bk][pos] = a;
                    mult[g][bk][pos] = 0;
                }
                mult[g][bk][pos]++;
            } else if (--mult[g][bk][pos] == 0) {
                const int last = --cnt[g][bk];
                addr[g][bk][pos] = addr[g][bk][last];
                mult[g][bk][pos] = mult[g][bk][last];
            }
        }
    }
    // wavefronts over the three gathers, and the sum of squared bank loads
    void cost(int &w, int &sq) const
    {
        w = 0;
        sq = 0;
        for (int g = 0; g < 3; g++) {
            int mx = 1;
            for (int k = 0; k < 32; k++) {
                mx = std::max(mx, cnt[g][k]);
                sq += cnt[g][k] * cnt[g][k];
            }
            w += mx;
        }
    }
    // distinct indices the trial would add to occupied banks
    int added(const int a3[3]) const
    {
        int c = 0;
        for (int g = 0; g < 3; g++) {
            const int a = a3[g], bk = a & 31;
            bool seen = false;
            for (int q = 0; q < cnt[g][bk]; q++) seen = seen || addr[g][bk][q] == a;
            if (!seen) c += cnt[g][bk];
        }
        return c;
    }
};

inline uint64_t mix64(uint64_t x)
{
    x += 0x9e3779b97f4a7c15ull;
    x = (x ^ (x >> 30)) * 0xbf58476d1ce4e5b9ull;
    x = (x ^ (x >> 27)) * 0x94d049bb133111ebull;
    return x ^ (x >> 31);
}

// The order of the warp whose first node is g0: ord[node * M + t * 32 + e] is
// the trial (of that node) that lane t of the node takes at slot e.  Returns
// R, the slots the warp runs: every weighted trial of its nodes sits at a
// slot e < R.
int order_warp(const std::vector<uint32_t> &idx, const std::vector<float> &b, int nv, int M, int g0, int iters,
               std::vector<int> &ord)
{
    const int HEt = 32, tpn = M / HEt, K = 32 / tpn;
    const int kn = std::min(K, nv - g0);
    auto weighted = [&](int nl, int k) { return b[(size_t)(g0 + nl) * M + k] != 0.0f; };
    // a weighted trial's three gather addresses; false for a zero-weight one
    auto trial = [&](int nl, int k, int a3[3]) -> bool {
        if (!weighted(nl, k)) return false;
        const size_t q = (size_t)(g0 + nl) * M + k;
        const uint32_t w0 = idx[2 * q], w1 = idx[2 * q + 1];
        a3[0] = (int)(w0 & 0xffffu);
        a3[1] = (int)(w0 >> 16);
        a3[2] = (int)w1;
        return true;
    };
    int kmax = 0;
    for (int nl = 0; nl < kn; nl++) {
        int c = 0;
        for (int k = 0; k < M; k++) c += weighted(nl, k);
        kmax = std::max(kmax, c);
    }
    const int R = (kmax + tpn - 1) / tpn;
    std::vector<BankSlot> S(HEt);
    std::vector<uint8_t> used((size_t)kn * M, 0);
    int a3[3];
    for (int e = 0; e < HEt; e++) {
        S[e].clear();
        for (int lane = 0; lane < kn * tpn; lane++) {
            const int nl = lane / tpn, t = lane % tpn;
            // slots e < R: the weighted trial that adds the fewest distinct
            // addresses to occupied banks, else a zero-weight filler; later
            // slots: the zero-weight trials left
            int best = -1, bestc = INT_MAX;
            for (int k = 0; k < M && bestc > 0; k++) {
                if (used[(size_t)nl * M + k] || !trial(nl, k, a3)) continue;
                const int c = S[e].added(a3);
                if (c < bestc) {
                    bestc = c;
                    best = k;
                }
            }
            if (best < 0)
                for (int k = 0; k < M && best < 0; k++)
                    if (!used[(size_t)nl * M + k]) best = k;
            used[(size_t)nl * M + best] = 1;
            if (trial(nl, best, a3)) S[e].add(a3, +1);
            ord[(size_t)(g0 + nl) * M + t * HEt + e] = best;
        }
    }
    int W[32], Q[32];
    for (int e = 0; e < HEt; e++) S[e].cost(W[e], Q[e]);
    uint64_t st = mix64(0x5eed0000ull + (uint64_t)g0);
    int b1[3], b2[3];
    for (int it = 0; it < iters && R > 1; it++) {
        st = mix64(st);
        // two of the node's slots below R
        const int nl = (int)(st % (uint64_t)kn);
        const int e1 = (int)((st >> 16) % (uint64_t)R), e2 = (int)((st >> 32) % (uint64_t)R);
        const int t1 = (int)((st >> 48) % (uint64_t)tpn), t2 = (int)((st >> 56) % (uint64_t)tpn);
        if (e1 == e2) continue;
        const int p1 = t1 * HEt + e1, p2 = t2 * HEt + e2;
        int *o1 = &ord[(size_t)(g0 + nl) * M + p1], *o2 = &ord[(size_t)(g0 + nl) * M + p2];
        const bool h1 = trial(nl, *o1, b1), h2 = trial(nl, *o2, b2);
        if (!h1 && !h2) continue;
        if (h1) S[e1].add(b1, -1);
        if (h2) S[e2].add(b2, -1);
        if (h2) S[e1].add(b2, +1);
        if (h1) S[e2].add(b1, +1);
        int w1, q1, w2, q2;
        S[e1].cost(w1, q1);
        S[e2].cost(w2, q2);
        const int dw = w1 + w2 - W[e1] - W[e2], dq = q1 + q2 - Q[e1] - Q[e2];
        if (dw < 0 || (dw == 0 && dq <= 0)) {
            std::swap(*o1, *o2);
            W[e1] = w1;
            Q[e1] = q1;
            W[e2] = w2;
            Q[e2] = q2;
        } else {
            if (h2) S[e1].add(b2, -1);
            if (h1) S[e2].add(b1, -1);
            if (h1) S[e1].add(b1, +1);
            if (h2) S[e2].add(b2, +1);
        }
    }
    return R;
}

}  // namespace

// idx/b: node-major tables as built; out_idx/out_b: the same entries in
// device order, the addresses of zero-weight trials below a warp's R slots
// replaced by those of a weighted lane of the same slot.
static void order_for_banks(const std::vector<uint32_t> &idx, const std::vector<float> &b, int nv, int M,
                            std::vector<uint32_t> &out_idx, std::vector<float> &out_b)
{
    const int HEt = 32, tpn = M / HEt, K = 32 / tpn;
    const int nwarps = (nv + K - 1) / K;
    std::vector<int> ord((size_t)nv * M);
    std::vector<uint8_t> rounds((size_t)nwarps, 0);
    const int iters = 60 * M * K;  // ~60 tries per trial of the warp
    const int nth = (int)std::max(1u, std::min(32u, std::thread::hardware_concurrency()));
    std::atomic<int> next{0};
    auto work = [&]() {
        for (int w = next++; w < nwarps; w = next++) rounds[w] = (uint8_t)order_warp(idx, b, nv, M, w * K, iters, ord);
    };
    std::vector<std::thread> pool;
    for (int i = 1; i < nth; i++) pool.emplace_back(work);
    work();
    for (auto &th : pool) th.join();
    out_idx.assign(idx.size(), 0u);
    out_b.assign(b.size(), 0.0f);
    for (int node = 0; node < nv; node++)
        for (int p = 0; p < M; p++) {
            const size_t src = (size_t)node * M + ord[(size_t)node * M + p], dst = (size_t)node * M + p;
            out_idx[2 * dst] = idx[2 * src];
            out_idx[2 * dst + 1] = idx[2 * src + 1];
            out_b[dst] = b[src];
        }
    // fillers: at each slot below R, a zero-weight trial takes the addresses of
    // the slot's first weighted lane (a repeated address costs no wavefront)
    for (int w = 0; w < nwarps; w++) {
        const int g0 = w * K, kn = std::min(K, nv - g0);
        for (int e = 0; e < rounds[w]; e++) {
            size_t ref = SIZE_MAX;
            for (int lane = 0; lane < kn * tpn && ref == SIZE_MAX; lane++) {
                const size_t q = (size_t)(g0 + lane / tpn) * M + (lane % tpn) * HEt + e;
                if (out_b[q] != 0.0f) ref = q;
            }
            if (ref == SIZE_MAX) continue;
            for (int lane = 0; lane < kn * tpn; lane++) {
                const size_t q = (size_t)(g0 + lane / tpn) * M + (lane % tpn) * HEt + e;
                if (out_b[q] == 0.0f) {
                    out_idx[2 * q] = out_idx[2 * ref];
                    out_idx[2 * q + 1] = out_idx[2 * ref + 1];
                }
            }
        }
    }
}

void hs_free(HsTables &t, const DevFree &dfree)
{
    if (t.d_idx) dfree(t.d_idx);
    if (t.d_b) dfree(t.d_b);
    if (t.d_xi) dfree(t.d_xi);
    if (t.d_jpk) dfree(t.d_jpk);
    if (t.d_bc) dfree(t.d_bc);
    t.d_idx = nullptr;
    t.d_b = nullptr;
    t.d_xi = nullptr;
    t.d_jpk = nullptr;
    t.d_bc = nullptr;
    t.bc_cells = 0;
    t.ready = false;
}

int hs_build(HsTables &t, const int n[3], const double lo[3], const double h[3],
             const std::vector<double> &xi, int trials, uint64_t seed, bool lattice, std::string &err,
             const DevAlloc &alloc, const DevFree &dfree)
{
    hs_free(t, dfree);
    const int nv = n[0] * n[1] * n[2];
    if (nv > 65535) { err = "hard-sphere tables need Nv < 65536"; return DVM_ENOTIMPL; }
    // the correction's exact integer basis (1, j, |j|^2) needs one spacing on
    // every axis and |j|^4 < 2^24 (n <= 32)
    if (h[0] != h[1] || h[0] != h[2] || n[0] > 32 || n[1] > 32 || n[2] > 32) {
        err = "hard-sphere collisions need the same velocity spacing on every axis and n <= 32";
        return DVM_ENOTIMPL;
    }
    if (!hs_trials_supported(trials)) {
        err = "trials per node must be 32, 64, ..., 1024 (a power-of-two multiple of 32)";
        return DVM_ENOTIMPL;
    }
    // natural (kx, ky, kz) -> storage index
    std::vector<int32_t> where((size_t)nv, -1);
    for (int v = 0; v < nv; v++) {
        int k[3];
        for (int d = 0; d < 3; d++) k[d] = (int)std::lround((xi[3 * (size_t)v + d] - lo[d]) / h[d] - 0.5);
        where[((size_t)k[0] * n[1] + k[1]) * n[2] + k[2]] = v;
    }
    const double dV = h[0] * h[1] * h[2];
    const double scale = (double)nv * dV / (std::sqrt(2.0) * (double)trials);
    t.host_idx.assign((size_t)trials * nv * 2, 0u);
    t.host_b.assign((size_t)trials * nv, 0.0f);
    t.discarded = 0;
    int64_t gen[5] = {1, 0, 0, 0, 0};
    if (lattice) {
        const int64_t am = korobov_multiplier(trials);
        for (int j = 1; j < 5; j++) gen[j] = gen[j - 1] * am % trials;
    }
    for (int i = 0; i < nv; i++) {
        const double *a = &xi[3 * (size_t)i];
        double shift[5] = {0, 0, 0, 0, 0};
        if (lattice)
            for (int j = 0; j < 5; j++) shift[j] = uniform01(seed, 5 * (uint64_t)i + (uint64_t)j);
        for (int k = 0; k < trials; k++) {
            int gam;
            double u1, u2;
            if (lattice) {
                double u[5];
                for (int j = 0; j < 5; j++) {
                    u[j] = (double)((int64_t)k * gen[j] % trials) / (double)trials + shift[j];
                    if (u[j] >= 1.0) u[j] -= 1.0;
                }
                int ax[3];
                for (int d = 0; d < 3; d++) ax[d] = std::min((int)(u[d] * (double)n[d]), n[d] - 1);
                gam = where[((size_t)ax[0] * n[1] + ax[1]) * n[2] + ax[2]];
                u1 = u[3];
                u2 = u[4];
            } else {
                const uint64_t s = (uint64_t)i * (uint64_t)trials + (uint64_t)k;
                gam = (int)(uniform01(seed, 3 * s) * (double)nv);
                u1 = uniform01(seed, 3 * s + 1);
                u2 = uniform01(seed, 3 * s + 2);
            }
            const double *b = &xi[3 * (size_t)gam];
            double g2 = 0.0;
            for (int d = 0; d < 3; d++) g2 += (a[d] - b[d]) * (a[d] - b[d]);
            const double gn = std::sqrt(g2);
            const double z = 2.0 * u1 - 1.0, phi = 2.0 * M_PI * u2;
            const double st = std::sqrt(std::fmax(0.0, 1.0 - z * z));
            const double om[3] = {st * std::cos(phi), st * std::sin(phi), z};
            int kp[3], kq[3];
            bool ok = true;
            for (int d = 0; d < 3 && ok; d++) {
                const double mid = 0.5 * (a[d] + b[d]);
                const double xp = mid + 0.5 * gn * om[d], xq = mid - 0.5 * gn * om[d];
                const double tp = std::round((xp - lo[d]) / h[d] - 0.5);
                const double tq = std::round((xq - lo[d]) / h[d] - 0.5);
                if (!(tp >= 0.0) || tp > n[d] - 1 || !(tq >= 0.0) || tq > n[d] - 1) ok = false;
                else { kp[d] = (int)tp; kq[d] = (int)tq; }
            }
            const size_t q = (size_t)i * trials + k;
            uint32_t *e = &t.host_idx[2 * q];
            if (!ok) {
                t.discarded++;
                e[0] = (uint32_t)i | ((uint32_t)i << 16);
                e[1] = (uint32_t)i;
                t.host_b[q] = 0.0f;
                continue;
            }
            const int l = where[((size_t)kp[0] * n[1] + kp[1]) * n[2] + kp[2]];
            const int m = where[((size_t)kq[0] * n[1] + kq[1]) * n[2] + kq[2]];
            e[0] = (uint32_t)gam | ((uint32_t)l << 16);
            e[1] = (uint32_t)m;
            t.host_b[q] = (float)(scale * gn);
        }
    }
    std::vector<float> xf(3 * (size_t)nv);
    std::vector<uint32_t> jp((size_t)nv);
    for (int v = 0; v < nv; v++) {
        uint32_t w = 0;
        for (int d = 0; d < 3; d++) {
            xf[(size_t)d * nv + v] = (float)xi[3 * (size_t)v + d];
            // node k of axis d: xi = lo + (k + 1/2) h = (h/2) (2k + 1 - n)
            const int k = (int)std::lround((xi[3 * (size_t)v + d] - lo[d]) / h[d] - 0.5);
            w |= (uint32_t)(2 * k + 1 - n[d] + 64) << (8 * d);
        }
        jp[v] = w;
    }
    t.hh = 0.5 * h[0];
    for (int d = 0; d < 3; d++) t.half[d] = n[d] / 2;
    t.d_idx = alloc(t.host_idx.size() * 4);
    t.d_b = static_cast<float *>(alloc(t.host_b.size() * 4));
    t.d_xi = static_cast<float *>(alloc(xf.size() * 4));
    t.d_jpk = static_cast<uint32_t *>(alloc(jp.size() * 4));
    if (!t.d_idx || !t.d_b || !t.d_xi || !t.d_jpk) { err = "device allocation (collision tables)"; return DVM_ENOMEM; }
    std::vector<uint32_t> didx;
    std::vector<float> db;
    order_for_banks(t.host_idx, t.host_b, nv, trials, didx, db);
    if (cudaMemcpy(t.d_idx, didx.data(), didx.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(t.d_b, db.data(), db.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(t.d_xi, xf.data(), xf.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(t.d_jpk, jp.data(), jp.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaGetLastError();
        err = "copy collision tables";
        return DVM_ECUDA;
    }
    t.trials = trials;
    t.seed = seed;
    t.nv = nv;
    t.ready = true;
    return DVM_OK;
}

}  // namespace dvm
