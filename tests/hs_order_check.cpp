// Host check of the hard-sphere trial order (the library's own ordering code,
// compiled in): reads node-major tables (gamma, l, m as uint32 triples and
// FP32 weights) for an n^3 grid with M trials per node, orders them for the
// gather kernel and checks that
//   * each node keeps its weighted trials (gamma, l, m, b) as a multiset;
//   * every weighted trial of a warp sits below the warp's last weighted slot
//     boundary R = ceil(largest weighted count / lanes per node);
//   * below R, a zero-weight trial gathers at addresses that a weighted lane of
//     the same slot gathers at too;
// and prints the mean shared-memory wavefronts per gather over all slots.
// Usage: hs_order_check n M tables.bin weights.bin
namespace dvm {
bool hs_trials_supported(int) { return true; }
}
#include "../paper_1503_00707_gb300/csrc/hs.cpp"

#include <cstdio>
#include <tuple>

int main(int argc, char **argv)
{
    if (argc != 5) return 2;
    const int n = std::atoi(argv[1]), M = std::atoi(argv[2]), nv = n * n * n;
    std::vector<uint32_t> a((size_t)nv * M * 3);
    std::vector<float> b((size_t)nv * M);
    FILE *f = std::fopen(argv[3], "rb");
    if (!f || std::fread(a.data(), 4, a.size(), f) != a.size()) return 3;
    std::fclose(f);
    f = std::fopen(argv[4], "rb");
    if (!f || std::fread(b.data(), 4, b.size(), f) != b.size()) return 3;
    std::fclose(f);
    std::vector<uint32_t> idx((size_t)nv * M * 2);
    for (size_t q = 0; q < (size_t)nv * M; q++) {
        idx[2 * q] = a[3 * q] | (a[3 * q + 1] << 16);
        idx[2 * q + 1] = a[3 * q + 2];
    }
    std::vector<uint32_t> o;
    std::vector<float> ob;
    dvm::order_for_banks(idx, b, nv, M, o, ob);
    const int tpn = M / 32, K = 32 / tpn;
    auto addr = [&](size_t q, int g) -> uint32_t { return g == 0 ? (o[2 * q] & 0xffffu) : g == 1 ? (o[2 * q] >> 16) : o[2 * q + 1]; };
    int bad_multiset = 0, bad_below = 0, bad_filler = 0;
    double wf = 0.0;
    long cnt = 0;
    for (int g0 = 0; g0 < nv; g0 += K) {
        const int kn = std::min(K, nv - g0);
        int kmax = 0;
        for (int nl = 0; nl < kn; nl++) {
            int c = 0;
            for (int k = 0; k < M; k++) c += b[(size_t)(g0 + nl) * M + k] != 0.0f;
            kmax = std::max(kmax, c);
        }
        const int R = (kmax + tpn - 1) / tpn;
        for (int e = 0; e < 32; e++) {
            for (int lane = 0; lane < kn * tpn; lane++) {
                const size_t q = (size_t)(g0 + lane / tpn) * M + (lane % tpn) * 32 + e;
                if (e >= R && ob[q] != 0.0f) bad_below++;
                if (e < R && ob[q] == 0.0f) {
                    bool shared = false;
                    for (int l2 = 0; l2 < kn * tpn && !shared; l2++) {
                        const size_t q2 = (size_t)(g0 + l2 / tpn) * M + (l2 % tpn) * 32 + e;
                        shared = ob[q2] != 0.0f && addr(q2, 0) == addr(q, 0) && addr(q2, 1) == addr(q, 1) &&
                                 addr(q2, 2) == addr(q, 2);
                    }
                    bool any_weighted = false;
                    for (int l2 = 0; l2 < kn * tpn; l2++)
                        any_weighted |= ob[(size_t)(g0 + l2 / tpn) * M + (l2 % tpn) * 32 + e] != 0.0f;
                    if (any_weighted && !shared) bad_filler++;
                }
            }
            for (int g = 0; g < 3; g++) {
                int c[32] = {0};
                uint32_t ad[32][32];
                for (int lane = 0; lane < 32; lane++) {
                    const int node = std::min(g0 + lane / tpn, nv - 1);
                    const size_t q = (size_t)node * M + (lane % tpn) * 32 + e;
                    const uint32_t v = addr(q, g);
                    const int bk = (int)(v & 31u);
                    bool seen = false;
                    for (int k = 0; k < c[bk]; k++) seen = seen || ad[bk][k] == v;
                    if (!seen) ad[bk][c[bk]++] = v;
                }
                int mx = 1;
                for (int k = 0; k < 32; k++) mx = std::max(mx, c[k]);
                wf += mx;
                cnt++;
            }
        }
    }
    for (int node = 0; node < nv; node++) {
        std::vector<std::tuple<uint32_t, uint32_t, float>> x, y;
        for (int k = 0; k < M; k++) {
            const size_t q = (size_t)node * M + k;
            if (b[q] != 0.0f) x.emplace_back(idx[2 * q], idx[2 * q + 1], b[q]);
            if (ob[q] != 0.0f) y.emplace_back(o[2 * q], o[2 * q + 1], ob[q]);
        }
        std::sort(x.begin(), x.end());
        std::sort(y.begin(), y.end());
        bad_multiset += x != y;
    }
    std::printf("%d %d %d %.4f\n", bad_multiset, bad_below, bad_filler, wf / cnt);
    return 0;
}
