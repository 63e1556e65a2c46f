// Host mesh construction: predicate refinement, 2:1 balance by a single
// finest-to-coarsest ripple sweep over a hash set of leaves, Morton sort,
// face enumeration and per-cell upwind stencils.
//
// Paper Sec. 2.1: boxes obtained by repeated halving, leaves are the cells,
// levels of direct and diagonal neighbours differ by at most one, N-order
// (Morton) traversal.  Sec. 3.1 step 4: per cell and per sign group, the
// count, indices and weights of the stencil of Eq. 2, rebuilt whenever the
// mesh changes.
#include "mesh.hpp"

#include <algorithm>
#include <array>
#include <cmath>
#include <unordered_map>
#include <unordered_set>

namespace dvm {
namespace {

constexpr int CBITS = 19;
constexpr uint64_t CMASK = (1ull << CBITS) - 1;

inline uint64_t node_code(int lev, const int32_t c[3])
{
    return ((uint64_t)lev << 58) | ((uint64_t)c[0] << (2 * CBITS)) |
           ((uint64_t)c[1] << CBITS) | (uint64_t)c[2];
}

// Spread the low 21 bits of v so that bit b lands on bit 3b (resp. 2b).
inline uint64_t spread3(uint64_t v)
{
    v &= 0x1fffff;
    v = (v | (v << 32)) & 0x1f00000000ffffull;
    v = (v | (v << 16)) & 0x1f0000ff0000ffull;
    v = (v | (v << 8)) & 0x100f00f00f00f00full;
    v = (v | (v << 4)) & 0x10c30c30c30c30c3ull;
    v = (v | (v << 2)) & 0x1249249249249249ull;
    return v;
}

inline uint64_t spread2(uint64_t v)
{
    v &= 0xffffffff;
    v = (v | (v << 16)) & 0x0000ffff0000ffffull;
    v = (v | (v << 8)) & 0x00ff00ff00ff00ffull;
    v = (v | (v << 4)) & 0x0f0f0f0f0f0f0f0full;
    v = (v | (v << 2)) & 0x3333333333333333ull;
    v = (v | (v << 1)) & 0x5555555555555555ull;
    return v;
}

struct Builder {
    const dvm_tree_spec &s;
    int dim, L;
    bool per[3];
    std::unordered_set<uint64_t> leaves;
    std::vector<std::vector<std::array<int32_t, 3>>> bylevel;

    explicit Builder(const dvm_tree_spec &sp) : s(sp), dim(sp.dim), L(sp.max_level)
    {
        for (int d = 0; d < 3; d++) per[d] = d < dim && sp.bc[2 * d] == DVM_BC_PERIODIC;
        bylevel.resize(L + 1);
    }

    // Box-to-centre squared distances on the dyadic box [c h, (c+1) h].
    double dist2_near(int lev, const int32_t c[3]) const
    {
        const double h = std::ldexp(1.0, -lev);
        double acc = 0.0;
        for (int d = 0; d < dim; d++) {
            const double lo = c[d] * h, hi = (c[d] + 1) * h;
            double t = 0.0;
            if (s.c[d] < lo) t = lo - s.c[d];
            else if (s.c[d] > hi) t = s.c[d] - hi;
            acc += t * t;
        }
        return acc;
    }

    double dist2_far(int lev, const int32_t c[3]) const
    {
        const double h = std::ldexp(1.0, -lev);
        double acc = 0.0;
        for (int d = 0; d < dim; d++) {
            const double a = std::fabs(c[d] * h - s.c[d]);
            const double b = std::fabs((c[d] + 1) * h - s.c[d]);
            const double t = std::max(a, b);
            acc += t * t;
        }
        return acc;
    }

    bool split_wanted(int lev, const int32_t c[3]) const
    {
        if (lev >= s.max_level) return false;
        switch (s.pred) {
        case DVM_PRED_BALL:
            return dist2_near(lev, c) <= s.r * s.r;
        case DVM_PRED_SHELL: {
            const double h = std::ldexp(1.0, -lev);
            const double outer = s.r + s.beta * h, inner = s.r - s.beta * h;
            if (!(dist2_near(lev, c) <= outer * outer)) return false;
            return inner <= 0.0 || dist2_far(lev, c) >= inner * inner;
        }
        default:
            return false;
        }
    }

    bool solid_leaf(int lev, const int32_t c[3]) const
    {
        if (!s.solid) return false;
        const double h = std::ldexp(1.0, -lev);
        double acc = 0.0;
        for (int d = 0; d < dim; d++) {
            const double t = (c[d] + 0.5) * h - s.c[d];
            acc += t * t;
        }
        return acc < s.r * s.r;
    }

    void emit(int lev, const int32_t c[3])
    {
        leaves.insert(node_code(lev, c));
        bylevel[lev].push_back({c[0], c[1], c[2]});
    }

    void descend(int lev, const int32_t c[3])
    {
        if (split_wanted(lev, c)) {
            for (int k = 0; k < (1 << dim); k++) {
                int32_t ch[3] = {0, 0, 0};
                for (int d = 0; d < dim; d++) ch[d] = 2 * c[d] + ((k >> d) & 1);
                descend(lev + 1, ch);
            }
        } else {
            emit(lev, c);
        }
    }

    // Level of the leaf containing node (lev, c), or -1 if the node is
    // subdivided into finer leaves.
    int owner_level(int lev, const int32_t c[3]) const
    {
        for (int m = lev; m >= 0; m--) {
            const int sh = lev - m;
            int32_t cc[3] = {c[0] >> sh, c[1] >> sh, c[2] >> sh};
            if (leaves.count(node_code(m, cc))) return m;
        }
        return -1;
    }

    void split_leaf(int lev, const int32_t c[3])
    {
        leaves.erase(node_code(lev, c));
        for (int k = 0; k < (1 << dim); k++) {
            int32_t ch[3] = {0, 0, 0};
            for (int d = 0; d < dim; d++) ch[d] = 2 * c[d] + ((k >> d) & 1);
            emit(lev + 1, ch);
        }
    }

    // Split the leaf (blev, ...) that contains node (tlev, t) until t is a leaf.
    void split_down(int blev, int tlev, const int32_t t[3])
    {
        for (int lev = blev; lev < tlev; lev++) {
            const int sh = tlev - lev;
            int32_t c[3] = {t[0] >> sh, t[1] >> sh, t[2] >> sh};
            split_leaf(lev, c);
        }
    }

    // Finest to coarsest: every leaf at level l needs each level-(l-1) node
    // that touches it to exist in the tree.  Splits made at level l create
    // leaves of level < l only, which later passes visit.
    void balance(int lowest)
    {
        for (int lev = L; lev >= lowest + 2; lev--) {
            const int32_t N = (int32_t)1 << (lev - 1);
            for (size_t q = 0; q < bylevel[lev].size(); q++) {
                const std::array<int32_t, 3> a = bylevel[lev][q];
                if (!leaves.count(node_code(lev, a.data()))) continue;
                const int nz = dim == 3 ? 3 : 1;
                for (int oz = 0; oz < nz; oz++)
                    for (int oy = 0; oy < 3; oy++)
                        for (int ox = 0; ox < 3; ox++) {
                            const int off[3] = {ox - 1, oy - 1, dim == 3 ? oz - 1 : 0};
                            if (off[0] == 0 && off[1] == 0 && off[2] == 0) continue;
                            int32_t n[3] = {0, 0, 0};
                            bool ok = true;
                            for (int d = 0; d < dim && ok; d++) {
                                // the neighbour of the parent touches this child only
                                // on the child's own side of the parent
                                if (off[d] == -1 && (a[d] & 1)) ok = false;
                                if (off[d] == 1 && !(a[d] & 1)) ok = false;
                                n[d] = (a[d] >> 1) + off[d];
                                if (n[d] < 0 || n[d] >= N) {
                                    if (per[d]) n[d] = (n[d] + N) % N;
                                    else ok = false;
                                }
                            }
                            if (!ok) continue;
                            const int m = owner_level(lev - 1, n);
                            if (m >= 0 && m < lev - 1) split_down(m, lev - 1, n);
                        }
            }
        }
    }
};

struct IFace { int64_t m, p; uint8_t ax; double area; uint64_t km, kp; };
struct BFace { int64_t l, o; uint8_t ax, side, kind; double area; uint64_t kl, ko; };

int check_spec(const dvm_tree_spec &s, std::string &err)
{
    if (s.dim != 2 && s.dim != 3) { err = "dim must be 2 or 3"; return DVM_EINVAL; }
    if (s.base_level < 1 || s.max_level < s.base_level || s.max_level > CBITS) {
        err = "need 1 <= base_level <= max_level <= 19";
        return DVM_EINVAL;
    }
    if (s.pred < DVM_PRED_NONE || s.pred > DVM_PRED_SHELL) { err = "unknown predicate"; return DVM_EINVAL; }
    for (int d = 0; d < s.dim; d++) {
        for (int q = 0; q < 2; q++)
            if (s.bc[2 * d + q] < DVM_BC_PERIODIC || s.bc[2 * d + q] > DVM_BC_WALL) {
                err = "unknown boundary kind";
                return DVM_EINVAL;
            }
        if ((s.bc[2 * d] == DVM_BC_PERIODIC) != (s.bc[2 * d + 1] == DVM_BC_PERIODIC)) {
            err = "periodic sides must come in pairs";
            return DVM_EINVAL;
        }
    }
    return DVM_OK;
}

int finish(Builder &b, Mesh &m, std::string &err)
{
    const int dim = b.dim, L = b.L;
    m.L = L;
    m.leaves.clear();
    m.leaves.reserve(b.leaves.size());
    for (uint64_t code : b.leaves) {
        Leaf x;
        x.lev = (int)(code >> 58);
        x.i[0] = (int32_t)((code >> (2 * CBITS)) & CMASK);
        x.i[1] = (int32_t)((code >> CBITS) & CMASK);
        x.i[2] = (int32_t)(code & CMASK);
        const int sh = L - x.lev;
        if (dim == 3)
            x.key = spread3((uint64_t)x.i[0] << sh) | (spread3((uint64_t)x.i[1] << sh) << 1) |
                    (spread3((uint64_t)x.i[2] << sh) << 2);
        else
            x.key = spread2((uint64_t)x.i[0] << sh) | (spread2((uint64_t)x.i[1] << sh) << 1);
        x.solid = b.solid_leaf(x.lev, x.i) ? 1 : 0;
        m.leaves.push_back(x);
    }
    std::sort(m.leaves.begin(), m.leaves.end(), [](const Leaf &a, const Leaf &c) { return a.key < c.key; });
    const int64_t nl = (int64_t)m.leaves.size();
    std::unordered_map<uint64_t, int64_t> index;
    index.reserve(nl * 2);
    for (int64_t q = 0; q < nl; q++) index[node_code(m.leaves[q].lev, m.leaves[q].i)] = q;
    m.cell_of_leaf.assign(nl, -1);
    m.leaf_of_cell.clear();
    m.max_cell_level = 0;
    for (int64_t q = 0; q < nl; q++)
        if (!m.leaves[q].solid) {
            m.cell_of_leaf[q] = (int64_t)m.leaf_of_cell.size();
            m.leaf_of_cell.push_back(q);
            m.max_cell_level = std::max(m.max_cell_level, m.leaves[q].lev);
        }
    if (m.leaf_of_cell.empty()) { err = "every leaf is solid"; return DVM_EINVAL; }

    // faces
    std::vector<IFace> fi;
    std::vector<BFace> fb;
    for (int64_t q = 0; q < nl; q++) {
        const Leaf &A = m.leaves[q];
        if (A.solid) continue;
        const int32_t N = (int32_t)1 << A.lev;
        for (int d = 0; d < dim; d++)
            for (int side = 0; side < 2; side++) {
                int32_t n[3] = {A.i[0], A.i[1], A.i[2]};
                n[d] += side ? 1 : -1;
                if (n[d] < 0 || n[d] >= N) {
                    if (b.per[d]) n[d] = (n[d] + N) % N;
                    else {
                        fb.push_back({q, -1, (uint8_t)d, (uint8_t)side, (uint8_t)b.s.bc[2 * d + side],
                                      std::ldexp(1.0, -A.lev * (dim - 1)), A.key, 0});
                        continue;
                    }
                }
                int64_t nb[4];
                int cnt = 0;
                double area;
                const int own = b.owner_level(A.lev, n);
                if (own >= 0) {
                    const int sh = A.lev - own;
                    int32_t cc[3] = {n[0] >> sh, n[1] >> sh, n[2] >> sh};
                    nb[cnt++] = index.at(node_code(own, cc));
                    area = std::ldexp(1.0, -A.lev * (dim - 1));
                } else {
                    for (int t = 0; t < (1 << (dim - 1)); t++) {
                        int32_t cc[3] = {0, 0, 0};
                        int bit = 0;
                        for (int e = 0; e < dim; e++)
                            cc[e] = e == d ? 2 * n[e] + (side ? 0 : 1) : 2 * n[e] + ((t >> bit++) & 1);
                        auto it = index.find(node_code(A.lev + 1, cc));
                        if (it == index.end()) { err = "mesh is not 2:1 balanced"; return DVM_EINVAL; }
                        nb[cnt++] = it->second;
                    }
                    area = std::ldexp(1.0, -(A.lev + 1) * (dim - 1));
                }
                for (int t = 0; t < cnt; t++) {
                    const Leaf &B = m.leaves[nb[t]];
                    if (B.solid)
                        fb.push_back({q, nb[t], (uint8_t)d, (uint8_t)side, (uint8_t)DVM_BC_WALL, area, A.key, B.key});
                    else if (side == 1)
                        fi.push_back({q, nb[t], (uint8_t)d, area, A.key, B.key});
                }
            }
    }
    std::sort(fi.begin(), fi.end(), [](const IFace &a, const IFace &c) {
        if (a.ax != c.ax) return a.ax < c.ax;
        if (a.km != c.km) return a.km < c.km;
        return a.kp < c.kp;
    });
    std::sort(fb.begin(), fb.end(), [](const BFace &a, const BFace &c) {
        if (a.kind != c.kind) return a.kind < c.kind;
        if (a.ax != c.ax) return a.ax < c.ax;
        if (a.side != c.side) return a.side < c.side;
        if (a.kl != c.kl) return a.kl < c.kl;
        return a.ko < c.ko;
    });
    m.fm.resize(fi.size()); m.fp.resize(fi.size()); m.fax.resize(fi.size()); m.farea.resize(fi.size());
    for (size_t q = 0; q < fi.size(); q++) {
        m.fm[q] = fi[q].m; m.fp[q] = fi[q].p; m.fax[q] = fi[q].ax; m.farea[q] = fi[q].area;
    }
    const size_t nb = fb.size();
    m.bl.resize(nb); m.bother.resize(nb); m.bax.resize(nb); m.bside.resize(nb); m.bkind.resize(nb); m.barea.resize(nb);
    for (size_t q = 0; q < nb; q++) {
        m.bl[q] = fb[q].l; m.bother[q] = fb[q].o; m.bax[q] = fb[q].ax;
        m.bside[q] = fb[q].side; m.bkind[q] = fb[q].kind; m.barea[q] = fb[q].area;
    }

    // stencils: list 2d+s of a cell gathers the faces on its side s of axis d
    const int64_t nc = (int64_t)m.leaf_of_cell.size();
    m.st_src.assign(nc * 6 * MAX_SRC, 0);
    m.st_w.assign(nc * 6 * MAX_SRC, 0.0);
    m.st_cnt.assign(nc * 8, 0);
    auto add = [&](int64_t cell, int list, int32_t src, double w) -> bool {
        uint8_t &c = m.st_cnt[cell * 8 + list];
        int32_t *s = &m.st_src[(cell * 6 + list) * MAX_SRC];
        double *ww = &m.st_w[(cell * 6 + list) * MAX_SRC];
        for (int e = 0; e < c; e++)
            if (s[e] == src && src < 0) { ww[e] += w; return true; }  // merge wall subfaces
        if (c >= MAX_SRC) return false;
        s[c] = src;
        ww[c] = w;
        c++;
        return true;
    };
    auto vol = [&](int64_t leaf) { return std::ldexp(1.0, -m.leaves[leaf].lev * dim); };
    for (size_t q = 0; q < fi.size(); q++) {
        const int64_t a = m.cell_of_leaf[fi[q].m], c = m.cell_of_leaf[fi[q].p];
        const int d = fi[q].ax;
        if (!add(a, 2 * d + 1, (int32_t)c, fi[q].area / vol(fi[q].m)) ||
            !add(c, 2 * d + 0, (int32_t)a, fi[q].area / vol(fi[q].p))) {
            err = "stencil overflow";
            return DVM_EINVAL;
        }
    }
    for (size_t q = 0; q < nb; q++) {
        const int64_t a = m.cell_of_leaf[fb[q].l];
        const int32_t src = fb[q].kind == DVM_BC_INFLOW ? SRC_INFLOW
                          : fb[q].kind == DVM_BC_OUTFLOW ? SRC_OUTFLOW : SRC_WALL;
        if (!add(a, 2 * fb[q].ax + fb[q].side, src, fb[q].area / vol(fb[q].l))) {
            err = "stencil overflow";
            return DVM_EINVAL;
        }
    }
    return DVM_OK;
}

}  // namespace

int build_mesh(const dvm_tree_spec &spec, Mesh &m, std::string &err)
{
    int rc = check_spec(spec, err);
    if (rc) return rc;
    Builder b(spec);
    const int32_t N = (int32_t)1 << spec.base_level;
    const int32_t nz = spec.dim == 3 ? N : 1;
    for (int32_t z = 0; z < nz; z++)
        for (int32_t y = 0; y < N; y++)
            for (int32_t x = 0; x < N; x++) {
                const int32_t c[3] = {x, y, z};
                b.descend(spec.base_level, c);
            }
    b.balance(spec.base_level);
    m = Mesh();
    m.spec = spec;
    return finish(b, m, err);
}

int refine_mesh(Mesh &m, const uint8_t *flag, int64_t n, std::string &err)
{
    if (n != (int64_t)m.leaves.size()) { err = "flag count differs from the leaf count"; return DVM_EINVAL; }
    Builder b(m.spec);
    for (int64_t q = 0; q < n; q++) {
        const Leaf &x = m.leaves[q];
        if (flag[q] && x.lev < m.spec.max_level) {
            for (int k = 0; k < (1 << b.dim); k++) {
                int32_t ch[3] = {0, 0, 0};
                for (int d = 0; d < b.dim; d++) ch[d] = 2 * x.i[d] + ((k >> d) & 1);
                b.emit(x.lev + 1, ch);
            }
        } else {
            b.emit(x.lev, x.i);
        }
    }
    b.balance(m.spec.base_level);
    const dvm_tree_spec spec = m.spec;
    m = Mesh();
    m.spec = spec;
    return finish(b, m, err);
}

// Coarsening (the inverse of refinement; the paper's adaptive runs refine
// and coarsen as the flow changes, Sec. 2.1, Sec. 4, Sec. 5): every group of
// 2^dim sibling leaves that are all flagged, whose parent is at or above the
// base level, merges into its parent, unless the parent would then touch a
// leaf two or more levels finer (2:1 balance across faces, edges and
// corners).  Groups are undone one by one until no parent breaks the
// balance; undoing only adds finer leaves, so this ends.
namespace {

bool parent_breaks_balance(const Builder &b, int lev, const int32_t c[3])
{
    const int dim = b.dim, nch = 1 << dim;
    const int32_t N = (int32_t)1 << lev;
    const int nz = dim == 3 ? 3 : 1;
    for (int oz = 0; oz < nz; oz++)
        for (int oy = 0; oy < 3; oy++)
            for (int ox = 0; ox < 3; ox++) {
                const int off[3] = {ox - 1, oy - 1, dim == 3 ? oz - 1 : 0};
                if (off[0] == 0 && off[1] == 0 && off[2] == 0) continue;
                int32_t nb[3] = {0, 0, 0};
                bool ok = true;
                for (int d = 0; d < dim && ok; d++) {
                    nb[d] = c[d] + off[d];
                    if (nb[d] < 0 || nb[d] >= N) {
                        if (b.per[d]) nb[d] = (nb[d] + N) % N;
                        else ok = false;
                    }
                }
                if (!ok) continue;
                // the neighbour's children on the side facing the parent
                for (int k = 0; k < nch; k++) {
                    int32_t ch[3] = {0, 0, 0};
                    bool touch = true;
                    for (int d = 0; d < dim; d++) {
                        const int bit = (k >> d) & 1;
                        if ((off[d] == -1 && bit != 1) || (off[d] == 1 && bit != 0)) touch = false;
                        ch[d] = 2 * nb[d] + bit;
                    }
                    if (touch && b.owner_level(lev + 1, ch) < 0) return true;
                }
            }
    return false;
}

}  // namespace

int coarsen_mesh(Mesh &m, const uint8_t *flag, int64_t n, std::string &err)
{
    if (n != (int64_t)m.leaves.size()) { err = "flag count differs from the leaf count"; return DVM_EINVAL; }
    Builder b(m.spec);
    const int dim = b.dim, nch = 1 << dim;
    for (const Leaf &x : m.leaves) b.leaves.insert(node_code(x.lev, x.i));
    struct Group { int lev; int32_t c[3]; bool on; };
    std::vector<Group> g;
    // the children of one parent are consecutive in Morton order
    for (int64_t q = 0; q + nch <= n;) {
        const Leaf &x = m.leaves[q];
        const int32_t pc[3] = {x.i[0] >> 1, x.i[1] >> 1, x.i[2] >> 1};
        bool ok = x.lev > m.spec.base_level;
        for (int k = 0; k < nch && ok; k++) {
            const Leaf &y = m.leaves[q + k];
            ok = flag[q + k] && y.lev == x.lev;
            for (int d = 0; d < dim && ok; d++) ok = (y.i[d] >> 1) == pc[d];
        }
        if (ok) {
            g.push_back({x.lev - 1, {pc[0], pc[1], pc[2]}, true});
            q += nch;
        } else {
            q++;
        }
    }
    auto child = [&](const Group &G, int k, int32_t ch[3]) {
        for (int d = 0; d < 3; d++) ch[d] = d < dim ? 2 * G.c[d] + ((k >> d) & 1) : 0;
    };
    for (const Group &G : g) {
        for (int k = 0; k < nch; k++) {
            int32_t ch[3];
            child(G, k, ch);
            b.leaves.erase(node_code(G.lev + 1, ch));
        }
        b.leaves.insert(node_code(G.lev, G.c));
    }
    for (bool changed = true; changed;) {
        changed = false;
        for (Group &G : g) {
            if (!G.on || !parent_breaks_balance(b, G.lev, G.c)) continue;
            b.leaves.erase(node_code(G.lev, G.c));
            for (int k = 0; k < nch; k++) {
                int32_t ch[3];
                child(G, k, ch);
                b.leaves.insert(node_code(G.lev + 1, ch));
            }
            G.on = false;
            changed = true;
        }
    }
    const dvm_tree_spec spec = m.spec;
    m = Mesh();
    m.spec = spec;
    return finish(b, m, err);
}

}  // namespace dvm
