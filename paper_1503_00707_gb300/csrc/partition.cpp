#include "partition.hpp"

#include <algorithm>

#include "mesh.hpp"

namespace dvm {

namespace {
constexpr int32_t CELL_MASK = 0x0fffffff;
}

void encode_stencils(const std::vector<int32_t> &st_src, int64_t ncells, std::vector<int32_t> &enc)
{
    // inflow: the extra cell `ncells` holding the freestream Maxwellian;
    // outflow: the cell itself; specular wall: the cell itself in the group
    // mirrored along the face's axis
    enc.resize(st_src.size());
    for (int64_t q = 0; q < ncells; q++)
        for (int list = 0; list < 6; list++)
            for (int e = 0; e < MAX_SRC; e++) {
                const size_t k = ((size_t)q * 6 + list) * MAX_SRC + e;
                const int32_t s0 = st_src[k];
                int32_t v;
                if (s0 >= 0) v = s0;
                else if (s0 == SRC_INFLOW) v = (int32_t)ncells;
                else if (s0 == SRC_OUTFLOW) v = (int32_t)q;
                else v = (int32_t)q | ((4 >> (list / 2)) << 28);
                enc[k] = v;
            }
}

void partition_cells(int64_t ncells, int nparts, const std::vector<int32_t> &enc,
                     const std::vector<uint8_t> &st_cnt, std::vector<Part> &parts, const double *weight)
{
    parts.assign(nparts, Part{});
    if (!weight) {
        const int64_t base = ncells / nparts, extra = ncells % nparts;
        int64_t c = 0;
        for (int p = 0; p < nparts; p++) {
            parts[p].c0 = c;
            c += base + (p < extra ? 1 : 0);
            parts[p].c1 = c;
        }
    } else {
        // cut p at the first cell where the weight before it reaches p W /
        // nparts, keeping at least one cell per part
        double W = 0.0;
        for (int64_t q = 0; q < ncells; q++) W += weight[q];
        int64_t c = 0;
        double acc = 0.0;
        for (int p = 0; p < nparts; p++) {
            parts[p].c0 = c;
            if (p == nparts - 1) {
                c = ncells;
            } else {
                const double target = W * (double)(p + 1) / (double)nparts;
                const int64_t hi = ncells - (nparts - 1 - p);  // leave a cell for each later part
                int64_t e = c + 1;
                acc += weight[c];
                while (e < hi && acc + 0.5 * weight[e] <= target) acc += weight[e++];
                c = e;
            }
            parts[p].c1 = c;
        }
    }
    for (Part &pt : parts) {
        std::vector<int64_t> g;
        for (int64_t q = pt.c0; q < pt.c1; q++)
            for (int list = 0; list < 6; list++)
                for (int e = 0; e < st_cnt[q * 8 + list]; e++) {
                    const int64_t s = enc[((size_t)q * 6 + list) * MAX_SRC + e] & CELL_MASK;
                    if (s != ncells && (s < pt.c0 || s >= pt.c1)) g.push_back(s);
                }
        std::sort(g.begin(), g.end());
        g.erase(std::unique(g.begin(), g.end()), g.end());
        pt.ghosts = std::move(g);
    }
}

void local_stencils(const Part &part, int64_t ncells, const std::vector<int32_t> &enc, std::vector<int32_t> &local)
{
    const int64_t nloc = part.c1 - part.c0;
    const size_t per = (size_t)6 * MAX_SRC;
    local.assign((size_t)nloc * per, 0);
    for (int64_t q = part.c0; q < part.c1; q++)
        for (size_t k = 0; k < per; k++) {
            const int32_t v = enc[(size_t)q * per + k];
            const int64_t s = v & CELL_MASK;
            int64_t ls;
            if (s == ncells) ls = nloc + (int64_t)part.ghosts.size();
            else if (s >= part.c0 && s < part.c1) ls = s - part.c0;
            else {
                const auto it = std::lower_bound(part.ghosts.begin(), part.ghosts.end(), s);
                // entries past a list's count are padding: any local index does
                ls = (it != part.ghosts.end() && *it == s) ? nloc + (it - part.ghosts.begin()) : 0;
            }
            local[(size_t)(q - part.c0) * per + k] = (int32_t)ls | (v & ~CELL_MASK);
        }
}

}  // namespace dvm
