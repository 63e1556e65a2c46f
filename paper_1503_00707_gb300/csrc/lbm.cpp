// Host side of the lattice Boltzmann step: velocity sets and upwind codes.
#include "lbm.hpp"

#include <cmath>

#include "../../include/dvm.h"

namespace dvm {

bool lbm_lattice(int kind, LbmLattice &out)
{
    // weights of the |c|^2 = 0, 1, 2, 3 classes; 4th-order isotropy of each
    // set fixes them, with c_s^2 = 1/3
    double wc[4];
    if (kind == DVM_LBM_D2Q9) { wc[0] = 4.0 / 9; wc[1] = 1.0 / 9; wc[2] = 1.0 / 36; wc[3] = 0; }
    else if (kind == DVM_LBM_D3Q19) { wc[0] = 1.0 / 3; wc[1] = 1.0 / 18; wc[2] = 1.0 / 36; wc[3] = 0; }
    else if (kind == DVM_LBM_D3Q27) { wc[0] = 8.0 / 27; wc[1] = 2.0 / 27; wc[2] = 1.0 / 54; wc[3] = 1.0 / 216; }
    else return false;
    out = LbmLattice{};
    out.kind = kind;
    for (int r2 = 0; r2 <= 3; r2++)
        for (int x = -1; x <= 1; x++)
            for (int y = -1; y <= 1; y++)
                for (int z = -1; z <= 1; z++) {
                    if (x * x + y * y + z * z != r2) continue;
                    if (kind == DVM_LBM_D2Q9 && z != 0) continue;
                    if (kind == DVM_LBM_D3Q19 && r2 == 3) continue;
                    out.c[out.q][0] = x;
                    out.c[out.q][1] = y;
                    out.c[out.q][2] = z;
                    out.w[out.q] = wc[r2];
                    out.q++;
                }
    return true;
}

int lbm_build_codes(const Mesh &m, std::vector<uint32_t> &codes, std::vector<uint32_t> &ovf,
                    std::vector<uint8_t> &lev, std::string &err)
{
    const int dim = m.spec.dim;
    const int64_t nc = (int64_t)m.leaf_of_cell.size();
    if (nc >= (int64_t)LBM_CELL) {
        err = "too many cells for the lattice Boltzmann codes";
        return DVM_EINVAL;
    }
    const int full = 1 << (dim - 1);
    codes.assign((size_t)2 * dim * nc, 0);
    ovf.clear();
    lev.assign((size_t)nc, 0);
    for (int64_t q = 0; q < nc; q++) {
        const int l = m.leaves[m.leaf_of_cell[q]].lev;
        lev[q] = (uint8_t)l;
        const double h = std::ldexp(1.0, -l);
        for (int list = 0; list < 2 * dim; list++) {
            const int cnt = m.st_cnt[q * 8 + list];
            uint32_t ent[MAX_SRC];
            int msum = 0;
            for (int e = 0; e < cnt; e++) {
                const size_t k = ((size_t)q * 6 + list) * MAX_SRC + e;
                const int32_t s = m.st_src[k];
                const double mm = m.st_w[k] * h * full;
                const int mi = (int)std::lround(mm);
                if (mi < 1 || mi > 4 || std::fabs(mm - mi) > 1e-9) {
                    err = "a stencil weight is not a multiple of the subface weight";
                    return DVM_EINVAL;
                }
                msum += mi;
                uint32_t v;
                if (s >= 0) v = (uint32_t)s;
                else if (s == SRC_INFLOW) v = (uint32_t)nc;
                else if (s == SRC_OUTFLOW) v = (uint32_t)q;
                else v = (uint32_t)q | LBM_WALL;
                ent[e] = v | ((uint32_t)(mi - 1) << LBM_M_SHIFT);
            }
            if (cnt < 1 || msum != full) {
                err = "a cell side is not covered by its upwind sources";
                return DVM_EINVAL;
            }
            uint32_t code;
            if (cnt == 1) {
                code = ent[0];
            } else {
                if (ovf.size() + cnt > (size_t)LBM_CELL) {
                    err = "too many overflow entries";
                    return DVM_EINVAL;
                }
                code = (uint32_t)ovf.size() | LBM_OVF | ((uint32_t)(cnt - 1) << LBM_M_SHIFT);
                for (int e = 0; e < cnt; e++) ovf.push_back(ent[e]);
            }
            codes[(size_t)list * nc + q] = code;
        }
    }
    return DVM_OK;
}

}  // namespace dvm
