// The uniform velocity grid (paper Sec. 3) in the sign-group storage order
// (Sec. 3.1 steps 1-3): host tables shared by the context and the per-rank
// solver.
#pragma once
#include <string>
#include <vector>

#include "../../include/dvm.h"

namespace dvm {

struct Vgrid {
    int n[3] = {0, 0, 0}, half[3] = {0, 0, 0};
    int nv = 0, P = 0;
    double lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0}, hv[3] = {0, 0, 0}, dV = 0;
    std::vector<double> xi;  // [nv][3] node values in storage order
    double amag[96] = {0};   // [3][32] |xi| of the positive-side nodes m = 0..half-1
    float amag_f[96] = {0};
};

// Checks and fills g: every n even and at most 64, lo = -hi > 0 per axis,
// n_z / 2 a multiple of vec (the vector width of the storage).  Nodes
// xi_d(k) = lo_d + (k + 1/2) h_d in FP64; group o = 4[xi_x>0] + 2[xi_y>0] +
// [xi_z>0]; inside a group node (mx, my, mz) (m = 0 nearest zero) at
// ((mx ny/2) + my) nz/2 + mz.
inline int make_vgrid(const int n[3], const double lo[3], const double hi[3], int vec, Vgrid &g, std::string &err)
{
    for (int d = 0; d < 3; d++) {
        if (n[d] < 2 || n[d] % 2 || n[d] > 64) { err = "each n must be even and at most 64"; return DVM_EINVAL; }
        if (!(hi[d] > 0.0) || lo[d] != -hi[d]) { err = "the velocity grid must be symmetric (lo = -hi)"; return DVM_EINVAL; }
    }
    if ((n[2] / 2) % vec) { err = "nz/2 must be a multiple of the vector width"; return DVM_EINVAL; }
    for (int d = 0; d < 3; d++) {
        g.n[d] = n[d];
        g.half[d] = n[d] / 2;
        g.lo[d] = lo[d];
        g.hi[d] = hi[d];
        g.hv[d] = (hi[d] - lo[d]) / n[d];
    }
    g.dV = g.hv[0] * g.hv[1] * g.hv[2];
    g.nv = n[0] * n[1] * n[2];
    g.P = g.nv / 8;
    g.xi.assign(3 * (size_t)g.nv, 0.0);
    int v = 0;
    for (int o = 0; o < 8; o++)
        for (int mx = 0; mx < g.half[0]; mx++)
            for (int my = 0; my < g.half[1]; my++)
                for (int mz = 0; mz < g.half[2]; mz++, v++) {
                    const int m3[3] = {mx, my, mz};
                    for (int d = 0; d < 3; d++) {
                        const bool pos = (o >> (2 - d)) & 1;
                        const int k = pos ? g.half[d] + m3[d] : g.half[d] - 1 - m3[d];
                        g.xi[3 * (size_t)v + d] = g.lo[d] + ((double)k + 0.5) * g.hv[d];
                    }
                }
    for (int d = 0; d < 3; d++)
        for (int m = 0; m < 32; m++) {
            const double val = m < g.half[d] ? g.lo[d] + ((double)(g.half[d] + m) + 0.5) * g.hv[d] : 0.0;
            g.amag[32 * d + m] = val;
            g.amag_f[32 * d + m] = (float)val;
        }
    return DVM_OK;
}

}  // namespace dvm
