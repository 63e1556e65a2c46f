// Lattice Boltzmann on the tree (paper Sec. 4): the DVM transport of Eq. 2 on
// a minimal velocity set (D2Q9, D3Q19, D3Q27) with the lattice BGK collision
// and its second-order equilibrium.  Host side: the velocity set and the
// compact per-cell upwind codes; device side: the fused step kernel.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "mesh.hpp"

namespace dvm {

// One upwind source of a cell side, 32 bits:
//   bits 0..26  source cell (the inflow ghost is cell ncells), or, with
//               LBM_OVF, the index of the first of the side's entries in the
//               overflow array;
//   bit 27      wall: the cell itself at the velocity mirrored along the side's axis;
//   bits 28..29 m - 1: the source's weight is m / (2^(dim-1) h) (a full side
//               sums to m = 2^(dim-1)); with LBM_OVF, the entry count - 1;
//   bit 30      LBM_OVF.
constexpr uint32_t LBM_CELL = (1u << 27) - 1, LBM_WALL = 1u << 27, LBM_OVF = 1u << 30;
constexpr int LBM_M_SHIFT = 28;

struct LbmLattice {
    int kind = 0, q = 0;
    int c[27][3] = {};
    double w[27] = {};
};

// The velocity set of DVM_LBM_D2Q9 / D3Q19 / D3Q27: velocities in order of
// increasing |c|^2, ties lexicographic in (c_x, c_y, c_z) with -1 < 0 < 1;
// weights by |c|^2.  Returns false for an unknown kind.
bool lbm_lattice(int kind, LbmLattice &out);

// codes [2 dim][ncells] (side list 2d + s, s = 0 the minus side), the
// overflow entries of sides with several sources, and each cell's level.
// Returns DVM_OK or a negative dvm_status with a message.
int lbm_build_codes(const Mesh &m, std::vector<uint32_t> &codes, std::vector<uint32_t> &ovf,
                    std::vector<uint8_t> &lev, std::string &err);

struct LbmParams {
    int prec;                 // DVM_F64 / DVM_F32
    int dim, q;
    int64_t ncells, ld;       // f is [q][ld], column ncells the inflow ghost
    const void *f_in;
    void *f_out;
    const uint32_t *codes;    // [2 dim][ncells]
    const uint32_t *ovf;
    const uint8_t *lev;       // [ncells]
    double dt, omega;         // omega = dt / tau
    int *status;              // bit 0: a cell with rho <= 0 or non-finite moments
    cudaStream_t stream;
};

int launch_lbm(const LbmParams &p);

// rho, u of every cell in FP64: out [ncells][4]
int launch_lbm_moments(int prec, int q, const void *f, int64_t ncells, int64_t ld, double *out,
                       cudaStream_t s);

}  // namespace dvm
