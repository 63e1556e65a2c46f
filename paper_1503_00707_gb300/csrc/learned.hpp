// Learned collision operator: host-side geometry for the local Knudsen
// sensor and the launch interface of its kernels (k_learned.cu).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>
#include <vector>

#include "mesh.hpp"

namespace dvm {

// Weighted least-squares gradient stencil: for cell c, entries
// start[c] .. start[c+1]-1 hold face neighbours nb[e] and coefficients
// coef[e][3] such that grad q(c) = sum_e coef[e] (q(nb[e]) - q(c)).
// coef = w N^{-1} d with d the centre offset (periodic sides wrapped),
// w = A_face / |d|^2 and N = sum w d d^T; a cell whose N is singular gets
// zero coefficients (zero gradient).
struct KnStencil {
    std::vector<int32_t> start, nb;
    std::vector<double> coef;
};
void build_kn_stencil(const Mesh &m, KnStencil &out);

// The velocity grids the learned kernels support: every n even and at most
// 32, and n_z / 2 a multiple of 4.
bool learned_grid_supported(const int n[3]);

// knl[c] = Kn_loc of cell c from the moments mom [ncells][5] (rho, u, T).
int launch_kn_local(const double *mom, const int32_t *start, const int32_t *nb, const double *coef,
                    int64_t ncells, double kn, double *knl, cudaStream_t s);

// out[r][64] = Hermite projection of row r of f (FP32 [.][nv], storage
// order): mode 0 gives a_m = sum f H_m dV / rho, mode 1 gives
// o_m = sum f H_m dV / (rho^2 sqrt(T)), with (rho, u, T) of the row's cell
// from mom.  With list != NULL, row r is cell list[r] for r < *count (the
// launch covers `rows` rows, those beyond *count do nothing).  In mode 0,
// out_eq (optional) receives a of the cell's Maxwellian M(rho, u, T)
// sampled at the nodes.
int launch_hermite_project(const float *f, const double *mom, const double *amag, int64_t rows, const int n[3],
                           double dV, int mode, const int32_t *list, const int *count, float *out, float *out_eq,
                           int *status, cudaStream_t s);

// Learned collision on f in place for every cell with knl < thr whose
// corrected term passes the checks: f += dtkn * Q, Q reconstructed from
// o - o_eq (o_eq optional: the network at the cell's Maxwellian).
// used[c] = 1 there;
// every other cell gets used[c] = 0 and is appended to list (*count, which
// must start at 0, counts them).  q_out (optional, [ncells][nv]) receives Q
// of the cells that used it.
int launch_learned_apply(float *f, const double *mom, const float *o, const float *o_eq, const double *knl, double thr,
                         const double *amag, int64_t ncells, const int n[3], double dtkn, int32_t *used,
                         int32_t *list, int *count, float *q_out, double dV, double *res, int *status,
                         cudaStream_t s);

}  // namespace dvm
