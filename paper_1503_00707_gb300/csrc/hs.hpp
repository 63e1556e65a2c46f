// Hard-sphere discrete collision integral (paper Sec. 3.2, Eqs. 3-6):
// seeded trial tables built on the host, collision kernel on the device.
#pragma once
#include <cstdint>
#include <functional>
#include <string>
#include <vector>

#include "../../include/dvm.h"
#include "kernels.hpp"

namespace dvm {

struct HsTables {
    bool ready = false;
    int trials = 0;
    uint64_t seed = 0;
    int nv = 0;
    int64_t discarded = 0;
    // Node-major tables, entry e = i*trials + k: idx {gamma | l << 16, m},
    // weight b (= c).  A discarded trial keeps b = 0 and points at node i.
    std::vector<uint32_t> host_idx;   // [nv*trials][2]
    std::vector<float> host_b;        // [nv*trials]
    void *d_idx = nullptr;
    float *d_b = nullptr;
    float *d_xi = nullptr;            // node velocities [3][nv], FP32
    uint32_t *d_jpk = nullptr;        // per node: xi_d = hh j_d, j_d odd, packed as bytes j_d + 64
    double hh = 0.0;                  // half the velocity spacing (the same on every axis)
    int half[3] = {0, 0, 0};          // nodes per axis / 2 (the grid's sign-group shape)
    float *d_bc = nullptr;            // scratch: B and C of every cell [ncells][nv][2]
    int64_t bc_cells = 0;
};

using DevAlloc = std::function<void *(size_t)>;
using DevFree = std::function<void(void *)>;

// Output n (0-based) of the SplitMix64 stream seeded with `seed`.
uint64_t splitmix64_at(uint64_t seed, uint64_t n);

// lattice = false: seeded random trials; true: trials on a shifted 5D
// Korobov lattice (partner by axis indices, omega from the last two
// coordinates).
int hs_build(HsTables &t, const int n[3], const double lo[3], const double h[3],
             const std::vector<double> &xi, int trials, uint64_t seed, bool lattice, std::string &err,
             const DevAlloc &alloc, const DevFree &dfree);

// Korobov multiplier of an M-point rank-1 lattice in five dimensions.
int64_t korobov_multiplier(int64_t M);
void hs_free(HsTables &t, const DevFree &dfree);

// Per-cell scratch for ncells cells (B, C and the correction sums).
int hs_prepare(HsTables &t, int64_t ncells, const DevAlloc &alloc, const DevFree &dfree);

// f (storage precision, already holding f* from the transport launch) is
// updated in place: f <- f* + dt/Kn * I(f*).
int launch_hs_collide(HsTables &t, const StepParams &p, void *f, double kn, double dt);

// The update restricted to the cells list[0 .. *count-1] (device list and
// count, count <= p.ncells), or, if q_out is not NULL, the term I(f) of every
// cell written to q_out [ncells][nv] with f left unchanged.  p.mom_out holds
// the moments of f per cell.
int launch_hs_general(HsTables &t, const StepParams &p, float *f, const int32_t *list, const int *count,
                      float *q_out, double kn, double dt);

// The same update on caller-owned f with a fixed, statically allocated
// device scratch (no allocation).  Needs p.ncells * (8 nv + 40) bytes of
// scratch at most DVM_HS_NOALLOC_SCRATCH_BYTES (else DVM_EINVAL); xi is the
// node table [nv][3] in FP64 and dV the velocity cell volume.
int launch_hs_collide_noalloc(HsTables &t, const StepParams &p, float *f, const double *xi, double dV,
                              double kn, double dt);

// Trials per node that the register-resident table layout supports.
bool hs_trials_supported(int trials);

}  // namespace dvm
