// Hard-sphere discrete collision integral (paper Sec. 3.2, Eqs. 3-6):
// seeded trial tables built on the host, collision kernel on the device.
#pragma once
#include <cstdint>
#include <functional>
#include <string>
#include <vector>

#include "kernels.hpp"

namespace dvm {

struct HsTables {
    bool ready = false;
    int trials = 0;
    uint64_t seed = 0;
    int nv = 0;
    int64_t discarded = 0;
    // [trials][nv] entries {gamma | l << 16, m, bits(b), 0}; a discarded
    // trial keeps b = 0 and points at the node itself.
    std::vector<uint32_t> host;
    void *dev = nullptr;
    double *d_corr = nullptr;   // per-cell scratch, see k_hs.cu
    float *d_bc = nullptr;      // per-cell B and C scratch [ncells][2][nv]
    int64_t bc_cells = 0;
};

using DevAlloc = std::function<void *(size_t)>;
using DevFree = std::function<void(void *)>;

// Output n (0-based) of the SplitMix64 stream seeded with `seed`.
uint64_t splitmix64_at(uint64_t seed, uint64_t n);

int hs_build(HsTables &t, const int n[3], const double lo[3], const double h[3],
             const std::vector<double> &xi, int trials, uint64_t seed, std::string &err,
             const DevAlloc &alloc, const DevFree &dfree);
void hs_free(HsTables &t, const DevFree &dfree);

// Per-cell scratch for ncells cells (B, C and the correction sums).
int hs_prepare(HsTables &t, int64_t ncells, const DevAlloc &alloc, const DevFree &dfree);

// f (storage precision, already holding f* from the transport launch) is
// updated in place: f <- f* + dt/Kn * I(f*).
int launch_hs_collide(HsTables &t, const StepParams &p, void *f, double kn, double dt);

}  // namespace dvm
