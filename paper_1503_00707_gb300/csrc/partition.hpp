// Space-filling-curve partition of the cells into contiguous Morton ranges,
// with each range's upwind halo (paper Sec. 3.3: the multi-GPU solver splits
// the Morton-ordered cells into pieces of equal work and exchanges the ghost
// cells that the advection stencils of a piece read from other pieces).
// Host work only.
#pragma once
#include <cstdint>
#include <vector>

namespace dvm {

struct Part {
    int64_t c0 = 0, c1 = 0;          // owned cells [c0, c1) in Morton order
    std::vector<int64_t> ghosts;     // other cells the owned stencils read, ascending
};

// Device stencil encoding of every list entry: source cell | group flip << 28,
// the inflow ghost as cell `ncells` (shared by the step and the partition).
// st_src / st_cnt are the mesh's [ncells][6][MAX_SRC] codes and [ncells][8]
// counts.
void encode_stencils(const std::vector<int32_t> &st_src, int64_t ncells, std::vector<int32_t> &enc);

// nparts contiguous ranges and the ghost list of each from the encoded
// stencils.  Without weights: ncells / nparts cells each (the first ncells %
// nparts ranges one cell longer: every cell carries the same work).  With
// per-cell weights (>= 0): range p ends at the first cell where the weight up
// to the cell's middle passes (p + 1) W / nparts, every range non-empty.
void partition_cells(int64_t ncells, int nparts, const std::vector<int32_t> &enc,
                     const std::vector<uint8_t> &st_cnt, std::vector<Part> &parts,
                     const double *weight = nullptr);

// The stencils of one part in its local numbering: owned cell c -> c - c0,
// ghost k -> (c1 - c0) + k, inflow ghost -> (c1 - c0) + ghosts.size().
void local_stencils(const Part &part, int64_t ncells, const std::vector<int32_t> &enc,
                    std::vector<int32_t> &local);

}  // namespace dvm
