// Host-side mesh: balanced quad/octree, Morton order, faces and per-cell
// upwind stencils (paper Sec. 2.1 and Sec. 3.1 step 4).  Built once per mesh
// on the host and copied to the device by the API layer.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/dvm.h"

namespace dvm {

struct Leaf {
    int lev;
    int32_t i[3];     // box coordinates at the box's own level
    uint64_t key;     // Morton key of the anchor at depth max_level
    uint8_t solid;
};

// Per-cell stencil: for axis d and side s (0 = minus, 1 = plus) list 2d+s
// holds the upwind sources on that side with weights A_face / V_cell.
// Source codes: >= 0 cell index; SRC_INFLOW freestream ghost; SRC_OUTFLOW
// the cell itself; SRC_WALL the cell itself at the velocity reflected
// along d.
enum : int32_t { SRC_INFLOW = -1, SRC_OUTFLOW = -2, SRC_WALL = -3 };
constexpr int MAX_SRC = 4;

struct Mesh {
    dvm_tree_spec spec{};
    int L = 0;
    std::vector<Leaf> leaves;              // Morton order
    std::vector<int64_t> cell_of_leaf;     // -1 for solid leaves
    std::vector<int64_t> leaf_of_cell;
    // interior faces
    std::vector<int64_t> fm, fp;
    std::vector<uint8_t> fax;
    std::vector<double> farea;
    // boundary faces
    std::vector<int64_t> bl, bother;
    std::vector<uint8_t> bax, bside, bkind;
    std::vector<double> barea;
    // stencils [ncells][6][MAX_SRC]
    std::vector<int32_t> st_src;
    std::vector<double> st_w;
    std::vector<uint8_t> st_cnt;           // [ncells][8], 6 used
    int max_cell_level = 0;
};

// Returns DVM_OK or a negative dvm_status, with a message in err.
int build_mesh(const dvm_tree_spec &spec, Mesh &m, std::string &err);
int refine_mesh(Mesh &m, const uint8_t *flag, int64_t n, std::string &err);
// Merge flagged sibling groups into their parents where 2:1 balance allows.
int coarsen_mesh(Mesh &m, const uint8_t *flag, int64_t n, std::string &err);

}  // namespace dvm
