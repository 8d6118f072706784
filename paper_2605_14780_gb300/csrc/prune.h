// Dead-ghost elimination (Sec. IV-C), host side: cut basic sub-matrices to
// the ghost values a stencil reads.  Used by bc_plan_create_pruned.
#pragma once

#include <cstdint>
#include <deque>
#include <vector>

#include "../../include/bc.h"

namespace bcg {

// A sub-matrix list built on the host (pruned pieces, lowered rows) and the
// payload arrays it points into (deque elements keep their addresses while
// more are added).
struct SubStore {
  std::vector<bc_submatrix> subs;
  std::vector<int> origin;  // index of each sub-matrix in the list it came from
  std::deque<std::vector<double>> dbl;
  std::deque<std::vector<int32_t>> i32;
  std::deque<std::vector<int64_t>> i64;
};

// Every sub-matrix box becomes the disjoint boxes of its live cells (a ghost
// cell g is live when g - o is a data cell of its block for one of the
// noffsets stencil offsets o = offsets[3n .. 3n+2]); sub-matrices with no
// live cell are dropped, and ones the plan would reject pass unchanged.
bc_status prune_submatrices(const bc_grid* grid, const bc_submatrix* subs, int nsubs,
                            const int32_t* offsets, int noffsets, SubStore& out);

}  // namespace bcg
