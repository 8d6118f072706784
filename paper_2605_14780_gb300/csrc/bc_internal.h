// Internal data structures shared by the plan builder (plan.cpp) and the
// sm_103a kernels (kernels.cu, geometry.cu) of libbcgb300.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace bcg {

// Work-item kinds.  A work item is a run of units of one basic sub-matrix
// (one component, or one rotated component pair); a unit is one ghost cell
// times a chunk of up to `ch` consecutive levels.  Items are processed by one
// warp each: these are the independent convex pieces the paper instantiates
// one by one (Sec. IV-C), sized for a warp.
enum ItemKind : int32_t {
  IK_ZERO = 0,
  IK_CONST = 1,
  IK_MAP = 2,
  IK_INTERP = 3,
  IK_CSR = 4,
  IK_INTERP_PAIR = 5,
  IK_ADJ = 6
};

constexpr int kPMax = 8;         // largest interpolation stencil
constexpr int kChunk = 8;        // levels of one unit (blocks with >= 8 levels)
constexpr int kFlatUnroll = 8;   // single-level units in flight per lane
constexpr int kUnitsPerWarp = 4; // 8-level units per lane and item
constexpr int kFlagSnap = 1;     // interpolation row is a unit copy of node 0

// Division of n < 2^31 by an invariant d >= 1: q = (umulhi(n, m) + n) >> s
// with s = ceil(log2 d), m = floor(2^32 (2^s - d) / d) + 1.
struct FastDiv {
  uint32_t d, m;
  int32_t s;
};

struct alignas(16) Item {
  int32_t kind;
  int32_t ch;              // levels per unit: 1 (flat) or kChunk
  int32_t u0, nunits;      // units [u0, u0 + nunits) of the unit space
  FastDiv vol;             // cells (rows) of the sub-matrix box / row group
  FastDiv w0, w1;          // box extents on axes 0 and 1
  int32_t L;               // levels of the block
  int32_t dst_slot, dst_slot2;
  int32_t src_slot, p;
  int32_t table;           // first table row of cell 0 of this component
  int32_t comp, comp2;     // INTERP: source components (pair: u, v)
  int32_t dst_org, dst_s0, dst_s1, dst_s2, dst_ls;   // element offsets
  int32_t src_org, src_s0, src_s1, src_s2, src_ls;   // MAP source
  int32_t pad[1];
};
static_assert(sizeof(Item) % 16 == 0, "Item must be a multiple of 16 bytes");

// Device-side view of a plan (passed by value to every kernel).
struct Ctx {
  void* const* slots;       // caller's device array of slot pointers
  const int32_t* slot_ls;   // level stride of every slot (elements)
  // interpolation: per table row {slot_base of source block, node-0 offset,
  // node step, flags}, weights [row][kPMax], rotation [row][4]
  const int4* itp_idx;
  const void* itp_w;
  const void* itp_m;
  // CSR rows (global row numbering): entry count per row, ELL entries
  // (a row's entries start at item.src_org + q * item.p), per-row constant
  const int32_t* csr_nnz;
  const int32_t* csr_slot;
  const int32_t* csr_off;
  const void* csr_val;
  const void* csr_rhs;
  // CONST values [row]
  const void* const_val;
  // transpose of A: rows are data values (slot, offset), entries the ghost
  // values that read them
  const int32_t* arow_slot;
  const int32_t* arow_off;
  const int64_t* adj_ptr;
  const int32_t* aent_slot;
  const int32_t* aent_off;
  const void* aent_w;
};

// Launchers (kernels.cu).  dtype: 0 = float, 1 = double.
// One warp per item; `threads` per CTA (a multiple of 32).
cudaError_t launch_items(int dtype, const Ctx& ctx, const Item* items,
                         int nitems, int threads, cudaStream_t s);
// Persistent: `grid` CTAs whose warps claim items from counter[0].
cudaError_t launch_persistent(int dtype, const Ctx& ctx, const Item* items,
                              int nitems, int threads, int grid,
                              unsigned* counter, cudaStream_t s);

// Cubed-sphere geometry (geometry.cu).
struct CsPanels {
  int32_t N, h, p, rotate;
  int32_t slot_base[6];
  int64_t s0[6], s1[6];
};
// cells: {panel index 0..5, i, j, table row}; writes itp_idx rows, FP64
// weights [row][kPMax] and rotations [row][4]; err gets error bits.
cudaError_t launch_cs_geometry(const CsPanels& pan, const int4* cells,
                               int ncells, int4* idx, double* w, double* m,
                               unsigned* err, cudaStream_t s);

// Sets the message bc_last_error() returns on this thread (plan.cpp).
void set_last_error(const char* msg);

enum CsError : unsigned {
  CS_ERR_NOT_EDGE = 1u,     // a cell is not an edge ghost
  CS_ERR_DEPTH = 2u,        // ghost point is not on a neighbour data row
  CS_ERR_NEIGHBOUR = 4u,    // neighbour panel is not adjacent
  CS_ERR_RANGE = 8u         // stencil outside the neighbour data region
};

}  // namespace bcg
