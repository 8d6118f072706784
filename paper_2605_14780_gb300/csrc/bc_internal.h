// Internal data structures shared by the plan builder (plan.cpp) and the
// sm_103a kernels (kernels.cu, geometry.cu) of libbcgb300.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace bcg {

// Work-item kinds.  A work item is a rectangular run of ghost cells of one
// basic sub-matrix (one component, or one rotated component pair) times a
// range of levels: the independent convex pieces the paper instantiates one
// by one (Sec. IV-C), here executed by one CTA each.
enum ItemKind : int32_t {
  IK_ZERO = 0,
  IK_CONST = 1,
  IK_MAP = 2,
  IK_INTERP = 3,
  IK_CSR = 4,
  IK_INTERP_PAIR = 5,
  IK_ADJ = 6
};

// CELL: each thread owns one cell and loops over the item's levels.
// FLAT: the item is a flat range of (cell, level) values, cell fastest; each
//       thread handles up to kFlatUnroll of them (used when levels are few).
enum ItemMode : int32_t { MODE_CELL = 0, MODE_FLAT = 1 };

constexpr int kPMax = 8;         // largest interpolation stencil
constexpr int kLevelUnroll = 8;  // levels in flight per thread (CELL mode)
constexpr int kFlatUnroll = 8;   // values in flight per thread (FLAT mode)
constexpr int kFlagSnap = 1;     // interpolation row is a unit copy of node 0

struct alignas(16) Item {
  int32_t kind, mode;
  int32_t ncell, q0;       // CELL: cells [q0, q0+ncell); FLAT: flat values
  int32_t l0, nlev;        // level range
  int32_t dst_slot, dst_slot2;
  int32_t src_slot, p;
  int32_t W0, W1;          // extents of the sub-matrix box, axes 0 and 1
  int32_t vol;             // cells of the sub-matrix box
  int32_t table;           // first table row of cell 0 of this component
  int32_t comp, comp2;     // INTERP: source components (pair: u, v)
  int64_t dst_org;         // dst offset of the box origin, level 0
  int64_t dst_s0, dst_s1, dst_s2, dst_ls;
  int64_t src_org;         // MAP: src offset of the image of the origin
  int64_t src_s0, src_s1, src_s2, src_ls;
};
static_assert(sizeof(Item) % 16 == 0, "Item must be a multiple of 16 bytes");
constexpr int kItemWords = sizeof(Item) / 4;

// Device-side view of a plan (passed by value to every kernel).
struct Ctx {
  void* const* slots;       // caller's device array of slot pointers
  const int64_t* slot_ls;   // level stride of every slot
  // interpolation: per table row {slot_base of source block, node-0 offset,
  // node step, flags}, weights [row][kPMax], rotation [row][4]
  const int4* itp_idx;
  const void* itp_w;
  const void* itp_m;
  // CSR rows (global row numbering), entries, per-row constant
  const int64_t* csr_ptr;
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
cudaError_t launch_items(int dtype, const Ctx& ctx, const Item* items,
                         int nitems, int threads, cudaStream_t s);
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

enum CsError : unsigned {
  CS_ERR_NOT_EDGE = 1u,     // a cell is not an edge ghost
  CS_ERR_DEPTH = 2u,        // ghost point is not on a neighbour data row
  CS_ERR_NEIGHBOUR = 4u,    // neighbour panel is not adjacent
  CS_ERR_RANGE = 8u         // stencil outside the neighbour data region
};

}  // namespace bcg
