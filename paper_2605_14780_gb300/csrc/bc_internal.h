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
  IK_ADJ = 6,
  IK_ADD = 7  // adjoint of unit copies: x_bar[dst + t] += y_bar[src + t] over runs
};

constexpr int kPMax = 8;         // largest interpolation stencil
constexpr int kChunk = 8;  // levels of one unit (blocks with >= 8 levels)
constexpr int kInterpChunk = 4;   // levels of one interpolation unit (6x768^2
                                  // cubed sphere, levels outermost: forward
                                  // 75.8 -> 65.0 us against 8)
constexpr int kFlatUnroll = 8;   // single-level units in flight per lane
#ifndef BC_RUN_UNROLL
#define BC_RUN_UNROLL 8
#endif
constexpr int kRunUnroll = BC_RUN_UNROLL;  // run values in flight per lane
constexpr int kUnitsPerWarp = 4; // 8-level units per lane and item
constexpr int kFlagSnap = 1;     // interpolation row is a unit copy of node 0

// Division of n < 2^31 by an invariant d >= 1: q = (umulhi(n, m) + n) >> s
// with s = ceil(log2 d), m = floor(2^32 (2^s - d) / d) + 1.
struct FastDiv {
  uint32_t d, m;
  int32_t s;
};

// Unit orders of a work item (Item::mode):
//   MODE_FLAT_CELL  one value (cell, level) per unit, cell fastest
//   MODE_FLAT_LEVEL one value per unit, level fastest (levels contiguous in
//                   memory: lanes of a warp then write one contiguous run)
//   mode >= 2       a unit is a cell times a chunk of `mode` levels; lanes
//                   take consecutive cells (levels far apart in memory)
//   MODE_RUNS       zero / map items only: a unit is a run of values that are
//                   contiguous in the destination and (maps) in the source;
//                   units [u0, u0 + nunits) index the run table (at most 32
//                   runs) and Item::p lanes (a power of two) share one run
//   MODE_TILE       interpolation items with levels far apart in memory:
//                   the cells' nodes lie in one small box of the source
//                   block, which the warp first copies to shared memory
//                   (cp.async) for its levels and components; the rows then
//                   read their nodes there (Item::l0 ... bwid, itp_box)
enum ItemMode : int32_t { MODE_TILE = -2, MODE_RUNS = -1, MODE_FLAT_CELL = 0, MODE_FLAT_LEVEL = 1 };

// itp_box row of a staged interpolation cell: node 0's index in the box
// (bits 0-15), nodes stepping along the box's second axis, a snapped row
constexpr int32_t kBoxIndex = 0xffff;
constexpr int32_t kBoxRows = 1 << 16;
constexpr int32_t kBoxSnap = 1 << 17;
// shared memory of one warp's staged box: interpolation and transpose
// tiles 2 KB, CSR tiles 4 KB (measured: the 4 x 4 reconstruction rows of a
// vector pair then stage 16-row tiles of 6 levels instead of 8-row tiles
// of 5, 135 -> 87 us on the 6 x 384^2 sphere; the interpolation tiles are
// 3 % faster with 2 KB)
constexpr int kStageBytesRows = 2048;
constexpr int kStageBytesCsr = 4096;
constexpr int kTileCells = 32;     // cells (rows) of one staged item, at most
constexpr int kTileLevels = 4;     // levels one lane of a staged CSR or transpose tile sums

struct alignas(16) Item {
  int32_t kind;
  int32_t mode;            // ItemMode, or the chunk length (>= 2)
  int32_t u0, nunits;      // units [u0, u0 + nunits) of the unit space
  FastDiv vol;             // cells (rows) of the sub-matrix box / row group
  FastDiv lev;             // levels of the block (lev.d)
  int32_t ctab;            // first row of the sub-matrix in the cell tables
  int32_t dst_slot, dst_slot2;
  int32_t src_slot;        // MAP source; CSR: the one slot all rows read, or -1
  int32_t p;               // INTERP: stencil points; CSR: ELL row width;
                           // MODE_RUNS: lanes per run
  int32_t table;           // CONST / INTERP / CSR: first table row of cell 0
  int32_t comp;            // INTERP source components: u | v << 16
  int32_t dst_ls, src_ls;  // level strides (elements)
  int32_t src_org;         // CSR: ELL entry of row 0 of this component
  // MODE_TILE items: levels [l0, l0 + nl) of the cells [u0, u0 + nunits)
  // (vol divides by nunits), reading a box of bw x bh cells at element
  // offset borg (level 0) of a block that steps bs0 / bs1 elements along
  // its two axes (bwid divides by bw); interpolation: the block's slots
  // start at bsrc; CSR: the entries read slot bsrc (selector 0) or bsrc2
  // (selector 1, or -1)
  int32_t l0, nl, bw, bh, bs0, bs1, bsrc;
  FastDiv bwid;
  int32_t bsrc2, borg;
};
static_assert(sizeof(Item) % 16 == 0, "Item must be a multiple of 16 bytes");

// Device-side view of a plan (passed by value to every kernel).
struct Ctx {
  void* const* slots;       // caller's device array of slot pointers
  int32_t vec_runs;         // 1: runs move 16-byte vectors (runs_vec)
  int32_t stage_warp;       // bytes of one warp's shared-memory stage in this launch
  const int32_t* slot_ls;   // level stride of every slot (elements)
  // cell tables, one row per cell of every sub-matrix box: the element
  // offset of the ghost cell (level 0) and, for maps, of its source cell
  const int32_t* ctab_d;
  const int32_t* ctab_s;
  // runs of zero / map items: {destination offset, source offset, length}
  const int4* runs;
  // interpolation: per table row {slot_base of source block, node-0 offset,
  // node step, flags}, weights [row][kPMax], rotation [row][4]
  const int4* itp_idx;
  const void* itp_w;
  const void* itp_m;
  const int32_t* itp_box;   // staged cells: node 0 in the item's box
  const int32_t* csr_box;   // staged CSR entries: place in a level's stage (slot-major)
  const int32_t* adj_box;   // staged transpose entries: the same
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

// Kernel families: item kinds that share one kernel (and one register
// budget).  Zero, constant and map items are FAM_STRUCT; interpolation and
// rotated pairs FAM_INTERP; CSR rows FAM_CSR; the transpose gather FAM_ADJ.
enum Family : int32_t { FAM_STRUCT = 0, FAM_INTERP = 1, FAM_CSR = 2, FAM_ADJ = 3 };
constexpr int kFamilies = 4;
// the persistent work-list kernel that runs every forward kind
constexpr int FAM_ALL = 4;

// Launcher (kernels.cu).  dtype: 0 = float, 1 = double.  One warp per item,
// `threads` per CTA (32..512).  grid <= 0: a plain grid with one warp per
// item; otherwise `grid` resident CTAs whose warps walk the items with a
// fixed stride, prefetching the next items' descriptors and slot pointers.
// stage: bytes of one warp's shared-memory stage that the list's staged
// tiles (MODE_TILE) need (kStageBytesRows or kStageBytesCsr), 0 when it has
// none: the launch requests that much dynamic shared memory per warp.
cudaError_t launch_family(int dtype, int family, const Ctx& ctx,
                          const Item* items, int nitems, int threads, int grid,
                          int stage, cudaStream_t s);
// CTAs of one family kernel that fit on an SM at once.
int resident_ctas(int dtype, int family, int threads, int stage);
// Persistent work-list launch: ctas_per_sm resident CTAs per SM (0: as many
// as fit) on `sms` SMs, whose warps claim the items through `counter`
// (kCtrWords words: a done count, then kSpread claim counters kCtrStride
// words apart; zero before the launch and zero again after it).  family:
// FAM_ALL (every forward kind) or one family.
constexpr unsigned kSpread = 8;      // claim counters per list
constexpr unsigned kCtrStride = 64;  // words between counters (own 256-byte lines)
constexpr unsigned kCtrWords = (kSpread + 1) * kCtrStride;
cudaError_t launch_persistent(int dtype, int family, const Ctx& ctx, const Item* items,
                              int nitems, int threads, int ctas_per_sm, int sms,
                              unsigned* counter, int stage, cudaStream_t s);
// CTAs of the persistent kernel of `family` that fit on an SM at once.
int persistent_fit(int dtype, int family, int threads, int stage);

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

// Ghost fill fused with a stencil (fused.cu).  One descriptor per slot;
// the launch's CTAs are cut per slot (cta0: the slot's first CTA): first
// one CTA per tile of kTileX x kTileY x tz data cells and level (the
// stencil outputs, read from a shared-memory copy of the tile and its
// halo), then CTAs of kFuseThreads ghost-frame values (ghost fills).
constexpr int kFuseThreads = 256;
constexpr int kFuseMaxPoints = 125;  // a 5 x 5 x 5 box
constexpr int kTileX = 32, kTileY = 8, kTileZ = 4;
constexpr int kTileVals = (kTileX + 4) * (kTileY + 4) * (kTileZ + 4);  // halo up to 2
struct FuseSlot {
  int32_t n[3], h[3];
  int32_t L, lfast;   // levels; 1: levels fastest in the value order
  int64_t s[3], ls;   // element strides of the axes and of the levels (0: one level)
  int64_t fbase;      // the slot's first frame-table entry
  int64_t cta0;       // the slot's first CTA
  int64_t tiles;      // tile CTAs of the slot (all levels); ghost CTAs follow
  int32_t nd, nf;     // data cells and ghost-frame cells of one level
  int32_t nt[3];      // tiles along each axis (tz cells deep along axis 2)
  int32_t tz;         // kTileZ, or 1 for 2-D blocks
  FastDiv dL, dnd, dnf, dn0, dn01;  // division by L, nd, nf, n[0], n[0] * n[1]
};
struct FuseCtx {
  int32_t nslots;
  const FuseSlot* slot;
  const int32_t* frame_row;  // per slot and frame cell: the row, or -1
  const int32_t* rptr;       // level-0 rows of A: entries [rptr[r], rptr[r + 1])
  const int32_t* eslot;
  const int32_t* eoff;
  const void* val;           // entry values and row constants b, plan dtype
  const void* rhs;
  const int32_t* slot_ls;    // level stride of every slot
};
struct FuseStencil {
  int32_t n;
  int32_t r[3];       // halo of the stencil along each axis (<= 2)
  int8_t o[kFuseMaxPoints][3];
  double c[kFuseMaxPoints];
};
cudaError_t launch_fused(int dtype, const FuseCtx& F, const FuseStencil& st, void* const* slots,
                         void* const* outs, int64_t nctas, cudaStream_t s);

// Box packing (pack.cu): one descriptor per box; CTAs are cut per box.
constexpr int kPackThreads = 256;
struct PackBox {
  int32_t slot0;          // slot of component 0 of the box's block
  int32_t lo[3], e[3];    // first cell (data coordinates) and extents
  int32_t L, ncomp;
  int64_t s[3], ls;       // element strides of the block (ls: 0 for one level)
  int64_t dst;            // first buffer element of the box
  int64_t count;          // values: ncomp * L * e[0] * e[1] * e[2]
  int64_t cta0;           // the box's first CTA
  FastDiv d0, d1, d2, dL; // division by e[0], e[1], e[2], L
};
cudaError_t launch_pack(int esize, const PackBox* boxes, int nboxes, int64_t nctas,
                        void* const* slots, void* buf, cudaStream_t s);

// Sets the message bc_last_error() returns on this thread (plan.cpp).
void set_last_error(const char* msg);

// Block-edge averaging (Sync rows on data cells, Sec. III-B), device side.
// Rows {slot, offset (level 0), staging offset, levels}, entries
// {slot, offset} with weights in the plan's dtype; for the adjoint, the
// columns the rows read {slot, offset, levels, 0} with their entries
// {staging offset of the row} and weights.  `stage` holds one value per row
// and level.
struct SyncCtx {
  int nrows = 0, ncols = 0;
  int lmax = 0;         // most levels of any Sync row / column
  int level_fast = 0;   // 1: consecutive threads take consecutive levels
                        //    (levels contiguous in memory), 0: consecutive
                        //    rows at one level
  const int4* row = nullptr;
  const int32_t* ptr = nullptr;
  const int2* ent = nullptr;
  const void* w = nullptr;
  const int4* col = nullptr;
  const int32_t* cptr = nullptr;
  const int32_t* cstage = nullptr;
  const void* cw = nullptr;
  void* stage = nullptr;
};
enum SyncStep : int32_t {
  SYNC_ROWS = 0,      // stage = A_sync x (reads data)
  SYNC_COMMIT = 1,    // data = stage
  SYNC_SNAPSHOT = 2,  // stage = y_bar of the Sync rows, then y_bar = 0
  SYNC_ADJOINT = 3    // x_bar += A_sync^T stage
};
cudaError_t launch_sync(int dtype, int step, const SyncCtx& s, void* const* slots,
                        const int32_t* slot_ls, cudaStream_t stream);

enum CsError : unsigned {
  CS_ERR_NOT_EDGE = 1u,     // a cell is not an edge ghost
  CS_ERR_DEPTH = 2u,        // ghost point is not on a neighbour data row
  CS_ERR_NEIGHBOUR = 4u,    // neighbour panel is not adjacent
  CS_ERR_RANGE = 8u         // stencil outside the neighbour data region
};

}  // namespace bcg
