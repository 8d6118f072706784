// Host side of libbcgb300: validation of the basic sub-matrices, the work
// list, the transpose of A, device tables and the C ABI of include/bc.h.
//
// A plan turns the user's basic sub-matrices (arxiv 2605.14780, Sec. IV-A,
// Table II) into
//   * explicit level-0 rows of A and b (FP64), kept on the host for the
//     transpose and for bc_plan_export_csr;
//   * kind-specific device tables (constants, interpolation stencils and
//     rotations, CSR rows) in the plan's dtype;
//   * a work list of rectangular cell runs x level ranges (the disjoint
//     convex pieces of Sec. IV-C), executed by the kernels of kernels.cu;
//   * the transpose of A (rows = data values read by some ghost, entries in
//     ascending ghost order) and its own work list, for the adjoint.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <memory>
#include <mutex>
#include <new>
#include <numeric>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include <map>
#include <unordered_map>
#include <unordered_set>

#include <nvtx3/nvToolsExt.h>

#include "../../include/bc.h"
#include "bc_internal.h"
#include "prune.h"
#include "quadrature.h"

using namespace bcg;

// cell (i, j, k) of block B at element offset `off` (defined with the C ABI)
bool decode_cell(const bc_block& B, int64_t off, int& i, int& j, int& k);

namespace {

thread_local std::string g_last_error;

bc_status fail(bc_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return st;
}

// Fault injection on the host, for tests of the error paths: with
// BC_FAULT_INJECT=alloc:<n> in the environment, the n-th device allocation
// of a plan creation or autotune call (counting from 1) fails with
// cudaErrorMemoryAllocation instead of allocating.  No GPU fault is made.
thread_local int g_alloc_countdown = 0;  // 0: off

void arm_fault_injection() {
  g_alloc_countdown = 0;
  const char* v = std::getenv("BC_FAULT_INJECT");
  if (v && std::strncmp(v, "alloc:", 6) == 0) g_alloc_countdown = std::max(0, std::atoi(v + 6));
}

cudaError_t dev_malloc(void** p, size_t bytes) {
  if (g_alloc_countdown > 0 && --g_alloc_countdown == 0) {
    *p = nullptr;
    return cudaErrorMemoryAllocation;
  }
  return cudaMalloc(p, bytes);
}

bc_status cuda_fail(cudaError_t e, const char* what) {
  return fail(e == cudaErrorMemoryAllocation ? BC_ERR_NOMEM : BC_ERR_CUDA,
              "%s: %s", what, cudaGetErrorString(e));
}

struct Sub {
  int kind = 0, block = 0;
  int lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0}, W[3] = {0, 0, 0};
  int vol = 0;
  std::vector<int> comps;
  int src_block = -1;
  int perm[3] = {0, 1, 2}, sign[3] = {1, 1, 1}, offset[3] = {0, 0, 0};
  int p = 0, geometry = 0, rot_u = -1, rot_v = -1;
  int table = 0;  // CONST/CSR: first row of comp 0; INTERP: first cell row
  int ell_base = 0, ell_w = 1;  // CSR: ELL entries of row 0, row width
  std::vector<int> csr_common;  // CSR: the one slot a component's rows read, or -1
  int ctab = 0;                 // first row in the cell tables
};

struct ExplicitRows {
  std::vector<int32_t> slot;
  std::vector<int64_t> off;
  std::vector<int64_t> ptr{0};
  std::vector<int32_t> cslot;
  std::vector<int64_t> coff;
  std::vector<double> val;
  std::vector<double> rhs;
  void begin_row(int32_t s, int64_t o, double b) {
    slot.push_back(s);
    off.push_back(o);
    rhs.push_back(b);
  }
  void entry(int32_t s, int64_t o, double v) {
    cslot.push_back(s);
    coff.push_back(o);
    val.push_back(v);
  }
  void end_row() { ptr.push_back((int64_t)val.size()); }
};

struct DevBuf {
  void* base = nullptr;
  size_t bytes = 0;
  ~DevBuf() {
    if (base) cudaFree(base);
  }
};

}  // namespace

struct bc_plan {
  int dtype = 0, esize = 4;
  std::vector<bc_block> blocks;
  std::vector<int32_t> slot_base, slot_block;
  std::vector<int32_t> slot_ls;
  int nslots = 0;
  std::vector<Sub> subs;
  // index into subs of every sub-matrix of the caller's list (-1: Sync rows,
  // or none); meaningless for pruned plans
  std::vector<int> sub_of_input;
  bool pruned = false;
  // user CSR rows that read ghost values (bc_plan_opts.ghost_sweeps) are
  // accepted only in the host-only plan that folds them; the ghost columns
  // met are recorded by (slot, offset) key
  bool allow_ghost_cols = false;
  std::unordered_set<int64_t> ghost_cols;
  ExplicitRows rows;  // level 0, in sub-matrix order
  // host tables (FP64 copies)
  std::vector<int4> itp_idx;
  std::vector<double> itp_w, itp_m;
  std::vector<int32_t> itp_box;  // staged interpolation: node 0 in its tile's box
  // staged CSR / transpose entries: the value's place in one level of its
  // tile's stage, selector * (box cells) + box index
  std::vector<int32_t> csr_box;
  std::vector<int32_t> adj_box;
  // user CSR rows stored as ELL blocks (one width per sub-matrix)
  std::vector<int32_t> csr_nnz;
  std::vector<int32_t> csr_slot, csr_off;
  std::vector<double> csr_val, csr_rhs;
  std::vector<double> const_val;
  // cell tables: ghost-cell offset and (maps) source-cell offset, level 0
  std::vector<int32_t> ctab_d, ctab_s;
  // runs of zero / map items (rebuilt with the work lists)
  std::vector<int4> runs;
  // transpose
  std::vector<int32_t> arow_slot, arow_off;
  std::vector<int64_t> adj_ptr{0};
  std::vector<int32_t> aent_slot, aent_off;
  std::vector<double> aent_w;
  int64_t adj_rows_total = 0, adj_nnz_total = 0;  // before unit copies leave the gather
  // adjoint of unit copies: runs {data offset, ghost offset, length} of the
  // transpose rows that hold one unit-weight entry, by (data slot, ghost slot)
  struct AddSeg {
    int32_t dslot, sslot, r0, nr;
  };
  std::vector<int4> add_runs;
  std::vector<AddSeg> add_segs;
  bool has_adjoint = false;
  // block-edge averaging (Sync rows on data cells): rows {slot, offset,
  // staging offset, levels}, CSR entries, and for the adjoint the columns
  // they read with {staging offset of the row, weight} entries
  struct SyncTabs {
    std::vector<int4> row;
    std::vector<int32_t> ptr{0};
    std::vector<int2> ent;
    std::vector<double> w;
    std::vector<int4> col;
    std::vector<int32_t> cptr{0};
    std::vector<int32_t> cstage;
    std::vector<double> cw;
    int64_t stage = 0;  // staging values (rows x levels)
  } sync;
  SyncCtx sync_ctx{};
  // work lists
  std::vector<Item> items, adj_items, adj_zero, adj_add;
  std::vector<Item> fam_items[kFamilies];  // batched form: per family, sub-matrix order
  std::vector<Item> all_items;  // persistent form: every forward item, longest first
  // per family (FAM_ADJ: also the adjoint gather) and FAM_ALL: bytes of a
  // warp's shared-memory stage that the list's staged tiles need (0: none)
  int staged[kFamilies + 1] = {0, 0, 0, 0, 0};
  std::vector<int> sub_begin, sub_end;
  int type_begin[5] = {0, 0, 0, 0, 0}, type_end[5] = {0, 0, 0, 0, 0};
  // device
  DevBuf tables, work, fuse;
  FuseCtx fuse_ctx{};
  int64_t fuse_ctas = 0;
  Ctx ctx{};
  Item* d_items = nullptr;
  Item* d_fam[kFamilies] = {nullptr, nullptr, nullptr, nullptr};
  // the batched form runs the families side by side: fork to these streams
  cudaStream_t aux[kFamilies - 1] = {nullptr, nullptr, nullptr};
  cudaEvent_t ev_fork = nullptr;
  cudaEvent_t ev_join[kFamilies - 1] = {nullptr, nullptr, nullptr};
  ~bc_plan() {
    for (auto& a : aux)
      if (a) cudaStreamDestroy(a);
    for (auto& e : ev_join)
      if (e) cudaEventDestroy(e);
    if (ev_fork) cudaEventDestroy(ev_fork);
  }
  Item* d_adj = nullptr;
  Item* d_adj_zero = nullptr;
  Item* d_all = nullptr;
  // work counters of the persistent launches: one pair per stream that
  // applies the plan (zero between launches)
  unsigned* d_ctr = nullptr;
  std::mutex ctr_mu;
  std::vector<void*> ctr_streams;
  int num_sms = 1;
  uint64_t hash = 0;  // of the rows, layouts and untuned options (autotune cache key)
  bc_plan_opts opts{};
  bc_stats stats{};
};

namespace {

int64_t cell_offset(const bc_block& b, int i, int j, int k) {
  return (int64_t)(i + b.h[0]) * b.stride[0] + (int64_t)(j + b.h[1]) * b.stride[1] +
         (int64_t)(k + b.h[2]) * b.stride[2];
}

bool in_data(const bc_block& b, int i, int j, int k) {
  return i >= 0 && i < b.n[0] && j >= 0 && j < b.n[1] && k >= 0 && k < b.n[2];
}

bool in_full(const bc_block& b, int i, int j, int k) {
  return i >= -b.h[0] && i < b.n[0] + b.h[0] && j >= -b.h[1] && j < b.n[1] + b.h[1] &&
         k >= -b.h[2] && k < b.n[2] + b.h[2];
}

int64_t col_key(int slot, int64_t off) { return ((int64_t)slot << 32) | (uint32_t)off; }

// A named NVTX range over one entry point (visible to Nsight tools, which
// can also filter kernels by it; without a tool attached it costs a branch).
struct TraceRange {
  explicit TraceRange(const char* name) { nvtxRangePushA(name); }
  ~TraceRange() { nvtxRangePop(); }
  TraceRange(const TraceRange&) = delete;
  TraceRange& operator=(const TraceRange&) = delete;
};

bc_status validate_grid(const bc_grid* g, bc_plan* P) {
  if (!g) return fail(BC_ERR_INVALID_ARG, "grid is NULL");
  if (g->dtype != BC_F32 && g->dtype != BC_F64)
    return fail(BC_ERR_INVALID_ARG, "unknown dtype %d", g->dtype);
  if (g->nblocks <= 0 || !g->blocks)
    return fail(BC_ERR_INVALID_ARG, "grid has no blocks");
  P->dtype = g->dtype;
  P->esize = g->dtype == BC_F64 ? 8 : 4;
  P->blocks.assign(g->blocks, g->blocks + g->nblocks);
  int64_t slots = 0;
  for (int b = 0; b < g->nblocks; ++b) {
    const bc_block& B = P->blocks[b];
    for (int d = 0; d < 3; ++d) {
      if (B.n[d] < 1) return fail(BC_ERR_INVALID_ARG, "block %d: n[%d] < 1", b, d);
      if (B.h[d] < 0) return fail(BC_ERR_INVALID_ARG, "block %d: h[%d] < 0", b, d);
      if (B.stride[d] < 1)
        return fail(BC_ERR_INVALID_ARG, "block %d: stride[%d] < 1", b, d);
    }
    if (B.nlevels < 1 || B.ncomp < 1 || B.ncomp > 32)
      return fail(BC_ERR_INVALID_ARG, "block %d: bad nlevels/ncomp", b);
    if (B.nlevels > 1 && B.level_stride < 1)
      return fail(BC_ERR_INVALID_ARG, "block %d: level_stride < 1", b);
    const int64_t maxoff = cell_offset(B, B.n[0] + B.h[0] - 1, B.n[1] + B.h[1] - 1,
                                       B.n[2] + B.h[2] - 1) +
                           (int64_t)(B.nlevels - 1) * (B.nlevels > 1 ? B.level_stride : 0);
    if (maxoff >= (int64_t(1) << 31) - 1)
      return fail(BC_ERR_UNSUPPORTED,
                  "block %d: one component spans >= 2^31 elements", b);
    P->slot_base.push_back((int32_t)slots);
    for (int c = 0; c < B.ncomp; ++c) {
      P->slot_block.push_back(b);
      P->slot_ls.push_back((int32_t)(B.nlevels > 1 ? B.level_stride : 0));
    }
    slots += B.ncomp;
    if (slots > (1 << 24)) return fail(BC_ERR_UNSUPPORTED, "too many slots");
  }
  P->nslots = (int)slots;
  return BC_OK;
}

// -- coverage bitmap ----------------------------------------------------------
struct Coverage {
  std::vector<std::vector<uint8_t>> map;  // per slot, over the full box
  const std::vector<bc_block>* blocks;
  const std::vector<int32_t>* slot_block;
  size_t index(const bc_block& B, int i, int j, int k) const {
    const size_t F0 = B.n[0] + 2 * B.h[0], F1 = B.n[1] + 2 * B.h[1];
    return ((size_t)(k + B.h[2]) * F1 + (size_t)(j + B.h[1])) * F0 + (size_t)(i + B.h[0]);
  }
  bool mark(int slot, int i, int j, int k) {
    const bc_block& B = (*blocks)[(*slot_block)[slot]];
    auto& m = map[slot];
    if (m.empty()) {
      const size_t F = (size_t)(B.n[0] + 2 * B.h[0]) * (B.n[1] + 2 * B.h[1]) *
                       (B.n[2] + 2 * B.h[2]);
      m.assign(F, 0);
    }
    uint8_t& c = m[index(B, i, j, k)];
    if (c) return false;
    c = 1;
    return true;
  }
};

template <typename F>
void for_box(const Sub& s, F f) {
  int q = 0;
  for (int k = s.lo[2]; k < s.hi[2]; ++k)
    for (int j = s.lo[1]; j < s.hi[1]; ++j)
      for (int i = s.lo[0]; i < s.hi[0]; ++i) f(q++, i, j, k);
}

bc_status read_sub(bc_plan* P, const bc_submatrix& m, int idx, Sub& s) {
  s.kind = m.kind;
  s.block = m.block;
  if (m.kind < BC_ZERO || m.kind > BC_SYNC)
    return fail(BC_ERR_INVALID_ARG, "sub-matrix %d: unknown kind %d", idx, m.kind);
  if (m.block < 0 || m.block >= (int)P->blocks.size())
    return fail(BC_ERR_INVALID_ARG, "sub-matrix %d: bad block %d", idx, m.block);
  const bc_block& B = P->blocks[m.block];
  int64_t vol = 1;
  for (int d = 0; d < 3; ++d) {
    s.lo[d] = m.lo[d];
    s.hi[d] = m.hi[d];
    if (m.hi[d] <= m.lo[d])
      return fail(BC_ERR_INVALID_ARG, "sub-matrix %d: empty box on axis %d", idx, d);
    if (m.lo[d] < -B.h[d] || m.hi[d] > B.n[d] + B.h[d])
      return fail(BC_ERR_OUT_OF_RANGE, "sub-matrix %d: box leaves the full region", idx);
    s.W[d] = m.hi[d] - m.lo[d];
    vol *= s.W[d];
  }
  if (vol > (int64_t(1) << 30))
    return fail(BC_ERR_UNSUPPORTED, "sub-matrix %d: box too large", idx);
  s.vol = (int)vol;
  if (m.ncomps < 1 || !m.comps)
    return fail(BC_ERR_INVALID_ARG, "sub-matrix %d: no components", idx);
  for (int c = 0; c < m.ncomps; ++c) {
    const int cc = m.comps[c];
    if (cc < 0 || cc >= B.ncomp)
      return fail(BC_ERR_INVALID_ARG, "sub-matrix %d: bad component %d", idx, cc);
    if (std::find(s.comps.begin(), s.comps.end(), cc) != s.comps.end())
      return fail(BC_ERR_INVALID_ARG, "sub-matrix %d: repeated component", idx);
    s.comps.push_back(cc);
  }
  return BC_OK;
}

bc_status add_zero_const(bc_plan* P, const bc_submatrix& m, int idx, Sub& s) {
  const bc_block& B = P->blocks[s.block];
  if (s.kind == BC_CONST) {
    if (!m.values) return fail(BC_ERR_INVALID_ARG, "sub-matrix %d: values is NULL", idx);
    s.table = (int)P->const_val.size();
    for (size_t c = 0; c < s.comps.size(); ++c)
      for (int q = 0; q < s.vol; ++q) {
        const double v = m.values[c * s.vol + q];
        if (!std::isfinite(v))
          return fail(BC_ERR_INVALID_ARG, "sub-matrix %d: non-finite value", idx);
        P->const_val.push_back(v);
      }
  }
  for (size_t c = 0; c < s.comps.size(); ++c) {
    const int slot = P->slot_base[s.block] + s.comps[c];
    for_box(s, [&](int q, int i, int j, int k) {
      P->rows.begin_row(slot, cell_offset(B, i, j, k),
                        s.kind == BC_CONST ? P->const_val[s.table + c * s.vol + q] : 0.0);
      P->rows.end_row();
    });
  }
  return BC_OK;
}

constexpr int kMaxMapScale = 1 << 16;

bc_status add_map(bc_plan* P, const bc_submatrix& m, int idx, Sub& s) {
  const bc_block& B = P->blocks[s.block];
  if (m.src_block < 0 || m.src_block >= (int)P->blocks.size())
    return fail(BC_ERR_INVALID_ARG, "sub-matrix %d: bad src_block", idx);
  s.src_block = m.src_block;
  const bc_block& S = P->blocks[m.src_block];
  bool seen[3] = {false, false, false};
  for (int d = 0; d < 3; ++d) {
    if (m.perm[d] < 0 || m.perm[d] > 2 || seen[m.perm[d]])
      return fail(BC_ERR_INVALID_ARG, "sub-matrix %d: perm is not a permutation", idx);
    seen[m.perm[d]] = true;
    // +-1: halo copies and reflections; |s| > 1: injection between blocks
    // whose grids are slices of one global grid with steps in ratio |s|
    if (m.sign[d] == 0 || m.sign[d] > kMaxMapScale || m.sign[d] < -kMaxMapScale)
      return fail(BC_ERR_INVALID_ARG, "sub-matrix %d: map scale must be nonzero, |scale| <= %d",
                  idx, kMaxMapScale);
    s.perm[d] = m.perm[d];
    s.sign[d] = m.sign[d];
    s.offset[d] = m.offset[d];
  }
  if (S.nlevels != B.nlevels)
    return fail(BC_ERR_INVALID_ARG, "sub-matrix %d: source has another level count", idx);
  for (int c : s.comps)
    if (c >= S.ncomp)
      return fail(BC_ERR_INVALID_ARG, "sub-matrix %d: source lacks component %d", idx, c);
  // the image of a box is a box: check its extent on every source axis
  for (int d = 0; d < 3; ++d) {
    const int e = s.perm[d];
    const int64_t a = (int64_t)s.sign[d] * s.lo[e] + s.offset[d];
    const int64_t b = (int64_t)s.sign[d] * (s.hi[e] - 1) + s.offset[d];
    const int64_t mn = std::min(a, b), mx = std::max(a, b);
    if (mn < 0 || mx >= S.n[d]) {
      const bool reflect = (m.src_block == s.block && e == d);
      return fail(reflect ? BC_ERR_HALO_TOO_WIDE : BC_ERR_COLUMN_NOT_DATA,
                  "sub-matrix %d: map image leaves the source data on axis %d", idx, d);
    }
  }
  for (int c : s.comps) {
    const int slot = P->slot_base[s.block] + c;
    const int sslot = P->slot_base[s.src_block] + c;
    for_box(s, [&](int, int i, int j, int k) {
      const int g[3] = {i, j, k};
      int src[3];
      for (int d = 0; d < 3; ++d) src[d] = s.sign[d] * g[s.perm[d]] + s.offset[d];
      P->rows.begin_row(slot, cell_offset(B, i, j, k), 0.0);
      P->rows.entry(sslot, cell_offset(S, src[0], src[1], src[2]), 1.0);
      P->rows.end_row();
    });
  }
  return BC_OK;
}

bc_status add_csr(bc_plan* P, const bc_submatrix& m, int idx, Sub& s) {
  const bc_block& B = P->blocks[s.block];
  if (!m.row_ptr || !m.col_block || !m.col_comp || !m.col_ijk || !m.val)
    return fail(BC_ERR_INVALID_ARG, "sub-matrix %d: CSR arrays missing", idx);
  const int64_t nrows = (int64_t)s.comps.size() * s.vol;
  if (m.row_ptr[0] != 0) return fail(BC_ERR_INVALID_ARG, "sub-matrix %d: row_ptr[0] != 0", idx);
  for (int64_t r = 0; r < nrows; ++r)
    if (m.row_ptr[r + 1] < m.row_ptr[r])
      return fail(BC_ERR_INVALID_ARG, "sub-matrix %d: row_ptr not monotone", idx);
  s.table = (int)P->csr_nnz.size();
  // ELL width of this sub-matrix: its longest row
  int64_t w = 1;
  for (int64_t r = 0; r < nrows; ++r) w = std::max<int64_t>(w, m.row_ptr[r + 1] - m.row_ptr[r]);
  // widths up to 8 are padded to 4 or 8, wider rows to a multiple of 8, and
  // rows start on 16-byte boundaries, so the kernels load a row's entries
  // as vectors (wide rows in blocks of 8)
  w = w <= 4 ? 4 : (w + 7) / 8 * 8;
  if (w * nrows > (int64_t(1) << 30))
    return fail(BC_ERR_UNSUPPORTED, "sub-matrix %d: CSR rows too long", idx);
  while (P->csr_slot.size() % 4) {
    P->csr_slot.push_back(0);
    P->csr_off.push_back(0);
    P->csr_val.push_back(0.0);
  }
  s.ell_w = (int)w;
  s.ell_base = (int)P->csr_slot.size();
  P->csr_slot.resize(P->csr_slot.size() + nrows * w, 0);
  P->csr_off.resize(P->csr_off.size() + nrows * w, 0);
  P->csr_val.resize(P->csr_val.size() + nrows * w, 0.0);
  for (size_t c = 0; c < s.comps.size(); ++c) {
    const int slot = P->slot_base[s.block] + s.comps[c];
    bc_status st = BC_OK;
    for_box(s, [&](int q, int i, int j, int k) {
      if (st != BC_OK) return;
      const int64_t r = (int64_t)c * s.vol + q;
      const double b = m.rhs ? m.rhs[r] : 0.0;
      if (!std::isfinite(b)) {
        st = fail(BC_ERR_INVALID_ARG, "sub-matrix %d: non-finite rhs", idx);
        return;
      }
      P->rows.begin_row(slot, cell_offset(B, i, j, k), b);
      for (int64_t e = m.row_ptr[r]; e < m.row_ptr[r + 1]; ++e) {
        const int cb = m.col_block[e], cc = m.col_comp[e];
        const int ci = m.col_ijk[3 * e], cj = m.col_ijk[3 * e + 1], ck = m.col_ijk[3 * e + 2];
        if (cb < 0 || cb >= (int)P->blocks.size() || cc < 0 || cc >= P->blocks[cb].ncomp) {
          st = fail(BC_ERR_INVALID_ARG, "sub-matrix %d: bad column block/component", idx);
          return;
        }
        const bc_block& C = P->blocks[cb];
        const bool ghost_col = !in_data(C, ci, cj, ck);
        if (ghost_col && !(P->allow_ghost_cols && in_full(C, ci, cj, ck))) {
          st = fail(BC_ERR_COLUMN_NOT_DATA, "sub-matrix %d: column (%d,%d,%d) of block %d is not data",
                    idx, ci, cj, ck, cb);
          return;
        }
        if (C.nlevels != B.nlevels) {
          st = fail(BC_ERR_INVALID_ARG, "sub-matrix %d: column block has another level count", idx);
          return;
        }
        if (!std::isfinite(m.val[e])) {
          st = fail(BC_ERR_INVALID_ARG, "sub-matrix %d: non-finite value", idx);
          return;
        }
        const int cs = P->slot_base[cb] + cc;
        const int64_t co = cell_offset(C, ci, cj, ck);
        if (ghost_col) P->ghost_cols.insert(col_key(cs, co));
        P->rows.entry(cs, co, m.val[e]);
        const int64_t pos = s.ell_base + r * w + (e - m.row_ptr[r]);
        P->csr_slot[pos] = cs;
        P->csr_off[pos] = (int32_t)co;
        P->csr_val[pos] = m.val[e];
      }
      P->rows.end_row();
      P->csr_rhs.push_back(b);
      P->csr_nnz.push_back((int32_t)(m.row_ptr[r + 1] - m.row_ptr[r]));
    });
    if (st != BC_OK) return st;
    // the one slot all rows of this component read, if there is one
    int common = -2;
    for (int64_t r = (int64_t)c * s.vol; r < (int64_t)(c + 1) * s.vol && common != -1; ++r)
      for (int64_t e = m.row_ptr[r]; e < m.row_ptr[r + 1]; ++e) {
        const int cs = P->slot_base[m.col_block[e]] + m.col_comp[e];
        if (common == -2) common = cs;
        else if (common != cs) { common = -1; break; }
      }
    s.csr_common.push_back(common < 0 ? -1 : common);
  }
  return BC_OK;
}

// INTERP rows are appended after the geometry is known (cubed sphere: after
// the GPU kernel); this records the stencil tables.
// Block-edge averaging (Sync of Sec. III-B): CSR rows on data cells of the
// box; every data cell may be overwritten by at most one Sync row.
bc_status add_sync(bc_plan* P, const bc_submatrix& m, int idx, Coverage& dcov) {
  Sub s;
  bc_status st = read_sub(P, m, idx, s);
  if (st != BC_OK) return st;
  const bc_block& B = P->blocks[s.block];
  if (!m.row_ptr || !m.col_block || !m.col_comp || !m.col_ijk || !m.val)
    return fail(BC_ERR_INVALID_ARG, "sub-matrix %d: Sync arrays missing", idx);
  const int64_t nrows = (int64_t)s.comps.size() * s.vol;
  if (m.row_ptr[0] != 0) return fail(BC_ERR_INVALID_ARG, "sub-matrix %d: row_ptr[0] != 0", idx);
  for (int64_t r = 0; r < nrows; ++r)
    if (m.row_ptr[r + 1] < m.row_ptr[r])
      return fail(BC_ERR_INVALID_ARG, "sub-matrix %d: row_ptr not monotone", idx);
  if (m.row_ptr[nrows] + (int64_t)P->sync.ent.size() > INT32_MAX)
    return fail(BC_ERR_UNSUPPORTED, "sub-matrix %d: too many Sync entries", idx);
  for (size_t c = 0; c < s.comps.size(); ++c) {
    const int slot = P->slot_base[s.block] + s.comps[c];
    bc_status err = BC_OK;
    for_box(s, [&](int q, int i, int j, int k) {
      if (err != BC_OK) return;
      if (!in_data(B, i, j, k)) {
        err = fail(BC_ERR_OUT_OF_RANGE, "sub-matrix %d: Sync box contains ghost cells", idx);
        return;
      }
      if (!dcov.mark(slot, i, j, k)) {
        err = fail(BC_ERR_OVERLAP, "sub-matrix %d: Sync rows overlap an earlier Sync box", idx);
        return;
      }
      const int64_t r = (int64_t)c * s.vol + q;
      if (m.rhs && m.rhs[r] != 0.0) {
        err = fail(BC_ERR_INVALID_ARG, "sub-matrix %d: Sync rows have b = 0", idx);
        return;
      }
      for (int64_t e = m.row_ptr[r]; e < m.row_ptr[r + 1]; ++e) {
        const int cb = m.col_block[e], cc = m.col_comp[e];
        const int ci = m.col_ijk[3 * e], cj = m.col_ijk[3 * e + 1], ck = m.col_ijk[3 * e + 2];
        if (cb < 0 || cb >= (int)P->blocks.size() || cc < 0 || cc >= P->blocks[cb].ncomp) {
          err = fail(BC_ERR_INVALID_ARG, "sub-matrix %d: bad column block/component", idx);
          return;
        }
        const bc_block& C = P->blocks[cb];
        if (!in_data(C, ci, cj, ck)) {
          err = fail(BC_ERR_COLUMN_NOT_DATA, "sub-matrix %d: column (%d,%d,%d) of block %d is not data",
                     idx, ci, cj, ck, cb);
          return;
        }
        if (C.nlevels != B.nlevels) {
          err = fail(BC_ERR_INVALID_ARG, "sub-matrix %d: column block has another level count", idx);
          return;
        }
        if (!std::isfinite(m.val[e])) {
          err = fail(BC_ERR_INVALID_ARG, "sub-matrix %d: non-finite value", idx);
          return;
        }
        P->sync.ent.push_back(make_int2(P->slot_base[cb] + cc, (int)cell_offset(C, ci, cj, ck)));
        P->sync.w.push_back(m.val[e]);
      }
      P->sync.row.push_back(make_int4(slot, (int)cell_offset(B, i, j, k), (int)P->sync.stage,
                                      B.nlevels));
      P->sync.ptr.push_back((int32_t)P->sync.ent.size());
      P->sync.stage += B.nlevels;
    });
    if (err != BC_OK) return err;
  }
  if (P->sync.stage > INT32_MAX) return fail(BC_ERR_UNSUPPORTED, "too many Sync values");
  return BC_OK;
}

// Columns read by Sync rows and their entries {staging offset, weight}, in
// ascending (row) order per column: the adjoint's gather table.
void build_sync_transpose(bc_plan* P) {
  auto& S = P->sync;
  struct E {
    int32_t slot, off, stage;
    double w;
    int L;
  };
  std::vector<E> ents;
  for (size_t r = 0; r < S.row.size(); ++r)
    for (int32_t e = S.ptr[r]; e < S.ptr[r + 1]; ++e)
      ents.push_back({S.ent[e].x, S.ent[e].y, S.row[r].z, S.w[e], S.row[r].w});
  std::stable_sort(ents.begin(), ents.end(), [](const E& a, const E& b) {
    return a.slot != b.slot ? a.slot < b.slot : a.off < b.off;
  });
  S.col.clear();
  S.cptr.assign(1, 0);
  S.cstage.clear();
  S.cw.clear();
  for (size_t e = 0; e < ents.size(); ++e) {
    if (e == 0 || ents[e].slot != ents[e - 1].slot || ents[e].off != ents[e - 1].off) {
      if (e) S.cptr.push_back((int32_t)S.cstage.size());
      S.col.push_back(make_int4(ents[e].slot, ents[e].off, ents[e].L, 0));
    }
    S.cstage.push_back(ents[e].stage);
    S.cw.push_back(ents[e].w);
  }
  if (!ents.empty()) S.cptr.push_back((int32_t)S.cstage.size());
}

bc_status read_interp(bc_plan* P, const bc_submatrix& m, int idx, Sub& s) {
  if (m.p < 1 || m.p > kPMax)
    return fail(BC_ERR_UNSUPPORTED, "sub-matrix %d: p must be in 1..%d", idx, kPMax);
  s.p = m.p;
  s.geometry = m.geometry;
  s.rot_u = m.rot_comp[0];
  s.rot_v = m.rot_comp[1];
  const bool rot = s.rot_u >= 0 || s.rot_v >= 0;
  if (rot) {
    auto has = [&](int c) { return std::find(s.comps.begin(), s.comps.end(), c) != s.comps.end(); };
    if (s.rot_u < 0 || s.rot_v < 0 || s.rot_u == s.rot_v || !has(s.rot_u) || !has(s.rot_v))
      return fail(BC_ERR_INVALID_ARG, "sub-matrix %d: rot_comp must name two listed components", idx);
  }
  s.table = (int)P->itp_idx.size();
  P->itp_idx.resize(P->itp_idx.size() + s.vol);
  P->itp_w.resize(P->itp_w.size() + (size_t)s.vol * kPMax, 0.0);
  P->itp_m.resize(P->itp_m.size() + (size_t)s.vol * 4, 0.0);
  if (m.geometry == BC_GEOM_USER) {
    if (!m.itp_src_block || !m.itp_start || !m.itp_axis || !m.itp_w || (rot && !m.itp_rot))
      return fail(BC_ERR_INVALID_ARG, "sub-matrix %d: interpolation tables missing", idx);
    const bc_block& B = P->blocks[s.block];
    for (int q = 0; q < s.vol; ++q) {
      const int sb = m.itp_src_block[q], ax = m.itp_axis[q];
      if (sb < 0 || sb >= (int)P->blocks.size() || ax < 0 || ax > 2)
        return fail(BC_ERR_INVALID_ARG, "sub-matrix %d: bad source block/axis", idx);
      const bc_block& S = P->blocks[sb];
      if (S.nlevels != B.nlevels)
        return fail(BC_ERR_INVALID_ARG, "sub-matrix %d: source has another level count", idx);
      for (int c : s.comps)
        if (c >= S.ncomp) return fail(BC_ERR_INVALID_ARG, "sub-matrix %d: source lacks a component", idx);
      int st[3] = {m.itp_start[3 * q], m.itp_start[3 * q + 1], m.itp_start[3 * q + 2]};
      int en[3] = {st[0], st[1], st[2]};
      en[ax] += m.p - 1;
      if (!in_data(S, st[0], st[1], st[2]) || !in_data(S, en[0], en[1], en[2]))
        return fail(BC_ERR_COLUMN_NOT_DATA, "sub-matrix %d: stencil leaves the source data", idx);
      const int64_t off = cell_offset(S, st[0], st[1], st[2]);
      P->itp_idx[s.table + q] = make_int4(P->slot_base[sb], (int)off, (int)S.stride[ax], 0);
      for (int k = 0; k < m.p; ++k) {
        const double w = m.itp_w[(size_t)q * m.p + k];
        if (!std::isfinite(w)) return fail(BC_ERR_INVALID_ARG, "sub-matrix %d: non-finite weight", idx);
        P->itp_w[(size_t)(s.table + q) * kPMax + k] = w;
      }
      double* M = &P->itp_m[(size_t)(s.table + q) * 4];
      if (rot) {
        for (int e = 0; e < 4; ++e) {
          M[e] = m.itp_rot[(size_t)q * 4 + e];
          if (!std::isfinite(M[e])) return fail(BC_ERR_INVALID_ARG, "sub-matrix %d: non-finite rotation", idx);
        }
      } else {
        M[0] = M[3] = 1.0;
      }
    }
  } else if (m.geometry == BC_GEOM_CUBED_SPHERE) {
    int panel = -1;
    for (int t = 0; t < 6; ++t) {
      const int pb = m.cs_panels[t];
      if (pb < 0 || pb >= (int)P->blocks.size())
        return fail(BC_ERR_INVALID_ARG, "sub-matrix %d: bad panel block", idx);
      if (pb == s.block) panel = t;
      const bc_block& A = P->blocks[pb];
      const bc_block& B0 = P->blocks[m.cs_panels[0]];
      if (A.n[0] != A.n[1] || A.n[0] != B0.n[0] || A.n[2] != 1 || A.h[0] != A.h[1] ||
          A.h[0] != B0.h[0] || A.nlevels != B0.nlevels || A.ncomp != B0.ncomp ||
          A.stride[0] != B0.stride[0] || A.stride[1] != B0.stride[1])
        return fail(BC_ERR_INVALID_ARG, "sub-matrix %d: panels must be equal N x N 2-D blocks", idx);
    }
    if (panel < 0) return fail(BC_ERR_INVALID_ARG, "sub-matrix %d: block is not a panel", idx);
    if (m.p > P->blocks[s.block].n[0])
      return fail(BC_ERR_INVALID_ARG, "sub-matrix %d: stencil wider than the panel", idx);
  } else {
    return fail(BC_ERR_INVALID_ARG, "sub-matrix %d: unknown geometry", idx);
  }
  return BC_OK;
}

void append_interp_rows(bc_plan* P, const Sub& s) {
  const bc_block& B = P->blocks[s.block];
  for (int c : s.comps) {
    if (c == s.rot_v) continue;  // the pair is emitted with its u component
    const bool pair = (c == s.rot_u);
    for (int comp_row = 0; comp_row < (pair ? 2 : 1); ++comp_row) {
      const int crow = pair ? (comp_row == 0 ? s.rot_u : s.rot_v) : c;
      const int slot = P->slot_base[s.block] + crow;
      for_box(s, [&](int q, int i, int j, int k) {
        const int4 ix = P->itp_idx[s.table + q];
        const double* w = &P->itp_w[(size_t)(s.table + q) * kPMax];
        const double* M = &P->itp_m[(size_t)(s.table + q) * 4];
        const int pe = (ix.w & kFlagSnap) ? 1 : s.p;
        P->rows.begin_row(slot, cell_offset(B, i, j, k), 0.0);
        if (!pair) {
          for (int n = 0; n < pe; ++n)
            P->rows.entry(ix.x + c, (int64_t)ix.y + (int64_t)n * ix.z, w[n]);
        } else {
          const double ma = M[comp_row * 2 + 0], mb = M[comp_row * 2 + 1];
          for (int n = 0; n < pe; ++n)
            P->rows.entry(ix.x + s.rot_u, (int64_t)ix.y + (int64_t)n * ix.z, ma * w[n]);
          for (int n = 0; n < pe; ++n)
            P->rows.entry(ix.x + s.rot_v, (int64_t)ix.y + (int64_t)n * ix.z, mb * w[n]);
        }
        P->rows.end_row();
      });
    }
  }
}

bc_status run_cubed_sphere(bc_plan* P, const std::vector<const bc_submatrix*>& cs_subs,
                           const std::vector<int>& cs_idx) {
  if (cs_subs.empty()) return BC_OK;
  // all cubed-sphere sub-matrices of one plan must share the panel set
  const bc_submatrix& m0 = *cs_subs[0];
  CsPanels pan{};
  const bc_block& B0 = P->blocks[m0.cs_panels[0]];
  pan.N = B0.n[0];
  pan.h = B0.h[0];
  pan.p = m0.p;
  pan.rotate = 0;
  for (int t = 0; t < 6; ++t) {
    const bc_block& A = P->blocks[m0.cs_panels[t]];
    pan.slot_base[t] = P->slot_base[m0.cs_panels[t]];
    pan.s0[t] = A.stride[0];
    pan.s1[t] = A.stride[1];
  }
  std::vector<int4> cells;
  for (size_t u = 0; u < cs_subs.size(); ++u) {
    const bc_submatrix& m = *cs_subs[u];
    for (int t = 0; t < 6; ++t)
      if (m.cs_panels[t] != m0.cs_panels[t])
        return fail(BC_ERR_UNSUPPORTED, "cubed-sphere sub-matrices must share one panel set");
    if (m.p != m0.p) return fail(BC_ERR_UNSUPPORTED, "cubed-sphere sub-matrices must share p");
    const Sub& s = P->subs[cs_idx[u]];
    if (s.rot_u >= 0) pan.rotate = 1;
    int panel = 0;
    for (int t = 0; t < 6; ++t)
      if (m.cs_panels[t] == s.block) panel = t;
    for_box(s, [&](int q, int i, int j, int) { cells.push_back(make_int4(panel, i, j, s.table + q)); });
  }
  const size_t nrow = P->itp_idx.size();
  int4 *d_cells = nullptr, *d_idx = nullptr;
  double *d_w = nullptr, *d_m = nullptr;
  unsigned* d_err = nullptr;
  auto cleanup = [&]() {
    cudaFree(d_cells);
    cudaFree(d_idx);
    cudaFree(d_w);
    cudaFree(d_m);
    cudaFree(d_err);
  };
  cudaError_t e;
  if ((e = dev_malloc(reinterpret_cast<void**>(&d_cells), cells.size() * sizeof(int4))) != cudaSuccess ||
      (e = dev_malloc(reinterpret_cast<void**>(&d_idx), nrow * sizeof(int4))) != cudaSuccess ||
      (e = dev_malloc(reinterpret_cast<void**>(&d_w), nrow * kPMax * sizeof(double))) != cudaSuccess ||
      (e = dev_malloc(reinterpret_cast<void**>(&d_m), nrow * 4 * sizeof(double))) != cudaSuccess ||
      (e = dev_malloc(reinterpret_cast<void**>(&d_err), sizeof(unsigned))) != cudaSuccess) {
    cleanup();
    return cuda_fail(e, "cubed-sphere geometry allocation");
  }
  unsigned herr = 0;
  if ((e = cudaMemcpy(d_cells, cells.data(), cells.size() * sizeof(int4), cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemcpy(d_idx, P->itp_idx.data(), nrow * sizeof(int4), cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemcpy(d_w, P->itp_w.data(), nrow * kPMax * sizeof(double), cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemcpy(d_m, P->itp_m.data(), nrow * 4 * sizeof(double), cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemset(d_err, 0, sizeof(unsigned))) != cudaSuccess ||
      (e = launch_cs_geometry(pan, d_cells, (int)cells.size(), d_idx, d_w, d_m, d_err, 0)) != cudaSuccess ||
      (e = cudaMemcpy(P->itp_idx.data(), d_idx, nrow * sizeof(int4), cudaMemcpyDeviceToHost)) != cudaSuccess ||
      (e = cudaMemcpy(P->itp_w.data(), d_w, nrow * kPMax * sizeof(double), cudaMemcpyDeviceToHost)) != cudaSuccess ||
      (e = cudaMemcpy(P->itp_m.data(), d_m, nrow * 4 * sizeof(double), cudaMemcpyDeviceToHost)) != cudaSuccess ||
      (e = cudaMemcpy(&herr, d_err, sizeof(unsigned), cudaMemcpyDeviceToHost)) != cudaSuccess) {
    cleanup();
    return cuda_fail(e, "cubed-sphere geometry kernel");
  }
  cleanup();
  if (herr & CS_ERR_NOT_EDGE)
    return fail(BC_ERR_GEOMETRY, "cubed sphere: a box cell is not an edge ghost");
  if (herr & CS_ERR_NEIGHBOUR)
    return fail(BC_ERR_GEOMETRY, "cubed sphere: neighbour panel check failed");
  if (herr & CS_ERR_DEPTH)
    return fail(BC_ERR_GEOMETRY, "cubed sphere: ghost point is off the neighbour rows");
  if (herr & CS_ERR_RANGE)
    return fail(BC_ERR_GEOMETRY, "cubed sphere: stencil outside the neighbour data");
  return BC_OK;
}

// -- work lists ----------------------------------------------------------------
int family_of_kind(int kind) {
  return kind == BC_INTERP ? FAM_INTERP : (kind == BC_CSR ? FAM_CSR : FAM_STRUCT);
}

FastDiv make_div(uint32_t d) {
  FastDiv f;
  f.d = d;
  f.s = 0;
  while ((uint64_t(1) << f.s) < d) ++f.s;
  f.m = (uint32_t)((((uint64_t(1) << 32) * ((uint64_t(1) << f.s) - d)) / d) + 1);
  return f;
}

void item_common(const bc_plan* P, const Sub& s, int comp, Item& it) {
  const bc_block& B = P->blocks[s.block];
  it.dst_slot = P->slot_base[s.block] + comp;
  it.dst_slot2 = -1;
  it.src_slot = -1;
  it.vol = make_div((uint32_t)s.vol);
  it.lev = make_div((uint32_t)B.nlevels);
  it.ctab = s.ctab;
  it.dst_ls = (int32_t)(B.nlevels > 1 ? B.level_stride : 0);
}

// Unit order of a block's items: level-fastest flat values when the levels
// are contiguous; otherwise cell-major chunks of up to 8 levels, or flat
// cell-fastest values when there are too few levels for a chunk.
// `order`: 0 auto, 1 cells fastest, 2 levels fastest (bc_plan_opts).
bool levels_fastest(const bc_block& B, int order) {
  if (B.nlevels <= 1 || order == 1) return false;
  return order == 2 || B.level_stride == 1;
}

int structured_mode(const bc_block& B, int order) {
  return levels_fastest(B, order) ? MODE_FLAT_LEVEL : MODE_FLAT_CELL;
}

int table_mode(const bc_block& B, int order, int chunk) {
  if (levels_fastest(B, order)) return MODE_FLAT_LEVEL;
  if (B.nlevels == 1 || chunk <= 1) return MODE_FLAT_CELL;
  return std::min(B.nlevels, chunk);
}

// levels per unit of the chunked unit order (bc_plan_opts.level_chunk; by
// default 4 for interpolation rows, whose pair path keeps two components'
// sums, and 8 for CSR and transpose rows); the persistent launch's kernel
// holds at most 4
int level_chunk(const bc_plan* P, bool interp) {
  int ch = P->opts.level_chunk;
  if (ch == 0) ch = interp ? 4 : 8;
  const bool all_kinds =
      P->opts.batch_mode == BC_BATCH_PERSISTENT || P->opts.batch_mode == BC_BATCH_SINGLE;
  return all_kinds ? std::min(ch, 4) : ch;
}

// split the unit space into warp-sized items: vol * L single values (flat
// modes) or vol * ceil(L / mode) chunks
void emit_units(std::vector<Item>& out, Item proto, int vol, int L, int mode, int per_item) {
  proto.mode = mode;
  const int64_t total = mode < 2 ? (int64_t)vol * L : (int64_t)vol * ((L + mode - 1) / mode);
  for (int64_t u0 = 0; u0 < total; u0 += per_item) {
    Item it = proto;
    it.u0 = (int)u0;
    it.nunits = (int)std::min<int64_t>(per_item, total - u0);
    out.push_back(it);
  }
}

#ifndef BC_RUN_ITEM
#define BC_RUN_ITEM 256  // values of a run item per unit of units_per_lane
#endif
#ifndef BC_FLAT_UPL_MAX
// largest units_per_lane of per-value (flat) items: one 8-value step per
// lane (512-block workload, levels innermost: the structured kernel alone
// 39.0 -> 30.3 us; items of 1024 values of the 2-cell edge strips of
// blocks with few levels ran up to 39 us each, the kernel's tail)
#define BC_FLAT_UPL_MAX 1
#endif
#ifndef BC_RUN_MIN_AVG
#define BC_RUN_MIN_AVG 16  // shortest average run (values) worth a run table
#endif

// Runs of a zero / map sub-matrix: maximal stretches of its ghost values
// that are contiguous in the destination and (maps) in the source, in the
// order the unit order visits them, cut into pieces of at most `cap` values.
// Returns false (use per-value units) when the runs would be short.
bool build_runs(bc_plan* P, const Sub& s, bool lev_fast, int cap, int& r0, int& nr) {
  const bc_block& B = P->blocks[s.block];
  const bool map = s.kind == BC_MAP;
  if (s.kind != BC_ZERO && !map) return false;
  const int L = B.nlevels;
  const int64_t dls = L > 1 ? B.level_stride : 0;
  const int64_t sls = map ? (P->blocks[s.src_block].nlevels > 1 ? P->blocks[s.src_block].level_stride : 0) : 0;
  // levels fastest: each cell's levels must be contiguous in the ghost and
  // in the source (a one-level block has nothing to check)
  if (lev_fast && L > 1 && (dls != 1 || (map && sls != 1))) return false;
  struct Run {
    int64_t d, s, n;
  };
  std::vector<Run> merged;
  const int len = lev_fast ? L : 1;
  for (int l = 0; l < (lev_fast ? 1 : L); ++l) {
    for (int q = s.ctab; q < s.ctab + s.vol; ++q) {
      const int64_t d = P->ctab_d[q] + (int64_t)l * dls;
      const int64_t sr = map ? P->ctab_s[q] + (int64_t)l * sls : 0;
      if (d + len > INT32_MAX || sr + len > INT32_MAX) return false;
      if (!merged.empty()) {
        Run& cur = merged.back();
        if (d == cur.d + cur.n && (!map || sr == cur.s + cur.n)) {
          cur.n += len;
          continue;
        }
      }
      merged.push_back({d, sr, len});
    }
  }
  const int64_t total = (int64_t)s.vol * L;
  if (merged.empty() || total < BC_RUN_MIN_AVG * (int64_t)merged.size()) return false;  // short runs
  r0 = (int)P->runs.size();
  for (const Run& m : merged)
    for (int64_t o = 0; o < m.n; o += cap)
      P->runs.push_back(make_int4((int)(m.d + o), (int)(m.s + (map ? o : 0)),
                                  (int)std::min<int64_t>(cap, m.n - o), 0));
  nr = (int)P->runs.size() - r0;
  return true;
}

// Lanes per run for the runs [a, b) of one item: the power of two g that
// needs the fewest U-value steps when 32 / g runs go side by side (ties to
// the larger g, for wider coalesced segments), and at least min(8, longest
// run) so a lane group covers a 32-byte sector where the runs allow it.
int run_lanes(const std::vector<int4>& runs, int a, int b) {
  int longest = 0;
  for (int r = a; r < b; ++r) longest = std::max(longest, runs[r].z);
  int gmin = 1;
  while (gmin < std::min(longest, 8)) gmin <<= 1;
  int best_g = 32;
  int64_t best = INT64_MAX;
  for (int g = 32; g >= gmin; g >>= 1) {
    const int side = 32 / g;
    int64_t steps = 0;
    for (int k = a; k < b; k += side) {
      int m = 0;
      for (int r = k; r < std::min(b, k + side); ++r) m = std::max(m, runs[r].z);
      steps += (m + g * kRunUnroll - 1) / (g * kRunUnroll);
    }
    if (steps < best) {
      best = steps;
      best_g = g;
    }
  }
  return best_g;
}

// split runs [r0, r0 + nr) into warp items of at most 32 runs and about
// `per_item` values
void emit_runs(std::vector<Item>& out, Item proto, const std::vector<int4>& runs, int r0, int nr,
               int per_item) {
  proto.mode = MODE_RUNS;
  int a = r0;
  while (a < r0 + nr) {
    int b = a, sum = 0;
    while (b < r0 + nr && b - a < 32 && (b == a || sum + runs[b].z <= per_item)) sum += runs[b++].z;
    Item it = proto;
    it.u0 = a;
    it.nunits = b - a;
    it.p = run_lanes(runs, a, b);
    out.push_back(it);
    a = b;
  }
}

// Staged interpolation items of sub-matrix s (levels in chunks of `chunk`):
// tiles of up to kTileCells consecutive box cells whose nodes all lie in one
// 2-D source block, with the node box of each tile small enough that `chunk`
// levels of its components (nc) fit a warp's staging area at least one
// level at a time.  Writes the cells' itp_box rows.  Returns false (the
// sub-matrix keeps the per-lane path) when some tile does not qualify.
bool emit_tiles(bc_plan* P, const Sub& s, const Item& proto, int chunk, int nc,
                std::vector<Item>& out) {
  const bc_block& B = P->blocks[s.block];
  const int L = B.nlevels;
  const int cap = kStageBytesRows / P->esize;
  std::vector<Item> tiles;
  std::vector<std::pair<int, int32_t>> boxes;  // (row, itp_box) to write on success
  for (int q0 = 0; q0 < s.vol; q0 += kTileCells) {
    const int nq = std::min(kTileCells, s.vol - q0);
    int base = -1;
    int imin = INT_MAX, imax = INT_MIN, jmin = INT_MAX, jmax = INT_MIN;
    struct Node0 {
      int i, j, rows, snap;
    };
    std::vector<Node0> n0(nq);
    for (int q = 0; q < nq; ++q) {
      const int4 ix = P->itp_idx[(size_t)(s.table + q0 + q)];
      if (base < 0) base = ix.x;
      if (ix.x != base) return false;
      const bc_block& S = P->blocks[P->slot_block[ix.x]];
      if (S.n[2] != 1 || S.h[2] != 0) return false;
      int i, j, k;
      if (!decode_cell(S, ix.y, i, j, k)) return false;
      const bool snap = ix.w & kFlagSnap;
      const int np = snap ? 1 : s.p;
      int ax;
      if (np == 1 || ix.z == S.stride[0]) ax = 0;
      else if (ix.z == S.stride[1]) ax = 1;
      else return false;
      const int i1 = ax == 0 ? i + np - 1 : i, j1 = ax == 1 ? j + np - 1 : j;
      imin = std::min(imin, i);
      imax = std::max(imax, i1);
      jmin = std::min(jmin, j);
      jmax = std::max(jmax, j1);
      n0[q] = {i, j, ax, snap ? 1 : 0};
    }
    const int bw = imax - imin + 1, bh = jmax - jmin + 1;
    if ((int64_t)bw * bh > kBoxIndex || (int64_t)bw * bh * nc > cap) return false;
    const int nl = std::min(chunk, cap / (bw * bh * nc));
    const bc_block& S = P->blocks[P->slot_block[base]];
    const int64_t org = cell_offset(S, imin, jmin, 0);
    if (org > INT32_MAX) return false;
    for (int q = 0; q < nq; ++q) {
      const int32_t bx = (n0[q].i - imin) + (n0[q].j - jmin) * bw;
      boxes.push_back({s.table + q0 + q,
                       bx | (n0[q].rows ? kBoxRows : 0) | (n0[q].snap ? kBoxSnap : 0)});
    }
    for (int l0 = 0; l0 < L; l0 += nl) {
      Item it = proto;
      it.mode = MODE_TILE;
      it.u0 = q0;
      it.nunits = nq;
      it.vol = make_div((uint32_t)nq);
      it.l0 = l0;
      it.nl = std::min(nl, L - l0);
      it.bw = bw;
      it.bh = bh;
      it.bs0 = (int32_t)S.stride[0];
      it.bs1 = (int32_t)S.stride[1];
      it.bsrc = base;
      it.bwid = make_div((uint32_t)bw);
      it.borg = (int32_t)org;
      it.bsrc2 = -1;
      it.src_ls = (int32_t)(S.nlevels > 1 ? S.level_stride : 0);
      tiles.push_back(it);
    }
  }
  for (const auto& b : boxes) P->itp_box[(size_t)b.first] = b.second;
  out.insert(out.end(), tiles.begin(), tiles.end());
  return true;
}

// A staged tile's box, the slots it reads and each entry's place in it.
struct TileBox {
  int blk = -1, nsel = 0, sl[2] = {-1, -1};
  int imin = INT_MAX, imax = INT_MIN, jmin = INT_MAX, jmax = INT_MIN;
  struct Ent {
    size_t e;
    int sel, i, j;
  };
  std::vector<Ent> ents;
  // entry e reads (slot, offset); false when it leaves one 2-D block or
  // its two slots
  bool add(const bc_plan* P, size_t e, int slot, int64_t off) {
    const int b = P->slot_block[slot];
    if (blk < 0) blk = b;
    if (b != blk) return false;
    int sel = slot == sl[0] ? 0 : (slot == sl[1] ? 1 : -1);
    if (sel < 0) {
      if (nsel == 2) return false;
      sl[nsel] = slot;
      sel = nsel++;
    }
    const bc_block& S = P->blocks[b];
    if (S.n[2] != 1 || S.h[2] != 0) return false;
    int i, j, k;
    if (!decode_cell(S, off, i, j, k)) return false;
    imin = std::min(imin, i);
    imax = std::max(imax, i);
    jmin = std::min(jmin, j);
    jmax = std::max(jmax, j);
    ents.push_back({e, sel, i, j});
    return true;
  }
};

// Staging pays only when a tile's entries read each staged value at least
// this often on average (a box mostly of values no row reads costs more
// loads than it saves).
constexpr int kMinTileReuse = 1;

// Items of one staged tile of nq rows from q0 (levels in chunks of `chunk`,
// L levels): 1 when the box holds at least `need` levels of its slots in a
// warp's staging area (items and box words appended), 0 when the box is
// too large for that, -1 when the rows cannot (or should not) be staged.
int finish_tile(const bc_plan* P, const TileBox& T, int q0, int nq, const Item& proto, int chunk,
                int L, int need, int stage_bytes, std::vector<Item>& tiles,
                std::vector<std::pair<size_t, int32_t>>& boxes) {
  if (T.blk < 0) return -1;
  const bc_block& S = P->blocks[T.blk];
  if (S.nlevels != L) return -1;
  const int cap = stage_bytes / P->esize;
  const int bw = T.imax - T.imin + 1, bh = T.jmax - T.jmin + 1;
  if ((int64_t)bw * bh > kBoxIndex) return 0;
  if ((int64_t)T.ents.size() < (int64_t)kMinTileReuse * bw * bh * T.nsel) return -1;
  const int64_t fit = cap / ((int64_t)bw * bh * T.nsel);
  if (fit < need) return 0;
  const int nl = (int)std::min<int64_t>(chunk, fit);
  const int64_t org = cell_offset(S, T.imin, T.jmin, 0);
  if (org > INT32_MAX) return -1;
  for (const TileBox::Ent& x : T.ents)
    boxes.push_back({x.e, (x.i - T.imin) + (x.j - T.jmin) * bw + x.sel * bw * bh});
  for (int l0 = 0; l0 < L; l0 += nl) {
    Item it = proto;
    it.mode = MODE_TILE;
    it.u0 = q0;
    it.nunits = nq;
    // lanes take (row, group of kTileLevels levels) units, rows fastest
    it.vol = make_div((uint32_t)nq);
    it.l0 = l0;
    it.nl = std::min(nl, L - l0);
    it.bw = bw;
    it.bh = bh;
    it.bs0 = (int32_t)S.stride[0];
    it.bs1 = (int32_t)S.stride[1];
    it.bsrc = T.sl[0];
    it.bsrc2 = T.sl[1];
    it.bwid = make_div((uint32_t)bw);
    it.borg = (int32_t)org;
    it.src_ls = (int32_t)(S.nlevels > 1 ? S.level_stride : 0);
    it.src_slot = -1;  // no common-slot lookup: the tile reads its slots itself
    tiles.push_back(it);
  }
  return 1;
}

// Levels a staged CSR or transpose tile must hold at once: a full lane
// group (fewer only when the chunk or the block has fewer).
int tile_need(int chunk, int L) { return std::min(kTileLevels, std::min(chunk, L)); }

// Staged CSR rows of component ci of sub-matrix s (levels in chunks of
// `chunk`): tiles of kTileCells rows (16 or 8 when the boxes of 32 rows are
// too large) whose entries all lie in one 2-D block, in at most two of its
// slots, inside a box of which a lane group of levels fits a warp's staging
// area.  Writes the entries' csr_box words.  Returns false (the component
// keeps the per-lane path) when some tile does not qualify.
bool emit_csr_tiles(bc_plan* P, const Sub& s, int ci, const Item& proto, int chunk,
                    std::vector<Item>& out) {
  const int L = P->blocks[s.block].nlevels;
  const int w = s.ell_w;
  const int need = tile_need(chunk, L);
  std::vector<Item> tiles;
  std::vector<std::pair<size_t, int32_t>> boxes;
  for (int rows = kTileCells; rows >= 8; rows /= 2) {
    tiles.clear();
    boxes.clear();
    bool smaller = false;
    for (int q0 = 0; q0 < s.vol && !smaller; q0 += rows) {
      const int nq = std::min(rows, s.vol - q0);
      TileBox T;
      for (int q = 0; q < nq; ++q) {
        const size_t row = (size_t)(s.table + ci * s.vol + q0 + q);
        const size_t e0 = (size_t)s.ell_base + ((size_t)ci * s.vol + q0 + q) * w;
        for (int k = 0; k < P->csr_nnz[row]; ++k)
          if (!T.add(P, e0 + k, P->csr_slot[e0 + k], P->csr_off[e0 + k])) return false;
      }
      const int r = finish_tile(P, T, q0, nq, proto, chunk, L, need, kStageBytesCsr, tiles, boxes);
      if (r < 0) return false;
      smaller = r == 0;
    }
    if (smaller) continue;
    for (const auto& b : boxes) P->csr_box[b.first] = b.second;
    out.insert(out.end(), tiles.begin(), tiles.end());
    return true;
  }
  return false;
}

// Staged transpose rows [r0, r0 + nrows) (one data slot, levels in chunks
// of `chunk`, the chunked unit order): tiles of kTileCells rows (16 or 8
// when some box of 32 rows is too large); a tile that does not qualify
// keeps the per-lane gather (one item of its rows per level chunk).
// Returns false, emitting nothing, when no tile qualifies.
bool emit_adj_tiles(bc_plan* P, int r0, int nrows, const Item& proto, int chunk, int L,
                    std::vector<Item>& out) {
  const int need = tile_need(chunk, L);
  std::vector<Item> items;
  std::vector<std::pair<size_t, int32_t>> boxes;
  int staged = 0;
  for (int rows = kTileCells; rows >= 8; rows /= 2) {
    items.clear();
    boxes.clear();
    staged = 0;
    bool smaller = false;
    for (int q0 = 0; q0 < nrows && !smaller; q0 += rows) {
      const int nq = std::min(rows, nrows - q0);
      TileBox T;
      bool ok = true;
      for (int q = 0; q < nq && ok; ++q) {
        const size_t r = (size_t)(r0 + q0 + q);
        for (int64_t e = P->adj_ptr[r]; e < P->adj_ptr[r + 1] && ok; ++e)
          ok = T.add(P, (size_t)e, P->aent_slot[(size_t)e], P->aent_off[(size_t)e]);
      }
      const int res =
          ok ? finish_tile(P, T, q0, nq, proto, chunk, L, need, kStageBytesRows, items, boxes) : -1;
      if (res > 0) {
        ++staged;
        continue;
      }
      if (res == 0 && rows > 8) {
        smaller = true;
        continue;
      }
      for (int c = 0; c * chunk < L; ++c) {
        Item it = proto;
        it.mode = chunk;
        it.u0 = q0 + c * nrows;
        it.nunits = nq;
        items.push_back(it);
      }
    }
    if (!smaller) break;
  }
  if (!staged) return false;
  for (const auto& b : boxes) P->adj_box[b.first] = b.second;
  out.insert(out.end(), items.begin(), items.end());
  return true;
}

void build_items(bc_plan* P) {
  P->runs.clear();
  P->adj_box.assign(P->aent_off.size(), 0);
  P->itp_box.assign(P->itp_idx.size(), 0);
  P->csr_box.assign(P->csr_off.size(), 0);
  // units per warp item: single-level values (flat) or 8-level chunks
  const int upl = std::max(1, std::min(P->opts.units_per_lane, 64));
  // A small plan still gets enough items to keep every SM busy: the value
  // budget of an item shrinks (down to one value per lane) until the plan's
  // values make about 16 items per SM (128^3 HPCG-like faces: 98 items of
  // 1024 values took 26.7 us; 1560 items of 64 values take far less).
  int64_t total_values = 0;
  for (const Sub& s : P->subs)
    total_values += (int64_t)s.comps.size() * s.vol * P->blocks[s.block].nlevels;
  const int64_t want_items = (int64_t)std::max(1, P->num_sms) * 16;
  const int small = (int)std::min<int64_t>(
      1 << 30, std::max<int64_t>(32, (total_values + want_items - 1) / want_items + 31) / 32 * 32);
  const int per_chunk_item = 32 * upl;
  const int per_flat_item = std::min(32 * kFlatUnroll * std::min(upl, BC_FLAT_UPL_MAX), small);
  // table-driven kinds (interpolation, CSR, transpose): one unit per lane, so
  // a warp's dependent table -> data chains run side by side, not in series
  const int per_table_item = 32;
  const int per_table_flat_item = std::min(32 * 8, small);
  auto structured_emit = [&](std::vector<Item>& out, const Item& it, const bc_block& B, int vol) {
    const int mode = structured_mode(B, P->opts.unit_order);
    emit_units(out, it, vol, B.nlevels, mode, mode < 2 ? per_flat_item : per_chunk_item);
  };
  // zero / map sub-matrices: runs when they are long, cached per sub-matrix
  const int per_run_item = std::min(BC_RUN_ITEM * upl, small);
  std::vector<int> run_r0(P->subs.size(), -1), run_n(P->subs.size(), 0);
  for (size_t si = 0; si < P->subs.size(); ++si) {
    const Sub& s = P->subs[si];
    const bc_block& B = P->blocks[s.block];
    int r0 = 0, nr = 0;
    if (!P->opts.no_runs &&
        build_runs(P, s, structured_mode(B, P->opts.unit_order) == MODE_FLAT_LEVEL,
                   per_run_item, r0, nr)) {
      run_r0[si] = r0;
      run_n[si] = nr;
    }
  }
  auto table_emit = [&](std::vector<Item>& out, const Item& it, const bc_block& B, int vol) {
    const bool interp = it.kind == IK_INTERP || it.kind == IK_INTERP_PAIR;
    const int mode = table_mode(B, P->opts.unit_order, level_chunk(P, interp));
    emit_units(out, it, vol, B.nlevels, mode, mode < 2 ? per_table_flat_item : per_table_item);
  };
  std::vector<std::pair<int, std::vector<Item>>> per_sub(P->subs.size());
  for (size_t si = 0; si < P->subs.size(); ++si) {
    const Sub& s = P->subs[si];
    const bc_block& B = P->blocks[s.block];
    std::vector<Item>& out = per_sub[si].second;
    per_sub[si].first = s.kind;
    for (size_t ci = 0; ci < s.comps.size(); ++ci) {
      const int c = s.comps[ci];
      Item it{};
      item_common(P, s, c, it);
      switch (s.kind) {
        case BC_ZERO:
        case BC_CONST:
        case BC_MAP: {
          it.kind = s.kind == BC_ZERO ? IK_ZERO : (s.kind == BC_CONST ? IK_CONST : IK_MAP);
          it.table = s.table + (int)ci * s.vol;
          if (s.kind == BC_MAP) {
            const bc_block& S = P->blocks[s.src_block];
            it.src_slot = P->slot_base[s.src_block] + c;
            it.src_ls = (int32_t)(S.nlevels > 1 ? S.level_stride : 0);
          }
          if (run_r0[si] >= 0)
            emit_runs(out, it, P->runs, run_r0[si], run_n[si], per_run_item);
          else
            structured_emit(out, it, B, s.vol);
          break;
        }
        case BC_INTERP: {
          if (c == s.rot_v) break;
          it.table = s.table;
          it.p = s.p;
          it.comp = c;
          if (c == s.rot_u) {
            it.kind = IK_INTERP_PAIR;
            it.comp = c | (s.rot_v << 16);
            it.dst_slot2 = P->slot_base[s.block] + s.rot_v;
          } else {
            it.kind = IK_INTERP;
          }
          // levels far apart in memory: stage the nodes of each tile in
          // shared memory when the tiles' boxes are small
          const int mode = table_mode(B, P->opts.unit_order, level_chunk(P, true));
          if (mode < 2 || P->opts.unstaged_rows ||
              !emit_tiles(P, s, it, mode, it.kind == IK_INTERP_PAIR ? 2 : 1, out))
            table_emit(out, it, B, s.vol);
          break;
        }
        case BC_CSR: {
          it.kind = IK_CSR;
          it.table = s.table + (int)ci * s.vol;
          it.p = s.ell_w;
          it.src_org = s.ell_base + (int)ci * s.vol * s.ell_w;
          it.src_slot = s.csr_common[ci];
          if (it.src_slot >= 0) {
            const bc_block& S = P->blocks[P->slot_block[it.src_slot]];
            it.src_ls = (int32_t)(S.nlevels > 1 ? S.level_stride : 0);
          }
          // levels far apart in memory: stage each tile's column box
          const int mode = table_mode(B, P->opts.unit_order, level_chunk(P, false));
          if (mode < 2 || P->opts.unstaged_rows ||
              !emit_csr_tiles(P, s, (int)ci, it, mode, out))
            table_emit(out, it, B, s.vol);
          break;
        }
      }
    }
  }
  // order: by kind, then sub-matrix (per-sub and per-kind ranges contiguous)
  P->items.clear();
  P->sub_begin.assign(P->subs.size(), 0);
  P->sub_end.assign(P->subs.size(), 0);
  for (int kind = 0; kind < 5; ++kind) {
    P->type_begin[kind] = (int)P->items.size();
    for (size_t si = 0; si < P->subs.size(); ++si) {
      if (per_sub[si].first != kind) continue;
      P->sub_begin[si] = (int)P->items.size();
      P->items.insert(P->items.end(), per_sub[si].second.begin(), per_sub[si].second.end());
      P->sub_end[si] = (int)P->items.size();
    }
    P->type_end[kind] = (int)P->items.size();
  }
  // batched launch: per family, longest items first
  for (auto& v : P->fam_items) v.clear();
  for (size_t si = 0; si < P->subs.size(); ++si) {
    const int f = family_of_kind(P->subs[si].kind);
    P->fam_items[f].insert(P->fam_items[f].end(), per_sub[si].second.begin(),
                           per_sub[si].second.end());
  }
  // longest items first, so the last wave of warps holds the short ones
  // (512-block workload, levels innermost: batched step 49.2 -> 48.1 us);
  // "longest" by the bytes an item moves (a map value twice a zero value):
  // 45.3 -> 44.9 us, the structured kernel alone 35.1 -> 33.2 us at 2 units
  // per lane
  auto work = [&](const Item& it) -> int64_t {
    if (it.mode == MODE_TILE) return (int64_t)it.nunits * it.nl;
    if (it.mode != MODE_RUNS) return it.nunits;
    int64_t n = 0;
    for (int r = it.u0; r < it.u0 + it.nunits; ++r) n += P->runs[r].z;
    return n;
  };
#ifndef BC_ITEM_COST
#define BC_ITEM_COST 1  // order of the family lists: 0 by values, 1 by bytes moved
#endif
  auto cost = [&](const Item& it) -> int64_t {
    const int64_t v = work(it);
    if (!BC_ITEM_COST) return v;
    return it.kind == IK_MAP ? 2 * v : (it.kind == IK_CSR ? v * (1 + it.p) : v);
  };
  for (auto& v : P->fam_items) {
    std::vector<std::pair<int64_t, size_t>> key(v.size());
    for (size_t t = 0; t < v.size(); ++t) key[t] = {-cost(v[t]), t};
    std::stable_sort(key.begin(), key.end());
    std::vector<Item> sorted(v.size());
    for (size_t t = 0; t < v.size(); ++t) sorted[t] = v[key[t].second];
    v.swap(sorted);
  }
  // persistent launch: every forward item, the most bytes first (values
  // times the bytes a value moves: one store, plus the loads of its row)
  {
    auto bytes = [&](const Item& it) -> int64_t {
      int64_t vals = work(it);
      if (it.mode >= 2) vals *= it.mode;
      switch (it.kind) {
        case IK_ZERO:
        case IK_CONST: return vals;
        case IK_MAP: return 2 * vals;
        case IK_INTERP: return vals * (2 + it.p / 2);
        case IK_INTERP_PAIR: return vals * 2 * (2 + it.p / 2);
        default: return vals * (1 + it.p);
      }
    };
    std::vector<Item> all;
    for (const auto& v : P->fam_items) all.insert(all.end(), v.begin(), v.end());
    std::vector<std::pair<int64_t, size_t>> key(all.size());
    for (size_t t = 0; t < all.size(); ++t) key[t] = {-bytes(all[t]), t};
    std::stable_sort(key.begin(), key.end());
    P->all_items.resize(all.size());
    for (size_t t = 0; t < all.size(); ++t) P->all_items[t] = all[key[t].second];
  }
  // adjoint: the zero pass over every covered ghost value
  P->adj_zero.clear();
  for (size_t si = 0; si < P->subs.size(); ++si) {
    const Sub& s = P->subs[si];
    // zero runs over the box: the same destination runs as a zero item
    int r0 = 0, nr = 0;
    Sub zs = s;
    zs.kind = BC_ZERO;
    const bool use_runs =
        !P->opts.no_runs &&
        build_runs(P, zs, structured_mode(P->blocks[s.block], P->opts.unit_order) == MODE_FLAT_LEVEL,
                   per_run_item, r0, nr);
    for (int c : s.comps) {
      Item z{};
      item_common(P, s, c, z);
      z.kind = IK_ZERO;
      if (use_runs)
        emit_runs(P->adj_zero, z, P->runs, r0, nr, per_run_item);
      else
        structured_emit(P->adj_zero, z, P->blocks[s.block], s.vol);
    }
  }
  // adjoint of unit copies: add-run items, launched with the gather items
  P->adj_add.clear();
  for (const auto& g : P->add_segs) {
    Item it{};
    it.kind = IK_ADD;
    it.dst_slot = g.dslot;
    it.dst_slot2 = -1;
    it.src_slot = g.sslot;
    const int base = (int)P->runs.size();
    P->runs.insert(P->runs.end(), P->add_runs.begin() + g.r0, P->add_runs.begin() + g.r0 + g.nr);
    emit_runs(P->adj_add, it, P->runs, base, g.nr, per_run_item);
  }
  // adjoint gather items over the other transpose rows, one data slot per
  // item (resolved once per item); when every entry of an item's rows reads
  // one ghost slot, that slot is resolved once too
  P->adj_items.clear();
  const int nar = (int)P->arow_slot.size();
  int r0 = 0;
  while (r0 < nar) {
    const int ds = P->arow_slot[r0];
    const bc_block& B0 = P->blocks[P->slot_block[ds]];
    int r1 = r0;
    while (r1 < nar && P->arow_slot[r1] == ds) ++r1;
    int common = -2;
    for (int64_t e = P->adj_ptr[r0]; e < P->adj_ptr[r1] && common != -1; ++e)
      common = common == -2 ? P->aent_slot[e] : (common == P->aent_slot[e] ? common : -1);
    Item it{};
    it.kind = IK_ADJ;
    it.vol = make_div((uint32_t)(r1 - r0));
    it.lev = make_div((uint32_t)B0.nlevels);
    it.table = r0;
    it.dst_slot = ds;
    it.dst_slot2 = -1;
    it.dst_ls = (int32_t)(B0.nlevels > 1 ? B0.level_stride : 0);
    it.src_slot = common >= 0 ? common : -1;
    if (common >= 0) {
      const bc_block& G = P->blocks[P->slot_block[common]];
      it.src_ls = (int32_t)(G.nlevels > 1 ? G.level_stride : 0);
    }
    // levels far apart in memory: stage each tile's box of ghost cotangents
    const int mode = table_mode(B0, P->opts.unit_order, level_chunk(P, false));
    if (mode < 2 || P->opts.unstaged_rows ||
        !emit_adj_tiles(P, r0, r1 - r0, it, mode, B0.nlevels, P->adj_items))
      table_emit(P->adj_items, it, B0, r1 - r0);
    r0 = r1;
  }
  P->adj_items.insert(P->adj_items.begin(), P->adj_add.begin(), P->adj_add.end());
  // the shared-memory stage each launch requests per warp
  auto stage_of = [](const std::vector<Item>& v) {
    int b = 0;
    for (const Item& it : v)
      if (it.mode == MODE_TILE) b = std::max(b, it.kind == IK_CSR ? kStageBytesCsr : kStageBytesRows);
    return b;
  };
  for (int f = 0; f < kFamilies; ++f) P->staged[f] = stage_of(P->fam_items[f]);
  P->staged[FAM_ADJ] = std::max(P->staged[FAM_ADJ], stage_of(P->adj_items));
  P->staged[FAM_ALL] = std::max(stage_of(P->all_items), stage_of(P->items));
}

// The adjoint of a unit copy is an add: a data value read by exactly one
// ghost value, with weight 1, gets x_bar_j = x_bar_j + y_bar_i.  Such
// transpose rows (consecutive in (data slot, offset) order, same ghost slot)
// become add-runs, contiguous in the data and in the ghost values; every
// other row stays in the gather.  A data value has one transpose row, so the
// two sets of targets are disjoint and the result is the gather's, bit for
// bit (x + 1 * y rounds once either way).
void split_unit_copies(bc_plan* P) {
  const int nar = (int)P->arow_slot.size();
  std::vector<char> keep(nar, 1);
  auto single = [&](int r) {
    const int64_t e = P->adj_ptr[r];
    return P->adj_ptr[r + 1] - e == 1 && P->aent_w[e] == 1.0;
  };
  int r = 0;
  while (r < nar) {
    if (!single(r)) {
      ++r;
      continue;
    }
    const int ds = P->arow_slot[r];
    const int gs = P->aent_slot[P->adj_ptr[r]];
    int r1 = r;
    while (r1 < nar && single(r1) && P->arow_slot[r1] == ds && P->aent_slot[P->adj_ptr[r1]] == gs)
      ++r1;
    const bc_block& D = P->blocks[P->slot_block[ds]];
    const bc_block& G = P->blocks[P->slot_block[gs]];
    const int L = D.nlevels;
    const int64_t dls = L > 1 ? D.level_stride : 0;
    const int64_t gls = G.nlevels > 1 ? G.level_stride : 0;
    const bool lev_fast = L == 1 || (dls == 1 && gls == 1);
    std::vector<int4> runs;
    bool fits = G.nlevels == L;
    for (int l = 0; fits && l < (lev_fast ? 1 : L); ++l) {
      for (int q = r; q < r1; ++q) {
        const int64_t d = P->arow_off[q] + (lev_fast ? 0 : l * dls);
        const int64_t g = P->aent_off[P->adj_ptr[q]] + (lev_fast ? 0 : l * gls);
        const int len = lev_fast ? L : 1;
        if (d + len > INT32_MAX || g + len > INT32_MAX) {
          fits = false;
          break;
        }
        if (!runs.empty() && d == runs.back().x + runs.back().z &&
            g == runs.back().y + runs.back().z && runs.back().z + len <= 2048) {
          runs.back().z += len;
          continue;
        }
        runs.push_back(make_int4((int)d, (int)g, len, 0));
      }
    }
    const int64_t total = (int64_t)(r1 - r) * L;
    if (fits && !runs.empty() && total >= BC_RUN_MIN_AVG * (int64_t)runs.size()) {
      P->add_segs.push_back({ds, gs, (int)P->add_runs.size(), (int)runs.size()});
      P->add_runs.insert(P->add_runs.end(), runs.begin(), runs.end());
      std::fill(keep.begin() + r, keep.begin() + r1, 0);
    }
    r = r1;
  }
  // the gather keeps the other rows
  std::vector<int32_t> rs, ro, es, eo;
  std::vector<int64_t> ptr{0};
  std::vector<double> ew;
  for (int q = 0; q < nar; ++q) {
    if (!keep[q]) continue;
    rs.push_back(P->arow_slot[q]);
    ro.push_back(P->arow_off[q]);
    for (int64_t e = P->adj_ptr[q]; e < P->adj_ptr[q + 1]; ++e) {
      es.push_back(P->aent_slot[e]);
      eo.push_back(P->aent_off[e]);
      ew.push_back(P->aent_w[e]);
    }
    ptr.push_back((int64_t)ew.size());
  }
  P->arow_slot.swap(rs);
  P->arow_off.swap(ro);
  P->aent_slot.swap(es);
  P->aent_off.swap(eo);
  P->aent_w.swap(ew);
  P->adj_ptr.swap(ptr);
}

// Within each data slot, the transpose rows read by one ghost slot (the
// slot of their first entry) are made consecutive, in data-offset order:
// consecutive rows then gather from one neighbour strip, so tiles of them
// can stage that strip (and more items find one common ghost slot).  Each
// data value keeps its one row and its entries' ghost order.
void group_rows_by_reader(bc_plan* P) {
  const size_t nr = P->arow_slot.size();
  std::vector<size_t> order(nr);
  std::iota(order.begin(), order.end(), size_t(0));
  auto reader = [&](size_t r) {
    return P->adj_ptr[r + 1] > P->adj_ptr[r] ? P->aent_slot[(size_t)P->adj_ptr[r]] : -1;
  };
  std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t b) {
    if (P->arow_slot[a] != P->arow_slot[b]) return P->arow_slot[a] < P->arow_slot[b];
    return reader(a) < reader(b);
  });
  std::vector<int32_t> rs(nr), ro(nr), es, eo;
  std::vector<int64_t> ptr{0};
  std::vector<double> ew;
  es.reserve(P->aent_slot.size());
  eo.reserve(P->aent_off.size());
  ew.reserve(P->aent_w.size());
  for (size_t t = 0; t < nr; ++t) {
    const size_t r = order[t];
    rs[t] = P->arow_slot[r];
    ro[t] = P->arow_off[r];
    for (int64_t e = P->adj_ptr[r]; e < P->adj_ptr[r + 1]; ++e) {
      es.push_back(P->aent_slot[(size_t)e]);
      eo.push_back(P->aent_off[(size_t)e]);
      ew.push_back(P->aent_w[(size_t)e]);
    }
    ptr.push_back((int64_t)ew.size());
  }
  P->arow_slot.swap(rs);
  P->arow_off.swap(ro);
  P->aent_slot.swap(es);
  P->aent_off.swap(eo);
  P->aent_w.swap(ew);
  P->adj_ptr.swap(ptr);
}

void build_transpose(bc_plan* P) {
  const ExplicitRows& R = P->rows;
  struct E {
    int32_t cs;
    int64_t co;
    int32_t rs;
    int64_t ro;
    double w;
  };
  std::vector<E> ents;
  ents.reserve(R.val.size());
  for (size_t r = 0; r < R.slot.size(); ++r)
    for (int64_t e = R.ptr[r]; e < R.ptr[r + 1]; ++e)
      ents.push_back({R.cslot[e], R.coff[e], R.slot[r], R.off[r], R.val[e]});
  std::stable_sort(ents.begin(), ents.end(), [](const E& a, const E& b) {
    if (a.cs != b.cs) return a.cs < b.cs;
    if (a.co != b.co) return a.co < b.co;
    if (a.rs != b.rs) return a.rs < b.rs;
    return a.ro < b.ro;
  });
  P->arow_slot.clear();
  P->arow_off.clear();
  P->adj_ptr.assign(1, 0);
  P->aent_slot.clear();
  P->aent_off.clear();
  P->aent_w.clear();
  for (size_t e = 0; e < ents.size(); ++e) {
    if (e == 0 || ents[e].cs != ents[e - 1].cs || ents[e].co != ents[e - 1].co) {
      if (e) P->adj_ptr.push_back((int64_t)P->aent_w.size());
      P->arow_slot.push_back(ents[e].cs);
      P->arow_off.push_back((int32_t)ents[e].co);
    }
    P->aent_slot.push_back(ents[e].rs);
    P->aent_off.push_back((int32_t)ents[e].ro);
    P->aent_w.push_back(ents[e].w);
  }
  if (!ents.empty()) P->adj_ptr.push_back((int64_t)P->aent_w.size());
  P->adj_rows_total = (int64_t)P->arow_slot.size();
  P->adj_nnz_total = (int64_t)P->aent_w.size();
  P->has_adjoint = true;
  if (!P->opts.no_runs) split_unit_copies(P);
  group_rows_by_reader(P);
}

// -- device upload -------------------------------------------------------------
// streams one plan's persistent launches can run on at the same time
constexpr int kCounterStreams = 64;

struct Layout {
  size_t off = 0;
  size_t take(size_t bytes) {
    const size_t o = off;
    off += (bytes + 255) & ~size_t(255);
    return o;
  }
};

template <typename T>
void put_dtype(std::vector<char>& host, size_t off, const std::vector<double>& v) {
  T* d = reinterpret_cast<T*>(host.data() + off);
  for (size_t i = 0; i < v.size(); ++i) d[i] = (T)v[i];
}

template <typename V>
void put_raw(std::vector<char>& host, size_t off, const std::vector<V>& v) {
  if (!v.empty()) std::memcpy(host.data() + off, v.data(), v.size() * sizeof(V));
}

bc_status upload_tables(bc_plan* P) {
  const size_t S = P->esize;
  Layout L;
  const size_t o_ls = L.take(P->slot_ls.size() * 4);
  const size_t o_cd = L.take(P->ctab_d.size() * 4);
  const size_t o_cs2 = L.take(P->ctab_s.size() * 4);
  const size_t o_idx = L.take(P->itp_idx.size() * sizeof(int4));
  const size_t o_w = L.take(P->itp_w.size() * S);
  const size_t o_m = L.take(P->itp_m.size() * S);
  const size_t o_cp = L.take(P->csr_nnz.size() * 4);
  const size_t o_cs = L.take(P->csr_slot.size() * 4);
  const size_t o_co = L.take(P->csr_off.size() * 4);
  const size_t o_cv = L.take(P->csr_val.size() * S);
  const size_t o_cr = L.take(P->csr_rhs.size() * S);
  const size_t o_k = L.take(P->const_val.size() * S);
  const size_t o_as = L.take(P->arow_slot.size() * 4);
  const size_t o_ao = L.take(P->arow_off.size() * 4);
  const size_t o_ap = L.take(P->adj_ptr.size() * 8);
  const size_t o_es = L.take(P->aent_slot.size() * 4);
  const size_t o_eo = L.take(P->aent_off.size() * 4);
  const size_t o_ew = L.take(P->aent_w.size() * S);
  const auto& Y = P->sync;
  const size_t o_yr = L.take(Y.row.size() * sizeof(int4));
  const size_t o_yp = L.take(Y.ptr.size() * 4);
  const size_t o_ye = L.take(Y.ent.size() * sizeof(int2));
  const size_t o_yw = L.take(Y.w.size() * S);
  const size_t o_yc = L.take(Y.col.size() * sizeof(int4));
  const size_t o_ycp = L.take(Y.cptr.size() * 4);
  const size_t o_ycs = L.take(Y.cstage.size() * 4);
  const size_t o_ycw = L.take(Y.cw.size() * S);
  const size_t o_yst = L.take((size_t)Y.stage * S);
  const size_t o_ctr = L.take(kCtrWords * kFamilies * kCounterStreams * sizeof(unsigned));  // zero
  std::vector<char> host(L.off + 256, 0);
  put_raw(host, o_yr, Y.row);
  put_raw(host, o_yp, Y.ptr);
  put_raw(host, o_ye, Y.ent);
  put_raw(host, o_yc, Y.col);
  put_raw(host, o_ycp, Y.cptr);
  put_raw(host, o_ycs, Y.cstage);
  put_raw(host, o_ls, P->slot_ls);
  put_raw(host, o_cd, P->ctab_d);
  put_raw(host, o_cs2, P->ctab_s);
  put_raw(host, o_idx, P->itp_idx);
  put_raw(host, o_cp, P->csr_nnz);
  put_raw(host, o_cs, P->csr_slot);
  put_raw(host, o_co, P->csr_off);
  put_raw(host, o_as, P->arow_slot);
  put_raw(host, o_ao, P->arow_off);
  put_raw(host, o_ap, P->adj_ptr);
  put_raw(host, o_es, P->aent_slot);
  put_raw(host, o_eo, P->aent_off);
  if (P->dtype == BC_F64) {
    put_dtype<double>(host, o_w, P->itp_w);
    put_dtype<double>(host, o_m, P->itp_m);
    put_dtype<double>(host, o_cv, P->csr_val);
    put_dtype<double>(host, o_cr, P->csr_rhs);
    put_dtype<double>(host, o_k, P->const_val);
    put_dtype<double>(host, o_ew, P->aent_w);
    put_dtype<double>(host, o_yw, Y.w);
    put_dtype<double>(host, o_ycw, Y.cw);
  } else {
    put_dtype<float>(host, o_w, P->itp_w);
    put_dtype<float>(host, o_m, P->itp_m);
    put_dtype<float>(host, o_cv, P->csr_val);
    put_dtype<float>(host, o_cr, P->csr_rhs);
    put_dtype<float>(host, o_k, P->const_val);
    put_dtype<float>(host, o_ew, P->aent_w);
    put_dtype<float>(host, o_yw, Y.w);
    put_dtype<float>(host, o_ycw, Y.cw);
  }
  cudaError_t e = dev_malloc(&P->tables.base, host.size());
  if (e != cudaSuccess) {
    P->tables.base = nullptr;
    return cuda_fail(e, "device tables");
  }
  P->tables.bytes = host.size();
  e = cudaMemcpy(P->tables.base, host.data(), host.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(e, "device tables upload");
  char* b = static_cast<char*>(P->tables.base);
  Ctx& c = P->ctx;
  c.slot_ls = reinterpret_cast<const int32_t*>(b + o_ls);
  c.ctab_d = reinterpret_cast<const int32_t*>(b + o_cd);
  c.ctab_s = reinterpret_cast<const int32_t*>(b + o_cs2);
  c.itp_idx = reinterpret_cast<const int4*>(b + o_idx);
  c.itp_w = b + o_w;
  c.itp_m = b + o_m;
  c.csr_nnz = reinterpret_cast<const int32_t*>(b + o_cp);
  c.csr_slot = reinterpret_cast<const int32_t*>(b + o_cs);
  c.csr_off = reinterpret_cast<const int32_t*>(b + o_co);
  c.csr_val = b + o_cv;
  c.csr_rhs = b + o_cr;
  c.const_val = b + o_k;
  c.arow_slot = reinterpret_cast<const int32_t*>(b + o_as);
  c.arow_off = reinterpret_cast<const int32_t*>(b + o_ao);
  c.adj_ptr = reinterpret_cast<const int64_t*>(b + o_ap);
  c.aent_slot = reinterpret_cast<const int32_t*>(b + o_es);
  c.aent_off = reinterpret_cast<const int32_t*>(b + o_eo);
  c.aent_w = b + o_ew;
  SyncCtx& y = P->sync_ctx;
  y.nrows = (int)Y.row.size();
  y.ncols = (int)Y.col.size();
  y.lmax = 0;
  y.level_fast = 1;
  for (const int4& r : Y.row) {
    y.lmax = std::max(y.lmax, r.w);
    if (r.w > 1 && P->slot_ls[r.x] != 1) y.level_fast = 0;
  }
  y.row = reinterpret_cast<const int4*>(b + o_yr);
  y.ptr = reinterpret_cast<const int32_t*>(b + o_yp);
  y.ent = reinterpret_cast<const int2*>(b + o_ye);
  y.w = b + o_yw;
  y.col = reinterpret_cast<const int4*>(b + o_yc);
  y.cptr = reinterpret_cast<const int32_t*>(b + o_ycp);
  y.cstage = reinterpret_cast<const int32_t*>(b + o_ycs);
  y.cw = b + o_ycw;
  y.stage = b + o_yst;
  P->d_ctr = reinterpret_cast<unsigned*>(b + o_ctr);
  return BC_OK;
}

bc_status upload_work(bc_plan* P) {
  if (P->work.base) {
    cudaFree(P->work.base);
    P->work.base = nullptr;
  }
  Layout L;
  const size_t o_i = L.take(P->items.size() * sizeof(Item));
  size_t o_f[kFamilies];
  for (int f = 0; f < kFamilies; ++f) o_f[f] = L.take(P->fam_items[f].size() * sizeof(Item));
  const size_t o_r = L.take(P->runs.size() * sizeof(int4));
  const size_t o_a = L.take(P->adj_items.size() * sizeof(Item));
  const size_t o_z = L.take(P->adj_zero.size() * sizeof(Item));
  const size_t o_all = L.take(P->all_items.size() * sizeof(Item));
  const size_t o_box = L.take(P->itp_box.size() * 4);
  const size_t o_cbox = L.take(P->csr_box.size() * 4);
  const size_t o_abox = L.take(P->adj_box.size() * 4);
  std::vector<char> host(L.off + 256, 0);
  put_raw(host, o_i, P->items);
  put_raw(host, o_all, P->all_items);
  put_raw(host, o_box, P->itp_box);
  put_raw(host, o_cbox, P->csr_box);
  put_raw(host, o_abox, P->adj_box);
  for (int f = 0; f < kFamilies; ++f) put_raw(host, o_f[f], P->fam_items[f]);
  put_raw(host, o_r, P->runs);
  put_raw(host, o_a, P->adj_items);
  put_raw(host, o_z, P->adj_zero);
  cudaError_t e = dev_malloc(&P->work.base, host.size());
  if (e != cudaSuccess) {
    P->work.base = nullptr;
    return cuda_fail(e, "device work list");
  }
  P->work.bytes = host.size();
  e = cudaMemcpy(P->work.base, host.data(), host.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(e, "device work list upload");
  char* b = static_cast<char*>(P->work.base);
  P->d_items = reinterpret_cast<Item*>(b + o_i);
  for (int f = 0; f < kFamilies; ++f) P->d_fam[f] = reinterpret_cast<Item*>(b + o_f[f]);
  P->ctx.runs = reinterpret_cast<const int4*>(b + o_r);
  P->d_adj = reinterpret_cast<Item*>(b + o_a);
  P->d_adj_zero = reinterpret_cast<Item*>(b + o_z);
  P->d_all = reinterpret_cast<Item*>(b + o_all);
  P->ctx.itp_box = reinterpret_cast<const int32_t*>(b + o_box);
  P->ctx.csr_box = reinterpret_cast<const int32_t*>(b + o_cbox);
  P->ctx.adj_box = reinterpret_cast<const int32_t*>(b + o_abox);
  return BC_OK;
}

void compute_stats(bc_plan* P) {
  bc_stats& st = P->stats;
  std::memset(&st, 0, sizeof(st));
  const int64_t S = P->esize;
  const ExplicitRows& R = P->rows;
  auto L_of_slot = [&](int s) { return (int64_t)P->blocks[P->slot_block[s]].nlevels; };
  // per-row kind, from the sub-matrices in order
  size_t r = 0;
  int64_t bytes = 0;
  std::vector<std::pair<int32_t, int64_t>> csr_cols;
  for (const Sub& s : P->subs) {
    const int64_t L = P->blocks[s.block].nlevels;
    const int64_t nrows = (int64_t)s.comps.size() * s.vol;
    const int64_t vals = nrows * L;
    st.ghost_values += vals;
    st.ghost_values_kind[s.kind] += vals;
    switch (s.kind) {
      case BC_ZERO: bytes += vals * S; break;
      case BC_CONST: bytes += vals * S + nrows * S; break;
      case BC_MAP: bytes += 2 * vals * S; break;
      case BC_INTERP: {
        const bool rot = s.rot_u >= 0;
        bytes += 2 * vals * S + (int64_t)s.vol * (16 + s.p * S + (rot ? 4 * S : 0));
        break;
      }
      case BC_CSR: {
        bytes += vals * S;
        for (int64_t q = 0; q < nrows; ++q, ++r) {
          bytes += 8 + S;
          for (int64_t e = R.ptr[r]; e < R.ptr[r + 1]; ++e) {
            bytes += 8 + S;
            csr_cols.push_back({R.cslot[e], R.coff[e]});
          }
        }
        continue;
      }
    }
    r += nrows;
  }
  std::sort(csr_cols.begin(), csr_cols.end());
  csr_cols.erase(std::unique(csr_cols.begin(), csr_cols.end()), csr_cols.end());
  for (auto& cc : csr_cols) bytes += L_of_slot(cc.first) * S;
  // Sync rows: written once, entries read per level, tables once
  const auto& Y = P->sync;
  st.sync_values = Y.stage;
  for (size_t q = 0; q < Y.row.size(); ++q)
    bytes += (int64_t)Y.row[q].w * S * (1 + Y.ptr[q + 1] - Y.ptr[q]) + 20 +
             (int64_t)(Y.ptr[q + 1] - Y.ptr[q]) * (8 + S);
  st.bytes_fwd = bytes;
  int64_t abytes = 4 * st.ghost_values * S;
  abytes += P->adj_rows_total * 16 + P->adj_nnz_total * (8 + S);
  // Sync: the rows' cotangents move to staging and back out through the
  // column entries (read-modify-write of every column value)
  for (size_t q = 0; q < Y.row.size(); ++q) abytes += 3 * (int64_t)Y.row[q].w * S;
  for (size_t q = 0; q < Y.col.size(); ++q)
    abytes += (int64_t)Y.col[q].z * S * (2 + Y.cptr[q + 1] - Y.cptr[q]);
  st.bytes_adj = abytes;
  st.nitems = (int64_t)P->items.size();
  st.nitems_adjoint = (int64_t)P->adj_items.size();
  st.nsubmatrices = (int64_t)P->subs.size();
  st.nslots = P->nslots;
  st.table_bytes = (int64_t)P->tables.bytes + (int64_t)P->work.bytes;
  st.transpose_nnz = P->adj_nnz_total;
  st.element_size = P->esize;
  st.form_threads = P->opts.threads;
  st.form_ctas_per_sm = P->opts.ctas_per_sm;
  st.units_per_lane = P->opts.units_per_lane;
  st.batch_mode = P->opts.batch_mode;
  st.level_chunk = P->opts.level_chunk;
  const int ys = P->sync_ctx.nrows > 0 ? 2 : 0;
  st.launches_fwd = ys;
  if (P->opts.batch_mode == BC_BATCH_PERSISTENT || P->opts.batch_mode == BC_BATCH_SINGLE)
    st.launches_fwd += P->all_items.empty() ? 0 : 1;
  else
    for (const auto& v : P->fam_items) st.launches_fwd += v.empty() ? 0 : 1;
  st.launches_adj = P->has_adjoint ? ys + !P->adj_items.empty() + !P->adj_zero.empty() : 0;
}

constexpr int kMaxGhostSweeps = 64;

bc_status normalise_opts(const bc_plan_opts* in, bc_plan_opts& o) {
  std::memset(&o, 0, sizeof(o));
  if (in) o = *in;
  if (o.threads == 0) o.threads = 128;
  if (o.threads != 32 && o.threads != 64 && o.threads != 128 && o.threads != 256 &&
      o.threads != 512)
    return fail(BC_ERR_INVALID_ARG, "threads must be 32, 64, 128, 256 or 512");
  if (o.units_per_lane == 0) o.units_per_lane = 4;
  if (o.units_per_lane < 1 || o.ctas_per_sm < 0 || o.unit_order < 0 || o.unit_order > 2 ||
      o.host_only < 0 || o.host_only > 1)
    return fail(BC_ERR_INVALID_ARG, "bad work-item options");
  if (o.ghost_sweeps < 0 || o.ghost_sweeps > kMaxGhostSweeps)
    return fail(BC_ERR_INVALID_ARG, "ghost_sweeps must be in 0..%d", kMaxGhostSweeps);
  if (o.batch_mode == 0) o.batch_mode = BC_BATCH_FAMILIES;
  if (o.batch_mode < BC_BATCH_PERSISTENT || o.batch_mode > BC_BATCH_SINGLE)
    return fail(BC_ERR_INVALID_ARG, "batch_mode must be 0 or a bc_batch_mode");
  if (o.scalar_runs < 0 || o.scalar_runs > 1)
    return fail(BC_ERR_INVALID_ARG, "scalar_runs must be 0 or 1");
  if (o.stencil_fusion < 0 || o.stencil_fusion > 1)
    return fail(BC_ERR_INVALID_ARG, "stencil_fusion must be 0 or 1");
  if (o.unstaged_rows < 0 || o.unstaged_rows > 1)
    return fail(BC_ERR_INVALID_ARG, "unstaged_rows must be 0 or 1");
  if (o.level_chunk != 0 && o.level_chunk != 1 && o.level_chunk != 2 && o.level_chunk != 4 &&
      o.level_chunk != 8)
    return fail(BC_ERR_INVALID_ARG, "level_chunk must be 0, 1, 2, 4 or 8");
  return BC_OK;
}

// live ghost cells of a block for a stencil (dead-ghost elimination): ghost
// cells g with g - o a data cell for some offset o
size_t live_ghosts(const bc_block& B, const int32_t* off, int noff) {
  size_t n = 0;
  for (int k = -B.h[2]; k < B.n[2] + B.h[2]; ++k)
    for (int j = -B.h[1]; j < B.n[1] + B.h[1]; ++j)
      for (int i = -B.h[0]; i < B.n[0] + B.h[0]; ++i) {
        if (i >= 0 && i < B.n[0] && j >= 0 && j < B.n[1] && k >= 0 && k < B.n[2]) continue;
        for (int o = 0; o < noff; ++o) {
          const int a = i - off[3 * o], b = j - off[3 * o + 1], c = k - off[3 * o + 2];
          if (a >= 0 && a < B.n[0] && b >= 0 && b < B.n[1] && c >= 0 && c < B.n[2]) {
            ++n;
            break;
          }
        }
      }
  return n;
}

// Tables of bc_apply_stencil: per slot a descriptor and the row of every
// ghost-frame cell (level 0, slab order: below, above, then per data plane
// the bands below and above and the two side columns), and the level-0 rows
// of A in CSR form, in the plan's dtype.
bc_status build_fusion(bc_plan* P) {
  const int S = P->esize;
  std::vector<FuseSlot> slots(P->nslots);
  int64_t fbase = 0, cta = 0;
  for (int sl = 0; sl < P->nslots; ++sl) {
    const bc_block& B = P->blocks[P->slot_block[sl]];
    FuseSlot& f = slots[sl];
    std::memset(&f, 0, sizeof(f));
    for (int d = 0; d < 3; ++d) {
      f.n[d] = B.n[d];
      f.h[d] = B.h[d];
      f.s[d] = B.stride[d];
    }
    f.L = B.nlevels;
    f.ls = B.nlevels > 1 ? B.level_stride : 0;
    f.lfast = B.nlevels > 1 && B.level_stride == 1;
    const int64_t F = (int64_t)(B.n[0] + 2 * B.h[0]) * (B.n[1] + 2 * B.h[1]) * (B.n[2] + 2 * B.h[2]);
    const int64_t D = (int64_t)B.n[0] * B.n[1] * B.n[2];
    if (F * B.nlevels >= INT32_MAX)
      return fail(BC_ERR_UNSUPPORTED, "stencil fusion: slot %d has 2^31 values or more", sl);
    f.nd = (int32_t)D;
    f.nf = (int32_t)(F - D);
    f.dL = make_div((uint32_t)f.L);
    f.dnd = make_div((uint32_t)std::max<int64_t>(D, 1));
    f.dnf = make_div((uint32_t)std::max<int64_t>(F - D, 1));
    f.dn0 = make_div((uint32_t)B.n[0]);
    f.dn01 = make_div((uint32_t)B.n[0] * (uint32_t)B.n[1]);
    f.fbase = fbase;
    f.cta0 = cta;
    f.tz = B.n[2] == 1 ? 1 : kTileZ;
    f.nt[0] = (B.n[0] + kTileX - 1) / kTileX;
    f.nt[1] = (B.n[1] + kTileY - 1) / kTileY;
    f.nt[2] = (B.n[2] + f.tz - 1) / f.tz;
    f.tiles = (int64_t)f.nt[0] * f.nt[1] * f.nt[2] * B.nlevels;
    fbase += F - D;
    cta += f.tiles + ((F - D) * B.nlevels + kFuseThreads - 1) / kFuseThreads;
  }
  P->fuse_ctas = cta;
  // frame index of a ghost cell (the device's frame_index)
  auto frame_index = [](const FuseSlot& f, int i, int j, int k) -> int64_t {
    const int64_t F0 = f.n[0] + 2 * f.h[0], F1 = f.n[1] + 2 * f.h[1];
    const int64_t slab = (int64_t)f.h[2] * F1 * F0;
    if (k < 0) return ((int64_t)(k + f.h[2]) * F1 + (j + f.h[1])) * F0 + (i + f.h[0]);
    if (k >= f.n[2]) return slab + ((int64_t)(k - f.n[2]) * F1 + (j + f.h[1])) * F0 + (i + f.h[0]);
    const int64_t plane = F1 * F0 - (int64_t)f.n[1] * f.n[0];
    const int64_t base = 2 * slab + (int64_t)k * plane;
    if (j < 0) return base + (int64_t)(j + f.h[1]) * F0 + (i + f.h[0]);
    if (j >= f.n[1]) return base + (int64_t)(f.h[1] + j - f.n[1]) * F0 + (i + f.h[0]);
    const int64_t b2 = base + 2 * (int64_t)f.h[1] * F0 + (int64_t)j * 2 * f.h[0];
    return i < 0 ? b2 + (i + f.h[0]) : b2 + f.h[0] + (i - f.n[0]);
  };
  std::vector<int32_t> frame((size_t)fbase, -1);
  const ExplicitRows& R = P->rows;
  if ((int64_t)R.val.size() >= INT32_MAX)
    return fail(BC_ERR_UNSUPPORTED, "stencil fusion: 2^31 row entries or more");
  for (size_t r = 0; r < R.slot.size(); ++r) {
    const int sl = R.slot[r];
    const bc_block& B = P->blocks[P->slot_block[sl]];
    int i, j, k;
    if (!decode_cell(B, R.off[r], i, j, k) || in_data(B, i, j, k))
      return fail(BC_ERR_UNSUPPORTED, "stencil fusion: a row is not a ghost cell");
    frame[(size_t)(slots[sl].fbase + frame_index(slots[sl], i, j, k))] = (int32_t)r;
  }
  std::vector<int32_t> rptr(R.ptr.size()), eslot(R.cslot.begin(), R.cslot.end()), eoff(R.coff.size());
  for (size_t r = 0; r < R.ptr.size(); ++r) rptr[r] = (int32_t)R.ptr[r];
  for (size_t e = 0; e < R.coff.size(); ++e) eoff[e] = (int32_t)R.coff[e];
  Layout L;
  const size_t o_s = L.take(slots.size() * sizeof(FuseSlot));
  const size_t o_f = L.take(frame.size() * 4);
  const size_t o_p = L.take(rptr.size() * 4);
  const size_t o_es = L.take(eslot.size() * 4);
  const size_t o_eo = L.take(eoff.size() * 4);
  const size_t o_v = L.take(R.val.size() * S);
  const size_t o_b = L.take(R.rhs.size() * S);
  std::vector<char> host(L.off + 256, 0);
  put_raw(host, o_s, slots);
  put_raw(host, o_f, frame);
  put_raw(host, o_p, rptr);
  put_raw(host, o_es, eslot);
  put_raw(host, o_eo, eoff);
  if (P->dtype == BC_F64) {
    put_dtype<double>(host, o_v, R.val);
    put_dtype<double>(host, o_b, R.rhs);
  } else {
    put_dtype<float>(host, o_v, R.val);
    put_dtype<float>(host, o_b, R.rhs);
  }
  cudaError_t e = dev_malloc(&P->fuse.base, host.size());
  if (e != cudaSuccess) {
    P->fuse.base = nullptr;
    return cuda_fail(e, "stencil fusion tables");
  }
  P->fuse.bytes = host.size();
  if ((e = cudaMemcpy(P->fuse.base, host.data(), host.size(), cudaMemcpyHostToDevice)) != cudaSuccess)
    return cuda_fail(e, "stencil fusion tables upload");
  char* b = static_cast<char*>(P->fuse.base);
  FuseCtx& F = P->fuse_ctx;
  F.nslots = P->nslots;
  F.slot = reinterpret_cast<const FuseSlot*>(b + o_s);
  F.frame_row = reinterpret_cast<const int32_t*>(b + o_f);
  F.rptr = reinterpret_cast<const int32_t*>(b + o_p);
  F.eslot = reinterpret_cast<const int32_t*>(b + o_es);
  F.eoff = reinterpret_cast<const int32_t*>(b + o_eo);
  F.val = b + o_v;
  F.rhs = b + o_b;
  F.slot_ls = P->ctx.slot_ls;
  return BC_OK;
}

// FNV-1a over the bytes that decide what the autotuner measures: dtype,
// block layouts, the explicit rows and the options it does not tune.
struct Fnv {
  uint64_t h = 1469598103934665603ull;
  void bytes(const void* p, size_t n) {
    const unsigned char* c = static_cast<const unsigned char*>(p);
    for (size_t i = 0; i < n; ++i) h = (h ^ c[i]) * 1099511628211ull;
  }
  template <typename V>
  void vec(const std::vector<V>& v) {
    const uint64_t n = v.size();
    bytes(&n, sizeof(n));
    if (!v.empty()) bytes(v.data(), v.size() * sizeof(V));
  }
  template <typename V>
  void val(const V& v) { bytes(&v, sizeof(V)); }
};

uint64_t plan_hash(const bc_plan* P) {
  Fnv f;
  f.val(P->dtype);
  for (const bc_block& b : P->blocks) {
    f.bytes(b.n, sizeof(b.n));
    f.bytes(b.h, sizeof(b.h));
    f.val(b.nlevels);
    f.val(b.ncomp);
    f.bytes(b.stride, sizeof(b.stride));
    f.val(b.level_stride);
  }
  const ExplicitRows& R = P->rows;
  f.vec(R.slot);
  f.vec(R.off);
  f.vec(R.ptr);
  f.vec(R.cslot);
  f.vec(R.coff);
  f.vec(R.val);
  f.vec(R.rhs);
  f.val(P->sync.stage);
  f.vec(P->sync.ptr);
  f.vec(P->sync.w);
  const bc_plan_opts& o = P->opts;
  const int32_t fixed[] = {o.unit_order, o.strict_cover, o.no_adjoint, o.no_runs,
                           o.ghost_sweeps, (int32_t)P->pruned};
  f.bytes(fixed, sizeof(fixed));
  return f.h;
}

bc_status plan_create_impl(const bc_grid* grid, const bc_submatrix* subs, int32_t nsubs,
                           const bc_plan_opts* opts, bc_plan* P,
                           const int32_t* stencil = nullptr, int nstencil = 0) {
  bc_status st = normalise_opts(opts, P->opts);
  if (st != BC_OK) return st;
  if ((st = validate_grid(grid, P)) != BC_OK) return st;
  if (nsubs < 0 || (nsubs > 0 && !subs)) return fail(BC_ERR_INVALID_ARG, "bad sub-matrix list");
  Coverage cov;
  cov.map.resize(P->nslots);
  cov.blocks = &P->blocks;
  cov.slot_block = &P->slot_block;
  std::vector<const bc_submatrix*> cs_subs;
  std::vector<int> cs_idx;
  // Sync rows (data cells) are kept apart from the ghost sub-matrices
  std::vector<int> reg, syn;
  for (int si = 0; si < nsubs; ++si) (subs[si].kind == BC_SYNC ? syn : reg).push_back(si);
  P->subs.resize(reg.size());
  P->sub_of_input.assign(nsubs, -1);
  for (size_t t = 0; t < reg.size(); ++t) P->sub_of_input[reg[t]] = (int)t;
  // pass 1: validation, coverage, tables of every kind but cubed-sphere rows
  for (size_t t = 0; t < reg.size(); ++t) {
    const int si = reg[t];
    const bc_submatrix& m = subs[si];
    Sub& s = P->subs[t];
    if ((st = read_sub(P, m, si, s)) != BC_OK) return st;
    const bc_block& B = P->blocks[s.block];
    bool ok = true, ghost = true;
    for (int c : s.comps) {
      const int slot = P->slot_base[s.block] + c;
      for_box(s, [&](int, int i, int j, int k) {
        if (in_data(B, i, j, k)) ghost = false;
        else if (!cov.mark(slot, i, j, k)) ok = false;
      });
    }
    if (!ghost) return fail(BC_ERR_OUT_OF_RANGE, "sub-matrix %d: box contains data cells", si);
    if (!ok) return fail(BC_ERR_OVERLAP, "sub-matrix %d overlaps an earlier sub-matrix", si);
    switch (m.kind) {
      case BC_ZERO:
      case BC_CONST: st = add_zero_const(P, m, si, s); break;
      case BC_MAP: st = add_map(P, m, si, s); break;
      case BC_CSR: st = add_csr(P, m, si, s); break;
      case BC_INTERP:
        st = read_interp(P, m, si, s);
        if (st == BC_OK && m.geometry == BC_GEOM_CUBED_SPHERE) {
          cs_subs.push_back(&m);
          cs_idx.push_back((int)t);
        }
        break;
    }
    if (st != BC_OK) return st;
  }
  {
    Coverage dcov;
    dcov.map.resize(P->nslots);
    dcov.blocks = &P->blocks;
    dcov.slot_block = &P->slot_block;
    for (int si : syn)
      if ((st = add_sync(P, subs[si], si, dcov)) != BC_OK) return st;
    build_sync_transpose(P);
  }
  // cell tables: every box cell's offset, and the source cell of maps
  for (Sub& s2 : P->subs) {
    const bc_block& B = P->blocks[s2.block];
    s2.ctab = (int)P->ctab_d.size();
    for_box(s2, [&](int, int i, int j, int k) {
      P->ctab_d.push_back((int32_t)cell_offset(B, i, j, k));
      if (s2.kind == BC_MAP) {
        const int g[3] = {i, j, k};
        int src[3];
        for (int d = 0; d < 3; ++d) src[d] = s2.sign[d] * g[s2.perm[d]] + s2.offset[d];
        P->ctab_s.push_back((int32_t)cell_offset(P->blocks[s2.src_block], src[0], src[1], src[2]));
      } else {
        P->ctab_s.push_back(0);
      }
    });
  }
  if (P->opts.strict_cover) {
    for (int slot = 0; slot < P->nslots; ++slot) {
      const bc_block& B = P->blocks[P->slot_block[slot]];
      const size_t F = (size_t)(B.n[0] + 2 * B.h[0]) * (B.n[1] + 2 * B.h[1]) * (B.n[2] + 2 * B.h[2]);
      const size_t D = (size_t)B.n[0] * B.n[1] * B.n[2];
      const auto& mm = cov.map[slot];
      const size_t covered = mm.empty() ? 0 : (size_t)std::count(mm.begin(), mm.end(), (uint8_t)1);
      // a pruned plan covers live ghost cells only, and must cover them all
      const size_t want = stencil ? live_ghosts(B, stencil, nstencil) : F - D;
      if (covered != want)
        return fail(BC_ERR_UNCOVERED, "slot %d: %zu ghost cells have no row", slot, want - covered);
    }
  }
  if (P->opts.host_only) {
    // no device work: the rows, the transpose and the work lists are built
    // on the host for inspection (stats, explicit rows)
    if (!cs_subs.empty())
      return fail(BC_ERR_UNSUPPORTED, "cubed-sphere geometry needs the GPU (host_only plan)");
    P->num_sms = 152;
  } else {
    // device from here on
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    e = cudaDeviceGetAttribute(&P->num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_fail(e, "device attributes");
    for (auto& a : P->aux)
      if ((e = cudaStreamCreateWithFlags(&a, cudaStreamNonBlocking)) != cudaSuccess)
        return cuda_fail(e, "plan streams");
    if ((e = cudaEventCreateWithFlags(&P->ev_fork, cudaEventDisableTiming)) != cudaSuccess)
      return cuda_fail(e, "plan events");
    for (auto& ev : P->ev_join)
      if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess)
        return cuda_fail(e, "plan events");
    if ((st = run_cubed_sphere(P, cs_subs, cs_idx)) != BC_OK) return st;
  }
  // explicit rows of interpolation sub-matrices, in sub-matrix order
  {
    ExplicitRows all;
    ExplicitRows& R = P->rows;
    size_t r = 0;
    for (Sub& s : P->subs) {
      if (s.kind == BC_INTERP) {
        ExplicitRows tmp;
        std::swap(tmp, P->rows);
        P->rows = ExplicitRows();
        append_interp_rows(P, s);
        std::swap(tmp, P->rows);
        for (size_t t = 0; t < tmp.slot.size(); ++t) {
          all.begin_row(tmp.slot[t], tmp.off[t], tmp.rhs[t]);
          for (int64_t q = tmp.ptr[t]; q < tmp.ptr[t + 1]; ++q)
            all.entry(tmp.cslot[q], tmp.coff[q], tmp.val[q]);
          all.end_row();
        }
      } else {
        const size_t nrows = s.comps.size() * (size_t)s.vol;
        for (size_t t = r; t < r + nrows; ++t) {
          all.begin_row(R.slot[t], R.off[t], R.rhs[t]);
          for (int64_t q = R.ptr[t]; q < R.ptr[t + 1]; ++q) all.entry(R.cslot[q], R.coff[q], R.val[q]);
          all.end_row();
        }
        r += nrows;
      }
    }
    P->rows = std::move(all);
  }
  if (!P->opts.no_adjoint) build_transpose(P);
  P->hash = plan_hash(P);
  build_items(P);
  if (!P->opts.host_only) {
    if ((st = upload_tables(P)) != BC_OK) return st;
    if ((st = upload_work(P)) != BC_OK) return st;
    if (P->opts.stencil_fusion && P->sync.row.empty() && (st = build_fusion(P)) != BC_OK)
      return st;
  }
  compute_stats(P);
  return BC_OK;
}

// streaming grid of a family: ctas_per_sm resident CTAs per SM (capped by
// what fits), or 0 for a plain grid with one warp per item
int stream_grid(const bc_plan* P, int fam) {
  if (P->opts.ctas_per_sm <= 0) return 0;
  const int fit = resident_ctas(P->dtype, fam, P->opts.threads, P->staged[fam]);
  return std::min(P->opts.ctas_per_sm, fit) * P->num_sms;
}

// The persistent launches' counter pair of `stream`, or nullptr when every
// pair is already bound to another stream.
unsigned* counter_for(bc_plan* P, cudaStream_t stream) {
  std::lock_guard<std::mutex> lock(P->ctr_mu);
  void* key = static_cast<void*>(stream);
  for (size_t i = 0; i < P->ctr_streams.size(); ++i)
    if (P->ctr_streams[i] == key) return P->d_ctr + kCtrWords * kFamilies * i;
  if ((int)P->ctr_streams.size() >= kCounterStreams) return nullptr;
  P->ctr_streams.push_back(key);
  return P->d_ctr + kCtrWords * kFamilies * (P->ctr_streams.size() - 1);
}

// Resident CTAs per SM of each family's persistent kernel when the families
// run side by side: shares of the SM in proportion to the family's bytes,
// at least one CTA each.
void persistent_split(bc_plan* P, int per_sm[kFamilies]) {
  double bytes[kFamilies] = {0, 0, 0, 0}, total = 0;
  for (int f = 0; f < kFamilies; ++f) {
    for (const Item& it : P->fam_items[f]) {
      double v = it.mode == MODE_RUNS ? 0 : (double)it.nunits * (it.mode >= 2 ? it.mode : 1);
      if (it.mode == MODE_RUNS)
        for (int r = it.u0; r < it.u0 + it.nunits; ++r) v += P->runs[(size_t)r].z;
      if (it.mode == MODE_TILE) v = (double)it.nunits * it.nl;
      bytes[f] += v * (it.kind == IK_MAP ? 2 : it.kind == IK_CSR ? 1 + it.p : it.kind >= IK_INTERP ? 3 : 1);
    }
    total += bytes[f];
  }
  for (int f = 0; f < kFamilies; ++f) {
    const int fit = persistent_fit(P->dtype, f, P->opts.threads, P->staged[f]);
    per_sm[f] = total > 0 ? std::max(1, (int)(fit * bytes[f] / total)) : 1;
  }
}

bc_status launch_forward(bc_plan* P, void* const* slots, int form, cudaStream_t s) {
  Ctx c = P->ctx;
  c.slots = slots;
  c.vec_runs = P->opts.scalar_runs ? 0 : 1;
  cudaError_t e = cudaSuccess;
  const int T = P->opts.threads;
  unsigned* ctr = nullptr;
  const bool single = form == BC_FORM_BATCHED && P->opts.batch_mode == BC_BATCH_SINGLE;
  if (form == BC_FORM_BATCHED && P->opts.batch_mode != BC_BATCH_FAMILIES && !single)
    ctr = counter_for(P, s);
  const bool all_in_one = single || (ctr && P->opts.batch_mode == BC_BATCH_PERSISTENT);
  // Sync rows read the input data: evaluate them into the staging buffer
  // while the ghost kernels run (they write only ghosts), write them back
  // after every kernel that reads data has run
  const bool sync = P->sync_ctx.nrows > 0;
  if (sync && form != BC_FORM_BATCHED &&
      (e = launch_sync(P->dtype, SYNC_ROWS, P->sync_ctx, slots, c.slot_ls, s)) != cudaSuccess)
    return cuda_fail(e, "Sync rows");
  if (all_in_one) {
    // one persistent launch over every item; the Sync rows beside it
    cudaStream_t ys = P->aux[kFamilies - 2];
    if (sync) {
      if ((e = cudaEventRecord(P->ev_fork, s)) != cudaSuccess ||
          (e = cudaStreamWaitEvent(ys, P->ev_fork, 0)) != cudaSuccess ||
          (e = launch_sync(P->dtype, SYNC_ROWS, P->sync_ctx, slots, c.slot_ls, ys)) != cudaSuccess ||
          (e = cudaEventRecord(P->ev_join[kFamilies - 2], ys)) != cudaSuccess)
        return cuda_fail(e, "Sync rows");
    }
    const int st = P->staged[FAM_ALL];
    e = single ? launch_family(P->dtype, FAM_ALL, c, P->d_all, (int)P->all_items.size(), T,
                               stream_grid(P, FAM_ALL), st, s)
               : launch_persistent(P->dtype, FAM_ALL, c, P->d_all, (int)P->all_items.size(), T,
                                   P->opts.ctas_per_sm, P->num_sms, ctr, st, s);
    if (sync && e == cudaSuccess) e = cudaStreamWaitEvent(s, P->ev_join[kFamilies - 2], 0);
  } else if (form == BC_FORM_BATCHED) {
    // one launch per kernel family, the families side by side
    int fams[kFamilies], nf = 0;
    for (int f = 0; f < kFamilies; ++f)
      if (!P->fam_items[f].empty()) fams[nf++] = f;
    // the Sync rows take the last plan stream (the forward has at most three
    // kernel families, so it is free)
    cudaStream_t ys = P->aux[kFamilies - 2];
    if ((nf > 1 || sync) && (e = cudaEventRecord(P->ev_fork, s)) != cudaSuccess)
      return cuda_fail(e, "fork event");
    if (sync) {
      if ((e = cudaStreamWaitEvent(ys, P->ev_fork, 0)) != cudaSuccess ||
          (e = launch_sync(P->dtype, SYNC_ROWS, P->sync_ctx, slots, c.slot_ls, ys)) != cudaSuccess ||
          (e = cudaEventRecord(P->ev_join[kFamilies - 2], ys)) != cudaSuccess)
        return cuda_fail(e, "Sync rows");
    }
    int split[kFamilies] = {0, 0, 0, 0};
    if (ctr) persistent_split(P, split);
    for (int t = 0; t < nf && e == cudaSuccess; ++t) {
      cudaStream_t st = t == 0 ? s : P->aux[t - 1];
      if (t > 0 && (e = cudaStreamWaitEvent(st, P->ev_fork, 0)) != cudaSuccess) break;
      const int f = fams[t];
      e = ctr ? launch_persistent(P->dtype, f, c, P->d_fam[f], (int)P->fam_items[f].size(), T,
                                  split[f], P->num_sms, ctr + kCtrWords * f, P->staged[f], st)
              : launch_family(P->dtype, f, c, P->d_fam[f], (int)P->fam_items[f].size(), T,
                              stream_grid(P, f), P->staged[f], st);
      if (e == cudaSuccess && t > 0) e = cudaEventRecord(P->ev_join[t - 1], st);
    }
    for (int t = 1; t < nf && e == cudaSuccess; ++t)
      e = cudaStreamWaitEvent(s, P->ev_join[t - 1], 0);
    if (sync && e == cudaSuccess) e = cudaStreamWaitEvent(s, P->ev_join[kFamilies - 2], 0);
  } else if (form == BC_FORM_TYPEWIDE) {
    for (int k = 0; k < 5 && e == cudaSuccess; ++k)
      e = launch_family(P->dtype, family_of_kind(k), c, P->d_items + P->type_begin[k],
                        P->type_end[k] - P->type_begin[k], T, 0, P->staged[FAM_ALL], s);
  } else if (form == BC_FORM_PER_BC) {
    for (size_t si = 0; si < P->subs.size() && e == cudaSuccess; ++si)
      e = launch_family(P->dtype, family_of_kind(P->subs[si].kind), c,
                        P->d_items + P->sub_begin[si], P->sub_end[si] - P->sub_begin[si], T,
                        0, P->staged[FAM_ALL], s);
  } else {
    return fail(BC_ERR_INVALID_ARG, "unknown form %d", form);
  }
  if (e == cudaSuccess) e = launch_sync(P->dtype, SYNC_COMMIT, P->sync_ctx, slots, c.slot_ls, s);
  if (e != cudaSuccess) return cuda_fail(e, "forward launch");
  return BC_OK;
}

}  // namespace

// ============================================================================
// C ABI
// ============================================================================
// Cell (i, j, k) of block B at element offset `off` from its slot pointer:
// the axes taken from the largest stride down, then checked by re-encoding
// (false for a layout whose strides do not nest).
bool decode_cell(const bc_block& B, int64_t off, int& i, int& j, int& k) {
  int ax[3] = {0, 1, 2};
  std::sort(ax, ax + 3, [&](int a, int b) { return B.stride[a] > B.stride[b]; });
  int64_t rem = off;
  int64_t c[3] = {0, 0, 0};
  for (int t = 0; t < 3; ++t) {
    c[ax[t]] = rem / B.stride[ax[t]];
    rem -= c[ax[t]] * B.stride[ax[t]];
  }
  i = (int)c[0] - B.h[0];
  j = (int)c[1] - B.h[1];
  k = (int)c[2] - B.h[2];
  return rem == 0 && in_full(B, i, j, k) && cell_offset(B, i, j, k) == off;
}

constexpr size_t kMaxFoldedRow = 4096;

// Rows that read ghost values (the iterative form HOPE(I) of Sec. II-B)
// become rows on data values only (HOPE(M)): every ghost starts at zero and
// all covered rows are evaluated together `ghost_sweeps` times, Jacobi
// style, which is one affine map of the data.  The rows of every kind come
// from a host-only plan that accepts ghost columns; each user CSR
// sub-matrix is then replaced by its folded rows (same box and components),
// all other sub-matrices pass unchanged.
bc_status fold_ghost_sweeps(const bc_grid* grid, const bc_submatrix* subs, int32_t nsubs,
                            const bc_plan_opts& opts, SubStore& out) {
  for (int32_t si = 0; si < nsubs; ++si)
    if (subs[si].kind == BC_INTERP && subs[si].geometry == BC_GEOM_CUBED_SPHERE)
      return fail(BC_ERR_UNSUPPORTED,
                  "ghost_sweeps: the cubed-sphere rows generated on the GPU cannot be folded");
  bc_plan T;
  T.allow_ghost_cols = true;
  bc_plan_opts o1 = opts;
  o1.host_only = 1;
  o1.no_adjoint = 1;
  o1.ghost_sweeps = 0;
  o1.strict_cover = 0;
  bc_status st = plan_create_impl(grid, subs, nsubs, &o1, &T);
  if (st != BC_OK) return st;
  const ExplicitRows& R = T.rows;
  const size_t nr = R.slot.size();
  std::unordered_map<int64_t, size_t> row_of;
  row_of.reserve(2 * nr);
  for (size_t r = 0; r < nr; ++r) row_of[col_key(R.slot[r], R.off[r])] = r;
  using Entries = std::vector<std::pair<int64_t, double>>;
  struct Row {
    Entries e;
    double b = 0.0;
  };
  // data entries and rhs of every row, and the ghost rows each row reads
  std::vector<Row> base(nr);
  std::vector<std::vector<std::pair<size_t, double>>> reads(nr);
  for (size_t r = 0; r < nr; ++r) {
    base[r].b = R.rhs[r];
    for (int64_t e = R.ptr[r]; e < R.ptr[r + 1]; ++e) {
      const int64_t key = col_key(R.cslot[e], R.coff[e]);
      if (T.ghost_cols.count(key)) {
        const auto it = row_of.find(key);
        if (it == row_of.end())
          return fail(BC_ERR_COLUMN_NOT_DATA,
                      "ghost_sweeps: a column is a ghost value no sub-matrix covers "
                      "(slot %d, offset %lld)", R.cslot[e], (long long)R.coff[e]);
        reads[r].push_back({it->second, R.val[e]});
      } else {
        base[r].e.push_back({key, R.val[e]});
      }
    }
  }
  // sweep 1 reads zero ghosts: every row is its data part; sweep m > 1 adds
  // the weighted rows of sweep m - 1
  std::vector<size_t> active;
  for (size_t r = 0; r < nr; ++r)
    if (!reads[r].empty()) active.push_back(r);
  std::vector<Row> cur(nr), next(nr);
  for (size_t r : active) cur[r] = base[r];
  std::unordered_map<int64_t, double> acc;
  for (int m = 2; m <= opts.ghost_sweeps; ++m) {
    for (size_t r : active) {
      acc.clear();
      double b = base[r].b;
      for (const auto& e : base[r].e) acc[e.first] += e.second;
      for (const auto& g : reads[r]) {
        const Row& src = reads[g.first].empty() ? base[g.first] : cur[g.first];
        b += g.second * src.b;
        for (const auto& e : src.e) acc[e.first] += g.second * e.second;
      }
      if (acc.size() > kMaxFoldedRow)
        return fail(BC_ERR_UNSUPPORTED, "ghost_sweeps: a folded row has more than %d entries",
                    (int)kMaxFoldedRow);
      Row& o = next[r];
      o.e.clear();
      for (const auto& e : acc)
        if (e.second != 0.0) o.e.push_back(e);  // terms that cancel exactly
      std::sort(o.e.begin(), o.e.end());
      o.b = b;
    }
    for (size_t r : active) std::swap(cur[r], next[r]);
  }
  // the user CSR sub-matrices, refilled with their folded rows
  out.subs.clear();
  out.origin.clear();
  for (int32_t si = 0; si < nsubs; ++si) {
    const bc_submatrix& m = subs[si];
    out.origin.push_back(si);
    if (m.kind != BC_CSR) {
      out.subs.push_back(m);
      continue;
    }
    const Sub& s = T.subs[(size_t)T.sub_of_input[(size_t)si]];
    const bc_block& B = T.blocks[(size_t)s.block];
    auto& rp = out.i64.emplace_back();
    auto& cb = out.i32.emplace_back();
    auto& cc = out.i32.emplace_back();
    auto& ck = out.i32.emplace_back();
    auto& cv = out.dbl.emplace_back();
    auto& rh = out.dbl.emplace_back();
    rp.push_back(0);
    for (int comp : s.comps) {
      const int slot = T.slot_base[(size_t)s.block] + comp;
      bc_status e2 = BC_OK;
      for_box(s, [&](int, int i, int j, int k) {
        if (e2 != BC_OK) return;
        const size_t r = row_of.at(col_key(slot, cell_offset(B, i, j, k)));
        const Row& row = reads[r].empty() ? base[r] : cur[r];
        for (const auto& e : row.e) {
          const int cs = (int)(e.first >> 32);
          const int64_t co = (int64_t)(uint32_t)(e.first & 0xffffffff);
          const int blk = T.slot_block[(size_t)cs];
          int ci, cj, ckk;
          if (!decode_cell(T.blocks[(size_t)blk], co, ci, cj, ckk)) {
            e2 = fail(BC_ERR_UNSUPPORTED, "ghost_sweeps: block %d's strides do not nest", blk);
            return;
          }
          cb.push_back(blk);
          cc.push_back(cs - T.slot_base[(size_t)blk]);
          ck.insert(ck.end(), {ci, cj, ckk});
          cv.push_back(e.second);
        }
        rh.push_back(row.b);
        rp.push_back((int64_t)cv.size());
      });
      if (e2 != BC_OK) return e2;
    }
    if (cv.empty()) {  // keep the arrays non-NULL
      cb.push_back(0);
      cc.push_back(0);
      ck.insert(ck.end(), {0, 0, 0});
      cv.push_back(0.0);
    }
    bc_submatrix s2 = m;
    s2.row_ptr = rp.data();
    s2.col_block = cb.data();
    s2.col_comp = cc.data();
    s2.col_ijk = ck.data();
    s2.val = cv.data();
    s2.rhs = rh.data();
    out.subs.push_back(s2);
  }
  return BC_OK;
}

// ---------------------------------------------------------------------------
// Host emulation of the work lists (test and debugging aid): replays, item by
// item, the values each forward and adjoint kernel writes, with the unit
// decompositions of the kernels (flat cell- or level-fastest units, chunks of
// levels, runs), and compares them with the plan's explicit rows.
// ---------------------------------------------------------------------------
struct WorkCheck {
  const bc_plan* P;
  int64_t problems = 0;
  std::string first;
  void problem(const char* what, int slot, int64_t off) {
    if (problems++ == 0) {
      char buf[200];
      snprintf(buf, sizeof(buf), "%s (slot %d, element %lld)", what, slot, (long long)off);
      first = buf;
    }
  }
  int64_t ls_of_slot(int slot) const {
    const bc_block& B = P->blocks[(size_t)P->slot_block[(size_t)slot]];
    return B.nlevels > 1 ? B.level_stride : 0;
  }
  int levels_of_slot(int slot) const {
    return P->blocks[(size_t)P->slot_block[(size_t)slot]].nlevels;
  }
  // every (q, l) unit of a non-run item
  template <typename F>
  void units(const Item& it, F f) const {
    const int vol = (int)it.vol.d, L = (int)it.lev.d;
    if (it.mode == MODE_TILE) {
      for (int l = it.l0; l < it.l0 + it.nl; ++l)
        for (int q = it.u0; q < it.u0 + it.nunits; ++q) f(q, l);
      return;
    }
    for (int u = it.u0; u < it.u0 + it.nunits; ++u) {
      if (it.mode == MODE_FLAT_LEVEL) {
        f(u / L, u % L);
      } else if (it.mode == MODE_FLAT_CELL) {
        f(u % vol, u / vol);
      } else {
        const int c = u / vol, q = u % vol;
        for (int l = c * it.mode; l < std::min(c * it.mode + it.mode, L); ++l) f(q, l);
      }
    }
  }
};

int64_t check_forward_list(WorkCheck& W, const std::vector<Item>& items, bool values = true) {
  const bc_plan* P = W.P;
  const ExplicitRows& R = P->rows;
  struct Want {
    size_t r;
    int l;
    int hits;
  };
  std::unordered_map<int64_t, Want> want;
  for (size_t r = 0; r < R.slot.size(); ++r)
    for (int l = 0; l < W.levels_of_slot(R.slot[r]); ++l)
      want[col_key(R.slot[r], R.off[r] + l * W.ls_of_slot(R.slot[r]))] = {r, l, 0};
  auto write = [&](int slot, int64_t E) -> Want* {
    const auto it = want.find(col_key(slot, E));
    if (it == want.end()) {
      W.problem("a forward item writes a value no row covers", slot, E);
      return nullptr;
    }
    if (++it->second.hits > 1) W.problem("a value is written twice", slot, E);
    return &it->second;
  };
  auto check_copy = [&](const Want* w, int src_slot, int64_t src_E, int slot, int64_t E) {
    const size_t r = w->r;
    const int64_t e = R.ptr[r];
    if (R.ptr[r + 1] - e != 1 || R.val[e] != 1.0 || R.rhs[r] != 0.0 || R.cslot[e] != src_slot ||
        R.coff[e] + w->l * W.ls_of_slot(R.cslot[e]) != src_E)
      W.problem("a copy reads another value than its row", slot, E);
  };
  auto check_const = [&](const Want* w, double v, int slot, int64_t E) {
    if (R.ptr[w->r + 1] != R.ptr[w->r] || R.rhs[w->r] != v)
      W.problem("a zero or constant value differs from its row", slot, E);
  };
  for (const Item& it : items) {
    if (it.mode == MODE_RUNS) {
      for (int k = it.u0; k < it.u0 + it.nunits; ++k) {
        const int4 run = P->runs[(size_t)k];
        for (int t = 0; t < run.z; ++t) {
          const Want* w = write(it.dst_slot, (int64_t)run.x + t);
          if (!w || !values) continue;
          if (it.kind == IK_MAP) check_copy(w, it.src_slot, (int64_t)run.y + t, it.dst_slot, run.x + t);
          else if (it.kind == IK_ZERO) check_const(w, 0.0, it.dst_slot, run.x + t);
          else W.problem("a run item of another kind than zero or map", it.dst_slot, run.x);
        }
      }
      continue;
    }
    W.units(it, [&](int q, int l) {
      const int64_t E = (int64_t)P->ctab_d[(size_t)(it.ctab + q)] + (int64_t)l * it.dst_ls;
      const Want* w = write(it.dst_slot, E);
      const Want* w2 = it.kind == IK_INTERP_PAIR ? write(it.dst_slot2, E) : nullptr;
      if (!w || !values) return;
      if (it.kind == IK_MAP)
        check_copy(w, it.src_slot, (int64_t)P->ctab_s[(size_t)(it.ctab + q)] + (int64_t)l * it.src_ls,
                   it.dst_slot, E);
      else if (it.kind == IK_ZERO)
        check_const(w, 0.0, it.dst_slot, E);
      else if (it.kind == IK_CONST)
        check_const(w, P->const_val[(size_t)(it.table + q)], it.dst_slot, E);
      else if (it.kind == IK_CSR) {
        // the ELL row as the CSR kernels read it (common source slot or one
        // slot per entry) against the row's own entries at this level
        const size_t row = (size_t)(it.table + q);
        const int nnz = P->csr_nnz[row];
        std::vector<std::pair<int64_t, double>> a, b;
        for (int k = 0; k < nnz; ++k) {
          const size_t e = (size_t)it.src_org + (size_t)q * (size_t)it.p + (size_t)k;
          int slot = it.src_slot >= 0 ? it.src_slot : P->csr_slot[e];
          int64_t off = P->csr_off[e];
          if (it.mode == MODE_TILE) {
            // a staged row reads its column from the tile's box
            const int32_t bx = P->csr_box[e], A = it.bw * it.bh;
            const int idx = bx % A;
            slot = bx / A ? it.bsrc2 : it.bsrc;
            off = it.borg + (int64_t)(idx % it.bw) * it.bs0 + (int64_t)(idx / it.bw) * it.bs1;
            if (bx < 0 || bx >= (it.bsrc2 >= 0 ? 2 : 1) * A || slot < 0)
              W.problem("a staged CSR entry lies outside its box", it.dst_slot, E);
          }
          const int64_t ls = it.src_slot >= 0 ? it.src_ls : W.ls_of_slot(slot);
          a.push_back({col_key(slot, off + l * ls), P->csr_val[e]});
        }
        for (int64_t e = R.ptr[w->r]; e < R.ptr[w->r + 1]; ++e)
          b.push_back({col_key(R.cslot[e], R.coff[e] + w->l * W.ls_of_slot(R.cslot[e])), R.val[e]});
        std::sort(a.begin(), a.end());
        std::sort(b.begin(), b.end());
        if (a != b || P->csr_rhs[row] != R.rhs[w->r] || nnz > it.p)
          W.problem("a CSR row reads other entries than its row", it.dst_slot, E);
      } else if (it.kind == IK_INTERP || it.kind == IK_INTERP_PAIR) {
        // the nodes and weights the interpolation kernels read (a snapped
        // row reads node 0 only), rotated for a pair, against the rows
        const size_t cell = (size_t)(it.table + q);
        int4 ix = P->itp_idx[cell];
        if (it.mode == MODE_TILE) {
          // the node offsets a staged item reads: from the cell's place in
          // its tile's box, not from the per-lane table
          const int32_t bx = P->itp_box[cell];
          const int idx = bx & kBoxIndex;
          ix.x = it.bsrc;
          ix.y = it.borg + (idx % it.bw) * it.bs0 + (idx / it.bw) * it.bs1;
          ix.z = (bx & kBoxRows) ? it.bs1 : it.bs0;
          ix.w = (bx & kBoxSnap) ? kFlagSnap : 0;
          if (idx >= it.bw * it.bh)
            W.problem("a staged row's node lies outside its box", it.dst_slot, E);
        }
        const int np_ = (ix.w & kFlagSnap) ? 1 : it.p;
        const int cu = it.comp & 0xffff, cv = it.comp >> 16;
        auto node = [&](int comp, int n) {
          const int slot = ix.x + comp;
          return col_key(slot, (int64_t)ix.y + (int64_t)n * ix.z + l * W.ls_of_slot(slot));
        };
        auto same = [&](const Want* ww, const std::vector<std::pair<int64_t, double>>& a0) {
          std::vector<std::pair<int64_t, double>> a = a0, b;
          for (int64_t e = R.ptr[ww->r]; e < R.ptr[ww->r + 1]; ++e)
            b.push_back({col_key(R.cslot[e], R.coff[e] + ww->l * W.ls_of_slot(R.cslot[e])),
                         R.val[e]});
          std::sort(a.begin(), a.end());
          std::sort(b.begin(), b.end());
          return a == b && R.rhs[ww->r] == 0.0;
        };
        const double* wt = &P->itp_w[cell * kPMax];
        if (it.kind == IK_INTERP) {
          std::vector<std::pair<int64_t, double>> a;
          for (int n = 0; n < np_; ++n) a.push_back({node(cu, n), wt[n]});
          if (!same(w, a)) W.problem("an interpolation row reads other nodes than its row",
                                     it.dst_slot, E);
        } else if (w2) {
          const double* M = &P->itp_m[cell * 4];
          for (int rr = 0; rr < 2; ++rr) {
            std::vector<std::pair<int64_t, double>> a;
            for (int n = 0; n < np_; ++n) a.push_back({node(cu, n), M[2 * rr] * wt[n]});
            for (int n = 0; n < np_; ++n) a.push_back({node(cv, n), M[2 * rr + 1] * wt[n]});
            if (!same(rr == 0 ? w : w2, a))
              W.problem("a rotated pair reads other nodes than its rows", it.dst_slot, E);
          }
        }
      }
    });
  }
  for (const auto& kv : want)
    if (kv.second.hits != 1)
      W.problem("a covered value is not written", (int)(kv.first >> 32),
                (int64_t)(uint32_t)(kv.first & 0xffffffff));
  return (int64_t)want.size();
}

int64_t check_adjoint_lists(WorkCheck& W, const std::vector<Item>& adj_items) {
  const bc_plan* P = W.P;
  const ExplicitRows& R = P->rows;
  using Terms = std::vector<std::pair<int64_t, double>>;
  // A^T by data value: the ghost values (and weights) that read it
  std::unordered_map<int64_t, Terms> want;
  for (size_t r = 0; r < R.slot.size(); ++r)
    for (int l = 0; l < W.levels_of_slot(R.slot[r]); ++l) {
      const int64_t g = col_key(R.slot[r], R.off[r] + l * W.ls_of_slot(R.slot[r]));
      for (int64_t e = R.ptr[r]; e < R.ptr[r + 1]; ++e)
        want[col_key(R.cslot[e], R.coff[e] + l * W.ls_of_slot(R.cslot[e]))].push_back({g, R.val[e]});
    }
  std::unordered_map<int64_t, Terms> got;
  std::unordered_map<int64_t, int> hits;
  for (const Item& it : adj_items) {
    if (it.kind == IK_ADD) {
      for (int k = it.u0; k < it.u0 + it.nunits; ++k) {
        const int4 run = P->runs[(size_t)k];
        for (int t = 0; t < run.z; ++t) {
          const int64_t d = col_key(it.dst_slot, (int64_t)run.x + t);
          ++hits[d];
          got[d].push_back({col_key(it.src_slot, (int64_t)run.y + t), 1.0});
        }
      }
      continue;
    }
    W.units(it, [&](int q, int l) {
      const size_t tr = (size_t)(it.table + q);
      const int64_t d = col_key(it.dst_slot, (int64_t)P->arow_off[tr] + (int64_t)l * it.dst_ls);
      ++hits[d];
      int64_t prev = INT64_MIN;
      for (int64_t e = P->adj_ptr[tr]; e < P->adj_ptr[tr + 1]; ++e) {
        int gs = P->aent_slot[(size_t)e];
        int64_t go = P->aent_off[(size_t)e];
        if (it.mode == MODE_TILE) {
          // a staged row reads its ghost value from the tile's box
          const int32_t bx = P->adj_box[(size_t)e], A = it.bw * it.bh;
          const int idx = bx % A;
          gs = bx / A ? it.bsrc2 : it.bsrc;
          go = it.borg + (int64_t)(idx % it.bw) * it.bs0 + (int64_t)(idx / it.bw) * it.bs1;
          if (bx < 0 || bx >= (it.bsrc2 >= 0 ? 2 : 1) * A || gs < 0)
            W.problem("a staged transpose entry lies outside its box", it.dst_slot, P->arow_off[tr]);
        }
        const int64_t order = col_key(gs, go);
        if (order < prev)
          W.problem("transpose entries out of ghost order", it.dst_slot, P->arow_off[tr]);
        prev = order;
        got[d].push_back({col_key(gs, go + l * W.ls_of_slot(gs)), P->aent_w[(size_t)e]});
      }
    });
  }
  for (auto& kv : want) {
    const int slot = (int)(kv.first >> 32);
    const int64_t off = (int64_t)(uint32_t)(kv.first & 0xffffffff);
    const auto h = hits.find(kv.first);
    if (h == hits.end() || h->second != 1) {
      W.problem("a data value is not gathered exactly once", slot, off);
      continue;
    }
    Terms a = kv.second, b = got[kv.first];
    std::sort(a.begin(), a.end());
    std::sort(b.begin(), b.end());
    if (a != b) W.problem("a data value gathers other terms than A^T holds", slot, off);
  }
  for (const auto& kv : hits)
    if (!want.count(kv.first))
      W.problem("the adjoint writes a data value no row reads", (int)(kv.first >> 32),
                (int64_t)(uint32_t)(kv.first & 0xffffffff));
  // the zero pass clears every covered ghost value once (coverage only)
  return (int64_t)want.size() + check_forward_list(W, P->adj_zero, false);
}

// Reconstruction-and-quadrature cubed-sphere sub-matrices become user CSR
// sub-matrices before anything else sees the list.
bc_status lower_subs(const bc_grid* grid, const bc_submatrix* subs, int32_t nsubs,
                     SubStore& low) {
  if (!has_cs_quadrature(subs, nsubs)) return BC_OK;
  std::string msg;
  const bc_status st = lower_cs_quadrature(grid, subs, nsubs, low, msg);
  return st == BC_OK ? st : fail(st, "%s", msg.c_str());
}

// The list plan creation works on: quadrature rows lowered to CSR, then rows
// that read ghost values folded (both one-to-one or one-to-two in order).
bc_status prepare_subs(const bc_grid* grid, const bc_plan_opts* opts, const bc_submatrix*& list,
                       int32_t& n, SubStore& low, SubStore& fold) {
  bc_status st = lower_subs(grid, list, n, low);
  if (st != BC_OK) return st;
  if (has_cs_quadrature(list, n)) {
    list = low.subs.data();
    n = (int32_t)low.subs.size();
  }
  if (opts && opts->ghost_sweeps != 0) {
    bc_plan_opts o;
    if ((st = normalise_opts(opts, o)) != BC_OK) return st;
    if ((st = fold_ghost_sweeps(grid, list, n, o, fold)) != BC_OK) return st;
    list = fold.subs.data();
    n = (int32_t)fold.subs.size();
  }
  return BC_OK;
}

extern "C" {

bc_status bc_plan_create(const bc_grid* grid, const bc_submatrix* subs, int32_t nsubs,
                         const bc_plan_opts* opts, bc_plan** out) {
  TraceRange trace("bc_plan_create");
  if (!out) return fail(BC_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  g_last_error.clear();
  arm_fault_injection();
  bc_plan* P = new (std::nothrow) bc_plan();
  if (!P) return fail(BC_ERR_NOMEM, "host allocation of the plan");
  bc_status st;
  try {
    SubStore low, fold;
    const bc_submatrix* list = subs;
    int32_t n = nsubs;
    st = prepare_subs(grid, opts, list, n, low, fold);
    if (st == BC_OK) {
      const bool lowered = has_cs_quadrature(subs, nsubs);
      st = plan_create_impl(grid, list, n, opts, P);
      if (st == BC_OK && lowered) {
        // back to the caller's numbering (a lowered sub-matrix maps to the
        // first of its CSR pieces)
        std::vector<int> user((size_t)nsubs, -1);
        for (size_t li = 0; li < low.origin.size(); ++li)
          if (user[(size_t)low.origin[li]] < 0) user[(size_t)low.origin[li]] = P->sub_of_input[li];
        P->sub_of_input.swap(user);
      }
    }
  } catch (const std::bad_alloc&) {
    st = fail(BC_ERR_NOMEM, "host allocation while building the plan");
  }
  if (st != BC_OK) {
    delete P;
    return st;
  }
  *out = P;
  return BC_OK;
}

bc_status bc_plan_create_pruned(const bc_grid* grid, const bc_submatrix* subs, int32_t nsubs,
                                const bc_plan_opts* opts, const int32_t* offsets,
                                int32_t noffsets, bc_plan** out) {
  TraceRange trace("bc_plan_create_pruned");
  if (!out) return fail(BC_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  g_last_error.clear();
  if (!offsets || noffsets <= 0) return fail(BC_ERR_INVALID_ARG, "empty stencil");
  arm_fault_injection();
  if (!grid || !grid->blocks || grid->nblocks < 0)
    return fail(BC_ERR_INVALID_ARG, "bad grid");
  bc_plan* P = new (std::nothrow) bc_plan();
  if (!P) return fail(BC_ERR_NOMEM, "host allocation of the plan");
  bc_status st;
  try {
    SubStore low, fold, pr;
    st = prepare_subs(grid, opts, subs, nsubs, low, fold);
    if (st == BC_OK) {
      P->pruned = true;
      st = prune_submatrices(grid, subs, nsubs, offsets, noffsets, pr);
      if (st != BC_OK)
        st = fail(st, "bad sub-matrix list");
      else
        st = plan_create_impl(grid, pr.subs.data(), (int32_t)pr.subs.size(), opts, P, offsets,
                              noffsets);
    }
  } catch (const std::bad_alloc&) {
    st = fail(BC_ERR_NOMEM, "host allocation while building the plan");
  }
  if (st != BC_OK) {
    delete P;
    return st;
  }
  *out = P;
  return BC_OK;
}

int32_t bc_plan_nslots(const bc_plan* plan) { return plan ? plan->nslots : 0; }

bc_status bc_apply_form(bc_plan* plan, void* const* slot_ptrs, int32_t form, void* stream) {
  TraceRange trace("bc_apply");
  if (!plan) return fail(BC_ERR_INVALID_ARG, "plan is NULL");
  if (plan->opts.host_only) return fail(BC_ERR_UNSUPPORTED, "host_only plan");
  if (!slot_ptrs && plan->nslots > 0) return fail(BC_ERR_INVALID_ARG, "slot_ptrs is NULL");
  return launch_forward(plan, slot_ptrs, form, static_cast<cudaStream_t>(stream));
}

bc_status bc_apply(bc_plan* plan, void* const* slot_ptrs, void* stream) {
  return bc_apply_form(plan, slot_ptrs, BC_FORM_BATCHED, stream);
}

bc_status bc_apply_adjoint(bc_plan* plan, void* const* slot_ptrs, void* stream) {
  TraceRange trace("bc_apply_adjoint");
  if (!plan) return fail(BC_ERR_INVALID_ARG, "plan is NULL");
  if (plan->opts.host_only) return fail(BC_ERR_UNSUPPORTED, "host_only plan");
  if (!plan->has_adjoint) return fail(BC_ERR_UNSUPPORTED, "plan was built without the transpose");
  if (!slot_ptrs && plan->nslots > 0) return fail(BC_ERR_INVALID_ARG, "slot_ptrs is NULL");
  Ctx c = plan->ctx;
  c.slots = slot_ptrs;
  c.vec_runs = plan->opts.scalar_runs ? 0 : 1;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int T = plan->opts.threads;
  // Sync rows: their data cells' cotangents move to the staging buffer
  // (consumed by the rows that overwrite them) before the gathers run
  cudaError_t e =
      launch_sync(plan->dtype, SYNC_SNAPSHOT, plan->sync_ctx, slot_ptrs, c.slot_ls, s);
  // one launch for the gather and the add-runs (disjoint targets), then the
  // Sync columns, then the zero pass over the ghost values they read
  if (e == cudaSuccess)
    e = launch_family(plan->dtype, FAM_ADJ, c, plan->d_adj, (int)plan->adj_items.size(), T,
                      stream_grid(plan, FAM_ADJ), plan->staged[FAM_ADJ], s);
  if (e == cudaSuccess)
    e = launch_sync(plan->dtype, SYNC_ADJOINT, plan->sync_ctx, slot_ptrs, c.slot_ls, s);
  if (e == cudaSuccess)
    e = launch_family(plan->dtype, FAM_STRUCT, c, plan->d_adj_zero,
                      (int)plan->adj_zero.size(), T, stream_grid(plan, FAM_STRUCT), 0, s);
  if (e != cudaSuccess) return cuda_fail(e, "adjoint launch");
  return BC_OK;
}

bc_status bc_apply_stencil(bc_plan* plan, void* const* slot_ptrs, void* const* out_ptrs,
                           const int32_t* offsets, const double* coeffs, int32_t npoints,
                           void* stream) {
  TraceRange trace("bc_apply_stencil");
  if (!plan) return fail(BC_ERR_INVALID_ARG, "plan is NULL");
  if (plan->opts.host_only) return fail(BC_ERR_UNSUPPORTED, "host_only plan");
  if (!plan->fuse.base)
    return fail(BC_ERR_UNSUPPORTED, plan->sync.row.empty()
                                        ? "plan built without bc_plan_opts.stencil_fusion"
                                        : "stencil fusion does not take Sync rows");
  if ((!slot_ptrs || !out_ptrs) && plan->nslots > 0)
    return fail(BC_ERR_INVALID_ARG, "slot_ptrs or out_ptrs is NULL");
  if (npoints < 1 || npoints > kFuseMaxPoints || !offsets || !coeffs)
    return fail(BC_ERR_INVALID_ARG, "need 1..%d stencil points", kFuseMaxPoints);
  FuseStencil st;
  std::memset(&st, 0, sizeof(st));
  st.n = npoints;
  for (int p = 0; p < npoints; ++p) {
    if (!std::isfinite(coeffs[p])) return fail(BC_ERR_INVALID_ARG, "stencil weight %d is not finite", p);
    for (int d = 0; d < 3; ++d) {
      const int o = offsets[3 * p + d];
      for (const bc_block& B : plan->blocks)
        if (o > B.h[d] || o < -B.h[d])
          return fail(BC_ERR_HALO_TOO_WIDE, "stencil point %d reaches %d cells along axis %d, "
                      "past a ghost width of %d", p, o, d, B.h[d]);
      if (o > 2 || o < -2)
        return fail(BC_ERR_UNSUPPORTED, "stencil point %d reaches %d cells along axis %d "
                    "(at most 2)", p, o, d);
      st.o[p][d] = (int8_t)o;
      st.r[d] = std::max(st.r[d], std::abs(o));
    }
    st.c[p] = coeffs[p];
  }
  cudaError_t e = launch_fused(plan->dtype, plan->fuse_ctx, st, slot_ptrs, out_ptrs,
                               plan->fuse_ctas, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "stencil launch");
  return BC_OK;
}

}  // extern "C"

struct bc_pack {
  int esize = 4;
  int64_t size = 0, nctas = 0;
  int nboxes = 0;
  DevBuf boxes;
};

extern "C" {

bc_status bc_pack_create(const bc_grid* grid, const bc_box* boxes, int32_t nboxes,
                         bc_pack** out) {
  if (!out) return fail(BC_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!grid || !grid->blocks || grid->nblocks <= 0 || nboxes < 0 || (nboxes > 0 && !boxes))
    return fail(BC_ERR_INVALID_ARG, "bad grid or box list");
  if (grid->dtype != BC_F32 && grid->dtype != BC_F64) return fail(BC_ERR_INVALID_ARG, "bad dtype");
  std::vector<int32_t> slot0(grid->nblocks);
  int32_t ns = 0;
  for (int b = 0; b < grid->nblocks; ++b) {
    slot0[b] = ns;
    ns += grid->blocks[b].ncomp;
  }
  std::vector<PackBox> desc(nboxes);
  int64_t pos = 0, cta = 0;
  for (int t = 0; t < nboxes; ++t) {
    const bc_box& x = boxes[t];
    if (x.block < 0 || x.block >= grid->nblocks)
      return fail(BC_ERR_INVALID_ARG, "box %d: block %d out of range", t, x.block);
    const bc_block& B = grid->blocks[x.block];
    PackBox& d = desc[t];
    std::memset(&d, 0, sizeof(d));
    int64_t cells = 1;
    for (int a = 0; a < 3; ++a) {
      if (x.hi[a] <= x.lo[a]) return fail(BC_ERR_INVALID_ARG, "box %d is empty along axis %d", t, a);
      if (x.lo[a] < -B.h[a] || x.hi[a] > B.n[a] + B.h[a])
        return fail(BC_ERR_OUT_OF_RANGE, "box %d leaves block %d's full region", t, x.block);
      d.lo[a] = x.lo[a];
      d.e[a] = x.hi[a] - x.lo[a];
      d.s[a] = B.stride[a];
      cells *= d.e[a];
    }
    d.slot0 = slot0[x.block];
    d.L = B.nlevels;
    d.ncomp = B.ncomp;
    d.ls = B.nlevels > 1 ? B.level_stride : 0;
    d.count = cells * B.nlevels * B.ncomp;
    if (d.count >= INT32_MAX) return fail(BC_ERR_UNSUPPORTED, "box %d holds 2^31 values or more", t);
    // offsets relative to the slot pointer, which addresses cell (-h, -h, -h)
    for (int a = 0; a < 3; ++a) d.lo[a] += B.h[a];
    d.dst = pos;
    d.cta0 = cta;
    d.d0 = make_div((uint32_t)d.e[0]);
    d.d1 = make_div((uint32_t)d.e[1]);
    d.d2 = make_div((uint32_t)d.e[2]);
    d.dL = make_div((uint32_t)d.L);
    pos += d.count;
    cta += (d.count + kPackThreads - 1) / kPackThreads;
  }
  std::unique_ptr<bc_pack> P(new (std::nothrow) bc_pack);
  if (!P) return fail(BC_ERR_NOMEM, "host allocation");
  P->esize = grid->dtype == BC_F64 ? 8 : 4;
  P->size = pos;
  P->nctas = cta;
  P->nboxes = nboxes;
  if (nboxes > 0) {
    arm_fault_injection();
    cudaError_t e = dev_malloc(&P->boxes.base, desc.size() * sizeof(PackBox));
    if (e != cudaSuccess) {
      P->boxes.base = nullptr;
      return cuda_fail(e, "pack descriptors");
    }
    if ((e = cudaMemcpy(P->boxes.base, desc.data(), desc.size() * sizeof(PackBox),
                        cudaMemcpyHostToDevice)) != cudaSuccess)
      return cuda_fail(e, "pack descriptors upload");
  }
  *out = P.release();
  return BC_OK;
}

int64_t bc_pack_size(const bc_pack* pack) { return pack ? pack->size : 0; }

bc_status bc_pack_run(bc_pack* pack, void* const* slot_ptrs, void* buffer, void* stream) {
  if (!pack) return fail(BC_ERR_INVALID_ARG, "pack is NULL");
  if (pack->nboxes == 0) return BC_OK;
  if (!slot_ptrs || !buffer) return fail(BC_ERR_INVALID_ARG, "slot_ptrs or buffer is NULL");
  cudaError_t e = launch_pack(pack->esize, static_cast<const PackBox*>(pack->boxes.base),
                              pack->nboxes, pack->nctas, slot_ptrs, buffer,
                              static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "pack launch");
  return BC_OK;
}

void bc_pack_destroy(bc_pack* pack) { delete pack; }

bc_status bc_fmap_submatrix(const bc_grid* grid, int32_t block, int32_t axis, int32_t side,
                            int32_t fmap, const int32_t* comps, int32_t ncomps,
                            bc_submatrix* out) {
  if (!grid || !grid->blocks || !out || !comps || ncomps <= 0)
    return fail(BC_ERR_INVALID_ARG, "NULL argument or no component");
  if (block < 0 || block >= grid->nblocks) return fail(BC_ERR_INVALID_ARG, "bad block %d", block);
  if (axis < 0 || axis > 2 || side < 0 || side > 1)
    return fail(BC_ERR_INVALID_ARG, "axis must be 0..2 and side 0 or 1");
  if (fmap != BC_FMAP_CIRCULAR && fmap != BC_FMAP_SYMMETRIC)
    return fail(BC_ERR_INVALID_ARG, "fmap must be BC_FMAP_CIRCULAR or BC_FMAP_SYMMETRIC");
  const bc_block& B = grid->blocks[block];
  for (int c = 0; c < ncomps; ++c)
    if (comps[c] < 0 || comps[c] >= B.ncomp)
      return fail(BC_ERR_INVALID_ARG, "component %d out of range", comps[c]);
  const int N = B.n[axis], h = B.h[axis];
  if (h <= 0) return fail(BC_ERR_OUT_OF_RANGE, "axis %d has no ghost cells", axis);
  if (h > N) return fail(BC_ERR_HALO_TOO_WIDE, "ghost width %d exceeds the extent %d", h, N);
  std::memset(out, 0, sizeof(*out));
  out->kind = BC_MAP;
  out->block = block;
  out->src_block = block;
  out->ncomps = ncomps;
  out->comps = comps;
  for (int d = 0; d < 3; ++d) {
    out->lo[d] = 0;
    out->hi[d] = B.n[d];
    out->perm[d] = d;
    out->sign[d] = 1;
    out->offset[d] = 0;
  }
  out->lo[axis] = side ? N : -h;
  out->hi[axis] = side ? N + h : 0;
  if (fmap == BC_FMAP_SYMMETRIC) {
    out->sign[axis] = -1;
    out->offset[axis] = side ? 2 * N - 1 : -1;
  } else {
    out->offset[axis] = side ? -N : N;
  }
  return BC_OK;
}

bc_status bc_apply_host(bc_plan* plan, void* const* host_ptrs, void* const* dev_ptrs,
                        void* const* slot_ptrs, void* stream) {
  TraceRange trace("bc_apply_host");
  if (!plan || !host_ptrs || !dev_ptrs || !slot_ptrs)
    return fail(BC_ERR_INVALID_ARG, "NULL argument");
  if (plan->opts.host_only) return fail(BC_ERR_UNSUPPORTED, "host_only plan");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // span of every slot, merged when host and device runs are both contiguous
  struct Run {
    char* h;
    char* d;
    size_t n;
  };
  std::vector<Run> runs;
  for (int slot = 0; slot < plan->nslots; ++slot) {
    const bc_block& B = plan->blocks[plan->slot_block[slot]];
    const int64_t last = cell_offset(B, B.n[0] + B.h[0] - 1, B.n[1] + B.h[1] - 1, B.n[2] + B.h[2] - 1) +
                         (int64_t)(B.nlevels - 1) * (B.nlevels > 1 ? B.level_stride : 0);
    const size_t n = (size_t)(last + 1) * plan->esize;
    char* h = static_cast<char*>(host_ptrs[slot]);
    char* d = static_cast<char*>(dev_ptrs[slot]);
    if (!runs.empty() && runs.back().h + runs.back().n == h && runs.back().d + runs.back().n == d)
      runs.back().n += n;
    else
      runs.push_back({h, d, n});
  }
  cudaError_t e = cudaSuccess;
  for (const Run& r : runs)
    if ((e = cudaMemcpyAsync(r.d, r.h, r.n, cudaMemcpyHostToDevice, s)) != cudaSuccess)
      return cuda_fail(e, "host-to-device copy");
  bc_status st = launch_forward(plan, slot_ptrs, BC_FORM_BATCHED, s);
  if (st != BC_OK) return st;
  for (const Run& r : runs)
    if ((e = cudaMemcpyAsync(r.h, r.d, r.n, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
      return cuda_fail(e, "device-to-host copy");
  return BC_OK;
}

namespace {

// Autotune results of this process, and of BC_AUTOTUNE_CACHE's file: the
// tuned options by "<plan hash>:<device name>:<SMs>".
struct TunedOpts {
  int32_t batch_mode, scalar_runs, units_per_lane, threads, level_chunk, ctas_per_sm,
      unstaged_rows;
};
std::mutex g_tune_mu;
std::map<std::string, TunedOpts> g_tuned;

std::string tune_key(const bc_plan* P) {
  int dev = 0;
  cudaDeviceProp prop{};
  std::string name = "unknown";
  if (cudaGetDevice(&dev) == cudaSuccess && cudaGetDeviceProperties(&prop, dev) == cudaSuccess)
    name = prop.name;
  for (char& ch : name)
    if (ch == ' ' || ch == ':') ch = '_';
  char buf[64];
  snprintf(buf, sizeof(buf), "%016llx", (unsigned long long)P->hash);
  return std::string(buf) + ":" + name + ":" + std::to_string(P->num_sms);
}

void set_tuned(bc_plan_opts& o, const TunedOpts& t) {
  o.batch_mode = t.batch_mode;
  o.scalar_runs = t.scalar_runs;
  o.units_per_lane = t.units_per_lane;
  o.threads = t.threads;
  o.level_chunk = t.level_chunk;
  o.ctas_per_sm = t.ctas_per_sm;
  o.unstaged_rows = t.unstaged_rows;
}

TunedOpts get_tuned(const bc_plan_opts& o) {
  return {o.batch_mode,  o.scalar_runs, o.units_per_lane, o.threads,
          o.level_chunk, o.ctas_per_sm, o.unstaged_rows};
}

// the cached choice for `key`, from memory or the cache file
bool cached_choice(const std::string& key, TunedOpts& out) {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  auto it = g_tuned.find(key);
  if (it != g_tuned.end()) {
    out = it->second;
    return true;
  }
  const char* path = std::getenv("BC_AUTOTUNE_CACHE");
  if (!path || !*path) return false;
  FILE* f = std::fopen(path, "r");
  if (!f) return false;
  char line[512];
  bool found = false;
  while (std::fgets(line, sizeof(line), f)) {
    char k[320];
    TunedOpts t{};
    if (std::sscanf(line, "%319s %d %d %d %d %d %d %d", k, &t.batch_mode, &t.scalar_runs,
                    &t.units_per_lane, &t.threads, &t.level_chunk, &t.ctas_per_sm,
                    &t.unstaged_rows) == 8 &&
        key == k) {
      out = t;
      found = true;  // the last line for a key wins
    }
  }
  std::fclose(f);
  if (found) g_tuned[key] = out;
  return found;
}

void store_choice(const std::string& key, const TunedOpts& t, float ms) {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  g_tuned[key] = t;
  const char* path = std::getenv("BC_AUTOTUNE_CACHE");
  if (!path || !*path) return;
  if (FILE* f = std::fopen(path, "a")) {
    std::fprintf(f, "%s %d %d %d %d %d %d %d %.6f\n", key.c_str(), t.batch_mode, t.scalar_runs,
                 t.units_per_lane, t.threads, t.level_chunk, t.ctas_per_sm, t.unstaged_rows, ms);
    std::fclose(f);
  }
}

}  // namespace

bc_status bc_plan_autotune(bc_plan* plan, void* const* slot_ptrs, void* stream) {
  TraceRange trace("bc_plan_autotune");
  if (plan && plan->opts.host_only) return fail(BC_ERR_UNSUPPORTED, "host_only plan");
  if (!plan || !slot_ptrs) return fail(BC_ERR_INVALID_ARG, "NULL argument");
  arm_fault_injection();
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const bc_plan_opts keep = plan->opts;
  const std::string key = tune_key(plan);
  TunedOpts hit{};
  if (cached_choice(key, hit)) {
    set_tuned(plan->opts, hit);
    build_items(plan);
    bc_status st = upload_work(plan);
    if (st != BC_OK) {
      plan->opts = keep;
      build_items(plan);
      upload_work(plan);
    }
    compute_stats(plan);
    return st;
  }
  int dev = 0, l2 = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev);
  if (e != cudaSuccess) return cuda_fail(e, "autotune device query");
  const size_t flush_bytes = std::max<size_t>((size_t)l2 * 2, size_t(64) << 20);
  void* flush = nullptr;
  e = dev_malloc(&flush, flush_bytes);
  if (e != cudaSuccess) return cuda_fail(e, "autotune flush buffer");
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if ((e = cudaEventCreate(&e0)) != cudaSuccess || (e = cudaEventCreate(&e1)) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    cudaFree(flush);
    return cuda_fail(e, "autotune events");
  }
  // one candidate: median of 6 launches after 2 warm-ups, an L2 flush before each
  auto time_candidate = [&](float& med) -> bc_status {
    build_items(plan);
    bc_status st = upload_work(plan);
    if (st != BC_OK) return st;
    std::vector<float> ts;
    for (int rep = 0; rep < 8; ++rep) {
      cudaError_t ee = cudaMemsetAsync(flush, rep & 0xff, flush_bytes, s);
      if (ee == cudaSuccess) ee = cudaEventRecord(e0, s);
      if (ee != cudaSuccess) return cuda_fail(ee, "autotune timing");
      if ((st = launch_forward(plan, slot_ptrs, BC_FORM_BATCHED, s)) != BC_OK) return st;
      if ((ee = cudaEventRecord(e1, s)) != cudaSuccess ||
          (ee = cudaEventSynchronize(e1)) != cudaSuccess)
        return cuda_fail(ee, "autotune timing");
      float ms = 0;
      if ((ee = cudaEventElapsedTime(&ms, e0, e1)) != cudaSuccess)
        return cuda_fail(ee, "autotune timing");
      if (rep >= 2) ts.push_back(ms);
    }
    std::sort(ts.begin(), ts.end());
    med = ts[ts.size() / 2];
    return BC_OK;
  };
  bool chunked = false, runs = false, staged = false;
  for (const Item& it : plan->items) {
    chunked |= it.mode >= 2 || (it.mode == MODE_FLAT_CELL && it.lev.d > 1);
    runs |= it.mode == MODE_RUNS;
    staged |= it.mode == MODE_TILE;
  }
  // one option at a time, from the plan's own options
  struct Knob {
    int32_t bc_plan_opts::*field;
    std::vector<int32_t> values;
  };
  std::vector<Knob> knobs = {{&bc_plan_opts::batch_mode,
                              {BC_BATCH_FAMILIES, BC_BATCH_SINGLE, BC_BATCH_FAMILIES_PERSISTENT,
                               BC_BATCH_PERSISTENT}}};
  if (runs) knobs.push_back({&bc_plan_opts::scalar_runs, {0, 1}});
  knobs.push_back({&bc_plan_opts::units_per_lane, {1, 2, 4, 8}});
  knobs.push_back({&bc_plan_opts::threads, {64, 128, 256}});
  if (chunked) knobs.push_back({&bc_plan_opts::level_chunk, {1, 2, 4, 8}});
  if (staged) knobs.push_back({&bc_plan_opts::unstaged_rows, {0, 1}});
  knobs.push_back({&bc_plan_opts::ctas_per_sm, {0, 1, 2}});
  float best_ms = 0;
  bc_status st = time_candidate(best_ms);
  bc_plan_opts best = plan->opts;
  for (const Knob& k : knobs) {
    for (int32_t v : k.values) {
      if (st != BC_OK || best.*(k.field) == v) continue;
      plan->opts = best;
      plan->opts.*(k.field) = v;
      float med = 0;
      st = time_candidate(med);
      if (st == BC_OK && med < best_ms) {
        best_ms = med;
        best = plan->opts;
      }
    }
  }
  plan->opts = st == BC_OK ? best : keep;
  build_items(plan);
  bc_status st2 = upload_work(plan);
  if (st == BC_OK) st = st2;
  if (st == BC_OK) store_choice(key, get_tuned(plan->opts), best_ms);
  compute_stats(plan);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(flush);
  return st;
}

// Sync rows (block-edge averaging): every row's staging range is its own,
// every Sync value is committed once, and the column lists of the adjoint
// hold exactly the rows' entries (the transpose) with the rows' staging
// offsets.
int64_t check_sync(WorkCheck& W) {
  const auto& Y = W.P->sync;
  std::vector<int> stage_hits((size_t)Y.stage, 0);
  std::unordered_set<int64_t> committed;
  std::map<int64_t, std::vector<std::pair<int, double>>> want, got;
  int64_t n = 0;
  for (size_t u = 0; u < Y.row.size(); ++u) {
    const int4 r = Y.row[u];
    if (r.w != W.levels_of_slot(r.x)) W.problem("a Sync row has another level count", r.x, r.y);
    for (int l = 0; l < r.w; ++l, ++n) {
      const int64_t idx = (int64_t)r.z + l;
      if (idx < 0 || idx >= Y.stage) {
        W.problem("a Sync row stages outside the buffer", r.x, r.y);
        continue;
      }
      ++stage_hits[(size_t)idx];
      if (!committed.insert(col_key(r.x, r.y + l * W.ls_of_slot(r.x))).second)
        W.problem("a Sync value is committed twice", r.x, r.y);
    }
    for (int32_t e = Y.ptr[u]; e < Y.ptr[u + 1]; ++e)
      want[col_key(Y.ent[(size_t)e].x, Y.ent[(size_t)e].y)].push_back({r.z, Y.w[(size_t)e]});
  }
  for (size_t i = 0; i < stage_hits.size(); ++i)
    if (stage_hits[i] != 1) W.problem("a staging value is not used exactly once", -1, (int64_t)i);
  for (size_t u = 0; u < Y.col.size(); ++u) {
    const int4 c = Y.col[u];
    if (c.z != W.levels_of_slot(c.x)) W.problem("a Sync column has another level count", c.x, c.y);
    for (int32_t e = Y.cptr[u]; e < Y.cptr[u + 1]; ++e)
      got[col_key(c.x, c.y)].push_back({Y.cstage[(size_t)e], Y.cw[(size_t)e]});
  }
  for (auto& kv : want) std::sort(kv.second.begin(), kv.second.end());
  for (auto& kv : got) std::sort(kv.second.begin(), kv.second.end());
  if (want != got) W.problem("the Sync column lists are not the transpose of the rows", -1, 0);
  return n;
}

bc_status bc_plan_check_work(const bc_plan* plan, int64_t* values, int64_t* problems) {
  if (!plan || !values || !problems) return fail(BC_ERR_INVALID_ARG, "NULL argument");
  WorkCheck W{plan};
  std::vector<Item> items = plan->items, fam, adj = plan->adj_items;
  for (const auto& f : plan->fam_items) fam.insert(fam.end(), f.begin(), f.end());
  // the checker's own test: BC_CHECK_PLANT=drop|dup|adjdrop alters the
  // copies replayed here (never the plan), which must then fail
  if (const char* plant = std::getenv("BC_CHECK_PLANT")) {
    const std::string w = plant;
    if (w == "drop" && !items.empty()) items.erase(items.begin());
    if (w == "dup" && !fam.empty()) fam.push_back(fam.front());
    if (w == "adjdrop" && !adj.empty()) adj.pop_back();
  }
  int64_t n = check_forward_list(W, items);
  n += check_forward_list(W, fam);
  n += check_forward_list(W, plan->all_items);
  if (plan->has_adjoint) n += check_adjoint_lists(W, adj);
  n += check_sync(W);
  *values = n;
  *problems = W.problems;
  if (W.problems) return fail(BC_OK, "%s", W.first.c_str());
  return BC_OK;
}

bc_status bc_plan_stats(const bc_plan* plan, bc_stats* out) {
  if (!plan || !out) return fail(BC_ERR_INVALID_ARG, "NULL argument");
  *out = plan->stats;
  return BC_OK;
}

bc_status bc_plan_const_values(bc_plan* plan, int32_t sub, void** values, int64_t* count) {
  if (!plan || !values || !count) return fail(BC_ERR_INVALID_ARG, "NULL argument");
  *values = nullptr;
  *count = 0;
  if (plan->opts.host_only) return fail(BC_ERR_UNSUPPORTED, "host-only plan: no device tables");
  if (plan->pruned)
    return fail(BC_ERR_UNSUPPORTED, "pruned plan: constant tables hold the live cells only");
  if (sub < 0 || sub >= (int32_t)plan->sub_of_input.size() || plan->sub_of_input[sub] < 0)
    return fail(BC_ERR_INVALID_ARG, "sub-matrix %d: no such ghost sub-matrix", sub);
  const Sub& s = plan->subs[plan->sub_of_input[sub]];
  if (s.kind != BC_CONST) return fail(BC_ERR_INVALID_ARG, "sub-matrix %d is not BC_CONST", sub);
  *values = static_cast<char*>(const_cast<void*>(plan->ctx.const_val)) +
            (size_t)s.table * (size_t)plan->esize;
  *count = (int64_t)s.comps.size() * s.vol;
  return BC_OK;
}

bc_status bc_plan_set_const(bc_plan* plan, int32_t sub, const void* values, void* stream) {
  void* dst = nullptr;
  int64_t n = 0;
  const bc_status st = bc_plan_const_values(plan, sub, &dst, &n);
  if (st != BC_OK) return st;
  if (!values) return fail(BC_ERR_INVALID_ARG, "values is NULL");
  const cudaError_t e = cudaMemcpyAsync(dst, values, (size_t)n * (size_t)plan->esize,
                                        cudaMemcpyDefault, static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? BC_OK : cuda_fail(e, "constant table copy");
}

bc_status bc_plan_export_csr(const bc_plan* plan, int64_t* nrows, int64_t* nnz, int32_t* row_slot,
                             int64_t* row_off, int64_t* row_ptr, int32_t* col_slot,
                             int64_t* col_off, double* val, double* rhs) {
  if (!plan || !nrows || !nnz) return fail(BC_ERR_INVALID_ARG, "NULL argument");
  // ghost rows, then the Sync rows (data cells) in one explicit row list
  ExplicitRows R = plan->rows;
  const auto& Y = plan->sync;
  for (size_t q = 0; q < Y.row.size(); ++q) {
    R.begin_row(Y.row[q].x, Y.row[q].y, 0.0);
    for (int32_t e = Y.ptr[q]; e < Y.ptr[q + 1]; ++e) R.entry(Y.ent[e].x, Y.ent[e].y, Y.w[e]);
    R.end_row();
  }
  *nrows = (int64_t)R.slot.size();
  *nnz = (int64_t)R.val.size();
  if (!row_slot) return BC_OK;
  if (!row_off || !row_ptr || !col_slot || !col_off || !val || !rhs)
    return fail(BC_ERR_INVALID_ARG, "NULL output array");
  std::vector<size_t> order(R.slot.size());
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t b) {
    if (R.slot[a] != R.slot[b]) return R.slot[a] < R.slot[b];
    return R.off[a] < R.off[b];
  });
  int64_t e = 0;
  row_ptr[0] = 0;
  for (size_t t = 0; t < order.size(); ++t) {
    const size_t r = order[t];
    row_slot[t] = R.slot[r];
    row_off[t] = R.off[r];
    rhs[t] = R.rhs[r];
    for (int64_t q = R.ptr[r]; q < R.ptr[r + 1]; ++q, ++e) {
      col_slot[e] = R.cslot[q];
      col_off[e] = R.coff[q];
      val[e] = R.val[q];
    }
    row_ptr[t + 1] = e;
  }
  return BC_OK;
}

void bc_plan_destroy(bc_plan* plan) { delete plan; }

const char* bc_status_string(bc_status status) {
  switch (status) {
    case BC_OK: return "BC_OK";
    case BC_ERR_INVALID_ARG: return "BC_ERR_INVALID_ARG";
    case BC_ERR_OVERLAP: return "BC_ERR_OVERLAP";
    case BC_ERR_COLUMN_NOT_DATA: return "BC_ERR_COLUMN_NOT_DATA";
    case BC_ERR_UNCOVERED: return "BC_ERR_UNCOVERED";
    case BC_ERR_HALO_TOO_WIDE: return "BC_ERR_HALO_TOO_WIDE";
    case BC_ERR_OUT_OF_RANGE: return "BC_ERR_OUT_OF_RANGE";
    case BC_ERR_NOMEM: return "BC_ERR_NOMEM";
    case BC_ERR_CUDA: return "BC_ERR_CUDA";
    case BC_ERR_UNSUPPORTED: return "BC_ERR_UNSUPPORTED";
    case BC_ERR_TIMEOUT: return "BC_ERR_TIMEOUT";
    case BC_ERR_GEOMETRY: return "BC_ERR_GEOMETRY";
  }
  return "BC_ERR_UNKNOWN";
}

const char* bc_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"

namespace bcg {
void set_last_error(const char* msg) { g_last_error = msg ? msg : ""; }
}  // namespace bcg

extern "C" {

}  // extern "C"
