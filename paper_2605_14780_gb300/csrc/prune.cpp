// Dead-ghost elimination (Sec. IV-C): keep only the ghost values that a
// stencil applied on the data cells reads, i.e. the effective space
// U(W) = { g : g - o is a data cell for some stencil offset o }, and cut every
// basic sub-matrix box to its live cells, split into disjoint boxes (the
// paper's disjoint convex sets).  The pieces carry slices of their
// sub-matrix's per-cell payload (constants, interpolation tables, CSR rows);
// maps and generated cubed-sphere geometry are position-independent and keep
// theirs.  Host code only; the pieces then go through bc_plan_create.
#include <algorithm>
#include <cstdint>
#include <vector>

#include "prune.h"

namespace bcg {

namespace {

struct Box {
  int lo[3], hi[3];
};

// live cells of one box as disjoint boxes: runs along axis 0 per (j, k) row,
// rows with equal runs merged along axis 1, then along axis 2
std::vector<Box> live_boxes(const bc_block& B, const Box& box, const int32_t* off, int noff) {
  auto live = [&](int i, int j, int k) {
    for (int o = 0; o < noff; ++o) {
      const int a = i - off[3 * o], b = j - off[3 * o + 1], c = k - off[3 * o + 2];
      if (a >= 0 && a < B.n[0] && b >= 0 && b < B.n[1] && c >= 0 && c < B.n[2]) return true;
    }
    return false;
  };
  // per (k): list of boxes spanning [j0, j1) with equal i-runs
  std::vector<Box> planes;  // merged over j, one k each
  for (int k = box.lo[2]; k < box.hi[2]; ++k) {
    std::vector<Box> open;  // boxes growing along j in this plane
    std::vector<Box> done;
    for (int j = box.lo[1]; j < box.hi[1]; ++j) {
      std::vector<std::pair<int, int>> runs;
      for (int i = box.lo[0]; i < box.hi[0];) {
        if (!live(i, j, k)) {
          ++i;
          continue;
        }
        int i1 = i + 1;
        while (i1 < box.hi[0] && live(i1, j, k)) ++i1;
        runs.push_back({i, i1});
        i = i1;
      }
      std::vector<Box> next;
      for (const auto& r : runs) {
        bool grown = false;
        for (auto it = open.begin(); it != open.end(); ++it)
          if (it->lo[0] == r.first && it->hi[0] == r.second && it->hi[1] == j) {
            Box b = *it;
            b.hi[1] = j + 1;
            next.push_back(b);
            open.erase(it);
            grown = true;
            break;
          }
        if (!grown) next.push_back(Box{{r.first, j, k}, {r.second, j + 1, k + 1}});
      }
      done.insert(done.end(), open.begin(), open.end());
      open.swap(next);
    }
    done.insert(done.end(), open.begin(), open.end());
    planes.insert(planes.end(), done.begin(), done.end());
  }
  // merge along k: equal (i, j) extents in consecutive planes
  std::vector<Box> out;
  for (const Box& b : planes) {
    bool merged = false;
    for (Box& o : out)
      if (o.lo[0] == b.lo[0] && o.hi[0] == b.hi[0] && o.lo[1] == b.lo[1] && o.hi[1] == b.hi[1] &&
          o.hi[2] == b.lo[2]) {
        o.hi[2] = b.hi[2];
        merged = true;
        break;
      }
    if (!merged) out.push_back(b);
  }
  return out;
}

}  // namespace

bc_status prune_submatrices(const bc_grid* grid, const bc_submatrix* subs, int nsubs,
                            const int32_t* offsets, int noffsets, SubStore& out) {
  if (!grid || !grid->blocks || grid->nblocks < 0 || nsubs < 0 || (nsubs > 0 && !subs))
    return BC_ERR_INVALID_ARG;
  if (noffsets <= 0 || !offsets) return BC_ERR_INVALID_ARG;
  out.subs.clear();
  for (int si = 0; si < nsubs; ++si) {
    const bc_submatrix& m = subs[si];
    // anything the plan would reject is passed through for it to report;
    // Sync rows are data cells, not ghost writes, and stay as they are
    if (m.kind == BC_SYNC || m.block < 0 || m.block >= grid->nblocks || m.ncomps < 0) {
      out.subs.push_back(m);
      continue;
    }
    const bc_block& B = grid->blocks[m.block];
    Box whole{{m.lo[0], m.lo[1], m.lo[2]}, {m.hi[0], m.hi[1], m.hi[2]}};
    int64_t vol = 1;
    for (int d = 0; d < 3; ++d) vol *= std::max(0, m.hi[d] - m.lo[d]);
    if (vol <= 0) {
      out.subs.push_back(m);
      continue;
    }
    const std::vector<Box> pieces = live_boxes(B, whole, offsets, noffsets);
    if (pieces.size() == 1) {
      const Box& p = pieces[0];
      bool same = true;
      for (int d = 0; d < 3; ++d) same = same && p.lo[d] == m.lo[d] && p.hi[d] == m.hi[d];
      if (same) {
        out.subs.push_back(m);
        continue;
      }
    }
    const int W0 = m.hi[0] - m.lo[0], W1 = m.hi[1] - m.lo[1];
    auto q_of = [&](int i, int j, int k) {
      return ((int64_t)(k - m.lo[2]) * W1 + (j - m.lo[1])) * W0 + (i - m.lo[0]);
    };
    for (const Box& p : pieces) {
      bc_submatrix s = m;
      for (int d = 0; d < 3; ++d) {
        s.lo[d] = p.lo[d];
        s.hi[d] = p.hi[d];
      }
      // original box index of every piece cell, in box order
      std::vector<int64_t> qs;
      for (int k = p.lo[2]; k < p.hi[2]; ++k)
        for (int j = p.lo[1]; j < p.hi[1]; ++j)
          for (int i = p.lo[0]; i < p.hi[0]; ++i) qs.push_back(q_of(i, j, k));
      if (m.kind == BC_CONST && m.values) {
        auto& v = out.dbl.emplace_back();
        for (int c = 0; c < m.ncomps; ++c)
          for (int64_t q : qs) v.push_back(m.values[c * vol + q]);
        s.values = v.data();
      }
      if (m.kind == BC_INTERP && m.geometry == BC_GEOM_USER) {
        if (m.itp_src_block) {
          auto& v = out.i32.emplace_back();
          for (int64_t q : qs) v.push_back(m.itp_src_block[q]);
          s.itp_src_block = v.data();
        }
        if (m.itp_axis) {
          auto& v = out.i32.emplace_back();
          for (int64_t q : qs) v.push_back(m.itp_axis[q]);
          s.itp_axis = v.data();
        }
        if (m.itp_start) {
          auto& v = out.i32.emplace_back();
          for (int64_t q : qs)
            for (int e = 0; e < 3; ++e) v.push_back(m.itp_start[3 * q + e]);
          s.itp_start = v.data();
        }
        if (m.itp_w && m.p > 0) {
          auto& v = out.dbl.emplace_back();
          for (int64_t q : qs)
            for (int e = 0; e < m.p; ++e) v.push_back(m.itp_w[q * m.p + e]);
          s.itp_w = v.data();
        }
        if (m.itp_rot) {
          auto& v = out.dbl.emplace_back();
          for (int64_t q : qs)
            for (int e = 0; e < 4; ++e) v.push_back(m.itp_rot[4 * q + e]);
          s.itp_rot = v.data();
        }
      }
      if (m.kind == BC_CSR && m.row_ptr) {
        auto& rp = out.i64.emplace_back();
        auto& cb = out.i32.emplace_back();
        auto& cc = out.i32.emplace_back();
        auto& ck = out.i32.emplace_back();
        auto& cv = out.dbl.emplace_back();
        std::vector<double>* rh = m.rhs ? &out.dbl.emplace_back() : nullptr;
        rp.push_back(0);
        for (int c = 0; c < m.ncomps; ++c)
          for (int64_t q : qs) {
            const int64_t r = c * vol + q;
            for (int64_t e = m.row_ptr[r]; e < m.row_ptr[r + 1]; ++e) {
              cb.push_back(m.col_block ? m.col_block[e] : 0);
              cc.push_back(m.col_comp ? m.col_comp[e] : 0);
              for (int d = 0; d < 3; ++d) ck.push_back(m.col_ijk ? m.col_ijk[3 * e + d] : 0);
              cv.push_back(m.val ? m.val[e] : 0.0);
            }
            rp.push_back((int64_t)cv.size());
            if (rh) rh->push_back(m.rhs[r]);
          }
        // keep the arrays non-NULL where the original had them
        if (cv.empty()) {
          cb.push_back(0);
          cc.push_back(0);
          ck.insert(ck.end(), {0, 0, 0});
          cv.push_back(0.0);
        }
        s.row_ptr = rp.data();
        s.col_block = m.col_block ? cb.data() : nullptr;
        s.col_comp = m.col_comp ? cc.data() : nullptr;
        s.col_ijk = m.col_ijk ? ck.data() : nullptr;
        s.val = m.val ? cv.data() : nullptr;
        s.rhs = rh ? rh->data() : nullptr;
      }
      out.subs.push_back(s);
    }
  }
  return BC_OK;
}

}  // namespace bcg
