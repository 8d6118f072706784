// Reconstruction-and-quadrature rows of cubed-sphere edge ghosts, built on
// the host in FP64 and handed to the plan as user CSR sub-matrices.
//
// The paper's HOPE example (Sec. II-B) fills a ghost cell with the quadrature
// of values at reconstruction points, each point reconstructed from the data
// of the neighbouring part of the grid; Sec. III-B writes the whole as one
// matrix Itp = Agg . Recons.  Here, for an edge ghost cell of panel P:
//
//   * Pts: the nq x nq Gauss-Legendre points of the cell in P's angles;
//   * Recons: each point is carried to the neighbour panel Q across the edge
//     and evaluated by the tensor-product polynomial of degree p - 1 per axis
//     whose averages over a p x p patch of Q's data cells are the data (cell
//     averages in Q's angles); the patch is fixed per ghost from its centre,
//     clamped into Q's data cells or (the centred variant) left centred, in
//     which case it may take Q's ghost cells and the plan folds the rows
//     that read ghosts by Jacobi sweeps;
//   * Agg: the tensor Gauss weights w_a w_b / 4 (the cell average in angle
//     coordinates);
//   * covariant vector pairs are rotated by M = e_P . e_Q^dual at every point
//     before the average.
//
// The geometry (panel frames, neighbour lookup, depth-row check) follows the
// same conventions as the device geometry of the point-interpolation rows.
#include "quadrature.h"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <vector>

namespace bcg {

namespace {

constexpr double kPi = 3.14159265358979323846;
constexpr int kQuadPMax = 8;
constexpr int kQuadMax = 8;
constexpr double kSnap = 1e-9;

struct D3 {
  double x, y, z;
};
D3 operator+(D3 a, D3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
D3 operator-(D3 a, D3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
D3 operator*(double s, D3 a) { return {s * a.x, s * a.y, s * a.z}; }
double dot(D3 a, D3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }

// outward normal and the directions of increasing first / second angle;
// panels 0..3 round the equator (+X, +Y, -X, -Y), 4 = +Z, 5 = -Z
void panel_frame(int P, D3& n, D3& ex, D3& ey) {
  static const double T[6][3][3] = {
      {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}},   {{0, 1, 0}, {-1, 0, 0}, {0, 0, 1}},
      {{-1, 0, 0}, {0, -1, 0}, {0, 0, 1}}, {{0, -1, 0}, {1, 0, 0}, {0, 0, 1}},
      {{0, 0, 1}, {0, 1, 0}, {-1, 0, 0}},  {{0, 0, -1}, {0, 1, 0}, {1, 0, 0}}};
  n = {T[P][0][0], T[P][0][1], T[P][0][2]};
  ex = {T[P][1][0], T[P][1][1], T[P][1][2]};
  ey = {T[P][2][0], T[P][2][1], T[P][2][2]};
}

D3 on_sphere(int P, double a, double b, double* cube_norm = nullptr) {
  D3 n, ex, ey;
  panel_frame(P, n, ex, ey);
  const D3 f = n + std::tan(a) * ex + std::tan(b) * ey;
  const double nf = std::sqrt(dot(f, f));
  if (cube_norm) *cube_norm = nf;
  return (1.0 / nf) * f;
}

int owner(D3 v) {
  int best = 0;
  double bp = -2.0;
  for (int P = 0; P < 6; ++P) {
    D3 n, ex, ey;
    panel_frame(P, n, ex, ey);
    if (dot(v, n) > bp) {
      bp = dot(v, n);
      best = P;
    }
  }
  return best;
}

void angles(int Q, D3 v, double& a, double& b) {
  D3 n, ex, ey;
  panel_frame(Q, n, ex, ey);
  const double dn = dot(v, n);
  a = std::atan(dot(v, ex) / dn);
  b = std::atan(dot(v, ey) / dn);
}

// d r / d a, d r / d b of the unit position on panel P
void covariant(int P, double a, double b, D3& ea, D3& eb) {
  D3 n, ex, ey;
  panel_frame(P, n, ex, ey);
  double nf;
  const D3 r = on_sphere(P, a, b, &nf);
  const double ca = std::cos(a), cb = std::cos(b);
  ea = (1.0 / (ca * ca * nf)) * (ex - dot(r, ex) * r);
  eb = (1.0 / (cb * cb * nf)) * (ey - dot(r, ey) * r);
}

// M_ij = e_P_i . e_Q^j (e^j the dual basis of Q's covariant basis)
void basis_change(int P, double a, double b, int Q, double aq, double bq, double M[4]) {
  D3 ea, eb, qa, qb;
  covariant(P, a, b, ea, eb);
  covariant(Q, aq, bq, qa, qb);
  const double g11 = dot(qa, qa), g12 = dot(qa, qb), g22 = dot(qb, qb);
  const double det = g11 * g22 - g12 * g12;
  const D3 da = (1.0 / det) * (g22 * qa - g12 * qb);
  const D3 db = (1.0 / det) * (g11 * qb - g12 * qa);
  M[0] = dot(ea, da);
  M[1] = dot(ea, db);
  M[2] = dot(eb, da);
  M[3] = dot(eb, db);
}

}  // namespace

void gauss_legendre(int n, double* x, double* w) {
  // Newton's iteration on P_n from Chebyshev-like first guesses; P_n and
  // P_{n-1} by the three-term recurrence k P_k = (2k-1) z P_{k-1} - (k-1) P_{k-2},
  // P_n'(z) = n (z P_n - P_{n-1}) / (z^2 - 1), weights 2 / ((1 - z^2) P_n'^2).
  for (int i = 0; i < (n + 1) / 2; ++i) {
    double z = std::cos(kPi * (i + 0.75) / (n + 0.5));
    double pn = 0.0, dpn = 1.0;
    for (int it = 0; it < 64; ++it) {
      double p_km1 = 1.0, p_km2 = 0.0;
      for (int k = 1; k <= n; ++k) {
        const double pk = ((2.0 * k - 1.0) * z * p_km1 - (k - 1.0) * p_km2) / k;
        p_km2 = p_km1;
        p_km1 = pk;
      }
      pn = p_km1;
      dpn = n * (z * pn - p_km2) / (z * z - 1.0);
      const double dz = pn / dpn;
      z -= dz;
      if (std::fabs(dz) <= 1e-16) break;
    }
    // derivative at the converged node
    double p_km1 = 1.0, p_km2 = 0.0;
    for (int k = 1; k <= n; ++k) {
      const double pk = ((2.0 * k - 1.0) * z * p_km1 - (k - 1.0) * p_km2) / k;
      p_km2 = p_km1;
      p_km1 = pk;
    }
    dpn = n * (z * p_km1 - p_km2) / (z * z - 1.0);
    x[i] = -z;
    x[n - 1 - i] = z;
    w[i] = w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dpn * dpn);
  }
  if (n % 2) x[n / 2] = 0.0;
}

void average_reconstruction(double x, int p, double* c) {
  // The primitive F(x) = int_{-1/2}^x P is known at the cell edges
  // e_m = m - 1/2 (the running sums of the averages) and has degree p, so
  // F = sum_m F(e_m) L_m with L_m the Lagrange basis of the p + 1 edges, and
  // P = F' gives c_k = sum_{m > k} L_m'(x).
  double dL[kQuadPMax + 1];
  for (int m = 0; m <= p; ++m) {
    const double em = m - 0.5;
    double s = 0.0;
    for (int j = 0; j <= p; ++j) {
      if (j == m) continue;
      double t = 1.0 / (em - (j - 0.5));
      for (int i = 0; i <= p; ++i)
        if (i != m && i != j) t *= (x - (i - 0.5)) / (em - (i - 0.5));
      s += t;
    }
    dL[m] = s;
  }
  double run = 0.0;
  for (int k = p - 1; k >= 0; --k) {
    run += dL[k + 1];
    c[k] = run;
  }
}

bool has_cs_quadrature(const bc_submatrix* subs, int nsubs) {
  if (!subs) return false;
  for (int i = 0; i < nsubs; ++i)
    if (subs[i].kind == BC_INTERP && (subs[i].geometry == BC_GEOM_CUBED_SPHERE_QUAD ||
                                      subs[i].geometry == BC_GEOM_CUBED_SPHERE_QUAD_CENTRED))
      return true;
  return false;
}

namespace {

bc_status bad(std::string& msg, bc_status st, int idx, const char* what) {
  char buf[256];
  snprintf(buf, sizeof(buf), "sub-matrix %d: %s", idx, what);
  msg = buf;
  return st;
}

// Weights of one ghost cell: its patch on Q and W[kn][kt] (scalar) or
// V[i][j][kn][kt] (own component i from neighbour component j).
struct GhostRow {
  int Q, dq, sn, st;
  double W[kQuadPMax][kQuadPMax];
  double V[2][2][kQuadPMax][kQuadPMax];
};

bc_status ghost_row(int P, int N, int h, int p, int nq, bool vec, bool centred, int i, int j,
                    const double* xg, const double* wg, GhostRow& g, std::string& msg,
                    int idx) {
  const double delta = kPi / (2.0 * N);
  const bool io = i < 0 || i >= N, jo = j < 0 || j >= N;
  if (io == jo) return bad(msg, BC_ERR_GEOMETRY, idx, "a box cell is not an edge ghost");
  const int d = io ? 0 : 1;
  const int side = io ? (i >= N) : (j >= N);
  // the neighbour across the edge and its axis normal to the edge
  double ref[2] = {0.0, 0.0};
  ref[d] = (kPi / 4 + delta / 2) * (side ? 1.0 : -1.0);
  const D3 vr = on_sphere(P, ref[0], ref[1]);
  const int Q = owner(vr);
  double ar, br;
  angles(Q, vr, ar, br);
  const int dq = std::fabs(ar) > std::fabs(br) ? 0 : 1;
  // the ghost centre on Q: depth row and along position
  const double a0 = -kPi / 4 + (i + 0.5) * delta, b0 = -kPi / 4 + (j + 0.5) * delta;
  const D3 vc = on_sphere(P, a0, b0);
  if (owner(vc) != Q || Q == P) return bad(msg, BC_ERR_GEOMETRY, idx, "neighbour panel check failed");
  double ac, bc_;
  angles(Q, vc, ac, bc_);
  const double fc[2] = {(ac + kPi / 4) / delta - 0.5, (bc_ + kPi / 4) / delta - 0.5};
  const double rq = std::rint(fc[dq]);
  if (std::fabs(fc[dq] - rq) > kSnap || rq < 0 || rq > N - 1)
    return bad(msg, BC_ERR_GEOMETRY, idx, "ghost centre is off the neighbour rows");
  g.Q = Q;
  g.dq = dq;
  g.sn = (int)rq - (p / 2 - 1);
  g.st = (int)std::floor(fc[1 - dq] + kSnap) - (p / 2 - 1);
  if (!centred) {
    g.sn = std::min(std::max(g.sn, 0), N - p);
    g.st = std::min(std::max(g.st, 0), N - p);
  } else if (g.sn < -h || g.sn + p > N + h || g.st < -h || g.st + p > N + h) {
    return bad(msg, BC_ERR_GEOMETRY, idx, "a centred patch leaves the neighbour's full region");
  }
  for (int a = 0; a < p; ++a)
    for (int b = 0; b < p; ++b) {
      g.W[a][b] = 0.0;
      for (int u = 0; u < 2; ++u)
        for (int v = 0; v < 2; ++v) g.V[u][v][a][b] = 0.0;
    }
  for (int ia = 0; ia < nq; ++ia)
    for (int ib = 0; ib < nq; ++ib) {
      const double a = a0 + xg[ia] * delta / 2, b = b0 + xg[ib] * delta / 2;
      const D3 v = on_sphere(P, a, b);
      if (owner(v) != Q)
        return bad(msg, BC_ERR_GEOMETRY, idx, "a quadrature point leaves the neighbour panel");
      double aq, bq;
      angles(Q, v, aq, bq);
      const double f[2] = {(aq + kPi / 4) / delta - 0.5, (bq + kPi / 4) / delta - 0.5};
      double cn[kQuadPMax], ct[kQuadPMax];
      average_reconstruction(f[dq] - g.sn, p, cn);
      average_reconstruction(f[1 - dq] - g.st, p, ct);
      const double om = wg[ia] * wg[ib] / 4.0;
      double M[4] = {1, 0, 0, 1};
      if (vec) basis_change(P, a, b, Q, aq, bq, M);
      for (int kn = 0; kn < p; ++kn)
        for (int kt = 0; kt < p; ++kt) {
          const double t = om * cn[kn] * ct[kt];
          g.W[kn][kt] += t;
          if (vec)
            for (int u = 0; u < 2; ++u)
              for (int v2 = 0; v2 < 2; ++v2) g.V[u][v2][kn][kt] += M[2 * u + v2] * t;
        }
    }
  return BC_OK;
}

}  // namespace

bc_status lower_cs_quadrature(const bc_grid* grid, const bc_submatrix* subs, int nsubs,
                              SubStore& out, std::string& msg) {
  out.subs.clear();
  out.origin.clear();
  if (!grid || !grid->blocks || grid->nblocks < 0 || nsubs < 0 || (nsubs > 0 && !subs)) {
    msg = "bad grid or sub-matrix list";
    return BC_ERR_INVALID_ARG;
  }
  for (int si = 0; si < nsubs; ++si) {
    const bc_submatrix& m = subs[si];
    const bool centred = m.geometry == BC_GEOM_CUBED_SPHERE_QUAD_CENTRED;
    if (!(m.kind == BC_INTERP && (m.geometry == BC_GEOM_CUBED_SPHERE_QUAD || centred))) {
      out.subs.push_back(m);
      out.origin.push_back(si);
      continue;
    }
    // panels: six equal N x N 2-D blocks, the box's block one of them
    int panel = -1;
    for (int t = 0; t < 6; ++t)
      if (m.cs_panels[t] < 0 || m.cs_panels[t] >= grid->nblocks)
        return bad(msg, BC_ERR_INVALID_ARG, si, "bad panel block");
    const bc_block& B0 = grid->blocks[m.cs_panels[0]];
    for (int t = 0; t < 6; ++t) {
      const int pb = m.cs_panels[t];
      const bc_block& A = grid->blocks[pb];
      if (A.n[0] != A.n[1] || A.n[0] != B0.n[0] || A.n[2] != 1 || A.h[0] != A.h[1] ||
          A.h[0] != B0.h[0] || A.nlevels != B0.nlevels || A.ncomp != B0.ncomp)
        return bad(msg, BC_ERR_INVALID_ARG, si, "panels must be equal N x N 2-D blocks");
      if (pb == m.block) panel = t;
    }
    if (m.block < 0 || m.block >= grid->nblocks || panel < 0)
      return bad(msg, BC_ERR_INVALID_ARG, si, "block is not a panel");
    const int N = grid->blocks[m.block].n[0];
    const int ncomp = grid->blocks[m.block].ncomp;
    if (m.p < 2 || m.p > kQuadPMax)
      return bad(msg, BC_ERR_UNSUPPORTED, si, "reconstruction order p must be in 2..8");
    if (m.p > N) return bad(msg, BC_ERR_INVALID_ARG, si, "stencil wider than the panel");
    if (m.nquad < 1 || m.nquad > kQuadMax)
      return bad(msg, BC_ERR_UNSUPPORTED, si, "nquad must be in 1..8");
    if (m.ncomps < 1 || !m.comps) return bad(msg, BC_ERR_INVALID_ARG, si, "no components");
    std::vector<int> scal;
    for (int c = 0; c < m.ncomps; ++c) {
      const int cc = m.comps[c];
      if (cc < 0 || cc >= ncomp) return bad(msg, BC_ERR_INVALID_ARG, si, "component out of range");
      for (int e = 0; e < c; ++e)
        if (m.comps[e] == cc) return bad(msg, BC_ERR_INVALID_ARG, si, "component listed twice");
      if (cc != m.rot_comp[0] && cc != m.rot_comp[1]) scal.push_back(cc);
    }
    const bool vec = m.rot_comp[0] >= 0 || m.rot_comp[1] >= 0;
    if (vec) {
      int found = 0;
      for (int c = 0; c < m.ncomps; ++c)
        found += (m.comps[c] == m.rot_comp[0]) + (m.comps[c] == m.rot_comp[1]);
      if (m.rot_comp[0] < 0 || m.rot_comp[1] < 0 || m.rot_comp[0] == m.rot_comp[1] || found != 2)
        return bad(msg, BC_ERR_INVALID_ARG, si, "rot_comp must name two listed components");
    }
    int64_t vol = 1;
    for (int d = 0; d < 3; ++d) vol *= std::max(0, m.hi[d] - m.lo[d]);
    if (vol <= 0) return bad(msg, BC_ERR_INVALID_ARG, si, "empty box");
    if (m.lo[2] != 0 || m.hi[2] != 1) return bad(msg, BC_ERR_GEOMETRY, si, "panels are 2-D");
    const int hh = grid->blocks[m.block].h[0];
    for (int d = 0; d < 2; ++d)
      if (m.lo[d] < -hh || m.hi[d] > N + hh)
        return bad(msg, BC_ERR_OUT_OF_RANGE, si, "box outside the panel's full region");
    double xg[kQuadMax], wg[kQuadMax];
    gauss_legendre(m.nquad, xg, wg);
    const int p = m.p, pp = p * p;
    // rows in box order (axis 0 fastest)
    std::vector<GhostRow> rows((size_t)vol);
    for (int j = m.lo[1], q = 0; j < m.hi[1]; ++j)
      for (int i = m.lo[0]; i < m.hi[0]; ++i, ++q) {
        bc_status st = ghost_row(panel, N, hh, p, m.nquad, vec, centred, i, j, xg, wg, rows[q],
                                 msg, si);
        if (st != BC_OK) return st;
      }
    // one CSR sub-matrix per group of components: the scalar ones, then the pair
    for (int grp = 0; grp < 2; ++grp) {
      std::vector<int> comps;
      if (grp == 0) comps = scal;
      else if (vec) comps = {m.rot_comp[0], m.rot_comp[1]};
      if (comps.empty()) continue;
      const int width = grp == 0 ? pp : 2 * pp;
      const int64_t nrows = (int64_t)comps.size() * vol;
      auto& rp = out.i64.emplace_back();
      auto& cb = out.i32.emplace_back();
      auto& cc = out.i32.emplace_back();
      auto& ck = out.i32.emplace_back();
      auto& cv = out.dbl.emplace_back();
      auto& cl = out.i32.emplace_back();
      rp.reserve((size_t)nrows + 1);
      cb.reserve((size_t)(nrows * width));
      cc.reserve((size_t)(nrows * width));
      ck.reserve((size_t)(nrows * width * 3));
      cv.reserve((size_t)(nrows * width));
      cl.assign(comps.begin(), comps.end());
      rp.push_back(0);
      for (size_t ci = 0; ci < comps.size(); ++ci)
        for (int64_t q = 0; q < vol; ++q) {
          const GhostRow& g = rows[(size_t)q];
          const int qb = m.cs_panels[g.Q];
          const int nsrc = grp == 0 ? 1 : 2;
          for (int sj = 0; sj < nsrc; ++sj) {
            const int col_c = grp == 0 ? comps[ci] : comps[sj];
            for (int kn = 0; kn < p; ++kn)
              for (int kt = 0; kt < p; ++kt) {
                int cell[2];
                cell[g.dq] = g.sn + kn;
                cell[1 - g.dq] = g.st + kt;
                cb.push_back(qb);
                cc.push_back(col_c);
                ck.push_back(cell[0]);
                ck.push_back(cell[1]);
                ck.push_back(0);
                cv.push_back(grp == 0 ? g.W[kn][kt] : g.V[ci][sj][kn][kt]);
              }
          }
          rp.push_back((int64_t)cv.size());
        }
      bc_submatrix s{};
      s.kind = BC_CSR;
      s.block = m.block;
      for (int d = 0; d < 3; ++d) {
        s.lo[d] = m.lo[d];
        s.hi[d] = m.hi[d];
      }
      s.ncomps = (int32_t)cl.size();
      s.comps = cl.data();
      s.row_ptr = rp.data();
      s.col_block = cb.data();
      s.col_comp = cc.data();
      s.col_ijk = ck.data();
      s.val = cv.data();
      s.rhs = nullptr;
      out.subs.push_back(s);
      out.origin.push_back(si);
    }
  }
  return BC_OK;
}

}  // namespace bcg
