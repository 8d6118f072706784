// Plan-time FP64 geometry of cubed-sphere panel-edge interpolation rows
// (arxiv 2605.14780, Sec. III-B user-defined interpolation; Sec. V-A vector
// components).  One thread per edge ghost cell computes, on the GPU:
//
//   * the equiangular gnomonic grid point of the ghost cell and the panel Q
//     whose outward normal has the largest projection on it,
//   * the data row of Q the point lies on (exactly, up to rounding) and its
//     fractional along-edge index t,
//   * either a unit copy (t within 1e-9 of a data index: grid lines align) or
//     the p-point Lagrange stencil start = clamp(floor(t) - (p/2 - 1), 0,
//     N - p) with weights prod_{m != k} (tau - m) / (k - m), tau = t - start,
//   * for covariant vector pairs, M_ij = e_own_i . e_Q^j with e = d r / d
//     angle on the unit sphere and e^j the dual basis of Q.
//
// FP64 stays here, at plan time; the per-apply kernels run in the plan's
// dtype.
#include <cmath>
#include <cstdint>

#include "bc_internal.h"

namespace bcg {
namespace {

struct V3 {
  double x, y, z;
};
__device__ __forceinline__ V3 add(V3 a, V3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
__device__ __forceinline__ V3 sub(V3 a, V3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ __forceinline__ V3 scl(double s, V3 a) { return {s * a.x, s * a.y, s * a.z}; }
__device__ __forceinline__ double dot(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }

// Panel frames: outward normal, then the directions of increasing first and
// second angle.  Panels 0..3 go round the equator (+X, +Y, -X, -Y), 4 is +Z
// and 5 is -Z.
__device__ __forceinline__ void frame(int P, V3& nrm, V3& ex, V3& ey) {
  switch (P) {
    case 0: nrm = {1, 0, 0};  ex = {0, 1, 0};  ey = {0, 0, 1}; break;
    case 1: nrm = {0, 1, 0};  ex = {-1, 0, 0}; ey = {0, 0, 1}; break;
    case 2: nrm = {-1, 0, 0}; ex = {0, -1, 0}; ey = {0, 0, 1}; break;
    case 3: nrm = {0, -1, 0}; ex = {1, 0, 0};  ey = {0, 0, 1}; break;
    case 4: nrm = {0, 0, 1};  ex = {0, 1, 0};  ey = {-1, 0, 0}; break;
    default: nrm = {0, 0, -1}; ex = {0, 1, 0}; ey = {1, 0, 0}; break;
  }
}

// cube point and unit-sphere point of angles (a, b) on panel P
__device__ V3 unit_point(int P, double a, double b, double* norm_out) {
  V3 nrm, ex, ey;
  frame(P, nrm, ex, ey);
  const V3 f = add(nrm, add(scl(tan(a), ex), scl(tan(b), ey)));
  const double nf = sqrt(dot(f, f));
  if (norm_out) *norm_out = nf;
  return scl(1.0 / nf, f);
}

__device__ int owner_panel(V3 v) {
  int best = 0;
  double bp = -2.0;
  for (int P = 0; P < 6; ++P) {
    V3 nrm, ex, ey;
    frame(P, nrm, ex, ey);
    const double pr = dot(v, nrm);
    if (pr > bp) {
      bp = pr;
      best = P;
    }
  }
  return best;
}

__device__ void angles_on(int Q, V3 v, double& a, double& b) {
  V3 nrm, ex, ey;
  frame(Q, nrm, ex, ey);
  const double dn = dot(v, nrm);
  a = atan(dot(v, ex) / dn);
  b = atan(dot(v, ey) / dn);
}

// d r / d a and d r / d b of the unit position on panel P
__device__ void basis(int P, double a, double b, V3& ea, V3& eb) {
  V3 nrm, ex, ey;
  frame(P, nrm, ex, ey);
  double nf;
  const V3 r = unit_point(P, a, b, &nf);
  const double ca = cos(a), cb = cos(b);
  const double sa = 1.0 / (ca * ca), sb = 1.0 / (cb * cb);
  ea = scl(sa / nf, sub(ex, scl(dot(r, ex), r)));
  eb = scl(sb / nf, sub(ey, scl(dot(r, ey), r)));
}

__global__ void k_cs_geometry(CsPanels pan, const int4* __restrict__ cells,
                              int ncells, int4* idx, double* w, double* m,
                              unsigned* err) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= ncells) return;
  const int4 cell = cells[g];
  const int P = cell.x, i = cell.y, j = cell.z, row = cell.w;
  const int N = pan.N, p = pan.p;
  const double pi = 3.14159265358979323846;
  const double delta = pi / (2.0 * N);
  // which edge strip: axis d out of range on side `side`
  const bool io = (i < 0 || i >= N), jo = (j < 0 || j >= N);
  int4 out = make_int4(0, 0, 0, 0);
  double* wr = w + (int64_t)row * kPMax;
  double* mr = m + (int64_t)row * 4;
  for (int n = 0; n < kPMax; ++n) wr[n] = 0.0;
  mr[0] = 1.0; mr[1] = 0.0; mr[2] = 0.0; mr[3] = 1.0;
  if (io == jo) {
    atomicOr(err, (unsigned)CS_ERR_NOT_EDGE);
    idx[row] = out;
    return;
  }
  const int d = io ? 0 : 1;
  const int side = io ? (i >= N) : (j >= N);
  // neighbour's depth axis from the middle of the strip
  double ref[2] = {0.0, 0.0};
  ref[d] = (pi / 4 + delta / 2) * (side ? 1.0 : -1.0);
  const V3 vr = unit_point(P, ref[0], ref[1], nullptr);
  const int Qr = owner_panel(vr);
  double ar, br;
  angles_on(Qr, vr, ar, br);
  const int dq = fabs(ar) > fabs(br) ? 0 : 1;
  // the ghost point
  const double a = -pi / 4 + (i + 0.5) * delta;
  const double b = -pi / 4 + (j + 0.5) * delta;
  const V3 v = unit_point(P, a, b, nullptr);
  const int Q = owner_panel(v);
  if (Q != Qr || Q == P) {
    atomicOr(err, (unsigned)CS_ERR_NEIGHBOUR);
    idx[row] = out;
    return;
  }
  double aq, bq;
  angles_on(Q, v, aq, bq);
  const double fa = (aq + pi / 4) / delta - 0.5;
  const double fb = (bq + pi / 4) / delta - 0.5;
  const double fdepth = dq == 0 ? fa : fb;
  const double t = dq == 0 ? fb : fa;
  const double rq = rint(fdepth);
  if (fabs(fdepth - rq) > 1e-9 || rq < 0 || rq > N - 1) {
    atomicOr(err, (unsigned)CS_ERR_DEPTH);
    idx[row] = out;
    return;
  }
  const double tr = rint(t);
  const bool snap = fabs(t - tr) < 1e-9 && tr >= 0 && tr <= N - 1;
  int start;
  if (snap) {
    start = (int)tr;
    wr[0] = 1.0;
  } else {
    start = (int)floor(t) - (p / 2 - 1);
    if (start < 0) start = 0;
    if (start > N - p) start = N - p;
    const double tau = t - start;
    for (int k = 0; k < p; ++k) {
      double acc = 1.0;
      for (int mm = 0; mm < p; ++mm)
        if (mm != k) acc *= (tau - mm) / (double)(k - mm);
      wr[k] = acc;
    }
  }
  if (start < 0 || start + (snap ? 1 : p) > N) atomicOr(err, (unsigned)CS_ERR_RANGE);
  // node 0 and step on Q (slot pointers address cell (-h, -h))
  const int cq0 = dq == 0 ? (int)rq : start;
  const int cq1 = dq == 0 ? start : (int)rq;
  const int64_t off = (int64_t)(cq0 + pan.h) * pan.s0[Q] + (int64_t)(cq1 + pan.h) * pan.s1[Q];
  const int64_t step = dq == 0 ? pan.s1[Q] : pan.s0[Q];
  out.x = pan.slot_base[Q];
  out.y = (int)off;
  out.z = (int)step;
  out.w = snap ? kFlagSnap : 0;
  idx[row] = out;
  if (pan.rotate) {
    V3 ea, eb, qa, qb;
    basis(P, a, b, ea, eb);
    basis(Q, aq, bq, qa, qb);
    const double g11 = dot(qa, qa), g12 = dot(qa, qb), g22 = dot(qb, qb);
    const double det = g11 * g22 - g12 * g12;
    const V3 da = scl(1.0 / det, sub(scl(g22, qa), scl(g12, qb)));
    const V3 db = scl(1.0 / det, sub(scl(g11, qb), scl(g12, qa)));
    mr[0] = dot(ea, da);
    mr[1] = dot(ea, db);
    mr[2] = dot(eb, da);
    mr[3] = dot(eb, db);
  }
}

}  // namespace

cudaError_t launch_cs_geometry(const CsPanels& pan, const int4* cells,
                               int ncells, int4* idx, double* w, double* m,
                               unsigned* err, cudaStream_t s) {
  if (ncells <= 0) return cudaSuccess;
  const int threads = 128;
  k_cs_geometry<<<(ncells + threads - 1) / threads, threads, 0, s>>>(
      pan, cells, ncells, idx, w, m, err);
  return cudaGetLastError();
}

}  // namespace bcg
