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
#include <cstdio>
#include <mutex>

#include "../../include/bc.h"
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

// The stencil of one edge ghost (i, j) of panel P (one coordinate out of
// range): the neighbour panel Q that owns the ghost's grid point, the axis dq
// of Q normal to the shared edge, the data row rq of Q the point lies on, the
// first node `start` along Q's other axis with the p Lagrange weights (or a
// unit copy of node `start` when grid lines align: snap), and, with
// `rotate`, the 2x2 basis change M.  Returns CsError bits (0: all found).
struct EdgeStencil {
  int Q, dq, rq, start, snap;
  double w[kPMax];
  double m[4];
};

__device__ unsigned edge_stencil(int P, int i, int j, int N, int p, bool rotate,
                                 EdgeStencil& o) {
  const double pi = 3.14159265358979323846;
  const double delta = pi / (2.0 * N);
  for (int n = 0; n < kPMax; ++n) o.w[n] = 0.0;
  o.m[0] = 1.0; o.m[1] = 0.0; o.m[2] = 0.0; o.m[3] = 1.0;
  o.Q = -1; o.dq = 0; o.rq = 0; o.start = 0; o.snap = 0;
  const bool io = (i < 0 || i >= N), jo = (j < 0 || j >= N);
  if (io == jo) return CS_ERR_NOT_EDGE;
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
  if (Q != Qr || Q == P) return CS_ERR_NEIGHBOUR;
  double aq, bq;
  angles_on(Q, v, aq, bq);
  const double fa = (aq + pi / 4) / delta - 0.5;
  const double fb = (bq + pi / 4) / delta - 0.5;
  const double fdepth = dq == 0 ? fa : fb;
  const double t = dq == 0 ? fb : fa;
  const double rq = rint(fdepth);
  if (fabs(fdepth - rq) > 1e-9 || rq < 0 || rq > N - 1) return CS_ERR_DEPTH;
  const double tr = rint(t);
  const bool snap = fabs(t - tr) < 1e-9 && tr >= 0 && tr <= N - 1;
  int start;
  if (snap) {
    start = (int)tr;
    o.w[0] = 1.0;
  } else {
    start = (int)floor(t) - (p / 2 - 1);
    if (start < 0) start = 0;
    if (start > N - p) start = N - p;
    const double tau = t - start;
    for (int k = 0; k < p; ++k) {
      double acc = 1.0;
      for (int mm = 0; mm < p; ++mm)
        if (mm != k) acc *= (tau - mm) / (double)(k - mm);
      o.w[k] = acc;
    }
  }
  o.Q = Q;
  o.dq = dq;
  o.rq = (int)rq;
  o.start = start;
  o.snap = snap ? 1 : 0;
  if (rotate) {
    V3 ea, eb, qa, qb;
    basis(P, a, b, ea, eb);
    basis(Q, aq, bq, qa, qb);
    const double g11 = dot(qa, qa), g12 = dot(qa, qb), g22 = dot(qb, qb);
    const double det = g11 * g22 - g12 * g12;
    const V3 da = scl(1.0 / det, sub(scl(g22, qa), scl(g12, qb)));
    const V3 db = scl(1.0 / det, sub(scl(g11, qb), scl(g12, qa)));
    o.m[0] = dot(ea, da);
    o.m[1] = dot(ea, db);
    o.m[2] = dot(eb, da);
    o.m[3] = dot(eb, db);
  }
  return (start < 0 || start + (snap ? 1 : p) > N) ? (unsigned)CS_ERR_RANGE : 0u;
}

__global__ void k_cs_geometry(CsPanels pan, const int4* __restrict__ cells,
                              int ncells, int4* idx, double* w, double* m,
                              unsigned* err) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= ncells) return;
  const int4 cell = cells[g];
  const int row = cell.w;
  EdgeStencil o;
  const unsigned e = edge_stencil(cell.x, cell.y, cell.z, pan.N, pan.p, pan.rotate != 0, o);
  double* wr = w + (int64_t)row * kPMax;
  double* mr = m + (int64_t)row * 4;
  for (int n = 0; n < kPMax; ++n) wr[n] = o.w[n];
  for (int n = 0; n < 4; ++n) mr[n] = o.m[n];
  if (e) atomicOr(err, e);
  if (o.Q < 0) {
    idx[row] = make_int4(0, 0, 0, 0);
    return;
  }
  // node 0 and step on Q (slot pointers address cell (-h, -h))
  const int cq0 = o.dq == 0 ? o.rq : o.start;
  const int cq1 = o.dq == 0 ? o.start : o.rq;
  const int64_t off =
      (int64_t)(cq0 + pan.h) * pan.s0[o.Q] + (int64_t)(cq1 + pan.h) * pan.s1[o.Q];
  const int64_t step = o.dq == 0 ? pan.s1[o.Q] : pan.s0[o.Q];
  idx[row] = make_int4(pan.slot_base[o.Q], (int)off, (int)step, o.snap ? kFlagSnap : 0);
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

// ---------------------------------------------------------------------------
// Allocation-free variant of the geometry kernel (bc_cubed_sphere_stencils_
// noalloc): the per-cell results and the error word go to one fixed device
// array instead of buffers the plan allocates.  Layout of the array:
//   [0, 256)                 error word (cleared by every call)
//   then, for kNoAllocMax cells: int4 {nb, i0, j0, axis | snap}
//   then FP64 weights [cell][kPMax], then FP64 rotations [cell][4].
// ---------------------------------------------------------------------------
namespace {

constexpr int kNoAllocMax = BC_NOALLOC_MAX_CELLS;
constexpr size_t kNoAllocIdx = 256;
constexpr size_t kNoAllocW = kNoAllocIdx + sizeof(int4) * (size_t)kNoAllocMax;
constexpr size_t kNoAllocM = kNoAllocW + sizeof(double) * kPMax * (size_t)kNoAllocMax;
constexpr size_t kNoAllocBytes = kNoAllocM + sizeof(double) * 4 * (size_t)kNoAllocMax;

// In host code this name is only a stand-in for the device symbol: host code
// passes the address cudaGetSymbolAddress returns for the current device.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

__global__ void k_cs_stencils_noalloc(int N, int h, int p, int rotate,
                                      unsigned char* scratch) {
  const int ncells = 24 * N * h;
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= ncells) return;
  unsigned* err = reinterpret_cast<unsigned*>(scratch);
  int4* idx = reinterpret_cast<int4*>(scratch + kNoAllocIdx);
  double* wr = reinterpret_cast<double*>(scratch + kNoAllocW) + (int64_t)g * kPMax;
  double* mr = reinterpret_cast<double*>(scratch + kNoAllocM) + (int64_t)g * 4;
  // canonical cell order: panel, strip (d, side), depth r, along s
  const int s = g % N;
  const int r = (g / N) % h;
  const int strip = (g / (N * h)) % 4;
  const int P = g / (4 * N * h);
  const int d = strip >> 1, side = strip & 1;
  const int gi = side ? N + r : -1 - r;
  EdgeStencil o;
  const unsigned e = edge_stencil(P, d == 0 ? gi : s, d == 0 ? s : gi, N, p, rotate != 0, o);
  for (int n = 0; n < kPMax; ++n) wr[n] = o.w[n];
  for (int n = 0; n < 4; ++n) mr[n] = o.m[n];
  if (e) atomicOr(err, e);
  idx[g] = o.Q < 0 ? make_int4(-1, 0, 0, 0)
                   : make_int4(o.Q, o.dq == 0 ? o.rq : o.start, o.dq == 0 ? o.start : o.rq,
                               (1 - o.dq) | (o.snap ? BC_NOALLOC_SNAP : 0));
}

std::mutex g_noalloc_mu;
void* g_noalloc_ptr[256] = {nullptr};  // device address of the array, per device

bc_status noalloc_fail(bc_status st, const char* msg) {
  set_last_error(msg);
  return st;
}

bc_status noalloc_cuda(cudaError_t e, const char* what) {
  char buf[256];
  snprintf(buf, sizeof(buf), "%s: %s", what, cudaGetErrorString(e));
  return noalloc_fail(BC_ERR_CUDA, buf);
}

}  // namespace
}  // namespace bcg

extern "C" bc_status bc_cubed_sphere_stencils_noalloc(int32_t N, int32_t h, int32_t p,
                                                      int32_t* nb, int32_t* node0,
                                                      int32_t* axis, double* w,
                                                      double* rot) {
  using namespace bcg;
  set_last_error("");
  if (p < 1 || p > kPMax) return noalloc_fail(BC_ERR_INVALID_ARG, "p must be in 1..8");
  if (h < 1 || N < p || h > N) return noalloc_fail(BC_ERR_INVALID_ARG, "need 1 <= h <= N and N >= p");
  if (!nb || !node0 || !axis || !w) return noalloc_fail(BC_ERR_INVALID_ARG, "NULL output array");
  if ((int64_t)24 * N * h > BC_NOALLOC_MAX_CELLS) {
    char buf[200];
    snprintf(buf, sizeof(buf), "24*N*h = %lld edge ghosts exceed the fixed scratch of %d cells",
             (long long)24 * N * h, BC_NOALLOC_MAX_CELLS);
    return noalloc_fail(BC_ERR_UNSUPPORTED, buf);
  }
  const int ncells = 24 * N * h;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return noalloc_cuda(e, "cudaGetDevice");
  if (dev < 0 || dev >= 256) return noalloc_fail(BC_ERR_UNSUPPORTED, "device index out of range");
  unsigned char* scratch = nullptr;
  {
    // set-up once per device, with that device current
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
      void* ptr = nullptr;
      e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
      if (e != cudaSuccess || !ptr) return noalloc_cuda(e, "cudaGetSymbolAddress of the scratch array");
      g_noalloc_ptr[dev] = ptr;
    }
    scratch = static_cast<unsigned char*>(g_noalloc_ptr[dev]);
  }
  // the error word must start at zero; results are fully rewritten
  if ((e = cudaMemset(scratch, 0, sizeof(unsigned))) != cudaSuccess)
    return noalloc_cuda(e, "clearing the error word");
  const int threads = 128;
  k_cs_stencils_noalloc<<<(ncells + threads - 1) / threads, threads>>>(N, h, p, rot ? 1 : 0, scratch);
  if ((e = cudaGetLastError()) != cudaSuccess) return noalloc_cuda(e, "stencil kernel launch");
  unsigned herr = 0;
  if ((e = cudaMemcpy(&herr, scratch, sizeof(unsigned), cudaMemcpyDeviceToHost)) != cudaSuccess)
    return noalloc_cuda(e, "stencil kernel");
  if (herr) return noalloc_fail(BC_ERR_GEOMETRY, "cubed sphere: neighbour or depth-row check failed");
  // scatter the int4 rows into the caller's arrays with strided copies
  const unsigned char* ix = scratch + kNoAllocIdx;
  if ((e = cudaMemcpy2D(nb, sizeof(int32_t), ix, sizeof(int4), sizeof(int32_t), ncells,
                        cudaMemcpyDeviceToHost)) != cudaSuccess ||
      (e = cudaMemcpy2D(node0, 2 * sizeof(int32_t), ix + sizeof(int32_t), sizeof(int4),
                        2 * sizeof(int32_t), ncells, cudaMemcpyDeviceToHost)) != cudaSuccess ||
      (e = cudaMemcpy2D(axis, sizeof(int32_t), ix + 3 * sizeof(int32_t), sizeof(int4),
                        sizeof(int32_t), ncells, cudaMemcpyDeviceToHost)) != cudaSuccess ||
      (e = cudaMemcpy2D(w, p * sizeof(double), scratch + kNoAllocW, kPMax * sizeof(double),
                        p * sizeof(double), ncells, cudaMemcpyDeviceToHost)) != cudaSuccess)
    return noalloc_cuda(e, "copying the stencils to the host");
  if (rot && (e = cudaMemcpy(rot, scratch + kNoAllocM, (size_t)ncells * 4 * sizeof(double),
                             cudaMemcpyDeviceToHost)) != cudaSuccess)
    return noalloc_cuda(e, "copying the rotations to the host");
  return BC_OK;
}
