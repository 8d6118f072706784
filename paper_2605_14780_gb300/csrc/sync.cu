// Block-edge averaging (Sync rows, Sec. III-B) on sm_103a.
//
// Sync rows overwrite data cells that several blocks store for one physical
// location, and read data cells themselves, so one apply runs in two steps
// around the other kernels: the rows are evaluated into a plan-owned staging
// buffer while every row of the operator still reads the input values, and
// the staged values are written to the data cells afterwards.  The adjoint
// mirrors it: the rows' cotangents are moved to the staging buffer (their
// data cells' own cotangent is consumed), the ghost gather runs, then every
// column the rows read gathers its staged contributions.  Sync sets are
// small (the shared edges of the blocks): one thread per (row or column,
// level), levels fastest when they are contiguous in memory, rows fastest
// otherwise, so the accesses of a warp stay coalesced in both layouts.
#include <cstdint>

#include "bc_internal.h"

namespace bcg {
namespace {

constexpr int kSyncThreads = 256;

template <typename T>
__device__ __forceinline__ T* slot_at(void* const* slots, int slot, int off) {
  return static_cast<T*>(slots[slot]) + off;
}

// thread t -> (row or column u, level l): levels fastest when the levels are
// contiguous in memory, else rows fastest (consecutive cells of a box)
__device__ __forceinline__ void split(const SyncCtx& s, int n, int64_t t, int& u, int& l) {
  if (s.level_fast) {
    u = (int)(t / s.lmax);
    l = (int)(t - (int64_t)u * s.lmax);
  } else {
    l = (int)(t / n);
    u = (int)(t - (int64_t)l * n);
  }
}

template <typename T>
__global__ void __launch_bounds__(kSyncThreads) k_sync(SyncCtx s, int step, void* const* slots,
                                                      const int32_t* slot_ls) {
  const int64_t t = (int64_t)blockIdx.x * kSyncThreads + threadIdx.x;
  T* stage = static_cast<T*>(s.stage);
  if (step == SYNC_ADJOINT) {
    if (t >= (int64_t)s.ncols * s.lmax) return;
    int u, l;
    split(s, s.ncols, t, u, l);
    const int4 c = s.col[u];
    if (l >= c.z) return;
    T* xb = slot_at<T>(slots, c.x, c.y + l * __ldg(slot_ls + c.x));
    const T* w = static_cast<const T*>(s.cw);
    const int e0 = __ldg(s.cptr + u), e1 = __ldg(s.cptr + u + 1);
    T acc = *xb;
    for (int e = e0; e < e1; ++e) acc = fma(__ldg(w + e), stage[__ldg(s.cstage + e) + l], acc);
    *xb = acc;
    return;
  }
  if (t >= (int64_t)s.nrows * s.lmax) return;
  int u, l;
  split(s, s.nrows, t, u, l);
  const int4 r = s.row[u];
  if (l >= r.w) return;
  T* d = slot_at<T>(slots, r.x, r.y + l * __ldg(slot_ls + r.x));
  if (step == SYNC_ROWS) {
    const T* w = static_cast<const T*>(s.w);
    const int e0 = __ldg(s.ptr + u), e1 = __ldg(s.ptr + u + 1);
    T acc = T(0);
    for (int e = e0; e < e1; ++e) {
      const int2 en = s.ent[e];
      acc = fma(__ldg(w + e), *slot_at<T>(slots, en.x, en.y + l * __ldg(slot_ls + en.x)), acc);
    }
    stage[r.z + l] = acc;
  } else if (step == SYNC_COMMIT) {
    *d = stage[r.z + l];
  } else {  // SYNC_SNAPSHOT
    stage[r.z + l] = *d;
    *d = T(0);
  }
}

}  // namespace

cudaError_t launch_sync(int dtype, int step, const SyncCtx& s, void* const* slots,
                        const int32_t* slot_ls, cudaStream_t stream) {
  const int64_t n = (int64_t)(step == SYNC_ADJOINT ? s.ncols : s.nrows) * s.lmax;
  if (n <= 0) return cudaSuccess;
  const int grid = (int)((n + kSyncThreads - 1) / kSyncThreads);
  if (dtype == 1)
    k_sync<double><<<grid, kSyncThreads, 0, stream>>>(s, step, slots, slot_ls);
  else
    k_sync<float><<<grid, kSyncThreads, 0, stream>>>(s, step, slots, slot_ls);
  return cudaGetLastError();
}

}  // namespace bcg
