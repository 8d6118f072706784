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
// small (the shared edges of the blocks): one warp per row or column, lanes
// over the levels.
#include <cstdint>

#include "bc_internal.h"

namespace bcg {
namespace {

constexpr int kSyncThreads = 128;

template <typename T>
__device__ __forceinline__ T* slot_at(void* const* slots, int slot, int off) {
  return static_cast<T*>(slots[slot]) + off;
}

template <typename T>
__global__ void __launch_bounds__(kSyncThreads) k_sync(SyncCtx s, int step, void* const* slots,
                                                      const int32_t* slot_ls) {
  const int warp = (blockIdx.x * kSyncThreads + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  T* stage = static_cast<T*>(s.stage);
  if (step == SYNC_ADJOINT) {
    if (warp >= s.ncols) return;
    const int4 c = s.col[warp];
    const int ls = __ldg(slot_ls + c.x);
    T* xb = slot_at<T>(slots, c.x, c.y);
    const T* w = static_cast<const T*>(s.cw);
    const int e0 = __ldg(s.cptr + warp), e1 = __ldg(s.cptr + warp + 1);
    for (int l = lane; l < c.z; l += 32) {
      T acc = xb[l * ls];
      for (int e = e0; e < e1; ++e) acc = fma(__ldg(w + e), stage[__ldg(s.cstage + e) + l], acc);
      xb[l * ls] = acc;
    }
    return;
  }
  if (warp >= s.nrows) return;
  const int4 r = s.row[warp];
  const int ls = __ldg(slot_ls + r.x);
  T* d = slot_at<T>(slots, r.x, r.y);
  if (step == SYNC_ROWS) {
    const T* w = static_cast<const T*>(s.w);
    const int e0 = __ldg(s.ptr + warp), e1 = __ldg(s.ptr + warp + 1);
    for (int l = lane; l < r.w; l += 32) {
      T acc = T(0);
      for (int e = e0; e < e1; ++e) {
        const int2 en = s.ent[e];
        acc = fma(__ldg(w + e), slot_at<T>(slots, en.x, en.y)[l * __ldg(slot_ls + en.x)], acc);
      }
      stage[r.z + l] = acc;
    }
  } else if (step == SYNC_COMMIT) {
    for (int l = lane; l < r.w; l += 32) d[l * ls] = stage[r.z + l];
  } else {  // SYNC_SNAPSHOT
    for (int l = lane; l < r.w; l += 32) {
      stage[r.z + l] = d[l * ls];
      d[l * ls] = T(0);
    }
  }
}

}  // namespace

cudaError_t launch_sync(int dtype, int step, const SyncCtx& s, void* const* slots,
                        const int32_t* slot_ls, cudaStream_t stream) {
  const int n = step == SYNC_ADJOINT ? s.ncols : s.nrows;
  if (n <= 0) return cudaSuccess;
  const int warps = kSyncThreads / 32;
  const int grid = (n + warps - 1) / warps;
  if (dtype == 1)
    k_sync<double><<<grid, kSyncThreads, 0, stream>>>(s, step, slots, slot_ls);
  else
    k_sync<float><<<grid, kSyncThreads, 0, stream>>>(s, step, slots, slot_ls);
  return cudaGetLastError();
}

}  // namespace bcg
