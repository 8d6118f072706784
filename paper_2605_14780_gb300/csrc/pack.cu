// Packing of block boxes into one contiguous buffer, for the exchange of
// ghost sources between processes that own different blocks (arxiv
// 2605.14780, Sec. V-B: each process receives the bounding box of the
// remote data its boundary rows read).  A box is a cell range of one block,
// taken with every component and level; in the buffer it is stored
// [component][level][k][j][i], boxes back to back.  One thread per value;
// the box of a CTA's first value is found by binary search and CTAs never
// straddle boxes.
#include <cstdint>

#include "bc_internal.h"

namespace bcg {
namespace {

__device__ __forceinline__ uint32_t pdiv(uint32_t n, const FastDiv& f) {
  return (__umulhi(n, f.m) + n) >> f.s;
}

template <typename B>
__global__ void __launch_bounds__(kPackThreads)
    k_pack(const PackBox* __restrict__ boxes, int nboxes, void* const* slots, B* buf) {
  __shared__ PackBox bx;
  if (threadIdx.x == 0) {
    int lo = 0, hi = nboxes - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (boxes[mid].cta0 <= (int64_t)blockIdx.x) lo = mid;
      else hi = mid - 1;
    }
    bx = boxes[lo];
  }
  __syncthreads();
  const int64_t v = ((int64_t)blockIdx.x - bx.cta0) * kPackThreads + threadIdx.x;
  if (v >= bx.count) return;
  // v -> (component, level, k, j, i), i fastest
  const uint32_t vv = (uint32_t)v;
  const uint32_t row = pdiv(vv, bx.d0);
  const int i = (int)(vv - row * (uint32_t)bx.e[0]);
  const uint32_t pl = pdiv(row, bx.d1);
  const int j = (int)(row - pl * (uint32_t)bx.e[1]);
  const uint32_t cl = pdiv(pl, bx.d2);
  const int k = (int)(pl - cl * (uint32_t)bx.e[2]);
  const uint32_t c = pdiv(cl, bx.dL);
  const int l = (int)(cl - c * (uint32_t)bx.L);
  const B* src = static_cast<const B*>(slots[bx.slot0 + (int)c]);
  const int64_t off = (int64_t)(bx.lo[0] + i) * bx.s[0] + (int64_t)(bx.lo[1] + j) * bx.s[1] +
                      (int64_t)(bx.lo[2] + k) * bx.s[2] + (int64_t)l * bx.ls;
  buf[bx.dst + v] = __ldg(src + off);
}

}  // namespace

cudaError_t launch_pack(int esize, const PackBox* boxes, int nboxes, int64_t nctas,
                        void* const* slots, void* buf, cudaStream_t s) {
  if (nctas <= 0 || nboxes <= 0) return cudaSuccess;
  if (esize == 8)
    k_pack<uint64_t><<<(unsigned)nctas, kPackThreads, 0, s>>>(boxes, nboxes, slots,
                                                               static_cast<uint64_t*>(buf));
  else
    k_pack<uint32_t><<<(unsigned)nctas, kPackThreads, 0, s>>>(boxes, nboxes, slots,
                                                               static_cast<uint32_t*>(buf));
  return cudaGetLastError();
}

}  // namespace bcg
