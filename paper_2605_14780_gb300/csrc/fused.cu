// Boundary conditions fused with the stencil that follows them (arxiv
// 2605.14780, Sec. IV-C: the boundary rows are only ever read by the next
// stencil, so they can be evaluated where that stencil reads them).  One
// launch over every slot computes
//
//   out[x] = sum_o c_o * f(x + o)   for every data value x,
//
// where f is the field as a forward apply leaves it: data values as stored,
// covered ghost values evaluated from their row of A and b at the point of
// use, uncovered ghost values as stored.  The same launch also writes every
// covered ghost value (f's ghosts), so the fields end as after bc_apply.
// Stencil threads never read covered ghost memory (they evaluate the row),
// so the ghost writes and the stencil reads do not race.
//
// Rows are the plan's level-0 rows of A in CSR form; each slot has a table
// that maps every cell of its ghost frame (the full region minus the data
// region, in slab order) to its row, or -1.  The stencil outputs go by
// tiles of 32 x 8 x 4 cells (x 1 for 2-D blocks) and one level: the CTA
// stages the tile and its halo in shared memory, evaluating each covered
// ghost of the halo once, and each thread sums the points for 4 cells
// along axis 2 from there.
#include <cstdint>

#include "bc_internal.h"

namespace bcg {
namespace {

__device__ __forceinline__ uint32_t fdivf(uint32_t n, const FastDiv& f) {
  return (__umulhi(n, f.m) + n) >> f.s;
}

template <typename T> struct FBits;
template <> struct FBits<float> { using type = uint32_t; };
template <> struct FBits<double> { using type = uint64_t; };

__device__ __forceinline__ uint32_t to_bits_f(float v) { return __float_as_uint(v); }
__device__ __forceinline__ uint64_t to_bits_f(double v) {
  return (uint64_t)__double_as_longlong(v);
}
template <typename T>
__device__ __forceinline__ T from_bits_f(typename FBits<T>::type b);
template <>
__device__ __forceinline__ float from_bits_f<float>(uint32_t b) { return __uint_as_float(b); }
template <>
__device__ __forceinline__ double from_bits_f<double>(uint64_t b) {
  return __longlong_as_double((long long)b);
}

// index of ghost cell (i, j, k) in the slot's frame table
__device__ __forceinline__ int64_t frame_index(const FuseSlot& S, int i, int j, int k) {
  const int64_t F0 = S.n[0] + 2 * S.h[0], F1 = S.n[1] + 2 * S.h[1];
  const int64_t slab = (int64_t)S.h[2] * F1 * F0;
  if (k < 0) return ((int64_t)(k + S.h[2]) * F1 + (j + S.h[1])) * F0 + (i + S.h[0]);
  if (k >= S.n[2]) return slab + ((int64_t)(k - S.n[2]) * F1 + (j + S.h[1])) * F0 + (i + S.h[0]);
  const int64_t plane = F1 * F0 - (int64_t)S.n[1] * S.n[0];
  const int64_t base = 2 * slab + (int64_t)k * plane;
  if (j < 0) return base + (int64_t)(j + S.h[1]) * F0 + (i + S.h[0]);
  if (j >= S.n[1]) return base + (int64_t)(S.h[1] + j - S.n[1]) * F0 + (i + S.h[0]);
  const int64_t b2 = base + 2 * (int64_t)S.h[1] * F0 + (int64_t)j * 2 * S.h[0];
  return i < 0 ? b2 + (i + S.h[0]) : b2 + S.h[0] + (i - S.n[0]);
}

// cell of frame entry f (the inverse of frame_index)
__device__ __forceinline__ void frame_cell(const FuseSlot& S, int64_t f, int& i, int& j, int& k) {
  const int64_t F0 = S.n[0] + 2 * S.h[0], F1 = S.n[1] + 2 * S.h[1];
  const int64_t slab = (int64_t)S.h[2] * F1 * F0;
  if (f < 2 * slab) {
    const bool top = f >= slab;
    const int64_t g = top ? f - slab : f;
    const int64_t kk = g / (F1 * F0), r = g - kk * F1 * F0;
    k = top ? S.n[2] + (int)kk : (int)kk - S.h[2];
    j = (int)(r / F0) - S.h[1];
    i = (int)(r % F0) - S.h[0];
    return;
  }
  const int64_t plane = F1 * F0 - (int64_t)S.n[1] * S.n[0];
  const int64_t g = f - 2 * slab;
  k = (int)(g / plane);
  int64_t r = g - (int64_t)k * plane;
  const int64_t band = (int64_t)S.h[1] * F0;
  if (r < 2 * band) {
    const bool top = r >= band;
    const int64_t rr = top ? r - band : r;
    j = top ? S.n[1] + (int)(rr / F0) : (int)(rr / F0) - S.h[1];
    i = (int)(rr % F0) - S.h[0];
    return;
  }
  r -= 2 * band;
  j = (int)(r / (2 * S.h[0]));
  const int t = (int)(r - (int64_t)j * 2 * S.h[0]);
  i = t < S.h[0] ? t - S.h[0] : S.n[0] + t - S.h[0];
}

__device__ __forceinline__ int64_t cell_off(const FuseSlot& S, int i, int j, int k) {
  return (int64_t)(i + S.h[0]) * S.s[0] + (int64_t)(j + S.h[1]) * S.s[1] +
         (int64_t)(k + S.h[2]) * S.s[2];
}

// row r of A at level l: bit pattern of a unit copy, else b_r + sum_e a_e x_e
template <typename T>
__device__ __forceinline__ T eval_row(const FuseCtx& F, void* const* slots, int r, int l,
                                      bool& copy, typename FBits<T>::type& bits) {
  using B = typename FBits<T>::type;
  const int e0 = __ldg(F.rptr + r), e1 = __ldg(F.rptr + r + 1);
  const T b = __ldg(static_cast<const T*>(F.rhs) + r);
  if (e1 - e0 == 1) {
    const T a = __ldg(static_cast<const T*>(F.val) + e0);
    if (a == T(1) && to_bits_f(b) == 0) {
      const int s = __ldg(F.eslot + e0);
      const B* x = static_cast<const B*>(slots[s]);
      bits = __ldg(x + (__ldg(F.eoff + e0) + (int64_t)l * __ldg(F.slot_ls + s)));
      copy = true;
      return from_bits_f<T>(bits);
    }
  }
  copy = false;
  T acc = b;
  for (int e = e0; e < e1; ++e) {
    const int s = __ldg(F.eslot + e);
    const T* x = static_cast<const T*>(slots[s]);
    acc = fma(__ldg(static_cast<const T*>(F.val) + e),
              __ldg(x + (__ldg(F.eoff + e) + (int64_t)l * __ldg(F.slot_ls + s))), acc);
  }
  return acc;
}

// f at cell (i, j, k) of slot S, level offset lo: a data value, a covered
// ghost evaluated from its row, or a stored (uncovered) ghost
template <typename T>
__device__ __forceinline__ T field_at(const FuseCtx& F, void* const* slots, const FuseSlot& S,
                                      const T* x, int i, int j, int k, int l, int64_t lo) {
  if (i >= 0 && i < S.n[0] && j >= 0 && j < S.n[1] && k >= 0 && k < S.n[2])
    return __ldg(x + (cell_off(S, i, j, k) + lo));
  const int r = __ldg(F.frame_row + S.fbase + frame_index(S, i, j, k));
  if (r < 0) return __ldg(x + (cell_off(S, i, j, k) + lo));
  bool copy;
  typename FBits<T>::type bits;
  return eval_row<T>(F, slots, r, l, copy, bits);
}

template <typename T>
__global__ void __launch_bounds__(kFuseThreads)
    k_fused(FuseCtx F, FuseStencil st, void* const* slots, void* const* outs) {
  using B = typename FBits<T>::type;
  __shared__ FuseSlot S;
  __shared__ int si;
  __shared__ T sm[kTileVals];
  __shared__ int dp[kFuseMaxPoints];
  __shared__ T cf[kFuseMaxPoints];
  const int tid = threadIdx.x;
  if (tid == 0) {
    // the slot of this CTA: the last slot whose first CTA is <= blockIdx.x
    int lo = 0, hi = F.nslots - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (F.slot[mid].cta0 <= (int64_t)blockIdx.x) lo = mid;
      else hi = mid - 1;
    }
    si = lo;
    S = F.slot[lo];
  }
  __syncthreads();
  const int64_t lc = (int64_t)blockIdx.x - S.cta0;
  const T* x = static_cast<const T*>(slots[si]);
  if (lc < S.tiles) {
    // stencil outputs of one tile at one level: stage the tile and its
    // halo (covered ghosts evaluated once each), then the sums
    int t = (int)lc;
    const int tx = t % S.nt[0];
    t /= S.nt[0];
    const int ty = t % S.nt[1];
    t /= S.nt[1];
    const int tzi = t % S.nt[2];
    const int l = t / S.nt[2];
    const int i0 = tx * kTileX, j0 = ty * kTileY, k0 = tzi * S.tz;
    const int SX = kTileX + 2 * st.r[0], SY = kTileY + 2 * st.r[1], SZ = S.tz + 2 * st.r[2];
    const int64_t lo = (int64_t)l * S.ls;
    for (int p = tid; p < st.n; p += kFuseThreads) {
      dp[p] = (st.o[p][2] * SY + st.o[p][1]) * SX + st.o[p][0];
      cf[p] = (T)st.c[p];
    }
    for (int e = tid; e < SX * SY * SZ; e += kFuseThreads) {
      const int li = e % SX, q = e / SX;
      const int lj = q % SY, lk = q / SY;
      const int i = i0 + li - st.r[0], j = j0 + lj - st.r[1], k = k0 + lk - st.r[2];
      const bool full = i >= -S.h[0] && i < S.n[0] + S.h[0] && j >= -S.h[1] &&
                        j < S.n[1] + S.h[1] && k >= -S.h[2] && k < S.n[2] + S.h[2];
      // cells past the full region only border outputs past the data region
      sm[e] = full ? field_at<T>(F, slots, S, x, i, j, k, l, lo) : T(0);
    }
    __syncthreads();
    const int ix = tid % kTileX, iy = tid / kTileX;
    const int i = i0 + ix, j = j0 + iy;
    if (i < S.n[0] && j < S.n[1]) {
      T* out = static_cast<T*>(outs[si]);
      for (int kz = 0; kz < S.tz; ++kz) {
        const int k = k0 + kz;
        if (k >= S.n[2]) break;
        const T* c = sm + ((kz + st.r[2]) * SY + (iy + st.r[1])) * SX + (ix + st.r[0]);
        T acc = T(0);
        for (int p = 0; p < st.n; ++p) acc = fma(cf[p], c[dp[p]], acc);
        out[cell_off(S, i, j, k) + lo] = acc;
      }
    }
    return;
  }
  // the ghost value at frame entry f, level l
  const int64_t w = (lc - S.tiles) * kFuseThreads + tid;
  if (w >= (int64_t)S.nf * S.L) return;
  B* xb = static_cast<B*>(slots[si]);
  int64_t f;
  int l;
  if (S.lfast) {
    f = (int64_t)fdivf((uint32_t)w, S.dL);
    l = (int)(w - f * S.L);
  } else {
    l = (int)fdivf((uint32_t)w, S.dnf);
    f = w - (int64_t)l * S.nf;
  }
  const int r = __ldg(F.frame_row + S.fbase + f);
  if (r < 0) return;
  int i, j, k;
  frame_cell(S, f, i, j, k);
  bool copy;
  B bits;
  const T val = eval_row<T>(F, slots, r, l, copy, bits);
  xb[cell_off(S, i, j, k) + (int64_t)l * S.ls] = copy ? bits : to_bits_f(val);
}

}  // namespace

cudaError_t launch_fused(int dtype, const FuseCtx& F, const FuseStencil& st, void* const* slots,
                         void* const* outs, int64_t nctas, cudaStream_t s) {
  if (nctas <= 0) return cudaSuccess;
  if (dtype == 1)
    k_fused<double><<<(unsigned)nctas, kFuseThreads, 0, s>>>(F, st, slots, outs);
  else
    k_fused<float><<<(unsigned)nctas, kFuseThreads, 0, s>>>(F, st, slots, outs);
  return cudaGetLastError();
}

}  // namespace bcg
