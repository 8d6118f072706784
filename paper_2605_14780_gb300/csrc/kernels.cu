// sm_103a kernels of the ghost-fill operator y_G = A x_D + b
// (arxiv 2605.14780, Sec. III-B) and of its adjoint.
//
// Every launch works on a list of work items (bc_internal.h).  One CTA
// processes one item at a time: either as a plain grid (one CTA per item,
// used by the per-sub-matrix and per-kind forms and by the batched form) or
// as a persistent grid whose CTAs claim items from an atomic counter.
//
// The path is a sparse gather/scatter bounded by HBM bandwidth, so it runs on
// the CUDA cores: coalesced strips along axis 0, several independent levels
// (or flat values) in flight per thread, copies done on integer bit patterns
// so they are exact, and table rows (stencils, CSR entries) loaded once per
// cell and reused for every level of that cell.
#include <cstdint>

#include "bc_internal.h"

namespace bcg {
namespace {

template <typename T> struct BitsOf;
template <> struct BitsOf<float> { using type = uint32_t; };
template <> struct BitsOf<double> { using type = uint64_t; };

template <typename T>
__device__ __forceinline__ T ldg(const T* p) { return __ldg(p); }

__device__ __forceinline__ void cell_of(int q, int W0, int W1, int& i, int& j,
                                        int& k) {
  i = q % W0;
  int r = q / W0;
  j = r % W1;
  k = r / W1;
}

__device__ __forceinline__ int64_t dst_offset(const Item& it, int i, int j,
                                              int k) {
  return it.dst_org + i * it.dst_s0 + j * it.dst_s1 + k * it.dst_s2;
}

// ---------------------------------------------------------------------------
// zero / constant / map (matrix-free rows, Sec. III-B)
// ---------------------------------------------------------------------------
template <typename T>
__device__ void structured_cell(const Item& it, const Ctx& c) {
  using B = typename BitsOf<T>::type;
  const int t = threadIdx.x;
  if (t >= it.ncell) return;
  const int q = it.q0 + t;
  int i, j, k;
  cell_of(q, it.W0, it.W1, i, j, k);
  B* dst = static_cast<B*>(c.slots[it.dst_slot]) + dst_offset(it, i, j, k);
  const int64_t ls = it.dst_ls;
  const int l1 = it.l0 + it.nlev;
  if (it.kind == IK_ZERO) {
    for (int l = it.l0; l < l1; ++l) dst[l * ls] = B(0);
  } else if (it.kind == IK_CONST) {
    const B v = ldg(static_cast<const B*>(c.const_val) + it.table + q);
    for (int l = it.l0; l < l1; ++l) dst[l * ls] = v;
  } else {
    const B* src = static_cast<const B*>(c.slots[it.src_slot]) + it.src_org +
                   i * it.src_s0 + j * it.src_s1 + k * it.src_s2;
    const int64_t sls = it.src_ls;
    for (int l = it.l0; l < l1; l += kLevelUnroll) {
      B v[kLevelUnroll];
#pragma unroll
      for (int u = 0; u < kLevelUnroll; ++u)
        if (l + u < l1) v[u] = ldg(src + (l + u) * sls);
#pragma unroll
      for (int u = 0; u < kLevelUnroll; ++u)
        if (l + u < l1) dst[(l + u) * ls] = v[u];
    }
  }
}

template <typename T>
__device__ void structured_flat(const Item& it, const Ctx& c) {
  using B = typename BitsOf<T>::type;
  const int end = it.q0 + it.ncell;
  B* dbase = static_cast<B*>(c.slots[it.dst_slot]);
  const B* sbase = it.kind == IK_MAP
                       ? static_cast<const B*>(c.slots[it.src_slot])
                       : nullptr;
  const B* cval = static_cast<const B*>(c.const_val);
  int64_t doff[kFlatUnroll];
  B v[kFlatUnroll];
#pragma unroll
  for (int u = 0; u < kFlatUnroll; ++u) {
    const int f = it.q0 + threadIdx.x + u * blockDim.x;
    doff[u] = -1;
    if (f < end) {
      const int q = f % it.vol;
      const int l = it.l0 + f / it.vol;
      int i, j, k;
      cell_of(q, it.W0, it.W1, i, j, k);
      doff[u] = dst_offset(it, i, j, k) + l * it.dst_ls;
      if (it.kind == IK_MAP) {
        v[u] = ldg(sbase + it.src_org + i * it.src_s0 + j * it.src_s1 +
                   k * it.src_s2 + l * it.src_ls);
      } else if (it.kind == IK_CONST) {
        v[u] = ldg(cval + it.table + q);
      } else {
        v[u] = B(0);
      }
    }
  }
#pragma unroll
  for (int u = 0; u < kFlatUnroll; ++u)
    if (doff[u] >= 0) dbase[doff[u]] = v[u];
}

// ---------------------------------------------------------------------------
// interpolation rows (user Itp, Sec. III-B) with optional 2x2 rotation of a
// covariant component pair (Sec. V-A): y = M (sum_k w_k x_u, sum_k w_k x_v)
// ---------------------------------------------------------------------------
template <typename T, bool PAIR>
__device__ void interp_cell(const Item& it, const Ctx& c) {
  using B = typename BitsOf<T>::type;
  const int t = threadIdx.x;
  if (t >= it.ncell) return;
  const int q = it.q0 + t;
  const int row = it.table + q;
  int i, j, k;
  cell_of(q, it.W0, it.W1, i, j, k);
  const int64_t doff = dst_offset(it, i, j, k);
  const int64_t ls = it.dst_ls;
  const int4 ix = __ldg(c.itp_idx + row);
  const int su = ix.x + it.comp;
  const T* xu = static_cast<const T*>(c.slots[su]) + ix.y;
  const int64_t sls = __ldg(c.slot_ls + su);
  const int64_t step = ix.z;
  const int p = it.p;
  const int l1 = it.l0 + it.nlev;
  if (!PAIR) {
    T* dst = static_cast<T*>(c.slots[it.dst_slot]) + doff;
    if (ix.w & kFlagSnap) {  // unit row: exact copy of node 0
      const B* s = reinterpret_cast<const B*>(xu);
      B* d = reinterpret_cast<B*>(dst);
      for (int l = it.l0; l < l1; l += kLevelUnroll) {
        B v[kLevelUnroll];
#pragma unroll
        for (int u = 0; u < kLevelUnroll; ++u)
          if (l + u < l1) v[u] = ldg(s + (l + u) * sls);
#pragma unroll
        for (int u = 0; u < kLevelUnroll; ++u)
          if (l + u < l1) d[(l + u) * ls] = v[u];
      }
      return;
    }
    T w[kPMax];
    const T* wr = static_cast<const T*>(c.itp_w) + (int64_t)row * kPMax;
#pragma unroll
    for (int n = 0; n < kPMax; ++n) w[n] = n < p ? ldg(wr + n) : T(0);
    for (int l = it.l0; l < l1; l += kLevelUnroll) {
      T acc[kLevelUnroll];
#pragma unroll
      for (int u = 0; u < kLevelUnroll; ++u) acc[u] = T(0);
#pragma unroll
      for (int n = 0; n < kPMax; ++n) {
        if (n < p) {
#pragma unroll
          for (int u = 0; u < kLevelUnroll; ++u)
            if (l + u < l1)
              acc[u] = fma(w[n], ldg(xu + n * step + (l + u) * sls), acc[u]);
        }
      }
#pragma unroll
      for (int u = 0; u < kLevelUnroll; ++u)
        if (l + u < l1) dst[(l + u) * ls] = acc[u];
    }
  } else {
    constexpr int LU = kLevelUnroll / 2;
    const int sv = ix.x + it.comp2;
    const T* xv = static_cast<const T*>(c.slots[sv]) + ix.y;
    const int64_t slsv = __ldg(c.slot_ls + sv);
    T* du = static_cast<T*>(c.slots[it.dst_slot]) + doff;
    T* dv = static_cast<T*>(c.slots[it.dst_slot2]) + doff;
    const T* mr = static_cast<const T*>(c.itp_m) + (int64_t)row * 4;
    const T m00 = ldg(mr), m01 = ldg(mr + 1), m10 = ldg(mr + 2),
            m11 = ldg(mr + 3);
    T w[kPMax];
    const bool snap = ix.w & kFlagSnap;
    const T* wr = static_cast<const T*>(c.itp_w) + (int64_t)row * kPMax;
#pragma unroll
    for (int n = 0; n < kPMax; ++n) w[n] = n < p ? ldg(wr + n) : T(0);
    const int pe = snap ? 1 : p;
    for (int l = it.l0; l < l1; l += LU) {
      T au[LU], av[LU];
#pragma unroll
      for (int u = 0; u < LU; ++u) au[u] = av[u] = T(0);
      if (snap) {
#pragma unroll
        for (int u = 0; u < LU; ++u)
          if (l + u < l1) {
            au[u] = ldg(xu + (l + u) * sls);
            av[u] = ldg(xv + (l + u) * slsv);
          }
      } else {
#pragma unroll
        for (int n = 0; n < kPMax; ++n) {
          if (n < pe) {
#pragma unroll
            for (int u = 0; u < LU; ++u)
              if (l + u < l1) {
                au[u] = fma(w[n], ldg(xu + n * step + (l + u) * sls), au[u]);
                av[u] = fma(w[n], ldg(xv + n * step + (l + u) * slsv), av[u]);
              }
          }
        }
      }
#pragma unroll
      for (int u = 0; u < LU; ++u)
        if (l + u < l1) {
          du[(l + u) * ls] = fma(m00, au[u], m01 * av[u]);
          dv[(l + u) * ls] = fma(m10, au[u], m11 * av[u]);
        }
    }
  }
}

// ---------------------------------------------------------------------------
// user CSR rows (Table III: F_NNZ / F_COL / F_DATA), one row per thread; the
// row's entries are loaded once per level chunk and reused for every level
// ---------------------------------------------------------------------------
template <typename T>
__device__ void csr_cell(const Item& it, const Ctx& c) {
  const int t = threadIdx.x;
  if (t >= it.ncell) return;
  const int q = it.q0 + t;
  const int row = it.table + q;
  int i, j, k;
  cell_of(q, it.W0, it.W1, i, j, k);
  T* dst = static_cast<T*>(c.slots[it.dst_slot]) + dst_offset(it, i, j, k);
  const int64_t ls = it.dst_ls;
  const int64_t e0 = __ldg(c.csr_ptr + row), e1 = __ldg(c.csr_ptr + row + 1);
  const T rhs = ldg(static_cast<const T*>(c.csr_rhs) + row);
  const T* val = static_cast<const T*>(c.csr_val);
  const int l1 = it.l0 + it.nlev;
  for (int l = it.l0; l < l1; l += kLevelUnroll) {
    T acc[kLevelUnroll];
#pragma unroll
    for (int u = 0; u < kLevelUnroll; ++u) acc[u] = T(0);
    for (int64_t e = e0; e < e1; ++e) {
      const int s = __ldg(c.csr_slot + e);
      const T a = ldg(val + e);
      const T* x = static_cast<const T*>(c.slots[s]) + __ldg(c.csr_off + e);
      const int64_t sls = __ldg(c.slot_ls + s);
#pragma unroll
      for (int u = 0; u < kLevelUnroll; ++u)
        if (l + u < l1) acc[u] = fma(a, ldg(x + (l + u) * sls), acc[u]);
    }
#pragma unroll
    for (int u = 0; u < kLevelUnroll; ++u)
      if (l + u < l1) dst[(l + u) * ls] = acc[u] + rhs;
  }
}

// ---------------------------------------------------------------------------
// adjoint gather: x_bar_j += sum_i A_ij y_bar_i over the stored transpose,
// entries in ascending ghost order (deterministic, no atomics)
// ---------------------------------------------------------------------------
template <typename T>
__device__ void adj_cell(const Item& it, const Ctx& c) {
  const int t = threadIdx.x;
  if (t >= it.ncell) return;
  const int r = it.q0 + t;
  const int slot = __ldg(c.arow_slot + r);
  T* xb = static_cast<T*>(c.slots[slot]) + __ldg(c.arow_off + r);
  const int64_t ls = __ldg(c.slot_ls + slot);
  const int64_t e0 = __ldg(c.adj_ptr + r), e1 = __ldg(c.adj_ptr + r + 1);
  const T* wv = static_cast<const T*>(c.aent_w);
  const int l1 = it.l0 + it.nlev;
  for (int l = it.l0; l < l1; l += kLevelUnroll) {
    T acc[kLevelUnroll];
#pragma unroll
    for (int u = 0; u < kLevelUnroll; ++u)
      acc[u] = (l + u < l1) ? xb[(l + u) * ls] : T(0);
    for (int64_t e = e0; e < e1; ++e) {
      const int gs = __ldg(c.aent_slot + e);
      const T a = ldg(wv + e);
      const T* y = static_cast<const T*>(c.slots[gs]) + __ldg(c.aent_off + e);
      const int64_t gls = __ldg(c.slot_ls + gs);
#pragma unroll
      for (int u = 0; u < kLevelUnroll; ++u)
        if (l + u < l1) acc[u] = fma(a, y[(l + u) * gls], acc[u]);
    }
#pragma unroll
    for (int u = 0; u < kLevelUnroll; ++u)
      if (l + u < l1) xb[(l + u) * ls] = acc[u];
  }
}

template <typename T>
__device__ __forceinline__ void run_item(const Item& it, const Ctx& c) {
  switch (it.kind) {
    case IK_ZERO:
    case IK_CONST:
    case IK_MAP:
      if (it.mode == MODE_FLAT)
        structured_flat<T>(it, c);
      else
        structured_cell<T>(it, c);
      break;
    case IK_INTERP:
      interp_cell<T, false>(it, c);
      break;
    case IK_INTERP_PAIR:
      interp_cell<T, true>(it, c);
      break;
    case IK_CSR:
      csr_cell<T>(it, c);
      break;
    case IK_ADJ:
      adj_cell<T>(it, c);
      break;
    default:
      break;
  }
}

__device__ __forceinline__ void load_item(Item* dst, const Item* src) {
  const int* s = reinterpret_cast<const int*>(src);
  int* d = reinterpret_cast<int*>(dst);
  if (threadIdx.x < kItemWords) d[threadIdx.x] = __ldg(s + threadIdx.x);
}

template <typename T, int THREADS>
__global__ void __launch_bounds__(THREADS)
    k_items(Ctx c, const Item* __restrict__ items, int nitems) {
  __shared__ Item sit;
  if (blockIdx.x >= nitems) return;
  load_item(&sit, items + blockIdx.x);
  __syncthreads();
  run_item<T>(sit, c);
}

// Persistent form: CTAs claim items from counter[0]; the last CTA to finish
// resets both counters for the next launch (no CTA ever waits on another).
template <typename T, int THREADS>
__global__ void __launch_bounds__(THREADS)
    k_persistent(Ctx c, const Item* __restrict__ items, int nitems,
                 unsigned* counter) {
  __shared__ Item sit;
  __shared__ int s_idx;
  for (;;) {
    if (threadIdx.x == 0) s_idx = (int)atomicAdd(counter, 1u);
    __syncthreads();
    const int idx = s_idx;
    if (idx >= nitems) break;
    load_item(&sit, items + idx);
    __syncthreads();
    run_item<T>(sit, c);
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned done = atomicAdd(counter + 1, 1u);
    if (done == gridDim.x - 1) {
      atomicExch(counter, 0u);
      atomicExch(counter + 1, 0u);
      __threadfence();
    }
  }
}

template <typename T>
cudaError_t launch_items_t(const Ctx& c, const Item* items, int nitems,
                           int threads, cudaStream_t s) {
  if (nitems <= 0) return cudaSuccess;
  switch (threads) {
    case 128: k_items<T, 128><<<nitems, 128, 0, s>>>(c, items, nitems); break;
    case 512: k_items<T, 512><<<nitems, 512, 0, s>>>(c, items, nitems); break;
    default: k_items<T, 256><<<nitems, 256, 0, s>>>(c, items, nitems); break;
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_persistent_t(const Ctx& c, const Item* items, int nitems,
                                int threads, int grid, unsigned* counter,
                                cudaStream_t s) {
  if (nitems <= 0) return cudaSuccess;
  if (grid > nitems) grid = nitems;
  switch (threads) {
    case 128:
      k_persistent<T, 128><<<grid, 128, 0, s>>>(c, items, nitems, counter);
      break;
    case 512:
      k_persistent<T, 512><<<grid, 512, 0, s>>>(c, items, nitems, counter);
      break;
    default:
      k_persistent<T, 256><<<grid, 256, 0, s>>>(c, items, nitems, counter);
      break;
  }
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_items(int dtype, const Ctx& ctx, const Item* items,
                         int nitems, int threads, cudaStream_t s) {
  return dtype == 1 ? launch_items_t<double>(ctx, items, nitems, threads, s)
                    : launch_items_t<float>(ctx, items, nitems, threads, s);
}

cudaError_t launch_persistent(int dtype, const Ctx& ctx, const Item* items,
                              int nitems, int threads, int grid,
                              unsigned* counter, cudaStream_t s) {
  return dtype == 1 ? launch_persistent_t<double>(ctx, items, nitems, threads,
                                                  grid, counter, s)
                    : launch_persistent_t<float>(ctx, items, nitems, threads,
                                                 grid, counter, s);
}

}  // namespace bcg
