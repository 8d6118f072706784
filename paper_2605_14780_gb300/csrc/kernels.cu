// sm_103a kernels of the ghost-fill operator y_G = A x_D + b
// (arxiv 2605.14780, Sec. III-B) and of its adjoint.
//
// Every launch works on a list of work items (bc_internal.h), one warp per
// item: as a plain grid (warp w of CTA b takes item b * warps + w; used by
// every launch form) or as a persistent grid whose warps claim items from an
// atomic counter.  No warp ever waits on another; there is no CTA barrier.
//
// The path is a sparse gather/scatter bounded by HBM bandwidth, so it runs on
// the CUDA cores: lanes take consecutive ghost cells (coalesced along axis 0),
// each lane keeps 8 independent levels (or 8 single-level values) in flight,
// copies move integer bit patterns so they are exact, and table rows
// (stencils, CSR entries) are loaded once per cell and reused for its levels.
#include <cstdint>

#include "bc_internal.h"

namespace bcg {
namespace {

template <typename T> struct BitsOf;
template <> struct BitsOf<float> { using type = uint32_t; };
template <> struct BitsOf<double> { using type = uint64_t; };

template <typename T>
__device__ __forceinline__ T ldg(const T* p) { return __ldg(p); }

__device__ __forceinline__ uint32_t fdiv(uint32_t n, const FastDiv& f) {
  return (__umulhi(n, f.m) + n) >> f.s;
}

// unit u -> cell q of the box and level chunk c (u = q + vol * c)
__device__ __forceinline__ void unit_of(int u, const Item& it, int& q, int& c) {
  c = (int)fdiv((uint32_t)u, it.vol);
  q = u - c * (int)it.vol.d;
}

// cell q of the box -> (i, j, k) relative to the box origin
__device__ __forceinline__ void cell_of(int q, const Item& it, int& i, int& j,
                                        int& k) {
  const int r = (int)fdiv((uint32_t)q, it.w0);
  i = q - r * (int)it.w0.d;
  k = (int)fdiv((uint32_t)r, it.w1);
  j = r - k * (int)it.w1.d;
}

__device__ __forceinline__ int dst_offset(const Item& it, int i, int j, int k) {
  return it.dst_org + i * it.dst_s0 + j * it.dst_s1 + k * it.dst_s2;
}

// ---------------------------------------------------------------------------
// zero / constant / map (matrix-free rows, Sec. III-B)
// ---------------------------------------------------------------------------
// Per-lane work batches: every load of a batch is issued before its first
// store, so a lane keeps up to kFlatUnroll * 2 (single-level values) or
// UnitsInFlight<T> * kChunk (8-level units) independent loads in flight.
template <typename T> struct UnitsInFlight { static constexpr int v = 4; };
template <> struct UnitsInFlight<double> { static constexpr int v = 2; };

template <typename T>
__device__ void structured_flat(const Item& it, const Ctx& c, int lane) {
  using B = typename BitsOf<T>::type;
  constexpr int U = 2 * kFlatUnroll;
  const int end = it.u0 + it.nunits;
  B* dbase = static_cast<B*>(c.slots[it.dst_slot]);
  const bool is_map = it.kind == IK_MAP;
  const B* sbase = is_map ? static_cast<const B*>(c.slots[it.src_slot]) : nullptr;
  const B* cval = static_cast<const B*>(c.const_val);
  for (int f0 = it.u0 + lane; f0 < end; f0 += 32 * U) {
    int doff[U];
    B v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int f = f0 + 32 * u;
      doff[u] = -1;
      v[u] = B(0);
      if (f < end) {
        int q, l, i, j, k;
        unit_of(f, it, q, l);
        cell_of(q, it, i, j, k);
        doff[u] = dst_offset(it, i, j, k) + l * it.dst_ls;
        if (is_map)
          v[u] = ldg(sbase + (it.src_org + i * it.src_s0 + j * it.src_s1 +
                              k * it.src_s2 + l * it.src_ls));
        else if (it.kind == IK_CONST)
          v[u] = ldg(cval + it.table + q);
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (doff[u] >= 0) dbase[doff[u]] = v[u];
  }
}

template <typename T>
__device__ void structured_chunk(const Item& it, const Ctx& c, int lane) {
  using B = typename BitsOf<T>::type;
  constexpr int R = UnitsInFlight<T>::v;
  const int end = it.u0 + it.nunits;
  B* dbase = static_cast<B*>(c.slots[it.dst_slot]);
  const bool is_map = it.kind == IK_MAP;
  const B* sbase = is_map ? static_cast<const B*>(c.slots[it.src_slot]) : nullptr;
  const int ls = it.dst_ls, sls = it.src_ls;
  for (int ub = it.u0 + lane; ub < end; ub += 32 * R) {
    B v[R][kChunk];
    int doff[R], nl[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int u = ub + 32 * r;
      nl[r] = 0;
      doff[r] = 0;
      if (u < end) {
        int q, ch, i, j, k;
        unit_of(u, it, q, ch);
        cell_of(q, it, i, j, k);
        const int l0 = ch * kChunk;
        nl[r] = min(kChunk, it.L - l0);
        doff[r] = dst_offset(it, i, j, k) + l0 * ls;
        if (is_map) {
          const B* s = sbase + (it.src_org + i * it.src_s0 + j * it.src_s1 +
                                k * it.src_s2 + l0 * sls);
#pragma unroll
          for (int l = 0; l < kChunk; ++l)
            if (l < nl[r]) v[r][l] = ldg(s + l * sls);
        } else {
          const B b = it.kind == IK_CONST
                          ? ldg(static_cast<const B*>(c.const_val) + it.table + q)
                          : B(0);
#pragma unroll
          for (int l = 0; l < kChunk; ++l) v[r][l] = b;
        }
      }
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
      B* d = dbase + doff[r];
#pragma unroll
      for (int l = 0; l < kChunk; ++l)
        if (l < nl[r]) d[l * ls] = v[r][l];
    }
  }
}

// ---------------------------------------------------------------------------
// interpolation rows (user Itp, Sec. III-B) with optional 2x2 rotation of a
// covariant component pair (Sec. V-A): y = M (sum_k w_k x_u, sum_k w_k x_v)
// ---------------------------------------------------------------------------
template <typename T>
__device__ void interp_scalar(const Item& it, const Ctx& c, int lane) {
  using B = typename BitsOf<T>::type;
  const int end = it.u0 + it.nunits;
  const int ls = it.dst_ls;
  const int p = it.p;
  const int chn = it.ch;
  for (int u = it.u0 + lane; u < end; u += 32) {
    int q, ch, i, j, k;
    unit_of(u, it, q, ch);
    cell_of(q, it, i, j, k);
    const int l0 = ch * chn;
    const int nl = min(chn, it.L - l0);
    const int row = it.table + q;
    const int4 ix = __ldg(c.itp_idx + row);
    const int su = ix.x + it.comp;
    const int sls = __ldg(c.slot_ls + su);
    const T* x = static_cast<const T*>(c.slots[su]) + (ix.y + l0 * sls);
    T* d = static_cast<T*>(c.slots[it.dst_slot]) + (dst_offset(it, i, j, k) + l0 * ls);
    if (ix.w & kFlagSnap) {  // unit row: exact copy of node 0
      const B* s = reinterpret_cast<const B*>(x);
      B* db = reinterpret_cast<B*>(d);
      B v[kChunk];
#pragma unroll
      for (int l = 0; l < kChunk; ++l)
        if (l < nl) v[l] = ldg(s + l * sls);
#pragma unroll
      for (int l = 0; l < kChunk; ++l)
        if (l < nl) db[l * ls] = v[l];
      continue;
    }
    const T* wr = static_cast<const T*>(c.itp_w) + row * kPMax;
    T acc[kChunk];
#pragma unroll
    for (int l = 0; l < kChunk; ++l) acc[l] = T(0);
#pragma unroll
    for (int n = 0; n < kPMax; ++n) {
      if (n < p) {
        const T w = ldg(wr + n);
        const T* xn = x + n * ix.z;
#pragma unroll
        for (int l = 0; l < kChunk; ++l)
          if (l < nl) acc[l] = fma(w, ldg(xn + l * sls), acc[l]);
      }
    }
#pragma unroll
    for (int l = 0; l < kChunk; ++l)
      if (l < nl) d[l * ls] = acc[l];
  }
}

template <typename T>
__device__ void interp_pair(const Item& it, const Ctx& c, int lane) {
  constexpr int LU = kChunk / 2;
  const int end = it.u0 + it.nunits;
  const int ls = it.dst_ls;
  const int p = it.p;
  const int chn = it.ch;
  for (int u = it.u0 + lane; u < end; u += 32) {
    int q, ch, i, j, k;
    unit_of(u, it, q, ch);
    cell_of(q, it, i, j, k);
    const int l0 = ch * chn;
    const int nl = min(chn, it.L - l0);
    const int row = it.table + q;
    const int4 ix = __ldg(c.itp_idx + row);
    const int su = ix.x + it.comp, sv = ix.x + it.comp2;
    const int slu = __ldg(c.slot_ls + su), slv = __ldg(c.slot_ls + sv);
    const T* xu = static_cast<const T*>(c.slots[su]) + (ix.y + l0 * slu);
    const T* xv = static_cast<const T*>(c.slots[sv]) + (ix.y + l0 * slv);
    const int doff = dst_offset(it, i, j, k) + l0 * ls;
    T* du = static_cast<T*>(c.slots[it.dst_slot]) + doff;
    T* dv = static_cast<T*>(c.slots[it.dst_slot2]) + doff;
    const T* mr = static_cast<const T*>(c.itp_m) + row * 4;
    const T* wr = static_cast<const T*>(c.itp_w) + row * kPMax;
    const int pe = (ix.w & kFlagSnap) ? 1 : p;
    for (int lb = 0; lb < nl; lb += LU) {
      T au[LU], av[LU];
#pragma unroll
      for (int l = 0; l < LU; ++l) au[l] = av[l] = T(0);
#pragma unroll
      for (int n = 0; n < kPMax; ++n) {
        if (n < pe) {
          const T w = (ix.w & kFlagSnap) ? T(1) : ldg(wr + n);
          const T* xun = xu + n * ix.z + lb * slu;
          const T* xvn = xv + n * ix.z + lb * slv;
#pragma unroll
          for (int l = 0; l < LU; ++l)
            if (lb + l < nl) {
              au[l] = fma(w, ldg(xun + l * slu), au[l]);
              av[l] = fma(w, ldg(xvn + l * slv), av[l]);
            }
        }
      }
      const T m00 = ldg(mr), m01 = ldg(mr + 1), m10 = ldg(mr + 2), m11 = ldg(mr + 3);
#pragma unroll
      for (int l = 0; l < LU; ++l)
        if (lb + l < nl) {
          du[(lb + l) * ls] = fma(m00, au[l], m01 * av[l]);
          dv[(lb + l) * ls] = fma(m10, au[l], m11 * av[l]);
        }
    }
  }
}

// ---------------------------------------------------------------------------
// user CSR rows (Table III: F_NNZ / F_COL / F_DATA): the row's entries are
// loaded once per unit and reused for its levels
// ---------------------------------------------------------------------------
template <typename T>
__device__ void csr_rows(const Item& it, const Ctx& c, int lane) {
  constexpr int E = 8;  // rows up to E entries: all entry loads issued at once
  const int end = it.u0 + it.nunits;
  const int ls = it.dst_ls;
  const int chn = it.ch;
  const int W = it.p;
  const T* val = static_cast<const T*>(c.csr_val);
  for (int u = it.u0 + lane; u < end; u += 32) {
    int q, ch, i, j, k;
    unit_of(u, it, q, ch);
    cell_of(q, it, i, j, k);
    const int l0 = ch * chn;
    const int nl = min(chn, it.L - l0);
    const int row = it.table + q;
    const int nnz = __ldg(c.csr_nnz + row);
    const int e0 = it.src_org + q * W;
    T* d = static_cast<T*>(c.slots[it.dst_slot]) + (dst_offset(it, i, j, k) + l0 * ls);
    T acc[kChunk];
#pragma unroll
    for (int l = 0; l < kChunk; ++l) acc[l] = T(0);
    if (W <= E) {
      int es[E], eo[E];
      T ea[E];
#pragma unroll
      for (int e = 0; e < E; ++e)
        if (e < nnz) {
          es[e] = __ldg(c.csr_slot + e0 + e);
          eo[e] = __ldg(c.csr_off + e0 + e);
          ea[e] = ldg(val + e0 + e);
        }
#pragma unroll
      for (int e = 0; e < E; ++e)
        if (e < nnz) {
          const int sls = __ldg(c.slot_ls + es[e]);
          const T* x = static_cast<const T*>(c.slots[es[e]]) + (eo[e] + l0 * sls);
#pragma unroll
          for (int l = 0; l < kChunk; ++l)
            if (l < nl) acc[l] = fma(ea[e], ldg(x + l * sls), acc[l]);
        }
    } else {
      for (int e = 0; e < nnz; ++e) {
        const int s = __ldg(c.csr_slot + e0 + e);
        const T a = ldg(val + e0 + e);
        const int sls = __ldg(c.slot_ls + s);
        const T* x = static_cast<const T*>(c.slots[s]) + (__ldg(c.csr_off + e0 + e) + l0 * sls);
#pragma unroll
        for (int l = 0; l < kChunk; ++l)
          if (l < nl) acc[l] = fma(a, ldg(x + l * sls), acc[l]);
      }
    }
    const T rhs = ldg(static_cast<const T*>(c.csr_rhs) + row);
#pragma unroll
    for (int l = 0; l < kChunk; ++l)
      if (l < nl) d[l * ls] = acc[l] + rhs;
  }
}

// ---------------------------------------------------------------------------
// adjoint gather: x_bar_j += sum_i A_ij y_bar_i over the stored transpose,
// entries in ascending ghost order (deterministic, no atomics)
// ---------------------------------------------------------------------------
template <typename T>
__device__ void adj_rows(const Item& it, const Ctx& c, int lane) {
  const int end = it.u0 + it.nunits;
  const int chn = it.ch;
  const T* wv = static_cast<const T*>(c.aent_w);
  for (int u = it.u0 + lane; u < end; u += 32) {
    int q, ch;
    unit_of(u, it, q, ch);
    const int l0 = ch * chn;
    const int nl = min(chn, it.L - l0);
    const int r = it.table + q;
    const int slot = __ldg(c.arow_slot + r);
    const int ls = __ldg(c.slot_ls + slot);
    T* xb = static_cast<T*>(c.slots[slot]) + (__ldg(c.arow_off + r) + l0 * ls);
    const int64_t e0 = __ldg(c.adj_ptr + r), e1 = __ldg(c.adj_ptr + r + 1);
    T acc[kChunk];
#pragma unroll
    for (int l = 0; l < kChunk; ++l) acc[l] = (l < nl) ? xb[l * ls] : T(0);
    for (int64_t e = e0; e < e1; ++e) {
      const int gs = __ldg(c.aent_slot + e);
      const T a = ldg(wv + e);
      const int gls = __ldg(c.slot_ls + gs);
      const T* y = static_cast<const T*>(c.slots[gs]) + (__ldg(c.aent_off + e) + l0 * gls);
#pragma unroll
      for (int l = 0; l < kChunk; ++l)
        if (l < nl) acc[l] = fma(a, y[l * gls], acc[l]);
    }
#pragma unroll
    for (int l = 0; l < kChunk; ++l)
      if (l < nl) xb[l * ls] = acc[l];
  }
}

template <typename T>
__device__ __forceinline__ void run_item(const Item& it, const Ctx& c, int lane) {
  switch (it.kind) {
    case IK_ZERO:
    case IK_CONST:
    case IK_MAP:
      if (it.ch == 1)
        structured_flat<T>(it, c, lane);
      else
        structured_chunk<T>(it, c, lane);
      break;
    case IK_INTERP: interp_scalar<T>(it, c, lane); break;
    case IK_INTERP_PAIR: interp_pair<T>(it, c, lane); break;
    case IK_CSR: csr_rows<T>(it, c, lane); break;
    case IK_ADJ: adj_rows<T>(it, c, lane); break;
    default: break;
  }
}

static_assert(sizeof(Item) == 32 * 4, "an Item is loaded as one word per lane");

__device__ __forceinline__ void load_item(Item* dst, const Item* src, int lane) {
  reinterpret_cast<int*>(dst)[lane] = __ldg(reinterpret_cast<const int*>(src) + lane);
  __syncwarp();
}

template <int THREADS> struct Occ {
  static constexpr int kMinBlocks = THREADS >= 512 ? 1 : 512 / THREADS;
};

template <typename T, int THREADS>
__global__ void __launch_bounds__(THREADS, Occ<THREADS>::kMinBlocks)
    k_items(Ctx c, const Item* __restrict__ items, int nitems) {
  __shared__ Item sit[THREADS / 32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int idx = blockIdx.x * (THREADS / 32) + warp;
  if (idx >= nitems) return;
  load_item(&sit[warp], items + idx, lane);
  run_item<T>(sit[warp], c, lane);
}

// Persistent form: warps claim items from counter[0]; the last warp to
// finish resets both counters for the next launch.  No warp waits on another.
template <typename T, int THREADS>
__global__ void __launch_bounds__(THREADS, Occ<THREADS>::kMinBlocks)
    k_persistent(Ctx c, const Item* __restrict__ items, int nitems,
                 unsigned* counter) {
  __shared__ Item sit[THREADS / 32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (;;) {
    int idx = 0;
    if (lane == 0) idx = (int)atomicAdd(counter, 1u);
    idx = __shfl_sync(0xffffffffu, idx, 0);
    if (idx >= nitems) break;
    load_item(&sit[warp], items + idx, lane);
    run_item<T>(sit[warp], c, lane);
    __syncwarp();
  }
  if (lane == 0) {
    __threadfence();
    const unsigned nwarps = gridDim.x * (THREADS / 32);
    if (atomicAdd(counter + 1, 1u) == nwarps - 1) {
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
  const int wpb = threads / 32;
  const int grid = (nitems + wpb - 1) / wpb;
  switch (threads) {
    case 32: k_items<T, 32><<<grid, 32, 0, s>>>(c, items, nitems); break;
    case 64: k_items<T, 64><<<grid, 64, 0, s>>>(c, items, nitems); break;
    case 128: k_items<T, 128><<<grid, 128, 0, s>>>(c, items, nitems); break;
    case 512: k_items<T, 512><<<grid, 512, 0, s>>>(c, items, nitems); break;
    default: k_items<T, 256><<<grid, 256, 0, s>>>(c, items, nitems); break;
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_persistent_t(const Ctx& c, const Item* items, int nitems,
                                int threads, int grid, unsigned* counter,
                                cudaStream_t s) {
  if (nitems <= 0) return cudaSuccess;
  const int wpb = threads / 32;
  const int need = (nitems + wpb - 1) / wpb;
  if (grid > need) grid = need;
  switch (threads) {
    case 32: k_persistent<T, 32><<<grid, 32, 0, s>>>(c, items, nitems, counter); break;
    case 64: k_persistent<T, 64><<<grid, 64, 0, s>>>(c, items, nitems, counter); break;
    case 128: k_persistent<T, 128><<<grid, 128, 0, s>>>(c, items, nitems, counter); break;
    case 512: k_persistent<T, 512><<<grid, 512, 0, s>>>(c, items, nitems, counter); break;
    default: k_persistent<T, 256><<<grid, 256, 0, s>>>(c, items, nitems, counter); break;
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
