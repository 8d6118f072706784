// sm_103a kernels of the ghost-fill operator y_G = A x_D + b
// (arxiv 2605.14780, Sec. III-B) and of its adjoint.
//
// Every launch works on a list of work items (bc_internal.h), one warp per
// item: as a plain grid (warp w of CTA b takes item b * warps + w; used by
// every launch form) or as a resident grid whose warps walk the items with a
// fixed stride.  No warp ever waits on another; there is no CTA barrier.
//
// The path is a sparse gather/scatter bounded by HBM bandwidth, so it runs on
// the CUDA cores.  The lanes of a warp are laid over the item's (cell, level)
// values in the order that is contiguous in memory -- consecutive cells when
// levels are far apart, consecutive levels when they are adjacent -- so a
// warp instruction touches as few 32-byte sectors as the layout allows; each
// lane keeps several independent values in flight; copies move integer bit
// patterns so they are exact; table rows (stencils, CSR entries) are loaded
// once per cell and level chunk.
#include <climits>
#include <cstddef>
#include <cstdint>

#include "bc_internal.h"

namespace bcg {
namespace {

template <typename T> struct BitsOf;
template <> struct BitsOf<float> { using type = uint32_t; };
template <> struct BitsOf<double> { using type = uint64_t; };

__device__ __forceinline__ uint32_t to_bits(float v) { return __float_as_uint(v); }
__device__ __forceinline__ uint64_t to_bits(double v) {
  return (uint64_t)__double_as_longlong(v);
}

template <typename T>
__device__ __forceinline__ T ldg(const T* p) { return __ldg(p); }

__device__ __forceinline__ uint32_t fdiv(uint32_t n, const FastDiv& f) {
  return (__umulhi(n, f.m) + n) >> f.s;
}

// flat unit f -> (cell q, level l)
__device__ __forceinline__ void flat_of(int f, const Item& it, int& q, int& l) {
  if (it.mode == MODE_FLAT_LEVEL) {
    q = (int)fdiv((uint32_t)f, it.lev);
    l = f - q * (int)it.lev.d;
  } else {
    l = (int)fdiv((uint32_t)f, it.vol);
    q = f - l * (int)it.vol.d;
  }
}

// chunk unit u -> cell q of the box and level chunk c (u = q + vol * c)
__device__ __forceinline__ void unit_of(int u, const Item& it, int& q, int& c) {
  c = (int)fdiv((uint32_t)u, it.vol);
  q = u - c * (int)it.vol.d;
}

// element offset (level 0) of cell q of the item's box, from the cell table
__device__ __forceinline__ int dst_cell(const Item& it, const Ctx& c, int q) {
  return __ldg(c.ctab_d + it.ctab + q);
}

// Base pointers of an item's destination slot(s) and of its source slot (MAP,
// or the common source slot of CSR rows), resolved once per item.
struct Ptrs {
  void* d;
  void* d2;
  const void* s;
  void* stage;  // this warp's shared-memory staging area (Ctx::stage_warp bytes), or null
};

// ---------------------------------------------------------------------------
// zero / constant / map (matrix-free rows, Sec. III-B)
// ---------------------------------------------------------------------------
// Flat: every lane keeps U single values in flight.  The item fields the
// loop needs are copied to registers first (the item itself sits in shared
// memory), and the loop is specialised on the unit order.
template <typename T, bool LEVEL>
__device__ void structured_flat_t(const Item& it, const Ptrs& P, const Ctx& c, int lane) {
  using B = typename BitsOf<T>::type;
  constexpr int U = kFlatUnroll;
  const int end = it.u0 + it.nunits;
  const FastDiv dv = LEVEL ? it.lev : it.vol;
  const int div = (int)dv.d;
  const int* __restrict__ cd = c.ctab_d + it.ctab;
  const int* __restrict__ cs = c.ctab_s + it.ctab;
  const int dls = it.dst_ls, sls = it.src_ls;
  const int kind = it.kind;
  B* dbase = static_cast<B*>(P.d);
  const B* sbase = static_cast<const B*>(P.s);
  const B* cval = static_cast<const B*>(c.const_val) + it.table;
  for (int f0 = it.u0 + lane; f0 < end; f0 += 32 * U) {
    int doff[U];
    B v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int f = f0 + 32 * u;
      doff[u] = -1;
      v[u] = B(0);
      if (f < end) {
        const int a = (int)fdiv((uint32_t)f, dv);
        const int q = LEVEL ? a : f - a * div;
        const int l = LEVEL ? f - a * div : a;
        doff[u] = __ldg(cd + q) + l * dls;
        if (kind == IK_MAP)
          v[u] = ldg(sbase + (__ldg(cs + q) + l * sls));
        else if (kind == IK_CONST)
          v[u] = ldg(cval + q);
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (doff[u] >= 0) dbase[doff[u]] = v[u];
  }
}

// Adjoint of unit copies over runs: x_bar[dst + t] += y_bar[src + t], the
// data values of P.d and the ghost values of P.s, with the lane layout of
// the copy runs below.  Runs in the transpose-gather kernel (its register
// budget), as items of the same launch.
template <typename T>
__device__ void add_runs(const Item& it, const Ptrs& P, const Ctx& c, int lane) {
  constexpr int U = 8;  // two arrays of U values: 8 keeps the gather's budget
  const int nr = it.nunits;
  const int lg = __ffs(it.p) - 1;
  const int g = 1 << lg, side = 32 >> lg;
  const int sub = lane >> lg, off = lane & (g - 1);
  int4 mine = make_int4(0, 0, 0, 0);
  if (lane < nr) mine = __ldg(c.runs + it.u0 + lane);
  for (int k = 0; k < nr; k += side) {
    const int r = k + sub;
    const int dof = __shfl_sync(0xffffffffu, mine.x, r & 31);
    const int sof = __shfl_sync(0xffffffffu, mine.y, r & 31);
    int len = __shfl_sync(0xffffffffu, mine.z, r & 31);
    if (r >= nr) len = 0;
    T* d = static_cast<T*>(P.d) + dof;
    const T* s = static_cast<const T*>(P.s) + sof;
    int t = off;
    for (; t + g * (U - 1) < len; t += g * U) {
      T y[U], x[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        y[u] = ldg(s + t + g * u);
        x[u] = d[t + g * u];
      }
#pragma unroll
      for (int u = 0; u < U; ++u) d[t + g * u] = x[u] + y[u];
    }
    if (t < len) {
      T y[U], x[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const bool on = t + g * u < len;
        y[u] = on ? ldg(s + t + g * u) : T(0);
        x[u] = on ? d[t + g * u] : T(0);
      }
#pragma unroll
      for (int u = 0; u < U; ++u)
        if (t + g * u < len) d[t + g * u] = x[u] + y[u];
    }
  }
}

// Runs: an item holds up to 32 runs, one descriptor per lane, loaded at
// once.  Groups of g = Item::p lanes (a power of two) each take one run, so
// 32 / g runs are copied side by side and short runs still fill the warp;
// within its run a lane keeps U values in flight.  A run is contiguous in the
// destination and, for maps, in the source: a value costs a load and a store.
template <typename T>
__device__ void structured_runs(const Item& it, const Ptrs& P, const Ctx& c, int lane) {
  using B = typename BitsOf<T>::type;
  constexpr int U = kRunUnroll;
  const bool is_map = it.kind == IK_MAP;
  const int nr = it.nunits;
  const int lg = __ffs(it.p) - 1;  // log2 of the lanes per run
  const int g = 1 << lg;
  const int side = 32 >> lg;       // runs side by side
  int4 mine = make_int4(0, 0, 0, 0);
  if (lane < nr) mine = __ldg(c.runs + it.u0 + lane);
  B* dbase = static_cast<B*>(P.d);
  const B* sbase = static_cast<const B*>(P.s);
  const int sub = lane >> lg, off = lane & (g - 1);
  for (int k = 0; k < nr; k += side) {
    const int r = k + sub;
    const int dof = __shfl_sync(0xffffffffu, mine.x, r & 31);
    const int sof = __shfl_sync(0xffffffffu, mine.y, r & 31);
    int len = __shfl_sync(0xffffffffu, mine.z, r & 31);
    if (r >= nr) len = 0;
    B* d = dbase + dof;
    if (is_map) {
      const B* s = sbase + sof;
      int t = off;
      for (; t + g * (U - 1) < len; t += g * U) {
        B v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) v[u] = ldg(s + t + g * u);
#pragma unroll
        for (int u = 0; u < U; ++u) d[t + g * u] = v[u];
      }
      if (t < len) {
        B v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) v[u] = t + g * u < len ? ldg(s + t + g * u) : B(0);
#pragma unroll
        for (int u = 0; u < U; ++u)
          if (t + g * u < len) d[t + g * u] = v[u];
      }
    } else {
      int t = off;
      for (; t + g * (U - 1) < len; t += g * U) {
#pragma unroll
        for (int u = 0; u < U; ++u) d[t + g * u] = B(0);
      }
#pragma unroll
      for (int u = 0; u < U; ++u)
        if (t + g * u < len) d[t + g * u] = B(0);
    }
  }
}

// ---------------------------------------------------------------------------
// 16-byte vector runs.  The runs of an item (at most 32, one descriptor per
// lane) are cut into destination-aligned 16-byte chunks -- E = 16 / S
// elements, the first and last chunk of a run partly outside it -- and the
// chunks of all runs form one sequence that the lanes take in order, lane t
// chunk t, t + 32, ..., U chunks in flight per lane.  So a warp instruction
// moves 512 contiguous bytes whatever the run lengths, and short runs do not
// leave lanes idle.  The alignment of a run depends on the caller's slot
// pointers, so it is worked out here: a chunk whose source is aligned the
// same way loads one 16-byte vector, otherwise the two aligned vectors that
// hold its elements and shifts them into place.  Every vector loaded holds
// at least one element of its run (so no load leaves the field's
// allocation); full chunks are stored as one vector, the chunks at the ends
// of a run element by element, so no value outside a run is written.
// ---------------------------------------------------------------------------
constexpr int kVecUnroll = 2;  // 4 spills under the 48-register budget
constexpr int kNoChunk = INT_MIN;  // a lane's chunk slot past the item's last chunk

enum RunOp : int { RUN_ZERO = 0, RUN_COPY = 1, RUN_ADD = 2 };

// words [ws, ws + 4) of the 8 words (a, b), ws in 1..3
__device__ __forceinline__ uint4 shift_words(const uint4& a, const uint4& b, int ws) {
  uint4 r;
  r.x = ws == 1 ? a.y : (ws == 2 ? a.z : a.w);
  r.y = ws == 1 ? a.z : (ws == 2 ? a.w : b.x);
  r.z = ws == 1 ? a.w : (ws == 2 ? b.x : b.y);
  r.w = ws == 1 ? b.x : (ws == 2 ? b.y : b.z);
  return r;
}

// bit pattern of element j (a constant after unrolling) of a 16-byte vector
template <typename T>
__device__ __forceinline__ typename BitsOf<T>::type vec_elem(const uint4& v, int j) {
  if constexpr (sizeof(T) == 4) {
    return j == 0 ? v.x : (j == 1 ? v.y : (j == 2 ? v.z : v.w));
  } else {
    return j == 0 ? ((uint64_t)v.y << 32 | v.x) : ((uint64_t)v.w << 32 | v.z);
  }
}

template <typename T>
__device__ __forceinline__ uint4 add_vec(const uint4& a, const uint4& b) {
  uint4 r;
  if constexpr (sizeof(T) == 4) {
    r.x = __float_as_uint(__uint_as_float(a.x) + __uint_as_float(b.x));
    r.y = __float_as_uint(__uint_as_float(a.y) + __uint_as_float(b.y));
    r.z = __float_as_uint(__uint_as_float(a.z) + __uint_as_float(b.z));
    r.w = __float_as_uint(__uint_as_float(a.w) + __uint_as_float(b.w));
  } else {
    const double a0 = __hiloint2double((int)a.y, (int)a.x), a1 = __hiloint2double((int)a.w, (int)a.z);
    const double b0 = __hiloint2double((int)b.y, (int)b.x), b1 = __hiloint2double((int)b.w, (int)b.z);
    const double r0 = a0 + b0, r1 = a1 + b1;
    r.x = (unsigned)__double2loint(r0);
    r.y = (unsigned)__double2hiint(r0);
    r.z = (unsigned)__double2loint(r1);
    r.w = (unsigned)__double2hiint(r1);
  }
  return r;
}

// OP: RUN_ZERO (d = 0), RUN_COPY (d = s, bit patterns), RUN_ADD (d = d + s
// in T; the adjoint of unit copies).  Runs {dst offset, src offset, length}.
template <typename T, int OP>
__device__ void runs_vec(const Item& it, const Ptrs& P, const Ctx& c, int lane) {
  using B = typename BitsOf<T>::type;
  constexpr int E = 16 / (int)sizeof(T);
  constexpr int LS = sizeof(T) == 4 ? 2 : 3;  // log2 of the element size
  constexpr int WPE = (int)sizeof(T) / 4;     // 32-bit words per element
  constexpr int U = kVecUnroll;
  constexpr unsigned FULL = 0xffffffffu;
  const int nr = it.nunits;
  int4 mine = make_int4(0, 0, 0, 0);
  if (lane < nr) mine = __ldg(c.runs + it.u0 + lane);
  B* dbase = static_cast<B*>(P.d);
  const B* sbase = static_cast<const B*>(P.s);
  const uint32_t dmis = (uint32_t)(reinterpret_cast<uintptr_t>(dbase) >> LS);
  const uint32_t smis = (uint32_t)(reinterpret_cast<uintptr_t>(sbase) >> LS);
  // chunks of this lane's run and their running count over the lanes
  const int ad = (int)((dmis + (uint32_t)mine.x) & (E - 1));
  const int nch = mine.z > 0 ? (mine.z + ad + E - 1) / E : 0;
  int incl = nch;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int t = __shfl_up_sync(FULL, incl, o);
    if (lane >= o) incl += t;
  }
  const int total = __shfl_sync(FULL, incl, 31);
  const int excl = incl - nch;
  for (int base = 0; base < total; base += 32 * U) {
    uint4 v[U];
    int dq[U], lo[U], hi[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int ch = base + lane + 32 * u;
      // the run of chunk ch: the last lane whose first chunk is <= ch
      int r = 0;
#pragma unroll
      for (int step = 16; step > 0; step >>= 1) {
        const int e = __shfl_sync(FULL, excl, r + step);
        if (e <= ch) r += step;
      }
      const int rd = __shfl_sync(FULL, mine.x, r);
      const int rs = __shfl_sync(FULL, mine.y, r);
      const int rn = __shfl_sync(FULL, mine.z, r);
      const int ra = __shfl_sync(FULL, ad, r);
      const int re = __shfl_sync(FULL, excl, r);
      const int e0 = (ch - re) * E - ra;  // run element in the chunk's first slot
      lo[u] = max(0, -e0);
      hi[u] = min(E, rn - e0);
      dq[u] = ch < total ? rd + e0 : kNoChunk;  // may be negative: slots before the slot base
      v[u] = make_uint4(0u, 0u, 0u, 0u);
      if (OP != RUN_ZERO && ch < total) {
        const int s0 = rs + e0;
        const int sa = (int)((smis + (uint32_t)s0) & (E - 1));
        const uint4* sp = reinterpret_cast<const uint4*>(sbase + (s0 - sa));
        if (sa == 0) {
          v[u] = __ldg(sp);
        } else {
          uint4 a = make_uint4(0u, 0u, 0u, 0u), b = a;
          if (sa + lo[u] < E) a = __ldg(sp);
          if (sa + hi[u] > E) b = __ldg(sp + 1);
          v[u] = shift_words(a, b, sa * WPE);
        }
      }
    }
    if (OP == RUN_ADD) {
#pragma unroll
      for (int u = 0; u < U; ++u)
        if (dq[u] != kNoChunk) {
          const uint4 x = *reinterpret_cast<const uint4*>(dbase + dq[u]);
          v[u] = add_vec<T>(x, v[u]);
        }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (dq[u] == kNoChunk) continue;
      B* d = dbase + dq[u];
      if (lo[u] == 0 && hi[u] == E) {
        *reinterpret_cast<uint4*>(d) = v[u];
      } else {
#pragma unroll
        for (int j = 0; j < E; ++j)
          if (j >= lo[u] && j < hi[u]) d[j] = vec_elem<T>(v[u], j);
      }
    }
  }
}

template <typename T>
__device__ __forceinline__ void structured_flat(const Item& it, const Ptrs& P, const Ctx& c,
                                                int lane) {
  if (it.mode == MODE_RUNS && c.vec_runs)
    it.kind == IK_MAP ? runs_vec<T, RUN_COPY>(it, P, c, lane)
                      : runs_vec<T, RUN_ZERO>(it, P, c, lane);
  else if (it.mode == MODE_RUNS)
    structured_runs<T>(it, P, c, lane);
  else if (it.mode == MODE_FLAT_LEVEL)
    structured_flat_t<T, true>(it, P, c, lane);
  else
    structured_flat_t<T, false>(it, P, c, lane);
}

// ---------------------------------------------------------------------------
// interpolation rows (user Itp, Sec. III-B) with optional 2x2 rotation of a
// covariant component pair (Sec. V-A): y = M (sum_k w_k x_u, sum_k w_k x_v)
// ---------------------------------------------------------------------------
// CH: the most levels of one unit (the arrays of a lane); the item's mode
// (its chunk length, <= CH) is the levels-per-lane split the plan chose.
template <typename T, int CH>
__device__ void interp_scalar_chunk(const Item& it, const Ptrs& P, const Ctx& c, int lane) {
  using B = typename BitsOf<T>::type;
  const int end = it.u0 + it.nunits;
  const int ls = it.dst_ls;
  const int p = it.p;
  const int chn = it.mode;
  const int comp = it.comp & 0xffff;
  for (int u = it.u0 + lane; u < end; u += 32) {
    int q, ch;
    unit_of(u, it, q, ch);
    const int l0 = ch * chn;
    const int nl = min(chn, (int)it.lev.d - l0);
    const int row = it.table + q;
    const int4 ix = __ldg(c.itp_idx + row);
    const int su = ix.x + comp;
    const int sls = __ldg(c.slot_ls + su);
    const T* x = static_cast<const T*>(c.slots[su]) + (ix.y + l0 * sls);
    T* d = static_cast<T*>(P.d) + (dst_cell(it, c, q) + l0 * ls);
    if (ix.w & kFlagSnap) {  // unit row: exact copy of node 0
      const B* s = reinterpret_cast<const B*>(x);
      B* db = reinterpret_cast<B*>(d);
      B v[CH];
#pragma unroll
      for (int l = 0; l < CH; ++l)
        if (l < nl) v[l] = ldg(s + l * sls);
#pragma unroll
      for (int l = 0; l < CH; ++l)
        if (l < nl) db[l * ls] = v[l];
      continue;
    }
    const T* wr = static_cast<const T*>(c.itp_w) + row * kPMax;
    T acc[CH];
#pragma unroll
    for (int l = 0; l < CH; ++l) acc[l] = T(0);
#pragma unroll
    for (int n = 0; n < kPMax; ++n) {
      if (n < p) {
        const T w = ldg(wr + n);
        const T* xn = x + n * ix.z;
#pragma unroll
        for (int l = 0; l < CH; ++l)
          if (l < nl) acc[l] = fma(w, ldg(xn + l * sls), acc[l]);
      }
    }
#pragma unroll
    for (int l = 0; l < CH; ++l)
      if (l < nl) d[l * ls] = acc[l];
  }
}

template <typename T, int CH>
__device__ void interp_pair_chunk(const Item& it, const Ptrs& P, const Ctx& c, int lane) {
  constexpr int LU = CH / 2;
  const int end = it.u0 + it.nunits;
  const int ls = it.dst_ls;
  const int p = it.p;
  const int chn = it.mode;
  for (int u = it.u0 + lane; u < end; u += 32) {
    int q, ch;
    unit_of(u, it, q, ch);
    const int l0 = ch * chn;
    const int nl = min(chn, (int)it.lev.d - l0);
    const int row = it.table + q;
    const int4 ix = __ldg(c.itp_idx + row);
    const int su = ix.x + (it.comp & 0xffff), sv = ix.x + (it.comp >> 16);
    const int slu = __ldg(c.slot_ls + su), slv = __ldg(c.slot_ls + sv);
    const T* xu = static_cast<const T*>(c.slots[su]) + (ix.y + l0 * slu);
    const T* xv = static_cast<const T*>(c.slots[sv]) + (ix.y + l0 * slv);
    const int doff = dst_cell(it, c, q) + l0 * ls;
    T* du = static_cast<T*>(P.d) + doff;
    T* dv = static_cast<T*>(P.d2) + doff;
    const T* mr = static_cast<const T*>(c.itp_m) + row * 4;
    const T* wr = static_cast<const T*>(c.itp_w) + row * kPMax;
    const bool snap = ix.w & kFlagSnap;
    const int pe = snap ? 1 : p;
    for (int lb = 0; lb < nl; lb += LU) {
      T au[LU], av[LU];
#pragma unroll
      for (int l = 0; l < LU; ++l) au[l] = av[l] = T(0);
#pragma unroll
      for (int n = 0; n < kPMax; ++n) {
        if (n < pe) {
          const T w = snap ? T(1) : ldg(wr + n);
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

// Staged interpolation (MODE_TILE): with levels far apart in memory, the
// nodes of a tile of up to 32 ghost cells lie in a small box of the
// neighbour block -- a strip of the edge rows or columns (the transposed
// strip when the nodes step along the neighbour's strided axis).  The warp
// copies the box, for the item's levels and components, into its shared
// memory with cp.async (each source value once, lanes over consecutive
// cells of a box row), then every lane evaluates its (cell, level) rows
// from shared memory: the p-point sums, the 2x2 rotation of a vector pair,
// and the store.  Same sums in the same order as the per-lane path.
template <typename T>
__device__ __forceinline__ void cp_async_elem(T* smem, const T* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  if constexpr (sizeof(T) == 4)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gmem) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem) : "memory");
}

__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_all;\n" ::: "memory");
}

template <typename T>
__device__ void interp_tile(const Item& it, const Ptrs& P, const Ctx& c, int lane) {
  using B = typename BitsOf<T>::type;
  T* sm = static_cast<T*>(P.stage);
  const bool pair = it.kind == IK_INTERP_PAIR;
  const int nc = pair ? 2 : 1;
  const int A = it.bw * it.bh;
  const int cu = it.comp & 0xffff, cv = it.comp >> 16;
  const int64_t lev0 = (int64_t)it.l0 * it.src_ls + it.borg;
  const T* xu = static_cast<const T*>(c.slots[it.bsrc + cu]) + lev0;
  const T* xv = pair ? static_cast<const T*>(c.slots[it.bsrc + cv]) + lev0 : xu;
  // stage: [level][component][box row][box column]
  for (int g = 0; g < it.nl * nc; ++g) {
    const int l = pair ? g >> 1 : g;
    const T* src = ((pair && (g & 1)) ? xv : xu) + (int64_t)l * it.src_ls;
    T* dst = sm + g * A;
    for (int e = lane; e < A; e += 32) {
      const int bj = (int)fdiv((uint32_t)e, it.bwid), bi = e - bj * it.bw;
      cp_async_elem<T>(dst + e, src + (bi * it.bs0 + bj * it.bs1));
    }
  }
  cp_async_wait_all();
  __syncwarp();
  // lanes take (cell, group of kTileLevels levels) units, cells fastest:
  // a cell's weights, box word and rotation load once for its group
  const int nq = it.nunits, tot = nq * ((it.nl + kTileLevels - 1) / kTileLevels);
  const int p = it.p;
  const int lstep = nc * A;  // stage values per level
  B* du = static_cast<B*>(P.d);
  B* dv = static_cast<B*>(P.d2);
  for (int u = lane; u < tot; u += 32) {
    const int g = (int)fdiv((uint32_t)u, it.vol), q = u - g * nq;
    const int lb = g * kTileLevels;
    const int row = it.table + it.u0 + q;
    const int bx = __ldg(c.itp_box + row);
    const int st = (bx & kBoxRows) ? it.bw : 1;
    const bool snap = bx & kBoxSnap;
    const int64_t off = (int64_t)dst_cell(it, c, it.u0 + q) + (int64_t)(it.l0 + lb) * it.dst_ls;
    const int64_t ls = it.dst_ls;
    const T* su = sm + lb * lstep + (bx & kBoxIndex);
    const T* wr = static_cast<const T*>(c.itp_w) + row * kPMax;
    if (!pair) {
      if (snap) {  // unit row: exact copy of node 0
#pragma unroll
        for (int l = 0; l < kTileLevels; ++l)
          if (lb + l < it.nl) du[off + l * ls] = reinterpret_cast<const B*>(su)[l * lstep];
        continue;
      }
      T acc[kTileLevels];
#pragma unroll
      for (int l = 0; l < kTileLevels; ++l) acc[l] = T(0);
#pragma unroll
      for (int n = 0; n < kPMax; ++n)
        if (n < p) {
          const T w = ldg(wr + n);
#pragma unroll
          for (int l = 0; l < kTileLevels; ++l)
            if (lb + l < it.nl) acc[l] = fma(w, su[l * lstep + n * st], acc[l]);
        }
#pragma unroll
      for (int l = 0; l < kTileLevels; ++l)
        if (lb + l < it.nl) du[off + l * ls] = to_bits(acc[l]);
    } else {
      const T* sv = su + A;
      const int pe = snap ? 1 : p;
      T au[kTileLevels], av[kTileLevels];
#pragma unroll
      for (int l = 0; l < kTileLevels; ++l) au[l] = av[l] = T(0);
#pragma unroll
      for (int n = 0; n < kPMax; ++n)
        if (n < pe) {
          const T w = snap ? T(1) : ldg(wr + n);
#pragma unroll
          for (int l = 0; l < kTileLevels; ++l)
            if (lb + l < it.nl) {
              au[l] = fma(w, su[l * lstep + n * st], au[l]);
              av[l] = fma(w, sv[l * lstep + n * st], av[l]);
            }
        }
      const T* mr = static_cast<const T*>(c.itp_m) + row * 4;
      const T m00 = ldg(mr), m01 = ldg(mr + 1), m10 = ldg(mr + 2), m11 = ldg(mr + 3);
#pragma unroll
      for (int l = 0; l < kTileLevels; ++l)
        if (lb + l < it.nl) {
          du[off + l * ls] = to_bits(fma(m00, au[l], m01 * av[l]));
          dv[off + l * ls] = to_bits(fma(m10, au[l], m11 * av[l]));
        }
    }
  }
  __syncwarp();  // every lane is done with the stage before the next item
}

// Staged CSR rows (MODE_TILE, levels far apart in memory): the entries of
// a tile of up to 32 rows lie in one small box of one block, in at most two
// of its slots (a vector pair's components); the warp copies the box for
// the item's levels and slots to shared memory, then each lane sums one row
// for a group of up to kTileLevels levels from there, loading each entry's
// weight and box word once for the group, in entry order (as the per-lane
// path: from zero, then + b).  Each entry carries its value's place in one
// level of the stage (csr_box: slot selector * box cells + box index).
template <typename T>
__device__ __forceinline__ void stage_box(const Item& it, const Ctx& c, T* sm, int lane) {
  const int nsel = it.bsrc2 >= 0 ? 2 : 1;
  const int A = it.bw * it.bh;
  const int64_t lev0 = (int64_t)it.l0 * it.src_ls + it.borg;
  const T* x0 = static_cast<const T*>(c.slots[it.bsrc]) + lev0;
  const T* x1 = nsel > 1 ? static_cast<const T*>(c.slots[it.bsrc2]) + lev0 : x0;
  // stage: [level][slot][box row][box column]
  for (int g = 0; g < it.nl * nsel; ++g) {
    const int l = nsel > 1 ? g >> 1 : g;
    const T* src = ((nsel > 1 && (g & 1)) ? x1 : x0) + (int64_t)l * it.src_ls;
    T* dst = sm + g * A;
    for (int e = lane; e < A; e += 32) {
      const int bj = (int)fdiv((uint32_t)e, it.bwid), bi = e - bj * it.bw;
      cp_async_elem<T>(dst + e, src + (bi * it.bs0 + bj * it.bs1));
    }
  }
  cp_async_wait_all();
  __syncwarp();
}

// four consecutive words / values from a 16-byte boundary
__device__ __forceinline__ void ld_words4(const int32_t* p, int* w) {
  const int4 v = __ldg(reinterpret_cast<const int4*>(p));
  w[0] = v.x;
  w[1] = v.y;
  w[2] = v.z;
  w[3] = v.w;
}

template <typename T>
__device__ __forceinline__ void ld_vals4(const T* p, T* a) {
  if constexpr (sizeof(T) == 4) {
    const float4 v = __ldg(reinterpret_cast<const float4*>(p));
    a[0] = v.x;
    a[1] = v.y;
    a[2] = v.z;
    a[3] = v.w;
  } else {
    const double2 v = __ldg(reinterpret_cast<const double2*>(p));
    const double2 u = __ldg(reinterpret_cast<const double2*>(p) + 1);
    a[0] = v.x;
    a[1] = v.y;
    a[2] = u.x;
    a[3] = u.y;
  }
}

template <typename T, int W>
__device__ void csr_tile(const Item& it, const Ptrs& P, const Ctx& c, int lane) {
  T* sm = static_cast<T*>(P.stage);
  stage_box<T>(it, c, sm, lane);
  const int lstep = (it.bsrc2 >= 0 ? 2 : 1) * it.bw * it.bh;  // stage values per level
  const int nq = it.nunits, tot = nq * ((it.nl + kTileLevels - 1) / kTileLevels);
  const T* val = static_cast<const T*>(c.csr_val);
  T* d = static_cast<T*>(P.d);
  for (int u = lane; u < tot; u += 32) {
    const int g = (int)fdiv((uint32_t)u, it.vol), q = u - g * nq;
    const int lb = g * kTileLevels;
    const int row = it.table + it.u0 + q;
    const int nnz = __ldg(c.csr_nnz + row);
    const int e0 = it.src_org + (it.u0 + q) * it.p;
    const T* s = sm + lb * lstep;
    T acc[kTileLevels];
#pragma unroll
    for (int l = 0; l < kTileLevels; ++l) acc[l] = T(0);
    // the row's entries W (4, or 8 when the row width is a multiple of 8)
    // at a time (rows start on 16-byte boundaries): the entries' stage
    // places (csr_box) and weights load as vectors, so a row costs one
    // memory latency per W entries; in the last, partial block the padding
    // entries (place 0, weight 0) read a staged value and are dropped
    for (int e = 0; e < nnz; e += W) {
      int bx[W];
      T w[W];
#pragma unroll
      for (int h = 0; h < W; h += 4) {
        ld_words4(c.csr_box + e0 + e + h, bx + h);
        ld_vals4<T>(val + e0 + e + h, w + h);
      }
      if (e + W <= nnz) {
#pragma unroll
        for (int j = 0; j < W; ++j)
#pragma unroll
          for (int l = 0; l < kTileLevels; ++l)
            if (lb + l < it.nl) acc[l] = fma(w[j], s[bx[j] + l * lstep], acc[l]);
      } else {
#pragma unroll
        for (int j = 0; j < W; ++j) {
          const bool live = e + j < nnz;
#pragma unroll
          for (int l = 0; l < kTileLevels; ++l)
            if (lb + l < it.nl) {
              const T xv = s[bx[j] + l * lstep];
              acc[l] = live ? fma(w[j], xv, acc[l]) : acc[l];
            }
        }
      }
    }
    const T b = ldg(static_cast<const T*>(c.csr_rhs) + row);
    T* dd = d + (int64_t)dst_cell(it, c, it.u0 + q) + (int64_t)(it.l0 + lb) * it.dst_ls;
#pragma unroll
    for (int l = 0; l < kTileLevels; ++l)
      if (lb + l < it.nl) dd[(int64_t)l * it.dst_ls] = acc[l] + b;
  }
  __syncwarp();  // every lane is done with the stage before the next item
}

// Staged transpose rows (MODE_TILE adjoint gather items, levels far apart in
// memory): the ghost values that a tile of up to 32 data values' transpose
// rows read lie in one small box of one block, in at most two slots; the
// warp copies the box of ghost cotangents for the item's levels to shared
// memory, then each lane updates one data value for a group of up to
// kTileLevels levels with the entries in ghost order from there (as
// adj_chunk: from the value's own cotangent).
template <typename T>
__device__ void adj_tile(const Item& it, const Ptrs& P, const Ctx& c, int lane) {
  T* sm = static_cast<T*>(P.stage);
  stage_box<T>(it, c, sm, lane);
  const int lstep = (it.bsrc2 >= 0 ? 2 : 1) * it.bw * it.bh;
  const int nq = it.nunits, tot = nq * ((it.nl + kTileLevels - 1) / kTileLevels);
  const T* wv = static_cast<const T*>(c.aent_w);
  for (int u = lane; u < tot; u += 32) {
    const int g = (int)fdiv((uint32_t)u, it.vol), q = u - g * nq;
    const int lb = g * kTileLevels;
    const int r = it.table + it.u0 + q;
    T* xb = static_cast<T*>(P.d) +
            ((int64_t)__ldg(c.arow_off + r) + (int64_t)(it.l0 + lb) * it.dst_ls);
    const int e0 = (int)__ldg(c.adj_ptr + r), e1 = (int)__ldg(c.adj_ptr + r + 1);
    const T* s = sm + lb * lstep;
    T acc[kTileLevels];
#pragma unroll
    for (int l = 0; l < kTileLevels; ++l)
      acc[l] = lb + l < it.nl ? xb[(int64_t)l * it.dst_ls] : T(0);
    // entries four at a time, their loads issued together
    for (int e = e0; e < e1; e += 4) {
      int bx[4];
      T w[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const bool live = e + j < e1;
        bx[j] = live ? __ldg(c.adj_box + e + j) : 0;
        w[j] = live ? ldg(wv + e + j) : T(0);
      }
#pragma unroll
      for (int j = 0; j < 4; ++j)
        if (e + j < e1) {
#pragma unroll
          for (int l = 0; l < kTileLevels; ++l)
            if (lb + l < it.nl) acc[l] = fma(w[j], s[bx[j] + l * lstep], acc[l]);
        }
    }
#pragma unroll
    for (int l = 0; l < kTileLevels; ++l)
      if (lb + l < it.nl) xb[(int64_t)l * it.dst_ls] = acc[l];
  }
  __syncwarp();  // every lane is done with the stage before the next item
}

// Flat interpolation: each lane keeps U values (cell, level) in flight; with
// level-fastest order the lanes of a warp share a cell, so its table row is
// one broadcast load and the node loads of the warp are contiguous.
template <typename T, bool PAIR>
__device__ void interp_flat(const Item& it, const Ptrs& P, const Ctx& c, int lane) {
  using B = typename BitsOf<T>::type;
  constexpr int U = 4;
  const int end = it.u0 + it.nunits;
  const int p = it.p;
  const int cu = it.comp & 0xffff, cv = it.comp >> 16;
  B* du = static_cast<B*>(P.d);
  B* dv = PAIR ? static_cast<B*>(P.d2) : nullptr;
  for (int f0 = it.u0 + lane; f0 < end; f0 += 32 * U) {
    int doff[U];
    B ou[U], ov[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int f = f0 + 32 * u;
      doff[u] = -1;
      ou[u] = ov[u] = B(0);
      if (f < end) {
        int q, l;
        flat_of(f, it, q, l);
        doff[u] = dst_cell(it, c, q) + l * it.dst_ls;
        const int row = it.table + q;
        const int4 ix = __ldg(c.itp_idx + row);
        const int su = ix.x + cu;
        const T* xu = static_cast<const T*>(c.slots[su]) + (ix.y + l * __ldg(c.slot_ls + su));
        const bool snap = ix.w & kFlagSnap;
        if (!PAIR && snap) {  // unit row: exact copy of node 0
          ou[u] = ldg(reinterpret_cast<const B*>(xu));
          continue;
        }
        const T* wr = static_cast<const T*>(c.itp_w) + row * kPMax;
        const int pe = snap ? 1 : p;
        T au = T(0), av = T(0);
        const T* xv = nullptr;
        if (PAIR) {
          const int sv = ix.x + cv;
          xv = static_cast<const T*>(c.slots[sv]) + (ix.y + l * __ldg(c.slot_ls + sv));
        }
#pragma unroll
        for (int n = 0; n < kPMax; ++n)
          if (n < pe) {
            const T w = snap ? T(1) : ldg(wr + n);
            au = fma(w, ldg(xu + n * ix.z), au);
            if (PAIR) av = fma(w, ldg(xv + n * ix.z), av);
          }
        if (PAIR) {
          const T* mr = static_cast<const T*>(c.itp_m) + row * 4;
          ou[u] = to_bits(fma(ldg(mr), au, ldg(mr + 1) * av));
          ov[u] = to_bits(fma(ldg(mr + 2), au, ldg(mr + 3) * av));
        } else {
          ou[u] = to_bits(au);
        }
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (doff[u] >= 0) {
        du[doff[u]] = ou[u];
        if (PAIR) dv[doff[u]] = ov[u];
      }
  }
}

// ---------------------------------------------------------------------------
// user CSR rows (Table III: F_NNZ / F_COL / F_DATA), ELL-packed: row q of the
// item's component has its entries at src_org + q * p
// ---------------------------------------------------------------------------
// When every entry of the item's rows reads one slot (P.s, level stride
// src_ls), the per-entry slot lookups are skipped.
template <typename T>
__device__ __forceinline__ const T* csr_src(const Item& it, const Ptrs& P, const Ctx& c,
                                             int e, int l, int& sls) {
  if (P.s) {
    sls = it.src_ls;
    return static_cast<const T*>(P.s) + (__ldg(c.csr_off + e) + l * sls);
  }
  const int s = __ldg(c.csr_slot + e);
  sls = __ldg(c.slot_ls + s);
  return static_cast<const T*>(c.slots[s]) + (__ldg(c.csr_off + e) + l * sls);
}

// A row of an ELL block of width W = 4 or 8 starts on a 16-byte boundary
// (the host pads the widths and aligns the blocks): its offsets, weights
// and (without a common slot) slots load as 16-byte vectors.
template <typename T> struct Vec16;
template <> struct Vec16<float> { using type = float4; static constexpr int n = 4; };
template <> struct Vec16<double> { using type = double2; static constexpr int n = 2; };

template <typename T, int W>
__device__ __forceinline__ void load_ell(const Ctx& c, int e0, bool common, int (&off)[W],
                                         T (&a)[W], int (&slot)[W]) {
  const int4* o4 = reinterpret_cast<const int4*>(c.csr_off + e0);
#pragma unroll
  for (int j = 0; j < W / 4; ++j) {
    const int4 v = __ldg(o4 + j);
    off[4 * j] = v.x;
    off[4 * j + 1] = v.y;
    off[4 * j + 2] = v.z;
    off[4 * j + 3] = v.w;
  }
  using V = typename Vec16<T>::type;
  constexpr int N = Vec16<T>::n;
  const V* a4 = reinterpret_cast<const V*>(static_cast<const T*>(c.csr_val) + e0);
#pragma unroll
  for (int j = 0; j < W / N; ++j) {
    const V v = __ldg(a4 + j);
    if constexpr (N == 4) {
      a[4 * j] = v.x;
      a[4 * j + 1] = v.y;
      a[4 * j + 2] = v.z;
      a[4 * j + 3] = v.w;
    } else {
      a[2 * j] = v.x;
      a[2 * j + 1] = v.y;
    }
  }
  if (!common) {
    const int4* s4 = reinterpret_cast<const int4*>(c.csr_slot + e0);
#pragma unroll
    for (int j = 0; j < W / 4; ++j) {
      const int4 v = __ldg(s4 + j);
      slot[4 * j] = v.x;
      slot[4 * j + 1] = v.y;
      slot[4 * j + 2] = v.z;
      slot[4 * j + 3] = v.w;
    }
  }
}

// One value per lane, a whole ELL row of width W per value.  With one
// common source slot the padding entries (offset 0 of that slot, in bounds)
// are loaded too and dropped by a select, so the W loads issue without
// branches; measured on the 512-block workload (levels innermost) this took
// the CSR kernel from 38 to 26 us.
template <typename T, int W, bool WIDE>
__device__ void csr_flat_w(const Item& it, const Ptrs& P, const Ctx& c, int lane) {
  const int end = it.u0 + it.nunits;
  T* dbase = static_cast<T*>(P.d);
  const T* sb = static_cast<const T*>(P.s);
  const bool common = sb != nullptr;
  const int RW = it.p;  // the row width: W, or a multiple of 8 for wide rows
  for (int f = it.u0 + lane; f < end; f += 32) {
    int q, l;
    flat_of(f, it, q, l);
    const int row = it.table + q;
    const int nnz = __ldg(c.csr_nnz + row);
    T acc = ldg(static_cast<const T*>(c.csr_rhs) + row);
    // wide rows (reconstruction-and-quadrature, folded rows) go in blocks
    // of W entries, each loaded as vectors, in entry order; a row of width
    // W is one block (the padded entries are dropped by the selects)
    const int nb = WIDE ? nnz : 1;
    for (int b0 = 0; b0 < nb; b0 += W) {
      int off[W], slot[W];
      T a[W], x[W];
      load_ell<T, W>(c, it.src_org + q * RW + b0, common, off, a, slot);
      if (common) {
        const T* xl = sb + l * it.src_ls;
#pragma unroll
        for (int j = 0; j < W; ++j) x[j] = ldg(xl + off[j]);
      } else {
#pragma unroll
        for (int j = 0; j < W; ++j) {
          x[j] = T(0);
          if (b0 + j < nnz)
            x[j] = ldg(static_cast<const T*>(c.slots[slot[j]]) +
                       (off[j] + l * __ldg(c.slot_ls + slot[j])));
        }
      }
#pragma unroll
      for (int j = 0; j < W; ++j) acc = b0 + j < nnz ? fma(a[j], x[j], acc) : acc;
    }
    dbase[dst_cell(it, c, q) + l * it.dst_ls] = acc;
  }
}

// A cell times a chunk of levels per lane, a whole ELL row of width W.
template <typename T, int W, int CH, bool WIDE>
__device__ void csr_chunk_w(const Item& it, const Ptrs& P, const Ctx& c, int lane) {
  const int end = it.u0 + it.nunits;
  const int ls = it.dst_ls;
  const int chn = it.mode;
  const T* sb = static_cast<const T*>(P.s);
  const bool common = sb != nullptr;
  const int RW = it.p;  // the row width: W, or a multiple of 8 for wide rows
  for (int u = it.u0 + lane; u < end; u += 32) {
    int q, ch;
    unit_of(u, it, q, ch);
    const int l0 = ch * chn;
    const int nl = min(chn, (int)it.lev.d - l0);
    const int row = it.table + q;
    const int nnz = __ldg(c.csr_nnz + row);
    T* d = static_cast<T*>(P.d) + (dst_cell(it, c, q) + l0 * ls);
    const T rhs = ldg(static_cast<const T*>(c.csr_rhs) + row);
    T acc[CH];
#pragma unroll
    for (int l = 0; l < CH; ++l) acc[l] = T(0);
    const int nb = WIDE ? nnz : 1;  // a row of width W: one block
    for (int b0 = 0; b0 < nb; b0 += W) {  // wide rows: blocks of W entries
      int off[W], slot[W];
      T a[W];
      load_ell<T, W>(c, it.src_org + q * RW + b0, common, off, a, slot);
      if (common) {  // padding entries read offset 0 of the slot, dropped below
        const int sls = it.src_ls;
#pragma unroll
        for (int j = 0; j < W; ++j) {
          const T* xs = sb + (off[j] + l0 * sls);
          const T aj = b0 + j < nnz ? a[j] : T(0);
#pragma unroll
          for (int l = 0; l < CH; ++l)
            if (l < nl) {
              const T xv = ldg(xs + l * sls);
              acc[l] = b0 + j < nnz ? fma(aj, xv, acc[l]) : acc[l];
            }
        }
      } else {
#pragma unroll
        for (int j = 0; j < W; ++j)
          if (b0 + j < nnz) {
            const int sls = __ldg(c.slot_ls + slot[j]);
            const T* xs = static_cast<const T*>(c.slots[slot[j]]) + (off[j] + l0 * sls);
#pragma unroll
            for (int l = 0; l < CH; ++l)
              if (l < nl) acc[l] = fma(a[j], ldg(xs + l * sls), acc[l]);
          }
      }
      }
#pragma unroll
      for (int l = 0; l < CH; ++l)
        if (l < nl) d[l * ls] = acc[l] + rhs;
    }
}

// Rows are processed E entries at a time: the E offsets and values load
// together, then the E x E-level source loads, so one row costs two memory
// latencies per E entries instead of two per entry.
constexpr int kCsrBatch = 8;

template <typename T, int CH>
__device__ void csr_chunk(const Item& it, const Ptrs& P, const Ctx& c, int lane) {
  constexpr int E = kCsrBatch;
  const int end = it.u0 + it.nunits;
  const int ls = it.dst_ls;
  const int chn = it.mode;
  const int W = it.p;
  const T* val = static_cast<const T*>(c.csr_val);
  for (int u = it.u0 + lane; u < end; u += 32) {
    int q, ch;
    unit_of(u, it, q, ch);
    const int l0 = ch * chn;
    const int nl = min(chn, (int)it.lev.d - l0);
    const int row = it.table + q;
    const int nnz = __ldg(c.csr_nnz + row);
    const int e0 = it.src_org + q * W;
    T* d = static_cast<T*>(P.d) + (dst_cell(it, c, q) + l0 * ls);
    T acc[CH];
#pragma unroll
    for (int l = 0; l < CH; ++l) acc[l] = T(0);
    for (int eb = 0; eb < nnz; eb += E) {
      const T* xs[E];
      int sl[E];
      T a[E];
#pragma unroll
      for (int e = 0; e < E; ++e)
        if (eb + e < nnz) {
          xs[e] = csr_src<T>(it, P, c, e0 + eb + e, l0, sl[e]);
          a[e] = ldg(val + e0 + eb + e);
        }
#pragma unroll
      for (int e = 0; e < E; ++e)
        if (eb + e < nnz) {
#pragma unroll
          for (int l = 0; l < CH; ++l)
            if (l < nl) acc[l] = fma(a[e], ldg(xs[e] + l * sl[e]), acc[l]);
        }
    }
    const T rhs = ldg(static_cast<const T*>(c.csr_rhs) + row);
#pragma unroll
    for (int l = 0; l < CH; ++l)
      if (l < nl) d[l * ls] = acc[l] + rhs;
  }
}

template <typename T>
__device__ void csr_flat(const Item& it, const Ptrs& P, const Ctx& c, int lane) {
  constexpr int E = kCsrBatch;
  const int end = it.u0 + it.nunits;
  const int W = it.p;
  const T* val = static_cast<const T*>(c.csr_val);
  T* dbase = static_cast<T*>(P.d);
  for (int f = it.u0 + lane; f < end; f += 32) {
    int q, l;
    flat_of(f, it, q, l);
    const int row = it.table + q;
    const int nnz = __ldg(c.csr_nnz + row);
    const int e0 = it.src_org + q * W;
    T acc = ldg(static_cast<const T*>(c.csr_rhs) + row);
    for (int eb = 0; eb < nnz; eb += E) {
      T x[E], a[E];
#pragma unroll
      for (int e = 0; e < E; ++e)
        if (eb + e < nnz) {
          int sls;
          x[e] = ldg(csr_src<T>(it, P, c, e0 + eb + e, l, sls));
          a[e] = ldg(val + e0 + eb + e);
        }
#pragma unroll
      for (int e = 0; e < E; ++e)
        if (eb + e < nnz) acc = fma(a[e], x[e], acc);
    }
    dbase[dst_cell(it, c, q) + l * it.dst_ls] = acc;
  }
}

// ---------------------------------------------------------------------------
// adjoint gather: x_bar_j += sum_i A_ij y_bar_i over the stored transpose,
// entries in ascending ghost order (deterministic, no atomics)
// ---------------------------------------------------------------------------
constexpr int kAdjBatch = 4;

template <typename T, int CH>
__device__ void adj_chunk(const Item& it, const Ptrs& P, const Ctx& c, int lane) {
  constexpr int E = kAdjBatch;
  const int end = it.u0 + it.nunits;
  const int chn = it.mode;
  const T* wv = static_cast<const T*>(c.aent_w);
  for (int u = it.u0 + lane; u < end; u += 32) {
    int q, ch;
    unit_of(u, it, q, ch);
    const int l0 = ch * chn;
    const int nl = min(chn, (int)it.lev.d - l0);
    const int r = it.table + q;
    const int ls = it.dst_ls;
    T* xb = static_cast<T*>(P.d) + (__ldg(c.arow_off + r) + l0 * ls);
    const int e0 = (int)__ldg(c.adj_ptr + r), e1 = (int)__ldg(c.adj_ptr + r + 1);
    T acc[CH];
#pragma unroll
    for (int l = 0; l < CH; ++l) acc[l] = (l < nl) ? xb[l * ls] : T(0);
    for (int eb = e0; eb < e1; eb += E) {
      const T* ys[E];
      int gl[E];
      T a[E];
#pragma unroll
      for (int e = 0; e < E; ++e)
        if (eb + e < e1) {
          const T* ybase;
          if (P.s) {
            ybase = static_cast<const T*>(P.s);
            gl[e] = it.src_ls;
          } else {
            const int gs = __ldg(c.aent_slot + eb + e);
            gl[e] = __ldg(c.slot_ls + gs);
            ybase = static_cast<const T*>(c.slots[gs]);
          }
          ys[e] = ybase + (__ldg(c.aent_off + eb + e) + l0 * gl[e]);
          a[e] = ldg(wv + eb + e);
        }
#pragma unroll
      for (int e = 0; e < E; ++e)
        if (eb + e < e1) {
#pragma unroll
          for (int l = 0; l < CH; ++l)
            if (l < nl) acc[l] = fma(a[e], ys[e][l * gl[e]], acc[l]);
        }
    }
#pragma unroll
    for (int l = 0; l < CH; ++l)
      if (l < nl) xb[l * ls] = acc[l];
  }
}

template <typename T>
__device__ void adj_flat(const Item& it, const Ptrs& P, const Ctx& c, int lane) {
  constexpr int E = kAdjBatch;
  const int end = it.u0 + it.nunits;
  const T* wv = static_cast<const T*>(c.aent_w);
  for (int f = it.u0 + lane; f < end; f += 32) {
    int q, l;
    flat_of(f, it, q, l);
    const int r = it.table + q;
    T* xb = static_cast<T*>(P.d) + (__ldg(c.arow_off + r) + l * it.dst_ls);
    const int e0 = (int)__ldg(c.adj_ptr + r), e1 = (int)__ldg(c.adj_ptr + r + 1);
    T acc = *xb;
    for (int eb = e0; eb < e1; eb += E) {
      T y[E], a[E];
#pragma unroll
      for (int e = 0; e < E; ++e)
        if (eb + e < e1) {
          const T* yp;
          if (P.s) {
            yp = static_cast<const T*>(P.s) + (__ldg(c.aent_off + eb + e) + l * it.src_ls);
          } else {
            const int gs = __ldg(c.aent_slot + eb + e);
            yp = static_cast<const T*>(c.slots[gs]) +
                 (__ldg(c.aent_off + eb + e) + l * __ldg(c.slot_ls + gs));
          }
          y[e] = *yp;
          a[e] = ldg(wv + eb + e);
        }
#pragma unroll
      for (int e = 0; e < E; ++e)
        if (eb + e < e1) acc = fma(a[e], y[e], acc);
    }
    *xb = acc;
  }
}

// Kernel families: one kernel per family keeps each family's register
// budget (and so its occupancy) independent of the others.
template <typename T, int FAM, int MAXCH>
__device__ __forceinline__ void run_item(const Item& it, const Ptrs& P, const Ctx& c, int lane) {
  const bool flat = it.mode < 2 && it.mode != MODE_TILE;
  const bool ch8 = MAXCH > 4 && it.mode > 4;  // level chunks of up to 8
  if constexpr (FAM == FAM_STRUCT) {
    structured_flat<T>(it, P, c, lane);
  } else if constexpr (FAM == FAM_INTERP) {
    if (it.mode == MODE_TILE) {
      interp_tile<T>(it, P, c, lane);
    } else if (it.kind == IK_INTERP_PAIR) {
      if (flat)
        interp_flat<T, true>(it, P, c, lane);
      else if (ch8)
        interp_pair_chunk<T, (MAXCH > 4 ? 8 : 4)>(it, P, c, lane);
      else
        interp_pair_chunk<T, 4>(it, P, c, lane);
    } else {
      if (flat)
        interp_flat<T, false>(it, P, c, lane);
      else if (ch8)
        interp_scalar_chunk<T, (MAXCH > 4 ? 8 : 4)>(it, P, c, lane);
      else
        interp_scalar_chunk<T, 4>(it, P, c, lane);
    }
  } else if constexpr (FAM == FAM_CSR) {
    if (it.mode == MODE_TILE) {
      if (it.p % 8 == 0)
        csr_tile<T, 8>(it, P, c, lane);
      else
        csr_tile<T, 4>(it, P, c, lane);
    } else if (it.p == 8) {
      if (flat)
        csr_flat_w<T, 8, false>(it, P, c, lane);
      else if (ch8)
        csr_chunk_w<T, 8, (MAXCH > 4 ? 8 : 4), false>(it, P, c, lane);
      else
        csr_chunk_w<T, 8, 4, false>(it, P, c, lane);
    } else if (it.p % 8 == 0) {  // wide rows in blocks of 8
      if (flat)
        csr_flat_w<T, 8, true>(it, P, c, lane);
      else if (ch8)
        csr_chunk_w<T, 8, (MAXCH > 4 ? 8 : 4), true>(it, P, c, lane);
      else
        csr_chunk_w<T, 8, 4, true>(it, P, c, lane);
    } else if (it.p == 4) {
      if (flat)
        csr_flat_w<T, 4, false>(it, P, c, lane);
      else if (ch8)
        csr_chunk_w<T, 4, (MAXCH > 4 ? 8 : 4), false>(it, P, c, lane);
      else
        csr_chunk_w<T, 4, 4, false>(it, P, c, lane);
    } else if (flat) {
      csr_flat<T>(it, P, c, lane);
    } else if (ch8) {
      csr_chunk<T, (MAXCH > 4 ? 8 : 4)>(it, P, c, lane);
    } else {
      csr_chunk<T, 4>(it, P, c, lane);
    }
  } else {
    if (it.mode == MODE_TILE)
      adj_tile<T>(it, P, c, lane);
    else if (it.kind == IK_ADD && c.vec_runs)
      runs_vec<T, RUN_ADD>(it, P, c, lane);
    else if (it.kind == IK_ADD)
      add_runs<T>(it, P, c, lane);
    else if (flat)
      adj_flat<T>(it, P, c, lane);
    else if (ch8)
      adj_chunk<T, (MAXCH > 4 ? 8 : 4)>(it, P, c, lane);
    else
      adj_chunk<T, 4>(it, P, c, lane);
  }
}

// All forward item kinds in one kernel (the persistent work-list launch):
// dispatch on the item's kind.  That kernel holds level chunks of at most 4
// (the plan cuts its units so), which keeps its register budget; the family
// kernels take chunks of up to 8.
template <typename T, int FAM>
__device__ __forceinline__ void run_work(const Item& it, const Ptrs& P, const Ctx& c, int lane) {
  if constexpr (FAM == FAM_ALL) {
    switch (it.kind) {
      case IK_ZERO:
      case IK_CONST:
      case IK_MAP: run_item<T, FAM_STRUCT, 4>(it, P, c, lane); break;
      case IK_INTERP:
      case IK_INTERP_PAIR: run_item<T, FAM_INTERP, 4>(it, P, c, lane); break;
      case IK_CSR: run_item<T, FAM_CSR, 4>(it, P, c, lane); break;
      default: run_item<T, FAM_ADJ, 4>(it, P, c, lane); break;
    }
  } else {
    run_item<T, FAM, 8>(it, P, c, lane);
  }
}

static_assert(sizeof(Item) == 32 * 4, "an Item is loaded as one word per lane");

// Resident CTAs the register budget is set for: the structured family is
// lean (48 registers, 40 warps per SM); the table families get 64.
template <int FAM, int THREADS> struct Occ {
#ifndef BC_STRUCT_WARPS
#define BC_STRUCT_WARPS 40
#endif
#ifndef BC_ALL_WARPS
#define BC_ALL_WARPS 32
#endif
  // the kernel of every kind carries the union of the paths at 64
  // registers (32 warps per SM): no spills in the plain grid; the
  // persistent loop spills some but measured faster than at 16 or 24 warps
  static constexpr int kWarps =
      FAM == FAM_STRUCT ? BC_STRUCT_WARPS : (FAM == FAM_ALL ? BC_ALL_WARPS : 32);
  // resident CTAs asked of the register allocator: the warp budget in CTAs,
  // at least 1 and at most 32 (the SM's CTA limit)
  static constexpr int kBlocksRaw = (kWarps * 32) / THREADS;
  static constexpr int kMinBlocks = kBlocksRaw < 1 ? 1 : (kBlocksRaw > 32 ? 32 : kBlocksRaw);
};

constexpr int kWordDst = offsetof(Item, dst_slot) / 4;
constexpr int kWordDst2 = offsetof(Item, dst_slot2) / 4;
constexpr int kWordSrc = offsetof(Item, src_slot) / 4;

// The lanes holding an item's slot words look up the slot pointers.
__device__ __forceinline__ void* lookup_slot(const Ctx& c, int word, int lane) {
  return ((lane == kWordDst || lane == kWordDst2 || lane == kWordSrc) && word >= 0)
             ? c.slots[word]
             : nullptr;
}

__device__ __forceinline__ Ptrs gather_ptrs(void* mine) {
  const unsigned long long v = reinterpret_cast<unsigned long long>(mine);
  Ptrs P;
  P.d = reinterpret_cast<void*>(__shfl_sync(0xffffffffu, v, kWordDst));
  P.d2 = reinterpret_cast<void*>(__shfl_sync(0xffffffffu, v, kWordDst2));
  P.s = reinterpret_cast<const void*>(__shfl_sync(0xffffffffu, v, kWordSrc));
  P.stage = nullptr;
  return P;
}

// Shared memory for staged boxes: one area per warp (Ctx::stage_warp bytes:
// 2 KB for interpolation and transpose tiles, 4 KB when the list has CSR
// tiles) in the kernels that run interpolation, CSR or transpose-gather
// items, as dynamic shared memory that only launches of lists with staged
// tiles request: a kernel that reserves no shared memory keeps the SM's
// default split of L1 and shared memory and shares SMs with the structured
// kernel beside it (the 512-block step, levels innermost: 51.1 us with a
// stage reserved in the CSR kernel, 44.9 us without).
template <int FAM, int THREADS>
struct Stage {
  static constexpr int kWarps = FAM != FAM_STRUCT ? THREADS / 32 : 0;
};

// dynamic shared memory of a launch with `stage` bytes per warp (the
// kernel's limit raised first where that exceeds 48 KB: 512 threads with
// CSR tiles)
template <int FAM, int THREADS, typename K>
int stage_smem(K kernel, int stage) {
  const int bytes = Stage<FAM, THREADS>::kWarps * stage;
  if (bytes > 48 * 1024)
    (void)cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  return bytes;
}

// Plain grid: warp w of CTA b processes item b * warps + w.
template <typename T, int THREADS, int FAM>
__global__ void __launch_bounds__(THREADS, (Occ<FAM, THREADS>::kMinBlocks))
    k_items(Ctx c, const Item* __restrict__ items, int nitems) {
  __shared__ Item sit[THREADS / 32];
  extern __shared__ __align__(16) unsigned char stage[];  // Stage, when requested
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int idx = blockIdx.x * (THREADS / 32) + warp;
  if (idx >= nitems) return;
  const int w = __ldg(reinterpret_cast<const int*>(items + idx) + lane);
  reinterpret_cast<int*>(&sit[warp])[lane] = w;
  Ptrs P = gather_ptrs(lookup_slot(c, w, lane));
  if (Stage<FAM, THREADS>::kWarps) P.stage = stage + warp * c.stage_warp;
  __syncwarp();
  run_work<T, FAM>(sit[warp], P, c, lane);
}

// Streaming form: a grid of resident warps walks the items with a fixed
// stride; while a warp works on one item, the descriptor of the item after
// next and the slot pointers of the next one are already in flight.  No warp
// waits on another.
template <typename T, int THREADS, int FAM>
__global__ void __launch_bounds__(THREADS, (Occ<FAM, THREADS>::kMinBlocks))
    k_stream(Ctx c, const Item* __restrict__ items, int nitems) {
  __shared__ Item sit[THREADS / 32];
  extern __shared__ __align__(16) unsigned char stage[];  // Stage, when requested
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int stride = gridDim.x * (THREADS / 32);
  const int* iw = reinterpret_cast<const int*>(items);
  int cur = blockIdx.x * (THREADS / 32) + warp;
  if (cur >= nitems) return;
  int w_cur = __ldg(iw + (int64_t)cur * 32 + lane);
  void* p_cur = lookup_slot(c, w_cur, lane);
  int nxt = cur + stride;
  int w_nxt = nxt < nitems ? __ldg(iw + (int64_t)nxt * 32 + lane) : 0;
  for (;;) {
    reinterpret_cast<int*>(&sit[warp])[lane] = w_cur;
    void* p_nxt = nxt < nitems ? lookup_slot(c, w_nxt, lane) : nullptr;
    const int nxt2 = nxt + stride;
    const int w_nxt2 = nxt2 < nitems ? __ldg(iw + (int64_t)nxt2 * 32 + lane) : 0;
    Ptrs P = gather_ptrs(p_cur);
    if (Stage<FAM, THREADS>::kWarps) P.stage = stage + warp * c.stage_warp;
    __syncwarp();
    run_work<T, FAM>(sit[warp], P, c, lane);
    __syncwarp();
    if (nxt >= nitems) break;
    w_cur = w_nxt;
    p_cur = p_nxt;
    nxt = nxt2;
    w_nxt = w_nxt2;
  }
}

// Persistent work-list form: a resident grid whose warps claim items from
// device counters (lane 0's atomic is issued while the warp still works on
// an earlier item; nothing ever waits on another warp).  Claims on one
// address serialise in its L2 slice, so the list is dealt over kSpread
// counters, each in its own 256-byte line: counter k hands out items k,
// k + kSpread, k + 2 kSpread, ... (longest first within each), a warp starts
// on counter (warp index mod kSpread) and moves to the next counter when its
// own runs dry, until it has found all kSpread dry in a row.  Three items
// are in a warp's pipeline: the one it works on, the next one (its slot
// pointers already loaded) and the one after (its descriptor in flight),
// plus the claim of a fourth.  A warp that stops counts itself done; the
// last warp of the launch puts every counter back to zero, so the next
// launch on the stream (or the next replay of a captured graph) starts
// from item 0.
template <typename T, int THREADS, int FAM>
__global__ void __launch_bounds__(THREADS, (Occ<FAM, THREADS>::kMinBlocks))
    k_persist(Ctx c, const Item* __restrict__ items, int nitems, unsigned* __restrict__ ctr) {
  constexpr unsigned FULL = 0xffffffffu;
  constexpr unsigned S = kSpread;
  __shared__ Item sit[THREADS / 32];
  extern __shared__ __align__(16) unsigned char stage[];  // Stage, when requested
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int* iw = reinterpret_cast<const int*>(items);
  const unsigned n = (unsigned)nitems;
  unsigned k = (blockIdx.x * (THREADS / 32) + warp) % S;  // this warp's counter
  unsigned dry = 0;                                        // dry counters in a row
  bool more = true;
  auto counter = [&](unsigned j) { return ctr + (1 + j) * kCtrStride; };
  auto issue = [&]() -> unsigned { return (more && lane == 0) ? atomicAdd(counter(k), 1u) : 0u; };
  // the item a claim `raw` on counter k gave, or the next counter's
  auto finish = [&](unsigned raw) -> unsigned {
    if (!more) return n;
    unsigned v = __shfl_sync(FULL, raw, 0) * S + k;
    while (v >= n) {
      if (++dry == S) {
        more = false;
        return n;
      }
      k = (k + 1) % S;
      const unsigned r = lane == 0 ? atomicAdd(counter(k), 1u) : 0u;
      v = __shfl_sync(FULL, r, 0) * S + k;
    }
    dry = 0;
    return v;
  };
  auto words = [&](unsigned i) -> int { return i < n ? __ldg(iw + (size_t)i * 32 + lane) : 0; };
  // prologue: the first three items
  unsigned a = finish(issue());
  int wa = words(a);
  unsigned b = finish(issue());
  int wb = words(b);
  void* pa = a < n ? lookup_slot(c, wa, lane) : nullptr;
  unsigned cn = finish(issue());
  int wc = words(cn);
  void* pb = b < n ? lookup_slot(c, wb, lane) : nullptr;
  while (a < n) {
    const unsigned raw = issue();  // claim of the fourth item, in flight
    reinterpret_cast<int*>(&sit[warp])[lane] = wa;
    Ptrs P = gather_ptrs(pa);
    if (Stage<FAM, THREADS>::kWarps) P.stage = stage + warp * c.stage_warp;
    __syncwarp();
    run_work<T, FAM>(sit[warp], P, c, lane);
    __syncwarp();
    const unsigned d = finish(raw);
    const int wd = words(d);
    void* pc = cn < n ? lookup_slot(c, wc, lane) : nullptr;
    a = b;
    wa = wb;
    pa = pb;
    b = cn;
    wb = wc;
    pb = pc;
    cn = d;
    wc = wd;
  }
  if (lane == 0) {
    __threadfence();
    const unsigned warps = gridDim.x * (THREADS / 32);
    if (atomicAdd(ctr, 1u) == warps - 1) {
      for (unsigned j = 0; j < S; ++j) atomicExch(counter(j), 0u);
      atomicExch(ctr, 0u);
    }
  }
}

template <typename T, int THREADS, int FAM>
cudaError_t launch_t(const Ctx& c, const Item* items, int nitems, int grid, int stage,
                     cudaStream_t s) {
  const int wpb = THREADS / 32;
  const int need = (nitems + wpb - 1) / wpb;
  if (grid <= 0) {
    const int smem = stage_smem<FAM, THREADS>(k_items<T, THREADS, FAM>, stage);
    k_items<T, THREADS, FAM><<<need, THREADS, smem, s>>>(c, items, nitems);
  } else {
    const int smem = stage_smem<FAM, THREADS>(k_stream<T, THREADS, FAM>, stage);
    k_stream<T, THREADS, FAM><<<grid < need ? grid : need, THREADS, smem, s>>>(c, items, nitems);
  }
  return cudaGetLastError();
}

template <typename T, int THREADS, int FAM>
cudaError_t persist_t(const Ctx& c, const Item* items, int nitems, int ctas_per_sm, int sms,
                      unsigned* ctr, int stage, cudaStream_t s) {
  const int smem = stage_smem<FAM, THREADS>(k_persist<T, THREADS, FAM>, stage);
  int fit = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fit, k_persist<T, THREADS, FAM>, THREADS,
                                                    smem) != cudaSuccess || fit < 1)
    fit = 1;
  const int per_sm = ctas_per_sm > 0 ? (ctas_per_sm < fit ? ctas_per_sm : fit) : fit;
  const int wpb = THREADS / 32;
  const int need = (nitems + wpb - 1) / wpb;
  const int grid = per_sm * sms < need ? per_sm * sms : need;
  k_persist<T, THREADS, FAM><<<grid, THREADS, smem, s>>>(c, items, nitems, ctr);
  return cudaGetLastError();
}

template <typename T, int FAM>
cudaError_t persist_fam(const Ctx& c, const Item* items, int nitems, int threads,
                        int ctas_per_sm, int sms, unsigned* ctr, int st, cudaStream_t s) {
  switch (threads) {
    case 64: return persist_t<T, 64, FAM>(c, items, nitems, ctas_per_sm, sms, ctr, st, s);
    case 128: return persist_t<T, 128, FAM>(c, items, nitems, ctas_per_sm, sms, ctr, st, s);
    case 512: return persist_t<T, 512, FAM>(c, items, nitems, ctas_per_sm, sms, ctr, st, s);
    default: return persist_t<T, 256, FAM>(c, items, nitems, ctas_per_sm, sms, ctr, st, s);
  }
}

template <typename T>
cudaError_t persist_any(int fam, const Ctx& c, const Item* items, int nitems, int threads,
                        int ctas_per_sm, int sms, unsigned* ctr, int st, cudaStream_t s) {
  switch (fam) {
    case FAM_STRUCT:
      return persist_fam<T, FAM_STRUCT>(c, items, nitems, threads, ctas_per_sm, sms, ctr, st, s);
    case FAM_INTERP:
      return persist_fam<T, FAM_INTERP>(c, items, nitems, threads, ctas_per_sm, sms, ctr, st, s);
    case FAM_CSR:
      return persist_fam<T, FAM_CSR>(c, items, nitems, threads, ctas_per_sm, sms, ctr, st, s);
    case FAM_ADJ:
      return persist_fam<T, FAM_ADJ>(c, items, nitems, threads, ctas_per_sm, sms, ctr, st, s);
    default:
      return persist_fam<T, FAM_ALL>(c, items, nitems, threads, ctas_per_sm, sms, ctr, st, s);
  }
}

// resident CTAs per SM of `kernel` with its stage requested or not
template <int FAM, int THREADS, typename K>
int fit_of(K kernel, int stage) {
  const int smem = stage_smem<FAM, THREADS>(kernel, stage);
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, THREADS, smem) != cudaSuccess)
    return 1;
  return n > 0 ? n : 1;
}

template <typename T, int FAM>
int persist_fit_fam(int threads, int st) {
  switch (threads) {
    case 64: return fit_of<FAM, 64>(k_persist<T, 64, FAM>, st);
    case 128: return fit_of<FAM, 128>(k_persist<T, 128, FAM>, st);
    case 512: return fit_of<FAM, 512>(k_persist<T, 512, FAM>, st);
    default: return fit_of<FAM, 256>(k_persist<T, 256, FAM>, st);
  }
}

template <typename T>
int persist_fit_any(int fam, int threads, int st) {
  switch (fam) {
    case FAM_STRUCT: return persist_fit_fam<T, FAM_STRUCT>(threads, st);
    case FAM_INTERP: return persist_fit_fam<T, FAM_INTERP>(threads, st);
    case FAM_CSR: return persist_fit_fam<T, FAM_CSR>(threads, st);
    case FAM_ADJ: return persist_fit_fam<T, FAM_ADJ>(threads, st);
    default: return persist_fit_fam<T, FAM_ALL>(threads, st);
  }
}

template <typename T, int FAM>
cudaError_t launch_fam(const Ctx& c, const Item* items, int nitems, int threads,
                       int grid, int st, cudaStream_t s) {
  switch (threads) {
    case 32: return launch_t<T, 32, FAM>(c, items, nitems, grid, st, s);
    case 64: return launch_t<T, 64, FAM>(c, items, nitems, grid, st, s);
    case 128: return launch_t<T, 128, FAM>(c, items, nitems, grid, st, s);
    case 512: return launch_t<T, 512, FAM>(c, items, nitems, grid, st, s);
    default: return launch_t<T, 256, FAM>(c, items, nitems, grid, st, s);
  }
}

template <typename T, int FAM>
int resident_fam(int threads, int st) {
  switch (threads) {
    case 32: return fit_of<FAM, 32>(k_stream<T, 32, FAM>, st);
    case 64: return fit_of<FAM, 64>(k_stream<T, 64, FAM>, st);
    case 128: return fit_of<FAM, 128>(k_stream<T, 128, FAM>, st);
    case 512: return fit_of<FAM, 512>(k_stream<T, 512, FAM>, st);
    default: return fit_of<FAM, 256>(k_stream<T, 256, FAM>, st);
  }
}

template <typename T>
cudaError_t launch_any(int fam, const Ctx& c, const Item* items, int nitems,
                       int threads, int grid, int st, cudaStream_t s) {
  switch (fam) {
    case FAM_STRUCT: return launch_fam<T, FAM_STRUCT>(c, items, nitems, threads, grid, st, s);
    case FAM_INTERP: return launch_fam<T, FAM_INTERP>(c, items, nitems, threads, grid, st, s);
    case FAM_CSR: return launch_fam<T, FAM_CSR>(c, items, nitems, threads, grid, st, s);
    case FAM_ALL: return launch_fam<T, FAM_ALL>(c, items, nitems, threads, grid, st, s);
    default: return launch_fam<T, FAM_ADJ>(c, items, nitems, threads, grid, st, s);
  }
}

template <typename T>
int resident_any(int fam, int threads, int st) {
  switch (fam) {
    case FAM_STRUCT: return resident_fam<T, FAM_STRUCT>(threads, st);
    case FAM_INTERP: return resident_fam<T, FAM_INTERP>(threads, st);
    case FAM_CSR: return resident_fam<T, FAM_CSR>(threads, st);
    case FAM_ALL: return resident_fam<T, FAM_ALL>(threads, st);
    default: return resident_fam<T, FAM_ADJ>(threads, st);
  }
}

}  // namespace

cudaError_t launch_family(int dtype, int family, const Ctx& ctx,
                          const Item* items, int nitems, int threads, int grid,
                          int stage, cudaStream_t s) {
  if (nitems <= 0) return cudaSuccess;
  Ctx c = ctx;
  c.stage_warp = stage;
  return dtype == 1 ? launch_any<double>(family, c, items, nitems, threads, grid, stage, s)
                    : launch_any<float>(family, c, items, nitems, threads, grid, stage, s);
}

cudaError_t launch_persistent(int dtype, int family, const Ctx& ctx, const Item* items,
                              int nitems, int threads, int ctas_per_sm, int sms,
                              unsigned* counter, int stage, cudaStream_t s) {
  if (nitems <= 0) return cudaSuccess;
  Ctx c = ctx;
  c.stage_warp = stage;
  return dtype == 1 ? persist_any<double>(family, c, items, nitems, threads, ctas_per_sm, sms,
                                          counter, stage, s)
                    : persist_any<float>(family, c, items, nitems, threads, ctas_per_sm, sms,
                                         counter, stage, s);
}

int persistent_fit(int dtype, int family, int threads, int stage) {
  return dtype == 1 ? persist_fit_any<double>(family, threads, stage)
                    : persist_fit_any<float>(family, threads, stage);
}

int resident_ctas(int dtype, int family, int threads, int stage) {
  return dtype == 1 ? resident_any<double>(family, threads, stage)
                    : resident_any<float>(family, threads, stage);
}

}  // namespace bcg
