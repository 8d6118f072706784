"""The boundary from plain C: the header compiles as strict C99, its struct
layouts match the Python binding's, and a C program links the library and
builds host-only plans (no GPU) -- a periodic 2-D block and the six panels
of a cubed sphere with reconstruction-and-quadrature edges -- reading the
rows back with bc_plan_export_csr and checking them against closed forms."""
import ctypes
import os
import shutil
import subprocess

import pytest

from paper_2605_14780_gb300 import bc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PROGRAM = r"""
#include <stddef.h>
#include <stdio.h>
#include <stdlib.h>
#include "bc.h"

static int check(bc_status st, const char* what) {
  if (st != BC_OK) {
    printf("FAIL %s: %s (%s)\n", what, bc_status_string(st), bc_last_error());
    return 1;
  }
  return 0;
}

/* one 2-D block, levels innermost, circular on both axes (Sec. III-B fmap),
   edges by the product of the two maps */
static int periodic_block(void) {
  const int n = 12, h = 2, L = 3;
  const int F = n + 2 * h;
  bc_block blk = {{n, n, 1}, {h, h, 0}, L, 1, {L, (int64_t)L * F, (int64_t)L * F * F}, 1};
  bc_grid grid = {BC_F64, 1, &blk};
  int32_t comp0 = 0;
  bc_submatrix subs[8];
  int ns = 0;
  for (int a = -1; a <= 1; ++a)
    for (int b = -1; b <= 1; ++b) {
      if (a == 0 && b == 0) continue;
      bc_submatrix m = {0};
      m.kind = BC_MAP;
      m.block = 0;
      m.ncomps = 1;
      m.comps = &comp0;
      m.src_block = 0;
      m.perm[0] = 0; m.perm[1] = 1; m.perm[2] = 2;
      m.sign[0] = m.sign[1] = m.sign[2] = 1;
      const int side[2] = {a, b};
      for (int d = 0; d < 2; ++d) {
        m.lo[d] = side[d] < 0 ? -h : (side[d] > 0 ? n : 0);
        m.hi[d] = side[d] < 0 ? 0 : (side[d] > 0 ? n + h : n);
        m.offset[d] = side[d] < 0 ? n : (side[d] > 0 ? -n : 0);
      }
      m.lo[2] = 0;
      m.hi[2] = 1;
      subs[ns++] = m;
    }
  bc_plan_opts opts = {0};
  opts.host_only = 1;
  opts.strict_cover = 1;
  bc_plan* plan = NULL;
  if (check(bc_plan_create(&grid, subs, ns, &opts, &plan), "periodic plan")) return 1;
  bc_stats st;
  if (check(bc_plan_stats(plan, &st), "stats")) return 1;
  int64_t nrows = 0, nnz = 0;
  if (check(bc_plan_export_csr(plan, &nrows, &nnz, NULL, NULL, NULL, NULL, NULL, NULL, NULL),
            "export sizes")) return 1;
  int32_t* rs = malloc(sizeof(int32_t) * nrows);
  int64_t* ro = malloc(sizeof(int64_t) * nrows);
  int64_t* rp = malloc(sizeof(int64_t) * (nrows + 1));
  int32_t* cs = malloc(sizeof(int32_t) * nnz);
  int64_t* co = malloc(sizeof(int64_t) * nnz);
  double* v = malloc(sizeof(double) * nnz);
  double* rhs = malloc(sizeof(double) * nrows);
  if (check(bc_plan_export_csr(plan, &nrows, &nnz, rs, ro, rp, cs, co, v, rhs), "export")) return 1;
  /* every row one unit entry at the periodic image of its cell */
  int bad = 0;
  for (int64_t r = 0; r < nrows; ++r) {
    const int64_t cell = ro[r] / L;
    const int i = (int)(cell % F) - h, j = (int)(cell / F) - h;
    const int si = (i + n) % n, sj = (j + n) % n;
    const int64_t want = ((int64_t)(sj + h) * F + (si + h)) * L;
    if (rp[r + 1] - rp[r] != 1 || v[rp[r]] != 1.0 || co[rp[r]] != want || rhs[r] != 0.0) ++bad;
  }
  printf("periodic %lld %lld %lld %d\n", (long long)st.ghost_values, (long long)nrows,
         (long long)nnz, bad);
  free(rs); free(ro); free(rp); free(cs); free(co); free(v); free(rhs);
  /* the apply entry points refuse a host-only plan */
  printf("apply %s\n", bc_status_string(bc_apply(plan, NULL, NULL)));
  bc_plan_destroy(plan);
  /* an overlap is reported with a message */
  subs[1] = subs[0];
  plan = NULL;
  const bc_status st2 = bc_plan_create(&grid, subs, ns, &opts, &plan);
  printf("overlap %s %d %d\n", bc_status_string(st2), plan == NULL, bc_last_error()[0] != 0);
  return 0;
}

/* six panels of N x N with halo h, edges by reconstruction-and-quadrature
   rows (p = 4, 2 x 2 Gauss points), corners left uncovered */
static int quadrature_sphere(void) {
  const int N = 8, h = 2, p = 4;
  const int F = N + 2 * h;
  bc_block blk = {{N, N, 1}, {h, h, 0}, 1, 1, {1, F, (int64_t)F * F}, 1};
  bc_block blocks[6];
  for (int t = 0; t < 6; ++t) blocks[t] = blk;
  bc_grid grid = {BC_F32, 6, blocks};
  int32_t comp0 = 0;
  bc_submatrix subs[24];
  int ns = 0;
  for (int P = 0; P < 6; ++P)
    for (int d = 0; d < 2; ++d)
      for (int side = 0; side < 2; ++side) {
        bc_submatrix m = {0};
        m.kind = BC_INTERP;
        m.block = P;
        m.ncomps = 1;
        m.comps = &comp0;
        m.p = p;
        m.geometry = BC_GEOM_CUBED_SPHERE_QUAD;
        m.nquad = 2;
        m.rot_comp[0] = m.rot_comp[1] = -1;
        for (int t = 0; t < 6; ++t) m.cs_panels[t] = t;
        m.lo[0] = m.lo[1] = 0;
        m.hi[0] = m.hi[1] = N;
        m.lo[d] = side ? N : -h;
        m.hi[d] = side ? N + h : 0;
        m.lo[2] = 0;
        m.hi[2] = 1;
        subs[ns++] = m;
      }
  bc_plan_opts opts = {0};
  opts.host_only = 1;
  bc_plan* plan = NULL;
  if (check(bc_plan_create(&grid, subs, ns, &opts, &plan), "quadrature plan")) return 1;
  int64_t nrows = 0, nnz = 0;
  if (check(bc_plan_export_csr(plan, &nrows, &nnz, NULL, NULL, NULL, NULL, NULL, NULL, NULL),
            "export sizes")) return 1;
  int32_t* rs = malloc(sizeof(int32_t) * nrows);
  int64_t* ro = malloc(sizeof(int64_t) * nrows);
  int64_t* rp = malloc(sizeof(int64_t) * (nrows + 1));
  int32_t* cs = malloc(sizeof(int32_t) * nnz);
  int64_t* co = malloc(sizeof(int64_t) * nnz);
  double* v = malloc(sizeof(double) * nnz);
  double* rhs = malloc(sizeof(double) * nrows);
  if (check(bc_plan_export_csr(plan, &nrows, &nnz, rs, ro, rp, cs, co, v, rhs), "export"))
    return 1;
  double worst = 0.0;
  for (int64_t r = 0; r < nrows; ++r) {
    double s = 0.0;
    for (int64_t e = rp[r]; e < rp[r + 1]; ++e) s += v[e];
    if (s - 1.0 > worst) worst = s - 1.0;
    if (1.0 - s > worst) worst = 1.0 - s;
  }
  printf("quadrature %lld %lld %.3g\n", (long long)nrows, (long long)nnz, worst);
  free(rs); free(ro); free(rp); free(cs); free(co); free(v); free(rhs);
  bc_plan_destroy(plan);
  return 0;
}

/* one 2-D block whose low x face extrapolates linearly, g_r = 2 v_{r-1} -
   v_{r-2}, reading the ghosts nearer the data: folded by h sweeps, every
   row holds two data entries (x0, x1) with weights (r + 2, -(r + 1)) */
static int folded_extrapolation(void) {
  const int n = 6, h = 3;
  const int F = n + 2 * h;
  bc_block blk = {{n, n, 1}, {h, h, 0}, 1, 1, {1, F, (int64_t)F * F}, 1};
  bc_grid grid = {BC_F64, 1, &blk};
  int32_t comp0 = 0;
  int64_t rp[3 * 6 + 1];
  int32_t cb[2 * 3 * 6], cc[2 * 3 * 6], ck[3 * 2 * 3 * 6];
  double v[2 * 3 * 6];
  int e = 0, r = 0;
  rp[0] = 0;
  for (int j = 0; j < n; ++j)
    for (int i = -h; i < 0; ++i) {       /* box order: axis 0 fastest */
      const int a = i + 1, b = i + 2;    /* v_{r-1}, v_{r-2} of depth r = -1 - i */
      cb[e] = 0; cc[e] = 0; ck[3 * e] = a; ck[3 * e + 1] = j; ck[3 * e + 2] = 0; v[e++] = 2.0;
      cb[e] = 0; cc[e] = 0; ck[3 * e] = b; ck[3 * e + 1] = j; ck[3 * e + 2] = 0; v[e++] = -1.0;
      rp[++r] = e;
    }
  bc_submatrix m = {0};
  m.kind = BC_CSR;
  m.block = 0;
  m.lo[0] = -h; m.hi[0] = 0;
  m.lo[1] = 0; m.hi[1] = n;
  m.lo[2] = 0; m.hi[2] = 1;
  m.ncomps = 1;
  m.comps = &comp0;
  m.row_ptr = rp;
  m.col_block = cb;
  m.col_comp = cc;
  m.col_ijk = ck;
  m.val = v;
  bc_plan_opts opts = {0};
  opts.host_only = 1;
  bc_plan* plan = NULL;
  const bc_status st0 = bc_plan_create(&grid, &m, 1, &opts, &plan);
  printf("unfolded %s\n", bc_status_string(st0));
  opts.ghost_sweeps = h;
  if (check(bc_plan_create(&grid, &m, 1, &opts, &plan), "folded plan")) return 1;
  int64_t nrows = 0, nnz = 0;
  if (check(bc_plan_export_csr(plan, &nrows, &nnz, NULL, NULL, NULL, NULL, NULL, NULL, NULL),
            "export sizes")) return 1;
  int32_t* rs = malloc(sizeof(int32_t) * nrows);
  int64_t* ro = malloc(sizeof(int64_t) * nrows);
  int64_t* p = malloc(sizeof(int64_t) * (nrows + 1));
  int32_t* cs = malloc(sizeof(int32_t) * nnz);
  int64_t* co = malloc(sizeof(int64_t) * nnz);
  double* w = malloc(sizeof(double) * nnz);
  double* rhs = malloc(sizeof(double) * nrows);
  if (check(bc_plan_export_csr(plan, &nrows, &nnz, rs, ro, p, cs, co, w, rhs), "export"))
    return 1;
  int bad = 0;
  for (int64_t q = 0; q < nrows; ++q) {
    const int i = (int)(ro[q] % F) - h;
    const int depth = -1 - i;
    const int64_t x0 = ro[q] - i, x1 = x0 + 1;      /* offsets of data cells (0, j), (1, j) */
    double w0 = 0.0, w1 = 0.0;
    for (int64_t t = p[q]; t < p[q + 1]; ++t) {
      if (co[t] == x0) w0 += w[t];
      else if (co[t] == x1) w1 += w[t];
      else ++bad;
    }
    if (w0 != depth + 2.0 || w1 != -(depth + 1.0)) ++bad;
  }
  printf("folded %lld %lld %d\n", (long long)nrows, (long long)nnz, bad);
  free(rs); free(ro); free(p); free(cs); free(co); free(w); free(rhs);
  bc_plan_destroy(plan);
  return 0;
}

int main(void) {
  printf("sizes %zu %zu %zu %zu %zu %zu\n", sizeof(bc_block), sizeof(bc_grid),
         sizeof(bc_submatrix), sizeof(bc_plan_opts), sizeof(bc_stats),
         offsetof(bc_submatrix, nquad));
  if (periodic_block()) return 1;
  if (quadrature_sphere()) return 1;
  if (folded_extrapolation()) return 1;
  return 0;
}
"""


@pytest.fixture(scope="module")
def program(tmp_path_factory):
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    lib = bc.library_path()
    if not os.path.exists(lib):
        from paper_2605_14780_gb300.build import build_library
        build_library()
    d = tmp_path_factory.mktemp("capi")
    src = d / "main.c"
    src.write_text(PROGRAM)
    exe = d / "main"
    libdir = os.path.dirname(lib)
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic",
                    "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe),
                    "-L", libdir, "-lbcgb300", f"-Wl,-rpath,{libdir}"], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0, out.stdout + out.stderr
    return {ln.split()[0]: ln.split()[1:] for ln in out.stdout.splitlines()}


def test_struct_layouts_match_the_binding(program):
    sizes = [int(x) for x in program["sizes"]]
    assert sizes == [ctypes.sizeof(bc.BcBlock), ctypes.sizeof(bc.BcGrid),
                     ctypes.sizeof(bc.BcSubmatrix), ctypes.sizeof(bc.BcPlanOpts),
                     ctypes.sizeof(bc.BcStats), bc.BcSubmatrix.nquad.offset]


def test_periodic_rows_from_c(program):
    ghost, nrows, nnz, bad = (int(x) for x in program["periodic"])
    n, h, L = 12, 2, 3
    assert nrows == nnz == (n + 2 * h) ** 2 - n * n
    assert ghost == nrows * L
    assert bad == 0
    assert program["apply"] == ["BC_ERR_UNSUPPORTED"]
    assert program["overlap"] == ["BC_ERR_OVERLAP", "1", "1"]


def test_quadrature_rows_from_c(program):
    nrows, nnz, worst = program["quadrature"]
    N, h, p = 8, 2, 4
    assert int(nrows) == 6 * 4 * h * N
    assert int(nnz) == int(nrows) * p * p
    assert float(worst) < 1e-12


def test_folded_ghost_rows_from_c(program):
    assert program["unfolded"] == ["BC_ERR_COLUMN_NOT_DATA"]
    nrows, nnz, bad = (int(x) for x in program["folded"])
    assert nrows == 3 * 6 and nnz == 2 * nrows and bad == 0
