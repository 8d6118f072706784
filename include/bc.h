/*
 * bc.h -- C ABI of libbcgb300, the GB300 (sm_103a) ghost-fill library.
 *
 * The library applies every boundary condition of a block-structured grid as
 * one affine sparse operator (arxiv 2605.14780, Sec. III-B):
 *
 *     y_G = A x_D + b
 *
 * where x_D is the data region of all blocks, y_G their ghost region, and A
 * has columns in the data region only.  The operator is described by a list
 * of basic sub-matrices (Sec. IV-A, Table II), each covering a box of ghost
 * cells of one block (its is_valid region) with one row pattern (its
 * iterator): zero padding, tabulated constants (pure-function boundary),
 * index maps (halo copies, circular and symmetric maps, rotated maps of
 * Alg. 1), interpolation rows (user Itp, or cubed-sphere panel edges
 * generated on the GPU) and user CSR rows (Table III: F_NNZ/F_COL/F_DATA);
 * block-edge averaging rows (Sync) overwrite data cells that several blocks
 * store for one location, and bc_plan_create_pruned keeps only the ghost
 * values a given stencil reads (Sec. IV-C).
 *
 * Memory model
 *   * Fields are caller-owned device memory.  Each (block, component) pair is
 *     a "slot"; slot s = slot_base(block) + comp, slot_base being the prefix
 *     sum of ncomp over the blocks in order.  The slot pointer addresses the
 *     element (i, j, k) = (-h0, -h1, -h2) of level 0; element (i, j, k, level)
 *     lives at  ptr + (i+h0)*stride[0] + (j+h1)*stride[1] + (k+h2)*stride[2]
 *                    + level*level_stride.
 *   * The apply entry points take a DEVICE array of slot pointers (like the
 *     pointer arrays of batched BLAS calls).  It is read by the kernels at
 *     run time, so it may be rewritten between calls, and a CUDA graph
 *     captured around an apply keeps working when the array is updated in
 *     stream order.
 *   * A plan owns its device tables; every host array passed to
 *     bc_plan_create is copied and may be freed afterwards.
 *   * bc_apply, bc_apply_form and bc_apply_adjoint allocate nothing, never
 *     synchronise the host, and only enqueue kernels on the given stream
 *     (the batched form forks them onto plan-owned streams and joins them
 *     back, so it is graph-capturable).  One plan's applies must not run
 *     concurrently on several streams: the fork/join events, and the
 *     staging buffer of Sync rows, belong to the plan.
 *
 * Errors
 *   For tests of the error paths, BC_FAULT_INJECT=alloc:<n> in the
 *   environment makes the n-th device allocation of a bc_plan_create,
 *   bc_plan_create_pruned or bc_plan_autotune call fail (BC_ERR_NOMEM); the
 *   failure is made on the host, not on the GPU.
 *   Every entry point returns a bc_status.  The message of the last error of
 *   the calling thread is returned by bc_last_error().  Invalid descriptions
 *   are rejected by bc_plan_create before any device work.  Launch errors are
 *   returned at once; faults inside a kernel surface at the next
 *   synchronisation of the stream.
 */
#ifndef BC_GB300_H
#define BC_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum bc_status {
  BC_OK = 0,
  BC_ERR_INVALID_ARG = 1,     /* malformed description or argument          */
  BC_ERR_OVERLAP = 2,         /* two sub-matrices cover one value            */
  BC_ERR_COLUMN_NOT_DATA = 3, /* a column is not a data cell (Sec. III-B)    */
  BC_ERR_UNCOVERED = 4,       /* strict cover: a ghost value has no row      */
  BC_ERR_HALO_TOO_WIDE = 5,   /* a map's ghost depth exceeds the data extent */
  BC_ERR_OUT_OF_RANGE = 6,    /* a row lies outside its region (ghost cells,
                                 data cells for Sync rows)                  */
  BC_ERR_NOMEM = 7,           /* a host or device allocation failed          */
  BC_ERR_CUDA = 8,            /* a CUDA runtime call failed                  */
  BC_ERR_UNSUPPORTED = 9,     /* valid, but outside what this build handles  */
  BC_ERR_TIMEOUT = 10,        /* reserved: a bounded device wait gave up     */
  BC_ERR_GEOMETRY = 11        /* cubed-sphere geometry check failed          */
} bc_status;

typedef enum bc_dtype { BC_F32 = 0, BC_F64 = 1 } bc_dtype;

/* Kinds of basic sub-matrix (Sec. III-B, Table III). */
typedef enum bc_kind {
  BC_ZERO = 0,   /* A_ij = 0, b_i = 0                                      */
  BC_CONST = 1,  /* A_ij = 0, b_i = values[i]  (pure-function boundary)    */
  BC_MAP = 2,    /* one unit entry at an affine image of the ghost index   */
  BC_INTERP = 3, /* p-point row along an axis of a source block            */
  BC_CSR = 4,    /* user CSR rows                                           */
  BC_SYNC = 5    /* block-edge averaging: CSR rows on shared data cells     */
} bc_kind;

typedef enum bc_geometry {
  BC_GEOM_USER = 0,              /* interpolation tables given by the caller */
  BC_GEOM_CUBED_SPHERE = 1,      /* generated on the GPU for gnomonic panels */
  BC_GEOM_CUBED_SPHERE_QUAD = 2, /* cell averages by reconstruction and
                                    Gauss quadrature, generated on the host */
  BC_GEOM_CUBED_SPHERE_QUAD_CENTRED = 3 /* the same with patches centred on
                                    the ghost, which may read ghost values
                                    (needs bc_plan_opts.ghost_sweeps)     */
} bc_geometry;

/* Execution forms of the forward apply. */
typedef enum bc_form {
  BC_FORM_BATCHED = 0,  /* all work items in one launch (the default)      */
  BC_FORM_TYPEWIDE = 1, /* one launch per sub-matrix kind                  */
  BC_FORM_PER_BC = 2    /* one launch per basic sub-matrix                 */
} bc_form;

/* One block of the grid.  2-D blocks use n[2] = 1, h[2] = 0. */
typedef struct bc_block {
  int32_t n[3];         /* data extents per axis, axis 0 fastest          */
  int32_t h[3];         /* ghost width per axis (same on both sides)      */
  int32_t nlevels;      /* vertical levels; every row repeats per level   */
  int32_t ncomp;        /* components, each a slot of its own (<= 32)     */
  int64_t stride[3];    /* element strides of the three axes (> 0)        */
  int64_t level_stride; /* element stride between levels (> 0 if L > 1)  */
} bc_block;

typedef struct bc_grid {
  int32_t dtype;          /* bc_dtype of every field                      */
  int32_t nblocks;
  const bc_block* blocks; /* host array [nblocks]                          */
} bc_grid;

/*
 * One basic sub-matrix: the rows of the ghost cells in the box [lo, hi) of
 * `block` (cell coordinates of the data region; ghosts are negative or
 * >= n), for the listed components.  Unused fields are ignored; set them to
 * zero.  All pointers are host pointers and are copied.
 *
 * BC_ZERO   -- no further fields.
 * BC_CONST  -- values[ncomps * volume]: component-major, then the box cells
 *              with axis 0 fastest; rounded to the plan's dtype.
 * BC_MAP    -- the ghost g of component c reads component c of src_block at
 *              src[d] = sign[d] * g[perm[d]] + offset[d]  (perm a permutation
 *              of 0..2): with sign +-1 the halo copy, circular and symmetric
 *              maps (Sec. III-B fmap) and the rotated map of Alg. 1; with
 *              |sign| > 1 (up to 65536) an injection that reads every
 *              |sign|-th cell, for blocks whose regions are slices of one
 *              global grid with different steps (Sec. III-A: staggered and
 *              multigrid layouts).  sign = 0 is rejected.
 * BC_INTERP -- row of cell q reads p consecutive data cells of one source
 *              block along one axis, y = sum_k w[q][k] x[node_k].
 *              geometry = BC_GEOM_USER: itp_src_block[vol], itp_start[vol*3]
 *              (data cell of node 0), itp_axis[vol] (axis the nodes step
 *              along, +1 each) and itp_w[vol*p] give each row.
 *              geometry = BC_GEOM_CUBED_SPHERE: `block` is one of the six
 *              panels cs_panels[0..5] (equal n, h, levels), every box cell
 *              must be an edge ghost (exactly one index out of range), and
 *              the GPU computes the neighbour panel, depth row, stencil and
 *              Lagrange weights in FP64 at plan creation.
 *              geometry = BC_GEOM_CUBED_SPHERE_QUAD: the finite-volume form
 *              of the user-defined interpolation (Sec. II-B; Itp = Agg .
 *              Recons, Sec. III-B).  Data values are cell averages in the
 *              panel's angle coordinates; the ghost value is the average of
 *              nquad x nquad Gauss-Legendre points of the ghost cell, each
 *              point evaluated on the neighbour panel by the tensor-product
 *              polynomial of degree p - 1 per axis whose averages over a
 *              p x p patch of data cells are the data (2 <= p <= 8,
 *              p <= N, 1 <= nquad <= 8).  The patch is chosen from the ghost
 *              centre (normal cells clamp(r - (p/2 - 1), 0, N - p) from its
 *              depth row r, along cells clamp(floor(t + 1e-9) - (p/2 - 1), 0,
 *              N - p) from its along position t).  Panel rules as for
 *              BC_GEOM_CUBED_SPHERE.  The rows are built in FP64 at plan
 *              creation and executed as user CSR rows (p^2 entries, 2 p^2
 *              for a vector pair); plan statistics and export count them as
 *              BC_CSR, and later error messages number sub-matrices after
 *              this expansion (one or two CSR sub-matrices each).  Errors:
 *              bad p or nquad BC_ERR_UNSUPPORTED (p > N: INVALID_ARG), a
 *              box beyond the panel's full region BC_ERR_OUT_OF_RANGE, a box
 *              cell that is not an edge ghost BC_ERR_GEOMETRY.
 *              geometry = BC_GEOM_CUBED_SPHERE_QUAD_CENTRED: the same rows
 *              with both clamps dropped, so that every patch stays centred
 *              on its ghost; near the panel corners and across the shared
 *              edge it then takes ghost values of the neighbour panel (the
 *              iterative form HOPE(I) of Sec. II-B), which the plan folds
 *              with bc_plan_opts.ghost_sweeps (0 sweeps:
 *              BC_ERR_COLUMN_NOT_DATA).  Patches must stay inside the
 *              neighbour's full region (h >= p/2), else BC_ERR_GEOMETRY.
 *              rot_comp = {cu, cv} (or {-1, -1}) names two listed components
 *              that form a covariant vector: for them the interpolated pair
 *              is multiplied by the 2x2 matrix M (user: itp_rot[vol*4],
 *              row-major; cubed sphere: generated, for the quadrature form at
 *              every point before the average) -- interpolate, then rotate.
 *              All other listed components use the plain row.
 * BC_CSR    -- row r = (listed comp r / volume, box cell r % volume) has the
 *              entries row_ptr[r] .. row_ptr[r+1]-1 with columns
 *              (col_block, col_comp, col_ijk[3]) and values val; rhs[r] (or
 *              NULL for zero) is added.  Rows repeat per level and read the
 *              same level of their column blocks.  Columns are data values;
 *              with bc_plan_opts.ghost_sweeps > 0 they may also be ghost
 *              values other sub-matrices (or this one) cover, folded at
 *              creation (see there).
 * BC_SYNC   -- block-edge averaging (Sync of Sec. III-B): the fields of
 *              BC_CSR, but the box lies in the *data* region and its rows
 *              overwrite those data cells (cells several blocks store for
 *              one physical location); rhs must be NULL or zero.  One apply
 *              is one application of A: every row reads the input values, so
 *              Sync rows are computed into a plan-owned staging buffer and
 *              written after all other rows have read the data.  Two Sync
 *              boxes must not share a data cell (BC_ERR_OVERLAP).  Because of
 *              the staging buffer, applies of one plan with Sync rows must
 *              not run concurrently on several streams.
 */
typedef struct bc_submatrix {
  int32_t kind;
  int32_t block;
  int32_t lo[3];
  int32_t hi[3];
  int32_t ncomps;
  const int32_t* comps;
  /* BC_CONST */
  const double* values;
  /* BC_MAP */
  int32_t src_block;
  int32_t perm[3];
  int32_t sign[3];
  int32_t offset[3];
  /* BC_INTERP */
  int32_t p;
  int32_t geometry;
  int32_t rot_comp[2];
  int32_t cs_panels[6];
  const int32_t* itp_src_block;
  const int32_t* itp_start;
  const int32_t* itp_axis;
  const double* itp_w;
  const double* itp_rot;
  /* BC_CSR */
  const int64_t* row_ptr;
  const int32_t* col_block;
  const int32_t* col_comp;
  const int32_t* col_ijk;
  const double* val;
  const double* rhs;
  /* BC_INTERP with BC_GEOM_CUBED_SPHERE_QUAD: Gauss points per axis */
  int32_t nquad;
} bc_submatrix;

/* Plan options; a zero-filled struct (or NULL) selects the defaults. */
typedef struct bc_plan_opts {
  int32_t units_per_lane;  /* work per lane of one warp item: 8-level units
                              (or 8 single-level values) (default 4); small
                              plans use smaller items so that they make
                              about 16 items per SM                         */
  int32_t unit_order;      /* 0: auto (levels fastest when they are adjacent
                              in memory), 1: cells fastest, 2: levels
                              fastest                                       */
  int32_t threads;         /* threads per CTA: 32, 64, 128, 256 or 512
                              (default 128)                                 */
  int32_t ctas_per_sm;     /* persistent CTAs per SM; 0 = a plain grid with
                              one warp per work item (default)              */
  int32_t strict_cover;    /* 1: every ghost value must be covered          */
  int32_t no_adjoint;      /* 1: skip the transpose tables                  */
  int32_t no_runs;         /* 1: zero and map sub-matrices always use
                              per-value units; 0 (default): they copy
                              contiguous runs when the average run holds 16
                              values or more                                */
  int32_t host_only;       /* 1: build the plan on the host only, with no
                              device work (no tables uploaded, no streams):
                              bc_plan_stats and bc_plan_export_csr work,
                              the apply entry points return
                              BC_ERR_UNSUPPORTED; BC_GEOM_CUBED_SPHERE
                              geometry (generated on the GPU) is
                              BC_ERR_UNSUPPORTED, the host-built
                              BC_GEOM_CUBED_SPHERE_QUAD rows are not      */
  int32_t ghost_sweeps;    /* 0 (default): every BC_CSR column must be a
                              data value.  k in 1..64: BC_CSR rows may also
                              read ghost values that a sub-matrix covers
                              (the iterative form HOPE(I) of Sec. II-B);
                              the plan folds k Jacobi sweeps, every ghost
                              starting at zero and all covered rows
                              evaluated together each sweep, into rows on
                              data values only (HOPE(M)) at creation, on
                              the host in FP64.  A column on an uncovered
                              ghost is BC_ERR_COLUMN_NOT_DATA; folded rows
                              over 4096 entries, or cubed-sphere rows
                              generated on the GPU in the same plan,
                              BC_ERR_UNSUPPORTED                             */
  int32_t batch_mode;      /* how BC_FORM_BATCHED runs: 0 default
                              (BC_BATCH_FAMILIES), BC_BATCH_PERSISTENT or
                              BC_BATCH_FAMILIES; bc_plan_autotune times both */
  int32_t scalar_runs;     /* 1: contiguous runs move one 4- or 8-byte value
                              per lane and load; 0 (default): 16-byte vectors,
                              whatever the runs' alignment                   */
  int32_t level_chunk;     /* levels one lane carries through a table row
                              when levels are far apart in memory
                              (interpolation, CSR and transpose rows): 0
                              default (4 for interpolation rows, 8 for CSR
                              and transpose rows), or 1, 2, 4, 8 for all;
                              the launches of every kind in one kernel
                              (BC_BATCH_PERSISTENT, BC_BATCH_SINGLE) take
                              at most 4                                     */
  int32_t unstaged_rows;   /* 1: interpolation, CSR and transpose rows
                              read their columns from global memory lane by
                              lane; 0 (default): with levels far apart in
                              memory, a warp first copies the small box of
                              cells a tile of 32 rows (16 or 8 when a group
                              of 4 levels of the box would not fit) reads,
                              in at most two slots of one block, into
                              shared memory                                 */
  int32_t stencil_fusion;  /* 1: also build the tables bc_apply_stencil
                              needs (a row per ghost-frame cell, and the
                              rows of A in CSR form); 0 (default): none     */
} bc_plan_opts;

/* Execution of BC_FORM_BATCHED (bc_plan_opts.batch_mode). */
typedef enum bc_batch_mode {
  BC_BATCH_PERSISTENT = 1, /* one resident grid whose warps claim the work
                              items of every kind from a device counter, the
                              longest first.  The counter (zero between
                              launches: the last warp resets it) lives in
                              the plan, one per stream the plan is applied
                              on; past 64 streams an apply runs as
                              BC_BATCH_FAMILIES                             */
  BC_BATCH_FAMILIES = 2,   /* one plain-grid kernel per kernel family
                              (structured, interpolation, CSR), forked onto
                              plan-owned streams and joined                 */
  BC_BATCH_FAMILIES_PERSISTENT = 3, /* one persistent kernel per family,
                              forked and joined, each claiming its family's
                              items from its own counter; the SMs are shared
                              out between the families in proportion to
                              their work, so the kernels run side by side  */
  BC_BATCH_SINGLE = 4      /* one plain-grid kernel over the work items of
                              every kind, the longest first (one launch, no
                              fork; the hardware hands the CTAs out)        */
} bc_batch_mode;

typedef struct bc_plan bc_plan;

/* Plan statistics (byte counts use the plan's element size S). */
typedef struct bc_stats {
  int64_t ghost_values;       /* ghost rows of A over all levels            */
  int64_t ghost_values_kind[5];
  int64_t nitems;             /* forward work items                         */
  int64_t nitems_adjoint;     /* adjoint gather items                       */
  int64_t nsubmatrices;
  int64_t nslots;
  int64_t bytes_fwd;          /* algorithmic bytes of one forward apply     */
  int64_t bytes_adj;          /* algorithmic bytes of one adjoint apply     */
  int64_t table_bytes;        /* device table bytes                         */
  int64_t transpose_nnz;      /* entries of the stored A^T (one level)      */
  int32_t element_size;
  int32_t form_threads;
  int32_t form_ctas_per_sm;
  int32_t units_per_lane;
  int32_t launches_fwd;       /* kernel launches of one batched forward      */
  int32_t launches_adj;       /* kernel launches of one adjoint              */
  int64_t sync_values;        /* Sync rows over all levels (data values)    */
  int32_t batch_mode;         /* the bc_batch_mode BC_FORM_BATCHED runs in  */
  int32_t level_chunk;        /* bc_plan_opts.level_chunk in use (0: the
                                 per-family default)                         */
} bc_stats;

/*
 * Build a plan from the grid and nsubs basic sub-matrices.  Checks the
 * description (boxes inside the ghost region, disjoint coverage, data-only
 * columns, fmap depth, finite weights), runs the FP64 cubed-sphere geometry
 * kernel when needed, builds the work list and the transpose of A, and
 * uploads everything to the current device.  Synchronous.  On error *out is
 * NULL and nothing is leaked.
 */
bc_status bc_plan_create(const bc_grid* grid, const bc_submatrix* subs,
                         int32_t nsubs, const bc_plan_opts* opts,
                         bc_plan** out);

/*
 * Dead-ghost elimination (Sec. IV-C: the effective space U(W) of the
 * boundary writes a following stencil reads).  Like bc_plan_create, but the
 * plan keeps only the ghost values that a stencil applied on the data cells
 * reads: ghost cell g of a block is live when g - o is a data cell of that
 * block for one of the stencil offsets o.  offsets: noffsets triples
 * (di, dj, dk), host memory, read during the call only.  Every sub-matrix
 * box is cut to its live cells, split into disjoint boxes that carry the
 * matching slices of its per-cell payload; sub-matrices without live cells
 * are dropped.  Apply then leaves dead ghost values untouched and the
 * adjoint neither reads nor zeroes them.  With strict_cover every live ghost
 * value must be covered.  Errors as bc_plan_create; BC_ERR_INVALID_ARG for
 * an empty stencil.
 */
bc_status bc_plan_create_pruned(const bc_grid* grid, const bc_submatrix* subs,
                                int32_t nsubs, const bc_plan_opts* opts,
                                const int32_t* offsets, int32_t noffsets,
                                bc_plan** out);

/* Number of slots (sum of ncomp) the slot-pointer arrays must hold. */
int32_t bc_plan_nslots(const bc_plan* plan);

/*
 * Forward apply in place: every covered ghost value of every slot becomes
 * (A x_D + b)_i.  slot_ptrs is a DEVICE array of nslots device pointers.
 * stream is a cudaStream_t (NULL = legacy default stream).  Copies, zero
 * rows and constants are written bit-exactly.  Equivalent to
 * bc_apply_form(plan, slot_ptrs, BC_FORM_BATCHED, stream).
 */
bc_status bc_apply(bc_plan* plan, void* const* slot_ptrs, void* stream);

/* Forward apply in one of the bc_form execution forms (same result bits). */
bc_status bc_apply_form(bc_plan* plan, void* const* slot_ptrs, int32_t form,
                        void* stream);

/*
 * Adjoint of the in-place forward apply, in place on the cotangent fields
 * given by slot_ptrs (device array): x_bar_j = y_bar_j + sum_i A_ij y_bar_i
 * for every data value j that no row overwrites, x_bar_j = sum_i A_ij
 * y_bar_i for the data values Sync rows overwrite, and 0 for covered ghost
 * values; uncovered ghosts are left as they are.  Deterministic: each data
 * value sums its entries in ascending order of (row slot, row offset),
 * without atomics.  Two launches (gather, then zero), plus two for Sync
 * rows (a snapshot of their cotangents before, their gather after).  Fails
 * with BC_ERR_UNSUPPORTED if the plan was built with no_adjoint.
 */
bc_status bc_apply_adjoint(bc_plan* plan, void* const* slot_ptrs,
                           void* stream);

/*
 * End-to-end apply on host fields: for every slot, copy host_ptrs[s] (host
 * memory, pinned for asynchronous copies) to dev_ptrs[s] (device memory;
 * host array of device pointers), apply (slot_ptrs: the same device
 * pointers as a device array), and copy every slot back to the host.
 * Adjacent slots whose host and device spans are both contiguous are copied
 * together.  Asynchronous on `stream`; the caller synchronises.
 */
bc_status bc_apply_host(bc_plan* plan, void* const* host_ptrs,
                        void* const* dev_ptrs, void* const* slot_ptrs,
                        void* stream);

/*
 * Boundary conditions fused with the stencil that reads them (Sec. IV-C:
 * the boundary rows only feed the next stencil).  One launch computes, for
 * every data value x of every slot,
 *     out[x] = sum_p coeffs[p] * f(x + offsets[p])
 * where f is the field as bc_apply leaves it: data values as stored,
 * covered ghost values evaluated from their row of A and b where the
 * stencil reads them, uncovered ghost values as stored.  The same launch
 * writes every covered ghost value of the fields (bit for bit as bc_apply
 * does for copies and zero rows), so afterwards the fields are those of a
 * bc_apply.  With a plan from bc_plan_create_pruned for the same stencil,
 * only the live ghosts are written.
 * slot_ptrs: the fields (device array, as bc_apply); out_ptrs: a device
 * array of nslots device pointers laid out with the same strides as the
 * fields, whose data values receive the stencil (ghost values of out are
 * not touched; out must not overlap the fields).  offsets: npoints triples
 * (di, dj, dk), coeffs: npoints FP64 weights (rounded to the plan's dtype),
 * both host memory read during the call (they travel as launch
 * parameters: no allocation, graph-capturable).  Each point's sum runs in
 * the order of the points.  Needs bc_plan_opts.stencil_fusion = 1 at
 * creation (else BC_ERR_UNSUPPORTED, as for plans with Sync rows);
 * BC_ERR_INVALID_ARG for npoints outside 1..125 or a non-finite weight;
 * BC_ERR_HALO_TOO_WIDE when an offset reaches past a block's ghost width,
 * BC_ERR_UNSUPPORTED past 2 cells (the kernel stages tiles with a halo of
 * at most 2).
 */
bc_status bc_apply_stencil(bc_plan* plan, void* const* slot_ptrs, void* const* out_ptrs,
                           const int32_t* offsets, const double* coeffs, int32_t npoints,
                           void* stream);

/*
 * Time candidate executions of BC_FORM_BATCHED on the caller's fields
 * (slot_ptrs, device array) and keep the fastest: the batch mode, the
 * scalar or vector runs, the work per item (units_per_lane), the threads
 * per CTA, the levels-per-lane split (level_chunk, when the plan has
 * chunked units), the staged or unstaged rows (unstaged_rows, when the
 * plan stages some) and the resident CTAs per SM of the persistent launch,
 * searched one option at a time from the plan's own options (median of
 * six launches, each after an L2 flush).  Overwrites the covered ghosts
 * (with the operator's own result).  Allocates a temporary L2-flush buffer;
 * synchronises the stream.
 *
 * Result cache: the choice is remembered under a hash of the plan's rows,
 * layouts and options, the device's name and SM count, for the rest of the
 * process; with BC_AUTOTUNE_CACHE=<file> in the environment it is also
 * read from and appended to that text file (one line per plan), so a later
 * process applies the stored choice without timing anything.
 */
bc_status bc_plan_autotune(bc_plan* plan, void* const* slot_ptrs,
                           void* stream);

/*
 * Pure-function boundary b_i = udf(i) (Sec. III-B) evaluated on the device
 * by the caller: *values receives the device address of the constant table
 * b of BC_CONST sub-matrix `sub` (its index in the list given to
 * bc_plan_create) and *count its length, ncomps * volume values in the
 * plan's dtype, in the order of bc_submatrix.values (component-major, box
 * cells with axis 0 fastest; one value per cell, used at every level).
 * Values the caller writes there (its own kernels or copies, ordered before
 * an apply on the stream that applies) are the b of every later apply and
 * graph replay: a time-dependent boundary needs no new plan.  The address
 * is valid until bc_plan_destroy.  bc_plan_export_csr keeps reporting the
 * values given at creation.  Errors: BC_ERR_INVALID_ARG (NULL argument, no
 * such sub-matrix, not BC_CONST), BC_ERR_UNSUPPORTED (host-only plan, or a
 * plan from bc_plan_create_pruned, whose tables hold the live cells only).
 */
bc_status bc_plan_const_values(bc_plan* plan, int32_t sub, void** values,
                               int64_t* count);

/*
 * Copy `count` values (bc_plan_const_values' count, in the plan's dtype)
 * from `values` (device memory, e.g. the caller's udf evaluated on the
 * device) into the constant table of BC_CONST sub-matrix `sub`, ordered on
 * `stream` (cudaStream_t; a stream capture records it as a copy node).
 * Errors as bc_plan_const_values; BC_ERR_INVALID_ARG for NULL values;
 * BC_ERR_CUDA if the copy cannot be issued.
 */
bc_status bc_plan_set_const(bc_plan* plan, int32_t sub, const void* values,
                            void* stream);

/*
 * Test and debugging aid: replay on the host the values every forward work
 * item (the per-kind list and the batched per-family lists) and every
 * adjoint item (gather, add-runs of unit copies, zero pass) would write,
 * with the kernels' unit decompositions, and compare them with the plan's
 * rows: each covered value written exactly once, copies reading their row's
 * column, zero and constant values equal to the row's b, CSR rows read from
 * the ELL tables and interpolation items read from their node and weight
 * tables equal to their rows, Sync rows staged and committed once with
 * column lists that are their transpose, each data value
 * gathering exactly the terms of A^T in ascending ghost order.  *values =
 * values checked, *problems = mismatches (the first is described by
 * bc_last_error).  Works on host-only plans; no device work.
 */
bc_status bc_plan_check_work(const bc_plan* plan, int64_t* values, int64_t* problems);

/* Fill *out with the plan's counters. */
bc_status bc_plan_stats(const bc_plan* plan, bc_stats* out);

/*
 * Export the rows of A and b at level 0 as CSR over (slot, element offset
 * from the slot pointer).  Call first with NULL arrays to get *nrows and
 * *nnz, then with arrays of those sizes.  Rows are sorted by (slot, offset)
 * and the entries of a row are in the order the forward kernels sum them.
 * Values are the plan's FP64 copies (before rounding to the plan's dtype).
 */
bc_status bc_plan_export_csr(const bc_plan* plan, int64_t* nrows,
                             int64_t* nnz, int32_t* row_slot,
                             int64_t* row_off, int64_t* row_ptr,
                             int32_t* col_slot, int64_t* col_off,
                             double* val, double* rhs);

/*
 * Cubed-sphere interpolation stencils without any device allocation.
 *
 * The paper has no counterpart: this is a convenience for callers that cannot
 * call cudaMalloc -- code inside a framework that owns all device memory
 * through its own pool and forbids raw allocations, or that runs under a
 * fixed device-memory budget.  bc_plan_create allocates device tables and
 * staging buffers, so such callers cannot build a plan; this call still
 * gives them the rows the plan's GPU geometry kernel generates for
 * BC_GEOM_CUBED_SPHERE sub-matrices (the same device function computes
 * both: FP64 geometry, snapping and stencil rules), written to HOST arrays.
 *
 * The kernel's scratch (results and an error word) lives in one fixed device
 * array inside the library, sized for BC_NOALLOC_MAX_CELLS cells (about
 * 7.3 MB); every GPU that loads the library holds it until the process
 * exits.  The call allocates nothing else on the device.
 *
 * Cells: the edge ghosts of six N x N panels with halo h, in the order
 * panel 0..5, strip (axis-0 low, axis-0 high, axis-1 low, axis-1 high), depth
 * 0..h-1 (0 next to the data), along index 0..N-1; ncells = 24 * N * h.
 * Outputs (host arrays) for cell c:
 *   nb[c]            neighbour panel 0..5
 *   node0[2c], node0[2c+1]   (i, j) data cell of stencil node 0 on nb[c]
 *   axis[c]          axis of nb[c] the nodes step along (+1 per node); the
 *                    bit BC_NOALLOC_SNAP marks a unit copy of node 0
 *   w[p*c .. p*c+p-1]  Lagrange weights (FP64)
 *   rot[4c .. 4c+3]  2x2 change of covariant vector components, row-major
 *                    (filled only when rot is not NULL)
 * Errors: BC_ERR_INVALID_ARG (p outside 1..8, h < 1, N < p, h > N, NULL
 * output), BC_ERR_UNSUPPORTED (24*N*h > BC_NOALLOC_MAX_CELLS),
 * BC_ERR_GEOMETRY, BC_ERR_CUDA.  After any status other than BC_OK the
 * contents of the output arrays are undefined.
 * Synchronous: it uses the legacy default stream of the current device and
 * returns when the results are on the host.  The first call on a device
 * looks up the scratch array's device address there (with that device
 * current) and keeps it for later calls; make that first call before any
 * stream capture begins.  The address belongs to the device's primary
 * context, so a cudaDeviceReset between calls is not supported.  All calls
 * share the one scratch array and it keeps the last call's results (the
 * error word is cleared by every call): calls that overlap on the GPU
 * (several host threads, or processes sharing a context) race with each
 * other.
 */
#define BC_NOALLOC_MAX_CELLS 65536
#define BC_NOALLOC_SNAP 0x100
bc_status bc_cubed_sphere_stencils_noalloc(int32_t N, int32_t h, int32_t p,
                                           int32_t* nb, int32_t* node0,
                                           int32_t* axis, double* w,
                                           double* rot);

/*
 * Packing of block boxes for an exchange between processes (Sec. V-B: a
 * process that owns only some blocks receives, for every remote block its
 * boundary rows read, the bounding box of the cells read).  A bc_box is the
 * cell range [lo, hi) of one block of `grid` (inside its full region),
 * taken with every component and level.  bc_pack_create checks the boxes
 * and uploads their descriptors (synchronous; allocates); bc_pack_run then
 * copies the boxes from the fields (slot_ptrs: device array of the grid's
 * nslots slot pointers, as bc_apply) into `buffer` (device memory of
 * bc_pack_size() elements of the grid's dtype): box after box, each stored
 * [component][level][k][j][i] -- the layout of a block of extents hi - lo,
 * no ghost cells, levels outermost.  bc_pack_run allocates nothing and does
 * not synchronise (graph-capturable); the values are copied bit for bit.
 * Errors: BC_ERR_INVALID_ARG (NULL, an empty box, a block out of range),
 * BC_ERR_OUT_OF_RANGE (a box outside its block's full region),
 * BC_ERR_UNSUPPORTED (a box of 2^31 values or more), BC_ERR_NOMEM / CUDA.
 */
typedef struct bc_box {
  int32_t block;
  int32_t lo[3];
  int32_t hi[3];
} bc_box;
typedef struct bc_pack bc_pack;
bc_status bc_pack_create(const bc_grid* grid, const bc_box* boxes, int32_t nboxes,
                         bc_pack** out);
int64_t bc_pack_size(const bc_pack* pack);
bc_status bc_pack_run(bc_pack* pack, void* const* slot_ptrs, void* buffer, void* stream);
void bc_pack_destroy(bc_pack* pack);

/*
 * The circular or symmetric face of Sec. III-B as a BC_MAP sub-matrix, so a
 * C caller need not derive the affine map.  On axis `axis` of block `block`
 * (grid->blocks[block], extent N = n[axis], ghost width h = h[axis]), side 0
 * is the low face (ghost indices -h..-1), side 1 the high face (N..N+h-1);
 * the box spans the data range along the other axes.  The paper's fmap:
 * BC_FMAP_SYMMETRIC reads the mirror image (low: -1-i; high: 2N-1-i),
 * BC_FMAP_CIRCULAR the periodic image (low: i+N; high: i-N), the other
 * axes unchanged.  comps (ncomps entries, the caller's array) is stored in
 * *out as given, so it must live until bc_plan_create has copied it.
 * Errors: BC_ERR_INVALID_ARG (NULL, bad block / axis / side / kind, a
 * component out of range), BC_ERR_HALO_TOO_WIDE (h > N: fmap is defined for
 * depths 0 < x <= N), BC_ERR_OUT_OF_RANGE (h = 0: the face has no ghosts).
 */
typedef enum bc_fmap { BC_FMAP_CIRCULAR = 0, BC_FMAP_SYMMETRIC = 1 } bc_fmap;
bc_status bc_fmap_submatrix(const bc_grid* grid, int32_t block, int32_t axis, int32_t side,
                            int32_t fmap, const int32_t* comps, int32_t ncomps,
                            bc_submatrix* out);

/* Release the plan and its device tables (NULL is a no-op). */
void bc_plan_destroy(bc_plan* plan);

const char* bc_status_string(bc_status status);

/* Message of the last failed call on this thread ("" if none). */
const char* bc_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* BC_GB300_H */
