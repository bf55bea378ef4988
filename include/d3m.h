/*
 * d3m.h -- C ABI of the GB300 D^3M library (Direct Domain Decomposition Method
 * for finite-element electromagnetics, Moshfegh & Vouvakis, ICEAA 2016).
 *
 * Problem (Theory section, decomposed BVP): curl curl E - k^2 eps_r E = 0 in
 * an axis-aligned box of nx*ny*nz lattice cells, meshed by bricks or by six
 * tetrahedra per cell, or on a general tetrahedral mesh (d3m_mesh), with
 * lowest-order Nedelec edge elements (complete first-order ones on general
 * meshes if asked), a first-order absorbing boundary condition on the whole
 * outer boundary driven by incident plane waves, mu_r = 1.  The domain is cut
 * into px*py*pz subdomains; the library assembles the decomposed system of
 * Eq. (1), [[A, D], [D^T, 0]] [E; lambda] = [f; 0], and factors it with the
 * paper's seven main steps: dense domain matrices K_D, assembly of the
 * block-sparse K = sum D_i^T A_i^{-1} D_i, block nested-dissection ordering of
 * its clique graph, symbolic factorisation, block LDL^T with restricted
 * Bunch-Kaufman pivots (Algorithm 1, in its multifrontal form), substitution
 * for lambda and recovery of E.
 *
 * Conventions for every entry point:
 *  - complex numbers are pairs of doubles (re, im) in consecutive memory;
 *  - global edge numbering: x-edges, then y-edges, then z-edges (then, on
 *    tetrahedral meshes, the diagonal families listed at d3m_mesh); each
 *    family runs its start node (i, j, k) x-fastest: x-edge (i,j,k) = i +
 *    nx*(j + (ny+1)*k), y-edge = NX + i + (nx+1)*(j + ny*k), z-edge = NX + NY
 *    + i + (nx+1)*(j + (ny+1)*k), NX = nx(ny+1)(nz+1), NY = (nx+1)ny(nz+1);
 *    every edge points from its start node towards increasing coordinates;
 *  - cells are numbered i + nx*(j + ny*k) (on general meshes: the
 *    tetrahedra in input order); subdomains ix + px*(iy + py*iz);
 *  - RHS / solution blocks are column-major n_edges x nrhs with a leading
 *    dimension >= n_edges, in global edge numbering with PEC edges present
 *    (their solution rows are returned as 0);
 *  - every call returns D3M_OK (0) or an error code; a message is available
 *    from d3m_last_error(ctx).  No call aborts the process or traps the GPU;
 *    device-side waits are bounded and report D3M_ETIMEOUT.
 *  - all device work is ordered on d3m_options.stream (a cudaStream_t, NULL =
 *    the legacy default stream); the library's internal streams (look-ahead,
 *    overlapped inverses) fork from and join back into it, and calls return
 *    after the work is complete (d3m_dense_ldlt_noalloc is the one exception:
 *    it only enqueues its work, see there).
 */
#ifndef D3M_H
#define D3M_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum d3m_status {
  D3M_OK = 0,
  D3M_EINVAL = 1,     /* bad argument (sizes, cuts, pointers) */
  D3M_ENOMEM = 2,     /* host or device allocation failed */
  D3M_ESINGULAR = 3,  /* a pivot column of a diagonal block is exactly zero */
  D3M_ENOCONV = 4,    /* iterative refinement did not reach refine_tol */
  D3M_ETIMEOUT = 5,   /* a bounded device-side wait expired */
  D3M_ECUDA = 6,      /* a CUDA runtime call failed */
  D3M_ESTATE = 7      /* call out of order (e.g. solve before factor) */
};

enum d3m_precision {
  D3M_FP64 = 0,       /* factors and substitutions in complex128 */
  D3M_MIXED = 1       /* factors in complex64; the pivot tests decide as fp64
                         tests on the complex64 values (fp32 comparisons,
                         re-evaluated in fp64 when within 2^-20 of a tie); the
                         1x1/2x2 pivot inverses are the fp32 inverses those
                         decisions computed; fp64 residuals and iterative
                         refinement against the fp64 sparse operator */
};

typedef struct d3m_ctx d3m_ctx;

enum d3m_element {
  D3M_BRICK = 0,      /* lowest-order Nedelec bricks on the axis-aligned grid */
  D3M_TET = 1,        /* lowest-order Nedelec (Whitney) tetrahedra, six per
                         cell (the Introduction's general FEM setting) */
  D3M_TET_MESH = 2    /* the same elements on a general tetrahedral mesh
                         (vertex and tetrahedron lists, any connectivity) */
};

/* Mesh of [0,lx] x [0,ly] x [0,lz] with nx*ny*nz lattice cells, or (element
 * D3M_TET_MESH) a general tetrahedral mesh.
 * element D3M_BRICK: axis-aligned bricks; vertices must be NULL.
 * element D3M_TET: every cell is split into six tetrahedra along its
 *   (0,0,0)-(1,1,1) diagonal (each cell face along its lowest-to-highest
 *   corner diagonal, so neighbouring cells conform).  The dof of an edge is
 *   the line average of E . t along it, as for bricks.  vertices: NULL for
 *   the regular lattice, or 3*(nx+1)*(ny+1)*(nz+1) doubles, the (x, y, z)
 *   position of node (i, j, k) at index i + (nx+1)*(j + (ny+1)*k), read
 *   during d3m_setup only (the caller keeps ownership).  Every tetrahedron
 *   must keep the orientation it has in the regular lattice, and nodes on the
 *   outer boundary must stay in their boundary planes (the absorbing
 *   condition takes the box's face normals): D3M_EINVAL otherwise.
 * Global edge numbering: edge families one after another, each x-fastest
 * over its own box of start nodes (i, j, k); directions (1,0,0), (0,1,0),
 * (0,0,1), and for D3M_TET then (1,1,0), (1,0,1), (0,1,1), (1,1,1).  Every
 * edge points from its start node to start + direction.
 * element D3M_TET_MESH: n_vertices positions in vertices (3 doubles each) and
 *   n_tets tetrahedra in tets (4 vertex ids each, any orientation, nonzero
 *   volume); nx..lz are not read.  Cells are the tetrahedra (eps_r has one
 *   value per tetrahedron, d3m_grad_eps one entry per tetrahedron).  Edges
 *   are the distinct vertex pairs (i < j) of the tetrahedra in lexicographic
 *   order, each pointing from vertex i to vertex j; boundary triangles (faces
 *   of one tetrahedron) carry the absorbing condition with their outward
 *   normal.  Subdomains are set by the coordinate cuts gx, gy, gz of the
 *   partition.  Both arrays are read during d3m_setup only. */
typedef struct {
  int32_t nx, ny, nz;
  double lx, ly, lz;
  int32_t element;          /* d3m_element */
  const double *vertices;   /* D3M_TET: NULL (regular lattice) or the lattice nodes;
                               D3M_TET_MESH: 3 * n_vertices doubles */
  int64_t n_vertices;       /* D3M_TET_MESH only */
  int64_t n_tets;           /* D3M_TET_MESH only */
  const int64_t *tets;      /* D3M_TET_MESH only: 4 * n_tets vertex ids */
  int32_t order;            /* D3M_TET_MESH: 0 or 1 = Whitney functions, one dof per
                               edge; 2 = complete first order (hierarchical): each
                               edge (i, j) also carries l_ij grad(lam_i lam_j) (no
                               curl, tangential component 1 - 2 s / l_ij along its
                               edge, s from i), dof 2e the Whitney function of edge
                               e and dof 2e+1 its gradient function; the "n_edges"
                               rows of every RHS/solution block and of pec_edge's
                               count are then 2 * edges (pec_edge: one byte per
                               dof, both dofs of an edge alike); 3 = curl-complete
                               second order: order 2 plus, on every face with
                               vertices a < b < c, l_ab lam_c W_ab and l_ac lam_b
                               W_ac (W the Whitney function without the length
                               factor), dofs 2*edges + 2f and + 1 for face f
                               (faces numbered as sorted vertex triples,
                               lexicographic).  Other elements: 0 or 1. */
} d3m_mesh;

/* Materials.  eps_r: 2*n_cells doubles (re, im) per cell, time convention
 * e^{jwt} so losses have negative imaginary part.  pec_edge: n_edges bytes or
 * NULL; 1 marks an edge whose tangential field is zero (its dof is removed:
 * a Dirichlet condition, used for the paper's PEC plates). */
typedef struct {
  const double *eps_r;
  const uint8_t *pec_edge;
} d3m_materials;

/* Subdomain cuts: cx has px+1 strictly increasing cell indices from 0 to nx
 * (likewise cy, cz).  Edges on an interior cut plane are copied into every
 * subdomain containing them.
 * General meshes (D3M_TET_MESH) use gx, gy, gz instead: px+1 (py+1, pz+1)
 * strictly increasing coordinates; a tetrahedron belongs to subdomain
 * (ix, iy, iz) when its centroid ((v0 + v1) + v2) + v3 over 4 satisfies
 * c_x >= gx[ix] (or ix = 0) and c_x < gx[ix+1] (or ix = px - 1), likewise in
 * y and z; every box must hold a tetrahedron (D3M_EINVAL otherwise).  An
 * edge is copied into every subdomain holding one of its tetrahedra; an
 * extra copy with no earlier copy in a grid-face-adjacent subdomain is tied
 * by its multiplier to the lowest-index copy. */
typedef struct {
  int32_t px, py, pz;
  const int32_t *cx, *cy, *cz;
  const double *gx, *gy, *gz;  /* D3M_TET_MESH only */
} d3m_partition;

typedef struct {
  int32_t precision;    /* d3m_precision */
  int32_t leaf_max;     /* nested-dissection leaf size (edges); 0 -> 64 */
  double refine_tol;    /* mixed: stop when ||f - A x||_inf / ||f||_inf <= tol;
                           0 -> 1e-10 */
  int32_t max_refine;   /* mixed: refinement step cap; 0 -> 10 */
  void *stream;         /* cudaStream_t */
  int32_t profile;      /* 1: time every kernel class with CUDA events on `stream`
                           (results in d3m_stats); 0: off */
  int32_t panel_kernel; /* 0: thread-block-cluster panels where the front fits the
                           cluster's shared memory (default); 1: always the
                           single-CTA global-memory panel (same arithmetic) */
  int32_t update_kernel;/* MIXED trailing/Schur updates: 0 = per level, the faster of
                           the two below as measured by the autotuner (default);
                           1 = fp32 FMA, right-looking after every panel; 2 =
                           deferred: the panels update only the pivot block, then
                           the update rows (W21 = F21 P^T L11^{-T}, L21 = W21
                           D^{-1}) and the Schur complement (F22 - L21 W21^T)
                           of every front of the level are two batched complex
                           products on the tcgen05 tensor cores: each fp32 operand
                           split into three bf16 planes (BF16x3), staged by TMA,
                           fp32 accumulation in tensor memory */
  int32_t autotune;     /* 0 = tune on the first d3m_factor (default): the update
                           kernel and the panel cluster size of every tree level
                           are timed with CUDA events over trial factorisations
                           (three in MIXED, two in FP64) and the faster kept; 1 =
                           off (fixed
                           defaults: FMA updates, smallest fitting cluster) */
  const char *autotune_cache; /* optional file: read the tuned schedule from it when
                           it matches this problem, write it after tuning; NULL = none */
  int32_t lookahead;    /* 0 = overlap (default): the Schur-complement part of each
                           trailing update runs on a second stream, launched with
                           the least urgent priority, while the next panels of the
                           front (which touch only its pivot block) proceed with
                           the most urgent one; 1 = off, every update completes
                           before the next panel.  Both give bitwise identical
                           factors. */
  int32_t refine_method;/* MIXED: 0 = plain iterative refinement (default): x +=
                           M^{-1} (f - A x) with M^{-1} the complex64 factors;
                           1 = GMRES-based refinement: each correction d solves
                           A d = f - A x by flexible GMRES in fp64, right
                           preconditioned by M^{-1}, for cases where plain
                           refinement stalls (conditioning times the factor
                           precision near one).  Every refinement step counts
                           toward max_refine. */
  int32_t gmres_restart;/* GMRES-IR: Krylov steps per correction; 0 -> 20 (<= 200) */
  double gmres_tol;     /* GMRES-IR: relative 2-norm reduction of each correction
                           equation's residual; 0 -> 1e-4 */
  double alpha_re, alpha_im; /* interface loss/gain coefficient alpha of the
                           subdomain matrices (+alpha T_f on the side facing the
                           higher subdomain index, -alpha T_f on the other; the
                           Theory section's "loss or gain at the interfaces"):
                           0, 0 -> jk.  The two sides cancel, so the solution E
                           does not depend on alpha; K_D, K and lambda do. */
  int32_t solve_kernel; /* MIXED substitution products (L11^{-1}, L21, their
                           transposes times the right-hand sides): 0 = complex
                           BF16x3 on the tcgen05 tensor cores (default): each
                           factorisation also writes these operands as bf16
                           planes in 128 x 32 blocks (about 12 bytes per complex
                           entry, blocks padded; extra device memory), the
                           right-hand sides are split inside the product
                           kernel, fp32 accumulation in tensor memory; 1 = fp32
                           FMA on the complex64 factors.  FP64 always uses fp64
                           FMA. */
  int32_t lm_weight;    /* multiplier map D of Eq. (1): 0 = signed Boolean (+1 on
                           the lower-index copy of an interface edge, -1 on the
                           other; default); 1 = the Galerkin form of the Theory
                           section's lambda = j +- e in the tangential edge basis:
                           D = D_bool T_lambda with T_lambda the tangential face
                           mass int_f N_m . N_l dS between the multipliers of one
                           interface block.  Symmetric positive definite per
                           block, so E does not change; lambda, K_D and K do
                           (lambda_1 = T_lambda^{-1} lambda_0).  Lattice meshes
                           only (D3M_EINVAL with D3M_TET_MESH, where a block
                           may join subdomains without a common face). */
} d3m_options;
/* d3m_setup returns D3M_EINVAL (and the context, for d3m_last_error) when an
 * option lies outside the values listed above. */

/* Per-solve report: per column relative residual (Numerical Results
 * section's ||A x - f||_inf / ||f||_inf) and refinement steps taken. */
typedef struct {
  double *resid;        /* caller array of nrhs doubles, or NULL */
  int32_t iters;        /* refinement steps (0 for FP64) */
  double max_resid;
  int32_t inner_iters;  /* GMRES-IR: Krylov steps summed over the corrections */
} d3m_solve_info;

/* Sizes and counts of a set-up problem. */
typedef struct {
  int64_t n_edges, n_free, n_lm, n_blocks, n_subdomains;
  int64_t n_m;            /* order of the saddle matrix [[A, D], [D^T, 0]] */
  int64_t n_fronts, n_levels, max_front;
  int64_t arena_bytes;    /* front storage of the chosen precision */
  double flops_interior;  /* real flops (8 per complex MAC) of the interior fronts */
  double flops_domain;    /* ... of the interface fronts (domain matrices K_D) */
  double flops_k;         /* ... of the fronts of K (Algorithm 1) */
  int64_t n_2x2;          /* 2x2 pivots taken by the last factorisation */
  double min_pivot_ratio; /* smallest |d| / max|column| seen (diagnostic) */
  /* last factorisation / solve (kernel launches always; times with profile=1) */
  int64_t launches_factor, launches_solve;
  double flops_update;    /* exact real flops of the trailing updates (device-counted) */
  double flops_panel;     /* exact real flops of the panel column updates */
  double ms_assemble, ms_panel, ms_update;        /* summed kernel durations */
  double ms_fwd, ms_bwd, ms_residual;             /* last solve, all refinement steps */
  double solve_flops;     /* real flops of the last solve's substitutions */
  double ms_inverse;      /* factor: building L11^{-1} of every front and, with
                             solve_kernel 0, the substitution's bf16 operand
                             blocks (profile=1) */
  int64_t tuned_levels_tc;/* levels whose updates the autotuner put on tensor cores */
  int64_t tuned_levels_cs2; /* levels whose panels run with the doubled cluster size */
  double ms_tuning;       /* wall time of the trial factorisations */
  /* MIXED, levels on the tensor cores: the deferred products W21 = F21 P^T
     L11^{-T} and C = F22 - L21 W21^T with their operand splits and the
     L21 = W21 D^{-1} scaling (profile=1), and their algorithmic real flops */
  double ms_tc;
  double flops_tc;
} d3m_stats;

/*
 * d3m_setup -- host-only analysis (no CUDA call is made).
 * Builds the element matrices, the subdomain matrices A_i with interface
 * loss/gain +-jk T_f (sign + on the side facing the higher subdomain index),
 * the signed multiplier map D (one multiplier per extra copy, tied to the
 * lowest-index face neighbour), the orderings (nested dissection inside each
 * subdomain with interface dofs last; block nested dissection of the clique
 * graph of K, main step 3) and the supernodal symbolic factorisation (main
 * step 4).  Host inputs are copied; the caller keeps ownership.  k is the
 * wavenumber (2*pi for wavelength 1).  Returns D3M_EINVAL on inconsistent
 * sizes or cuts.  *out receives a context to pass to d3m_free.
 */
int d3m_setup(const d3m_mesh *mesh, const d3m_materials *mat, double k,
              const d3m_partition *part, const d3m_options *opt, d3m_ctx **out);

/*
 * d3m_factor -- numeric factorisation on the GPU (main steps 1, 2, 5).
 * First call uploads the plan and allocates the device arena (all device
 * memory is owned by the context).  Runs, level by level over the assembly
 * tree, the front assembly (extend-add), restricted Bunch-Kaufman panels and
 * trailing updates of every front: subdomain interiors, interface fronts whose
 * contribution blocks are -K_D^(i), and the fronts of K.  D3M_ESINGULAR if a
 * pivot column is exactly zero.  The first call also tunes the per-level
 * schedule (d3m_options.autotune) with two timed trial factorisations; an
 * unprofiled call captures its launch sequence into a CUDA graph that later
 * unprofiled calls replay (the same arithmetic, bit for bit).  Call it again
 * after the materials change (a new d3m_setup) or to refactor the same
 * operator.
 */
int d3m_factor(d3m_ctx *ctx);

/*
 * d3m_solve -- main steps 6-7 for nrhs excitations, DEVICE pointers.
 * rhs: n_edges x nrhs complex column-major (ld >= n_edges), read only.
 * x:   n_edges x nrhs complex column-major (ld >= n_edges), written.
 * Multiplier values can be read afterwards with d3m_structure(D3M_LAMBDA).
 * MIXED precision refines until the residual criterion holds (D3M_ENOCONV
 * otherwise; x then holds the last iterate).  info may be NULL.
 */
int d3m_solve(d3m_ctx *ctx, const double *rhs, int64_t ldb, double *x, int64_t ldx,
              int32_t nrhs, d3m_solve_info *info);

/* d3m_solve_host -- as d3m_solve with HOST pointers (pinned memory gives
 * asynchronous copies); the host<->device copies run on the context stream. */
int d3m_solve_host(d3m_ctx *ctx, const double *rhs, int64_t ldb, double *x, int64_t ldx,
                   int32_t nrhs, d3m_solve_info *info);

/*
 * d3m_solve_adjoint -- y = A^{-H} b with the same factors (DEVICE pointers,
 * layouts as d3m_solve).  A is complex symmetric (A = A^T, the paper's
 * discussion of K), so A^{-H} b = conj(A^{-1} conj(b)): the conjugations are
 * applied inside the library and the factorisation is reused as it is.  This
 * is the adjoint solve of a field objective's gradient; MIXED precision
 * refines it like d3m_solve.
 */
int d3m_solve_adjoint(d3m_ctx *ctx, const double *rhs, int64_t ldb, double *y, int64_t ldy,
                      int32_t nrhs, d3m_solve_info *info);

/*
 * d3m_grad_eps -- per-cell gradient of a real objective J(x) of the solution
 * with respect to the real part of eps_r:
 *   grad[c] = k^2 * Re( sum_r conj(y_r)_c^T M_c x_r,c ),
 * where x = A^{-1} f is the forward solution, y = A^{-H} (dJ/dx) the adjoint
 * solution from d3m_solve_adjoint (dJ/dx in PyTorch's convention, e.g. 2 x at
 * the probes for J = sum |x_probe|^2), M_c the mass matrix of cell c over its
 * 12 edges (bricks), 19 edges (the six tetrahedra of a D3M_TET cell) or the
 * 6, 12 or 20 dofs of a D3M_TET_MESH tetrahedron of order 1, 2 or 3
 * (dA/deps_c = -k^2 M_c) and the sum runs over the nrhs columns.  DEVICE
 * pointers: x, y as in d3m_solve (PEC rows ignored), grad: n_cells doubles,
 * overwritten.  FP64 regardless of the factor precision.
 */
int d3m_grad_eps(d3m_ctx *ctx, const double *x, int64_t ldx, const double *y, int64_t ldy,
                 int32_t nrhs, double *grad);

/*
 * d3m_rhs_planewave -- host computation of the ABC right-hand side for
 * incident plane waves E_inc = p exp(-jk khat.r):  f_v = -sum over outer
 * faces of int (n x curl E_inc - jk E_inc,t) . N_v dS, 3x3 Gauss-Legendre
 * points per face.  khat_pol: nrhs rows of 9 doubles (khat xyz, then p as
 * re x, im x, re y, im y, re z, im z).  rhs: host, n_edges x nrhs complex,
 * column-major, ld >= n_edges.
 */
int d3m_rhs_planewave(d3m_ctx *ctx, const double *khat_pol, int32_t nrhs, double *rhs,
                      int64_t ldb);

/* Structure / diagnostics export (host memory).  Call with buf = NULL to get
 * the size in bytes in *bytes; then with a buffer of that size. */
enum d3m_structure_kind {
  D3M_SN_RANGE = 0,    /* int64 [n_fronts][2]: pivot range [start, end) in M order */
  D3M_SN_PARENT = 1,   /* int64 [n_fronts]: supernodal elimination tree, -1 = root */
  D3M_SN_KIND = 2,     /* int64 [n_fronts][2]: kind (0 interior ND node, 1 interface
                          dofs B_i, 2 block of K) and owner (subdomain or block id) */
  D3M_SN_STRUCT = 3,   /* int64 [n_fronts + 1] offsets, then the concatenated sorted
                          update-row lists (M indices) */
  D3M_M_MAP = 4,       /* int64 [n_m][2]: (subdomain, global edge) of each M index,
                          (-1, multiplier id) for multipliers */
  D3M_LM = 5,          /* int64 [n_lm][3]: (global edge, + subdomain, - subdomain) */
  D3M_BLOCKS = 6,      /* int64 [n_blocks][3]: (a, b, first multiplier id) in block order */
  D3M_LAMBDA = 7,      /* double [n_lm][nrhs][2]: multipliers of the last solve,
                          column-major complex */
  D3M_STATS = 8,       /* d3m_stats */
  D3M_M_ENTRIES = 9,   /* double [nnz][4]: (row, col, re, im) of the lower triangle of
                          M = [[A, D], [D^T, 0]] in M order, as assembled */
  D3M_LEVELS = 10      /* double [n_levels][10] per level of the assembly tree
                          (leaves first): fronts, largest pivot block, largest
                          front, algorithmic real flops, then from the last
                          factorisation run with d3m_options.profile = 1 (else
                          0): panel ms, update ms, 1 if the deferred tcgen05
                          products ran, panel cluster size (0 = single-CTA
                          panel), L11^{-1} ms, tcgen05 products ms */
};
int d3m_structure(d3m_ctx *ctx, int32_t which, void *buf, size_t *bytes);

/*
 * d3m_dense_ldlt -- the front kernel alone: restricted Bunch-Kaufman partial
 * LDL^T of `batch` dense complex-symmetric m x m matrices (DEVICE pointers,
 * column-major, lower triangle read, consecutive matrices m*m complex apart),
 * pivots restricted to the leading p x p block (the paper's block-restricted
 * pivoting).  On return, in place: columns 0..p-1 hold unit-lower L in pivot
 * order (rows 0..m-1; the diagonal holds the diagonal of D and the (k+1,k)
 * entry of a 2x2 block is 0), rows/cols p..m-1 hold the Schur complement C
 * (lower).
 * perm (device int32, batch*m): pivot position -> original index.
 * dinv (device double, batch*p*6): per pivot (re,im) of D^{-1}(k,k), of the
 * coupling entry of its 2x2 block (0 for 1x1) and a block-size code
 * (1, 2 = first of a pair, -2 = second) in the real slot of the third pair.
 * info (device int32, batch): 0 or 1 + first zero-pivot column.
 * fp64 only; stream and panel_kernel as in d3m_options.  Does not need a context.
 */
int d3m_dense_ldlt(int32_t m, int32_t p, int32_t batch, double *A, int32_t *perm, double *dinv,
                   int32_t *info, void *stream, int32_t panel_kernel);

/*
 * d3m_export_front -- diagnostics: copy front `front` (M-order supernode id)
 * of the last factorisation to host memory.  F: m*m complex (column-major,
 * after factorisation: L in the pivot columns, D on the diagonal / 2x2
 * couplings, contribution block below-right), perm: p int32 (pivot position
 * -> local index), dinv: 6*p doubles as in d3m_dense_ldlt.  Any pointer may be
 * NULL.  Values are widened to fp64 for the MIXED precision.  *m_out, *p_out
 * receive the front sizes (call with NULL buffers first to size them).
 */
int d3m_export_front(d3m_ctx *ctx, int64_t front, int32_t *m_out, int32_t *p_out, double *F,
                     int32_t *perm, double *dinv);

/*
 * d3m_dense_ldlt_noalloc -- d3m_dense_ldlt for callers that cannot allocate
 * memory.  The paper has no counterpart: this is a service entry point of the
 * library.  Some callers run where cudaMalloc/cudaFree are not allowed --
 * code inside a stream-ordered region that must not synchronise the device,
 * allocator hooks and custom memory pools that would recurse into
 * themselves, or processes whose device memory budget is fixed up front.
 * This variant computes the same factorisation with every piece of scratch
 * (front tables, panel workspace, pivot state) in one fixed device array of
 * D3M_NOALLOC_SCRATCH_BYTES that is part of the library image; it calls no
 * cudaMalloc, cudaFree or other allocating routine, on the host or the device.
 * Arguments, layout and results are exactly those of d3m_dense_ldlt, but the
 * call is asynchronous: it returns as soon as its kernels are enqueued on
 * `stream` (NULL = the legacy default stream) and never waits for the device;
 * A, perm, dinv and info hold the results once the stream has reached that
 * point.  A non-OK return means that a launch was refused (D3M_ECUDA) or the
 * request was invalid (D3M_EINVAL): after D3M_ECUDA, A may be partly factored
 * and perm, dinv, info are undefined.
 * Limits: the scratch must hold 16*NB*m*batch bytes of panel workspace (NB =
 * 32) plus about 96 bytes per matrix and 37 bytes per pivot; larger requests
 * return D3M_EINVAL without touching the GPU.  The first call on a device
 * looks the array up (cudaGetSymbolAddress, once per device, with that device
 * current), so make that first call before any stream capture.  Every GPU
 * that loads the library holds the array until the process exits.  All calls
 * share the array and it keeps the previous call's contents (the state that
 * must start at zero is cleared by each call), so calls whose GPU work
 * overlaps (different streams, or different host threads on the same device)
 * race with each other: serialise them.
 */
#define D3M_NOALLOC_SCRATCH_BYTES (8u << 20)
int d3m_dense_ldlt_noalloc(int32_t m, int32_t p, int32_t batch, double *A, int32_t *perm, double *dinv,
                           int32_t *info, void *stream);

int d3m_stats_get(d3m_ctx *ctx, d3m_stats *out);

/* Turn the per-kernel-class CUDA-event timing (d3m_options.profile) on (1)
 * or off (0) for the following calls.  Unprofiled factorisations replay the
 * launch sequence captured into a CUDA graph at their first call; profiled
 * ones launch eagerly with events around every kernel group, which costs host
 * time.  D3M_EINVAL for a NULL context. */
int d3m_set_profile(d3m_ctx *ctx, int32_t on);
const char *d3m_last_error(const d3m_ctx *ctx);
void d3m_free(d3m_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* D3M_H */
