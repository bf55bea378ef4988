// Internal state shared by the host set-up (host_setup.cpp) and the device
// factor/solve engine (engine.cu).  Not part of the public ABI.
#pragma once

#include <array>
#include <complex>
#include <cstdint>
#include <string>
#include <utility>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/d3m.h"

namespace d3m {

// Named range over one call of the ABI (NVTX; free unless a profiler such as
// Nsight Systems is attached): d3m_setup, d3m_factor, d3m_solve, ...
struct NvtxRange {
  explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange &) = delete;
  NvtxRange &operator=(const NvtxRange &) = delete;
};

using cplx = std::complex<double>;

struct DeviceState;  // engine.cu

struct Plan {
  // ---- problem
  int nx = 0, ny = 0, nz = 0;
  double lx = 0, ly = 0, lz = 0, k = 0, h[3] = {0, 0, 0};
  std::vector<cplx> eps;
  std::vector<uint8_t> pec;  // per edge, 1 = removed
  int parts[3] = {1, 1, 1};
  std::vector<int> cuts[3];
  int64_t nex = 0, ney = 0, nez = 0, n_edges = 0, n_free = 0;
  // ---- element kind and edge families (d3m_mesh)
  int element = 0;                    // D3M_BRICK or D3M_TET
  int nfam = 3;                       // edge families: 3 (bricks) or 7 (tetrahedra)
  int cell_ne = 12;                   // edges per cell: 12 or 19
  int64_t fam_off[8] = {0};           // first edge id of each family
  int64_t fam_n[7][3] = {};           // start-node box of each family
  std::vector<double> vert;           // tetrahedra: 3 doubles per node (empty: lattice)
  int64_t n_cells = 0;                // lattice cells, or the tetrahedra of a general mesh
  // ---- general tetrahedral meshes (D3M_TET_MESH)
  std::vector<int64_t> tet_v;         // 4 vertex ids per tetrahedron
  std::vector<int64_t> tet_e;         // 6 edge ids per tetrahedron (local pairs 01 02 03 12 13 23)
  std::vector<int8_t> tet_s;          // 6 orientation signs per tetrahedron
  int dpe = 1;                        // dofs per edge (mesh order): dof dpe*e + q
  int order = 1;                      // mesh order 1, 2 or 3 (3: two dofs per face too)
  int64_t n_geo = 0, n_faces = 0;     // edges and faces of a general mesh
  std::vector<int64_t> tet_f;         // 4 face ids per tetrahedron (face q omits vertex q)
  std::vector<std::array<int64_t, 3>> mface;  // sorted vertex triple of each face
  std::vector<std::array<int64_t, 4>> bface;  // boundary triangles: sorted vertices + opposite vertex
  std::vector<std::pair<int64_t, int64_t>> medge;  // vertex pair (i < j) of each edge
  double bS[12][12], bM[12][12], bT[6][12][12];  // brick element and face matrices

  // ---- decomposition
  int nsub = 0;
  std::vector<std::array<int, 3>> sub_lo, sub_hi;
  std::vector<std::vector<int64_t>> sub_edges;  // sorted global ids of free edges
  std::vector<int64_t> lm_edge, lm_plus, lm_minus;  // multipliers in block order
  std::vector<std::array<int64_t, 3>> blocks;       // (a, b, first multiplier)

  // ---- ordering of M = [[A, D], [D^T, 0]]
  int64_t n_m = 0;
  std::vector<int64_t> m_sub, m_edge;  // (subdomain, edge) or (-1, multiplier)
  std::vector<int64_t> owner_m;        // per global edge: M index of its owner copy, -1 for PEC
  int64_t lam_start = 0;               // M index of multiplier 0

  // ---- supernodes == fronts (same ids, elimination order)
  std::vector<int64_t> sn_start, sn_end, sn_kind, sn_owner, parent;
  std::vector<int64_t> struct_ptr, struct_idx;  // update rows per front (sorted M indices)
  std::vector<int32_t> emap;                    // per struct entry: local row in the parent front
  std::vector<int32_t> child_rank;              // position among the parent's children
  std::vector<int32_t> level;                   // height in the assembly tree
  int n_levels = 0;
  std::vector<int32_t> level_fronts, level_ptr;   // fronts grouped by level
  std::vector<int32_t> ea_child, ea_ptr;          // per (level, pass): children to extend-add
  std::vector<int32_t> ea_pass_ptr;               // level -> first pass index into ea_ptr
  std::vector<int64_t> front_off;                 // element offset of the m x m front in the arena
  std::vector<int64_t> piv_off, y_off;            // offsets in pivot arrays / solve buffers
  int64_t arena_elems = 0, piv_total = 0, y_rows = 0;
  int max_front = 0;

  // ---- original entries of M, lower triangle, grouped by level
  std::vector<int64_t> ent_off;   // arena element offset
  std::vector<cplx> ent_val;
  std::vector<int64_t> ent_ptr;   // per level
  std::vector<int64_t> ent_row, ent_col;  // M indices of each entry (diagnostics)

  // ---- global operator A (free edges, full CSR, global numbering) for residuals
  std::vector<int64_t> csr_ptr;
  std::vector<int32_t> csr_col;
  std::vector<cplx> csr_val;

  // ---- flop counts
  double flops[3] = {0, 0, 0};
};

struct Ctx {
  Plan plan;
  d3m_options opt{};
  std::string cache_path;  // copy of opt.autotune_cache
  std::string fault;       // host-side fault injection (environment D3M_FAULT): "", alloc, pivot, nan, timeout
  std::string err;
  DeviceState *dev = nullptr;
  d3m_stats stats{};
  std::vector<double> lvl_ms_panel, lvl_ms_update;  // last profiled factorisation, per level
  std::vector<double> lvl_ms_inv, lvl_ms_tc;
  std::vector<int> lvl_tc, lvl_cs;                   // schedule of the last factorisation
  std::vector<cplx> lambda_host;  // last solve's multipliers, column-major n_lm x nrhs
  int32_t lambda_nrhs = 0;
  bool factored = false;
};

// host_setup.cpp
int build_plan(Ctx &c, const d3m_mesh *mesh, const d3m_materials *mat, double k,
               const d3m_partition *part);
void element_matrices(const double h[3], double S[12][12], double M[12][12]);
void face_matrix(const double h[3], int axis, int side, double T[12][12]);
constexpr int MAX_CELL_NE = 20;  // dofs per cell: 12 bricks, 19 lattice tetrahedra, 6/12/20 mesh orders 1-3
int cell_edges(const Plan &p, int ci, int cj, int ck, int64_t e[MAX_CELL_NE]);
int cell_matrices(const Plan &p, int ci, int cj, int ck, double S[MAX_CELL_NE][MAX_CELL_NE],
                  double M[MAX_CELL_NE][MAX_CELL_NE]);
// Edges and mass matrix of cell c (any element kind; c = i + nx*(j + ny*k)
// on lattices, the tetrahedron index on general meshes); returns the count.
int cell_dofs_mass(const Plan &p, int64_t c, int64_t e[MAX_CELL_NE], double M[MAX_CELL_NE][MAX_CELL_NE]);
int rhs_planewave(const Plan &p, const double *khat_pol, int nrhs, double *rhs, int64_t ldb);

// engine.cu
int dev_factor(Ctx &c);
int dev_solve(Ctx &c, const double *rhs, int64_t ldb, double *x, int64_t ldx, int nrhs,
              d3m_solve_info *info, bool host_ptrs, bool adjoint = false);
int dev_grad_eps(Ctx &c, const double *x, int64_t ldx, const double *y, int64_t ldy, int nrhs,
                 double *grad);
void dev_free(Ctx &c);
int dense_ldlt(int m, int p, int batch, double *A, int32_t *perm, double *dinv, int32_t *info,
               void *stream, std::string &err);

}  // namespace d3m

struct d3m_ctx {
  d3m::Ctx c;
};
