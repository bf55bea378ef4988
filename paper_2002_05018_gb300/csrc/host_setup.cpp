// Host-side set-up of the D^3M plan (no CUDA calls): discretisation of the
// decomposed BVP (Theory section), the multiplier map D of Eq. (1), the
// orderings of main step 3 and the symbolic factorisation of main step 4.
// Everything here runs once per problem; the numeric work is in engine.cu.
#include <algorithm>
#include <cstdlib>
#include <cmath>
#include <cstring>
#include <map>
#include <numeric>
#include <set>
#include <stdexcept>
#include <array>
#include <tuple>

#include "d3m_internal.h"

namespace d3m {

// ------------------------------------------------------------ element algebra
// 1-D integrals of the linear hat pair phi_0 = 1 - t, phi_1 = t on [0, 1]:
// int phi_a phi_b = m1(a, b); phi_a' = sgn(a).
static inline double m1(int a, int b) { return a == b ? 1.0 / 3.0 : 1.0 / 6.0; }
static inline double sgn(int a) { return a ? 1.0 : -1.0; }
static const int OFF[4][2] = {{0, 0}, {1, 0}, {0, 1}, {1, 1}};

// Closed-form stiffness int curl N_a . curl N_b and mass int N_a . N_b of the
// 12 edge functions of a brick (x-edges (a,b): x^ phi_a(y) phi_b(z); y-edges:
// y^ phi_a(x) phi_b(z); z-edges: z^ phi_a(x) phi_b(y)).
void element_matrices(const double h[3], double S[12][12], double M[12][12]) {
  const double hx = h[0], hy = h[1], hz = h[2], vol = hx * hy * hz;
  std::memset(S, 0, sizeof(double) * 144);
  std::memset(M, 0, sizeof(double) * 144);
  // second derivative scale per family: (first curl term axis, second term axis)
  const double dA[3] = {hz, hz, hy};  // term with m_aa' s_b s_b'
  const double dB[3] = {hy, hx, hx};  // term with s_a s_a' m_bb'
  for (int f = 0; f < 3; ++f)
    for (int i = 0; i < 4; ++i)
      for (int j = 0; j < 4; ++j) {
        int a = OFF[i][0], b = OFF[i][1], a2 = OFF[j][0], b2 = OFF[j][1];
        M[4 * f + i][4 * f + j] = vol * m1(a, a2) * m1(b, b2);
        S[4 * f + i][4 * f + j] = vol * (m1(a, a2) * sgn(b) * sgn(b2) / (dA[f] * dA[f]) +
                                         sgn(a) * sgn(a2) * m1(b, b2) / (dB[f] * dB[f]));
      }
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) {
      int a = OFF[i][0], b = OFF[i][1], a2 = OFF[j][0], b2 = OFF[j][1];
      double xy = -sgn(a) * sgn(a2) * m1(b, b2) * vol / (hx * hy);
      double xz = -sgn(b) * sgn(a2) * m1(a, b2) * vol / (hz * hx);
      double yz = -sgn(b) * sgn(b2) * m1(a, a2) * vol / (hz * hy);
      S[i][4 + j] = S[4 + j][i] = xy;
      S[i][8 + j] = S[8 + j][i] = xz;
      S[4 + i][8 + j] = S[8 + j][4 + i] = yz;
    }
}

// Tangential face mass int_face N_t . N_t dS on face {axis = side}.
void face_matrix(const double h[3], int axis, int side, double T[12][12]) {
  std::memset(T, 0, sizeof(double) * 144);
  const double hx = h[0], hy = h[1], hz = h[2];
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) {
      int a = OFF[i][0], b = OFF[i][1], a2 = OFF[j][0], b2 = OFF[j][1];
      if (axis == 2) {  // x-edges and y-edges with z-offset == side
        if (b == side && b2 == side) {
          T[i][j] = hx * hy * m1(a, a2);
          T[4 + i][4 + j] = hx * hy * m1(a, a2);
        }
      } else if (axis == 1) {  // x-edges with y-offset == side, z-edges with y-offset == side
        if (a == side && a2 == side) T[i][j] = hx * hz * m1(b, b2);
        if (b == side && b2 == side) T[8 + i][8 + j] = hx * hz * m1(a, a2);
      } else {  // y-edges and z-edges with x-offset == side
        if (a == side && a2 == side) {
          T[4 + i][4 + j] = hy * hz * m1(b, b2);
          T[8 + i][8 + j] = hy * hz * m1(b, b2);
        }
      }
    }
}

// ------------------------------------------------------------ edge families
// Directions of the edge families; bricks use the first three.
static const int DIRS[7][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}, {1, 1, 0},
                               {1, 0, 1}, {0, 1, 1}, {1, 1, 1}};

static inline int64_t EID(const Plan &p, int d, int64_t i, int64_t j, int64_t k) {
  return p.fam_off[d] + i + p.fam_n[d][0] * (j + p.fam_n[d][1] * k);
}
static inline int64_t EX(const Plan &p, int64_t i, int64_t j, int64_t k) { return EID(p, 0, i, j, k); }
static inline int64_t EY(const Plan &p, int64_t i, int64_t j, int64_t k) { return EID(p, 1, i, j, k); }
static inline int64_t EZ(const Plan &p, int64_t i, int64_t j, int64_t k) { return EID(p, 2, i, j, k); }

// Edges of cell (ci, cj, ck): the 12 brick edges (x-edges at (dy, dz) =
// OFF[q], y-edges at (dx, dz), z-edges at (dx, dy)); tetrahedral cells add
// the (1,1,0) diagonals at dz = 0, 1, the (1,0,1) diagonals at dy = 0, 1, the
// (0,1,1) diagonals at dx = 0, 1 and the cell diagonal.  Returns the count.
int cell_edges(const Plan &p, int ci, int cj, int ck, int64_t e[MAX_CELL_NE]) {
  for (int q = 0; q < 4; ++q) {
    int a = OFF[q][0], b = OFF[q][1];
    e[q] = EX(p, ci, cj + a, ck + b);
    e[4 + q] = EY(p, ci + a, cj, ck + b);
    e[8 + q] = EZ(p, ci + a, cj + b, ck);
  }
  if (p.element != D3M_TET) return 12;
  for (int b = 0; b < 2; ++b) {
    e[12 + b] = EID(p, 3, ci, cj, ck + b);
    e[14 + b] = EID(p, 4, ci, cj + b, ck);
    e[16 + b] = EID(p, 5, ci + b, cj, ck);
  }
  e[18] = EID(p, 6, ci, cj, ck);
  return 19;
}

// Position in cell_edges of the cell edge that starts at vertex offset o
// (each 0/1) with direction d.
static int local_edge(const int o[3], const int d[3]) {
  switch (d[0] + 2 * d[1] + 4 * d[2]) {
    case 1: return o[1] + 2 * o[2];      // (1,0,0)
    case 2: return 4 + o[0] + 2 * o[2];  // (0,1,0)
    case 4: return 8 + o[0] + 2 * o[1];  // (0,0,1)
    case 3: return 12 + o[2];            // (1,1,0)
    case 5: return 14 + o[1];            // (1,0,1)
    case 6: return 16 + o[0];            // (0,1,1)
    default: return 18;                  // (1,1,1)
  }
}

// family and start node of an edge
static inline void edge_info(const Plan &p, int64_t e, int &d, int64_t &i, int64_t &j,
                             int64_t &k) {
  d = 0;
  while (d + 1 < p.nfam && e >= p.fam_off[d + 1]) ++d;
  const int64_t q = e - p.fam_off[d];
  i = q % p.fam_n[d][0];
  const int64_t r = q / p.fam_n[d][0];
  j = r % p.fam_n[d][1];
  k = r / p.fam_n[d][1];
}

// All edges of the cells in box [lo, hi), increasing global id: per family,
// the start nodes in [lo, hi - direction].
template <class F>
static void for_box_edges(const Plan &p, const int lo[3], const int hi[3], F &&fn) {
  for (int d = 0; d < p.nfam; ++d)
    for (int64_t k = lo[2]; k <= hi[2] - DIRS[d][2]; ++k)
      for (int64_t j = lo[1]; j <= hi[1] - DIRS[d][1]; ++j)
        for (int64_t i = lo[0]; i <= hi[0] - DIRS[d][0]; ++i) fn(EID(p, d, i, j, k));
}

// ------------------------------------------------------------ Whitney tetrahedra
// Six tetrahedra per cell: the monotone lattice paths (0,0,0) -> e_a ->
// e_a + e_b -> (1,1,1), one per order (a, b, c) of the axes.  With
// barycentric coordinates lam_i, the edge (a, b) of a tetrahedron carries
// N_ab = l_ab (lam_a grad lam_b - lam_b grad lam_a) (l_ab its length, so the
// dof is the line average of E . t), curl N_ab = 2 l_ab grad lam_a x grad lam_b,
// and int lam_i lam_j = V (1 + [i == j]) / 20 (/ 12 on a triangle of area A).
static const int TET_AXES[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
static const int TET_E[6][2] = {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}};
static const int TRI_E[3][2] = {{0, 1}, {0, 2}, {1, 2}};

static inline void sub3(const double a[3], const double b[3], double o[3]) {
  o[0] = a[0] - b[0];
  o[1] = a[1] - b[1];
  o[2] = a[2] - b[2];
}
static inline void cross3(const double a[3], const double b[3], double o[3]) {
  o[0] = a[1] * b[2] - a[2] * b[1];
  o[1] = a[2] * b[0] - a[0] * b[2];
  o[2] = a[0] * b[1] - a[1] * b[0];
}
static inline double dot3(const double a[3], const double b[3]) {
  return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

static inline void node_pos(const Plan &p, int64_t i, int64_t j, int64_t k, double x[3]) {
  if (p.vert.empty()) {
    x[0] = (double)i * p.h[0];
    x[1] = (double)j * p.h[1];
    x[2] = (double)k * p.h[2];
  } else {
    const double *v = p.vert.data() + 3 * (i + (int64_t)(p.nx + 1) * (j + (int64_t)(p.ny + 1) * k));
    x[0] = v[0];
    x[1] = v[1];
    x[2] = v[2];
  }
}

// Vertex offsets of tetrahedron t of a cell.
static void tet_offsets(int t, int o[4][3]) {
  for (int q = 0; q < 3; ++q) o[0][q] = 0;
  for (int v = 1; v < 4; ++v) {
    for (int q = 0; q < 3; ++q) o[v][q] = o[v - 1][q];
    o[v][TET_AXES[t][v - 1]] = 1;
  }
}

// Barycentric gradients and signed 6 x volume of tetrahedron X.
static double tet_grads(const double X[4][3], double g[4][3]) {
  double e1[3], e2[3], e3[3], c[3];
  sub3(X[1], X[0], e1);
  sub3(X[2], X[0], e2);
  sub3(X[3], X[0], e3);
  cross3(e2, e3, c);
  const double det = dot3(e1, c);
  cross3(e2, e3, g[1]);
  cross3(e3, e1, g[2]);
  cross3(e1, e2, g[3]);
  for (int q = 0; q < 3; ++q) {
    g[1][q] /= det;
    g[2][q] /= det;
    g[3][q] /= det;
    g[0][q] = -(g[1][q] + g[2][q] + g[3][q]);
  }
  return det;
}

// int (lam_a grad lam_b - lam_b grad lam_a) . (lam_c grad lam_d - lam_d grad lam_c)
// in units of the simplex measure / (20 or 12): the bracket of the mass formula.
static inline double whitney_pair(const double g[][3], int a, int b, int c, int d) {
  return (1.0 + (a == c)) * dot3(g[b], g[d]) - (1.0 + (a == d)) * dot3(g[b], g[c]) -
         (1.0 + (b == c)) * dot3(g[a], g[d]) + (1.0 + (b == d)) * dot3(g[a], g[c]);
}

// Orientation sign of tetrahedron t in the regular lattice.
static double tet_parity(int t) {
  int o[4][3];
  tet_offsets(t, o);
  double X[4][3], g[4][3];
  for (int v = 0; v < 4; ++v)
    for (int q = 0; q < 3; ++q) X[v][q] = o[v][q];
  return tet_grads(X, g) > 0 ? 1.0 : -1.0;
}

static void cell_tet(const Plan &p, int ci, int cj, int ck, int t, int o[4][3], double X[4][3]) {
  tet_offsets(t, o);
  for (int v = 0; v < 4; ++v) node_pos(p, ci + o[v][0], cj + o[v][1], ck + o[v][2], X[v]);
}

// Local S and M (6 x 6, edge pairs 01 02 03 12 13 23, each local function
// pointing from its lower to its higher local vertex) of tetrahedron X.
static void tet_local(const double X[4][3], double S[6][6], double M[6][6]) {
  double g[4][3], ell[6], cu[6][3];
  const double vol = std::fabs(tet_grads(X, g)) / 6.0;
  for (int q = 0; q < 6; ++q) {
    const int a = TET_E[q][0], b = TET_E[q][1];
    double ev[3];
    sub3(X[b], X[a], ev);
    ell[q] = std::sqrt(dot3(ev, ev));
    cross3(g[a], g[b], cu[q]);
    for (int r = 0; r < 3; ++r) cu[q][r] *= 2.0 * ell[q];
  }
  for (int q = 0; q < 6; ++q)
    for (int r = 0; r < 6; ++r) {
      S[q][r] = vol * dot3(cu[q], cu[r]);
      M[q][r] = vol / 20.0 * ell[q] * ell[r] * whitney_pair(g, TET_E[q][0], TET_E[q][1], TET_E[r][0], TET_E[r][1]);
    }
}

// int (lam_a grad lam_b + s1 lam_b grad lam_a) . (lam_c grad lam_d + s2 lam_d grad lam_c)
// in units of the simplex measure / (20 or 12); s = -1 for a Whitney
// function, +1 for an edge-gradient function l grad(lam_a lam_b) / l.
static inline double pair_mass(const double g[][3], int a, int b, double s1, int c, int d, double s2) {
  return (1.0 + (a == c)) * dot3(g[b], g[d]) + s2 * (1.0 + (a == d)) * dot3(g[b], g[c]) +
         s1 * (1.0 + (b == c)) * dot3(g[a], g[d]) + s1 * s2 * (1.0 + (b == d)) * dot3(g[a], g[c]);
}

// Order 2: local S and M (12 x 12) of tetrahedron X, the six Whitney functions
// (pairs 01 02 03 12 13 23) then the six edge-gradient functions.
static void tet_local2(const double X[4][3], double S[12][12], double M[12][12]) {
  double S6[6][6], M6[6][6], g[4][3], ell[6];
  tet_local(X, S6, M6);
  const double vol = std::fabs(tet_grads(X, g)) / 6.0;
  for (int q = 0; q < 6; ++q) {
    double ev[3];
    sub3(X[TET_E[q][1]], X[TET_E[q][0]], ev);
    ell[q] = std::sqrt(dot3(ev, ev));
  }
  for (int q = 0; q < 12; ++q)
    for (int r = 0; r < 12; ++r) {
      if (q < 6 && r < 6) {
        S[q][r] = S6[q][r];
        M[q][r] = M6[q][r];
        continue;
      }
      S[q][r] = 0.0;  // the gradient functions have no curl
      const int qq = q % 6, rr = r % 6;
      M[q][r] = vol / 20.0 * ell[qq] * ell[rr] *
                pair_mass(g, TET_E[qq][0], TET_E[qq][1], q < 6 ? -1.0 : 1.0, TET_E[rr][0], TET_E[rr][1],
                          r < 6 ? -1.0 : 1.0);
    }
}

// ---- order 3 (curl-complete second order): functions as sums of terms
// c lam^a v (a monomial in the barycentric coordinates times a constant
// vector); products integrate in closed form,
//   int_T lam^a = (d! |T|) prod a_i! / (|a| + d)!   (d = 3 tetrahedra, 2 triangles).
struct VTerm {
  double c;
  int a[4];
  double v[3];
};
struct VFun {
  int n = 0;
  VTerm t[4];
  void add(double c, const int a[4], const double v[3]) {
    t[n].c = c;
    for (int i = 0; i < 4; ++i) t[n].a[i] = a[i];
    for (int i = 0; i < 3; ++i) t[n].v[i] = v[i];
    ++n;
  }
};

static double fact(int n) {
  double f = 1.0;
  for (int i = 2; i <= n; ++i) f *= i;
  return f;
}

// int lam^a over a simplex of dimension d and measure meas (k vertices)
static double mono_int(const int a[4], int k, int d, double meas) {
  double num = 1.0;
  int deg = 0;
  for (int i = 0; i < k; ++i) {
    num *= fact(a[i]);
    deg += a[i];
  }
  return meas * fact(d) * num / fact(deg + d);
}

static double vfun_dot(const VFun &f, const VFun &g, int k, int d, double meas) {
  double s = 0.0;
  for (int i = 0; i < f.n; ++i)
    for (int j = 0; j < g.n; ++j) {
      int a[4];
      for (int q = 0; q < 4; ++q) a[q] = f.t[i].a[q] + g.t[j].a[q];
      s += f.t[i].c * g.t[j].c * dot3(f.t[i].v, g.t[j].v) * mono_int(a, k, d, meas);
    }
  return s;
}

// curl(lam^a v) = sum_i a_i lam^(a - e_i) grad lam_i x v
static VFun vfun_curl(const VFun &f, const double g[][3]) {
  VFun c;
  for (int i = 0; i < f.n; ++i)
    for (int q = 0; q < 4; ++q)
      if (f.t[i].a[q] > 0) {
        int a[4];
        for (int r = 0; r < 4; ++r) a[r] = f.t[i].a[r];
        a[q] -= 1;
        double v[3];
        cross3(g[q], f.t[i].v, v);
        if (c.n < 4) c.add(f.t[i].c * f.t[i].a[q], a, v);
      }
  return c;
}

// The functions of order 3 on a simplex with barycentric gradients g and
// vertex positions X: the Whitney and the gradient function of each pair
// in `pairs`, then the face functions l_AB lam_C W_AB and l_AC lam_B W_AC of
// the faces listed in `faces` (local vertex indices sorted by global id).
static int order3_functions(const double X[][3], const double g[][3], const int (*pairs)[2], int np,
                            const int (*faces)[3], int nf, VFun *F) {
  int n = 0;
  auto e = [](int i, int j, int a[4]) {
    for (int q = 0; q < 4; ++q) a[q] = 0;
    a[i] += 1;
    if (j >= 0) a[j] += 1;
  };
  auto len = [&](int i, int j) {
    double ev[3];
    sub3(X[j], X[i], ev);
    return std::sqrt(dot3(ev, ev));
  };
  for (int sgn = -1; sgn <= 1; sgn += 2)
    for (int q = 0; q < np; ++q) {
      const int a = pairs[q][0], b = pairs[q][1];
      const double l = len(a, b);
      int ea[4], eb[4];
      e(a, -1, ea);
      e(b, -1, eb);
      VFun f;
      f.add(l, ea, g[b]);
      f.add(sgn * l, eb, g[a]);
      F[n++] = f;
    }
  for (int q = 0; q < nf; ++q) {
    const int A = faces[q][0], B = faces[q][1], C = faces[q][2];
    int e1[4], e2[4];
    VFun f1, f2;
    const double lab = len(A, B), lac = len(A, C);
    e(A, C, e1);
    e(B, C, e2);
    f1.add(lab, e1, g[B]);
    f1.add(-lab, e2, g[A]);
    e(A, B, e1);
    e(C, B, e2);
    f2.add(lac, e1, g[C]);
    f2.add(-lac, e2, g[A]);
    F[n++] = f1;
    F[n++] = f2;
  }
  return n;
}

// S = int curl N . curl N and M = int N . N of a cell, in cell_edges order.
int cell_matrices(const Plan &p, int ci, int cj, int ck, double S[MAX_CELL_NE][MAX_CELL_NE],
                  double M[MAX_CELL_NE][MAX_CELL_NE]) {
  if (p.element != D3M_TET) {
    for (int a = 0; a < 12; ++a)
      for (int b = 0; b < 12; ++b) {
        S[a][b] = p.bS[a][b];
        M[a][b] = p.bM[a][b];
      }
    return 12;
  }
  std::memset(S, 0, sizeof(double) * MAX_CELL_NE * MAX_CELL_NE);
  std::memset(M, 0, sizeof(double) * MAX_CELL_NE * MAX_CELL_NE);
  for (int t = 0; t < 6; ++t) {
    int o[4][3];
    double X[4][3], Sl[6][6], Ml[6][6];
    cell_tet(p, ci, cj, ck, t, o, X);
    tet_local(X, Sl, Ml);
    int loc[6];
    for (int q = 0; q < 6; ++q) {
      const int a = TET_E[q][0], b = TET_E[q][1];
      int d[3] = {o[b][0] - o[a][0], o[b][1] - o[a][1], o[b][2] - o[a][2]};
      loc[q] = local_edge(o[a], d);
    }
    for (int q = 0; q < 6; ++q)
      for (int r = 0; r < 6; ++r) {
        S[loc[q]][loc[r]] += Sl[q][r];
        M[loc[q]][loc[r]] += Ml[q][r];
      }
  }
  return 19;
}

// Signed local matrices of tetrahedron t of a general mesh (global edge
// orientation: from the lower to the higher vertex id; the edge-gradient
// functions of order 2 carry no sign); returns the local dof count.
static const int FACE_OF[4][3] = {{1, 2, 3}, {0, 2, 3}, {0, 1, 3}, {0, 1, 2}};  // face q omits vertex q

static int mesh_tet_matrices(const Plan &p, int64_t t, double S[20][20], double M[20][20]) {
  double X[4][3];
  for (int v = 0; v < 4; ++v) {
    const double *x = p.vert.data() + 3 * p.tet_v[4 * t + v];
    X[v][0] = x[0];
    X[v][1] = x[1];
    X[v][2] = x[2];
  }
  const int nl = p.order == 3 ? 20 : 6 * p.dpe;
  if (p.order == 3) {
    // the local vertices of each face in the order of their global ids
    int faces[4][3];
    for (int q = 0; q < 4; ++q) {
      for (int w = 0; w < 3; ++w) faces[q][w] = FACE_OF[q][w];
      std::sort(faces[q], faces[q] + 3,
                [&](int a, int b) { return p.tet_v[4 * t + a] < p.tet_v[4 * t + b]; });
    }
    double g[4][3];
    const double vol = std::fabs(tet_grads(X, g)) / 6.0;
    VFun F[20], Cu[20];
    order3_functions(X, g, TET_E, 6, faces, 4, F);
    for (int q = 0; q < 20; ++q) Cu[q] = vfun_curl(F[q], g);
    for (int q = 0; q < 20; ++q)
      for (int r = 0; r < 20; ++r) {
        M[q][r] = vfun_dot(F[q], F[r], 4, 3, vol);
        S[q][r] = vfun_dot(Cu[q], Cu[r], 4, 3, vol);
      }
  } else if (p.dpe == 2) {
    double S12[12][12], M12[12][12];
    tet_local2(X, S12, M12);
    for (int q = 0; q < 12; ++q)
      for (int r = 0; r < 12; ++r) {
        S[q][r] = S12[q][r];
        M[q][r] = M12[q][r];
      }
  } else {
    double S6[6][6], M6[6][6];
    tet_local(X, S6, M6);
    for (int q = 0; q < 6; ++q)
      for (int r = 0; r < 6; ++r) {
        S[q][r] = S6[q][r];
        M[q][r] = M6[q][r];
      }
  }
  const int8_t *sg = p.tet_s.data() + 6 * t;
  for (int q = 0; q < nl; ++q)
    for (int r = 0; r < nl; ++r) {
      const double s = (double)((q < 6 ? sg[q] : 1) * (r < 6 ? sg[r] : 1));
      S[q][r] *= s;
      M[q][r] *= s;
    }
  return nl;
}

// Global dof of local function q of tetrahedron t (Whitney q < 6, gradient
// 6 <= q < 12, face functions 12 + 2 k + j of local face k).
static inline int64_t mesh_tet_dof(const Plan &p, int64_t t, int q) {
  if (q < 6) return p.dpe * p.tet_e[6 * t + q];
  if (q < 12) return p.dpe * p.tet_e[6 * t + q - 6] + 1;
  return 2 * p.n_geo + 2 * p.tet_f[4 * t + (q - 12) / 2] + (q - 12) % 2;
}

int cell_dofs_mass(const Plan &p, int64_t c, int64_t e[MAX_CELL_NE], double M[MAX_CELL_NE][MAX_CELL_NE]) {
  if (p.element == D3M_TET_MESH) {
    if (6 * p.dpe + (p.order == 3 ? 8 : 0) > MAX_CELL_NE) return 0;
    double S20[20][20], M20[20][20];
    const int nl = mesh_tet_matrices(p, c, S20, M20);
    for (int q = 0; q < nl; ++q) {
      e[q] = mesh_tet_dof(p, c, q);
      for (int r = 0; r < nl; ++r) M[q][r] = M20[q][r];
    }
    return nl;
  }
  const int ci = (int)(c % p.nx), cj = (int)((c / p.nx) % p.ny), ck = (int)(c / ((int64_t)p.nx * p.ny));
  double S[MAX_CELL_NE][MAX_CELL_NE];
  cell_edges(p, ci, cj, ck, e);
  return cell_matrices(p, ci, cj, ck, S, M);
}

// The two triangles of cell face {axis = side}, split along the diagonal
// from its lowest to its highest corner: vertex offsets.
static void face_tris(int axis, int side, int o[2][3][3]) {
  const int u = axis == 0 ? 1 : 0, v = axis == 2 ? 1 : 2;
  for (int t = 0; t < 2; ++t) {
    for (int w = 0; w < 3; ++w)
      for (int q = 0; q < 3; ++q) o[t][w][q] = 0;
    for (int w = 0; w < 3; ++w) o[t][w][axis] = side;
    o[t][1][t ? v : u] = 1;
    o[t][2][u] = 1;
    o[t][2][v] = 1;
  }
}

// In-plane barycentric gradients of triangle Q: grad mu_i = n x (Q_{i+2} -
// Q_{i+1}) / (2A), n the unit normal; returns the area.
static double tri_grads(const double Q[3][3], double g[3][3]) {
  double e1[3], e2[3], nrm[3];
  sub3(Q[1], Q[0], e1);
  sub3(Q[2], Q[0], e2);
  cross3(e1, e2, nrm);
  const double twoA = std::sqrt(dot3(nrm, nrm));
  for (int q = 0; q < 3; ++q) nrm[q] /= twoA;
  for (int i = 0; i < 3; ++i) {
    double ev[3];
    sub3(Q[(i + 2) % 3], Q[(i + 1) % 3], ev);
    cross3(nrm, ev, g[i]);
    for (int q = 0; q < 3; ++q) g[i][q] /= twoA;
  }
  return 0.5 * twoA;
}

// Local tangential face mass (3 x 3, pairs 01 02 12) of triangle Q.
static void tri_local(const double Q[3][3], double T[3][3]) {
  double g[3][3], ell[3];
  const double area = tri_grads(Q, g);
  for (int q = 0; q < 3; ++q) {
    double ev[3];
    sub3(Q[TRI_E[q][1]], Q[TRI_E[q][0]], ev);
    ell[q] = std::sqrt(dot3(ev, ev));
  }
  for (int q = 0; q < 3; ++q)
    for (int r = 0; r < 3; ++r)
      T[q][r] = area / 12.0 * ell[q] * ell[r] * whitney_pair(g, TRI_E[q][0], TRI_E[q][1], TRI_E[r][0], TRI_E[r][1]);
}

// Order 2: local tangential face mass (6 x 6) of triangle Q (Whitney, then gradients).
static void tri_local2(const double Q[3][3], double T[6][6]) {
  double g[3][3], ell[3];
  const double area = tri_grads(Q, g);
  for (int q = 0; q < 3; ++q) {
    double ev[3];
    sub3(Q[TRI_E[q][1]], Q[TRI_E[q][0]], ev);
    ell[q] = std::sqrt(dot3(ev, ev));
  }
  for (int q = 0; q < 6; ++q)
    for (int r = 0; r < 6; ++r) {
      const int qq = q % 3, rr = r % 3;
      T[q][r] = area / 12.0 * ell[qq] * ell[rr] *
                pair_mass(g, TRI_E[qq][0], TRI_E[qq][1], q < 3 ? -1.0 : 1.0, TRI_E[rr][0], TRI_E[rr][1],
                          r < 3 ? -1.0 : 1.0);
    }
}

// Order 3: local tangential face mass (8 x 8) of triangle Q with vertices in
// the order of their global ids: Whitney and gradient functions of the pairs
// 01 02 12, then the face's l_01 mu_2 W_01 and l_02 mu_1 W_02.
static void tri_local3(const double Q[3][3], double T[8][8]) {
  double g[3][3];
  const double area = tri_grads(Q, g);
  static const int face[1][3] = {{0, 1, 2}};
  VFun F[8];
  order3_functions(Q, g, TRI_E, 3, face, 1, F);
  for (int q = 0; q < 8; ++q)
    for (int r = 0; r < 8; ++r) T[q][r] = vfun_dot(F[q], F[r], 3, 2, area);
}

struct FaceTri {
  double Q[3][3], g[3][3], area, ell[3];
  int loc[3];
};
static void cell_face_tri(const Plan &p, int ci, int cj, int ck, const int o[3][3], FaceTri &f) {
  for (int w = 0; w < 3; ++w) node_pos(p, ci + o[w][0], cj + o[w][1], ck + o[w][2], f.Q[w]);
  f.area = tri_grads(f.Q, f.g);
  for (int q = 0; q < 3; ++q) {
    const int a = TRI_E[q][0], b = TRI_E[q][1];
    int d[3] = {o[b][0] - o[a][0], o[b][1] - o[a][1], o[b][2] - o[a][2]};
    f.loc[q] = local_edge(o[a], d);
    double ev[3];
    sub3(f.Q[b], f.Q[a], ev);
    f.ell[q] = std::sqrt(dot3(ev, ev));
  }
}

// Tangential face mass int_face N_t . N_t dS of face {axis = side} of a cell.
static void cell_face_matrix(const Plan &p, int ci, int cj, int ck, int axis, int side,
                             double T[MAX_CELL_NE][MAX_CELL_NE]) {
  if (p.element != D3M_TET) {
    for (int a = 0; a < 12; ++a)
      for (int b = 0; b < 12; ++b) T[a][b] = p.bT[2 * axis + side][a][b];
    return;
  }
  std::memset(T, 0, sizeof(double) * MAX_CELL_NE * MAX_CELL_NE);
  int o[2][3][3];
  face_tris(axis, side, o);
  for (int t = 0; t < 2; ++t) {
    FaceTri f;
    cell_face_tri(p, ci, cj, ck, o[t], f);
    for (int q = 0; q < 3; ++q)
      for (int r = 0; r < 3; ++r)
        T[f.loc[q]][f.loc[r]] += f.area / 12.0 * f.ell[q] * f.ell[r] *
                                 whitney_pair(f.g, TRI_E[q][0], TRI_E[q][1], TRI_E[r][0], TRI_E[r][1]);
  }
}

static inline int sub_id(const Plan &p, int x, int y, int z) {
  return x + p.parts[0] * (y + p.parts[1] * z);
}
static inline void sub_pos(const Plan &p, int s, int pos[3]) {
  pos[0] = s % p.parts[0];
  pos[1] = (s / p.parts[0]) % p.parts[1];
  pos[2] = s / (p.parts[0] * p.parts[1]);
}
static bool face_adj(const Plan &p, int a, int b) {
  int pa[3], pb[3];
  sub_pos(p, a, pa);
  sub_pos(p, b, pb);
  int diff = 0, tot = 0;
  for (int q = 0; q < 3; ++q) {
    int d = std::abs(pa[q] - pb[q]);
    tot += d;
    diff += d != 0;
  }
  return tot == 1 && diff == 1;
}

// ------------------------------------------------------------ orderings
// Block nested dissection of the subdomain grid (main step 3 reading): split
// the box at the middle cut of its longest axis (ties x < y < z); the
// separator is every block of the box whose two subdomains lie on opposite
// sides of the cut (face neighbours across it on lattice meshes; on general
// meshes also subdomains meeting only along an edge or at a point); order =
// left, right, separator sorted by (a, b).
static void block_nd(const Plan &p, const std::vector<std::pair<int, int>> &pairs, const int lo[3],
                     const int hi[3], std::vector<std::pair<int, int>> &out) {
  int ext[3] = {hi[0] - lo[0], hi[1] - lo[1], hi[2] - lo[2]};
  int axis = 0;
  for (int q = 1; q < 3; ++q)
    if (ext[q] > ext[axis]) axis = q;
  if (ext[axis] <= 1) return;
  const int mid = lo[axis] + ext[axis] / 2;
  std::vector<std::pair<int, int>> left, right, sep;
  for (auto &ab : pairs) {
    int pa[3], pb[3];
    sub_pos(p, ab.first, pa);
    sub_pos(p, ab.second, pb);
    if (pa[axis] < mid && pb[axis] < mid)
      left.push_back(ab);
    else if (pa[axis] >= mid && pb[axis] >= mid)
      right.push_back(ab);
    else
      sep.push_back(ab);
  }
  int lhi[3] = {hi[0], hi[1], hi[2]}, rlo[3] = {lo[0], lo[1], lo[2]};
  lhi[axis] = mid;
  rlo[axis] = mid;
  block_nd(p, left, lo, lhi, out);
  block_nd(p, right, rlo, hi, out);
  std::sort(sep.begin(), sep.end());
  out.insert(out.end(), sep.begin(), sep.end());
}

// Geometric nested dissection of a subdomain's non-interface edges.
static void sub_nd(const Plan &p, std::vector<char> &avail, const int lo[3], const int hi[3],
                   int leaf_max, std::vector<std::vector<int64_t>> &nodes) {
  std::vector<int64_t> E;
  for_box_edges(p, lo, hi, [&](int64_t e) {
    if (avail[e]) E.push_back(e);
  });
  int ext[3] = {hi[0] - lo[0], hi[1] - lo[1], hi[2] - lo[2]};
  int axis = 0;
  for (int q = 1; q < 3; ++q)
    if (ext[q] > ext[axis]) axis = q;
  if ((int64_t)E.size() <= leaf_max || ext[axis] < 2) {
    if (!E.empty()) {
      for (int64_t e : E) avail[e] = 0;
      std::sort(E.begin(), E.end());
      nodes.push_back(std::move(E));
    }
    return;
  }
  int c = lo[axis] + ext[axis] / 2;
  std::vector<int64_t> sep;
  for (int64_t e : E) {
    int d;
    int64_t ijk[3];
    edge_info(p, e, d, ijk[0], ijk[1], ijk[2]);
    if (!DIRS[d][axis] && ijk[axis] == c) sep.push_back(e);  // the edges lying in plane c
  }
  for (int64_t e : sep) avail[e] = 0;
  int lhi[3] = {hi[0], hi[1], hi[2]}, rlo[3] = {lo[0], lo[1], lo[2]};
  lhi[axis] = c;
  rlo[axis] = c;
  sub_nd(p, avail, lo, lhi, leaf_max, nodes);
  sub_nd(p, avail, rlo, hi, leaf_max, nodes);
  if (!sep.empty()) {
    std::sort(sep.begin(), sep.end());
    nodes.push_back(std::move(sep));
  }
}

// ------------------------------------------------------------ assembly helpers
struct Trip {
  int64_t r, c;
  cplx v;
};

// Which subdomain interval(s) along one axis contain node coordinate x
// (closed intervals) -- 1 or 2 results; cell-interval for an along-edge axis.
static int node_intervals(const std::vector<int> &cut, int64_t x, int out[2]) {
  int n = (int)cut.size() - 1;
  int cnt = 0;
  for (int q = 0; q < n; ++q)
    if (cut[q] <= x && x <= cut[q + 1]) out[cnt++] = q;
  return cnt;
}
static int cell_interval(const std::vector<int> &cut, int64_t x) {
  int n = (int)cut.size() - 1;
  for (int q = 0; q < n; ++q)
    if (cut[q] <= x && x < cut[q + 1]) return q;
  return -1;
}

// ------------------------------------------------------------ build
static int finish_plan(Ctx &ctx, std::vector<Trip> &trips, std::vector<Trip> &g);

// ------------------------------------------------------------ general tetrahedral meshes
static inline int64_t mesh_edge_id(const Plan &p, int64_t a, int64_t b) {
  auto it = std::lower_bound(p.medge.begin(), p.medge.end(), std::make_pair(a, b));
  return (it != p.medge.end() && it->first == a && it->second == b) ? (int64_t)(it - p.medge.begin()) : -1;
}

static inline void mesh_vertex(const Plan &p, int64_t v, double x[3]) {
  x[0] = p.vert[3 * v];
  x[1] = p.vert[3 * v + 1];
  x[2] = p.vert[3 * v + 2];
}

// Centroid of tetrahedron t: ((v0 + v1) + v2) + v3 over 4.
static void mesh_centroid(const Plan &p, int64_t t, double c[3]) {
  for (int a = 0; a < 3; ++a) {
    double s = p.vert[3 * p.tet_v[4 * t] + a];
    s += p.vert[3 * p.tet_v[4 * t + 1] + a];
    s += p.vert[3 * p.tet_v[4 * t + 2] + a];
    s += p.vert[3 * p.tet_v[4 * t + 3] + a];
    c[a] = s / 4.0;
  }
}

// Face mass of a triangle with sorted vertices (every local edge along its
// global orientation) and its dofs (Whitney functions of the pairs 01 02 12,
// then at order 2 their gradient functions); returns the dof count.
static int mesh_face(const Plan &p, const int64_t v[3], double T[8][8], int64_t e[8]) {
  double Q[3][3];
  for (int w = 0; w < 3; ++w) mesh_vertex(p, v[w], Q[w]);
  if (p.order == 3) {
    tri_local3(Q, T);
    const std::array<int64_t, 3> key = {v[0], v[1], v[2]};
    const int64_t f = std::lower_bound(p.mface.begin(), p.mface.end(), key) - p.mface.begin();
    for (int q = 0; q < 3; ++q) {
      const int64_t ge = mesh_edge_id(p, v[TRI_E[q][0]], v[TRI_E[q][1]]);
      e[q] = 2 * ge;
      e[3 + q] = 2 * ge + 1;
    }
    e[6] = 2 * p.n_geo + 2 * f;
    e[7] = e[6] + 1;
    return 8;
  }
  if (p.dpe == 2) {
    double T6[6][6];
    tri_local2(Q, T6);
    for (int q = 0; q < 6; ++q)
      for (int r = 0; r < 6; ++r) T[q][r] = T6[q][r];
  } else {
    double T3[3][3];
    tri_local(Q, T3);
    for (int q = 0; q < 3; ++q)
      for (int r = 0; r < 3; ++r) T[q][r] = T3[q][r];
  }
  for (int q = 0; q < 3; ++q) {
    const int64_t ge = mesh_edge_id(p, v[TRI_E[q][0]], v[TRI_E[q][1]]);
    e[q] = p.dpe * ge;
    if (p.dpe == 2) e[3 + q] = 2 * ge + 1;
  }
  return 3 * p.dpe;
}

// Interior ordering of a subdomain of a general mesh: bisection of its
// tetrahedra T at the middle of their centroids' bounding box along its
// longest axis (ties x < y < z; left: centroid below the middle); the still
// unassigned entities (edges; at order 3 also faces, numbered after the
// edges) shared by both halves form the separator; left, right, separator; a
// region of at most leaf_max unassigned entities, or one that does not
// split, is a leaf.  Inside a node entities follow their index.  tent: ept
// entities per tetrahedron.
static void mesh_nd(const Plan &p, const std::vector<double> &cent, std::vector<char> &avail,
                    const std::vector<int64_t> &tent, int ept, const std::vector<int64_t> &T, int leaf_max,
                    std::vector<std::vector<int64_t>> &nodes) {
  auto edges_of = [&](const std::vector<int64_t> &TT, bool only_avail) {
    std::vector<int64_t> E;
    E.reserve(TT.size() * ept);
    for (int64_t t : TT)
      for (int q = 0; q < ept; ++q) {
        const int64_t e = tent[ept * t + q];
        if (!only_avail || avail[e]) E.push_back(e);
      }
    std::sort(E.begin(), E.end());
    E.erase(std::unique(E.begin(), E.end()), E.end());
    return E;
  };
  std::vector<int64_t> E = edges_of(T, true);
  auto leaf = [&]() {
    if (E.empty()) return;
    for (int64_t e : E) avail[e] = 0;
    nodes.push_back(std::move(E));
  };
  if ((int64_t)E.size() <= leaf_max || T.size() < 2) return leaf();
  double lo[3], hi[3];
  for (int a = 0; a < 3; ++a) lo[a] = hi[a] = cent[3 * T[0] + a];
  for (int64_t t : T)
    for (int a = 0; a < 3; ++a) {
      lo[a] = std::min(lo[a], cent[3 * t + a]);
      hi[a] = std::max(hi[a], cent[3 * t + a]);
    }
  const double ext[3] = {hi[0] - lo[0], hi[1] - lo[1], hi[2] - lo[2]};
  int axis = 0;
  for (int q = 1; q < 3; ++q)
    if (ext[q] > ext[axis]) axis = q;
  const double mid = (lo[axis] + hi[axis]) / 2.0;
  std::vector<int64_t> L, R;
  for (int64_t t : T) (cent[3 * t + axis] < mid ? L : R).push_back(t);
  if (L.empty() || R.empty()) return leaf();
  const std::vector<int64_t> EL = edges_of(L, false), ER = edges_of(R, false);
  std::vector<int64_t> both, sep;
  std::set_intersection(EL.begin(), EL.end(), ER.begin(), ER.end(), std::back_inserter(both));
  for (int64_t e : both)
    if (avail[e]) sep.push_back(e);
  for (int64_t e : sep) avail[e] = 0;
  mesh_nd(p, cent, avail, tent, ept, L, leaf_max, nodes);
  mesh_nd(p, cent, avail, tent, ept, R, leaf_max, nodes);
  if (!sep.empty()) nodes.push_back(std::move(sep));
}

// Front half of the plan for a general tetrahedral mesh: edges, faces,
// subdomains by centroid, copies and multipliers, the ordering of M, its
// entries and the global operator.
static int build_plan_mesh(Ctx &ctx, const d3m_mesh *mesh, const d3m_materials *mat, double k,
                           const d3m_partition *part) {
  Plan &p = ctx.plan;
  const int leaf_max = ctx.opt.leaf_max > 0 ? ctx.opt.leaf_max : 64;
  p.k = k;
  p.element = D3M_TET_MESH;
  p.nfam = 0;
  p.nx = p.ny = p.nz = 0;
  if (mesh->order < 0 || mesh->order > 3) {
    ctx.err = "d3m_setup: mesh order must be 0, 1, 2 or 3";
    return D3M_EINVAL;
  }
  p.order = mesh->order <= 1 ? 1 : mesh->order;
  p.dpe = p.order >= 2 ? 2 : 1;
  p.cell_ne = 6 * p.dpe + (p.order == 3 ? 8 : 0);
  const int dpe = p.dpe;
  const int64_t nv = mesh->n_vertices, nt = mesh->n_tets;
  if (nv < 4 || nt < 1 || !mesh->vertices || !mesh->tets) {
    ctx.err = "d3m_setup: a general mesh needs n_vertices >= 4, n_tets >= 1, vertices and tets";
    return D3M_EINVAL;
  }
  if (ctx.opt.lm_weight != 0) {
    ctx.err = "d3m_setup: lm_weight = 1 needs a lattice mesh";
    return D3M_EINVAL;
  }
  p.vert.assign(mesh->vertices, mesh->vertices + 3 * nv);
  for (double x : p.vert)
    if (!std::isfinite(x)) {
      ctx.err = "d3m_setup: non-finite vertex position";
      return D3M_EINVAL;
    }
  p.tet_v.assign(mesh->tets, mesh->tets + 4 * nt);
  p.n_cells = nt;
  for (int64_t t = 0; t < nt; ++t) {
    const int64_t *v = p.tet_v.data() + 4 * t;
    double X[4][3], g[4][3], lmax = 0.0;
    for (int a = 0; a < 4; ++a) {
      if (v[a] < 0 || v[a] >= nv) {
        ctx.err = "d3m_setup: tetrahedron vertex id out of range";
        return D3M_EINVAL;
      }
      mesh_vertex(p, v[a], X[a]);
    }
    for (int q = 0; q < 6; ++q) {
      double ev[3];
      sub3(X[TET_E[q][1]], X[TET_E[q][0]], ev);
      lmax = std::max(lmax, std::sqrt(dot3(ev, ev)));
    }
    const double det = tet_grads(X, g);
    if (!(std::fabs(det) > 1e-12 * lmax * lmax * lmax)) {
      ctx.err = "d3m_setup: a tetrahedron is degenerate";
      return D3M_EINVAL;
    }
  }
  // ---- edges: distinct vertex pairs, lexicographic
  p.medge.clear();
  p.medge.reserve(6 * nt);
  for (int64_t t = 0; t < nt; ++t)
    for (int q = 0; q < 6; ++q) {
      const int64_t a = p.tet_v[4 * t + TET_E[q][0]], b = p.tet_v[4 * t + TET_E[q][1]];
      p.medge.push_back({std::min(a, b), std::max(a, b)});
    }
  std::sort(p.medge.begin(), p.medge.end());
  p.medge.erase(std::unique(p.medge.begin(), p.medge.end()), p.medge.end());
  const int64_t n_geo = (int64_t)p.medge.size();
  p.n_geo = n_geo;
  p.tet_e.resize(6 * nt);
  p.tet_s.resize(6 * nt);
  for (int64_t t = 0; t < nt; ++t)
    for (int q = 0; q < 6; ++q) {
      const int64_t a = p.tet_v[4 * t + TET_E[q][0]], b = p.tet_v[4 * t + TET_E[q][1]];
      p.tet_e[6 * t + q] = mesh_edge_id(p, std::min(a, b), std::max(a, b));
      p.tet_s[6 * t + q] = a < b ? 1 : -1;
    }
  // ---- faces: boundary triangles (one tetrahedron) and shared ones (two)
  struct FRec {
    std::array<int64_t, 3> v;
    int64_t t, opp;
    int q;
  };
  std::vector<FRec> fr;
  fr.reserve(4 * nt);
  for (int64_t t = 0; t < nt; ++t)
    for (int q = 0; q < 4; ++q) {
      std::array<int64_t, 3> v;
      int w = 0;
      for (int a = 0; a < 4; ++a)
        if (a != q) v[w++] = p.tet_v[4 * t + a];
      std::sort(v.begin(), v.end());
      fr.push_back({v, t, p.tet_v[4 * t + q], q});
    }
  std::sort(fr.begin(), fr.end(), [](const FRec &a, const FRec &b) { return a.v != b.v ? a.v < b.v : a.t < b.t; });
  p.bface.clear();
  p.mface.clear();
  p.tet_f.assign(4 * nt, -1);
  std::vector<int64_t> bface_tet;
  std::vector<std::array<int64_t, 5>> iface;  // sorted vertices, the two tetrahedra
  for (size_t i = 0; i < fr.size();) {
    size_t j = i;
    while (j < fr.size() && fr[j].v == fr[i].v) ++j;
    for (size_t r = i; r < j; ++r) p.tet_f[4 * fr[r].t + fr[r].q] = (int64_t)p.mface.size();
    p.mface.push_back(fr[i].v);
    if (j - i == 1) {
      p.bface.push_back({fr[i].v[0], fr[i].v[1], fr[i].v[2], fr[i].opp});
      bface_tet.push_back(fr[i].t);
    } else if (j - i == 2) {
      iface.push_back({fr[i].v[0], fr[i].v[1], fr[i].v[2], fr[i].t, fr[i + 1].t});
    } else {
      ctx.err = "d3m_setup: a triangle is shared by more than two tetrahedra";
      return D3M_EINVAL;
    }
    i = j;
  }
  p.n_faces = (int64_t)p.mface.size();
  p.n_edges = dpe * n_geo + (p.order == 3 ? 2 * p.n_faces : 0);  // dofs
  // ---- materials
  if (!mat || !mat->eps_r) {
    ctx.err = "d3m_setup: eps_r is required";
    return D3M_EINVAL;
  }
  p.eps.resize(nt);
  for (int64_t t = 0; t < nt; ++t) p.eps[t] = cplx(mat->eps_r[2 * t], mat->eps_r[2 * t + 1]);
  p.pec.assign(p.n_edges, 0);
  if (mat->pec_edge)
    for (int64_t e = 0; e < p.n_edges; ++e) p.pec[e] = mat->pec_edge[e] ? 1 : 0;
  for (int64_t e = 0; dpe == 2 && e < p.n_edges / 2; ++e)
    if (p.pec[2 * e] != p.pec[2 * e + 1]) {
      ctx.err = "d3m_setup: pec_edge must mark both dofs of an edge (or face) alike";
      return D3M_EINVAL;
    }
  p.n_free = 0;
  for (int64_t e = 0; e < p.n_edges; ++e) p.n_free += !p.pec[e];
  // ---- subdomains: coordinate boxes, a tetrahedron goes where its centroid is
  p.parts[0] = part->px;
  p.parts[1] = part->py;
  p.parts[2] = part->pz;
  const double *gc[3] = {part->gx, part->gy, part->gz};
  std::vector<double> gcut[3];
  for (int a = 0; a < 3; ++a) {
    if (p.parts[a] < 1 || !gc[a]) {
      ctx.err = "d3m_setup: a general mesh needs partition counts >= 1 with coordinate cuts gx, gy, gz";
      return D3M_EINVAL;
    }
    gcut[a].assign(gc[a], gc[a] + p.parts[a] + 1);
    for (int q = 0; q < p.parts[a]; ++q)
      if (!(gcut[a][q + 1] > gcut[a][q])) {
        ctx.err = "d3m_setup: coordinate cuts must be strictly increasing";
        return D3M_EINVAL;
      }
  }
  p.nsub = p.parts[0] * p.parts[1] * p.parts[2];
  std::vector<double> cent(3 * nt);
  std::vector<int> tsub(nt);
  std::vector<std::vector<int64_t>> sub_tets(p.nsub);
  for (int64_t t = 0; t < nt; ++t) {
    mesh_centroid(p, t, &cent[3 * t]);
    int ix[3];
    for (int a = 0; a < 3; ++a)
      ix[a] = (int)(std::upper_bound(gcut[a].begin() + 1, gcut[a].end() - 1, cent[3 * t + a]) - (gcut[a].begin() + 1));
    tsub[t] = sub_id(p, ix[0], ix[1], ix[2]);
    sub_tets[tsub[t]].push_back(t);
  }
  for (int s = 0; s < p.nsub; ++s)
    if (sub_tets[s].empty()) {
      ctx.err = "d3m_setup: a subdomain box holds no tetrahedron";
      return D3M_EINVAL;
    }
  p.sub_lo.assign(p.nsub, {0, 0, 0});
  p.sub_hi.assign(p.nsub, {0, 0, 0});
  // entities carrying dofs: the edges, then (order 3) the faces
  const int ept = p.order == 3 ? 10 : 6;
  const int64_t n_ent = n_geo + (p.order == 3 ? p.n_faces : 0);
  std::vector<int64_t> tent((size_t)ept * nt);
  for (int64_t t = 0; t < nt; ++t) {
    for (int q = 0; q < 6; ++q) tent[ept * t + q] = p.tet_e[6 * t + q];
    if (p.order == 3)
      for (int q = 0; q < 4; ++q) tent[ept * t + 6 + q] = n_geo + p.tet_f[4 * t + q];
  }
  const int de = p.order == 1 ? 1 : 2;  // dofs per entity
  auto ent_dof = [&](int64_t e, int q) { return e < n_geo ? dpe * e + q : 2 * n_geo + 2 * (e - n_geo) + q; };
  auto dof_ent = [&](int64_t d) { return d < dpe * n_geo ? d / dpe : n_geo + (d - 2 * n_geo) / 2; };
  p.sub_edges.assign(p.nsub, {});  // free dofs of each subdomain
  std::vector<std::vector<int64_t>> sub_geo(p.nsub);  // its entities
  for (int s = 0; s < p.nsub; ++s) {
    auto &G = sub_geo[s];
    for (int64_t t : sub_tets[s])
      for (int q = 0; q < ept; ++q) G.push_back(tent[ept * t + q]);
    std::sort(G.begin(), G.end());
    G.erase(std::unique(G.begin(), G.end()), G.end());
    for (int64_t e : G)
      for (int q = 0; q < de; ++q)
        if (!p.pec[ent_dof(e, q)]) p.sub_edges[s].push_back(ent_dof(e, q));
  }
  // ---- copies and multipliers (per dof)
  std::vector<std::vector<int>> copies(p.n_edges);
  for (int s = 0; s < p.nsub; ++s)
    for (int64_t e : p.sub_edges[s]) copies[e].push_back(s);
  std::map<std::pair<int, int>, std::vector<int64_t>> pair_edges;
  for (int64_t e = 0; e < p.n_edges; ++e) {
    const auto &cs = copies[e];
    for (size_t kk = 1; kk < cs.size(); ++kk) {
      int sj = cs[0];
      for (size_t j = 0; j < kk; ++j)
        if (face_adj(p, cs[j], cs[kk])) {
          sj = cs[j];
          break;
        }
      pair_edges[{sj, cs[kk]}].push_back(e);
    }
  }
  std::vector<std::pair<int, int>> pairs, border;
  for (auto &kv : pair_edges) pairs.push_back(kv.first);
  {
    int lo[3] = {0, 0, 0}, hi[3] = {p.parts[0], p.parts[1], p.parts[2]};
    block_nd(p, pairs, lo, hi, border);
  }
  p.lm_edge.clear();
  p.lm_plus.clear();
  p.lm_minus.clear();
  p.blocks.clear();
  for (auto &ab : border) {
    auto &es = pair_edges[ab];
    p.blocks.push_back({ab.first, ab.second, (int64_t)p.lm_edge.size()});
    for (int64_t e : es) {
      p.lm_edge.push_back(e);
      p.lm_plus.push_back(ab.first);
      p.lm_minus.push_back(ab.second);
    }
  }
  const int64_t n_lm = (int64_t)p.lm_edge.size();
  // ---- ordering of M and supernodes
  p.m_sub.clear();
  p.m_edge.clear();
  p.sn_start.clear();
  p.sn_end.clear();
  p.sn_kind.clear();
  p.sn_owner.clear();
  auto push_node = [&](int s, const std::vector<int64_t> &nd, int kind, int64_t owner) {
    p.sn_start.push_back((int64_t)p.m_sub.size());
    for (int64_t e : nd) {
      p.m_sub.push_back(s);
      p.m_edge.push_back(e);
    }
    p.sn_end.push_back((int64_t)p.m_sub.size());
    p.sn_kind.push_back(kind);
    p.sn_owner.push_back(owner);
  };
  std::vector<char> avail(n_ent, 0);  // per entity
  std::vector<int64_t> sub_m0(p.nsub);
  for (int s = 0; s < p.nsub; ++s) {
    sub_m0[s] = (int64_t)p.m_sub.size();
    // an entity is ordered inside the subdomain when it has a free dof there
    // and none of its dofs is an interface dof
    for (int64_t d : p.sub_edges[s]) avail[dof_ent(d)] = 1;
    for (int64_t d : p.sub_edges[s])
      if (copies[d].size() >= 2) avail[dof_ent(d)] = 0;
    std::vector<std::vector<int64_t>> nodes;
    mesh_nd(p, cent, avail, tent, ept, sub_tets[s], leaf_max, nodes);
    for (auto &nd : nodes) {
      std::vector<int64_t> dofs;
      for (int64_t e : nd)
        for (int q = 0; q < de; ++q) dofs.push_back(ent_dof(e, q));
      push_node(s, dofs, 0, s);
    }
    for (int64_t e : sub_geo[s]) avail[e] = 0;
    std::vector<int64_t> B;
    for (int64_t e : p.sub_edges[s])
      if (copies[e].size() >= 2) B.push_back(e);
    if (!B.empty()) push_node(s, B, 1, s);
  }
  p.lam_start = (int64_t)p.m_sub.size();
  for (size_t b = 0; b < p.blocks.size(); ++b) {
    const int64_t first = p.blocks[b][2], last = b + 1 < p.blocks.size() ? p.blocks[b + 1][2] : n_lm;
    std::vector<int64_t> ls;
    for (int64_t l = first; l < last; ++l) ls.push_back(l);
    push_node(-1, ls, 2, (int64_t)b);
  }
  p.n_m = (int64_t)p.m_sub.size();
  std::vector<int64_t> gm(p.n_edges, -1);
  p.owner_m.assign(p.n_edges, -1);
  for (int64_t v = 0; v < p.lam_start; ++v) {
    const int64_t e = p.m_edge[v];
    const int s = (int)p.m_sub[v];
    if (!copies[e].empty() && copies[e][0] == s) p.owner_m[e] = v;
  }
  // ---- entries of M (lower triangle), per subdomain
  const cplx jk(0.0, k);
  const cplx alpha = (ctx.opt.alpha_re == 0.0 && ctx.opt.alpha_im == 0.0) ? jk
                                                                         : cplx(ctx.opt.alpha_re, ctx.opt.alpha_im);
  // faces of each subdomain: (face record, coefficient)
  std::vector<std::vector<std::pair<std::array<int64_t, 3>, cplx>>> sub_faces(p.nsub);
  for (size_t f = 0; f < p.bface.size(); ++f)
    sub_faces[tsub[bface_tet[f]]].push_back({{p.bface[f][0], p.bface[f][1], p.bface[f][2]}, jk});
  for (auto &f : iface) {
    const int s0 = tsub[f[3]], s1 = tsub[f[4]];
    if (s0 == s1) continue;
    sub_faces[s0].push_back({{f[0], f[1], f[2]}, s1 > s0 ? alpha : -alpha});
    sub_faces[s1].push_back({{f[0], f[1], f[2]}, s0 > s1 ? alpha : -alpha});
  }
  std::vector<Trip> trips;
  for (int s = 0; s < p.nsub; ++s) {
    const int64_t m0 = sub_m0[s];
    const int64_t m1_ = s + 1 < p.nsub ? sub_m0[s + 1] : p.lam_start;
    for (int64_t v = m0; v < m1_; ++v) gm[p.m_edge[v]] = v;
    for (int64_t t : sub_tets[s]) {
      double S20[20][20], M20[20][20];
      const int nl = mesh_tet_matrices(p, t, S20, M20);
      int64_t e[20];
      for (int q = 0; q < nl; ++q) e[q] = mesh_tet_dof(p, t, q);
      for (int a = 0; a < nl; ++a) {
        const int64_t ra = p.pec[e[a]] ? -1 : gm[e[a]];
        if (ra < 0) continue;
        for (int b = 0; b < nl; ++b) {
          const int64_t rb = p.pec[e[b]] ? -1 : gm[e[b]];
          if (rb < 0 || ra < rb) continue;
          const cplx v = S20[a][b] - k * k * p.eps[t] * M20[a][b];
          if (v != cplx(0.0)) trips.push_back({ra, rb, v});
        }
      }
    }
    for (auto &fc : sub_faces[s]) {
      double T8[8][8];
      int64_t e[8];
      const int nf = mesh_face(p, fc.first.data(), T8, e);
      for (int a = 0; a < nf; ++a) {
        const int64_t ra = p.pec[e[a]] ? -1 : gm[e[a]];
        if (ra < 0) continue;
        for (int b = 0; b < nf; ++b) {
          const int64_t rb = p.pec[e[b]] ? -1 : gm[e[b]];
          if (rb < 0 || ra < rb || T8[a][b] == 0.0) continue;
          trips.push_back({ra, rb, fc.second * T8[a][b]});
        }
      }
    }
    // multipliers: +1 on the lower-index copy, -1 on the other
    for (int64_t l = 0; l < n_lm; ++l) {
      if (p.lm_plus[l] == s) trips.push_back({p.lam_start + l, gm[p.lm_edge[l]], cplx(1.0, 0.0)});
      if (p.lm_minus[l] == s) trips.push_back({p.lam_start + l, gm[p.lm_edge[l]], cplx(-1.0, 0.0)});
    }
    for (int64_t v = m0; v < m1_; ++v) gm[p.m_edge[v]] = -1;
  }
  // ---- global operator: every tetrahedron and the boundary triangles
  std::vector<Trip> g;
  g.reserve((size_t)nt * 36 * dpe * dpe);
  for (int64_t t = 0; t < nt; ++t) {
    double S20[20][20], M20[20][20];
    const int nl = mesh_tet_matrices(p, t, S20, M20);
    int64_t e[20];
    for (int q = 0; q < nl; ++q) e[q] = mesh_tet_dof(p, t, q);
    for (int a = 0; a < nl; ++a) {
      if (p.pec[e[a]]) continue;
      for (int b = 0; b < nl; ++b) {
        if (p.pec[e[b]]) continue;
        const cplx v = S20[a][b] - k * k * p.eps[t] * M20[a][b];
        if (v != cplx(0.0)) g.push_back({e[a], e[b], v});
      }
    }
  }
  for (auto &bf : p.bface) {
    double T8[8][8];
    int64_t e[8];
    const int nf = mesh_face(p, bf.data(), T8, e);
    for (int a = 0; a < nf; ++a) {
      if (p.pec[e[a]]) continue;
      for (int b = 0; b < nf; ++b)
        if (!p.pec[e[b]] && T8[a][b] != 0.0) g.push_back({e[a], e[b], jk * T8[a][b]});
    }
  }
  return finish_plan(ctx, trips, g);
}


int build_plan(Ctx &ctx, const d3m_mesh *mesh, const d3m_materials *mat, double k,
               const d3m_partition *part) {
  if (mesh->element == D3M_TET_MESH) return build_plan_mesh(ctx, mesh, mat, k, part);
  Plan &p = ctx.plan;
  const int leaf_max = ctx.opt.leaf_max > 0 ? ctx.opt.leaf_max : 64;
  p.nx = mesh->nx;
  p.ny = mesh->ny;
  p.nz = mesh->nz;
  p.lx = mesh->lx;
  p.ly = mesh->ly;
  p.lz = mesh->lz;
  p.k = k;
  if (p.nx < 1 || p.ny < 1 || p.nz < 1 || !(p.lx > 0) || !(p.ly > 0) || !(p.lz > 0)) {
    ctx.err = "d3m_setup: mesh sizes must be positive";
    return D3M_EINVAL;
  }
  p.h[0] = p.lx / p.nx;
  p.h[1] = p.ly / p.ny;
  p.h[2] = p.lz / p.nz;
  p.element = mesh->element;
  if (p.element != D3M_BRICK && p.element != D3M_TET) {
    ctx.err = "d3m_setup: mesh element must be D3M_BRICK, D3M_TET or D3M_TET_MESH";
    return D3M_EINVAL;
  }
  if (mesh->order != 0 && mesh->order != 1) {
    ctx.err = "d3m_setup: order 2 is for general meshes (D3M_TET_MESH)";
    return D3M_EINVAL;
  }
  if (mesh->vertices && p.element != D3M_TET) {
    ctx.err = "d3m_setup: vertex positions are for tetrahedral meshes only";
    return D3M_EINVAL;
  }
  p.nfam = p.element == D3M_TET ? 7 : 3;
  p.cell_ne = p.element == D3M_TET ? 19 : 12;
  p.fam_off[0] = 0;
  for (int d = 0; d < p.nfam; ++d) {
    p.fam_n[d][0] = p.nx + 1 - DIRS[d][0];
    p.fam_n[d][1] = p.ny + 1 - DIRS[d][1];
    p.fam_n[d][2] = p.nz + 1 - DIRS[d][2];
    p.fam_off[d + 1] = p.fam_off[d] + p.fam_n[d][0] * p.fam_n[d][1] * p.fam_n[d][2];
  }
  p.nex = p.fam_off[1];
  p.ney = p.fam_off[2] - p.fam_off[1];
  p.nez = p.fam_off[3] - p.fam_off[2];
  p.n_edges = p.fam_off[p.nfam];
  const int64_t ncell = (int64_t)p.nx * p.ny * p.nz;
  p.n_cells = ncell;
  p.vert.clear();
  if (mesh->vertices) {
    const int64_t nn3 = 3 * (int64_t)(p.nx + 1) * (p.ny + 1) * (p.nz + 1);
    p.vert.assign(mesh->vertices, mesh->vertices + nn3);
    const int nmax[3] = {p.nx, p.ny, p.nz};
    const double len[3] = {p.lx, p.ly, p.lz};
    for (int64_t k = 0; k <= p.nz; ++k)
      for (int64_t j = 0; j <= p.ny; ++j)
        for (int64_t i = 0; i <= p.nx; ++i) {
          const int64_t ijk[3] = {i, j, k};
          double x[3];
          node_pos(p, i, j, k, x);
          for (int a = 0; a < 3; ++a) {
            if (!std::isfinite(x[a])) {
              ctx.err = "d3m_setup: non-finite vertex position";
              return D3M_EINVAL;
            }
            const bool lo = ijk[a] == 0, hi = ijk[a] == nmax[a];
            if ((lo && std::fabs(x[a]) > 1e-12 * len[a]) || (hi && std::fabs(x[a] - len[a]) > 1e-12 * len[a])) {
              ctx.err = "d3m_setup: a boundary vertex left its boundary plane";
              return D3M_EINVAL;
            }
          }
        }
  }
  if (p.element == D3M_TET) {
    for (int t = 0; t < 6; ++t) {
      const double par = tet_parity(t);
      for (int ck = 0; ck < p.nz; ++ck)
        for (int cj = 0; cj < p.ny; ++cj)
          for (int ci = 0; ci < p.nx; ++ci) {
            int o[4][3];
            double X[4][3], g[4][3];
            cell_tet(p, ci, cj, ck, t, o, X);
            if (!(par * tet_grads(X, g) > 0.0)) {
              ctx.err = "d3m_setup: a tetrahedron is inverted or degenerate";
              return D3M_EINVAL;
            }
          }
    }
  }
  element_matrices(p.h, p.bS, p.bM);
  for (int axis = 0; axis < 3; ++axis)
    for (int side = 0; side < 2; ++side) face_matrix(p.h, axis, side, p.bT[2 * axis + side]);
  if (!mat || !mat->eps_r) {
    ctx.err = "d3m_setup: eps_r is required";
    return D3M_EINVAL;
  }
  p.eps.resize(ncell);
  for (int64_t c = 0; c < ncell; ++c) p.eps[c] = cplx(mat->eps_r[2 * c], mat->eps_r[2 * c + 1]);
  p.pec.assign(p.n_edges, 0);
  if (mat->pec_edge)
    for (int64_t e = 0; e < p.n_edges; ++e) p.pec[e] = mat->pec_edge[e] ? 1 : 0;
  p.parts[0] = part->px;
  p.parts[1] = part->py;
  p.parts[2] = part->pz;
  const int32_t *cp[3] = {part->cx, part->cy, part->cz};
  const int nn[3] = {p.nx, p.ny, p.nz};
  for (int a = 0; a < 3; ++a) {
    if (p.parts[a] < 1 || !cp[a]) {
      ctx.err = "d3m_setup: partition counts must be >= 1 with cut arrays";
      return D3M_EINVAL;
    }
    p.cuts[a].assign(cp[a], cp[a] + p.parts[a] + 1);
    if (p.cuts[a].front() != 0 || p.cuts[a].back() != nn[a]) {
      ctx.err = "d3m_setup: cuts must start at 0 and end at the cell count";
      return D3M_EINVAL;
    }
    for (int q = 0; q < p.parts[a]; ++q)
      if (p.cuts[a][q + 1] <= p.cuts[a][q]) {
        ctx.err = "d3m_setup: cuts must be strictly increasing";
        return D3M_EINVAL;
      }
  }
  p.nsub = p.parts[0] * p.parts[1] * p.parts[2];
  p.n_free = 0;
  for (int64_t e = 0; e < p.n_edges; ++e) p.n_free += !p.pec[e];

  // ---- subdomain boxes and edges
  p.sub_lo.resize(p.nsub);
  p.sub_hi.resize(p.nsub);
  p.sub_edges.assign(p.nsub, {});
  for (int s = 0; s < p.nsub; ++s) {
    int pos[3];
    sub_pos(p, s, pos);
    for (int a = 0; a < 3; ++a) {
      p.sub_lo[s][a] = p.cuts[a][pos[a]];
      p.sub_hi[s][a] = p.cuts[a][pos[a] + 1];
    }
    for_box_edges(p, p.sub_lo[s].data(), p.sub_hi[s].data(), [&](int64_t e) {
      if (!p.pec[e]) p.sub_edges[s].push_back(e);
    });
  }

  // ---- copies of each edge (sorted subdomain lists) and multipliers
  // copies are only needed for edges on interior cut planes
  std::vector<int> ncopy(p.n_edges, 0);
  std::vector<std::array<int, 4>> copies(p.n_edges);
  for (int64_t e = 0; e < p.n_edges; ++e) {
    if (p.pec[e]) continue;
    int d;
    int64_t ijk[3];
    edge_info(p, e, d, ijk[0], ijk[1], ijk[2]);
    int iv[3][2], cnt[3];
    for (int a = 0; a < 3; ++a) {
      if (DIRS[d][a]) {
        iv[a][0] = cell_interval(p.cuts[a], ijk[a]);
        cnt[a] = 1;
      } else {
        cnt[a] = node_intervals(p.cuts[a], ijk[a], iv[a]);
      }
    }
    std::vector<int> lst;
    for (int z = 0; z < cnt[2]; ++z)
      for (int y = 0; y < cnt[1]; ++y)
        for (int x = 0; x < cnt[0]; ++x) lst.push_back(sub_id(p, iv[0][x], iv[1][y], iv[2][z]));
    std::sort(lst.begin(), lst.end());
    ncopy[e] = (int)lst.size();
    for (size_t q = 0; q < lst.size(); ++q) copies[e][q] = lst[q];
  }
  std::map<std::pair<int, int>, std::vector<int64_t>> pair_edges;
  for (int64_t e = 0; e < p.n_edges; ++e) {
    for (int kk = 1; kk < ncopy[e]; ++kk) {
      int sk = copies[e][kk], sj = -1;
      for (int j = 0; j < kk; ++j)
        if (face_adj(p, copies[e][j], sk)) {
          sj = copies[e][j];
          break;
        }
      if (sj < 0) {
        ctx.err = "d3m_setup: internal error (copy without face neighbour)";
        return D3M_EINVAL;
      }
      pair_edges[{sj, sk}].push_back(e);
    }
  }
  std::vector<std::pair<int, int>> pairs;
  for (auto &kv : pair_edges) pairs.push_back(kv.first);
  std::vector<std::pair<int, int>> border;
  {
    int lo[3] = {0, 0, 0}, hi[3] = {p.parts[0], p.parts[1], p.parts[2]};
    block_nd(p, pairs, lo, hi, border);
  }
  p.lm_edge.clear();
  p.lm_plus.clear();
  p.lm_minus.clear();
  p.blocks.clear();
  for (auto &ab : border) {
    auto &es = pair_edges[ab];  // already increasing
    p.blocks.push_back({ab.first, ab.second, (int64_t)p.lm_edge.size()});
    for (int64_t e : es) {
      p.lm_edge.push_back(e);
      p.lm_plus.push_back(ab.first);
      p.lm_minus.push_back(ab.second);
    }
  }
  const int64_t n_lm = (int64_t)p.lm_edge.size();

  // ---- M ordering and supernodes
  p.m_sub.clear();
  p.m_edge.clear();
  p.sn_start.clear();
  p.sn_end.clear();
  p.sn_kind.clear();
  p.sn_owner.clear();
  std::vector<char> avail(p.n_edges, 0);
  std::vector<int64_t> sub_m0(p.nsub);  // first M index of each subdomain
  std::vector<std::vector<int64_t>> sub_mindex(p.nsub);  // M index of each local edge
  for (int s = 0; s < p.nsub; ++s) {
    sub_m0[s] = (int64_t)p.m_sub.size();
    for (int64_t e : p.sub_edges[s]) avail[e] = ncopy[e] < 2;  // interface dofs excluded
    std::vector<std::vector<int64_t>> nodes;
    sub_nd(p, avail, p.sub_lo[s].data(), p.sub_hi[s].data(), leaf_max, nodes);
    for (auto &nd : nodes) {
      p.sn_start.push_back((int64_t)p.m_sub.size());
      for (int64_t e : nd) {
        p.m_sub.push_back(s);
        p.m_edge.push_back(e);
      }
      p.sn_end.push_back((int64_t)p.m_sub.size());
      p.sn_kind.push_back(0);
      p.sn_owner.push_back(s);
    }
    for (int64_t e : p.sub_edges[s]) avail[e] = 0;
    std::vector<int64_t> B;
    for (int64_t e : p.sub_edges[s])
      if (ncopy[e] >= 2) B.push_back(e);
    if (!B.empty()) {
      p.sn_start.push_back((int64_t)p.m_sub.size());
      for (int64_t e : B) {
        p.m_sub.push_back(s);
        p.m_edge.push_back(e);
      }
      p.sn_end.push_back((int64_t)p.m_sub.size());
      p.sn_kind.push_back(1);
      p.sn_owner.push_back(s);
    }
  }
  p.lam_start = (int64_t)p.m_sub.size();
  for (size_t b = 0; b < p.blocks.size(); ++b) {
    int64_t first = p.blocks[b][2];
    int64_t last = b + 1 < p.blocks.size() ? p.blocks[b + 1][2] : n_lm;
    p.sn_start.push_back((int64_t)p.m_sub.size());
    for (int64_t l = first; l < last; ++l) {
      p.m_sub.push_back(-1);
      p.m_edge.push_back(l);
    }
    p.sn_end.push_back((int64_t)p.m_sub.size());
    p.sn_kind.push_back(2);
    p.sn_owner.push_back((int64_t)b);
  }
  p.n_m = (int64_t)p.m_sub.size();

  // per subdomain: global edge -> M index (dense scratch reused)
  std::vector<int64_t> gm(p.n_edges, -1);
  p.owner_m.assign(p.n_edges, -1);
  for (int64_t v = 0; v < p.lam_start; ++v) {
    int64_t e = p.m_edge[v];
    int s = (int)p.m_sub[v];
    if (ncopy[e] >= 1 && copies[e][0] == s) p.owner_m[e] = v;
  }

  // ---- entries of M (lower triangle), per subdomain
  const cplx jk(0.0, k);
  // interface loss/gain coefficient (d3m_options.alpha_re/im; 0 -> jk)
  const cplx alpha = (ctx.opt.alpha_re == 0.0 && ctx.opt.alpha_im == 0.0) ? jk
                                                                         : cplx(ctx.opt.alpha_re, ctx.opt.alpha_im);
  std::vector<Trip> trips;
  double Sc[MAX_CELL_NE][MAX_CELL_NE], Mc[MAX_CELL_NE][MAX_CELL_NE], Tf[MAX_CELL_NE][MAX_CELL_NE];
  for (int s = 0; s < p.nsub; ++s) {
    int64_t m0 = sub_m0[s];
    int64_t m1_ = s + 1 < p.nsub ? sub_m0[s + 1] : p.lam_start;
    for (int64_t v = m0; v < m1_; ++v) gm[p.m_edge[v]] = v;
    auto add_block = [&](const int64_t *e, int ne, const double (*X)[MAX_CELL_NE], cplx coef) {
      for (int a = 0; a < ne; ++a) {
        int64_t ra = p.pec[e[a]] ? -1 : gm[e[a]];
        if (ra < 0) continue;
        for (int b = 0; b < ne; ++b) {
          if (X[a][b] == 0.0) continue;
          int64_t rb = p.pec[e[b]] ? -1 : gm[e[b]];
          if (rb < 0 || ra < rb) continue;
          trips.push_back({ra, rb, coef * X[a][b]});
        }
      }
    };
    const auto &lo = p.sub_lo[s];
    const auto &hi = p.sub_hi[s];
    int pos[3];
    sub_pos(p, s, pos);
    for (int ck = lo[2]; ck < hi[2]; ++ck)
      for (int cj = lo[1]; cj < hi[1]; ++cj)
        for (int ci = lo[0]; ci < hi[0]; ++ci) {
          int64_t e[MAX_CELL_NE];
          const int ne = cell_edges(p, ci, cj, ck, e);
          cell_matrices(p, ci, cj, ck, Sc, Mc);
          cplx eps = p.eps[ci + (int64_t)p.nx * (cj + (int64_t)p.ny * ck)];
          for (int a = 0; a < ne; ++a) {
            int64_t ra = p.pec[e[a]] ? -1 : gm[e[a]];
            if (ra < 0) continue;
            for (int b = 0; b < ne; ++b) {
              int64_t rb = p.pec[e[b]] ? -1 : gm[e[b]];
              if (rb < 0 || ra < rb) continue;
              cplx v = Sc[a][b] - k * k * eps * Mc[a][b];
              if (v != cplx(0.0)) trips.push_back({ra, rb, v});
            }
          }
          int c3[3] = {ci, cj, ck};
          for (int axis = 0; axis < 3; ++axis)
            for (int side = 0; side < 2; ++side) {
              int layer = side ? hi[axis] - 1 : lo[axis];
              if (c3[axis] != layer) continue;
              int node = side ? hi[axis] : lo[axis];
              cell_face_matrix(p, ci, cj, ck, axis, side, Tf);
              if (node == 0 || node == nn[axis]) {
                add_block(e, ne, Tf, jk);  // first-order ABC
              } else {
                int npos[3] = {pos[0], pos[1], pos[2]};
                npos[axis] += side ? 1 : -1;
                int nb = sub_id(p, npos[0], npos[1], npos[2]);
                add_block(e, ne, Tf, nb > s ? alpha : -alpha);  // interface loss / gain
              }
            }
        }
    for (int64_t v = m0; v < m1_; ++v) gm[p.m_edge[v]] = -1;
  }
  // multiplier couplings.  lm_weight 0: D is the signed Boolean map (+1 on
  // the lower-index copy, -1 on the other).  lm_weight 1: D = D_bool T_lambda,
  // the Galerkin form of the Theory section's multiplier lambda = j +- e
  // expanded in the same tangential edge basis: T_lambda couples the
  // multipliers of one interface block (a, b) by the tangential face mass
  // int_f N_m . N_l dS over the cut face between a and b, so column l of D
  // holds +T(m, l) on a's copy and -T(m, l) on b's copy of every multiplier
  // edge m of the block.  T_lambda is symmetric positive definite per block,
  // so E is unchanged and lambda becomes T_lambda^{-1} lambda_bool.
  {
    // (edge, lm, value) per subdomain; M indices are resolved with a
    // per-subdomain scratch pass (no binary search per entry)
    std::vector<std::vector<std::tuple<int64_t, int64_t, double>>> by_sub(p.nsub);
    if (ctx.opt.lm_weight == 0) {
      for (int64_t l = 0; l < n_lm; ++l) {
        by_sub[p.lm_plus[l]].push_back({p.lm_edge[l], l, 1.0});
        by_sub[p.lm_minus[l]].push_back({p.lm_edge[l], l, -1.0});
      }
    } else {
      // multiplier of edge e in block (a, b): sorted (edge, a, b, l) records
      std::vector<std::array<int64_t, 4>> key(n_lm);
      for (int64_t l = 0; l < n_lm; ++l) key[l] = {p.lm_edge[l], p.lm_plus[l], p.lm_minus[l], l};
      std::sort(key.begin(), key.end());
      auto find_lm = [&](int64_t e, int64_t a, int64_t b) -> int64_t {
        auto it = std::lower_bound(key.begin(), key.end(), std::array<int64_t, 4>{e, a, b, -1});
        return (it != key.end() && (*it)[0] == e && (*it)[1] == a && (*it)[2] == b) ? (*it)[3] : -1;
      };
      for (int a = 0; a < p.nsub; ++a) {
        const auto &lo = p.sub_lo[a];
        const auto &hi = p.sub_hi[a];
        int pos[3];
        sub_pos(p, a, pos);
        for (int axis = 0; axis < 3; ++axis)
          for (int side = 0; side < 2; ++side) {
            int npos[3] = {pos[0], pos[1], pos[2]};
            npos[axis] += side ? 1 : -1;
            if (npos[axis] < 0 || npos[axis] >= p.parts[axis]) continue;
            const int b = sub_id(p, npos[0], npos[1], npos[2]);
            if (b < a) continue;  // each cut face once, from its lower-index side
            const int layer = side ? hi[axis] - 1 : lo[axis];
            int c0[3] = {lo[0], lo[1], lo[2]}, c1[3] = {hi[0], hi[1], hi[2]};
            c0[axis] = layer;
            c1[axis] = layer + 1;
            for (int ck = c0[2]; ck < c1[2]; ++ck)
              for (int cj = c0[1]; cj < c1[1]; ++cj)
                for (int ci = c0[0]; ci < c1[0]; ++ci) {
                  int64_t e[MAX_CELL_NE];
                  const int ne = cell_edges(p, ci, cj, ck, e);
                  cell_face_matrix(p, ci, cj, ck, axis, side, Tf);
                  for (int j = 0; j < ne; ++j) {
                    const int64_t l = find_lm(e[j], a, b);
                    if (l < 0) continue;
                    for (int i = 0; i < ne; ++i) {
                      if (Tf[i][j] == 0.0 || find_lm(e[i], a, b) < 0) continue;
                      by_sub[a].push_back({e[i], l, Tf[i][j]});
                      by_sub[b].push_back({e[i], l, -Tf[i][j]});
                    }
                  }
                }
          }
      }
    }
    for (int s = 0; s < p.nsub; ++s) {
      int64_t m0 = sub_m0[s];
      int64_t m1_ = s + 1 < p.nsub ? sub_m0[s + 1] : p.lam_start;
      for (int64_t v = m0; v < m1_; ++v) gm[p.m_edge[v]] = v;
      for (auto &q : by_sub[s]) trips.push_back({p.lam_start + std::get<1>(q), gm[std::get<0>(q)], cplx(std::get<2>(q), 0.0)});
      for (int64_t v = m0; v < m1_; ++v) gm[p.m_edge[v]] = -1;
    }
  }
  // ---- global operator A on free edges (all cells and the outer boundary),
  // summed and stored as CSR by finish_plan
  std::vector<Trip> g;
  {
    g.reserve((size_t)ncell * p.cell_ne * p.cell_ne);
    double Tb[6][MAX_CELL_NE][MAX_CELL_NE];  // the cell's outer-boundary face matrices
    for (int ck = 0; ck < p.nz; ++ck)
      for (int cj = 0; cj < p.ny; ++cj)
        for (int ci = 0; ci < p.nx; ++ci) {
          int64_t e[MAX_CELL_NE];
          const int ne = cell_edges(p, ci, cj, ck, e);
          cell_matrices(p, ci, cj, ck, Sc, Mc);
          cplx eps = p.eps[ci + (int64_t)p.nx * (cj + (int64_t)p.ny * ck)];
          int c3[3] = {ci, cj, ck};
          bool bnd[6];
          for (int axis = 0; axis < 3; ++axis) {
            bnd[2 * axis] = c3[axis] == 0;
            bnd[2 * axis + 1] = c3[axis] == nn[axis] - 1;
            for (int side = 0; side < 2; ++side)
              if (bnd[2 * axis + side]) cell_face_matrix(p, ci, cj, ck, axis, side, Tb[2 * axis + side]);
          }
          for (int a = 0; a < ne; ++a) {
            if (p.pec[e[a]]) continue;
            for (int b = 0; b < ne; ++b) {
              if (p.pec[e[b]]) continue;
              cplx v = Sc[a][b] - k * k * eps * Mc[a][b];
              for (int f = 0; f < 6; ++f)
                if (bnd[f]) v += jk * Tb[f][a][b];
              if (v != cplx(0.0)) g.push_back({e[a], e[b], v});
            }
          }
        }
  }
  return finish_plan(ctx, trips, g);
}

// Symbolic factorisation, assembly tree, arena layout and the entries of M
// grouped by level (main step 4), from the entries of M (trips, lower
// triangle, M indices) and the triplets of the global operator (g, global
// edge ids); common to every element kind.
static int finish_plan(Ctx &ctx, std::vector<Trip> &trips, std::vector<Trip> &g) {
  Plan &p = ctx.plan;
  const int64_t nsn = (int64_t)p.sn_start.size();
  std::vector<int64_t> sn_of(p.n_m);
  for (int64_t s = 0; s < nsn; ++s)
    for (int64_t v = p.sn_start[s]; v < p.sn_end[s]; ++v) sn_of[v] = s;
  std::sort(trips.begin(), trips.end(), [](const Trip &a, const Trip &b) {
    return a.c != b.c ? a.c < b.c : a.r < b.r;
  });
  {
    size_t w = 0;
    for (size_t i = 0; i < trips.size(); ++i) {
      if (w > 0 && trips[w - 1].r == trips[i].r && trips[w - 1].c == trips[i].c)
        trips[w - 1].v += trips[i].v;
      else
        trips[w++] = trips[i];
    }
    trips.resize(w);
  }
  std::vector<int64_t> col_ptr(p.n_m + 1, 0);
  for (auto &t : trips) col_ptr[t.c + 1]++;
  for (int64_t c = 0; c < p.n_m; ++c) col_ptr[c + 1] += col_ptr[c];

  // ---- supernodal symbolic factorisation (child-merge)
  p.parent.assign(nsn, -1);
  std::vector<std::vector<int64_t>> children(nsn), st(nsn);
  std::vector<int64_t> mark(p.n_m, -1);
  for (int64_t s = 0; s < nsn; ++s) {
    int64_t a = p.sn_start[s], b = p.sn_end[s];
    auto &L = st[s];
    for (int64_t c = a; c < b; ++c)
      for (int64_t q = col_ptr[c]; q < col_ptr[c + 1]; ++q) {
        int64_t r = trips[q].r;
        if (r >= b && mark[r] != s) {
          mark[r] = s;
          L.push_back(r);
        }
      }
    for (int64_t ch : children[s])
      for (int64_t r : st[ch])
        if (r >= b && mark[r] != s) {
          mark[r] = s;
          L.push_back(r);
        }
    std::sort(L.begin(), L.end());
    if (!L.empty()) {
      p.parent[s] = sn_of[L[0]];
      children[p.parent[s]].push_back(s);
    }
  }
  p.struct_ptr.assign(nsn + 1, 0);
  for (int64_t s = 0; s < nsn; ++s) p.struct_ptr[s + 1] = p.struct_ptr[s] + (int64_t)st[s].size();
  p.struct_idx.resize(p.struct_ptr[nsn]);
  for (int64_t s = 0; s < nsn; ++s)
    std::copy(st[s].begin(), st[s].end(), p.struct_idx.begin() + p.struct_ptr[s]);

  // ---- extend-add maps, child ranks, levels
  p.emap.assign(p.struct_idx.size(), -1);
  p.child_rank.assign(nsn, -1);
  p.level.assign(nsn, 0);
  for (int64_t s = 0; s < nsn; ++s) {
    int64_t q = p.parent[s];
    if (q < 0) continue;
    int64_t pq = p.sn_end[q] - p.sn_start[q];
    const int64_t *qs = p.struct_idx.data() + p.struct_ptr[q];
    int64_t nq = p.struct_ptr[q + 1] - p.struct_ptr[q];
    for (int64_t t = p.struct_ptr[s]; t < p.struct_ptr[s + 1]; ++t) {
      int64_t v = p.struct_idx[t];
      int64_t loc;
      if (v < p.sn_end[q]) {
        loc = v - p.sn_start[q];
      } else {
        const int64_t *it = std::lower_bound(qs, qs + nq, v);
        if (it == qs + nq || *it != v) {
          ctx.err = "d3m_setup: internal error (child row missing in parent front)";
          return D3M_EINVAL;
        }
        loc = pq + (it - qs);
      }
      p.emap[t] = (int32_t)loc;
    }
  }
  for (int64_t s = 0; s < nsn; ++s) {
    for (size_t r = 0; r < children[s].size(); ++r) p.child_rank[children[s][r]] = (int32_t)r;
    int lv = 0;
    for (int64_t ch : children[s]) lv = std::max(lv, p.level[ch] + 1);
    p.level[s] = lv;
  }
  p.n_levels = 0;
  for (int64_t s = 0; s < nsn; ++s) p.n_levels = std::max(p.n_levels, p.level[s] + 1);
  p.level_ptr.assign(p.n_levels + 1, 0);
  for (int64_t s = 0; s < nsn; ++s) p.level_ptr[p.level[s] + 1]++;
  for (int l = 0; l < p.n_levels; ++l) p.level_ptr[l + 1] += p.level_ptr[l];
  p.level_fronts.resize(nsn);
  {
    std::vector<int32_t> fill(p.level_ptr.begin(), p.level_ptr.end() - 1);
    for (int64_t s = 0; s < nsn; ++s) p.level_fronts[fill[p.level[s]]++] = (int32_t)s;
  }
  // extend-add passes: pass r of level l adds the r-th child of each front
  p.ea_pass_ptr.assign(p.n_levels + 1, 0);
  p.ea_ptr.assign(1, 0);
  p.ea_child.clear();
  for (int l = 0; l < p.n_levels; ++l) {
    size_t maxc = 0;
    for (int i = p.level_ptr[l]; i < p.level_ptr[l + 1]; ++i)
      maxc = std::max(maxc, children[p.level_fronts[i]].size());
    for (size_t r = 0; r < maxc; ++r) {
      for (int i = p.level_ptr[l]; i < p.level_ptr[l + 1]; ++i) {
        auto &ch = children[p.level_fronts[i]];
        if (r < ch.size()) p.ea_child.push_back((int32_t)ch[r]);
      }
      p.ea_ptr.push_back((int32_t)p.ea_child.size());
    }
    p.ea_pass_ptr[l + 1] = (int32_t)p.ea_ptr.size() - 1;
  }

  // ---- arena layout (level-major, so a level's fronts are contiguous)
  p.front_off.assign(nsn, 0);
  p.piv_off.assign(nsn, 0);
  p.y_off.assign(nsn, 0);
  int64_t off = 0, poff = 0, yoff = 0;
  p.max_front = 0;
  for (int i = 0; i < (int)nsn; ++i) {
    int32_t s = p.level_fronts[i];
    int64_t pp = p.sn_end[s] - p.sn_start[s];
    int64_t m = pp + p.struct_ptr[s + 1] - p.struct_ptr[s];
    p.front_off[s] = off;
    off += m * m;
    p.piv_off[s] = poff;
    poff += pp;
    p.y_off[s] = yoff;
    yoff += m;
    p.max_front = std::max<int>(p.max_front, (int)m);
    // algorithmic flops of the partial LDL^T: sum_{k<p} (m-k-1)(m-k)/2 complex MACs
    double cm = 0;
    for (int64_t kk = 0; kk < pp; ++kk) cm += 0.5 * double(m - kk - 1) * double(m - kk);
    p.flops[p.sn_kind[s]] += 8.0 * cm;
  }
  p.arena_elems = off;
  p.piv_total = poff;
  p.y_rows = yoff;

  // ---- entries grouped by level with arena offsets
  {
    std::vector<int64_t> cnt(p.n_levels + 1, 0);
    for (auto &t : trips) cnt[p.level[sn_of[t.c]] + 1]++;
    for (int l = 0; l < p.n_levels; ++l) cnt[l + 1] += cnt[l];
    p.ent_ptr = cnt;
    p.ent_off.resize(trips.size());
    p.ent_val.resize(trips.size());
    p.ent_row.resize(trips.size());
    p.ent_col.resize(trips.size());
    std::vector<int64_t> fill(cnt.begin(), cnt.end() - 1);
    for (auto &t : trips) {
      int64_t s = sn_of[t.c];
      int64_t a = p.sn_start[s], b = p.sn_end[s];
      int64_t pp = b - a;
      int64_t m = pp + p.struct_ptr[s + 1] - p.struct_ptr[s];
      int64_t lr;
      if (t.r < b) {
        lr = t.r - a;
      } else {
        const int64_t *qs = p.struct_idx.data() + p.struct_ptr[s];
        const int64_t *it = std::lower_bound(qs, qs + (m - pp), t.r);
        lr = pp + (it - qs);
      }
      int64_t lc = t.c - a;
      int64_t slot = fill[p.level[s]]++;
      p.ent_off[slot] = p.front_off[s] + lc * m + lr;
      p.ent_val[slot] = t.v;
      p.ent_row[slot] = t.r;
      p.ent_col[slot] = t.c;
    }
  }

  // ---- global operator A on free edges (full CSR) for fp64 residuals
  std::sort(g.begin(), g.end(), [](const Trip &a, const Trip &b) {
    return a.r != b.r ? a.r < b.r : a.c < b.c;
  });
  p.csr_ptr.assign(p.n_edges + 1, 0);
  p.csr_col.clear();
  p.csr_val.clear();
  for (size_t i = 0; i < g.size();) {
    size_t j = i;
    cplx v = 0;
    while (j < g.size() && g[j].r == g[i].r && g[j].c == g[i].c) v += g[j++].v;
    p.csr_col.push_back((int32_t)g[i].c);
    p.csr_val.push_back(v);
    p.csr_ptr[g[i].r + 1]++;
    i = j;
  }
  for (int64_t r = 0; r < p.n_edges; ++r) p.csr_ptr[r + 1] += p.csr_ptr[r];
  return D3M_OK;
}

// ------------------------------------------------------------ plane-wave RHS
// U = n x curl E_inc - jk (E_inc)_t at point xyz for the plane wave kp (3
// direction components, complex polarisation as re/im pairs), outward normal n.
static void incident_u(const Plan &p, const double *kp, const double xyz[3], const double nvec[3], cplx U[3]) {
  const cplx J(0.0, 1.0);
  cplx pol[3] = {cplx(kp[3], kp[4]), cplx(kp[5], kp[6]), cplx(kp[7], kp[8])};
  double kr = kp[0] * xyz[0] + kp[1] * xyz[1] + kp[2] * xyz[2];
  cplx ph = std::exp(-J * p.k * kr);
  cplx E[3] = {pol[0] * ph, pol[1] * ph, pol[2] * ph};
  // curl E = -jk khat x E
  cplx cE[3] = {-J * p.k * (kp[1] * E[2] - kp[2] * E[1]), -J * p.k * (kp[2] * E[0] - kp[0] * E[2]),
                -J * p.k * (kp[0] * E[1] - kp[1] * E[0])};
  cplx ndotE = nvec[0] * E[0] + nvec[1] * E[1] + nvec[2] * E[2];
  cplx nxc[3] = {nvec[1] * cE[2] - nvec[2] * cE[1], nvec[2] * cE[0] - nvec[0] * cE[2],
                 nvec[0] * cE[1] - nvec[1] * cE[0]};
  for (int a = 0; a < 3; ++a) U[a] = nxc[a] - J * p.k * (E[a] - nvec[a] * ndotE);
}

// Radon's 7-point degree-5 triangle rule: barycentric points (1/3,1/3,1/3)
// and the permutations of (a, a, 1 - 2a), a = (6 -+ sqrt 15)/21; weights 9/40
// and (155 -+ sqrt 15)/1200 of the area.
struct TriRule {
  double b[7][3], w[7];
};
static TriRule radon7() {
  TriRule R;
  const double r15 = std::sqrt(15.0);
  R.b[0][0] = R.b[0][1] = R.b[0][2] = 1.0 / 3.0;
  R.w[0] = 9.0 / 40.0;
  for (int g = 0; g < 2; ++g) {
    const double a = g ? (6.0 + r15) / 21.0 : (6.0 - r15) / 21.0;
    const double wt = g ? (155.0 + r15) / 1200.0 : (155.0 - r15) / 1200.0;
    for (int r = 0; r < 3; ++r) {
      double *b = R.b[1 + 3 * g + r];
      b[0] = b[1] = b[2] = a;
      b[2 - r] = 1.0 - 2.0 * a;
      R.w[1 + 3 * g + r] = wt;
    }
  }
  return R;
}

// f_v -= int U . N_v dS over triangle Q with outward normal nvec; eids: the
// dofs of the Whitney functions of the vertex pairs 01 02 12 (each pointing
// from the lower to the higher local vertex), then, when nfun >= 6, of their
// edge-gradient functions, and when nfun = 8 of the face functions
// l_01 mu_2 W_01 and l_02 mu_1 W_02 (vertices in the order of their ids).
static void rhs_triangle(const Plan &p, const TriRule &R, const double Q[3][3], const double nvec[3],
                         const int64_t *eids, int nfun, const double *khat_pol, int nrhs, double *rhs,
                         int64_t ldb) {
  double g[3][3], ell[3];
  const double area = tri_grads(Q, g);
  for (int m = 0; m < 3; ++m) {
    double ev[3];
    sub3(Q[TRI_E[m][1]], Q[TRI_E[m][0]], ev);
    ell[m] = std::sqrt(dot3(ev, ev));
  }
  for (int q = 0; q < 7; ++q) {
    const double *mu = R.b[q];
    double xyz[3], N[8][3];
    for (int a = 0; a < 3; ++a) xyz[a] = mu[0] * Q[0][a] + mu[1] * Q[1][a] + mu[2] * Q[2][a];
    for (int m = 0; m < nfun && m < 6; ++m) {
      const int mm = m % 3, a = TRI_E[mm][0], b = TRI_E[mm][1];
      const double sb = m < 3 ? -1.0 : 1.0;
      for (int c = 0; c < 3; ++c) N[m][c] = ell[mm] * (mu[a] * g[b][c] + sb * mu[b] * g[a][c]);
    }
    if (nfun == 8)
      for (int c = 0; c < 3; ++c) {
        N[6][c] = ell[0] * mu[2] * (mu[0] * g[1][c] - mu[1] * g[0][c]);
        N[7][c] = ell[1] * mu[1] * (mu[0] * g[2][c] - mu[2] * g[0][c]);
      }
    const double w = R.w[q] * area;
    for (int r = 0; r < nrhs; ++r) {
      cplx U[3];
      incident_u(p, khat_pol + 9 * r, xyz, nvec, U);
      for (int m = 0; m < nfun; ++m) {
        const cplx dot = U[0] * N[m][0] + U[1] * N[m][1] + U[2] * N[m][2];
        const int64_t idx = eids[m] + ldb * r;
        rhs[2 * idx] -= w * dot.real();
        rhs[2 * idx + 1] -= w * dot.imag();
      }
    }
  }
}

// Lattice tetrahedra: the two triangles of every outer-boundary cell face.
static int rhs_planewave_tet(const Plan &p, const double *khat_pol, int nrhs, double *rhs, int64_t ldb) {
  const TriRule R = radon7();
  const int nn[3] = {p.nx, p.ny, p.nz};
  for (int axis = 0; axis < 3; ++axis)
    for (int side = 0; side < 2; ++side) {
      double nvec[3] = {0, 0, 0};
      nvec[axis] = side ? 1.0 : -1.0;
      int o[2][3][3];
      face_tris(axis, side, o);
      const int layer = side ? nn[axis] - 1 : 0;
      for (int ck = 0; ck < p.nz; ++ck)
        for (int cj = 0; cj < p.ny; ++cj)
          for (int ci = 0; ci < p.nx; ++ci) {
            const int c3[3] = {ci, cj, ck};
            if (c3[axis] != layer) continue;
            int64_t e[MAX_CELL_NE];
            cell_edges(p, ci, cj, ck, e);
            for (int t = 0; t < 2; ++t) {
              FaceTri f;
              cell_face_tri(p, ci, cj, ck, o[t], f);
              const int64_t eids[3] = {e[f.loc[0]], e[f.loc[1]], e[f.loc[2]]};
              rhs_triangle(p, R, f.Q, nvec, eids, 3, khat_pol, nrhs, rhs, ldb);
            }
          }
    }
  return D3M_OK;
}

// General meshes: every boundary triangle with the outward normal of its
// tetrahedron.
static int rhs_planewave_mesh(const Plan &p, const double *khat_pol, int nrhs, double *rhs, int64_t ldb) {
  const TriRule R = radon7();
  for (const auto &bf : p.bface) {
    double Q[3][3], X[3], e1[3], e2[3], nvec[3];
    for (int w = 0; w < 3; ++w) mesh_vertex(p, bf[w], Q[w]);
    mesh_vertex(p, bf[3], X);
    sub3(Q[1], Q[0], e1);
    sub3(Q[2], Q[0], e2);
    cross3(e1, e2, nvec);
    const double len = std::sqrt(dot3(nvec, nvec));
    for (int a = 0; a < 3; ++a) nvec[a] /= len;
    double to_opp[3];
    sub3(X, Q[0], to_opp);
    if (dot3(nvec, to_opp) > 0)
      for (int a = 0; a < 3; ++a) nvec[a] *= -1.0;
    int64_t eids[8];
    for (int m = 0; m < 3; ++m) {
      const int64_t ge = mesh_edge_id(p, bf[TRI_E[m][0]], bf[TRI_E[m][1]]);
      eids[m] = p.dpe * ge;
      eids[3 + m] = 2 * ge + 1;
    }
    int nfun = 3 * p.dpe;
    if (p.order == 3) {
      const std::array<int64_t, 3> key = {bf[0], bf[1], bf[2]};
      const int64_t f = std::lower_bound(p.mface.begin(), p.mface.end(), key) - p.mface.begin();
      eids[6] = 2 * p.n_geo + 2 * f;
      eids[7] = eids[6] + 1;
      nfun = 8;
    }
    rhs_triangle(p, R, Q, nvec, eids, nfun, khat_pol, nrhs, rhs, ldb);
  }
  return D3M_OK;
}

int rhs_planewave(const Plan &p, const double *khat_pol, int nrhs, double *rhs, int64_t ldb) {
  for (int r = 0; r < nrhs; ++r)
    for (int64_t e = 0; e < p.n_edges; ++e) {
      rhs[2 * (e + ldb * r)] = 0.0;
      rhs[2 * (e + ldb * r) + 1] = 0.0;
    }
  if (p.element == D3M_TET) return rhs_planewave_tet(p, khat_pol, nrhs, rhs, ldb);
  if (p.element == D3M_TET_MESH) return rhs_planewave_mesh(p, khat_pol, nrhs, rhs, ldb);
  const double gq[3] = {0.5 - 0.5 * std::sqrt(0.6), 0.5, 0.5 + 0.5 * std::sqrt(0.6)};
  const double gw[3] = {5.0 / 18.0, 8.0 / 18.0, 5.0 / 18.0};
  const int nn[3] = {p.nx, p.ny, p.nz};
  const cplx J(0.0, 1.0);
  for (int axis = 0; axis < 3; ++axis) {
    int u = axis == 0 ? 1 : 0, v = axis == 2 ? 1 : 2;
    double area = p.h[u] * p.h[v];
    for (int side = 0; side < 2; ++side) {
      double nvec[3] = {0, 0, 0};
      nvec[axis] = side ? 1.0 : -1.0;
      int layer = side ? nn[axis] - 1 : 0;
      int lim[3] = {p.nx, p.ny, p.nz};
      for (int ck = 0; ck < lim[2]; ++ck)
        for (int cj = 0; cj < lim[1]; ++cj)
          for (int ci = 0; ci < lim[0]; ++ci) {
            int c3[3] = {ci, cj, ck};
            if (c3[axis] != layer) continue;
            int64_t e[MAX_CELL_NE];
            cell_edges(p, ci, cj, ck, e);
            for (int qa = 0; qa < 3; ++qa)
              for (int qb = 0; qb < 3; ++qb) {
                double ref[3];
                ref[axis] = side;
                ref[u] = gq[qa];
                ref[v] = gq[qb];
                double xyz[3] = {(ci + ref[0]) * p.h[0], (cj + ref[1]) * p.h[1],
                                 (ck + ref[2]) * p.h[2]};
                // basis values at the point (12 x 3)
                double N[12][3] = {};
                for (int q = 0; q < 4; ++q) {
                  int a = OFF[q][0], b = OFF[q][1];
                  auto ph = [](double t, int s) { return s ? t : 1.0 - t; };
                  N[q][0] = ph(ref[1], a) * ph(ref[2], b);
                  N[4 + q][1] = ph(ref[0], a) * ph(ref[2], b);
                  N[8 + q][2] = ph(ref[0], a) * ph(ref[1], b);
                }
                double w = gw[qa] * gw[qb] * area;
                for (int r = 0; r < nrhs; ++r) {
                  const double *kp = khat_pol + 9 * r;
                  cplx pol[3] = {cplx(kp[3], kp[4]), cplx(kp[5], kp[6]), cplx(kp[7], kp[8])};
                  double kr = kp[0] * xyz[0] + kp[1] * xyz[1] + kp[2] * xyz[2];
                  cplx ph = std::exp(-J * p.k * kr);
                  cplx E[3] = {pol[0] * ph, pol[1] * ph, pol[2] * ph};
                  // curl E = -jk khat x E
                  cplx cE[3] = {-J * p.k * (kp[1] * E[2] - kp[2] * E[1]),
                                -J * p.k * (kp[2] * E[0] - kp[0] * E[2]),
                                -J * p.k * (kp[0] * E[1] - kp[1] * E[0])};
                  cplx ndotE = nvec[0] * E[0] + nvec[1] * E[1] + nvec[2] * E[2];
                  cplx U[3];
                  cplx nxc[3] = {nvec[1] * cE[2] - nvec[2] * cE[1], nvec[2] * cE[0] - nvec[0] * cE[2],
                                 nvec[0] * cE[1] - nvec[1] * cE[0]};
                  for (int a = 0; a < 3; ++a) U[a] = nxc[a] - J * p.k * (E[a] - nvec[a] * ndotE);
                  for (int a = 0; a < 12; ++a) {
                    cplx dot = U[0] * N[a][0] + U[1] * N[a][1] + U[2] * N[a][2];
                    if (dot == cplx(0.0)) continue;
                    int64_t idx = e[a] + ldb * r;
                    rhs[2 * idx] -= w * dot.real();
                    rhs[2 * idx + 1] -= w * dot.imag();
                  }
                }
              }
          }
    }
  }
  return D3M_OK;
}

}  // namespace d3m

// ============================================================ C ABI (host part)
using d3m::Ctx;

extern "C" int d3m_setup(const d3m_mesh *mesh, const d3m_materials *mat, double k,
                         const d3m_partition *part, const d3m_options *opt, d3m_ctx **out) {
  if (!out) return D3M_EINVAL;
  *out = nullptr;
  if (!mesh || !mat || !part) return D3M_EINVAL;
  d3m_ctx *h = nullptr;
  try {
    h = new d3m_ctx();
  } catch (...) {
    return D3M_ENOMEM;
  }
  Ctx &c = h->c;
  if (opt) c.opt = *opt;
  if (opt && opt->autotune_cache) c.cache_path = opt->autotune_cache;
  if (const char *f = std::getenv("D3M_FAULT")) c.fault = f;
  c.opt.autotune_cache = nullptr;  // the context keeps its own copy
  if (c.opt.refine_tol <= 0) c.opt.refine_tol = 1e-10;
  if (c.opt.max_refine <= 0) c.opt.max_refine = 10;
  if (c.opt.gmres_restart == 0) c.opt.gmres_restart = 20;
  if (c.opt.gmres_tol == 0) c.opt.gmres_tol = 1e-4;
  if (c.opt.precision != D3M_FP64 && c.opt.precision != D3M_MIXED) {
    c.err = "d3m_setup: unknown precision";
    *out = h;
    return D3M_EINVAL;
  }
  const char *bad = nullptr;
  if (c.opt.leaf_max < 0) bad = "leaf_max < 0";
  else if (c.opt.panel_kernel != 0 && c.opt.panel_kernel != 1) bad = "panel_kernel not 0 or 1";
  else if (c.opt.update_kernel < 0 || c.opt.update_kernel > 2) bad = "update_kernel not 0, 1 or 2";
  else if (c.opt.autotune != 0 && c.opt.autotune != 1) bad = "autotune not 0 or 1";
  else if (c.opt.lookahead != 0 && c.opt.lookahead != 1) bad = "lookahead not 0 or 1";
  else if (c.opt.refine_method != 0 && c.opt.refine_method != 1) bad = "refine_method not 0 or 1";
  else if (c.opt.gmres_restart < 1 || c.opt.gmres_restart > 200) bad = "gmres_restart not in 1..200";
  else if (!(c.opt.gmres_tol > 0 && c.opt.gmres_tol < 1)) bad = "gmres_tol not in (0, 1)";
  else if (c.opt.solve_kernel != 0 && c.opt.solve_kernel != 1) bad = "solve_kernel not 0 or 1";
  else if (c.opt.lm_weight != 0 && c.opt.lm_weight != 1) bad = "lm_weight not 0 or 1";
  else if (!c.fault.empty() && c.fault != "alloc" && c.fault != "pivot" && c.fault != "nan" && c.fault != "timeout" &&
           c.fault != "solve_timeout")
    bad = "D3M_FAULT not one of alloc, pivot, nan, timeout, solve_timeout";
  if (bad) {
    c.err = std::string("d3m_setup: ") + bad;
    *out = h;
    return D3M_EINVAL;
  }
  int rc;
  d3m::NvtxRange range("d3m_setup");
  try {
    rc = d3m::build_plan(c, mesh, mat, k, part);
  } catch (const std::bad_alloc &) {
    c.err = "d3m_setup: host allocation failed";
    rc = D3M_ENOMEM;
  }
  const d3m::Plan &p = c.plan;
  if (rc == D3M_OK) {
    d3m_stats &st = c.stats;
    st.n_edges = p.n_edges;
    st.n_free = p.n_free;
    st.n_lm = (int64_t)p.lm_edge.size();
    st.n_blocks = (int64_t)p.blocks.size();
    st.n_subdomains = p.nsub;
    st.n_m = p.n_m;
    st.n_fronts = (int64_t)p.sn_start.size();
    st.n_levels = p.n_levels;
    st.max_front = p.max_front;
    st.arena_bytes = p.arena_elems * (c.opt.precision == D3M_FP64 ? 16 : 8);
    st.flops_interior = p.flops[0];
    st.flops_domain = p.flops[1];
    st.flops_k = p.flops[2];
    st.min_pivot_ratio = 0;
  }
  *out = h;
  return rc;
}

extern "C" int d3m_rhs_planewave(d3m_ctx *h, const double *khat_pol, int32_t nrhs, double *rhs,
                                 int64_t ldb) {
  if (!h || !khat_pol || !rhs || nrhs < 0 || ldb < h->c.plan.n_edges) return D3M_EINVAL;
  return d3m::rhs_planewave(h->c.plan, khat_pol, nrhs, rhs, ldb);
}

template <class T>
static int put(void *buf, size_t *bytes, const std::vector<T> &v) {
  size_t need = v.size() * sizeof(T);
  if (!buf) {
    *bytes = need;
    return D3M_OK;
  }
  if (*bytes < need) return D3M_EINVAL;
  std::memcpy(buf, v.data(), need);
  *bytes = need;
  return D3M_OK;
}

extern "C" int d3m_structure(d3m_ctx *h, int32_t which, void *buf, size_t *bytes) {
  if (!h || !bytes) return D3M_EINVAL;
  const d3m::Plan &p = h->c.plan;
  const size_t nsn = p.sn_start.size();
  std::vector<int64_t> v;
  switch (which) {
    case D3M_SN_RANGE:
      for (size_t s = 0; s < nsn; ++s) {
        v.push_back(p.sn_start[s]);
        v.push_back(p.sn_end[s]);
      }
      return put(buf, bytes, v);
    case D3M_SN_PARENT:
      return put(buf, bytes, p.parent);
    case D3M_SN_KIND:
      for (size_t s = 0; s < nsn; ++s) {
        v.push_back(p.sn_kind[s]);
        v.push_back(p.sn_owner[s]);
      }
      return put(buf, bytes, v);
    case D3M_SN_STRUCT:
      v = p.struct_ptr;
      v.insert(v.end(), p.struct_idx.begin(), p.struct_idx.end());
      return put(buf, bytes, v);
    case D3M_M_MAP:
      for (int64_t i = 0; i < p.n_m; ++i) {
        v.push_back(p.m_sub[i]);
        v.push_back(p.m_edge[i]);
      }
      return put(buf, bytes, v);
    case D3M_LM:
      for (size_t l = 0; l < p.lm_edge.size(); ++l) {
        v.push_back(p.lm_edge[l]);
        v.push_back(p.lm_plus[l]);
        v.push_back(p.lm_minus[l]);
      }
      return put(buf, bytes, v);
    case D3M_BLOCKS:
      for (auto &b : p.blocks) {
        v.push_back(b[0]);
        v.push_back(b[1]);
        v.push_back(b[2]);
      }
      return put(buf, bytes, v);
    case D3M_LAMBDA: {
      std::vector<double> d(2 * h->c.lambda_host.size());
      for (size_t i = 0; i < h->c.lambda_host.size(); ++i) {
        d[2 * i] = h->c.lambda_host[i].real();
        d[2 * i + 1] = h->c.lambda_host[i].imag();
      }
      return put(buf, bytes, d);
    }
    case D3M_M_ENTRIES: {
      std::vector<double> d(4 * p.ent_val.size());
      for (size_t i = 0; i < p.ent_val.size(); ++i) {
        d[4 * i] = (double)p.ent_row[i];
        d[4 * i + 1] = (double)p.ent_col[i];
        d[4 * i + 2] = p.ent_val[i].real();
        d[4 * i + 3] = p.ent_val[i].imag();
      }
      return put(buf, bytes, d);
    }
    case D3M_LEVELS: {
      const d3m::Ctx &c = h->c;
      std::vector<double> d((size_t)p.n_levels * 10, 0.0);
      for (int l = 0; l < p.n_levels; ++l) {
        double *o = d.data() + (size_t)l * 10;
        for (int i = p.level_ptr[l]; i < p.level_ptr[l + 1]; ++i) {
          int32_t f = p.level_fronts[i];
          int64_t pp = p.sn_end[f] - p.sn_start[f];
          int64_t m = pp + p.struct_ptr[f + 1] - p.struct_ptr[f];
          o[0] += 1;
          o[1] = std::max(o[1], (double)pp);
          o[2] = std::max(o[2], (double)m);
          for (int64_t kk = 0; kk < pp; ++kk) o[3] += 4.0 * double(m - kk - 1) * double(m - kk);
        }
        if ((size_t)l < c.lvl_ms_panel.size()) o[4] = c.lvl_ms_panel[l];
        if ((size_t)l < c.lvl_ms_update.size()) o[5] = c.lvl_ms_update[l];
        if ((size_t)l < c.lvl_tc.size()) o[6] = c.lvl_tc[l];
        if ((size_t)l < c.lvl_cs.size()) o[7] = c.lvl_cs[l];
        if ((size_t)l < c.lvl_ms_inv.size()) o[8] = c.lvl_ms_inv[l];
        if ((size_t)l < c.lvl_ms_tc.size()) o[9] = c.lvl_ms_tc[l];
      }
      return put(buf, bytes, d);
    }
    case D3M_STATS: {
      std::vector<d3m_stats> s(1, h->c.stats);
      return put(buf, bytes, s);
    }
    default:
      return D3M_EINVAL;
  }
}

extern "C" int d3m_stats_get(d3m_ctx *h, d3m_stats *out) {
  if (!h || !out) return D3M_EINVAL;
  *out = h->c.stats;
  return D3M_OK;
}

extern "C" const char *d3m_last_error(const d3m_ctx *h) {
  if (!h) return "null context";
  return h->c.err.c_str();
}

extern "C" void d3m_free(d3m_ctx *h) {
  if (!h) return;
  d3m::dev_free(h->c);
  delete h;
}
