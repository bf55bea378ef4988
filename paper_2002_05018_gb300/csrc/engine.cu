// Device engine of the D^3M library: numeric factorisation (main steps 1, 2
// and 5) and substitution (main steps 6-7) on one GB300.
//
// The decomposed system of Eq. (1), M = [[A, D], [D^T, 0]], is factored as one
// sparse complex-symmetric LDL^T in the multifrontal form that the paper
// allows for Algorithm 1.  The ordering puts, per subdomain, its interior
// (nested dissection) then its interface dofs B_i, and finally the interface
// blocks of K; fronts are processed level by level (all subdomains at once):
//   - interior fronts: partial LDL^T, Schur complement passed up;
//   - interface fronts [B_i ; lambda_i]: eliminating B_i leaves the
//     contribution -D_i^T A_i^{-1} D_i = -K_D^(i) on the multipliers (main
//     step 1), which extend-add scatters into the fronts of K (main step 2);
//   - fronts of K: block LDL^T with Bunch-Kaufman pivots restricted to the
//     block (main step 5, Algorithm 1).
// Every front is dense, column-major, lower triangle, in one arena.  A front
// is factored by panels of NB columns (restricted Bunch-Kaufman with
// left-looking updates inside the panel, one CTA per front) followed by a
// trailing update of all fronts of the level (64x64 tiles).
#include <cooperative_groups.h>
#include <cuda.h>  // CUtensorMap (the encoder is fetched through the runtime, no driver link)
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "d3m_internal.h"

namespace d3m {

// ------------------------------------------------------------ complex helpers
template <typename T>
struct cx {
  T re, im;
};
template <typename T>
__host__ __device__ __forceinline__ cx<T> mk(T r, T i) {
  cx<T> z;
  z.re = r;
  z.im = i;
  return z;
}
template <typename T>
__device__ __forceinline__ cx<T> cmul(cx<T> a, cx<T> b) {
  return mk<T>(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
// a - b*c
template <typename T>
__device__ __forceinline__ cx<T> cfms(cx<T> a, cx<T> b, cx<T> c) {
  a.re -= b.re * c.re;
  a.re += b.im * c.im;
  a.im -= b.re * c.im;
  a.im -= b.im * c.re;
  return a;
}
// a + b*c
template <typename T>
__device__ __forceinline__ cx<T> cfma(cx<T> a, cx<T> b, cx<T> c) {
  a.re += b.re * c.re;
  a.re -= b.im * c.im;
  a.im += b.re * c.im;
  a.im += b.im * c.re;
  return a;
}
template <typename T>
__device__ __forceinline__ double cabs1(cx<T> a) {
  return fabs((double)a.re) + fabs((double)a.im);
}
__device__ __forceinline__ double2 zdiv1(double2 a) {  // 1 / a
  double d = a.x * a.x + a.y * a.y;
  return make_double2(a.x / d, -a.y / d);
}
__device__ __forceinline__ double2 zmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename T>
__device__ __forceinline__ double2 to_d(cx<T> a) {
  return make_double2((double)a.re, (double)a.im);
}
template <typename T>
__device__ __forceinline__ cx<T> from_d(double2 a) {
  return mk<T>((T)a.x, (T)a.y);
}

#define CUDA_TRY(call)                                                              \
  do {                                                                              \
    cudaError_t e_ = (call);                                                        \
    if (e_ != cudaSuccess) {                                                        \
      c.err = std::string("CUDA error ") + cudaGetErrorString(e_) + " at " #call; \
      return D3M_ECUDA;                                                             \
    }                                                                               \
  } while (0)

constexpr int NB = 32;         // panel width (columns per panel kernel)
constexpr int LSTR = NB + 2;   // shared-memory row stride of the cluster panel (16-byte rows, bank spread)
constexpr int UT = 64;         // trailing-update tile edge
constexpr int UK = 16;         // trailing-update k chunk
constexpr int PANEL_THREADS = 512;
constexpr double BK_ALPHA = 0.6403882032022076;  // (1 + sqrt(17)) / 8

// ------------------------------------------------------------ front tables
struct FrontTab {
  const int32_t *m, *p;
  const int64_t *off, *piv, *soff, *start, *yoff;
  const int32_t *parent;
};

// ------------------------------------------------------------ assembly kernels
template <typename T>
__global__ void k_assemble(int64_t n, const int64_t *__restrict__ off, const double2 *__restrict__ val,
                           cx<T> *__restrict__ arena) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) arena[off[i]] = from_d<T>(val[i]);
}

// pass: children list; adds child contribution blocks (lower) into parents
template <typename T>
__global__ void __launch_bounds__(256) k_extend_add(const int32_t *__restrict__ kids, FrontTab ft,
                                                    const int32_t *__restrict__ emap,
                                                    cx<T> *__restrict__ arena) {
  const int c = kids[blockIdx.y];
  const int mc = ft.m[c], pc = ft.p[c], n = mc - pc;
  const int nt = (n + 31) / 32;
  const int t = blockIdx.x;
  if (t >= nt * (nt + 1) / 2) return;
  int I = (int)((sqrt(8.0 * t + 1.0) - 1.0) * 0.5);
  while (I * (I + 1) / 2 > t) --I;
  while ((I + 1) * (I + 2) / 2 <= t) ++I;
  const int J = t - I * (I + 1) / 2;
  const int q = ft.parent[c];
  const int mq = ft.m[q];
  const cx<T> *C = arena + ft.off[c];
  cx<T> *F = arena + ft.off[q];
  const int32_t *map = emap + ft.soff[c];
  const int i = I * 32 + (threadIdx.x & 31);
  if (i >= n) return;
  const int64_t ri = map[i];
  // all loads (child entries, map, parent entries) before the first store
  cx<T> v[4], o[4];
  int64_t cj[4];
  bool ok[4];
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int j = J * 32 + (threadIdx.x >> 5) + 8 * u;
    ok[u] = j <= i && j < n;
    v[u] = ok[u] ? C[(int64_t)(pc + i) + (int64_t)(pc + j) * mc] : mk<T>(0, 0);
    cj[u] = ok[u] ? (int64_t)map[j] : 0;
  }
#pragma unroll
  for (int u = 0; u < 4; ++u) o[u] = ok[u] ? F[ri + cj[u] * mq] : mk<T>(0, 0);
#pragma unroll
  for (int u = 0; u < 4; ++u)
    if (ok[u]) F[ri + cj[u] * mq] = mk<T>(o[u].re + v[u].re, o[u].im + v[u].im);
}

// ------------------------------------------------------------ reciprocal
// 1/s for s > 0 in fp64 by Newton-Raphson from an fp32 seed: r <- r (2 - s r)
// doubles the correct bits per step (24 -> 48 -> 96), so two steps reach
// fp64 accuracy with a handful of fp64 FMAs instead of a full fp64 divide.
// Outside the fp32 range the plain fp64 division is used.
__device__ __forceinline__ double recip_nr(double s) {
  if (!(s > 1e-30 && s < 1e30)) return 1.0 / s;
  double r = (double)(1.0f / (float)s);
  r = r * fma(-s, r, 2.0);
  r = r * fma(-s, r, 2.0);
  return r;
}
__device__ __forceinline__ double2 zinv_nr(double2 a) {  // 1 / a, a != 0
  double rs = recip_nr(fma(a.x, a.x, a.y * a.y));
  return make_double2(a.x * rs, -a.y * rs);
}

// ------------------------------------------------------------ block reductions
// Arg-max in the factor precision T (magnitudes |Re|+|Im| of T values),
// lowest index on ties.
template <typename T>
struct ArgMaxT {
  T v;
  int i;
};
template <typename T>
__device__ __forceinline__ ArgMaxT<T> amaxT(ArgMaxT<T> a, ArgMaxT<T> b) {
  if (b.v > a.v || (b.v == a.v && b.i < a.i)) return b;
  return a;
}
template <typename T>
__device__ __forceinline__ T cabs1T(cx<T> a) {
  return fabs(a.re) + fabs(a.im);
}
struct ArgMax {
  double v;
  int i;
};
__device__ __forceinline__ ArgMax amax(ArgMax a, ArgMax b) {
  if (b.v > a.v || (b.v == a.v && b.i < a.i)) return b;
  return a;
}
__device__ ArgMax block_argmax(ArgMax x, ArgMax *sh) {
  for (int o = 16; o > 0; o >>= 1) {
    ArgMax y;
    y.v = __shfl_down_sync(0xffffffffu, x.v, o);
    y.i = __shfl_down_sync(0xffffffffu, x.i, o);
    x = amax(x, y);
  }
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[w] = x;
  __syncthreads();
  if (w == 0) {
    x = l < (int)(blockDim.x >> 5) ? sh[l] : ArgMax{-1.0, 0x7fffffff};
    for (int o = 16; o > 0; o >>= 1) {
      ArgMax y;
      y.v = __shfl_down_sync(0xffffffffu, x.v, o);
      y.i = __shfl_down_sync(0xffffffffu, x.i, o);
      x = amax(x, y);
    }
    if (l == 0) sh[0] = x;
  }
  __syncthreads();
  ArgMax r = sh[0];
  __syncthreads();
  return r;
}

// ------------------------------------------------------------ panel kernel
// Restricted Bunch-Kaufman factorisation of up to NB columns of each front
// of the level (one CTA per front).  Left-looking inside the panel: the
// updated column k is W[:, j] = F[:, k] - L[:, k0:k] W[k, 0:j]^T with
// W = L D.  Pivot candidates are rows k+1 .. p-1 only (the pivot block); no
// pivot is delayed.  Interchanges are applied to all previously factored
// columns of the front so L ends in pivot order.
template <typename T>
__global__ void __launch_bounds__(PANEL_THREADS)
    k_panel(const int32_t *__restrict__ lvl, FrontTab ft, const int64_t *__restrict__ wofs,
            cx<T> *__restrict__ arena, cx<T> *__restrict__ Wbuf, int32_t *__restrict__ perm,
            double2 *__restrict__ dinv_d, double2 *__restrict__ dinv_o, int8_t *__restrict__ psize,
            int32_t *__restrict__ st_k0, int32_t *__restrict__ st_kb, int32_t *__restrict__ st_info,
            double *__restrict__ st_minpiv, double *__restrict__ flop_cnt, int2 *__restrict__ snap) {
  const int f = lvl[blockIdx.x];
  const int m = ft.m[f], p = ft.p[f];
  const int k0 = st_k0[f];
  const int tid = threadIdx.x, nth = blockDim.x;
  if (k0 >= p) {
    if (tid == 0) {
      st_kb[f] = 0;
      snap[blockIdx.x] = make_int2(k0, 0);
    }
    return;
  }
  cx<T> *F = arena + ft.off[f];
  cx<T> *W = Wbuf + wofs[blockIdx.x];
  int32_t *pv = perm + ft.piv[f];
  double2 *dd = dinv_d + ft.piv[f];
  double2 *dof = dinv_o + ft.piv[f];
  int8_t *ps = psize + ft.piv[f];
  const int64_t ld = m;
  __shared__ cx<T> wrow[NB];
  __shared__ ArgMax red[32];
  __shared__ int s_kp, s_kstep, s_imax;
  __shared__ double s_minpiv, s_cmac;
  __shared__ double2 s_dinv;
  if (tid == 0) {
    s_minpiv = 1e300;
    s_cmac = 0.0;
  }
  int k = k0, j = 0;
  while (k < p && j < NB - 1) {
    // (1) updated column k -> W[:, j]
    if (tid < NB) wrow[tid] = tid < j ? W[k + (int64_t)tid * ld] : mk<T>(0, 0);
    __syncthreads();
    for (int i = k + tid; i < m; i += nth) {
      cx<T> acc = F[i + (int64_t)k * ld];
      const cx<T> *Li = F + i + (int64_t)k0 * ld;
      for (int t0 = 0; t0 < j; t0 += 8) {  // 8 independent loads in flight
        cx<T> l[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) l[u] = t0 + u < j ? Li[(int64_t)(t0 + u) * ld] : mk<T>(0, 0);
#pragma unroll
        for (int u = 0; u < 8; ++u) acc = cfms(acc, l[u], wrow[min(t0 + u, NB - 1)]);
      }
      W[i + (int64_t)j * ld] = acc;
    }
    __syncthreads();
    // (2) pivot test on the restricted column
    ArgMax loc{-1.0, 0x7fffffff};
    for (int i = k + 1 + tid; i < p; i += nth) loc = amax(loc, ArgMax{cabs1(W[i + (int64_t)j * ld]), i});
    ArgMax cm = block_argmax(loc, red);
    const double absakk = cabs1(W[k + (int64_t)j * ld]);
    const double colmax = cm.i < p ? cm.v : 0.0;
    const int imax = cm.i;
    if (tid == 0) {
      s_kstep = 1;
      s_kp = k;
      s_imax = imax;
      s_cmac += (double)(m - k) * (j + 1);
    }
    if (fmax(absakk, colmax) == 0.0) {
      if (tid == 0 && st_info[f] == 0) st_info[f] = k + 1;
    } else if (absakk < BK_ALPHA * colmax) {
      // (3) updated column imax -> W[:, j+1]
      if (tid < NB) wrow[tid] = tid < j ? W[imax + (int64_t)tid * ld] : mk<T>(0, 0);
      __syncthreads();
      for (int i = k + tid; i < m; i += nth) {
        cx<T> acc = i < imax ? F[imax + (int64_t)i * ld] : F[i + (int64_t)imax * ld];
        const cx<T> *Li = F + i + (int64_t)k0 * ld;
        for (int t0 = 0; t0 < j; t0 += 8) {
          cx<T> l[8];
#pragma unroll
          for (int u = 0; u < 8; ++u) l[u] = t0 + u < j ? Li[(int64_t)(t0 + u) * ld] : mk<T>(0, 0);
#pragma unroll
          for (int u = 0; u < 8; ++u) acc = cfms(acc, l[u], wrow[min(t0 + u, NB - 1)]);
        }
        W[i + (int64_t)(j + 1) * ld] = acc;
      }
      __syncthreads();
      ArgMax rl{-1.0, 0x7fffffff};
      for (int i = k + tid; i < p; i += nth)
        if (i != imax) rl = amax(rl, ArgMax{cabs1(W[i + (int64_t)(j + 1) * ld]), i});
      ArgMax rm = block_argmax(rl, red);
      const double rowmax = rm.v > 0 ? rm.v : 0.0;
      if (tid == 0) {
        s_cmac += (double)(m - k) * j;
        if (absakk * rowmax >= BK_ALPHA * colmax * colmax) {
          s_kp = k;
        } else if (cabs1(W[imax + (int64_t)(j + 1) * ld]) >= BK_ALPHA * rowmax) {
          s_kp = imax;
          s_kstep = -1;  // 1x1 at imax: copy column j+1 into j below
        } else {
          s_kp = imax;
          s_kstep = 2;
        }
      }
      __syncthreads();
      if (s_kstep == -1) {
        for (int i = k + tid; i < m; i += nth) W[i + (int64_t)j * ld] = W[i + (int64_t)(j + 1) * ld];
      }
    }
    __syncthreads();
    const int kstep = s_kstep == 2 ? 2 : 1;
    const int kp = s_kp;
    const int kk = k + kstep - 1;
    if (kp != kk) {
      // copy the non-updated column kk into position kp (its old content is in W)
      if (tid == 0) F[kp + (int64_t)kp * ld] = F[kk + (int64_t)kk * ld];
      for (int i = kk + 1 + tid; i < kp; i += nth) F[kp + (int64_t)i * ld] = F[i + (int64_t)kk * ld];
      for (int i = kp + 1 + tid; i < m; i += nth) F[i + (int64_t)kp * ld] = F[i + (int64_t)kk * ld];
      __syncthreads();
      // interchange rows kk and kp in the factored columns and in W
      for (int cidx = tid; cidx < kk; cidx += nth) {
        cx<T> a = F[kk + (int64_t)cidx * ld], b = F[kp + (int64_t)cidx * ld];
        F[kk + (int64_t)cidx * ld] = b;
        F[kp + (int64_t)cidx * ld] = a;
      }
      for (int t = tid; t < j + kstep; t += nth) {
        cx<T> a = W[kk + (int64_t)t * ld], b = W[kp + (int64_t)t * ld];
        W[kk + (int64_t)t * ld] = b;
        W[kp + (int64_t)t * ld] = a;
      }
      if (tid == 0) {
        int32_t a = pv[kk];
        pv[kk] = pv[kp];
        pv[kp] = a;
      }
    }
    __syncthreads();
    if (kstep == 1) {
      cx<T> d = W[k + (int64_t)j * ld];
      double2 dd0 = to_d(d);
      if (tid == 0) s_dinv = (dd0.x == 0.0 && dd0.y == 0.0) ? make_double2(0.0, 0.0) : zdiv1(dd0);
      __syncthreads();
      double2 di = s_dinv;
      cx<T> dinv = from_d<T>(di);
      for (int i = k + 1 + tid; i < m; i += nth) F[i + (int64_t)k * ld] = cmul(W[i + (int64_t)j * ld], dinv);
      if (tid == 0) {
        F[k + (int64_t)k * ld] = d;
        dd[k] = di;
        dof[k] = make_double2(0.0, 0.0);
        ps[k] = 1;
        double r = colmax > 0 ? (fabs(dd0.x) + fabs(dd0.y)) / colmax : 1e300;
        s_minpiv = fmin(s_minpiv, r);
      }
    } else {
      double2 d11 = to_d(W[k + (int64_t)j * ld]);
      double2 d21 = to_d(W[k + 1 + (int64_t)j * ld]);
      double2 d22 = to_d(W[k + 1 + (int64_t)(j + 1) * ld]);
      double2 det = zmul(d11, d22);
      double2 d2 = zmul(d21, d21);
      det.x -= d2.x;
      det.y -= d2.y;
      double2 idet = zdiv1(det);
      double2 i11 = zmul(d22, idet), i22 = zmul(d11, idet), i21 = zmul(d21, idet);
      i21.x = -i21.x;
      i21.y = -i21.y;
      cx<T> a11 = from_d<T>(i11), a21 = from_d<T>(i21), a22 = from_d<T>(i22);
      for (int i = k + 2 + tid; i < m; i += nth) {
        cx<T> w1 = W[i + (int64_t)j * ld], w2 = W[i + (int64_t)(j + 1) * ld];
        cx<T> l1 = cfma(cmul(w1, a11), w2, a21);
        cx<T> l2 = cfma(cmul(w1, a21), w2, a22);
        F[i + (int64_t)k * ld] = l1;
        F[i + (int64_t)(k + 1) * ld] = l2;
      }
      if (tid == 0) {
        // D on the diagonal; L(k+1, k) of a 2x2 pair is 0 (the coupling of D
        // lives only in the inverse arrays), so every consumer may read the
        // pivot columns as a plain unit-lower L
        F[k + (int64_t)k * ld] = W[k + (int64_t)j * ld];
        F[k + 1 + (int64_t)k * ld] = mk<T>(0, 0);
        F[k + 1 + (int64_t)(k + 1) * ld] = W[k + 1 + (int64_t)(j + 1) * ld];
        dd[k] = i11;
        dd[k + 1] = i22;
        dof[k] = i21;
        dof[k + 1] = i21;
        ps[k] = 2;
        ps[k + 1] = -2;
      }
    }
    __syncthreads();
    k += kstep;
    j += kstep;
  }
  if (tid == 0) {
    st_k0[f] = k;
    st_kb[f] = j;
    snap[blockIdx.x] = make_int2(k, j);
    if (s_minpiv < st_minpiv[f]) st_minpiv[f] = s_minpiv;
    if (flop_cnt) {
      const double n = (double)(m - k);
      atomicAdd(flop_cnt, 8.0 * j * n * (n + 1.0) * 0.5);  // trailing update of this panel
      atomicAdd(flop_cnt + 1, 8.0 * s_cmac);                 // column updates inside the panel
    }
  }
}

// ------------------------------------------------------------ cluster panel kernel
// The same restricted Bunch-Kaufman panel as k_panel, run by a thread-block
// cluster of CS CTAs per front on the pivot rows [k0, p) (the update rows are
// k_l21's), with the panel's L rows resident in the cluster's distributed
// shared memory.  The rows are split into CS contiguous slot ranges; a row
// interchange only permutes the replicated logical-row <-> slot tables (data
// stays in its slot) and moves the not yet factored column in the global front.
// Per column: every CTA updates its slots of the column (original column from
// global, L from its shared memory, the pivot row of L from the owner CTA via
// DSMEM) and reduces its local pivot search; with CS > 1 it posts the result
// in a mailbox and, after one cluster barrier, every thread reads all
// mailboxes.  Every thread then takes the same pivot decision (fp32 path:
// tests in fp32 with an exact fp64 re-evaluation when the two sides are
// within rounding; fp64 path: one thread, published through shared memory,
// because an fp64 instruction issued by all 512 threads costs hundreds of
// cycles on GB300).  The panel's L and D columns, W = L D and the row
// interchanges of the earlier panels' columns are written once, after the
// last column, in the final row order.
namespace cg = cooperative_groups;

// inverse of a pivot in the factor precision (scales the panel's L columns);
// fp32 scales against overflow, fp64 uses the Newton reciprocal below
__device__ __forceinline__ cx<float> cinv_t(cx<float> a) {
  // conj(a) / |a|^2 with a scaled by its largest component (no overflow);
  // two correctly rounded reciprocals instead of three divisions
  float s = fmaxf(fabsf(a.re), fabsf(a.im));
  if (s == 0.0f) return mk<float>(0, 0);
  const float is = __frcp_rn(s);
  float ar = a.re * is, ai = a.im * is;
  float r = __frcp_rn(s * (ar * ar + ai * ai));
  return mk<float>(ar * r, -ai * r);
}
__device__ __forceinline__ cx<double> cinv_t(cx<double> a) {
  if (a.re == 0.0 && a.im == 0.0) return mk<double>(0, 0);
  double2 z = zinv_nr(make_double2(a.re, a.im));
  return mk<double>(z.x, z.y);
}
__device__ __forceinline__ double cabs1_d(cx<float> a) { return fabs((double)a.re) + fabs((double)a.im); }
__device__ __forceinline__ double cabs1_d(cx<double> a) { return fabs(a.re) + fabs(a.im); }

// lhs < rhs for magnitudes evaluated in T; for T = float the comparison is
// re-evaluated in fp64 from the exact operands when the two sides agree to
// within 2^-20 (the rounding of their fp32 evaluation is below 2^-21), so the
// outcome is the exact fp64 test's
template <typename T, typename Exact>
__device__ __forceinline__ bool bk_less(T lhs, T rhs, Exact exact) {
  if (sizeof(T) == 8) return lhs < rhs;
  const T g = (T)9.5367431640625e-07;
  if (lhs < rhs * ((T)1 - g)) return true;
  if (lhs > rhs * ((T)1 + g)) return false;
  return exact();
}

// warp arg-max, the same result in every lane (uniform even for NaN input)
template <typename T>
__device__ __forceinline__ ArgMaxT<T> warp_argmaxT(ArgMaxT<T> x) {
  for (int o = 16; o > 0; o >>= 1) {
    ArgMaxT<T> y;
    y.v = __shfl_down_sync(0xffffffffu, x.v, o);
    y.i = __shfl_down_sync(0xffffffffu, x.i, o);
    x = amaxT(x, y);
  }
  x.v = __shfl_sync(0xffffffffu, x.v, 0);
  x.i = __shfl_sync(0xffffffffu, x.i, 0);
  return x;
}
// fp32: two warp reductions (redux.sync).  Non-negative floats order like
// their bit patterns; "no candidate" (-1) and NaN map to key 0, so they never
// beat a real candidate; among equal maxima the lowest index wins, as in amaxT.
template <>
__device__ __forceinline__ ArgMaxT<float> warp_argmaxT<float>(ArgMaxT<float> x) {
  const unsigned key = x.v >= 0.0f ? __float_as_uint(x.v) : 0u;
  const unsigned km = __reduce_max_sync(0xffffffffu, key);
  const unsigned idx = __reduce_min_sync(0xffffffffu, key == km ? (unsigned)x.i : 0x7fffffffu);
  ArgMaxT<float> r;
  r.i = (int)idx;
  r.v = idx == 0x7fffffffu ? -1.0f : __uint_as_float(km);
  return r;
}
// Block arg-max with one barrier: the warp results go to half `par` of sh
// (2 x 32 entries) and every warp reduces them itself.  Consecutive calls use
// alternate halves, so a half is rewritten only after the barrier of the call
// in between has been passed by every thread.
template <typename T>
__device__ __forceinline__ ArgMaxT<T> block_argmax1(ArgMaxT<T> x, ArgMaxT<T> *sh, int &par) {
  x = warp_argmaxT(x);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  ArgMaxT<T> *h = sh + 32 * par;
  if (l == 0) h[w] = x;
  __syncthreads();
  x = l < (int)(blockDim.x >> 5) ? h[l] : ArgMaxT<T>{(T)-1, 0x7fffffff};
  par ^= 1;
  return warp_argmaxT(x);
}

// acc - sum_{t<j} L[t] w[t]: the column update of one panel row.  For fp32,
// two complex terms per 16-byte shared-memory load and two independent
// accumulators (the dependent FMA chain halves); rows and w are 16-byte aligned.
__device__ __forceinline__ cx<float> col_update(cx<float> acc, const cx<float> *__restrict__ L,
                                                const cx<float> *__restrict__ w, int j) {
  cx<float> acc1 = mk<float>(0.f, 0.f);
  int t = 0;
#pragma unroll 4
  for (; t + 1 < j; t += 2) {
    const float4 l = *reinterpret_cast<const float4 *>(L + t);
    const float4 v = *reinterpret_cast<const float4 *>(w + t);
    acc = cfms(acc, mk<float>(l.x, l.y), mk<float>(v.x, v.y));
    acc1 = cfms(acc1, mk<float>(l.z, l.w), mk<float>(v.z, v.w));
  }
  if (t < j) acc = cfms(acc, L[t], w[t]);
  acc.re += acc1.re;
  acc.im += acc1.im;
  return acc;
}
__device__ __forceinline__ cx<double> col_update(cx<double> acc, const cx<double> *__restrict__ L,
                                                 const cx<double> *__restrict__ w, int j) {
#pragma unroll 4
  for (int t = 0; t < j; ++t) acc = cfms(acc, L[t], w[t]);
  return acc;
}

// the pivot decision of one column
template <typename T>
struct PivotDec {
  int imax, kstep, kp;
  int need2, singular, use_r;
  T colmax, absakk;
  cx<T> akk, vmax;
  cx<T> d11, d21, d22;  // D block in the factor precision
  cx<T> a11, a21, a22;  // its inverse in the factor precision
};
// what one CTA posts for the others (CS > 1)
template <typename T>
struct PanelBox {
  T cmax;           // local max |w_i| over candidate rows
  int cidx;         // its logical row
  int has;          // 1 if this CTA owns the queried row
  cx<T> vmax;       // the local winner itself
  cx<T> v1, v2;     // owner-published values (w at row k / at row imax)
};

// first half of the decision: column maximum and the 1x1 test on a_kk
template <typename T>
__device__ __forceinline__ void bk_decide1(PivotDec<T> &d, int k, int p, int cidx, cx<T> akk, cx<T> vmax) {
  d.akk = akk;
  d.vmax = vmax;
  d.imax = cidx;
  d.colmax = cabs1T(vmax);
  if (!(cidx < p)) {
    d.colmax = (T)0;
    d.vmax = mk<T>(0, 0);
    d.imax = k;
  }
  d.absakk = cabs1T(akk);
  d.singular = d.absakk == (T)0 && d.colmax == (T)0;
  const cx<T> va = d.akk, vm = d.vmax;
  d.need2 = !d.singular &&
            bk_less(d.absakk, (T)BK_ALPHA * d.colmax, [&] { return cabs1_d(va) < BK_ALPHA * cabs1_d(vm); });
}
// record the chosen block and its inverse in the factor precision
template <typename T>
__device__ __forceinline__ void bk_finish(PivotDec<T> &d, int kstep, int kp, int use_r, cx<T> d11, cx<T> d21,
                                          cx<T> d22) {
  d.kstep = kstep;
  d.kp = kp;
  d.use_r = use_r;
  d.d11 = d11;
  d.d21 = d21;
  d.d22 = d22;
  if (kstep == 1) {
    d.a11 = cinv_t(d11);
  } else {
    const cx<T> idet = cinv_t(cfms(cmul(d11, d22), d21, d21));
    d.a11 = cmul(d22, idet);
    d.a22 = cmul(d11, idet);
    const cx<T> n = cmul(d21, idet);
    d.a21 = mk<T>(-n.re, -n.im);
  }
}
// second half: the tests on the row maximum of column imax
template <typename T>
__device__ __forceinline__ void bk_decide2(PivotDec<T> &d, int k, T rowmax, cx<T> rwin, cx<T> wki, cx<T> wri) {
  const cx<T> va = d.akk, vm = d.vmax;
  const double cm = cabs1_d(vm);
  if (!bk_less(d.absakk * rowmax, (T)BK_ALPHA * d.colmax * d.colmax,
               [&] { return cabs1_d(va) * cabs1_d(rwin) < BK_ALPHA * cm * cm; })) {
    bk_finish(d, 1, k, 0, d.akk, mk<T>(0, 0), mk<T>(0, 0));
  } else if (!bk_less(cabs1T(wri), (T)BK_ALPHA * rowmax,
                      [&] { return cabs1_d(wri) < BK_ALPHA * cabs1_d(rwin); })) {
    bk_finish(d, 1, d.imax, 1, wri, mk<T>(0, 0), mk<T>(0, 0));
  } else {
    bk_finish(d, 2, d.imax, 0, d.akk, wki, wri);
  }
}

template <typename T>
__global__ void __launch_bounds__(512)
    k_panel_cl(const int32_t *__restrict__ lvl, FrontTab ft, const int64_t *__restrict__ wofs,
               cx<T> *__restrict__ arena, cx<T> *__restrict__ Wbuf, int32_t *__restrict__ perm,
               double2 *__restrict__ dinv_d, double2 *__restrict__ dinv_o, int8_t *__restrict__ psize,
               int32_t *__restrict__ st_k0, int32_t *__restrict__ st_kb, int32_t *__restrict__ st_info,
               double *__restrict__ st_minpiv, double *__restrict__ flop_cnt, int2 *__restrict__ swp, int rcap,
               int mcap, int2 *__restrict__ snap) {
  // fp32: every thread takes the decisions; fp64: one thread, then a barrier
  constexpr bool ONE = sizeof(T) == 8;
  cg::cluster_group cl = cg::this_cluster();
  const int CS = (int)cl.num_blocks();
  const int rank = (int)cl.block_rank();
  const int fi = blockIdx.x / CS;
  const int f = lvl[fi];
  const int m = ft.m[f], p = ft.p[f];
  const int k0 = st_k0[f];
  const int tid = threadIdx.x, nth = blockDim.x;
  if (k0 >= p) {  // uniform over the cluster
    if (rank == 0 && tid == 0) {
      st_kb[f] = 0;
      snap[fi] = make_int2(k0, 0);
    }
    return;
  }
  cx<T> *F = arena + ft.off[f];
  cx<T> *W = Wbuf + wofs[fi];
  int32_t *pv = perm + ft.piv[f];
  double2 *dd = dinv_d + ft.piv[f];
  double2 *dof = dinv_o + ft.piv[f];
  int8_t *ps = psize + ft.piv[f];
  const int64_t ld = m;
  const int nr = p - k0;  // pivot rows only: update rows (>= p) are done by k_l21
  const int R = (nr + CS - 1) / CS;
  const int s_lo = rank * R;                 // first global slot of this CTA
  const int ns = max(0, min(R, nr - s_lo));  // slots owned
  // shared memory layout
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<T> *Ls = reinterpret_cast<cx<T> *>(smem_raw);       // [rcap][LSTR]
  cx<T> *wk = Ls + (size_t)rcap * LSTR;                   // [rcap]
  cx<T> *wr = wk + rcap;                                  // [rcap]
  int *spos = reinterpret_cast<int *>(wr + rcap);         // [rcap] logical row of each own slot
  int *p2s = spos + rcap;                                 // [mcap] logical row - k0 -> global slot
  // per-column mailbox of the cluster: every CTA's thread 0 writes its record
  // into slot [rank] of every CTA's copy before the cluster barrier, so the
  // records are read from local shared memory after it ([0]: the column
  // arg-max, [1]: the row arg-max of the 2x2 test)
  __shared__ PanelBox<T> box[2][16];
  __shared__ __align__(16) cx<T> wrow[(512 / 32) * NB];   // one staged row per warp
  __shared__ __align__(16) cx<T> wrow2[(512 / 32) * NB];
  __shared__ cx<T> Dd[NB], Do[NB];    // D of the panel's pivots: diag / 2x2 coupling
  __shared__ cx<T> Ei[NB], Eo[NB];    // D^{-1} in the factor precision (fp32 path): diag / 2x2 coupling
  __shared__ PivotDec<T> pd;          // fp64 path: the decision of thread 0
  __shared__ int Dz[NB];              // 1, 2 (first of a pair), -2
  __shared__ ArgMaxT<T> red[64];
  __shared__ int s_nmv, s_nout;
  __shared__ int2 s_mv[2 * NB];       // rows moved by the panel: (destination, source)
  for (int q = tid; q < nr; q += nth) p2s[q] = q;  // slot q holds row k0 + q initially
  if (rank == 0 && tid < 2 * NB) swp[(int64_t)fi * 2 * NB + tid] = make_int2(-1, -1);
  for (int q = tid; q < ns; q += nth) spos[q] = k0 + s_lo + q;
  if (tid == 0) s_nmv = s_nout = 0;
  __syncthreads();
  if (CS > 1) cl.sync();
  // a cluster of one synchronises like a plain block
  auto csync = [&]() {
    if (CS == 1)
      __syncthreads();
    else
      cl.sync();
  };
  // Original (not yet updated) data of the column being processed (cur) and
  // of the next column (nx, loaded at the start of the current column), for
  // the own slots q = tid and tid + nth (a CTA owns at most 2 nth slots).
  // An interchange moves data with the slots, so nx stays valid for the next
  // column except for one entry, passed through fixv (see below).
  cx<T> cur0 = mk<T>(0, 0), cur1 = mk<T>(0, 0), nx0 = mk<T>(0, 0), nx1 = mk<T>(0, 0);
  if (tid < ns) cur0 = F[spos[tid] + (int64_t)k0 * ld];
  if (tid + nth < ns) cur1 = F[spos[tid + nth] + (int64_t)k0 * ld];
  __shared__ cx<T> fixv;
  int k = k0, j = 0, par = 0;
  long long cmac = 0;        // complex MACs of the column updates (thread 0)
  float minpiv = 3.0e38f;    // smallest |d| / colmax of the 1x1 pivots (thread 0)
  // W row of logical row `row` for the panel columns 0..j-1: L[row, :] D
  // Every warp stages the row into its own buffer (lane t: element t), so
  // only a warp barrier separates the staging from its use.
  auto load_wrow = [&](int row, cx<T> *dst) {
    int g = p2s[row - k0];
    int o = g / R, sl = g - o * R;
    const cx<T> *Lr = (CS == 1 ? Ls : cl.map_shared_rank(Ls, o)) + (size_t)sl * LSTR;
    const int lane = tid & 31;
    {
      cx<T> v = mk<T>(0, 0);
      if (lane < j) {
        int t = lane;
        cx<T> l = Lr[t];
        if (Dz[t] == 1) {
          v = cmul(l, Dd[t]);
        } else if (Dz[t] == 2) {  // [l_t l_t+1] [[d11 d21][d21 d22]] column t
          v = cfma(cmul(l, Dd[t]), Lr[t + 1], Do[t]);
        } else {  // second of a pair: column t = [d21 d22]^T
          v = cfma(cmul(Lr[t - 1], Do[t]), l, Dd[t]);
        }
      }
      dst[(tid >> 5) * NB + lane] = v;
    }
    __syncwarp();
  };
  // value of own-CTA slot array a at logical row `row` (CS == 1: any row)
  auto own_at = [&](const cx<T> *a, int row) { return a[p2s[row - k0] - rank * R]; };
  while (k < p && j < NB - 1) {
    if (k + 1 < p) {  // the next column, in flight during this one
      if (tid < ns && spos[tid] >= k + 1) nx0 = F[spos[tid] + (int64_t)(k + 1) * ld];
      if (tid + nth < ns && spos[tid + nth] >= k + 1) nx1 = F[spos[tid + nth] + (int64_t)(k + 1) * ld];
    }
    // ---- (1) updated column k for own slots, local pivot search
    load_wrow(k, wrow);
    const cx<T> *wrw = wrow + (tid >> 5) * NB;  // this warp's copy
    ArgMaxT<T> loc{(T)-1, 0x7fffffff};
    for (int q = tid, qi = 0; q < ns; q += nth, ++qi) {
      int i = spos[q];
      if (i < k) continue;
      cx<T> acc = qi == 0 ? cur0 : cur1;
      const cx<T> *Lq = Ls + (size_t)q * LSTR;
      acc = col_update(acc, Lq, wrw, j);  // j terms (not NB predicated)
      wk[q] = acc;
      if (i > k && i < p) loc = amaxT(loc, ArgMaxT<T>{cabs1T(acc), i});
    }
    cmac += (long long)(p - k) * (j + 1);
    ArgMaxT<T> cm = block_argmax1(loc, red, par);
    cx<T> akk, vmax;
    if (CS == 1) {
      akk = own_at(wk, k);
      vmax = cm.i < p ? own_at(wk, cm.i) : mk<T>(0, 0);
    } else {
      const int gk = p2s[k - k0];
      if (tid == 0) {
        PanelBox<T> mb;
        mb.cmax = cm.v;
        mb.cidx = cm.i;
        mb.has = gk / R == rank;
        mb.v1 = gk / R == rank ? wk[gk - rank * R] : mk<T>(0, 0);
        mb.vmax = cm.i < p ? own_at(wk, cm.i) : mk<T>(0, 0);
        mb.v2 = mk<T>(0, 0);
        for (int c = 0; c < CS; ++c) cl.map_shared_rank(&box[0][0], c)[rank] = mb;
      }
      cl.sync();  // #1
      ArgMaxT<T> best{(T)-1, 0x7fffffff};
      vmax = mk<T>(0, 0);
      akk = mk<T>(0, 0);
      for (int c = 0; c < CS; ++c) {
        const PanelBox<T> *b = &box[0][c];
        const T v = b->cmax;
        const int i = b->cidx;
        if (v > best.v || (v == best.v && i < best.i)) {
          best = ArgMaxT<T>{v, i};
          vmax = b->vmax;
        }
        if (b->has) akk = b->v1;
      }
      cm = best;
    }
    PivotDec<T> d;
    if (ONE) {
      if (tid == 0) {
        bk_decide1(pd, k, p, cm.i, akk, vmax);
        if (!pd.need2) bk_finish(pd, 1, k, 0, akk, mk<T>(0, 0), mk<T>(0, 0));
      }
      __syncthreads();
      d = pd;
    } else {
      bk_decide1(d, k, p, cm.i, akk, vmax);
      if (!d.need2) bk_finish(d, 1, k, 0, akk, mk<T>(0, 0), mk<T>(0, 0));
    }
    if (d.need2) {
      const int imax = d.imax;
      // ---- (2) updated column imax for own slots
      // original column imax of the own rows: loads issued first, in flight
      // while row imax's W entries are staged
      cx<T> g0 = mk<T>(0, 0), g1 = mk<T>(0, 0);
      if (tid < ns) {
        const int i = spos[tid];
        if (i >= k) g0 = i < imax ? F[imax + (int64_t)i * ld] : F[i + (int64_t)imax * ld];
      }
      if (tid + nth < ns) {
        const int i = spos[tid + nth];
        if (i >= k) g1 = i < imax ? F[imax + (int64_t)i * ld] : F[i + (int64_t)imax * ld];
      }
      load_wrow(imax, wrow2);
      const cx<T> *wrw2 = wrow2 + (tid >> 5) * NB;
      ArgMaxT<T> rl{(T)-1, 0x7fffffff};
      for (int q = tid, qi = 0; q < ns; q += nth, ++qi) {
        int i = spos[q];
        if (i < k) continue;
        cx<T> acc = qi == 0 ? g0 : g1;
        const cx<T> *Lq = Ls + (size_t)q * LSTR;
        acc = col_update(acc, Lq, wrw2, j);
        wr[q] = acc;
        if (i != imax && i < p) rl = amaxT(rl, ArgMaxT<T>{cabs1T(acc), i});
      }
      cmac += (long long)(p - k) * j;
      ArgMaxT<T> rm = block_argmax1(rl, red, par);
      cx<T> rwin, wki, wri;
      T rowmax;
      if (CS == 1) {
        rowmax = rm.i < p ? rm.v : (T)0;
        rwin = rm.i < p ? own_at(wr, rm.i) : mk<T>(0, 0);
        wki = own_at(wk, imax);
        wri = own_at(wr, imax);
      } else {
        const int gi = p2s[imax - k0];
        if (tid == 0) {
          PanelBox<T> mb;
          mb.cmax = rm.i < p ? rm.v : (T)-1;
          mb.cidx = rm.i;
          mb.vmax = rm.i < p ? own_at(wr, rm.i) : mk<T>(0, 0);
          mb.has = gi / R == rank;
          mb.v1 = gi / R == rank ? wk[gi - rank * R] : mk<T>(0, 0);  // w_k at row imax
          mb.v2 = gi / R == rank ? wr[gi - rank * R] : mk<T>(0, 0);  // w_r at row imax
          for (int c = 0; c < CS; ++c) cl.map_shared_rank(&box[1][0], c)[rank] = mb;
        }
        cl.sync();  // #2
        rowmax = (T)0;
        double rex = 0.0;  // exact magnitude of the largest winner
        rwin = mk<T>(0, 0);
        wki = wri = mk<T>(0, 0);
        for (int c = 0; c < CS; ++c) {
          const PanelBox<T> *b = &box[1][c];
          if (b->cmax > rowmax) rowmax = b->cmax;
          if (b->cmax >= (T)0 && cabs1_d(b->vmax) > rex) {
            rex = cabs1_d(b->vmax);
            rwin = b->vmax;
          }
          if (b->has) {
            wki = b->v1;
            wri = b->v2;
          }
        }
      }
      if (ONE) {
        if (tid == 0) bk_decide2(pd, k, rowmax, rwin, wki, wri);
        __syncthreads();
        d = pd;
      } else {
        bk_decide2(d, k, rowmax, rwin, wki, wri);
      }
    }
    const int kstep = d.kstep, kp = d.kp;
    const int kk = k + kstep - 1;
    if (tid == 0) {
      if (d.singular && rank == 0 && st_info[f] == 0) st_info[f] = k + 1;
      if (kstep == 1 && d.colmax > (T)0) minpiv = fminf(minpiv, (float)cabs1_d(d.d11) / (float)d.colmax);
    }
    if (kp != kk) {
      // ---- interchange kk <-> kp: the not yet factored column kk (original
      // data: cur for kk = k, nx for kk = k + 1) moves to position kp in the
      // global front; each thread writes the rows of its own slots
      for (int q = tid, qi = 0; q < ns; q += nth, ++qi) {
        const int i = spos[q];
        const cx<T> v = kstep == 1 ? (qi == 0 ? cur0 : cur1) : (qi == 0 ? nx0 : nx1);
        if (i > kk && i < kp) F[kp + (int64_t)i * ld] = v;
        else if (i > kp) F[i + (int64_t)kp * ld] = v;
        else if (i == kk) F[kp + (int64_t)kp * ld] = v;
        // after a 1x1 interchange with kp > k + 1 the slot now at row kp needs
        // A[kp, k+1] = A[k+1, k] (original), held by the slot of row k + 1
        if (kstep == 1 && kp > k + 1 && i == k + 1) fixv = qi == 0 ? cur0 : cur1;
      }
      csync();  // the moves have read their sources; every thread has read p2s
      for (int q = tid; q < ns; q += nth) {
        if (spos[q] == kk) spos[q] = kp;
        else if (spos[q] == kp) spos[q] = kk;
      }
      if (tid == 0) {
        int ga = p2s[kk - k0];
        p2s[kk - k0] = p2s[kp - k0];
        p2s[kp - k0] = ga;
      }
    }
    // ---- original data of the next column for the own slots
    if (kstep == 1 && k + 1 < p) {
      if (kp == k + 1) {  // the next column is the old column k
        nx0 = cur0;
        nx1 = cur1;
      } else if (kp != kk) {
        const int g1 = p2s[k + 1 - k0];  // row k + 1 did not move
        const cx<T> fv = CS == 1 ? fixv : *cl.map_shared_rank(&fixv, g1 / R);
        if (tid < ns && spos[tid] == kp) nx0 = fv;
        if (tid + nth < ns && spos[tid + nth] == kp) nx1 = fv;
      }
      cur0 = nx0;
      cur1 = nx1;
    } else if (kstep == 2 && k + 2 < p) {
      if (kp == k + 2) {  // the next column is the old column k + 1
        cur0 = nx0;
        cur1 = nx1;
      } else {  // loaded after the interchange (which may have written row kp of it)
        if (tid < ns && spos[tid] >= k + 2) cur0 = F[spos[tid] + (int64_t)(k + 2) * ld];
        if (tid + nth < ns && spos[tid + nth] >= k + 2) cur1 = F[spos[tid + nth] + (int64_t)(k + 2) * ld];
      }
    }
    // ---- scale: L columns of own slots (in shared memory; written to the
    // front after the last column)
    if (kstep == 1) {
      const cx<T> dinv = d.a11;
      const cx<T> *src = d.use_r ? wr : wk;
      for (int q = tid; q < ns; q += nth) {
        int i = spos[q];
        if (i < k) continue;
        Ls[(size_t)q * LSTR + j] = i == k ? mk<T>(1, 0) : cmul(src[q], dinv);
      }
      if (tid == 0) {
        Dd[j] = d.d11;
        Do[j] = mk<T>(0, 0);
        Dz[j] = 1;
        Ei[j] = d.a11;
        Eo[j] = mk<T>(0, 0);
      }
    } else {
      const cx<T> a11 = d.a11, a21 = d.a21, a22 = d.a22;
      for (int q = tid; q < ns; q += nth) {
        int i = spos[q];
        if (i < k) continue;
        cx<T> l1, l2;
        if (i == k) {
          l1 = mk<T>(1, 0);
          l2 = mk<T>(0, 0);
        } else if (i == k + 1) {
          l1 = mk<T>(0, 0);
          l2 = mk<T>(1, 0);
        } else {
          cx<T> w1 = wk[q], w2 = wr[q];
          l1 = cfma(cmul(w1, a11), w2, a21);
          l2 = cfma(cmul(w1, a21), w2, a22);
        }
        Ls[(size_t)q * LSTR + j] = l1;
        Ls[(size_t)q * LSTR + j + 1] = l2;
      }
      if (tid == 0) {
        Dd[j] = d.d11;
        Dd[j + 1] = d.d22;
        Do[j] = d.d21;
        Do[j + 1] = d.d21;
        Dz[j] = 2;
        Dz[j + 1] = -2;
        Ei[j] = d.a11;
        Ei[j + 1] = d.a22;
        Eo[j] = d.a21;
        Eo[j + 1] = d.a21;
      }
    }
    csync();  // #3: L rows, D and the tables are consistent for the next column
    k += kstep;
    j += kstep;
  }
  // ---- D^{-1} of the panel's pivots (one thread per pivot), stored in fp64.
  // fp32 path: the inverses the decisions computed (every consumer of the
  // complex64 factors uses D^{-1} in fp32); fp64 path: computed here.
  if (sizeof(T) == 4 && rank == 0 && tid < j) {
    const int t = tid, z = Dz[t];
    const bool zero = z == 1 && Dd[t].re == (T)0 && Dd[t].im == (T)0;
    dd[k0 + t] = zero ? make_double2(0, 0) : to_d(Ei[t]);
    dof[k0 + t] = to_d(Eo[t]);
    ps[k0 + t] = (int8_t)z;
  } else if (rank == 0 && tid < j) {
    const int t = tid, z = Dz[t];
    if (z == 1) {
      const double2 d11 = to_d(Dd[t]);
      dd[k0 + t] = (d11.x == 0.0 && d11.y == 0.0) ? make_double2(0, 0) : zinv_nr(d11);
      dof[k0 + t] = make_double2(0, 0);
      ps[k0 + t] = 1;
    } else if (z == 2) {
      const double2 d11 = to_d(Dd[t]), d22 = to_d(Dd[t + 1]), d21 = to_d(Do[t]);
      double2 det = zmul(d11, d22), d2 = zmul(d21, d21);
      det.x -= d2.x;
      det.y -= d2.y;
      const double2 idet = zinv_nr(det), t21 = zmul(d21, idet);
      dd[k0 + t] = zmul(d22, idet);
      dd[k0 + t + 1] = zmul(d11, idet);
      dof[k0 + t] = make_double2(-t21.x, -t21.y);
      dof[k0 + t + 1] = make_double2(-t21.x, -t21.y);
      ps[k0 + t] = 2;
      ps[k0 + t + 1] = -2;
    }
  }
  // ---- the panel's columns in the final row order: L below the diagonal,
  // D on it (the coupling entry L(k+1, k) of a 2x2 pair is stored as 0, so
  // every consumer may read the pivot columns as a plain unit-lower L), and
  // W = L D for the rows below the panel (trailing update input)
  // (thread -> logical rows k0 + tid, k0 + tid + nth, ...: consecutive threads
  // write consecutive rows; the slot of a row comes from p2s)
  for (int i = k0 + tid; i < p; i += nth) {
    const int g = p2s[i - k0];
    if (g / R != rank) continue;  // another CTA of the cluster holds the row
    const cx<T> *Lq = Ls + (size_t)(g - rank * R) * LSTR;
#pragma unroll 4
    for (int t = 0; t < j; ++t) {
      const int c = k0 + t;
      if (c < i) F[i + (int64_t)c * ld] = Lq[t];
      else if (c == i) F[i + (int64_t)c * ld] = Dd[t];
    }
    if (i < k) continue;
#pragma unroll 4
    for (int t = 0; t < j; ++t) {
      cx<T> l = Lq[t], acc;
      if (Dz[t] == 1) {
        acc = cmul(l, Dd[t]);
      } else if (Dz[t] == 2) {
        acc = cfma(cmul(l, Dd[t]), Lq[t + 1], Do[t]);
      } else {
        acc = cfma(cmul(Lq[t - 1], Do[t]), l, Dd[t]);
      }
      W[i + (int64_t)t * ld] = acc;
    }
  }
  // ---- the panel's row interchanges on the earlier panels' columns [0, k0):
  // logical row r now holds what row k0 + p2s[r - k0] held
  for (int q = tid; q < nr; q += nth)
    if (p2s[q] != q) {
      int a = atomicAdd(&s_nmv, 1);
      s_mv[a] = make_int2(k0 + q, k0 + p2s[q]);
    }
  __syncthreads();  // Ls is free from here on: staging buffer for the moves
  const int nmv = s_nmv;
  // the panel's interchanges on the pivot order (rank 0): position r now holds
  // what position k0 + p2s[r - k0] held (staged, since the gather is in place)
  if (rank == 0 && nmv > 0) {
    int32_t *pvs = reinterpret_cast<int32_t *>(Ls);  // nr ints fit: 4 nr <= 8 LSTR rcap
    for (int q = tid; q < nr; q += nth) pvs[q] = pv[k0 + p2s[q]];
    __syncthreads();
    for (int q = tid; q < nr; q += nth)
      if (p2s[q] != q) pv[k0 + q] = pvs[q];
    __syncthreads();
  }
  // the panel's column permutation for k_l21 (update rows): per panel column
  // its source column, then the moves (destination, source) of the columns
  // right of the panel
  if (rank == 0) {
    int2 *rec = swp + (int64_t)fi * 2 * NB;
    if (tid < j) rec[tid] = make_int2(k0 + p2s[tid], 0);
    if (tid < nmv && s_mv[tid].x >= k0 + j) rec[NB + atomicAdd(&s_nout, 1)] = s_mv[tid];
  }
  if (nmv > 0 && k0 > 0) {
    const int cap = rcap * LSTR;
    const int cpc = cap / nmv;  // columns per chunk (nmv <= min(2 NB, nr) <= LSTR rcap)
    const int ncol = (k0 + CS - 1) / CS, c_lo = rank * ncol, c_hi = min(k0, c_lo + ncol);
    for (int cb = c_lo; cb < c_hi; cb += cpc) {
      const int nc = min(cpc, c_hi - cb), ne = nc * nmv;
      for (int e0 = tid; e0 < ne; e0 += 8 * nth) {  // 8 loads in flight per thread
        cx<T> v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int e = e0 + u * nth;
          if (e < ne) {
            const int2 mv = s_mv[e % nmv];
            v[u] = F[mv.y + (int64_t)(cb + e / nmv) * ld];
          }
        }
#pragma unroll
        for (int u = 0; u < 8; ++u)
          if (e0 + u * nth < ne) Ls[e0 + u * nth] = v[u];
      }
      __syncthreads();
      for (int e = tid; e < ne; e += nth) {
        const int2 mv = s_mv[e % nmv];
        F[mv.x + (int64_t)(cb + e / nmv) * ld] = Ls[e];
      }
      __syncthreads();
    }
  }
  if (rank == 0 && tid == 0) {
    st_k0[f] = k;
    st_kb[f] = j;
    snap[fi] = make_int2(k, j);  // this step's (k0 + kb, kb) for the trailing updates
  }
  if (tid == 0) {
    if (flop_cnt && rank == 0) {
      const double n = (double)(m - k);
      atomicAdd(flop_cnt, 8.0 * j * n * (n + 1.0) * 0.5);
      atomicAdd(flop_cnt + 1, 8.0 * (double)cmac);
    }
    if (minpiv < 3.0e38f)
      atomicMin(reinterpret_cast<unsigned long long *>(st_minpiv + f),
                (unsigned long long)__double_as_longlong((double)minpiv));
  }
  csync();  // no CTA leaves while others may still read its shared memory
}

static size_t panel_cl_smem(int rcap, int mcap, size_t esz) {
  return (size_t)rcap * LSTR * esz + 2 * (size_t)rcap * esz + (size_t)rcap * 4 + (size_t)mcap * 4;
}

// Update rows of the panel's columns (rows p..m-1), Algorithm 1's triangular
// solve: apply the panel's column permutation to the row (the panel columns
// gathered from their source columns, the moved columns right of the panel
// rewritten; all loads before any store), then w = a L11^{-T}
// (forward substitution with the panel's unit-lower block), L21 = w D^{-1};
// L21 goes to the front, w (= L21 D) to the workspace for the trailing update.
// One thread per update row, all fronts of the level.
// The step is read from the panel's (k0 + kb, kb) snapshot, so the kernel may
// run behind later panels on another stream.  With w21 given (mixed path,
// deferred Schur products), w goes to the front's W21 block of that buffer
// (column-major (m - p) x p at w21_off[level position]) instead of the
// workspace.
template <typename T>
__global__ void __launch_bounds__(128) k_l21(const int32_t *__restrict__ lvl, FrontTab ft,
                                             const int64_t *__restrict__ wofs, cx<T> *__restrict__ arena,
                                             cx<T> *__restrict__ Wbuf, const double2 *__restrict__ dinv_d,
                                             const double2 *__restrict__ dinv_o, const int8_t *__restrict__ psize,
                                             const int2 *__restrict__ snap, const int2 *__restrict__ swp,
                                             double *__restrict__ flop_cnt, float2 *__restrict__ w21,
                                             const int64_t *__restrict__ w21_off) {
  const int fi = blockIdx.y;
  const int f = lvl[fi];
  const int kb = snap[fi].y;
  if (kb == 0) return;
  const int m = ft.m[f], p = ft.p[f];
  const int r = p + blockIdx.x * blockDim.x + threadIdx.x;
  if (p + (int)(blockIdx.x * blockDim.x) >= m) return;  // uniform per CTA
  const int k0 = snap[fi].x - kb;
  cx<T> *F = arena + ft.off[f];
  cx<T> *W = Wbuf + wofs[fi];
  float2 *W21 = w21 ? w21 + w21_off[fi] + (r - p) : nullptr;
  const int64_t ld = m;
  __shared__ cx<T> L11[NB][NB + 1];
  __shared__ cx<T> Di[NB], Do[NB];
  __shared__ int Dz[NB];
  __shared__ int s_src[NB];   // source column of panel column t
  __shared__ int2 s_out[NB];  // moves right of the panel: (destination, source)
  __shared__ int s_nout;
  {  // L11 of the panel: every load issued before the first shared store
    constexpr int NE = NB * NB / 128;
    cx<T> v[NE];
#pragma unroll
    for (int u = 0; u < NE; ++u) {
      const int e = threadIdx.x + 128 * u, a = e % NB, b = e / NB;
      v[u] = (a < kb && b < a) ? F[k0 + a + (int64_t)(k0 + b) * ld] : mk<T>(0, 0);
    }
#pragma unroll
    for (int u = 0; u < NE; ++u) {
      const int e = threadIdx.x + 128 * u;
      L11[e % NB][e / NB] = v[u];
    }
  }
  if (threadIdx.x < NB) {
    int t = threadIdx.x;
    const int2 *rec = swp + (int64_t)fi * 2 * NB;
    s_src[t] = t < kb ? rec[t].x : k0 + t;
    s_out[t] = rec[NB + t];
    const unsigned ball = __ballot_sync(0xffffffffu, rec[NB + t].x >= 0);
    if (t == 0) s_nout = __popc(ball);
    if (t < kb) {
      Di[t] = from_d<T>(dinv_d[ft.piv[f] + k0 + t]);
      Do[t] = from_d<T>(dinv_o[ft.piv[f] + k0 + t]);
      Dz[t] = psize[ft.piv[f] + k0 + t];
    }
  }
  __syncthreads();
  // 2x2 couplings inside L11 are zero by construction (stored as 0)
  if (r < m) {
    // the panel's column permutation on this row (the thread owns the row):
    // the panel columns gathered from their sources, then the columns right
    // of the panel, whose sources are panel columns that no move rewrites
    const int nout = s_nout;
    cx<T> a[NB];
#pragma unroll
    for (int t = 0; t < NB; ++t) a[t] = t < kb ? F[r + (int64_t)s_src[t] * ld] : mk<T>(0, 0);
    for (int u0 = 0; u0 < nout; u0 += 8) {
      cx<T> o[8];
#pragma unroll
      for (int u = 0; u < 8; ++u)
        if (u0 + u < nout) o[u] = F[r + (int64_t)s_out[u0 + u].y * ld];
#pragma unroll
      for (int u = 0; u < 8; ++u)
        if (u0 + u < nout) F[r + (int64_t)s_out[u0 + u].x * ld] = o[u];
    }
    // forward substitution: w[t] = a[t] - sum_{u<t} L11[t][u] w[u]
#pragma unroll
    for (int t = 1; t < NB; ++t) {
      if (t < kb) {
        cx<T> acc = a[t];
#pragma unroll
        for (int u = 0; u < NB - 1; ++u)
          if (u < t) acc = cfms(acc, L11[t][u], a[u]);
        a[t] = acc;
      }
    }
#pragma unroll
    for (int t = 0; t < NB; ++t) {
      if (t < kb) {
        if (W21)
          W21[(int64_t)(k0 + t) * (m - p)] = make_float2((float)a[t].re, (float)a[t].im);
        else
          W[r + (int64_t)t * ld] = a[t];
        cx<T> l;
        if (Dz[t] == 1) {
          l = cmul(a[t], Di[t]);
        } else if (Dz[t] == 2) {
          l = cfma(cmul(a[t], Di[t]), a[min(t + 1, NB - 1)], Do[t]);
        } else {
          l = cfma(cmul(a[max(t - 1, 0)], Do[t]), a[t], Di[t]);
        }
        F[r + (int64_t)(k0 + t) * ld] = l;
      }
    }
  }
  if (flop_cnt && threadIdx.x == 0 && blockIdx.x == 0) {
    atomicAdd(flop_cnt + 1, 8.0 * (double)(m - p) * (0.5 * kb * (kb - 1) + kb));
  }
}

constexpr size_t PANEL_SMEM_MAX = 200 * 1024;
// Cluster size for a level whose largest front has mmax rows: the smallest of
// 1, 2, 4, 8, 16 whose per-CTA shared memory fits; 0 = use the global panel.
static int panel_cluster_size(int mmax, size_t esz) {
  for (int cs = 1; cs <= 16; cs *= 2) {
    int rcap = (mmax + cs - 1) / cs;
    if (panel_cl_smem(rcap, mmax, esz) <= PANEL_SMEM_MAX) return cs;
  }
  return 0;
}

// Kernel launch with an optional scheduling priority (lower = more urgent, as
// for streams; 0 = the stream's own).  The attribute travels with the launch
// into a captured graph's kernel node, where stream priorities do not.
// Programmatic dependent launch (the substitution sweeps): a kernel launched
// with launch_pdl may start while its predecessor in the stream finishes;
// pdl_wait() blocks the calling thread until the predecessor grid has
// completed and its writes are visible, so every thread calls it before it
// touches memory the predecessor writes or reads.  pdl_trigger() lets the
// successor launch.  Both are no-ops in a kernel launched without the
// attribute.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
template <typename... KArgs, typename... Args>
static cudaError_t launch_pdl(bool on, void (*k)(KArgs...), dim3 g, dim3 b, size_t smem, cudaStream_t s,
                              Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = g;
  cfg.blockDim = b;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = on ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, k, args...);
}

template <typename... KArgs, typename... Args>
static cudaError_t launch_prio(void (*k)(KArgs...), dim3 g, dim3 b, size_t smem, cudaStream_t s, int prio,
                               Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = g;
  cfg.blockDim = b;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributePriority;
  at[0].val.priority = prio;
  cfg.attrs = at;
  cfg.numAttrs = prio != 0 ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, k, args...);
}

// Kernel attributes are per device: one "set" flag per device ordinal
// (ordinals beyond the table set the attributes on every call).
constexpr int ATTR_MAX_DEVICES = 64;
static bool *attr_flag(bool *tab) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= ATTR_MAX_DEVICES) return nullptr;
  return tab + dev;
}
template <typename T>
static cudaError_t panel_attrs() {
  static bool done[ATTR_MAX_DEVICES] = {};
  bool *f = attr_flag(done);
  if (f && *f) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(k_panel_cl<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)PANEL_SMEM_MAX);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_panel_cl<T>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (f) *f = e == cudaSuccess;
  return e;
}

// One panel step for the nf fronts listed at lvl.
// One panel step for the nf fronts listed at lvl.  cs > 0: cluster panel on
// the pivot rows (pmax = largest pivot block of the level) followed by k_l21
// on the update rows (mmax = largest front); cs == 0: single-CTA panel over
// all rows.
template <typename T>
static cudaError_t launch_panel(int cs, int pmax, int mmax, int nf, const int32_t *lvl, FrontTab ft,
                                const int64_t *wofs, cx<T> *arena, cx<T> *W, int32_t *perm, double2 *dd,
                                double2 *dof, int8_t *ps, int32_t *k0, int32_t *kb, int32_t *info, double *minpiv,
                                double *flops, int2 *swp, int2 *snap, cudaStream_t s, int prio = 0) {
  if (cs <= 0)
    return launch_prio(k_panel<T>, dim3(nf), dim3(PANEL_THREADS), 0, s, prio, lvl, ft, wofs, arena, W, perm, dd, dof,
                       ps, k0, kb, info, minpiv, flops, snap);
  cudaError_t e = panel_attrs<T>();
  if (e != cudaSuccess) return e;
  int rcap = (pmax + cs - 1) / cs;
  if (rcap > 2 * 512) return cudaErrorInvalidValue;  // k_panel_cl keeps two slots per thread
  const int mcap = pmax;
  // as many threads as one slot per row needs (whole warps, 64 to 512): warps
  // without rows would only add their share of every column's staging,
  // reductions and decision to the issue slots
  const int nth = std::min(512, std::max(64, (rcap + 31) / 32 * 32));
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(nf * cs));
  cfg.blockDim = dim3(nth);
  cfg.dynamicSmemBytes = panel_cl_smem(rcap, mcap, sizeof(cx<T>));
  cfg.stream = s;
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = cs;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  attr[1].id = cudaLaunchAttributePriority;
  attr[1].val.priority = prio;
  cfg.attrs = attr;
  cfg.numAttrs = prio != 0 ? 2 : 1;
  e = cudaLaunchKernelEx(&cfg, k_panel_cl<T>, lvl, ft, wofs, arena, W, perm, dd, dof, ps, k0, kb, info, minpiv,
                         flops, swp, rcap, mcap, snap);
  if (e != cudaSuccess) return e;
  if (mmax > 0) {
    dim3 g((unsigned)std::max(1, (mmax + 127) / 128), (unsigned)nf);
    e = launch_prio(k_l21<T>, g, dim3(128), 0, s, prio, lvl, ft, wofs, arena, W, (const double2 *)dd,
                    (const double2 *)dof, (const int8_t *)ps, (const int2 *)snap, (const int2 *)swp, flops,
                    (float2 *)nullptr, (const int64_t *)nullptr);
  }
  return e;
}

// ------------------------------------------------------------ trailing update
// F[i, c] -= sum_t L[i, k0+t] W[c, t] for k0+kb <= c <= i < m (lower triangle)
template <typename T>
__global__ void __launch_bounds__(256)
    k_update(const int32_t *__restrict__ lvl, FrontTab ft, const int64_t *__restrict__ wofs,
             cx<T> *__restrict__ arena, const cx<T> *__restrict__ Wbuf, const int2 *__restrict__ snap,
             int mode) {
  const int f = lvl[blockIdx.y];
  const int2 sk = snap[blockIdx.y];
  const int kb = sk.y;
  if (kb == 0) return;
  const int c0 = sk.x;
  const int k0 = c0 - kb;
  const int m = ft.m[f], p = ft.p[f];
  // column window: mode 0 every trailing column, 1 those of the pivot block
  // (< p), 2 those of the Schur complement (>= p); mode 3 the pivot block's
  // columns and rows only (the update rows and the Schur complement are left
  // to the deferred tensor-core products)
  // (to the deferred tensor-core products); mode 4 the update rows (>= p)
  // of the pivot block's columns, a rectangle of tiles
  const int clo = mode == 2 ? max(c0, p) : c0, chi = (mode == 1 || mode == 3 || mode == 4) ? p : m;
  const int rhi = mode == 3 ? p : m, rlo = mode == 4 ? p : 0;
  const int I0 = c0 / UT;
  const int nt = (rhi + UT - 1) / UT - I0;
  const int R4 = (p / UT) * UT, nr4 = (m - R4 + UT - 1) / UT, nc4 = (p - I0 * UT + UT - 1) / UT;
  const int ntl = mode == 4 ? (c0 < p ? nr4 * nc4 : 0) : (nt > 0 ? nt * (nt + 1) / 2 : 0);
  // tiles of the trailing lower triangle, grid-strided (a launch may use
  // fewer CTAs than tiles, leaving room on every SM for other kernels)
  for (int t = blockIdx.x; t < ntl; t += gridDim.x) {
  int r0, cc0;
  if (mode == 4) {
    r0 = R4 + (t % nr4) * UT;
    cc0 = (I0 + t / nr4) * UT;
  } else {
    int ii = (int)((sqrt(8.0 * t + 1.0) - 1.0) * 0.5);
    while (ii * (ii + 1) / 2 > t) --ii;
    while ((ii + 1) * (ii + 2) / 2 <= t) ++ii;
    const int jj = t - ii * (ii + 1) / 2;
    r0 = (I0 + ii) * UT;
    cc0 = (I0 + jj) * UT;
  }
  if (cc0 + UT <= clo || cc0 >= chi) continue;  // uniform per CTA
  cx<T> *F = arena + ft.off[f];
  const cx<T> *W = Wbuf + wofs[blockIdx.y];
  const int64_t ld = m;
  // K chunk: the whole panel (32 KB of shared memory) in fp32, half of it in fp64
  constexpr int KC = sizeof(T) == 4 ? NB : UK;
  __shared__ cx<T> Ls[KC][UT];
  __shared__ cx<T> Ws[KC][UT];
  // the fast thread index runs along the rows (column-major front), so every
  // warp access to the C tile covers two 128-byte column segments
  const int tr = threadIdx.x & 15, tc = threadIdx.x >> 4;
  // C tile first: its loads are in flight while L and W are staged
  cx<T> cv[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int i = r0 + tr + 16 * a;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int cidx = cc0 + tc + 16 * b;
      cv[a][b] = (i >= rlo && i < rhi && cidx >= clo && cidx < chi && cidx <= i) ? F[i + (int64_t)cidx * ld]
                                                                                 : mk<T>(0, 0);
    }
  }
  for (int t0 = 0; t0 < kb; t0 += KC) {
    // every load of the chunk is issued before the first shared store
    constexpr int NE = KC * UT / 256;
    cx<T> lr[NE], wr[NE];
#pragma unroll
    for (int u = 0; u < NE; ++u) {
      const int e = threadIdx.x + 256 * u;
      const int r = e % UT, tt = e / UT;
      const int gi = r0 + r, gc = cc0 + r;
      const bool ok = t0 + tt < kb;
      lr[u] = (ok && gi >= rlo && gi < rhi) ? F[gi + (int64_t)(k0 + t0 + tt) * ld] : mk<T>(0, 0);
      wr[u] = (ok && gc < chi) ? W[gc + (int64_t)(t0 + tt) * ld] : mk<T>(0, 0);
    }
    if (t0 > 0) __syncthreads();
#pragma unroll
    for (int u = 0; u < NE; ++u) {
      const int e = threadIdx.x + 256 * u;
      Ls[e / UT][e % UT] = lr[u];
      Ws[e / UT][e % UT] = wr[u];
    }
    __syncthreads();
    const int nt = min(KC, kb - t0);
#pragma unroll 4
    for (int tt = 0; tt < nt; ++tt) {
      cx<T> lv[4], wv[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) lv[a] = Ls[tt][tr + 16 * a];
#pragma unroll
      for (int b = 0; b < 4; ++b) wv[b] = Ws[tt][tc + 16 * b];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) cv[a][b] = cfms(cv[a][b], lv[a], wv[b]);
    }
  }
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int i = r0 + tr + 16 * a;
    if (i < rlo || i >= rhi) continue;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int cidx = cc0 + tc + 16 * b;
      if (cidx < clo || cidx >= chi || cidx > i) continue;
      F[i + (int64_t)cidx * ld] = cv[a][b];
    }
  }
  __syncthreads();  // the shared tiles are restaged for the next tile
  }
}

// ------------------------------------------------------------ tensor-core helpers
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
// Bounded wait on phase `parity` of an mbarrier: true once the phase has
// completed, false after `iters` unsuccessful polls.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t mbar, uint32_t parity, int iters) {
  uint32_t done = 0;
  for (int it = 0; it < iters && !done; ++it) {
    asm volatile(
        "{\n\t.reg .pred q;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}\n"
        : "=r"(done)
        : "r"(mbar), "r"(parity)
        : "memory");
  }
  return done != 0;
}

#include "tc_gemm.cuh"
#include "gmres_ir.cuh"

// ------------------------------------------------------------ solve kernels
// Vectors in M space and front-local vectors are row-major (RHS fastest).
// The forward sweep's right-hand side of every front of a level, in one
// pass: row k (pivot order) of front f is its entry of bM (pivot rows) plus
// the child update rows that extend-add into it, listed in a static CSR
// keyed by the parent's original row (gptr / gsrc: Y rows of the children);
// the pivot order maps position k to original row pv[k] at run time.
// One read of each source and one write of each row (no read-modify-write
// passes over the parent rows, one launch per level).
template <typename T>
__global__ void k_fwd_gather(const int32_t *__restrict__ lvl, FrontTab ft, const int32_t *__restrict__ perm,
                             const cx<T> *__restrict__ bM, const int64_t *__restrict__ gptr,
                             const int64_t *__restrict__ gsrc, cx<T> *__restrict__ Y, int r) {
  pdl_wait();  // the predecessor in the sweep has finished
  pdl_trigger();
  const int f = lvl[blockIdx.y];
  const int m = ft.m[f], p = ft.p[f];
  const int64_t n = (int64_t)m * r, y0 = ft.yoff[f];
  cx<T> *Yf = Y + y0 * r;
  const int32_t *pv = perm + ft.piv[f];
  const int64_t st = ft.start[f];
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const int k = (int)(e / r), c = (int)(e % r);
    const int o = k < p ? pv[k] : k;
    cx<T> v = k < p ? bM[(st + o) * r + c] : mk<T>(0, 0);
    const int64_t q0 = gptr[y0 + o], q1 = gptr[y0 + o + 1];
    for (int64_t q = q0; q < q1; ++q) {
      const cx<T> u = Y[gsrc[q] * r + c];
      v.re += u.re;
      v.im += u.im;
    }
    Yf[e] = v;
  }
}

// Forward substitution with unit-lower L11 (pivot rows only), then
// z = D^{-1} y written to zM in pivot order.  One CTA per (front, RC RHS).
template <typename T, int RC>
__global__ void __launch_bounds__(256) k_fwd_solve(const int32_t *__restrict__ lvl, FrontTab ft,
                                                   const cx<T> *__restrict__ arena,
                                                   const double2 *__restrict__ dinv_d,
                                                   const double2 *__restrict__ dinv_o,
                                                   const int8_t *__restrict__ psize, cx<T> *__restrict__ Y,
                                                   cx<T> *__restrict__ zM, int r) {
  pdl_wait();  // the predecessor in the sweep has finished
  pdl_trigger();
  const int f = lvl[blockIdx.y];
  const int m = ft.m[f], p = ft.p[f];
  const int c0 = blockIdx.x * RC;
  const int nc = min(RC, r - c0);
  const cx<T> *F = arena + ft.off[f];
  const int64_t ld = m;
  cx<T> *Yf = Y + ft.yoff[f] * r;
  const int8_t *ps = psize + ft.piv[f];
  __shared__ cx<T> Ld[32][33];
  __shared__ cx<T> ys[32][RC];
  const int tid = threadIdx.x;
  for (int kb0 = 0; kb0 < p; kb0 += 32) {
    const int nbk = min(32, p - kb0);
    for (int e = tid; e < 32 * 32; e += 256) {
      int a = e % 32, b = e / 32;
      cx<T> v = mk<T>(0, 0);
      if (a < nbk && b < nbk && a > b) {
        v = F[kb0 + a + (int64_t)(kb0 + b) * ld];
        if (a == b + 1 && ps[kb0 + b] == 2) v = mk<T>(0, 0);
      }
      Ld[a][b] = v;
    }
    for (int e = tid; e < 32 * RC; e += 256) {
      int a = e / RC, cc = e % RC;
      ys[a][cc] = (a < nbk && cc < nc) ? Yf[(int64_t)(kb0 + a) * r + c0 + cc] : mk<T>(0, 0);
    }
    __syncthreads();
    for (int b = 0; b < nbk - 1; ++b) {
      for (int e = tid; e < 32 * RC; e += 256) {
        int a = e / RC, cc = e % RC;
        if (a > b && a < nbk) ys[a][cc] = cfms(ys[a][cc], Ld[a][b], ys[b][cc]);
      }
      __syncthreads();
    }
    for (int e = tid; e < nbk * RC; e += 256) {
      int a = e / RC, cc = e % RC;
      if (cc < nc) Yf[(int64_t)(kb0 + a) * r + c0 + cc] = ys[a][cc];
    }
    // pivot rows below the block (the update rows are done by the L21 GEMM, k_cgemm)
    for (int i = kb0 + nbk + tid; i < p; i += 256) {
      cx<T> acc[RC];
#pragma unroll
      for (int cc = 0; cc < RC; ++cc) acc[cc] = mk<T>(0, 0);
      const cx<T> *Li = F + i + (int64_t)kb0 * ld;
      for (int b0 = 0; b0 < nbk; b0 += 8) {
        cx<T> l[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) l[u] = b0 + u < nbk ? Li[(int64_t)(b0 + u) * ld] : mk<T>(0, 0);
#pragma unroll
        for (int u = 0; u < 8; ++u)
#pragma unroll
          for (int cc = 0; cc < RC; ++cc) acc[cc] = cfma(acc[cc], l[u], ys[min(b0 + u, 31)][cc]);
      }
      cx<T> *yi = Yf + (int64_t)i * r + c0;
#pragma unroll
      for (int cc = 0; cc < RC; ++cc)
        if (cc < nc) {
          cx<T> v = yi[cc];
          v.re -= acc[cc].re;
          v.im -= acc[cc].im;
          yi[cc] = v;
        }
    }
    __syncthreads();
  }
  // z = D^{-1} y (block diagonal), pivot order
  const double2 *di = dinv_d + ft.piv[f];
  const double2 *dof = dinv_o + ft.piv[f];
  const int64_t st = ft.start[f];
  for (int e = tid; e < p * RC; e += 256) {
    int k = e / RC, cc = e % RC;
    if (cc >= nc) continue;
    double2 y = to_d(Yf[(int64_t)k * r + c0 + cc]);
    double2 z = zmul(di[k], y);
    int s = ps[k];
    if (s == 2 || s == -2) {
      int o = s == 2 ? k + 1 : k - 1;
      double2 yo = to_d(Yf[(int64_t)o * r + c0 + cc]);
      double2 t2 = zmul(dof[k], yo);
      z.x += t2.x;
      z.y += t2.y;
    }
    zM[(st + k) * r + c0 + cc] = from_d<T>(z);
  }
}

// Backward substitution with L11^T on the pivot rows, right-looking: start
// from w = z - sum_s part_s (the split partial products L21^T x_upd of
// the L21^T GEMM, k_cgemm), then for each 32-block from the last: solve the diagonal
// block, publish x, and subtract L[blk, k]^T x_blk from every earlier pivot
// row k.  x is written to xM at the original (un-permuted) positions.
template <typename T, int RC>
__global__ void __launch_bounds__(256) k_bwd_solve(const int32_t *__restrict__ lvl, FrontTab ft,
                                                   const cx<T> *__restrict__ arena,
                                                   const int32_t *__restrict__ perm,
                                                   const int8_t *__restrict__ psize,
                                                   const int32_t *__restrict__ nsplit,
                                                   const int64_t *__restrict__ part_off,
                                                   const cx<T> *__restrict__ part, cx<T> *__restrict__ Y,
                                                   const cx<T> *__restrict__ zM, cx<T> *__restrict__ xM, int r) {
  pdl_wait();  // the predecessor in the sweep has finished
  pdl_trigger();
  const int f = lvl[blockIdx.y];
  const int m = ft.m[f], p = ft.p[f];
  (void)m;
  const int c0 = blockIdx.x * RC;
  const int nc = min(RC, r - c0);
  const cx<T> *F = arena + ft.off[f];
  const int64_t ld = ft.m[f];
  cx<T> *Yf = Y + ft.yoff[f] * r;
  const int8_t *ps = psize + ft.piv[f];
  const int32_t *pv = perm + ft.piv[f];
  const int64_t st = ft.start[f];
  const int tid = threadIdx.x;
  const int S = nsplit[blockIdx.y];
  const cx<T> *pt = part + part_off[blockIdx.y] * r;
  for (int e = tid; e < p * RC; e += 256) {
    int k = e / RC, cc = e % RC;
    if (cc >= nc) continue;
    cx<T> w = zM[(st + k) * r + c0 + cc];
    for (int q = 0; q < S; ++q) {
      cx<T> u = pt[((int64_t)q * p + k) * r + c0 + cc];
      w.re -= u.re;
      w.im -= u.im;
    }
    Yf[(int64_t)k * r + c0 + cc] = w;
  }
  __syncthreads();
  __shared__ cx<T> Ls[32][33];
  __shared__ cx<T> v[32][RC];
  const int last = ((p - 1) / 32) * 32;
  const int b = tid / RC, cc = tid % RC;  // 32 x RC threads own (pivot, rhs)
  for (int kb0 = last; kb0 >= 0; kb0 -= 32) {
    const int nbk = min(32, p - kb0);
    if (b < 32) v[b][cc] = (b < nbk && cc < nc) ? Yf[(int64_t)(kb0 + b) * r + c0 + cc] : mk<T>(0, 0);
    for (int e = tid; e < 32 * 32; e += 256) {
      int a = e % 32, col = e / 32;
      cx<T> val = mk<T>(0, 0);
      if (a < nbk && col < nbk && a > col) {
        val = F[kb0 + a + (int64_t)(kb0 + col) * ld];
        if (a == col + 1 && ps[kb0 + col] == 2) val = mk<T>(0, 0);
      }
      Ls[a][col] = val;
    }
    __syncthreads();
    for (int a = nbk - 1; a > 0; --a) {
      if (b < a && cc < nc) v[b][cc] = cfms(v[b][cc], Ls[a][b], v[a][cc]);
      __syncthreads();
    }
    if (b < nbk && cc < nc) {
      Yf[(int64_t)(kb0 + b) * r + c0 + cc] = v[b][cc];
      xM[(st + pv[kb0 + b]) * r + c0 + cc] = v[b][cc];
    }
    // earlier pivot rows: w[k] -= sum_b L[kb0+b, k] x[kb0+b]
    for (int k = tid; k < kb0; k += 256) {
      cx<T> acc[RC];
#pragma unroll
      for (int q = 0; q < RC; ++q) acc[q] = mk<T>(0, 0);
      const cx<T> *Lk = F + kb0 + (int64_t)k * ld;
      for (int b0 = 0; b0 < nbk; b0 += 8) {
        cx<T> l[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) l[u] = b0 + u < nbk ? Lk[b0 + u] : mk<T>(0, 0);
#pragma unroll
        for (int u = 0; u < 8; ++u)
#pragma unroll
          for (int q = 0; q < RC; ++q) acc[q] = cfma(acc[q], l[u], v[min(b0 + u, 31)][q]);
      }
      cx<T> *yk = Yf + (int64_t)k * r + c0;
#pragma unroll
      for (int q = 0; q < RC; ++q)
        if (q < nc) {
          cx<T> t = yk[q];
          t.re -= acc[q].re;
          t.im -= acc[q].im;
          yk[q] = t;
        }
    }
    __syncthreads();
  }
}

// Backward update rows are split into blocks of BSPLIT rows; each block's
// partial sums L21^T x (per pivot) are added up by k_bwd_solve / k_bwd_w.
constexpr int BSPLIT = 256;

// ------------------------------------------------------------ batched complex GEMM
// C = alpha op(A) B (+ C) over a list of items (all fronts of a level), one
// CTA per BM x 64 output tile (BM = 32, 64 or 128, chosen per launch: small
// tiles for the levels with few fronts): 256 threads with (BM/16) x 4 complex
// accumulators each, K in chunks of 16 staged through shared memory, the next
// chunk loaded into registers while the current one is multiplied.  Operands
// are addressed by (row stride, column stride) into one of six buffers; B's
// rows may be gathered through an index list (gath >= 0).  The fast thread
// index runs along A's and C's contiguous dimension, so loads and stores
// coalesce for column- and row-major operands alike.  Triangular operands
// (stored with explicit zeros) bound the k range of a tile: mode 1 A lower
// (k <= i), 2 B lower (k >= j), 3 A upper (k >= i).
// koff: the item's first k in the full product (split-K pieces of a
// triangular product bound their k range with the global index).
struct CgItem {
  int64_t a, b, c, gath;
  int32_t a_rs, a_cs, b_rs, b_cs, c_rs, c_cs;
  int32_t M, N, K, mode, abuf, bbuf, cbuf, beta;
  float alpha;
  int32_t tile0;
  int32_t koff;
  // tensor-core kernel only: the pre-split block of the item's A operand for
  // row tile 0 and its first k chunk, and the blocks per row tile (k chunks)
  int64_t qa;
  int32_t qnk;
};
template <typename T>
struct CgBufs {
  cx<T> *p[7];
};
constexpr int CG_BN = 64;
// K chunk: 48 for the small fp32 tiles (the launches of the levels with few
// fronts are latency bound, so each round trip carries more of K), else 16
template <typename T, int BM>
__host__ __device__ constexpr int cg_kc() {
  return sizeof(T) == 4 && BM == 32 ? 48 : 16;
}
// Buffer i of a launch's buffer table, read from the kernel parameters by a
// switch (an indexed read would copy the table to local memory first).
template <typename T>
__device__ __forceinline__ cx<T> *cg_buf(const CgBufs<T> &b, int i) {
  switch (i) {
    case 0: return b.p[0];
    case 1: return b.p[1];
    case 2: return b.p[2];
    case 3: return b.p[3];
    case 4: return b.p[4];
    case 5: return b.p[5];
    default: return b.p[6];
  }
}
// The item of output tile t of a launch: one load from the launch's
// tile -> item map when there is one, else a binary search over the items'
// first tiles (a chain of dependent loads, kept for the small launches of
// the factor-time inverse).
__device__ __forceinline__ int cg_item_of(const CgItem *__restrict__ items, int nitems, int t,
                                          const int32_t *__restrict__ tmap) {
  if (tmap) return tmap[t];
  int lo = 0, hi = nitems - 1;  // last item with tile0 <= t
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (items[mid].tile0 <= t) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}
template <typename T, int BM>
__global__ void __launch_bounds__(256, (sizeof(T) == 4 && BM <= 64) ? 2 : 1) k_cgemm(const CgItem *__restrict__ items, int nitems, int ntiles,
                                               CgBufs<T> bufs, const int64_t *__restrict__ gidx,
                                               const int32_t *__restrict__ tmap) {
  constexpr int BN = CG_BN, KC = cg_kc<T, BM>(), RA = BM / 16, RB = BN / 16;
  constexpr int LA = BM * KC / 256, LB = BN * KC / 256;  // staged elements per thread
  const int t = blockIdx.x;
  if (t >= ntiles) return;
  const CgItem it = items[cg_item_of(items, nitems, t, tmap)];  // static tables: before the wait
  pdl_wait();
  pdl_trigger();
  const cx<T> *A = cg_buf(bufs, it.abuf) + it.a;
  const cx<T> *B = cg_buf(bufs, it.bbuf) + it.b;
  cx<T> *C = cg_buf(bufs, it.cbuf) + it.c;
  const int64_t *G = it.gath >= 0 ? gidx + it.gath : nullptr;
  const int ntm = (it.M + BM - 1) / BM;
  const int ti = t - it.tile0, tm = ti % ntm, tn = ti / ntm;
  const int i0 = tm * BM, j0 = tn * BN;
  int klo = 0, khi = it.K;
  if (it.mode == 1) khi = min(it.K, i0 + BM - it.koff);
  if (it.mode == 2) klo = max(0, j0 - it.koff);
  if (it.mode == 3) klo = max(0, i0 - it.koff);
  __shared__ cx<T> As[KC][BM + 1];
  __shared__ cx<T> Bs[KC][BN + 1];
  // thread -> (row, column) of its outputs: rows fast for column-major C
  const bool cfast = it.c_rs == 1;
  const int tr = cfast ? (threadIdx.x & 15) : (threadIdx.x >> 4);
  const int tc = cfast ? (threadIdx.x >> 4) : (threadIdx.x & 15);
  // staging maps: the fast index along each operand's contiguous dimension
  const bool afast = it.a_rs == 1, bfast = it.b_cs == 1;
  cx<T> ra[LA], rb[LB];
  auto load = [&](int k0) {
#pragma unroll
    for (int u = 0; u < LA; ++u) {
      const int e = threadIdx.x + 256 * u;
      const int x = afast ? e % BM : e / KC, kk = afast ? e / BM : e % KC;
      const int i = i0 + x, k = k0 + kk;
      ra[u] = (i < it.M && k < khi) ? A[(int64_t)i * it.a_rs + (int64_t)k * it.a_cs] : mk<T>(0, 0);
    }
#pragma unroll
    for (int u = 0; u < LB; ++u) {
      const int e = threadIdx.x + 256 * u;
      const int x = bfast ? e % BN : e / KC, kk = bfast ? e / BN : e % KC;
      const int j = j0 + x, k = k0 + kk;
      cx<T> v = mk<T>(0, 0);
      if (j < it.N && k < khi) {
        const int64_t kr = G ? G[k] : (int64_t)k;
        v = B[kr * it.b_rs + (int64_t)j * it.b_cs];
      }
      rb[u] = v;
    }
  };
  auto stage = [&]() {
#pragma unroll
    for (int u = 0; u < LA; ++u) {
      const int e = threadIdx.x + 256 * u;
      const int x = afast ? e % BM : e / KC, kk = afast ? e / BM : e % KC;
      As[kk][x] = ra[u];
    }
#pragma unroll
    for (int u = 0; u < LB; ++u) {
      const int e = threadIdx.x + 256 * u;
      const int x = bfast ? e % BN : e / KC, kk = bfast ? e / BN : e % KC;
      Bs[kk][x] = rb[u];
    }
  };
  cx<T> acc[RA][RB];
#pragma unroll
  for (int a = 0; a < RA; ++a)
#pragma unroll
    for (int b = 0; b < RB; ++b) acc[a][b] = mk<T>(0, 0);
  if (klo < khi) load(klo);
  for (int k0 = klo; k0 < khi; k0 += KC) {
    __syncthreads();  // the previous chunk has been read
    stage();
    __syncthreads();
    if (k0 + KC < khi) load(k0 + KC);  // in flight during the multiply
#pragma unroll 4
    for (int kk = 0; kk < KC; ++kk) {
      cx<T> av[RA], bv[RB];
#pragma unroll
      for (int a = 0; a < RA; ++a) av[a] = As[kk][tr + 16 * a];
#pragma unroll
      for (int b = 0; b < RB; ++b) bv[b] = Bs[kk][tc + 16 * b];
#pragma unroll
      for (int a = 0; a < RA; ++a)
#pragma unroll
        for (int b = 0; b < RB; ++b) acc[a][b] = cfma(acc[a][b], av[a], bv[b]);
    }
  }
  const T al = (T)it.alpha;
  // beta: the old values are loaded before the stores (the stores could alias
  // later loads, so the compiler would otherwise serialise every element):
  // all of them at once in fp32; one tile row (RB values) at a time in fp64,
  // whose wider accumulators leave no registers for all of them
  constexpr int GA = sizeof(T) == 4 ? RA : 1;
#pragma unroll
  for (int a0 = 0; a0 < RA; a0 += GA) {
#pragma unroll
    for (int a = a0; a < a0 + GA; ++a)
#pragma unroll
      for (int b = 0; b < RB; ++b) {
        const int i = i0 + tr + 16 * a, j = j0 + tc + 16 * b;
        acc[a][b] = mk<T>(al * acc[a][b].re, al * acc[a][b].im);
        if (it.beta && i < it.M && j < it.N) {
          const cx<T> o = C[(int64_t)i * it.c_rs + (int64_t)j * it.c_cs];
          acc[a][b].re += o.re;
          acc[a][b].im += o.im;
        }
      }
#pragma unroll
    for (int a = a0; a < a0 + GA; ++a) {
      const int i = i0 + tr + 16 * a;
      if (i >= it.M) continue;
#pragma unroll
      for (int b = 0; b < RB; ++b) {
        const int j = j0 + tc + 16 * b;
        if (j >= it.N) continue;
        C[(int64_t)i * it.c_rs + (int64_t)j * it.c_cs] = acc[a][b];
      }
    }
  }
}

#include "tc_solve.cuh"

// bm: the row tile of the FMA kernel (32, 64 or 128), or 0 for the tensor-core
// kernel (128 x 64 tiles, complex64 operands only); qpl / err / wait_cap are
// that kernel's pre-split A blocks, error flag and first-wait bound; tmap, if
// given, maps each output tile to its item (index relative to `items`);
// pdl: launched as a programmatic dependent of the stream's previous kernel.
template <typename T>
static void launch_cgemm(int bm, int ntiles, const CgItem *items, int nitems, const CgBufs<T> &bufs,
                         const int64_t *gidx, cudaStream_t s, const uint16_t *qpl = nullptr,
                         int32_t *err = nullptr, int wait_cap = 0, const int32_t *tmap = nullptr,
                         bool pdl = false) {
  if constexpr (sizeof(T) == 4) {
    if (bm == 0) {
      if (pdl)
        launch_pdl(true, k_tc_cgemm, dim3(ntiles), dim3(Q_THREADS), Q_SMEM, s, items, nitems, ntiles, bufs, gidx, tmap, qpl,
                   err, wait_cap);
      else
        k_tc_cgemm<<<ntiles, Q_THREADS, Q_SMEM, s>>>(items, nitems, ntiles, bufs, gidx, tmap, qpl, err, wait_cap);
      return;
    }
  }
  void (*k)(const CgItem *, int, int, CgBufs<T>, const int64_t *, const int32_t *) =
      bm == 32 ? k_cgemm<T, 32> : (bm == 64 || sizeof(T) == 8) ? k_cgemm<T, 64> : k_cgemm<T, (sizeof(T) == 4 ? 128 : 64)>;
  if (pdl)
    launch_pdl(true, k, dim3(ntiles), dim3(256), 0, s, items, nitems, ntiles, bufs, gidx, tmap);
  else
    k<<<ntiles, 256, 0, s>>>(items, nitems, ntiles, bufs, gidx, tmap);
}

// Split-K: a product whose launch has few output tiles and a long k range is
// cut into S pieces along k, each written (scaled by alpha, beta = 0) to its
// own M x N block of a partial buffer (row-major, RHS fastest); this item
// list then adds them to the target in a fixed order (deterministic).
struct SkItem {
  int64_t c, p;        // target offset in buffer cbuf; first partial block in the partial buffer
  int32_t c_rs, c_cs, M, N, S, cbuf, beta;
  int32_t elem0;       // first element index of this item in the launch
  int32_t f;           // front of the item (its rows are the front's pivot rows for kinds 0 and 3)
};
template <typename T>
__global__ void k_splitk_reduce(const SkItem *__restrict__ items, int nitems, int64_t nelem, CgBufs<T> bufs,
                                const cx<T> *__restrict__ part) {
  pdl_wait();  // the predecessor in the sweep has finished
  pdl_trigger();
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nelem; e += (int64_t)gridDim.x * blockDim.x) {
    int lo = 0, hi = nitems - 1;  // last item with elem0 <= e
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (items[mid].elem0 <= e) lo = mid;
      else hi = mid - 1;
    }
    const SkItem it = items[lo];
    const int64_t q = e - it.elem0;
    const int i = (int)(q / it.N), j = (int)(q % it.N);
    const int64_t mn = (int64_t)it.M * it.N;
    cx<T> acc = mk<T>(0, 0);
    for (int s2 = 0; s2 < it.S; ++s2) {
      const cx<T> v = part[it.p + s2 * mn + q];
      acc.re += v.re;
      acc.im += v.im;
    }
    cx<T> *d = cg_buf(bufs, it.cbuf) + it.c + (int64_t)i * it.c_rs + (int64_t)j * it.c_cs;
    if (it.beta) {
      const cx<T> o = *d;
      acc.re += o.re;
      acc.im += o.im;
    }
    *d = acc;
  }
}

// The split-K reduction of a level's L11^{-1} product fused with the next
// sweep step (levels whose products are split, the narrow ones near the
// root): mode 0 (forward) writes y = L11^{-1} b to Y2 and z = D^{-1} y to
// zM, summing the partials of a 2x2 pivot's partner row as well (the same
// operations in the same order as the reduction followed by k_fwd_dinv);
// mode 3 (backward) writes x = L11^{-T} w straight to its original
// positions in xM (the reduction followed by k_bwd_out).  Kind-0 and kind-3
// items have beta = 0 and row-major targets.
template <typename T>
__global__ void k_splitk_reduce_sweep(const SkItem *__restrict__ items, int nitems, int64_t nelem, CgBufs<T> bufs,
                                      const cx<T> *__restrict__ part, FrontTab ft, const double2 *__restrict__ dinv_d,
                                      const double2 *__restrict__ dinv_o, const int8_t *__restrict__ psize,
                                      const int32_t *__restrict__ perm, cx<T> *__restrict__ zM, cx<T> *__restrict__ xM,
                                      int r, int mode) {
  pdl_wait();  // the predecessor in the sweep has finished
  pdl_trigger();
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nelem; e += (int64_t)gridDim.x * blockDim.x) {
    int lo = 0, hi = nitems - 1;  // last item with elem0 <= e
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (items[mid].elem0 <= e) lo = mid;
      else hi = mid - 1;
    }
    const SkItem it = items[lo];
    const int64_t q = e - it.elem0, mn = (int64_t)it.M * it.N;
    const int i = (int)(q / it.N), j = (int)(q % it.N);
    auto sum_row = [&](int row) {
      cx<T> acc = mk<T>(0, 0);
      for (int s2 = 0; s2 < it.S; ++s2) {
        const cx<T> v = part[it.p + s2 * mn + (int64_t)row * it.N + j];
        acc.re += v.re;
        acc.im += v.im;
      }
      return acc;
    };
    const cx<T> y = sum_row(i);
    const int64_t piv = ft.piv[it.f], st = ft.start[it.f];
    if (mode == 0) {
      cg_buf(bufs, it.cbuf)[it.c + (int64_t)i * it.c_rs + (int64_t)j * it.c_cs] = y;
      cx<T> z = cmul(y, from_d<T>(dinv_d[piv + i]));
      const int sz = psize[piv + i];
      if (sz == 2 || sz == -2) z = cfma(z, sum_row(sz == 2 ? i + 1 : i - 1), from_d<T>(dinv_o[piv + i]));
      zM[(st + i) * r + j] = z;
    } else {
      xM[(st + perm[piv + i]) * r + j] = y;
    }
  }
}

// Inverse of each 32x32 unit-lower diagonal block of L11 (2x2 couplings are
// zero in L), written to the front's L11^{-1} (p x p, column-major, zeros
// above the diagonal).  One CTA per (front, block); thread j builds column j.
template <typename T>
__global__ void __launch_bounds__(32) k_trinv_diag(const int32_t *__restrict__ lvl, FrontTab ft,
                                                   const cx<T> *__restrict__ arena, const int64_t *__restrict__ loff,
                                                   cx<T> *__restrict__ Linv) {
  const int f = lvl[blockIdx.y];
  const int p = ft.p[f], m = ft.m[f];
  const int b0 = blockIdx.x * 32;
  if (b0 >= p) return;
  const int nb = min(32, p - b0);
  const cx<T> *F = arena + ft.off[f];
  cx<T> *X = Linv + loff[blockIdx.y];
  __shared__ cx<T> Ls[32][33];
  __shared__ cx<T> Xs[32][33];
  const int jj = threadIdx.x;
  for (int a = 0; a < 32; ++a)
    Ls[a][jj] = (a < nb && jj < nb && a > jj) ? F[b0 + a + (int64_t)(b0 + jj) * m] : mk<T>(0, 0);
  __syncthreads();
  // column jj: X[jj][jj] = 1, X[i][jj] = -sum_{k=jj}^{i-1} L[i][k] X[k][jj]
  for (int a = 0; a < 32; ++a) Xs[a][jj] = a == jj ? mk<T>(1, 0) : mk<T>(0, 0);
  for (int i = jj + 1; i < nb; ++i) {
    cx<T> acc = mk<T>(0, 0);
    for (int k = jj; k < i; ++k) acc = cfma(acc, Ls[i][k], Xs[k][jj]);
    Xs[i][jj] = mk<T>(-acc.re, -acc.im);
  }
  __syncthreads();
  for (int a = 0; a < nb; ++a)
    if (jj < nb) X[b0 + a + (int64_t)(b0 + jj) * p] = Xs[a][jj];
}

// z = D^{-1} y for the pivot rows (y in Y2, pivot order) -> zM
template <typename T>
__global__ void k_fwd_dinv(const int32_t *__restrict__ lvl, FrontTab ft, const double2 *__restrict__ dinv_d,
                           const double2 *__restrict__ dinv_o, const int8_t *__restrict__ psize,
                           const cx<T> *__restrict__ Y2, cx<T> *__restrict__ zM, int r) {
  pdl_wait();  // the predecessor in the sweep has finished
  pdl_trigger();
  const int f = lvl[blockIdx.y];
  const int p = ft.p[f];
  const cx<T> *Yf = Y2 + ft.yoff[f] * r;
  const double2 *di = dinv_d + ft.piv[f];
  const double2 *dof = dinv_o + ft.piv[f];
  const int8_t *ps = psize + ft.piv[f];
  const int64_t st = ft.start[f];
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)p * r;
       e += (int64_t)gridDim.x * blockDim.x) {
    int k = (int)(e / r), c = (int)(e % r);
    cx<T> z = cmul(Yf[(int64_t)k * r + c], from_d<T>(di[k]));
    int sz = ps[k];
    if (sz == 2 || sz == -2) {
      int o = sz == 2 ? k + 1 : k - 1;
      z = cfma(z, Yf[(int64_t)o * r + c], from_d<T>(dof[k]));
    }
    zM[(st + k) * r + c] = z;
  }
}

// w = z - sum_s part_s into Yf[0:p] (pivot order)
template <typename T>
__global__ void k_bwd_w(const int32_t *__restrict__ lvl, FrontTab ft, const int32_t *__restrict__ nsplit,
                        const int64_t *__restrict__ part_off, const cx<T> *__restrict__ part,
                        const cx<T> *__restrict__ zM, cx<T> *__restrict__ Y, int r) {
  pdl_wait();  // the predecessor in the sweep has finished
  pdl_trigger();
  const int f = lvl[blockIdx.y];
  const int p = ft.p[f];
  cx<T> *Yf = Y + ft.yoff[f] * r;
  const int S = nsplit[blockIdx.y];
  const cx<T> *pt = part + part_off[blockIdx.y] * r;
  const int64_t st = ft.start[f];
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)p * r;
       e += (int64_t)gridDim.x * blockDim.x) {
    int k = (int)(e / r), c = (int)(e % r);
    cx<T> w = zM[(st + k) * r + c];
    for (int q = 0; q < S; ++q) {
      cx<T> u = pt[((int64_t)q * p + k) * r + c];
      w.re -= u.re;
      w.im -= u.im;
    }
    Yf[(int64_t)k * r + c] = w;
  }
}

// x (pivot order, in Y2) -> xM at the original positions
template <typename T>
__global__ void k_bwd_out(const int32_t *__restrict__ lvl, FrontTab ft, const int32_t *__restrict__ perm,
                          const cx<T> *__restrict__ Y2, cx<T> *__restrict__ xM, int r) {
  pdl_wait();  // the predecessor in the sweep has finished
  pdl_trigger();
  const int f = lvl[blockIdx.y];
  const int p = ft.p[f];
  const cx<T> *Yf = Y2 + ft.yoff[f] * r;
  const int32_t *pv = perm + ft.piv[f];
  const int64_t st = ft.start[f];
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)p * r;
       e += (int64_t)gridDim.x * blockDim.x) {
    int k = (int)(e / r), c = (int)(e % r);
    xM[(st + pv[k]) * r + c] = Yf[(int64_t)k * r + c];
  }
}

// ------------------------------------------------------------ edge-space kernels
// column-major user block -> row-major edge vector (conjugated for the adjoint)
__global__ void k_cm_to_rm(const double2 *__restrict__ in, int64_t ld, double2 *__restrict__ out, int64_t n,
                           int r, int conj) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * r; e += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = e / r;
    int c = (int)(e % r);
    double2 v = in[i + ld * c];
    if (conj) v.y = -v.y;
    out[e] = v;
  }
}
__global__ void k_rm_to_cm(const double2 *__restrict__ in, double2 *__restrict__ out, int64_t ld, int64_t n,
                           int r, const uint8_t *__restrict__ pec, int conj) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * r; e += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = e / r;
    int c = (int)(e % r);
    double2 v = pec[i] ? make_double2(0.0, 0.0) : in[e];
    if (conj) v.y = -v.y;
    out[i + ld * c] = v;
  }
}

// grad[c] = k^2 Re( sum_r conj(y)_c^T M_e x_c ), one thread per cell, fp64
struct ElemMass {
  double M[12][12];
};
__global__ void k_grad_eps(int nx, int ny, int nz, double k2, ElemMass Me, const double2 *__restrict__ x, int64_t ldx,
                           const double2 *__restrict__ y, int64_t ldy, int r, const uint8_t *__restrict__ pec,
                           double *__restrict__ grad) {
  const int64_t ncell = (int64_t)nx * ny * nz;
  const int64_t nex = (int64_t)nx * (ny + 1) * (nz + 1), ney = (int64_t)(nx + 1) * ny * (nz + 1);
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < ncell; c += (int64_t)gridDim.x * blockDim.x) {
    int ci = (int)(c % nx), cj = (int)((c / nx) % ny), ck = (int)(c / ((int64_t)nx * ny));
    int64_t e[12];
    for (int q = 0; q < 4; ++q) {
      int a = q & 1, b = q >> 1;
      e[q] = (ci) + (int64_t)nx * ((cj + a) + (int64_t)(ny + 1) * (ck + b));
      e[4 + q] = nex + (ci + a) + (int64_t)(nx + 1) * (cj + (int64_t)ny * (ck + b));
      e[8 + q] = nex + ney + (ci + a) + (int64_t)(nx + 1) * ((cj + b) + (int64_t)(ny + 1) * ck);
    }
    double acc = 0.0;
    for (int rr = 0; rr < r; ++rr) {
      double2 xv[12], yv[12];
      for (int a = 0; a < 12; ++a) {
        bool z = pec[e[a]] != 0;
        xv[a] = z ? make_double2(0, 0) : x[e[a] + ldx * rr];
        yv[a] = z ? make_double2(0, 0) : y[e[a] + ldy * rr];
      }
      for (int a = 0; a < 12; ++a) {
        double2 mx = make_double2(0, 0);
        for (int b = 0; b < 12; ++b) {
          mx.x += Me.M[a][b] * xv[b].x;
          mx.y += Me.M[a][b] * xv[b].y;
        }
        acc += yv[a].x * mx.x + yv[a].y * mx.y;  // Re(conj(y) * mx)
      }
    }
    grad[c] = k2 * acc;
  }
}
// The same gradient with per-cell dof lists and mass matrices (ne <=
// MAX_CELL_NE dofs per cell, checked on the host: 19 for the six Whitney
// tetrahedra of a lattice cell, 6, 12 or 20 for a tetrahedron of a general
// mesh of order 1, 2 or 3, its orientation signs inside the mass).
__global__ void k_grad_eps_cells(int64_t ncell, int ne, const int64_t *__restrict__ cell_edge,
                                 const double *__restrict__ cell_mass, double k2, const double2 *__restrict__ x,
                                 int64_t ldx, const double2 *__restrict__ y, int64_t ldy, int r,
                                 const uint8_t *__restrict__ pec, double *__restrict__ grad) {
  constexpr int NE = MAX_CELL_NE;
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < ncell; c += (int64_t)gridDim.x * blockDim.x) {
    const int64_t *e = cell_edge + c * ne;
    const double *Mc = cell_mass + c * ne * ne;
    double acc = 0.0;
    for (int rr = 0; rr < r; ++rr) {
      double2 xv[NE], yv[NE];
      for (int a = 0; a < ne; ++a) {
        bool z = pec[e[a]] != 0;
        xv[a] = z ? make_double2(0, 0) : x[e[a] + ldx * rr];
        yv[a] = z ? make_double2(0, 0) : y[e[a] + ldy * rr];
      }
      for (int a = 0; a < ne; ++a) {
        double2 mx = make_double2(0, 0);
        for (int b = 0; b < ne; ++b) {
          mx.x += Mc[a * ne + b] * xv[b].x;
          mx.y += Mc[a * ne + b] * xv[b].y;
        }
        acc += yv[a].x * mx.x + yv[a].y * mx.y;  // Re(conj(y) * mx)
      }
    }
    grad[c] = k2 * acc;
  }
}
template <typename T>
__global__ void k_scatter(const double2 *__restrict__ fe, const int64_t *__restrict__ owner, cx<T> *__restrict__ bM,
                          int64_t n, int r) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * r; e += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = e / r;
    int c = (int)(e % r);
    int64_t v = owner[i];
    if (v >= 0) bM[v * r + c] = from_d<T>(fe[e]);
  }
}
// x_e (+)= xM[owner]
template <typename T>
__global__ void k_gather(const cx<T> *__restrict__ xM, const int64_t *__restrict__ owner, double2 *__restrict__ xe,
                         int64_t n, int r, int accumulate) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * r; e += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = e / r;
    int c = (int)(e % r);
    int64_t v = owner[i];
    double2 val = v >= 0 ? to_d(xM[v * r + c]) : make_double2(0.0, 0.0);
    if (accumulate) {
      double2 o = xe[e];
      val.x += o.x;
      val.y += o.y;
    }
    xe[e] = val;
  }
}
template <typename T>
__global__ void k_lambda_acc(const cx<T> *__restrict__ xM, int64_t lam0, int64_t nlm, int r, double2 *__restrict__ lam,
                             int accumulate) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nlm * r; e += (int64_t)gridDim.x * blockDim.x) {
    double2 v = to_d(xM[lam0 * r + e]);
    if (accumulate) {
      v.x += lam[e].x;
      v.y += lam[e].y;
    }
    lam[e] = v;
  }
}

__device__ __forceinline__ void atomic_max_pos(double *addr, double v) {
  // non-negative doubles order like their bit patterns
  atomicMax(reinterpret_cast<unsigned long long *>(addr), (unsigned long long)__double_as_longlong(v));
}

// r = f - A x (fp64) with per-column max |r|^2 (and max |f|^2 when fnorm is
// given); one warp per row, lanes over the right-hand sides, a bounded grid of
// CTAs looping over the rows.  The maxima are reduced per CTA in shared memory
// (2 r doubles of dynamic shared memory when smem_max != 0) and leave with
// one atomic per column and CTA.
__global__ void __launch_bounds__(256)
    k_residual(int64_t n, const int64_t *__restrict__ ptr, const int32_t *__restrict__ col,
               const double *__restrict__ vre, const int64_t *__restrict__ iptr, const int32_t *__restrict__ icol,
               const double *__restrict__ vim, const double2 *__restrict__ x, const double2 *__restrict__ f,
               double2 *__restrict__ res, int r, double *__restrict__ rnorm, double *__restrict__ fnorm,
               int smem_max) {
  extern __shared__ double s_nrm[];  // [2][r]
  if (smem_max)
    for (int c = threadIdx.x; c < 2 * r; c += blockDim.x) s_nrm[c] = 0.0;
  __syncthreads();
  double *rmax = smem_max ? s_nrm : rnorm;
  double *fmax_ = smem_max ? s_nrm + r : fnorm;
  const int lane = threadIdx.x & 31;
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t row = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); row < n; row += nw) {
    const int64_t a = ptr[row], b = ptr[row + 1];
    if (a == b) {  // removed (PEC) edge: no equation, r = f
      for (int c = lane; c < r; c += 32) res[row * r + c] = f[row * r + c];
      continue;
    }
    for (int c = lane; c < r; c += 32) {
      const double2 fv = f[row * r + c];
      double2 acc = fv;
      for (int64_t q = a; q < b; ++q) {  // real part
        const double av = vre[q];
        const double2 xv = x[(int64_t)col[q] * r + c];
        acc.x -= av * xv.x;
        acc.y -= av * xv.y;
      }
      for (int64_t q = iptr[row]; q < iptr[row + 1]; ++q) {  // j * imaginary part
        const double av = vim[q];
        const double2 xv = x[(int64_t)icol[q] * r + c];
        acc.x += av * xv.y;
        acc.y -= av * xv.x;
      }
      res[row * r + c] = acc;
      atomic_max_pos(rmax + c, acc.x * acc.x + acc.y * acc.y);
      if (fnorm) atomic_max_pos(fmax_ + c, fv.x * fv.x + fv.y * fv.y);
    }
  }
  if (smem_max) {
    __syncthreads();
    for (int c = threadIdx.x; c < r; c += blockDim.x) {
      if (s_nrm[c] > 0.0) atomic_max_pos(rnorm + c, s_nrm[c]);
      if (fnorm && s_nrm[r + c] > 0.0) atomic_max_pos(fnorm + c, s_nrm[r + c]);
    }
  }
}

// ------------------------------------------------------------ profiling
// CUDA events around each launch group, on the launching stream; durations
// are summed per kernel class after the stream is synchronised.
enum ProfClass { PC_ASSEMBLE = 0, PC_PANEL, PC_UPDATE, PC_FWD, PC_BWD, PC_RESID, PC_INV, PC_TC, PC_N };
struct Profiler {
  bool on = false;
  cudaStream_t s = nullptr;
  std::vector<cudaEvent_t> pool;
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> marks;
  std::vector<int> mark_level;
  int cur_level = -1;
  size_t used = 0;
  cudaEvent_t get() {
    if (used == pool.size()) {
      cudaEvent_t e;
      cudaEventCreate(&e);
      pool.push_back(e);
    }
    return pool[used++];
  }
  void begin(int cls, cudaEvent_t &e0, cudaStream_t st = nullptr) {
    if (!on) return;
    e0 = get();
    cudaEventRecord(e0, st ? st : s);
    (void)cls;
  }
  void end(int cls, cudaEvent_t e0, cudaStream_t st = nullptr) {
    if (!on) return;
    cudaEvent_t e1 = get();
    cudaEventRecord(e1, st ? st : s);
    marks.push_back({cls, {e0, e1}});
    mark_level.push_back(cur_level);
  }
  void reset() {
    marks.clear();
    mark_level.clear();
    used = 0;
  }
  // per-level sums of one class (after the stream has been synchronised)
  std::vector<double> per_level(int cls, int nlev) {
    std::vector<double> v(nlev, 0.0);
    for (size_t q = 0; q < marks.size(); ++q) {
      if (marks[q].first != cls || mark_level[q] < 0) continue;
      float t = 0;
      cudaEventElapsedTime(&t, marks[q].second.first, marks[q].second.second);
      v[mark_level[q]] += t;
    }
    return v;
  }
  void collect(double ms[PC_N]) {
    for (int q = 0; q < PC_N; ++q) ms[q] = 0;
    for (auto &mk : marks) {
      float t = 0;
      cudaEventElapsedTime(&t, mk.second.first, mk.second.second);
      ms[mk.first] += t;
    }
    reset();
  }
  ~Profiler() {
    for (auto e : pool) cudaEventDestroy(e);
  }
};
#define PROF_BEGIN(cls)   \
  cudaEvent_t pe_##cls{}; \
  d->prof.begin(cls, pe_##cls)
#define PROF_END(cls) d->prof.end(cls, pe_##cls)
#define PROF_BEGIN_ON(cls, st) \
  cudaEvent_t pb_##cls{};      \
  d->prof.begin(cls, pb_##cls, st)
#define PROF_END_ON(cls, st) d->prof.end(cls, pb_##cls, st)

// ------------------------------------------------------------ device state
struct DeviceState {
  Profiler prof;
  int64_t inv_launches = 0;
  double *flop_cnt = nullptr;  // [0] trailing-update flops, [1] panel flops
  int64_t launches = 0;
  double solve_flops_per_rhs = 0;
  int precision = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;       // created here when the caller passed the legacy NULL stream
  cudaEvent_t legacy_ev = nullptr;
  // look-ahead: the Schur-complement part of each trailing update runs on a
  // second, low-priority stream while the next panels proceed on the first;
  // W and the per-step (k0 + kb, kb) snapshots rotate through three slots
  cudaStream_t stream_b = nullptr;
  cudaEvent_t ev_step[3] = {}, ev_schur[3] = {}, ev_b = nullptr;
  // the mixed path's L11^{-1} of a finished level runs on a third stream while
  // the next level proceeds (it reads only the level's pivot blocks)
  cudaStream_t stream_c = nullptr;
  cudaEvent_t ev_lvl = nullptr, ev_c = nullptr;
  int2 *snap = nullptr;          // [3][level position]
  int64_t wslot = 0;             // elements per W slot
  bool lookahead_off = false;    // set while the autotuner times the kernels
  int prio_lo = 0, prio_hi = 0;  // least / most urgent scheduling priority
  // plan tables
  int32_t *f_m = nullptr, *f_p = nullptr, *f_parent = nullptr;
  int64_t *f_off = nullptr, *f_piv = nullptr, *f_soff = nullptr, *f_start = nullptr, *f_y = nullptr;
  int32_t *lvl_fronts = nullptr, *ea_child = nullptr, *emap = nullptr;
  int64_t *g_ptr = nullptr, *g_src = nullptr;  // forward gather: parent row -> child Y rows (CSR)
  int64_t *sidx = nullptr, *ent_off = nullptr, *wofs = nullptr, *owner = nullptr;
  double2 *ent_val = nullptr;
  // factors
  void *arena = nullptr;
  int32_t *perm = nullptr, *iperm = nullptr;
  double2 *dinv_d = nullptr, *dinv_o = nullptr;
  int8_t *psize = nullptr;
  int32_t *st_k0 = nullptr, *st_kb = nullptr, *st_info = nullptr;
  double *st_minpiv = nullptr;
  void *W = nullptr;
  // operator for residuals
  int64_t *csr_ptr = nullptr;  // A = Ar + j Ai: Ar on the full pattern,
  int32_t *csr_col = nullptr;  // Ai (absorbing faces, lossy cells) on its own
  double *csr_re = nullptr;
  int64_t *csi_ptr = nullptr;
  int32_t *csi_col = nullptr;
  double *csi_val = nullptr;
  uint8_t *pec = nullptr;
  int64_t *gc_edge = nullptr;  // tetrahedral meshes: per cell its 19 edges and
  double *gc_mass = nullptr;   // 19 x 19 mass matrix (uploaded by the first gradient)
  // solve buffers (capacity in RHS)
  int cap = 0;
  void *bM = nullptr, *zM = nullptr, *xM = nullptr, *Y = nullptr;
  double2 *fe = nullptr, *xe = nullptr, *re = nullptr, *ucm = nullptr, *lam = nullptr;
  double *norms = nullptr;
  // host launch data
  std::vector<int64_t> w_level_base;  // per level: index of first front in wofs (== level_ptr)
  std::vector<int> level_steps;
  std::vector<std::vector<int>> update_grid;  // per level, per step: grid.x upper bound
  std::vector<int> ea_grid;                   // per pass: grid.x (tiles) upper bound
  std::vector<int> level_maxm, pass_maxn;
  // explicit L11^{-1} of every front (p x p column-major), built after each level
  void *linv = nullptr;
  int64_t *linv_off = nullptr;                 // per level position
  std::vector<int64_t> linv_off_h;
  void *tmp_inv = nullptr;                     // doubling-stage temporaries
  CgItem *inv_items = nullptr;                 // all factor-time doubling items
  std::vector<std::vector<std::array<int, 4>>> inv_stage;  // per level: (item0, nitems, ntiles, row tile)
  CgItem *sol_items = nullptr;                 // solve GEMM items for sol_r RHS
  // per level, (item0, nitems, ntiles) of: forward L11^{-1}, forward L21,
  // backward L21^T (split partials), backward L11^{-T}
  std::vector<std::array<int, 16>> sol_lvl;  // (item0, nitems, ntiles, row tile) per kind
  int32_t *sol_tmap = nullptr;               // per solve launch: output tile -> item (relative)
  std::vector<std::array<int64_t, 4>> sol_tofs;  // per level and kind: offset in sol_tmap
  std::vector<std::array<int, 12>> sk_lvl;   // per kind: split-K reduce (item0, nitems, elements)
  SkItem *sk_items = nullptr;
  void *skp = nullptr;                       // split-K partial blocks
  int sol_r = 0;
  void *Y2 = nullptr;
  cudaGraphExec_t g_fwd = nullptr, g_bwd = nullptr;  // captured substitution sweeps
  cudaGraphExec_t g_factor = nullptr;                // captured factorisation (unprofiled calls)
  int64_t g_factor_launches = 0;
  int g_r = 0;
  int64_t g_launches[2] = {0, 0};
  int2 *swp = nullptr;           // per level position: the current panel's column permutation (2 NB each)
  int32_t *tc_err = nullptr;     // set by k_tc_gemm when a bounded wait expires
  int32_t *fin_err = nullptr;    // set when a pivot inverse is not finite
  int tc_wait_cap = 1 << 22;     // first-attempt bound of k_tc_gemm's mbarrier waits
  int32_t *sv_err = nullptr;     // set by k_tc_cgemm (substitution products) when a bounded wait expires
  int sv_wait_cap = 1 << 22;     // first-attempt bound of k_tc_cgemm's mbarrier waits
  std::vector<uint8_t> lvl_tc;   // per level: deferred tensor-core products (mixed)
  std::vector<int> lvl_cs;       // per level: panel cluster size (0 = global panel)
  bool tuned = false;
  std::vector<double> tune_panel, tune_update, tune_inv, tune_tc;  // per-level ms of the last profiled factor
  std::vector<std::vector<int>> update_grid_p;  // per level, per step: tiles of the pivot-block update
  std::vector<std::vector<int>> update_grid_r;  // ... of the update rows of the pivot-block columns
  // deferred Schur products of the mixed path on the tensor cores
  // (tc_gemm.cuh), per level: operand-split blocks (L21, W21) and product tiles
  struct TcLevel {
    int kpitch = 0;                 // K pitch of the level's planes (0: nothing to do)
    int64_t rowsA = 0, rowsB = 0;   // plane rows of the A / B operands
    int sx0 = 0, nsx = 0, sl0 = 0, nsl = 0, g20 = 0, ng2 = 0;  // L21 / W21 split blocks, Schur tiles
    double flops = 0;               // algorithmic real flops of the Schur products
    CUtensorMap tmA, tmB;
  };
  std::vector<TcLevel> tcl;
  TcSplit *tc_split = nullptr;
  TcTile *tc_tiles = nullptr;
  int64_t *w21_off = nullptr;     // per level position: the front's W21 block in tc_w
  uint16_t *planesA = nullptr, *planesB = nullptr;  // bf16 operand planes
  // tensor-core substitution: pre-split 48 KB blocks of the A operands
  // (L11^{-1}, L21 and their transposes, per level position and kind 0-3),
  // written after each level is factored (k_tc_presplit)
  uint16_t *qpl = nullptr;
  QPre *qpre = nullptr;
  std::vector<std::array<int64_t, 4>> qblk_h;  // first block of each operand
  std::vector<std::array<int32_t, 4>> qnk_h;   // its k chunks (blocks per row tile)
  std::vector<std::array<int64_t, 2>> qpre_lvl;  // per level: first job, job count
  int64_t qblocks = 0;
  float2 *tc_w = nullptr;         // W21 of every front of a level (fp32 complex)
  std::vector<int> level_maxp;   // largest pivot block per level
  int32_t *nsplit = nullptr;     // per level position: row splits of the backward partials
  std::vector<int64_t> part_off_h;  // per level position: first partial row
  int64_t *part_off = nullptr;   // per level position: partial-buffer offset (units of r)
  int64_t part_rows = 0;         // max over levels of sum(nsplit * p)
  void *part = nullptr;
  // GMRES-IR work space (edge space, fp64): basis V (m + 1 vectors), the
  // preconditioned directions Z (m), their multiplier parts, w, reductions
  int gm_r = 0, gm_m = 0;
  double2 *gm_V = nullptr, *gm_Z = nullptr, *gm_lamZ = nullptr, *gm_w = nullptr, *gm_y = nullptr;
  double *gm_h = nullptr, *gm_s = nullptr;
  std::vector<void *> allocs;
};

template <class X>
static cudaError_t dalloc(DeviceState *d, X **ptr, size_t count) {
  void *p = nullptr;
  cudaError_t e = cudaMalloc(&p, std::max<size_t>(count, 1) * sizeof(X));
  if (e == cudaSuccess) {
    d->allocs.push_back(p);
    *ptr = (X *)p;
  }
  return e;
}
template <class X>
static cudaError_t upload(DeviceState *d, X **ptr, const std::vector<X> &v) {
  cudaError_t e = dalloc(d, ptr, v.size());
  if (e != cudaSuccess) return e;
  if (!v.empty()) e = cudaMemcpy(*ptr, v.data(), v.size() * sizeof(X), cudaMemcpyHostToDevice);
  return e;
}

static FrontTab tab(const DeviceState *d) {
  FrontTab t;
  t.m = d->f_m;
  t.p = d->f_p;
  t.off = d->f_off;
  t.piv = d->f_piv;
  t.soff = d->f_soff;
  t.start = d->f_start;
  t.yoff = d->f_y;
  t.parent = d->f_parent;
  return t;
}

// Row tile (32, 64 or 128) of one batched k_cgemm launch over `items`: the
// fewest efficiency-weighted rows per SM over the waves of CTAs (1 resident
// CTA per SM for 128-row tiles, 2 for the smaller ones); assigns the items'
// first tiles and returns (tiles, row tile).
static std::pair<int, int> cg_assign(std::vector<CgItem> &items, bool allow128) {
  int best = 64;
  double bcost = 1e300;
  for (int bm : {32, 64, 128}) {
    if (bm == 128 && !allow128) continue;
    int64_t t = 0;
    for (const CgItem &g : items) t += (int64_t)((g.M + bm - 1) / bm) * ((g.N + CG_BN - 1) / CG_BN);
    const int occ = bm == 128 ? 1 : 2;
    const double eff = bm == 128 ? 1.0 : bm == 64 ? 0.85 : 0.6;
    const double cost = (double)((t + 152 * occ - 1) / (152 * occ)) * bm / eff;
    if (cost < bcost) {
      bcost = cost;
      best = bm;
    }
  }
  int tiles = 0;
  for (CgItem &g : items) {
    g.tile0 = tiles;
    tiles += ((g.M + best - 1) / best) * ((g.N + CG_BN - 1) / CG_BN);
  }
  return {tiles, best};
}

// ---- deferred tensor-core products: the driver entry point of the tensor-map
// encoder, fetched through the runtime (no link against the driver library)
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
static EncodeTiledFn encode_tiled() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)p;
  }
  return fn;
}
// Tensor map over the six bf16 planes of one operand: dims (k, row, plane),
// 32 x 128 x 1 boxes with 64-byte swizzle (the K-major shared-memory layout
// that k_tc_gemm's descriptors describe).
static bool encode_planes(CUtensorMap *tm, uint16_t *base, int kpitch, int64_t rows) {
  EncodeTiledFn fn = encode_tiled();
  if (!fn) return false;
  const cuuint64_t dims[3] = {(cuuint64_t)kpitch, (cuuint64_t)rows, (cuuint64_t)G_NPL};
  const cuuint64_t strides[2] = {(cuuint64_t)kpitch * 2, (cuuint64_t)rows * kpitch * 2};
  const cuuint32_t box[3] = {(cuuint32_t)G_BK, (cuuint32_t)G_BM, 1};
  const cuuint32_t es[3] = {1, 1, 1};
  return fn(tm, CU_TENSOR_MAP_DATA_TYPE_UINT16, 3, base, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Per level: the fronts with a pivot block and update rows get an A-operand
// block (their Mr = m - p update rows of L21, padded to 128 rows) and a
// B-operand block (W21, same shape) in the plane buffers, a W21 slot (Mr x p,
// written by the update-row solve), the 32 x 32 split blocks of both operands
// and the 128 x 128 tiles of the lower triangle of the Schur product
// C = F22 - L21 W21^T.
// Whether substitution product `kind` (0: L11^{-1} y, 1: L21 y, 2: L21^T x,
// 3: L11^{-T} w) of tree level l runs on the tensor cores: when its fronts'
// operands fill at least 30 % of the padded 128 x 32 blocks they take (the
// bf16x3 kernel then outruns fp32 FMA; the small fronts near the leaves
// stay on FMA, which also spares their mostly-padding operand blocks).
static bool tc_solve_launch(const Plan &P, int l, int kind) {
  double use = 0, pad = 0;
  for (int i = P.level_ptr[l]; i < P.level_ptr[l + 1]; ++i) {
    const int f = P.level_fronts[i];
    const int64_t pf = P.sn_end[f] - P.sn_start[f], uf = P.struct_ptr[f + 1] - P.struct_ptr[f];
    const int64_t M = kind == 1 ? uf : pf, K = kind == 2 ? uf : pf;
    if (M <= 0 || K <= 0) continue;
    use += (double)M * K;
    pad += (double)((M + Q_BM - 1) / Q_BM * Q_BM) * ((K + Q_BK - 1) / Q_BK * Q_BK);
  }
  return pad > 0 && use >= 0.3 * pad;
}

static int tc_plan(Ctx &c, DeviceState *d, const std::vector<int32_t> &m, const std::vector<int32_t> &pp) {
  const Plan &P = c.plan;
  std::vector<TcSplit> sp;
  std::vector<TcTile> tl;
  std::vector<int64_t> w21_off((size_t)P.sn_start.size(), 0);
  d->tcl.assign(P.n_levels, DeviceState::TcLevel{});
  int64_t maxA = 0, maxW = 0;
  auto rup = [](int64_t v, int64_t q) { return (v + q - 1) / q * q; };
  struct Fo {
    int f, i, pf, mf, Mr;
    int64_t row, woff;
  };
  for (int l = 0; l < P.n_levels; ++l) {
    DeviceState::TcLevel &L = d->tcl[l];
    std::vector<Fo> fo;
    int64_t ra = 0, wo = 0;
    int kp = 0;
    for (int i = P.level_ptr[l]; i < P.level_ptr[l + 1]; ++i) {
      const int f = P.level_fronts[i], pf = pp[f], mf = m[f], Mr = mf - pf;
      if (pf == 0 || Mr == 0) continue;
      fo.push_back({f, i, pf, mf, Mr, ra, wo});
      w21_off[i] = wo;
      ra += rup(Mr, G_BM);
      wo += (int64_t)Mr * pf;
      kp = std::max<int>(kp, (int)rup(pf, G_KPAD));
      L.flops += 8.0 * 0.5 * (double)pf * Mr * (Mr + 1.0);
    }
    if (fo.empty()) continue;
    L.kpitch = kp;
    L.rowsA = L.rowsB = ra;
    maxA = std::max(maxA, ra * kp);
    maxW = std::max(maxW, wo);
    L.sx0 = (int)sp.size();
    for (const Fo &q : fo)  // L21: rows p.. of the front's pivot columns (pivot order)
      for (int r0 = 0; r0 < rup(q.Mr, G_BM); r0 += 32)
        for (int k0 = 0; k0 < rup(q.pf, G_KPAD); k0 += 32)
          sp.push_back({q.f, r0, k0, q.Mr, q.pf, (int32_t)q.row, P.front_off[q.f] + q.pf, q.mf, 0});
    L.nsx = (int)sp.size() - L.sx0;
    L.sl0 = (int)sp.size();
    for (const Fo &q : fo)  // W21 = L21 D (column-major Mr x p in the W21 buffer)
      for (int r0 = 0; r0 < rup(q.Mr, G_BM); r0 += 32)
        for (int k0 = 0; k0 < rup(q.pf, G_KPAD); k0 += 32)
          sp.push_back({q.f, r0, k0, q.Mr, q.pf, (int32_t)q.row, q.woff, q.Mr, 0});
    L.nsl = (int)sp.size() - L.sl0;
    L.g20 = (int)tl.size();
    for (const Fo &q : fo)  // C -= L21 W21^T, lower triangle of tiles
      for (int I = 0; I * G_BM < q.Mr; ++I)
        for (int J = 0; J <= I; ++J) {
          TcTile t{};
          t.arow = (int32_t)(q.row + I * G_BM);
          t.brow = (int32_t)(q.row + J * G_BN);
          t.M = std::min(G_BM, q.Mr - I * G_BM);
          t.N = std::min(G_BN, q.Mr - J * G_BN);
          t.nk = (q.pf + G_BK - 1) / G_BK;
          t.mode = 1;
          t.diag = I == J;
          t.ldc = q.mf;
          t.c_off = P.front_off[q.f] + (int64_t)(q.pf + I * G_BM) + (int64_t)(q.pf + J * G_BN) * q.mf;
          tl.push_back(t);
        }
    L.ng2 = (int)tl.size() - L.g20;
  }
  if (tl.empty()) return D3M_OK;
  CUDA_TRY(upload(d, &d->tc_split, sp));
  CUDA_TRY(upload(d, &d->tc_tiles, tl));
  CUDA_TRY(upload(d, &d->w21_off, w21_off));
  CUDA_TRY(dalloc(d, &d->planesA, (size_t)maxA * G_NPL));
  CUDA_TRY(dalloc(d, &d->planesB, (size_t)maxA * G_NPL));
  CUDA_TRY(dalloc(d, &d->tc_w, (size_t)maxW));
  for (int l = 0; l < P.n_levels; ++l) {
    DeviceState::TcLevel &L = d->tcl[l];
    if (L.kpitch == 0) continue;
    if (!encode_planes(&L.tmA, d->planesA, L.kpitch, L.rowsA) || !encode_planes(&L.tmB, d->planesB, L.kpitch, L.rowsB)) {
      c.err = "d3m_factor: tensor map encoding of the operand planes failed";
      return D3M_ECUDA;
    }
  }
  CUDA_TRY(cudaFuncSetAttribute(k_tc_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, G_SMEM));
  return D3M_OK;
}

static int dev_init(Ctx &c) {
  if (c.dev) return D3M_OK;
  const Plan &P = c.plan;
  if (c.fault == "alloc") {  // host-side fault injection: the first device allocation fails
    c.err = "d3m_factor: device allocation failed (injected by D3M_FAULT=alloc)";
    return D3M_ENOMEM;
  }
  DeviceState *d = new DeviceState();
  c.dev = d;
  d->precision = c.opt.precision;
  d->stream = (cudaStream_t)c.opt.stream;
  int prio_lo = 0, prio_hi = 0;
  CUDA_TRY(cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi));
  d->prio_lo = prio_lo;
  d->prio_hi = prio_hi;
  if (!d->stream) {
    // CUDA graphs cannot be captured on the legacy NULL stream: work on an own
    // non-blocking stream, ordered after the caller's legacy-stream work at
    // every entry point (enter()) and synchronised before returning
    CUDA_TRY(cudaStreamCreateWithPriority(&d->stream, cudaStreamNonBlocking, prio_hi));
    CUDA_TRY(cudaEventCreateWithFlags(&d->legacy_ev, cudaEventDisableTiming));
    d->own_stream = true;
  }
  CUDA_TRY(cudaStreamCreateWithPriority(&d->stream_b, cudaStreamNonBlocking, prio_lo));
  for (int q = 0; q < 3; ++q) {
    CUDA_TRY(cudaEventCreateWithFlags(&d->ev_step[q], cudaEventDisableTiming));
    CUDA_TRY(cudaEventCreateWithFlags(&d->ev_schur[q], cudaEventDisableTiming));
  }
  CUDA_TRY(cudaEventCreateWithFlags(&d->ev_b, cudaEventDisableTiming));
  CUDA_TRY(cudaStreamCreateWithPriority(&d->stream_c, cudaStreamNonBlocking, prio_lo));
  CUDA_TRY(cudaEventCreateWithFlags(&d->ev_lvl, cudaEventDisableTiming));
  CUDA_TRY(cudaEventCreateWithFlags(&d->ev_c, cudaEventDisableTiming));
  const int64_t nsn = (int64_t)P.sn_start.size();
  std::vector<int32_t> m(nsn), pp(nsn), par(nsn);
  std::vector<int64_t> soff(nsn);
  for (int64_t s = 0; s < nsn; ++s) {
    pp[s] = (int32_t)(P.sn_end[s] - P.sn_start[s]);
    m[s] = pp[s] + (int32_t)(P.struct_ptr[s + 1] - P.struct_ptr[s]);
    par[s] = (int32_t)P.parent[s];
    soff[s] = P.struct_ptr[s];
  }
  CUDA_TRY(upload(d, &d->f_m, m));
  CUDA_TRY(upload(d, &d->f_p, pp));
  CUDA_TRY(upload(d, &d->f_parent, par));
  CUDA_TRY(upload(d, &d->f_off, P.front_off));
  CUDA_TRY(upload(d, &d->f_piv, P.piv_off));
  CUDA_TRY(upload(d, &d->f_soff, soff));
  CUDA_TRY(upload(d, &d->f_start, P.sn_start));
  CUDA_TRY(upload(d, &d->f_y, P.y_off));
  CUDA_TRY(upload(d, &d->lvl_fronts, P.level_fronts));
  CUDA_TRY(upload(d, &d->ea_child, P.ea_child));
  CUDA_TRY(upload(d, &d->emap, P.emap));
  {
    // forward gather: for every front row (original order, Y row y_off + o)
    // the Y rows of the child update rows that extend-add into it
    int64_t ny = 0;
    for (int64_t s2 = 0; s2 < nsn; ++s2) ny = std::max<int64_t>(ny, P.y_off[s2] + m[s2]);
    std::vector<int64_t> gp((size_t)ny + 1, 0), gs;
    for (int64_t c2 = 0; c2 < nsn; ++c2) {
      const int64_t q = P.parent[c2];
      if (q < 0) continue;
      for (int i = 0; i < m[c2] - pp[c2]; ++i) gp[(size_t)(P.y_off[q] + P.emap[P.struct_ptr[c2] + i]) + 1]++;
    }
    for (int64_t g = 0; g < ny; ++g) gp[(size_t)g + 1] += gp[(size_t)g];
    gs.resize((size_t)gp[(size_t)ny]);
    std::vector<int64_t> fill(gp.begin(), gp.end() - 1);
    for (int64_t c2 = 0; c2 < nsn; ++c2) {
      const int64_t q = P.parent[c2];
      if (q < 0) continue;
      for (int i = 0; i < m[c2] - pp[c2]; ++i)
        gs[(size_t)fill[(size_t)(P.y_off[q] + P.emap[P.struct_ptr[c2] + i])]++] = P.y_off[c2] + pp[c2] + i;
    }
    if (gs.empty()) gs.push_back(0);
    CUDA_TRY(upload(d, &d->g_ptr, gp));
    CUDA_TRY(upload(d, &d->g_src, gs));
  }
  CUDA_TRY(upload(d, &d->sidx, P.struct_idx));
  CUDA_TRY(upload(d, &d->ent_off, P.ent_off));
  CUDA_TRY(upload(d, &d->owner, P.owner_m));
  {
    std::vector<double2> v(P.ent_val.size());
    for (size_t i = 0; i < v.size(); ++i) v[i] = make_double2(P.ent_val[i].real(), P.ent_val[i].imag());
    // host-side fault injection on the uploaded copy of the entries of M:
    // "pivot" zeroes row and column of the first pivot of front 0 (an exactly
    // zero pivot column), "nan" makes its diagonal entry NaN
    if ((c.fault == "pivot" || c.fault == "nan") && !P.sn_start.empty()) {
      const int64_t j0 = P.sn_start[0];
      for (size_t i = 0; i < v.size(); ++i) {
        if (c.fault == "pivot" && (P.ent_row[i] == j0 || P.ent_col[i] == j0)) v[i] = make_double2(0.0, 0.0);
        if (c.fault == "nan" && P.ent_row[i] == j0 && P.ent_col[i] == j0) v[i] = make_double2(NAN, 0.0);
      }
    }
    CUDA_TRY(upload(d, &d->ent_val, v));
    // the residual's operator as Ar + j Ai: most entries are real, so the
    // fp64 product costs two multiply-adds per entry instead of four
    std::vector<double> re(P.csr_val.size()), iv;
    std::vector<int64_t> ip(P.csr_ptr.size(), 0);
    std::vector<int32_t> ic;
    for (int64_t r = 0; r + 1 < (int64_t)P.csr_ptr.size(); ++r) {
      for (int64_t q = P.csr_ptr[r]; q < P.csr_ptr[r + 1]; ++q) {
        re[q] = P.csr_val[q].real();
        if (P.csr_val[q].imag() != 0.0) {
          ic.push_back(P.csr_col[q]);
          iv.push_back(P.csr_val[q].imag());
        }
      }
      ip[r + 1] = (int64_t)ic.size();
    }
    if (ic.empty()) {  // keep the device arrays non-null
      ic.push_back(0);
      iv.push_back(0.0);
    }
    CUDA_TRY(upload(d, &d->csr_re, re));
    CUDA_TRY(upload(d, &d->csi_ptr, ip));
    CUDA_TRY(upload(d, &d->csi_col, ic));
    CUDA_TRY(upload(d, &d->csi_val, iv));
  }
  CUDA_TRY(upload(d, &d->csr_ptr, P.csr_ptr));
  CUDA_TRY(upload(d, &d->csr_col, P.csr_col));
  CUDA_TRY(upload(d, &d->pec, P.pec));
  // W offsets: per level, fronts laid out one after the other (m x NB each)
  std::vector<int64_t> wofs(nsn);
  int64_t wmax = 0;
  d->level_steps.assign(P.n_levels, 0);
  d->update_grid.assign(P.n_levels, {});
  d->level_maxm.assign(P.n_levels, 0);
  std::vector<int32_t> nsplit_h(nsn, 0);
  d->part_off_h.assign(nsn, 0);
  d->part_rows = 0;
  for (int l = 0; l < P.n_levels; ++l) {
    int64_t prow = 0;
    for (int i = P.level_ptr[l]; i < P.level_ptr[l + 1]; ++i) {
      int s = P.level_fronts[i];
      int S = (m[s] - pp[s] + BSPLIT - 1) / BSPLIT;
      nsplit_h[i] = S;
      d->part_off_h[i] = prow;
      prow += (int64_t)S * pp[s];
    }
    d->part_rows = std::max(d->part_rows, prow);
    int64_t w = 0;
    int steps = 0, maxm = 0;
    for (int i = P.level_ptr[l]; i < P.level_ptr[l + 1]; ++i) {
      int s = P.level_fronts[i];
      wofs[i] = w;
      w += (int64_t)m[s] * NB;
      steps = std::max(steps, (pp[s] + NB - 2) / (NB - 1));
      maxm = std::max(maxm, m[s]);
    }
    wmax = std::max(wmax, w);
    d->level_steps[l] = steps;
    d->level_maxm[l] = maxm;
    for (int stp = 0; stp < steps; ++stp) {
      int g = 0;
      for (int i = P.level_ptr[l]; i < P.level_ptr[l + 1]; ++i) {
        int s = P.level_fronts[i];
        int cmin = std::min<int>(pp[s], (stp + 1) * (NB - 1));
        int nt = (m[s] + UT - 1) / UT - cmin / UT;
        g = std::max(g, nt * (nt + 1) / 2);
      }
      d->update_grid[l].push_back(std::max(g, 1));
    }
  }
  CUDA_TRY(upload(d, &d->wofs, wofs));
  {
    // L11^{-1} storage (level-major) and the factor-time doubling stages:
    // for blocks A = [i0, i0+s), C = [i0+s, i0+2s) of the pivot range,
    //   T1 = L[C, A] A^{-1}  (mode 2),   L^{-1}[C, A] = -C^{-1} T1  (mode 1)
    std::vector<CgItem> items;
    d->linv_off_h.assign(nsn, 0);
    int64_t lo = 0, tmax = 0;
    for (int i = 0; i < (int)nsn; ++i) {
      int s = P.level_fronts[i];
      d->linv_off_h[i] = lo;
      lo += (int64_t)pp[s] * pp[s];
    }
    const bool mixed = c.opt.precision == D3M_MIXED;
    d->inv_stage.assign(P.n_levels, {});
    for (int l = 0; l < P.n_levels; ++l) {
      int pmax = 0;
      for (int i = P.level_ptr[l]; i < P.level_ptr[l + 1]; ++i) pmax = std::max(pmax, pp[P.level_fronts[i]]);
      for (int sz = 32; sz < pmax; sz *= 2) {
        std::vector<CgItem> g1, g2;
        int64_t toff = 0;
        for (int i = P.level_ptr[l]; i < P.level_ptr[l + 1]; ++i) {
          int f = P.level_fronts[i];
          int pf = pp[f], mf = m[f];
          int64_t lf = d->linv_off_h[i];
          for (int i0 = 0; i0 + sz < pf; i0 += 2 * sz) {
            int cs = std::min(sz, pf - i0 - sz);
            CgItem a{};
            a.gath = -1;
            a.a = P.front_off[f] + (i0 + sz) + (int64_t)i0 * mf;  // L[C, A]
            a.a_rs = 1; a.a_cs = mf;
            a.b = lf + i0 + (int64_t)i0 * pf;                      // A^{-1}
            a.b_rs = 1; a.b_cs = pf;
            a.c = toff;                                            // T1 (cs x sz, column-major)
            a.c_rs = 1; a.c_cs = cs;
            a.M = cs; a.N = sz; a.K = sz; a.mode = 2;
            a.abuf = 0; a.bbuf = 1; a.cbuf = 2; a.beta = 0; a.alpha = 1.f;
            g1.push_back(a);
            CgItem b{};
            b.gath = -1;
            b.a = lf + (i0 + sz) + (int64_t)(i0 + sz) * pf;      // C^{-1}
            b.a_rs = 1; b.a_cs = pf;
            b.b = toff; b.b_rs = 1; b.b_cs = cs;                   // T1
            b.c = lf + (i0 + sz) + (int64_t)i0 * pf;               // L^{-1}[C, A]
            b.c_rs = 1; b.c_cs = pf;
            b.M = cs; b.N = sz; b.K = cs; b.mode = 1;
            b.abuf = 1; b.bbuf = 2; b.cbuf = 1; b.beta = 0; b.alpha = -1.f;
            g2.push_back(b);
            toff += (int64_t)cs * sz;
          }
        }
        tmax = std::max(tmax, toff);
        if (g1.empty()) continue;
        auto t1 = cg_assign(g1, mixed), t2 = cg_assign(g2, mixed);
        d->inv_stage[l].push_back({(int)items.size(), (int)g1.size(), t1.first, t1.second});
        items.insert(items.end(), g1.begin(), g1.end());
        d->inv_stage[l].push_back({(int)items.size(), (int)g2.size(), t2.first, t2.second});
        items.insert(items.end(), g2.begin(), g2.end());
      }
    }
    const size_t esz0 = c.opt.precision == D3M_FP64 ? sizeof(cx<double>) : sizeof(cx<float>);
    CUDA_TRY(cudaMalloc(&d->linv, std::max<int64_t>(lo, 1) * esz0));
    d->allocs.push_back(d->linv);
    CUDA_TRY(cudaMalloc(&d->tmp_inv, std::max<int64_t>(tmax, 1) * esz0));
    d->allocs.push_back(d->tmp_inv);
    CUDA_TRY(upload(d, &d->inv_items, items));
    CUDA_TRY(upload(d, &d->linv_off, d->linv_off_h));
    if (mixed && c.opt.solve_kernel == 0) {
      // the A operands of the tensor-core substitution, as 128 x 32 blocks
      // (only the blocks inside the k range of each row tile of the
      // triangular L11^{-1} and L11^{-T} are written and read)
      std::vector<QPre> pre;
      d->qblk_h.assign(nsn, {});
      d->qnk_h.assign(nsn, {});
      d->qpre_lvl.assign(P.n_levels, {});
      int64_t nb = 0;
      for (int l = 0; l < P.n_levels; ++l) {
        d->qpre_lvl[l][0] = (int64_t)pre.size();
        bool on[4];
        for (int kind = 0; kind < 4; ++kind) on[kind] = tc_solve_launch(P, l, kind);
        for (int i = P.level_ptr[l]; i < P.level_ptr[l + 1]; ++i) {
          const int f = P.level_fronts[i];
          const int pf = pp[f], mf = m[f];
          for (int kind = 0; kind < 4; ++kind) {
            QPre q{};
            int mode = 0;
            if (kind == 0 || kind == 3) {
              q.src = d->linv_off_h[i]; q.abuf = 1; q.M = pf; q.K = pf;
              q.a_rs = kind == 0 ? 1 : pf; q.a_cs = kind == 0 ? pf : 1;
              mode = kind == 0 ? 1 : 3;
            } else {
              q.src = P.front_off[f] + pf; q.abuf = 0;
              q.M = kind == 1 ? mf - pf : pf; q.K = kind == 1 ? pf : mf - pf;
              q.a_rs = kind == 1 ? 1 : mf; q.a_cs = kind == 1 ? mf : 1;
            }
            if (q.M <= 0 || q.K <= 0 || !on[kind]) continue;
            const int nkc = (q.K + Q_BK - 1) / Q_BK, ntm = (q.M + Q_BM - 1) / Q_BM;
            d->qblk_h[i][kind] = nb;
            d->qnk_h[i][kind] = nkc;
            for (int tm = 0; tm < ntm; ++tm) {
              // the chunks the row tile's k range reaches (all, or those of a triangle)
              const int c0 = mode == 3 ? tm * (Q_BM / Q_BK) : 0;
              const int c1 = mode == 1 ? std::min(nkc, (tm + 1) * (Q_BM / Q_BK)) : nkc;
              for (int kc = c0; kc < c1; ++kc) {
                QPre b = q;
                b.blk = nb + q_rowbase(mode, nkc, tm) + kc;
                b.r0 = tm * Q_BM;
                b.k0 = kc * Q_BK;
                pre.push_back(b);
              }
            }
            nb += q_rowbase(mode, nkc, ntm) + (mode == 3 ? (int64_t)ntm * (Q_BM / Q_BK) : 0);
          }
        }
        d->qpre_lvl[l][1] = (int64_t)pre.size() - d->qpre_lvl[l][0];
      }
      d->qblocks = nb;
      if (!pre.empty()) {
        CUDA_TRY(upload(d, &d->qpre, pre));
        CUDA_TRY(dalloc(d, &d->qpl, (size_t)nb * (Q_ABLK / 2)));
      }
    }
  }
  CUDA_TRY(upload(d, &d->nsplit, nsplit_h));
  CUDA_TRY(upload(d, &d->part_off, d->part_off_h));
  const size_t esz = c.opt.precision == D3M_FP64 ? sizeof(cx<double>) : sizeof(cx<float>);
  d->wslot = std::max<int64_t>(wmax, 1);
  CUDA_TRY(cudaMalloc(&d->W, 3 * d->wslot * esz));
  CUDA_TRY(dalloc(d, &d->snap, (size_t)3 * nsn));
  d->allocs.push_back(d->W);
  CUDA_TRY(cudaMalloc(&d->arena, std::max<int64_t>(P.arena_elems, 1) * esz));
  d->allocs.push_back(d->arena);
  CUDA_TRY(dalloc(d, &d->perm, P.piv_total));
  CUDA_TRY(dalloc(d, &d->iperm, P.piv_total));
  CUDA_TRY(dalloc(d, &d->dinv_d, P.piv_total));
  CUDA_TRY(dalloc(d, &d->dinv_o, P.piv_total));
  CUDA_TRY(dalloc(d, &d->psize, P.piv_total));
  CUDA_TRY(dalloc(d, &d->st_k0, nsn));
  CUDA_TRY(dalloc(d, &d->st_kb, nsn));
  CUDA_TRY(dalloc(d, &d->st_info, nsn));
  CUDA_TRY(dalloc(d, &d->st_minpiv, nsn));
  CUDA_TRY(dalloc(d, &d->flop_cnt, 2));
  CUDA_TRY(dalloc(d, &d->swp, (size_t)3 * nsn * 2 * NB));  // three look-ahead slots
  CUDA_TRY(dalloc(d, &d->tc_err, 1));
  CUDA_TRY(dalloc(d, &d->fin_err, 1));
  CUDA_TRY(dalloc(d, &d->sv_err, 1));
  CUDA_TRY(cudaFuncSetAttribute(k_tc_cgemm, cudaFuncAttributeMaxDynamicSharedMemorySize, Q_SMEM));
  if (c.fault == "timeout") d->tc_wait_cap = 0;  // every first wait of k_tc_gemm expires at once
  if (c.fault == "solve_timeout") d->sv_wait_cap = 0;  // the same for k_tc_cgemm (the substitution)
  d->update_grid_p.assign(P.n_levels, {});
  d->update_grid_r.assign(P.n_levels, {});
  for (int l = 0; l < P.n_levels; ++l)
    for (int stp = 0; stp < d->level_steps[l]; ++stp) {
      int g = 0, gr = 0;
      for (int i = P.level_ptr[l]; i < P.level_ptr[l + 1]; ++i) {
        int s = P.level_fronts[i];
        int cmin = std::min<int>(pp[s], (stp + 1) * (NB - 1));
        int nt = (pp[s] + UT - 1) / UT - cmin / UT;
        g = std::max(g, nt * (nt + 1) / 2);
        const int nr = (m[s] - (pp[s] / UT) * UT + UT - 1) / UT, nc = (pp[s] - (cmin / UT) * UT + UT - 1) / UT;
        gr = std::max(gr, nr * nc);
      }
      d->update_grid_p[l].push_back(std::max(g, 1));
      d->update_grid_r[l].push_back(std::max(gr, 1));
    }
  if (c.opt.precision == D3M_MIXED) {
    const int rc = tc_plan(c, d, m, pp);
    if (rc) return rc;
  }
  d->level_maxp.assign(P.n_levels, 0);
  for (int l = 0; l < P.n_levels; ++l)
    for (int i = P.level_ptr[l]; i < P.level_ptr[l + 1]; ++i)
      d->level_maxp[l] = std::max(d->level_maxp[l], pp[P.level_fronts[i]]);
  d->lvl_tc.assign(P.n_levels, 0);
  d->lvl_cs.assign(P.n_levels, 0);
  for (int l = 0; l < P.n_levels; ++l)
    d->lvl_cs[l] = panel_cluster_size(d->level_maxp[l], c.opt.precision == D3M_FP64 ? sizeof(cx<double>)
                                                                                      : sizeof(cx<float>));
  d->prof.on = c.opt.profile != 0;
  d->prof.s = d->stream;
  d->solve_flops_per_rhs = 0;
  for (int64_t s = 0; s < nsn; ++s)  // forward + backward, 8 real flops per complex MAC
    d->solve_flops_per_rhs += 16.0 * (0.5 * pp[s] * (pp[s] - 1.0) + (double)(m[s] - pp[s]) * pp[s]);
  // extend-add grids
  d->ea_grid.clear();
  for (size_t q = 0; q + 1 < P.ea_ptr.size(); ++q) {
    int g = 1;
    for (int i = P.ea_ptr[q]; i < P.ea_ptr[q + 1]; ++i) {
      int s = P.ea_child[i];
      int n = m[s] - pp[s];
      int nt = (n + 31) / 32;
      g = std::max(g, nt * (nt + 1) / 2);
    }
    d->ea_grid.push_back(g);
  }
  return D3M_OK;
}

__global__ void k_init_perm(int64_t nsn, const int32_t *__restrict__ fp, const int64_t *__restrict__ fpiv,
                            int32_t *__restrict__ perm) {
  int64_t s = blockIdx.x;
  if (s >= nsn) return;
  for (int i = threadIdx.x; i < fp[s]; i += blockDim.x) perm[fpiv[s] + i] = i;
}
__global__ void k_iperm(int64_t nsn, const int32_t *__restrict__ fp, const int64_t *__restrict__ fpiv,
                        const int32_t *__restrict__ perm, int32_t *__restrict__ iperm) {
  int64_t s = blockIdx.x;
  if (s >= nsn) return;
  for (int i = threadIdx.x; i < fp[s]; i += blockDim.x) iperm[fpiv[s] + perm[fpiv[s] + i]] = i;
}
// flag = 1 if an entry of the pivot inverses is not finite
__global__ void k_check_finite(const double2 *__restrict__ v, int64_t n, int32_t *__restrict__ flag) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    if (!isfinite(v[i].x) || !isfinite(v[i].y)) *flag = 1;
}
__global__ void k_fill_double(double *x, int64_t n, double v) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) x[i] = v;
}

template <typename T>
static int factor_t(Ctx &c) {
  const Plan &P = c.plan;
  DeviceState *d = c.dev;
  cudaStream_t s = d->stream;
  const int64_t nsn = (int64_t)P.sn_start.size();
  cx<T> *arena = (cx<T> *)d->arena;
  cx<T> *W = (cx<T> *)d->W;
  FrontTab ft = tab(d);
  CUDA_TRY(panel_attrs<T>());
  // Without profiling the launch sequence (fixed once the schedule is tuned)
  // is captured into a CUDA graph at the first call and replayed after.
  const bool use_graph = !d->prof.on;
  int64_t nl = 0;
  auto enqueue = [&]() -> int {
    CUDA_TRY(cudaMemsetAsync(d->st_k0, 0, nsn * sizeof(int32_t), s));
    CUDA_TRY(cudaMemsetAsync(d->st_kb, 0, nsn * sizeof(int32_t), s));
    CUDA_TRY(cudaMemsetAsync(d->st_info, 0, nsn * sizeof(int32_t), s));
    CUDA_TRY(cudaMemsetAsync(d->flop_cnt, 0, 2 * sizeof(double), s));
    CUDA_TRY(cudaMemsetAsync(d->tc_err, 0, sizeof(int32_t), s));
    CUDA_TRY(cudaMemsetAsync(d->fin_err, 0, sizeof(int32_t), s));
    d->prof.reset();
    // (profiled runs are sequential, so that every kernel class's events time
  // that class alone)
  const bool la = c.opt.lookahead == 0 && !d->lookahead_off && !d->prof.on;
    bool used_c = false;  // stream_c carried an L11^{-1} (join it before the end)
    k_fill_double<<<(unsigned)((nsn + 255) / 256), 256, 0, s>>>(d->st_minpiv, nsn, 1e300);
    k_init_perm<<<(unsigned)nsn, 128, 0, s>>>(nsn, d->f_p, d->f_piv, d->perm);
    nl += 2;
    for (int l = 0; l < P.n_levels; ++l) {
      const int nf = P.level_ptr[l + 1] - P.level_ptr[l];
      const int32_t *lvl = d->lvl_fronts + P.level_ptr[l];
      d->prof.cur_level = l;
      // deferred products on the tensor cores (mixed): the panels update only
      // the pivot blocks; the update rows and Schur complements follow as two
      // batched tcgen05 products after the level's L11^{-1}
      const bool defer = sizeof(T) == 4 && (c.opt.update_kernel == 2 || (c.opt.update_kernel == 0 && d->lvl_tc[l]));
      // zero the level's fronts (contiguous) and assemble the entries of M
      int64_t first = P.front_off[P.level_fronts[P.level_ptr[l]]];
      int last_s = P.level_fronts[P.level_ptr[l + 1] - 1];
      int64_t mlast = (P.sn_end[last_s] - P.sn_start[last_s]) + (P.struct_ptr[last_s + 1] - P.struct_ptr[last_s]);
      int64_t end = P.front_off[last_s] + mlast * mlast;
      {
        PROF_BEGIN(PC_ASSEMBLE);
        CUDA_TRY(cudaMemsetAsync(arena + first, 0, (end - first) * sizeof(cx<T>), s));
        int64_t ne = P.ent_ptr[l + 1] - P.ent_ptr[l];
        if (ne > 0) {
          k_assemble<T><<<(unsigned)((ne + 255) / 256), 256, 0, s>>>(ne, d->ent_off + P.ent_ptr[l],
                                                                      d->ent_val + P.ent_ptr[l], arena);
          ++nl;
        }
        for (int q = P.ea_pass_ptr[l]; q < P.ea_pass_ptr[l + 1]; ++q) {
          int nk = P.ea_ptr[q + 1] - P.ea_ptr[q];
          if (nk == 0) continue;
          dim3 g(d->ea_grid[q], nk);
          k_extend_add<T><<<g, 256, 0, s>>>(d->ea_child + P.ea_ptr[q], ft, d->emap, arena);
          ++nl;
        }
        PROF_END(PC_ASSEMBLE);
      }
      const int64_t *wofs = d->wofs + P.level_ptr[l];
      // trailing update of one step: mode 0 all trailing columns, 1 the pivot
      // block's, 2 the Schur complement's (on stream st)
      // (priorities under look-ahead: the panel chain urgent, the overlapped
      // Schur part least urgent)
      auto update = [&](int stp, const cx<T> *Ws, const int2 *sn, int mode, cudaStream_t st) {
        const int prio = !la ? 0 : mode == 2 ? d->prio_lo : d->prio_hi;
        dim3 g(mode == 3 ? d->update_grid_p[l][stp] : mode == 4 ? d->update_grid_r[l][stp] : d->update_grid[l][stp],
               nf);
        launch_prio(k_update<T>, g, dim3(256), 0, st, prio, lvl, ft, wofs, arena, (const cx<T> *)Ws, sn, mode);
      };
      // Deferred levels: each step's panel and its pivot-block update (mode
      // 3) form the critical chain on stream s; the update rows of the step
      // (Algorithm 1's triangular solve, k_l21, writing W21 = L21 D to the
      // W21 buffer) and their trailing update (mode 4) follow on stream_b with
      // the least urgent priority.  W, the snapshots and the column
      // permutations rotate through three slots, as in the look-ahead below.
      // The Schur complements are one tensor-core product after the level.
      if (defer && la) {
        CUDA_TRY(cudaEventRecord(d->ev_b, s));
        CUDA_TRY(cudaStreamWaitEvent(d->stream_b, d->ev_b, 0));
      }
      for (int stp = 0; defer && stp < d->level_steps[l]; ++stp) {
        const int slot = stp % 3;
        cx<T> *Ws = W + slot * d->wslot;
        int2 *sn = d->snap + slot * nsn + P.level_ptr[l];
        int2 *sw = d->swp + ((int64_t)slot * nsn + P.level_ptr[l]) * 2 * NB;
        cudaStream_t sb = la ? d->stream_b : s;
        if (la && stp >= 3) CUDA_TRY(cudaStreamWaitEvent(s, d->ev_schur[slot], 0));
        {
          PROF_BEGIN(PC_PANEL);
          int cs = c.opt.panel_kernel == 1 ? 0 : d->lvl_cs[l];
          CUDA_TRY(launch_panel<T>(cs, d->level_maxp[l], 0, nf, lvl, ft, wofs, arena, Ws, d->perm, d->dinv_d,
                                   d->dinv_o, d->psize, d->st_k0, d->st_kb, d->st_info, d->st_minpiv, d->flop_cnt, sw,
                                   sn, s, la ? d->prio_hi : 0));
          PROF_END(PC_PANEL);
        }
        {
          PROF_BEGIN(PC_UPDATE);
          update(stp, Ws, sn, 3, s);
          PROF_END(PC_UPDATE);
        }
        if (la) {
          CUDA_TRY(cudaEventRecord(d->ev_step[slot], s));
          CUDA_TRY(cudaStreamWaitEvent(sb, d->ev_step[slot], 0));
        }
        if (d->level_maxm[l] > d->level_maxp[l]) {
          {
            PROF_BEGIN_ON(PC_PANEL, sb);
            dim3 g((unsigned)std::max(1, (d->level_maxm[l] + 127) / 128), (unsigned)nf);
            CUDA_TRY(launch_prio(k_l21<T>, g, dim3(128), 0, sb, la ? d->prio_lo : 0, lvl, ft, wofs, arena, Ws,
                                 (const double2 *)d->dinv_d, (const double2 *)d->dinv_o, (const int8_t *)d->psize,
                                 (const int2 *)sn, (const int2 *)sw, d->flop_cnt, d->tc_w,
                                 (const int64_t *)(d->w21_off + P.level_ptr[l])));
            PROF_END_ON(PC_PANEL, sb);
          }
          {
            PROF_BEGIN_ON(PC_UPDATE, sb);
            update(stp, Ws, sn, 4, sb);
            PROF_END_ON(PC_UPDATE, sb);
          }
          nl += 2;
        }
        if (la) CUDA_TRY(cudaEventRecord(d->ev_schur[slot], sb));
        nl += 2;
      }
      if (defer && la) {
        CUDA_TRY(cudaEventRecord(d->ev_b, d->stream_b));
        CUDA_TRY(cudaStreamWaitEvent(s, d->ev_b, 0));
      }
      if (la && !defer) {  // stream_b starts after everything issued so far on the factor stream
        CUDA_TRY(cudaEventRecord(d->ev_b, s));
        CUDA_TRY(cudaStreamWaitEvent(d->stream_b, d->ev_b, 0));
      }
      for (int stp = 0; !defer && stp < d->level_steps[l]; ++stp) {
        // Look-ahead: the panels of a front read and write only its pivot
        // block (columns < p), so the Schur-complement part of step stp's
        // update (columns >= p) runs on stream_b while step stp + 1 proceeds
        // here.  Slot stp % 3 of W and of the snapshots is rewritten by the
        // panel of step stp + 3, which first waits for that update.
        const int slot = stp % 3;
        cx<T> *Ws = W + (la ? slot * d->wslot : 0);
        int2 *sn = d->snap + (la ? slot * nsn : 0) + P.level_ptr[l];
        if (la && stp >= 3) CUDA_TRY(cudaStreamWaitEvent(s, d->ev_schur[slot], 0));
        {
          PROF_BEGIN(PC_PANEL);
          int cs = c.opt.panel_kernel == 1 ? 0 : d->lvl_cs[l];
          CUDA_TRY(launch_panel<T>(cs, d->level_maxp[l], d->level_maxm[l], nf, lvl, ft, wofs, arena, Ws, d->perm,
                                   d->dinv_d, d->dinv_o, d->psize, d->st_k0, d->st_kb, d->st_info, d->st_minpiv,
                                   d->flop_cnt, d->swp + (int64_t)P.level_ptr[l] * 2 * NB, sn, s,
                                   la ? d->prio_hi : 0));
          PROF_END(PC_PANEL);
        }
        if (!la) {
          PROF_BEGIN(PC_UPDATE);
          update(stp, Ws, sn, 0, s);
          PROF_END(PC_UPDATE);
          nl += 2;
          continue;
        }
        CUDA_TRY(cudaEventRecord(d->ev_step[slot], s));
        {
          PROF_BEGIN(PC_UPDATE);
          update(stp, Ws, sn, 1, s);
          PROF_END(PC_UPDATE);
        }
        CUDA_TRY(cudaStreamWaitEvent(d->stream_b, d->ev_step[slot], 0));
        {
          PROF_BEGIN_ON(PC_UPDATE, d->stream_b);
          update(stp, Ws, sn, 2, d->stream_b);
          PROF_END_ON(PC_UPDATE, d->stream_b);
        }
        CUDA_TRY(cudaEventRecord(d->ev_schur[slot], d->stream_b));
        nl += 3;
      }
      // the next level's extend-add reads these Schur complements
      if (la && !defer) {
        CUDA_TRY(cudaEventRecord(d->ev_b, d->stream_b));
        CUDA_TRY(cudaStreamWaitEvent(s, d->ev_b, 0));
      }
      // L11^{-1} of the level's fronts (mixed precision only: it turns every
      // substitution into tile GEMMs; the fp64 path keeps the triangular-solve
      // kernels, since on the fp64 pipe the extra p^3/6 flops cost more than
      // the sequential blocks): diagonal 32-blocks, then doubling stages
      if (sizeof(T) == 4) {
        // under look-ahead on stream_c, after everything of this level
        cudaStream_t si = s;
        if (la) {
          si = d->stream_c;
          used_c = true;
          CUDA_TRY(cudaEventRecord(d->ev_lvl, s));
          CUDA_TRY(cudaStreamWaitEvent(si, d->ev_lvl, 0));
        }
        PROF_BEGIN(PC_INV);
        cx<T> *Li = (cx<T> *)d->linv;
        int lf = P.level_fronts[P.level_ptr[l]];
        int ll = P.level_fronts[P.level_ptr[l + 1] - 1];
        int64_t a0 = d->linv_off_h[P.level_ptr[l]];
        int64_t pl = P.sn_end[ll] - P.sn_start[ll];
        int64_t a1 = d->linv_off_h[P.level_ptr[l + 1] - 1] + pl * pl;
        (void)lf;
        CUDA_TRY(cudaMemsetAsync(Li + a0, 0, (a1 - a0) * sizeof(cx<T>), si));
        dim3 gd((unsigned)((d->level_maxp[l] + 31) / 32), nf);
        k_trinv_diag<T><<<gd, 32, 0, si>>>(lvl, ft, arena, d->linv_off + P.level_ptr[l], Li);
        ++nl;
        const CgBufs<T> ib{{arena, Li, (cx<T> *)d->tmp_inv, nullptr, nullptr, nullptr, nullptr}};
        for (auto &st : d->inv_stage[l]) {
          launch_cgemm<T>(st[3], st[2], d->inv_items + st[0], st[1], ib, nullptr, si);
          ++nl;
        }
        // the level's substitution operands as pre-split tensor-core blocks
        if (d->qpl && d->qpre_lvl[l][1] > 0) {
          CgBufs<float> fb;
          for (int q = 0; q < 7; ++q) fb.p[q] = reinterpret_cast<cx<float> *>(ib.p[q]);
          k_tc_presplit<<<(unsigned)d->qpre_lvl[l][1], 256, 0, si>>>(d->qpre + d->qpre_lvl[l][0], fb, d->qpl);
          ++nl;
        }
        PROF_END(PC_INV);
      }
      if (defer && sizeof(T) == 4 && d->tcl[l].kpitch > 0) {
        const DeviceState::TcLevel &L = d->tcl[l];
        cx<float> *ar = (cx<float> *)d->arena;
        PROF_BEGIN(PC_TC);
        // operands of C = F22 - L21 W21^T as bf16 planes, then the product
        k_tc_split<<<L.nsx, 256, 0, s>>>(d->tc_split + L.sx0, ar, d->perm, d->f_piv, d->planesA, L.rowsA,
                                         L.kpitch);
        k_tc_split<<<L.nsl, 256, 0, s>>>(d->tc_split + L.sl0, (const cx<float> *)d->tc_w, d->perm, d->f_piv,
                                         d->planesB, L.rowsB, L.kpitch);
        k_tc_gemm<<<L.ng2, 128, G_SMEM, s>>>(L.tmA, L.tmB, d->tc_tiles + L.g20, ar, d->tc_w, d->tc_err,
                                             d->tc_wait_cap);
        PROF_END(PC_TC);
        nl += 3;
      }
    }
    if (used_c) {  // join the inverses before the factor completes
      CUDA_TRY(cudaEventRecord(d->ev_c, d->stream_c));
      CUDA_TRY(cudaStreamWaitEvent(s, d->ev_c, 0));
    }
    d->prof.cur_level = -1;
    k_iperm<<<(unsigned)nsn, 128, 0, s>>>(nsn, d->f_p, d->f_piv, d->perm, d->iperm);
    k_check_finite<<<(unsigned)std::max<int64_t>(1, std::min<int64_t>((P.piv_total + 255) / 256, 1216)), 256, 0, s>>>(
        d->dinv_d, P.piv_total, d->fin_err);
    nl += 2;
  return D3M_OK;
  };
  if (use_graph && d->g_factor) {
    CUDA_TRY(cudaGraphLaunch(d->g_factor, s));
    nl = d->g_factor_launches;
  } else if (use_graph) {
    CUDA_TRY(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    const int rc = enqueue();
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(s, &g);
    if (rc != D3M_OK) {
      if (g) cudaGraphDestroy(g);
      return rc;
    }
    if (e == cudaSuccess) {
      // node priorities (look-ahead) apply only with this flag
      const cudaError_t ei =
          cudaGraphInstantiateWithFlags(&d->g_factor, g, cudaGraphInstantiateFlagUseNodePriority);
      cudaGraphDestroy(g);
      CUDA_TRY(ei);
    } else {
      CUDA_TRY(e);
    }
    d->g_factor_launches = nl;
    CUDA_TRY(cudaGraphLaunch(d->g_factor, s));
  } else {
    const int rc = enqueue();
    if (rc != D3M_OK) return rc;
  }
  c.stats.launches_factor = nl + d->inv_launches;
  CUDA_TRY(cudaGetLastError());
  CUDA_TRY(cudaStreamSynchronize(s));
  std::vector<int32_t> info(nsn);
  std::vector<double> mp(nsn);
  CUDA_TRY(cudaMemcpy(info.data(), d->st_info, nsn * sizeof(int32_t), cudaMemcpyDeviceToHost));
  CUDA_TRY(cudaMemcpy(mp.data(), d->st_minpiv, nsn * sizeof(double), cudaMemcpyDeviceToHost));
  std::vector<int8_t> ps(P.piv_total);
  CUDA_TRY(cudaMemcpy(ps.data(), d->psize, P.piv_total, cudaMemcpyDeviceToHost));
  int64_t n2 = 0;
  for (int8_t v : ps) n2 += v == 2;
  c.stats.n_2x2 = n2;
  double mn = 1e300;
  for (double v : mp) mn = std::min(mn, v);
  c.stats.min_pivot_ratio = mn;
  double fc[2];
  CUDA_TRY(cudaMemcpy(fc, d->flop_cnt, sizeof fc, cudaMemcpyDeviceToHost));
  int32_t tce = 0;
  CUDA_TRY(cudaMemcpy(&tce, d->tc_err, sizeof tce, cudaMemcpyDeviceToHost));
  if (tce) {
    c.err = "d3m_factor: a tensor-core product tile gave up a bounded wait (its results were discarded)";
    return D3M_ETIMEOUT;
  }
  int32_t fin = 0;
  CUDA_TRY(cudaMemcpy(&fin, d->fin_err, sizeof fin, cudaMemcpyDeviceToHost));
  c.lvl_cs = d->lvl_cs;
  c.lvl_tc.assign(P.n_levels, 0);
  double ftc = 0.0;
  for (int l = 0; l < P.n_levels; ++l) {
    c.lvl_tc[l] = sizeof(T) == 4 && (c.opt.update_kernel == 2 || (c.opt.update_kernel == 0 && d->lvl_tc[l]));
    if (c.lvl_tc[l] && !d->tcl.empty()) ftc += d->tcl[l].flops;
  }
  // the panels count each step's whole trailing triangle; on deferred levels
  // the update rows and Schur complements are the tensor-core products' share
  c.stats.flops_tc = ftc;
  c.stats.flops_update = fc[0] - ftc;
  c.stats.flops_panel = fc[1];
  if (c.opt.panel_kernel == 1) c.lvl_cs.assign(P.n_levels, 0);
  if (d->prof.on) {
    d->tune_panel = d->prof.per_level(PC_PANEL, P.n_levels);
    d->tune_update = d->prof.per_level(PC_UPDATE, P.n_levels);
    d->tune_inv = d->prof.per_level(PC_INV, P.n_levels);
    d->tune_tc = d->prof.per_level(PC_TC, P.n_levels);
    c.lvl_ms_panel = d->tune_panel;
    c.lvl_ms_update = d->tune_update;
    c.lvl_ms_inv = d->tune_inv;
    c.lvl_ms_tc = d->tune_tc;
    double ms[PC_N];
    d->prof.collect(ms);
    c.stats.ms_assemble = ms[PC_ASSEMBLE];
    c.stats.ms_panel = ms[PC_PANEL];
    c.stats.ms_update = ms[PC_UPDATE];
    c.stats.ms_inverse = ms[PC_INV];
    c.stats.ms_tc = ms[PC_TC];
  }
  if (fin) {
    c.err = "d3m_factor: a pivot is not finite (non-finite entries in the operator or its factors)";
    return D3M_ESINGULAR;
  }
  for (int64_t q = 0; q < nsn; ++q)
    if (info[q] != 0) {
      char buf[160];
      snprintf(buf, sizeof buf, "d3m_factor: zero pivot column %d in front %lld (kind %lld)", info[q] - 1,
               (long long)q, (long long)P.sn_kind[q]);
      c.err = buf;
      return D3M_ESINGULAR;
    }
  return D3M_OK;
}

// Order the library stream after the caller's legacy-stream work.
static int enter(Ctx &c) {
  DeviceState *d = c.dev;
  if (d->own_stream) {
    CUDA_TRY(cudaEventRecord(d->legacy_ev, 0));
    CUDA_TRY(cudaStreamWaitEvent(d->stream, d->legacy_ev, 0));
  }
  return D3M_OK;
}

// ---- autotuner: per tree level, the trailing-update kernel (mixed: fp32 FMA
// or tcgen05) and the panel cluster size (smallest that fits, or twice that),
// chosen by timing trial factorisations with CUDA events per level (three in
// mixed precision, two in fp64: trials A, B and C below).
static std::string tune_signature(const Ctx &c) {
  const Plan &P = c.plan;
  char buf[256];
  snprintf(buf, sizeof buf, "d3m-autotune-v1 nm=%lld fronts=%lld levels=%d prec=%d arena=%lld", (long long)P.n_m,
           (long long)P.sn_start.size(), P.n_levels, c.opt.precision, (long long)P.arena_elems);
  return buf;
}
static bool tune_load(Ctx &c) {
  if (c.cache_path.empty()) return false;
  FILE *fp = fopen(c.cache_path.c_str(), "r");
  if (!fp) return false;
  char line[512];
  bool ok = fgets(line, sizeof line, fp) != nullptr;
  std::string sig = tune_signature(c);
  ok = ok && std::string(line).substr(0, sig.size()) == sig;
  DeviceState *d = c.dev;
  std::vector<uint8_t> tc(c.plan.n_levels, 0);
  std::vector<int> cs(c.plan.n_levels, 0);
  for (int l = 0; ok && l < c.plan.n_levels; ++l) {
    int ll, a, b;
    ok = fscanf(fp, "%d %d %d", &ll, &a, &b) == 3 && ll == l && b >= 0 && b <= 16;
    if (ok) {
      tc[l] = (uint8_t)(a != 0);
      cs[l] = b;
    }
  }
  fclose(fp);
  if (!ok) return false;
  // a cached cluster size must still fit this level
  for (int l = 0; l < c.plan.n_levels; ++l)
    if (cs[l] != 0 && cs[l] < d->lvl_cs[l]) return false;
  int64_t ncs2 = 0, ntc = 0;
  for (int l = 0; l < c.plan.n_levels; ++l) {
    ntc += tc[l];
    ncs2 += cs[l] != d->lvl_cs[l];
  }
  d->lvl_tc = tc;
  d->lvl_cs = cs;
  c.stats.tuned_levels_tc = ntc;
  c.stats.tuned_levels_cs2 = ncs2;
  c.stats.ms_tuning = 0.0;
  return true;
}
static void tune_save(const Ctx &c) {
  if (c.cache_path.empty()) return;
  FILE *fp = fopen(c.cache_path.c_str(), "w");
  if (!fp) return;
  fprintf(fp, "%s\n", tune_signature(c).c_str());
  for (int l = 0; l < c.plan.n_levels; ++l) fprintf(fp, "%d %d %d\n", l, (int)c.dev->lvl_tc[l], c.dev->lvl_cs[l]);
  fclose(fp);
}

static int factor_any(Ctx &c) { return c.opt.precision == D3M_FP64 ? factor_t<double>(c) : factor_t<float>(c); }

static int autotune(Ctx &c) {
  DeviceState *d = c.dev;
  const int nlev = c.plan.n_levels;
  if (tune_load(c)) {
    d->tuned = true;
    return D3M_OK;
  }
  auto t0 = std::chrono::steady_clock::now();
  const bool prof = d->prof.on;
  const int uk = c.opt.update_kernel;
  d->prof.on = true;
  d->lookahead_off = true;  // per-kernel times without the overlap
  // trial A: right-looking fp32/fp64-FMA updates, smallest cluster
  std::vector<int> csA = d->lvl_cs, csB(nlev);
  // (clusters stay within the portable size 8)
  for (int l = 0; l < nlev; ++l) csB[l] = csA[l] > 0 && csA[l] <= 4 ? csA[l] * 2 : csA[l];
  const bool mixed = c.opt.precision == D3M_MIXED;
  c.opt.update_kernel = 1;
  int rc = factor_any(c);
  auto total = [&]() {  // per-level time of everything but the assembly
    std::vector<double> t(nlev, 0.0);
    for (int l = 0; l < nlev; ++l)
      t[l] = d->tune_panel[l] + d->tune_update[l] + (d->tune_inv.empty() ? 0.0 : d->tune_inv[l]) +
             (d->tune_tc.empty() ? 0.0 : d->tune_tc[l]);
    return t;
  };
  std::vector<double> tA = total(), pA = d->tune_panel, tB(nlev, 1e300), pB(nlev, 1e300);
  // trial B (mixed): deferred tensor-core products, smallest cluster
  if (rc == D3M_OK && mixed) {
    c.opt.update_kernel = 2;
    rc = factor_any(c);
    tB = total();
    pB = d->tune_panel;
  }
  // trial C: doubled cluster, with the faster update scheme of each level
  if (rc == D3M_OK) {
    c.opt.update_kernel = 0;
    for (int l = 0; l < nlev; ++l) d->lvl_tc[l] = mixed && tB[l] < tA[l] ? 1 : 0;
    d->lvl_cs = csB;
    rc = factor_any(c);
  }
  std::vector<double> pC = d->tune_panel;
  c.opt.update_kernel = uk;
  d->prof.on = prof;
  d->lookahead_off = false;
  if (rc != D3M_OK) {
    d->lvl_cs = csA;
    return rc;
  }
  // cluster size per level: trial C's panels against the smallest cluster's
  // panels under the same update scheme (trial B for deferred levels, A else)
  int64_t ntc = 0, ncs2 = 0;
  for (int l = 0; l < nlev; ++l) {
    const double ref = d->lvl_tc[l] ? pB[l] : pA[l];
    d->lvl_cs[l] = pC[l] < ref ? csB[l] : csA[l];
    ntc += d->lvl_tc[l];
    ncs2 += d->lvl_cs[l] != csA[l];
  }
  c.stats.tuned_levels_tc = ntc;
  c.stats.tuned_levels_cs2 = ncs2;
  c.stats.ms_tuning =
      std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  d->tuned = true;
  tune_save(c);
  return D3M_OK;
}

int dev_factor(Ctx &c) {
  int rc = dev_init(c);
  if (rc) return rc;
  rc = enter(c);
  if (rc) return rc;
  if (!c.dev->tuned && c.opt.autotune == 0 && c.opt.panel_kernel != 1) {
    rc = autotune(c);
    if (rc) return rc;
  }
  rc = factor_any(c);
  c.factored = rc == D3M_OK;
  return rc;
}

static int ensure_rhs(Ctx &c, int r) {
  DeviceState *d = c.dev;
  if (d->cap >= r) return D3M_OK;
  const Plan &P = c.plan;
  for (void *p : {d->bM, d->zM, d->xM, d->Y, d->Y2, d->part, (void *)d->fe, (void *)d->xe, (void *)d->re, (void *)d->ucm,
                  (void *)d->lam, (void *)d->norms})
    if (p) {
      cudaFree(p);
      d->allocs.erase(std::remove(d->allocs.begin(), d->allocs.end(), p), d->allocs.end());
    }
  const size_t esz = d->precision == D3M_FP64 ? sizeof(cx<double>) : sizeof(cx<float>);
  auto A = [&](void **p, size_t bytes) -> cudaError_t {
    cudaError_t e = cudaMalloc(p, std::max<size_t>(bytes, 16));
    if (e == cudaSuccess) d->allocs.push_back(*p);
    return e;
  };
  for (cudaGraphExec_t *g : {&d->g_fwd, &d->g_bwd})
    if (*g) {
      cudaGraphExecDestroy(*g);
      *g = nullptr;
    }
  d->g_r = 0;
  CUDA_TRY(A(&d->bM, P.n_m * r * esz));
  CUDA_TRY(A(&d->zM, P.n_m * r * esz));
  CUDA_TRY(A(&d->xM, P.n_m * r * esz));
  CUDA_TRY(A(&d->Y, P.y_rows * r * esz));
  CUDA_TRY(A(&d->Y2, P.y_rows * r * esz));
  CUDA_TRY(A(&d->part, std::max<int64_t>(d->part_rows, 1) * r * esz));
  CUDA_TRY(A((void **)&d->fe, P.n_edges * r * sizeof(double2)));
  CUDA_TRY(A((void **)&d->xe, P.n_edges * r * sizeof(double2)));
  CUDA_TRY(A((void **)&d->re, P.n_edges * r * sizeof(double2)));
  CUDA_TRY(A((void **)&d->ucm, P.n_edges * r * sizeof(double2)));
  CUDA_TRY(A((void **)&d->lam, (int64_t)P.lm_edge.size() * r * sizeof(double2)));
  CUDA_TRY(A((void **)&d->norms, 2 * r * sizeof(double)));
  d->cap = r;
  return D3M_OK;
}

// Work lists of the solve GEMMs for r right-hand sides, per level:
//   forward   Y2[0:p] = L11^{-1} Y[0:p]                       (mixed factors)
//             Y[p:m] -= L21 y[0:p]   (y = Y2 mixed, Y fp64)
//   backward  part[q] = L21[split q]^T x[struct rows of split q]
//             Y2[0:p] = L11^{-T} Y[0:p]                       (mixed factors)
// Buffers: 0 arena, 1 L^{-1}, 2 Y, 3 Y2, 4 xM, 5 partials; B rows of the
// backward items are gathered through the fronts' update-row lists.
static int solve_items(Ctx &c, int r) {
  DeviceState *d = c.dev;
  if (d->sol_r == r && d->sol_items) return D3M_OK;
  const Plan &P = c.plan;
  const bool mixed = c.opt.precision == D3M_MIXED;
  const bool tcs = mixed && c.opt.solve_kernel == 0;  // complex64 products on the tensor cores
  std::vector<CgItem> items;
  std::vector<SkItem> skitems;
  int64_t skmax = 0;
  d->sol_lvl.assign(P.n_levels, {});
  d->sk_lvl.assign(P.n_levels, {});
  int BM = 128;
  auto tiles_of = [&](const CgItem &g) { return ((g.M + BM - 1) / BM) * ((g.N + CG_BN - 1) / CG_BN); };
  for (int l = 0; l < P.n_levels; ++l) {
    for (int kind = 0; kind < 4; ++kind) {
      // row tile of this launch: the fewest (efficiency-weighted) rows per SM
      // over the waves of CTAs (1 resident CTA per SM for 128-row tiles, 2 for
      // the smaller ones, by their register use)
      int best = 64;
      double bcost = 1e300;
      const bool tcl = tcs && tc_solve_launch(P, l, kind);  // this launch on the tensor cores
      for (int bm : {32, 64, 128}) {
        if (bm == 128 && !mixed) continue;
        if (tcl && bm != 128) continue;  // the tensor-core kernel's tiles are 128 rows
        BM = bm;
        int64_t t = 0;
        for (int i = P.level_ptr[l]; i < P.level_ptr[l + 1]; ++i) {
          const int f = P.level_fronts[i];
          const int pf = (int)(P.sn_end[f] - P.sn_start[f]);
          const int mf = pf + (int)(P.struct_ptr[f + 1] - P.struct_ptr[f]);
          const int M = kind == 1 ? mf - pf : pf;
          const int S = kind == 2 ? (mf - pf + BSPLIT - 1) / BSPLIT : 1;
          t += (int64_t)S * ((M + bm - 1) / bm) * ((r + CG_BN - 1) / CG_BN);
        }
        const int occ = bm == 128 ? 1 : 2;
        const double eff = bm == 128 ? 1.0 : bm == 64 ? 0.85 : 0.6;
        const double cost = (double)((t + 152 * occ - 1) / (152 * occ)) * bm / eff;
        if (cost < bcost) {
          bcost = cost;
          best = bm;
        }
      }
      BM = best;
      int first = (int)items.size(), tiles = 0;
      std::vector<CgItem> kitems;  // this launch's items before any split
      std::vector<int32_t> kfront;  // the front of each of them
      for (int i = P.level_ptr[l]; i < P.level_ptr[l + 1]; ++i) {
        const int f = P.level_fronts[i];
        const int pf = (int)(P.sn_end[f] - P.sn_start[f]);
        const int mf = pf + (int)(P.struct_ptr[f + 1] - P.struct_ptr[f]);
        CgItem g{};
        g.gath = -1;
        g.N = r;
        if (kind == 0 || kind == 3) {  // L11^{-1} (lower) or its transpose (upper)
          if (!mixed) continue;
          g.a = d->linv_off_h[i];
          if (kind == 0) {
            g.a_rs = 1; g.a_cs = pf; g.mode = 1;
          } else {
            g.a_rs = pf; g.a_cs = 1; g.mode = 3;
          }
          g.b = P.y_off[f] * r; g.b_rs = r; g.b_cs = 1;
          g.c = P.y_off[f] * r; g.c_rs = r; g.c_cs = 1;
          g.M = pf; g.K = pf;
          g.abuf = 1; g.bbuf = 2; g.cbuf = 3; g.beta = 0; g.alpha = 1.f;
          if (tcl) { g.qa = d->qblk_h[i][kind]; g.qnk = d->qnk_h[i][kind]; }
          kitems.push_back(g);
          kfront.push_back(f);
        } else if (kind == 1) {  // Y[p:m] -= L21 y[0:p]
          if (mf == pf || pf == 0) continue;
          g.a = P.front_off[f] + pf; g.a_rs = 1; g.a_cs = mf;
          g.b = P.y_off[f] * r; g.b_rs = r; g.b_cs = 1;
          g.c = (P.y_off[f] + pf) * r; g.c_rs = r; g.c_cs = 1;
          g.M = mf - pf; g.K = pf;
          g.abuf = 0; g.bbuf = mixed ? 3 : 2; g.cbuf = 2; g.beta = 1; g.alpha = -1.f;
          if (tcl) { g.qa = d->qblk_h[i][1]; g.qnk = d->qnk_h[i][1]; }
          kitems.push_back(g);
          kfront.push_back(f);
        } else {  // partials of L21^T x over row splits
          if (mf == pf || pf == 0) continue;
          const int S = (mf - pf + BSPLIT - 1) / BSPLIT;
          for (int q = 0; q < S; ++q) {
            CgItem h = g;
            const int rb = q * BSPLIT;
            h.a = P.front_off[f] + pf + rb; h.a_rs = mf; h.a_cs = 1;
            h.b = 0; h.b_rs = r; h.b_cs = 1; h.gath = P.struct_ptr[f] + rb;
            h.c = (d->part_off_h[i] + (int64_t)q * pf) * r; h.c_rs = r; h.c_cs = 1;
            h.M = pf; h.K = std::min(BSPLIT, mf - pf - rb);
            h.abuf = 0; h.bbuf = 4; h.cbuf = 5; h.beta = 0; h.alpha = 1.f;
            if (tcl) { h.qa = d->qblk_h[i][2] + rb / Q_BK; h.qnk = d->qnk_h[i][2]; }
            kitems.push_back(h);
            kfront.push_back(f);
          }
        }
      }
      // split-K for narrow launches with a long k range (the top levels of
      // the tree: few fronts, p of a few hundred): S pieces along k into the
      // partial buffer, added to their targets by k_splitk_reduce
      int64_t nt0 = 0, kmax = 0;
      for (const CgItem &g : kitems) {
        nt0 += tiles_of(g);
        kmax = std::max<int64_t>(kmax, g.K);
      }
      int S = 1;
      if (kind != 2 && nt0 > 0 && nt0 < 152 && kmax >= 96)
        S = (int)std::min<int64_t>({8, (304 + nt0 - 1) / nt0, kmax / 48});
      const int sk_first = (int)skitems.size();
      int64_t sk_elems = 0, pofs = 0;
      for (size_t ki = 0; ki < kitems.size(); ++ki) {
        const CgItem &g = kitems[ki];
        if (S <= 1) {
          CgItem h = g;
          h.tile0 = tiles;
          tiles += tiles_of(h);
          items.push_back(h);
          continue;
        }
        const int kq = tcl ? Q_BK : 16;  // the tensor-core pieces start on A-block boundaries
        const int Kc = ((g.K + S - 1) / S + kq - 1) / kq * kq;
        const int64_t mn = (int64_t)g.M * g.N;
        int pieces = 0;
        for (int kb = 0; kb < g.K; kb += Kc, ++pieces) {
          CgItem h = g;
          h.koff = kb;
          h.K = std::min(Kc, g.K - kb);
          h.qa = g.qa + kb / Q_BK;
          h.a += (int64_t)kb * g.a_cs;
          if (g.gath >= 0) h.gath += kb;
          else h.b += (int64_t)kb * g.b_rs;
          h.c = pofs + (int64_t)pieces * mn;
          h.c_rs = g.N;
          h.c_cs = 1;
          h.cbuf = 6;
          h.beta = 0;
          h.tile0 = tiles;
          tiles += tiles_of(h);
          items.push_back(h);
        }
        SkItem q{};
        q.c = g.c;
        q.p = pofs;
        q.c_rs = g.c_rs;
        q.c_cs = g.c_cs;
        q.M = g.M;
        q.N = g.N;
        q.S = pieces;
        q.cbuf = g.cbuf;
        q.beta = g.beta;
        q.elem0 = (int32_t)sk_elems;
        q.f = kfront[ki];
        skitems.push_back(q);
        sk_elems += mn;
        pofs += (int64_t)pieces * mn;
      }
      skmax = std::max(skmax, pofs);
      d->sk_lvl[l][3 * kind + 0] = sk_first;
      d->sk_lvl[l][3 * kind + 1] = (int)skitems.size() - sk_first;
      d->sk_lvl[l][3 * kind + 2] = (int)sk_elems;
      d->sol_lvl[l][4 * kind + 0] = first;
      d->sol_lvl[l][4 * kind + 1] = (int)items.size() - first;
      d->sol_lvl[l][4 * kind + 2] = tiles;
      d->sol_lvl[l][4 * kind + 3] = tcl ? 0 : BM;  // 0: k_tc_cgemm
    }
  }
  if (d->sol_items) {
    cudaFree(d->sol_items);
    d->allocs.erase(std::remove(d->allocs.begin(), d->allocs.end(), (void *)d->sol_items), d->allocs.end());
    d->sol_items = nullptr;
  }
  // tile -> item maps of every launch (an item's tiles run from its tile0 to
  // the next item's tile0, or to the launch's tile count)
  std::vector<int32_t> tmap;
  d->sol_tofs.assign(P.n_levels, {});
  for (int l = 0; l < P.n_levels; ++l)
    for (int kind = 0; kind < 4; ++kind) {
      const auto &sl = d->sol_lvl[l];
      const int first = sl[4 * kind], n = sl[4 * kind + 1], tiles = sl[4 * kind + 2];
      d->sol_tofs[l][kind] = (int64_t)tmap.size();
      for (int q = 0; q < n; ++q) {
        const int t1 = q + 1 < n ? items[first + q + 1].tile0 : tiles;
        for (int t = items[first + q].tile0; t < t1; ++t) tmap.push_back(q);
      }
    }
  if (d->sol_tmap) {
    cudaFree(d->sol_tmap);
    d->allocs.erase(std::remove(d->allocs.begin(), d->allocs.end(), (void *)d->sol_tmap), d->allocs.end());
    d->sol_tmap = nullptr;
  }
  if (tmap.empty()) tmap.push_back(0);
  CUDA_TRY(upload(d, &d->sol_tmap, tmap));
  if (items.empty()) items.push_back(CgItem{});
  CUDA_TRY(upload(d, &d->sol_items, items));
  for (void *q : {(void *)d->sk_items, d->skp})
    if (q) {
      cudaFree(q);
      d->allocs.erase(std::remove(d->allocs.begin(), d->allocs.end(), q), d->allocs.end());
    }
  d->sk_items = nullptr;
  d->skp = nullptr;
  if (skitems.empty()) skitems.push_back(SkItem{});
  CUDA_TRY(upload(d, &d->sk_items, skitems));
  const size_t esz = c.opt.precision == D3M_FP64 ? sizeof(cx<double>) : sizeof(cx<float>);
  CUDA_TRY(cudaMalloc(&d->skp, std::max<int64_t>(skmax, 1) * esz));
  d->allocs.push_back(d->skp);
  d->sol_r = r;
  return D3M_OK;
}

// x-extent of the grid of a per-front sweep kernel (256 threads, grid-strided
// over `work` elements of each of nf fronts): one element per thread up to
// about 2048 CTAs in all (every grid-stride step of these kernels is a chain
// of dependent loads), at least 64 CTAs per front.
static unsigned sweep_grid(int64_t work, int nf) {
  const int64_t cap = std::max<int64_t>(64, 2048 / std::max(1, nf));
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>((work + 255) / 256, cap));
}

// One pass of the factored operator: xM = M^{-1} bM (in the factor precision).
// dir: 1 forward sweep only, 2 backward sweep only, 3 both (eager).
template <typename T>
static int64_t apply_inverse(Ctx &c, int r, int dir = 3) {
  const Plan &P = c.plan;
  DeviceState *d = c.dev;
  cudaStream_t s = d->stream;
  FrontTab ft = tab(d);
  cx<T> *arena = (cx<T> *)d->arena;
  cx<T> *Y = (cx<T> *)d->Y;
  cx<T> *Y2 = (cx<T> *)d->Y2;
  cx<T> *Li = (cx<T> *)d->linv;
  const bool use_inv = sizeof(T) == 4;  // L11^{-1} exists for the mixed factors only
  // programmatic dependent launches on the mixed sweeps only: the fp64
  // sweep's long triangular-solve kernels ran slower beside the early
  // launched, waiting CTAs of their successors
  const bool pdl = sizeof(T) == 4;
  constexpr int RC = 8;
  const CgBufs<T> bufs{{arena, Li, Y, Y2, (cx<T> *)d->xM, (cx<T> *)d->part, (cx<T> *)d->skp}};
  // the split-K reduction of launch `kind` of level l (if that launch was split)
  auto reduce = [&](int l, int kind) -> int64_t {
    const auto &k3 = d->sk_lvl[l];
    if (k3[3 * kind + 1] == 0) return 0;
    const int64_t ne = k3[3 * kind + 2];
    launch_pdl(pdl, k_splitk_reduce<T>, dim3((unsigned)std::max<int64_t>(1, std::min<int64_t>((ne + 255) / 256, 1216))),
               dim3(256), 0, s, (const SkItem *)(d->sk_items + k3[3 * kind + 0]), k3[3 * kind + 1], ne, bufs,
               (const cx<T> *)d->skp);
    return 1;
  };
  // the split-K reduction of kind 0 (mode 0) or 3 (mode 3) fused with the
  // sweep step that follows it (k_splitk_reduce_sweep)
  auto reduce_sweep = [&](int l, int kind) {
    const auto &k3 = d->sk_lvl[l];
    const int64_t ne = k3[3 * kind + 2];
    launch_pdl(pdl, k_splitk_reduce_sweep<T>,
               dim3((unsigned)std::max<int64_t>(1, std::min<int64_t>((ne + 255) / 256, 1216))), dim3(256), 0, s,
               (const SkItem *)(d->sk_items + k3[3 * kind + 0]), k3[3 * kind + 1], ne, bufs, (const cx<T> *)d->skp,
               ft, (const double2 *)d->dinv_d, (const double2 *)d->dinv_o, (const int8_t *)d->psize,
               (const int32_t *)d->perm, (cx<T> *)d->zM, (cx<T> *)d->xM, r, kind);
  };
  int64_t nl = 0;
  if (dir & 1) {
  PROF_BEGIN(PC_FWD);
  for (int l = 0; l < P.n_levels; ++l) {
    const int nf = P.level_ptr[l + 1] - P.level_ptr[l];
    const int32_t *lvl = d->lvl_fronts + P.level_ptr[l];
    int64_t work = (int64_t)d->level_maxm[l] * r;
    ++nl;
    dim3 gi(sweep_grid(work, nf), nf);
    launch_pdl(pdl, k_fwd_gather<T>, gi, dim3(256), 0, s, lvl, ft, (const int32_t *)d->perm, (const cx<T> *)d->bM,
               (const int64_t *)d->g_ptr, (const int64_t *)d->g_src, Y, r);
    const auto &sl = d->sol_lvl[l];
    if (use_inv) {
      launch_cgemm<T>(sl[3], sl[2], d->sol_items + sl[0], sl[1], bufs, d->sidx, s, d->qpl,
                      d->sv_err, d->sv_wait_cap, d->sol_tmap + d->sol_tofs[l][0], pdl);
      if (d->sk_lvl[l][1] > 0) {  // split: the reduction also applies D^{-1}
        reduce_sweep(l, 0);
      } else {
        dim3 gdv(sweep_grid((int64_t)d->level_maxp[l] * r, nf), nf);
        launch_pdl(pdl, k_fwd_dinv<T>, gdv, dim3(256), 0, s, lvl, ft, (const double2 *)d->dinv_d,
                   (const double2 *)d->dinv_o, (const int8_t *)d->psize, (const cx<T> *)Y2, (cx<T> *)d->zM, r);
      }
    } else {
      dim3 gs((r + RC - 1) / RC, nf);
      launch_pdl(pdl, k_fwd_solve<T, RC>, gs, dim3(256), 0, s, lvl, ft, (const cx<T> *)arena, (const double2 *)d->dinv_d,
                 (const double2 *)d->dinv_o, (const int8_t *)d->psize, Y, (cx<T> *)d->zM, r);
    }
    nl += 2;
    if (sl[5] > 0) {
      launch_cgemm<T>(sl[7], sl[6], d->sol_items + sl[4], sl[5], bufs, d->sidx, s, d->qpl,
                      d->sv_err, d->sv_wait_cap, d->sol_tmap + d->sol_tofs[l][1], pdl);
      nl += reduce(l, 1);
      ++nl;
    }
  }
  PROF_END(PC_FWD);
  }
  if (dir & 2) {
  PROF_BEGIN(PC_BWD);
  for (int l = P.n_levels - 1; l >= 0; --l) {
    const int nf = P.level_ptr[l + 1] - P.level_ptr[l];
    const int32_t *lvl = d->lvl_fronts + P.level_ptr[l];
    const int32_t *ns = d->nsplit + P.level_ptr[l];
    const int64_t *po = d->part_off + P.level_ptr[l];
    const auto &sl = d->sol_lvl[l];
    if (sl[9] > 0) {
      launch_cgemm<T>(sl[11], sl[10], d->sol_items + sl[8], sl[9], bufs, d->sidx, s, d->qpl,
                      d->sv_err, d->sv_wait_cap, d->sol_tmap + d->sol_tofs[l][2], pdl);
      ++nl;
    }
    if (use_inv) {
      dim3 gw(sweep_grid((int64_t)d->level_maxp[l] * r, nf), nf);
      launch_pdl(pdl, k_bwd_w<T>, gw, dim3(256), 0, s, lvl, ft, ns, po, (const cx<T> *)d->part, (const cx<T> *)d->zM, Y,
                 r);
      launch_cgemm<T>(sl[15], sl[14], d->sol_items + sl[12], sl[13], bufs, d->sidx, s, d->qpl,
                      d->sv_err, d->sv_wait_cap, d->sol_tmap + d->sol_tofs[l][3], pdl);
      if (d->sk_lvl[l][3 * 3 + 1] > 0)  // split: the reduction also scatters x to xM
        reduce_sweep(l, 3);
      else
        launch_pdl(pdl, k_bwd_out<T>, gw, dim3(256), 0, s, lvl, ft, (const int32_t *)d->perm, (const cx<T> *)Y2,
                   (cx<T> *)d->xM, r);
      nl += 3;
    } else {
      dim3 gs((r + RC - 1) / RC, nf);
      launch_pdl(pdl, k_bwd_solve<T, RC>, gs, dim3(256), 0, s, lvl, ft, (const cx<T> *)arena, (const int32_t *)d->perm,
                 (const int8_t *)d->psize, ns, po, (const cx<T> *)d->part, Y, (const cx<T> *)d->zM, (cx<T> *)d->xM,
                 r);
      ++nl;
    }
  }
  PROF_END(PC_BWD);
  }
  return nl;
}

// The two sweeps of apply_inverse captured as CUDA graphs for r right-hand
// sides (rebuilt when r or the solve buffers change); each replay is timed
// with events on the stream when profiling.
template <typename T>
static int graph_sweeps(Ctx &c, int r) {
  DeviceState *d = c.dev;
  if (d->g_r == r && d->g_fwd && d->g_bwd) return D3M_OK;
  for (cudaGraphExec_t *g : {&d->g_fwd, &d->g_bwd})
    if (*g) {
      cudaGraphExecDestroy(*g);
      *g = nullptr;
    }
  const bool prof = d->prof.on;
  d->prof.on = false;  // no event nodes inside the graphs
  for (int dir = 1; dir <= 2; ++dir) {
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(d->stream, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      d->g_launches[dir - 1] = apply_inverse<T>(c, r, dir);
      e = cudaStreamEndCapture(d->stream, &g);
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(dir == 1 ? &d->g_fwd : &d->g_bwd, g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      d->prof.on = prof;
      c.err = std::string("CUDA graph capture of the substitution failed: ") + cudaGetErrorString(e);
      return D3M_ECUDA;
    }
  }
  d->prof.on = prof;
  d->g_r = r;
  return D3M_OK;
}

template <typename T>
static int64_t run_sweeps(Ctx &c, int r) {
  DeviceState *d = c.dev;
  cudaStream_t s = d->stream;
  {
    PROF_BEGIN(PC_FWD);
    cudaGraphLaunch(d->g_fwd, s);
    PROF_END(PC_FWD);
  }
  {
    PROF_BEGIN(PC_BWD);
    cudaGraphLaunch(d->g_bwd, s);
    PROF_END(PC_BWD);
  }
  return d->g_launches[0] + d->g_launches[1];
}

static unsigned grid1(int64_t n) { return (unsigned)std::min<int64_t>((n + 255) / 256, 152 * 16); }

static int gmres_buffers(Ctx &c, int r, int m) {
  DeviceState *d = c.dev;
  if (d->gm_r >= r && d->gm_m >= m) return D3M_OK;
  for (void *p : {(void *)d->gm_V, (void *)d->gm_Z, (void *)d->gm_lamZ, (void *)d->gm_w, (void *)d->gm_y,
                  (void *)d->gm_h, (void *)d->gm_s})
    if (p) {
      cudaFree(p);
      d->allocs.erase(std::remove(d->allocs.begin(), d->allocs.end(), p), d->allocs.end());
    }
  const int64_t n = c.plan.n_edges, nlm = std::max<int64_t>((int64_t)c.plan.lm_edge.size(), 1);
  CUDA_TRY(dalloc(d, &d->gm_V, (size_t)(m + 1) * n * r));
  CUDA_TRY(dalloc(d, &d->gm_Z, (size_t)m * n * r));
  CUDA_TRY(dalloc(d, &d->gm_lamZ, (size_t)m * nlm * r));
  CUDA_TRY(dalloc(d, &d->gm_w, (size_t)n * r));
  CUDA_TRY(dalloc(d, &d->gm_y, (size_t)m * r));
  CUDA_TRY(dalloc(d, &d->gm_h, (size_t)2 * (m + 1) * r));
  CUDA_TRY(dalloc(d, &d->gm_s, (size_t)r));
  d->gm_r = r;
  d->gm_m = m;
  return D3M_OK;
}

// One GMRES-IR correction: solve A d = re (the current fp64 residual) by
// flexible GMRES with right preconditioner M^{-1} (the factors, through the
// substitution sweeps) to a relative 2-norm reduction gmres_tol per column,
// at most gmres_restart steps, then x += d and lambda += its multipliers.
// Adds the Krylov steps taken to `inner`.
template <typename T>
static int gmres_correction(Ctx &c, int r, int &inner, int64_t &nl) {
  DeviceState *d = c.dev;
  const Plan &P = c.plan;
  cudaStream_t s = d->stream;
  const int m = c.opt.gmres_restart;
  const int64_t n = P.n_edges, nlm = (int64_t)P.lm_edge.size();
  const int64_t vst = n * r, lst = std::max<int64_t>(nlm, 1) * r;
  const size_t esz = sizeof(cx<T>);
  int rc = gmres_buffers(c, r, m);
  if (rc) return rc;
  const unsigned gd = (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 511) / 512, 304));
  auto dots = [&](int nv, const double2 *V, const double2 *w) -> int {  // -> d->gm_h
    CUDA_TRY(cudaMemsetAsync(d->gm_h, 0, sizeof(double) * 2 * nv * r, s));
    k_dots<<<gd, 256, 0, s>>>(n, r, nv, V, vst, w, d->gm_h);
    ++nl;
    return D3M_OK;
  };
  std::vector<double> hh(2 * (m + 1) * r), h1(2 * (m + 1) * r);
  // v_0 = r / beta
  k_mask_rows<<<grid1(n * r), 256, 0, s>>>(n, r, d->pec, d->re);
  if ((rc = dots(1, d->re, d->re))) return rc;
  CUDA_TRY(cudaMemcpyAsync(hh.data(), d->gm_h, sizeof(double) * 2 * r, cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  std::vector<double> beta(r), sc(r);
  for (int q = 0; q < r; ++q) {
    beta[q] = std::sqrt(std::max(hh[2 * q], 0.0));
    sc[q] = beta[q] > 0 ? 1.0 / beta[q] : 0.0;
  }
  CUDA_TRY(cudaMemcpyAsync(d->gm_s, sc.data(), sizeof(double) * r, cudaMemcpyHostToDevice, s));
  k_scale_cols<<<grid1(n * r), 256, 0, s>>>(n, r, d->re, d->gm_s, d->gm_V);
  nl += 3;
  // per column: Hessenberg (column-major (m+1) x m), Givens rotations, g
  std::vector<cplx> H((size_t)(m + 1) * m * r, 0.0), cs((size_t)m * r, 0.0), sn((size_t)m * r, 0.0),
      g((size_t)(m + 1) * r, 0.0);
  for (int q = 0; q < r; ++q) g[(size_t)q * (m + 1)] = beta[q];
  int kdone = 0;
  for (int k = 0; k < m; ++k) {
    double2 *Vk = d->gm_V + (int64_t)k * vst, *Zk = d->gm_Z + (int64_t)k * vst;
    // z_k = M^{-1} v_k (and its multiplier part)
    CUDA_TRY(cudaMemsetAsync(d->bM, 0, P.n_m * r * esz, s));
    k_scatter<T><<<grid1(n * r), 256, 0, s>>>(Vk, d->owner, (cx<T> *)d->bM, n, r);
    nl += run_sweeps<T>(c, r) + 1;
    k_gather<T><<<grid1(n * r), 256, 0, s>>>((const cx<T> *)d->xM, d->owner, Zk, n, r, 0);
    if (nlm)
      k_lambda_acc<T><<<grid1(nlm * r), 256, 0, s>>>((const cx<T> *)d->xM, P.lam_start, nlm, r,
                                                     d->gm_lamZ + (int64_t)k * lst, 0);
    // w = A z_k, orthogonalised twice against v_0..v_k
    const unsigned gs = (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 7) / 8, 152 * 8));
    k_spmv<<<gs, 256, 0, s>>>(n, d->csr_ptr, d->csr_col, d->csr_re, d->csi_ptr, d->csi_col, d->csi_val, Zk, d->gm_w,
                               r);
    nl += 3;
    for (int pass = 0; pass < 2; ++pass) {
      if ((rc = dots(k + 1, d->gm_V, d->gm_w))) return rc;
      k_sub_many<<<grid1(n * r), 256, 0, s>>>(n, r, k + 1, d->gm_V, vst, (const double2 *)d->gm_h, d->gm_w);
      CUDA_TRY(cudaMemcpyAsync(pass == 0 ? h1.data() : hh.data(), d->gm_h, sizeof(double) * 2 * (k + 1) * r,
                               cudaMemcpyDeviceToHost, s));
      ++nl;
    }
    if ((rc = dots(1, d->gm_w, d->gm_w))) return rc;
    std::vector<double> nn(2 * r);
    CUDA_TRY(cudaMemcpyAsync(nn.data(), d->gm_h, sizeof(double) * 2 * r, cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    bool all = true;
    for (int q = 0; q < r; ++q) {
      const double hn = std::sqrt(std::max(nn[2 * q], 0.0));
      sc[q] = hn > 0 ? 1.0 / hn : 0.0;
      if (beta[q] == 0) continue;
      cplx *Hq = &H[(size_t)q * (m + 1) * m + (size_t)k * (m + 1)];
      for (int i = 0; i <= k; ++i)
        Hq[i] = cplx(h1[2 * ((size_t)i * r + q)] + hh[2 * ((size_t)i * r + q)],
                     h1[2 * ((size_t)i * r + q) + 1] + hh[2 * ((size_t)i * r + q) + 1]);
      Hq[k + 1] = hn;
      cplx *cq = &cs[(size_t)q * m], *sq = &sn[(size_t)q * m], *gq = &g[(size_t)q * (m + 1)];
      for (int i = 0; i < k; ++i) {  // earlier rotations
        const cplx t = cq[i] * Hq[i] + sq[i] * Hq[i + 1];
        Hq[i + 1] = -std::conj(sq[i]) * Hq[i] + std::conj(cq[i]) * Hq[i + 1];
        Hq[i] = t;
      }
      const cplx a = Hq[k], b = Hq[k + 1];
      const double den = std::sqrt(std::norm(a) + std::norm(b));
      if (den == 0) {
        cq[k] = 1.0;
        sq[k] = 0.0;
      } else {
        cq[k] = std::conj(a) / den;
        sq[k] = std::conj(b) / den;
      }
      Hq[k] = cq[k] * a + sq[k] * b;
      Hq[k + 1] = 0.0;
      gq[k + 1] = -std::conj(sq[k]) * gq[k];
      gq[k] = cq[k] * gq[k];
      if (std::abs(gq[k + 1]) > c.opt.gmres_tol * beta[q] && Hq[k] != cplx(0.0)) all = false;
    }
    CUDA_TRY(cudaMemcpyAsync(d->gm_s, sc.data(), sizeof(double) * r, cudaMemcpyHostToDevice, s));
    k_scale_cols<<<grid1(n * r), 256, 0, s>>>(n, r, d->gm_w, d->gm_s, d->gm_V + (int64_t)(k + 1) * vst);
    nl += 2;
    ++inner;
    kdone = k + 1;
    if (all) break;
  }
  // y = H^{-1} g per column (upper triangular), then x += Z y, lambda += ...
  std::vector<double> yv(2 * (size_t)kdone * r, 0.0);
  for (int q = 0; q < r; ++q) {
    if (beta[q] == 0) continue;
    const cplx *Hq = &H[(size_t)q * (m + 1) * m];
    std::vector<cplx> y(kdone);
    for (int i = kdone - 1; i >= 0; --i) {
      cplx acc = g[(size_t)q * (m + 1) + i];
      for (int j = i + 1; j < kdone; ++j) acc -= Hq[(size_t)j * (m + 1) + i] * y[j];
      const cplx dg = Hq[(size_t)i * (m + 1) + i];
      y[i] = dg != cplx(0.0) ? acc / dg : cplx(0.0);
    }
    for (int i = 0; i < kdone; ++i) {
      yv[2 * ((size_t)i * r + q)] = y[i].real();
      yv[2 * ((size_t)i * r + q) + 1] = y[i].imag();
    }
  }
  CUDA_TRY(cudaMemcpyAsync(d->gm_y, yv.data(), yv.size() * sizeof(double), cudaMemcpyHostToDevice, s));
  k_add_combo<<<grid1(n * r), 256, 0, s>>>(n, r, kdone, d->gm_Z, vst, d->gm_y, d->xe);
  if (nlm) k_add_combo<<<grid1(nlm * r), 256, 0, s>>>(nlm, r, kdone, d->gm_lamZ, lst, d->gm_y, d->lam);
  nl += 2;
  CUDA_TRY(cudaStreamSynchronize(s));  // the host vectors above outlive their copies
  return D3M_OK;
}

template <typename T>
static int solve_t(Ctx &c, const double *rhs, int64_t ldb, double *x, int64_t ldx, int r,
                   d3m_solve_info *info, bool host_ptrs, bool adjoint) {
  const int cj = adjoint ? 1 : 0;
  const Plan &P = c.plan;
  DeviceState *d = c.dev;
  cudaStream_t s = d->stream;
  const int64_t n = P.n_edges;
  const int64_t nlm = (int64_t)P.lm_edge.size();
  const size_t esz = sizeof(cx<T>);
  // user RHS -> row-major fp64 edge vector fe
  if (host_ptrs) {
    CUDA_TRY(cudaMemcpy2DAsync(d->ucm, n * sizeof(double2), rhs, ldb * sizeof(double2), n * sizeof(double2), r,
                               cudaMemcpyHostToDevice, s));
    k_cm_to_rm<<<grid1(n * r), 256, 0, s>>>(d->ucm, n, d->fe, n, r, cj);
  } else {
    k_cm_to_rm<<<grid1(n * r), 256, 0, s>>>((const double2 *)rhs, ldb, d->fe, n, r, cj);
  }
  CUDA_TRY(cudaMemsetAsync(d->sv_err, 0, sizeof(int32_t), s));
  // first solve from f
  d->prof.reset();
  int64_t nl = 3;
  int napply = 1;
  CUDA_TRY(cudaMemsetAsync(d->bM, 0, P.n_m * r * esz, s));
  k_scatter<T><<<grid1(n * r), 256, 0, s>>>(d->fe, d->owner, (cx<T> *)d->bM, n, r);
  {
    int grc = graph_sweeps<T>(c, r);
    if (grc) return grc;
  }
  nl += run_sweeps<T>(c, r);
  k_gather<T><<<grid1(n * r), 256, 0, s>>>((const cx<T> *)d->xM, d->owner, d->xe, n, r, 0);
  if (nlm) k_lambda_acc<T><<<grid1(nlm * r), 256, 0, s>>>((const cx<T> *)d->xM, P.lam_start, nlm, r, d->lam, 0);
  std::vector<double> nh(2 * r);
  int iters = 0, inner = 0;
  double maxres = 0;
  const bool refine = d->precision == D3M_MIXED;
  for (;;) {
    // max |r|^2 per column each time, max |f|^2 on the first pass only
    const bool first = iters == 0;
    CUDA_TRY(cudaMemsetAsync(d->norms, 0, (first ? 2 : 1) * r * sizeof(double), s));
    {
      PROF_BEGIN(PC_RESID);
      const int smem_max = r <= 2048;
      const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 7) / 8, 152 * 8));
      k_residual<<<grid, 256, smem_max ? 2 * r * sizeof(double) : 0, s>>>(
          n, d->csr_ptr, d->csr_col, d->csr_re, d->csi_ptr, d->csi_col, d->csi_val, d->xe, d->fe, d->re, r, d->norms, first ? d->norms + r : nullptr,
          smem_max);
      PROF_END(PC_RESID);
    }
    ++nl;
    CUDA_TRY(cudaMemcpyAsync(nh.data(), d->norms, (first ? 2 : 1) * r * sizeof(double), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    maxres = 0;
    for (int q = 0; q < r; ++q) {
      const double rn = std::sqrt(nh[q]), fn = std::sqrt(nh[r + q]);
      double rr = fn > 0 ? rn / fn : rn;
      if (info && info->resid) info->resid[q] = rr;
      maxres = std::max(maxres, rr);
    }
    if (!refine || maxres <= c.opt.refine_tol || iters >= c.opt.max_refine || !std::isfinite(maxres)) break;
    if (c.opt.refine_method == 1) {
      // GMRES-IR correction (flexible GMRES on A d = r, preconditioned by the factors)
      const int before = inner;
      const int grc = gmres_correction<T>(c, r, inner, nl);
      if (grc) return grc;
      napply += inner - before;
    } else {
      // correction: solve with the residual, accumulate in fp64
      CUDA_TRY(cudaMemsetAsync(d->bM, 0, P.n_m * r * esz, s));
      k_scatter<T><<<grid1(n * r), 256, 0, s>>>(d->re, d->owner, (cx<T> *)d->bM, n, r);
      nl += run_sweeps<T>(c, r) + 3;
      ++napply;
      k_gather<T><<<grid1(n * r), 256, 0, s>>>((const cx<T> *)d->xM, d->owner, d->xe, n, r, 1);
      if (nlm) k_lambda_acc<T><<<grid1(nlm * r), 256, 0, s>>>((const cx<T> *)d->xM, P.lam_start, nlm, r, d->lam, 1);
    }
    ++iters;
  }
  if (host_ptrs) {
    k_rm_to_cm<<<grid1(n * r), 256, 0, s>>>(d->xe, d->ucm, n, n, r, d->pec, cj);
    CUDA_TRY(cudaMemcpy2DAsync(x, ldx * sizeof(double2), d->ucm, n * sizeof(double2), n * sizeof(double2), r,
                               cudaMemcpyDeviceToHost, s));
  } else {
    k_rm_to_cm<<<grid1(n * r), 256, 0, s>>>(d->xe, (double2 *)x, ldx, n, r, d->pec, cj);
  }
  CUDA_TRY(cudaGetLastError());
  CUDA_TRY(cudaStreamSynchronize(s));
  int32_t sve = 0;
  CUDA_TRY(cudaMemcpy(&sve, d->sv_err, sizeof sve, cudaMemcpyDeviceToHost));
  if (sve) {
    c.err = "d3m_solve: a tensor-core substitution tile gave up a bounded wait (its results were discarded)";
    return D3M_ETIMEOUT;
  }
  if (info) {
    info->iters = iters;
    info->max_resid = maxres;
    info->inner_iters = inner;
  }
  c.stats.launches_solve = nl + 2;
  c.stats.solve_flops = d->solve_flops_per_rhs * r * napply;
  if (d->prof.on) {
    double ms[PC_N];
    d->prof.collect(ms);
    c.stats.ms_fwd = ms[PC_FWD];
    c.stats.ms_bwd = ms[PC_BWD];
    c.stats.ms_residual = ms[PC_RESID];
  }
  c.lambda_nrhs = 0;
  if (!std::isfinite(maxres)) {
    c.err = "d3m_solve: the residual is not finite (non-finite input or factors)";
    return D3M_ENOCONV;
  }
  if (refine && maxres > c.opt.refine_tol) {
    char buf[128];
    snprintf(buf, sizeof buf, "d3m_solve: refinement stopped at residual %.3e after %d steps", maxres, iters);
    c.err = buf;
    return D3M_ENOCONV;
  }
  return D3M_OK;
}

int dev_solve(Ctx &c, const double *rhs, int64_t ldb, double *x, int64_t ldx, int nrhs, d3m_solve_info *info,
              bool host_ptrs, bool adjoint) {
  if (!c.factored) {
    c.err = "d3m_solve: call d3m_factor first";
    return D3M_ESTATE;
  }
  int rc = ensure_rhs(c, nrhs);
  if (rc) return rc;
  rc = solve_items(c, nrhs);
  if (rc) return rc;
  rc = enter(c);
  if (rc) return rc;
  rc = c.opt.precision == D3M_FP64 ? solve_t<double>(c, rhs, ldb, x, ldx, nrhs, info, host_ptrs, adjoint)
                                   : solve_t<float>(c, rhs, ldb, x, ldx, nrhs, info, host_ptrs, adjoint);
  // keep the multipliers for d3m_structure(D3M_LAMBDA)
  const int64_t nlm = (int64_t)c.plan.lm_edge.size();
  if (rc == D3M_OK || rc == D3M_ENOCONV) {
    std::vector<double2> tmp(nlm * nrhs);
    if (nlm) {
      cudaError_t e = cudaMemcpy(tmp.data(), c.dev->lam, nlm * nrhs * sizeof(double2), cudaMemcpyDeviceToHost);
      if (e != cudaSuccess) {
        c.err = cudaGetErrorString(e);
        return D3M_ECUDA;
      }
    }
    c.lambda_host.assign(nlm * nrhs, cplx(0));
    for (int64_t l = 0; l < nlm; ++l)
      for (int q = 0; q < nrhs; ++q) c.lambda_host[l + nlm * q] = cplx(tmp[l * nrhs + q].x, tmp[l * nrhs + q].y);
    c.lambda_nrhs = nrhs;
  }
  return rc;
}

int dev_grad_eps(Ctx &c, const double *x, int64_t ldx, const double *y, int64_t ldy, int nrhs, double *grad) {
  int rc = dev_init(c);
  if (rc) return rc;
  rc = enter(c);
  if (rc) return rc;
  const Plan &P = c.plan;
  cudaStream_t s = c.dev->stream;
  const int64_t ncell = P.n_cells;
  if (P.element != D3M_BRICK) {
    DeviceState *d = c.dev;
    if (!d->gc_edge) {
      const int ne = P.cell_ne;
      std::vector<int64_t> ce((size_t)ncell * ne);
      std::vector<double> cm((size_t)ncell * ne * ne);
      double M[MAX_CELL_NE][MAX_CELL_NE];
      for (int64_t cc = 0; cc < ncell; ++cc) {
        int64_t e[MAX_CELL_NE];
        cell_dofs_mass(P, cc, e, M);
        for (int a = 0; a < ne; ++a) {
          ce[cc * ne + a] = e[a];
          for (int b = 0; b < ne; ++b) cm[(cc * ne + a) * ne + b] = M[a][b];
        }
      }
      CUDA_TRY(upload(d, &d->gc_edge, ce));
      CUDA_TRY(upload(d, &d->gc_mass, cm));
    }
    k_grad_eps_cells<<<grid1(ncell), 128, 0, s>>>(ncell, P.cell_ne, d->gc_edge, d->gc_mass, P.k * P.k,
                                                 (const double2 *)x, ldx, (const double2 *)y, ldy, nrhs, d->pec,
                                                 grad);
  } else {
    ElemMass Me;
    double S[12][12];
    element_matrices(P.h, S, Me.M);
    k_grad_eps<<<grid1(ncell), 256, 0, s>>>(P.nx, P.ny, P.nz, P.k * P.k, Me, (const double2 *)x, ldx,
                                            (const double2 *)y, ldy, nrhs, c.dev->pec, grad);
  }
  CUDA_TRY(cudaGetLastError());
  CUDA_TRY(cudaStreamSynchronize(s));
  return D3M_OK;
}

void dev_free(Ctx &c) {
  if (!c.dev) return;
  for (cudaGraphExec_t g : {c.dev->g_fwd, c.dev->g_bwd, c.dev->g_factor})
    if (g) cudaGraphExecDestroy(g);
  if (c.dev->stream_b) {
    cudaStreamSynchronize(c.dev->stream_b);
    cudaStreamDestroy(c.dev->stream_b);
    for (int q = 0; q < 3; ++q) {
      cudaEventDestroy(c.dev->ev_step[q]);
      cudaEventDestroy(c.dev->ev_schur[q]);
    }
    cudaEventDestroy(c.dev->ev_b);
  }
  if (c.dev->stream_c) {
    cudaStreamSynchronize(c.dev->stream_c);
    cudaStreamDestroy(c.dev->stream_c);
    cudaEventDestroy(c.dev->ev_lvl);
    cudaEventDestroy(c.dev->ev_c);
  }
  if (c.dev->own_stream) {
    cudaStreamSynchronize(c.dev->stream);
    cudaStreamDestroy(c.dev->stream);
    cudaEventDestroy(c.dev->legacy_ev);
  }
  for (void *p : c.dev->allocs) cudaFree(p);
  delete c.dev;
  c.dev = nullptr;
}

// ------------------------------------------------------------ dense entry
int dense_ldlt(int m, int p, int batch, double *A, int32_t *perm, double *dinv, int32_t *info, void *stream,
               int panel_kernel, std::string &err) {
  cudaStream_t s = (cudaStream_t)stream;
  std::vector<int32_t> fm(batch, m), fp(batch, p), par(batch, -1), lvl(batch);
  std::vector<int64_t> off(batch), piv(batch), wofs(batch), zero(batch, 0);
  for (int b = 0; b < batch; ++b) {
    lvl[b] = b;
    off[b] = (int64_t)b * m * m;
    piv[b] = (int64_t)b * p;
    wofs[b] = (int64_t)b * m * NB;
  }
  DeviceState tmp;
  Ctx c;  // for CUDA_TRY error text
  auto fail = [&](int rc) {
    for (void *q : tmp.allocs) cudaFree(q);
    err = c.err;
    return rc;
  };
#define DTRY(call)                                                       \
  do {                                                                   \
    cudaError_t e_ = (call);                                             \
    if (e_ != cudaSuccess) {                                             \
      c.err = std::string("CUDA error ") + cudaGetErrorString(e_);       \
      return fail(D3M_ECUDA);                                            \
    }                                                                    \
  } while (0)
  DTRY(upload(&tmp, &tmp.f_m, fm));
  DTRY(upload(&tmp, &tmp.f_p, fp));
  DTRY(upload(&tmp, &tmp.f_parent, par));
  DTRY(upload(&tmp, &tmp.f_off, off));
  DTRY(upload(&tmp, &tmp.f_piv, piv));
  DTRY(upload(&tmp, &tmp.f_soff, zero));
  DTRY(upload(&tmp, &tmp.f_start, zero));
  DTRY(upload(&tmp, &tmp.f_y, zero));
  DTRY(upload(&tmp, &tmp.lvl_fronts, lvl));
  DTRY(upload(&tmp, &tmp.wofs, wofs));
  cx<double> *W = nullptr;
  DTRY(dalloc(&tmp, &W, (size_t)batch * m * NB));
  int32_t *pv = nullptr, *k0 = nullptr, *kb = nullptr;
  int2 *swp = nullptr;
  double2 *dd = nullptr, *dof = nullptr;
  int8_t *ps = nullptr;
  double *mp = nullptr;
  DTRY(dalloc(&tmp, &pv, (size_t)batch * p));
  DTRY(dalloc(&tmp, &dd, (size_t)batch * p));
  DTRY(dalloc(&tmp, &dof, (size_t)batch * p));
  DTRY(dalloc(&tmp, &ps, (size_t)batch * p));
  DTRY(dalloc(&tmp, &k0, batch));
  DTRY(dalloc(&tmp, &kb, batch));
  DTRY(dalloc(&tmp, &mp, batch));
  DTRY(dalloc(&tmp, &swp, (size_t)batch * 2 * NB));
  int2 *snap = nullptr;
  DTRY(dalloc(&tmp, &snap, batch));
  DTRY(cudaMemsetAsync(k0, 0, batch * sizeof(int32_t), s));
  DTRY(cudaMemsetAsync(kb, 0, batch * sizeof(int32_t), s));
  DTRY(cudaMemsetAsync(info, 0, batch * sizeof(int32_t), s));
  k_fill_double<<<(batch + 255) / 256, 256, 0, s>>>(mp, batch, 1e300);
  FrontTab ft = tab(&tmp);
  k_init_perm<<<batch, 128, 0, s>>>(batch, tmp.f_p, tmp.f_piv, pv);
  int steps = (p + NB - 2) / (NB - 1);
  cx<double> *arena = (cx<double> *)A;
  for (int stp = 0; stp < steps; ++stp) {
    int cs = panel_kernel == 1 ? 0 : panel_cluster_size(p, sizeof(cx<double>));
    DTRY(launch_panel<double>(cs, p, m, batch, tmp.lvl_fronts, ft, tmp.wofs, arena, W, pv, dd, dof, ps, k0, kb, info,
                              mp, nullptr, swp, snap, s));
    int cmin = std::min(p, (stp + 1) * (NB - 1));
    int nt = (m + UT - 1) / UT - cmin / UT;
    dim3 g(std::max(1, nt * (nt + 1) / 2), batch);
    k_update<double><<<g, 256, 0, s>>>(tmp.lvl_fronts, ft, tmp.wofs, arena, W, snap, 0);
  }
  DTRY(cudaGetLastError());
  DTRY(cudaStreamSynchronize(s));
  // outputs
  std::vector<int32_t> hp((size_t)batch * p), out((size_t)batch * m);
  std::vector<double2> hd((size_t)batch * p), ho((size_t)batch * p);
  std::vector<int8_t> hs((size_t)batch * p);
  DTRY(cudaMemcpy(hp.data(), pv, hp.size() * 4, cudaMemcpyDeviceToHost));
  DTRY(cudaMemcpy(hd.data(), dd, hd.size() * 16, cudaMemcpyDeviceToHost));
  DTRY(cudaMemcpy(ho.data(), dof, ho.size() * 16, cudaMemcpyDeviceToHost));
  DTRY(cudaMemcpy(hs.data(), ps, hs.size(), cudaMemcpyDeviceToHost));
  std::vector<double> hdi((size_t)batch * p * 6);
  for (int b = 0; b < batch; ++b) {
    for (int i = 0; i < m; ++i) out[(size_t)b * m + i] = i < p ? hp[(size_t)b * p + i] : i;
    for (int i = 0; i < p; ++i) {
      size_t q = (size_t)b * p + i;
      hdi[6 * q + 0] = hd[q].x;
      hdi[6 * q + 1] = hd[q].y;
      hdi[6 * q + 2] = ho[q].x;
      hdi[6 * q + 3] = ho[q].y;
      hdi[6 * q + 4] = hs[q];
      hdi[6 * q + 5] = 0;
    }
  }
  DTRY(cudaMemcpy(perm, out.data(), out.size() * 4, cudaMemcpyHostToDevice));
  DTRY(cudaMemcpy(dinv, hdi.data(), hdi.size() * 8, cudaMemcpyHostToDevice));
  for (void *q : tmp.allocs) cudaFree(q);
  return D3M_OK;
#undef DTRY
}

// ------------------------------------------------------------ allocation-free dense entry
// Scratch of d3m_dense_ldlt_noalloc: one fixed array in the library image.
// Host code must not use g_noalloc_scratch's name as an address (it is a
// host-side shadow); its device address is looked up once per device.
static __device__ __align__(256) unsigned char g_noalloc_scratch[D3M_NOALLOC_SCRATCH_BYTES];
constexpr int NOALLOC_MAX_DEVICES = 64;
static void *g_noalloc_addr[NOALLOC_MAX_DEVICES] = {};

struct NoallocLayout {
  size_t f_m, f_p, f_parent, lvl, f_off, f_piv, f_zero, wofs, W, pv, dd, dof, k0, kb, mp, ps, swp, snap, total;
};
static NoallocLayout noalloc_layout(int m, int p, int batch) {
  NoallocLayout L{};
  size_t o = 0;
  auto take = [&](size_t bytes) {
    size_t at = o;
    o += (bytes + 255) / 256 * 256;
    return at;
  };
  const size_t b = (size_t)batch, pp = (size_t)std::max(p, 1);
  L.f_m = take(4 * b);
  L.f_p = take(4 * b);
  L.f_parent = take(4 * b);
  L.lvl = take(4 * b);
  L.f_off = take(8 * b);
  L.f_piv = take(8 * b);
  L.f_zero = take(8 * b);
  L.wofs = take(8 * b);
  L.W = take(sizeof(cx<double>) * b * (size_t)m * NB);
  L.pv = take(4 * b * pp);
  L.dd = take(16 * b * pp);
  L.dof = take(16 * b * pp);
  L.k0 = take(4 * b);
  L.kb = take(4 * b);
  L.mp = take(8 * b);
  L.ps = take(b * pp);
  L.swp = take(8 * b * 2 * NB);
  L.snap = take(8 * b);
  L.total = o;
  return L;
}

__global__ void k_noalloc_init(int m, int p, int batch, int32_t *fm, int32_t *fp, int32_t *par, int32_t *lvl,
                               int64_t *off, int64_t *piv, int64_t *zero, int64_t *wofs, int32_t *k0, int32_t *kb,
                               int32_t *info, double *mp, int32_t *pv) {
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < batch; b += gridDim.x * blockDim.x) {
    fm[b] = m;
    fp[b] = p;
    par[b] = -1;
    lvl[b] = b;
    off[b] = (int64_t)b * m * m;
    piv[b] = (int64_t)b * p;
    zero[b] = 0;
    wofs[b] = (int64_t)b * m * NB;
    k0[b] = 0;
    kb[b] = 0;
    info[b] = 0;
    mp[b] = 1e300;
  }
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < (int64_t)batch * p;
       q += (int64_t)gridDim.x * blockDim.x)
    pv[q] = (int32_t)(q % p);
}

__global__ void k_noalloc_out(int m, int p, int batch, const int32_t *pv, const double2 *dd, const double2 *dof,
                              const int8_t *ps, int32_t *perm, double *dinv) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < (int64_t)batch * m;
       q += (int64_t)gridDim.x * blockDim.x) {
    int64_t b = q / m;
    int i = (int)(q % m);
    perm[q] = i < p ? pv[b * p + i] : i;
  }
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < (int64_t)batch * p;
       q += (int64_t)gridDim.x * blockDim.x) {
    dinv[6 * q + 0] = dd[q].x;
    dinv[6 * q + 1] = dd[q].y;
    dinv[6 * q + 2] = dof[q].x;
    dinv[6 * q + 3] = dof[q].y;
    dinv[6 * q + 4] = ps[q];
    dinv[6 * q + 5] = 0.0;
  }
}

static int dense_ldlt_noalloc(int m, int p, int batch, double *A, int32_t *perm, double *dinv, int32_t *info,
                              void *stream) {
  const NoallocLayout Lo = noalloc_layout(m, p, batch);
  if (Lo.total > (size_t)D3M_NOALLOC_SCRATCH_BYTES) return D3M_EINVAL;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return D3M_ECUDA;
  if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return D3M_EINVAL;
  if (!g_noalloc_addr[dev]) {  // once per device, with that device current
    void *ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) return D3M_ECUDA;
    g_noalloc_addr[dev] = ptr;
  }
  unsigned char *base = static_cast<unsigned char *>(g_noalloc_addr[dev]);
  cudaStream_t s = (cudaStream_t)stream;
  FrontTab ft;
  ft.m = reinterpret_cast<int32_t *>(base + Lo.f_m);
  ft.p = reinterpret_cast<int32_t *>(base + Lo.f_p);
  ft.parent = reinterpret_cast<int32_t *>(base + Lo.f_parent);
  ft.off = reinterpret_cast<int64_t *>(base + Lo.f_off);
  ft.piv = reinterpret_cast<int64_t *>(base + Lo.f_piv);
  ft.soff = ft.start = ft.yoff = reinterpret_cast<int64_t *>(base + Lo.f_zero);
  int32_t *lvl = reinterpret_cast<int32_t *>(base + Lo.lvl);
  int64_t *wofs = reinterpret_cast<int64_t *>(base + Lo.wofs);
  cx<double> *W = reinterpret_cast<cx<double> *>(base + Lo.W);
  int32_t *pv = reinterpret_cast<int32_t *>(base + Lo.pv);
  double2 *dd = reinterpret_cast<double2 *>(base + Lo.dd);
  double2 *dof = reinterpret_cast<double2 *>(base + Lo.dof);
  int32_t *k0 = reinterpret_cast<int32_t *>(base + Lo.k0);
  int32_t *kb = reinterpret_cast<int32_t *>(base + Lo.kb);
  double *mp = reinterpret_cast<double *>(base + Lo.mp);
  int8_t *ps = reinterpret_cast<int8_t *>(base + Lo.ps);
  // every launch reports its own status (cudaLaunchKernelEx), so an error
  // left behind by the caller's earlier work is neither reported nor cleared
  const dim3 gi((unsigned)std::min<int64_t>(((int64_t)batch * std::max(p, 1) + 255) / 256 + 1, 1024));
  if (launch_prio(k_noalloc_init, gi, dim3(256), 0, s, 0, m, p, batch, const_cast<int32_t *>(ft.m),
                  const_cast<int32_t *>(ft.p), const_cast<int32_t *>(ft.parent), lvl, const_cast<int64_t *>(ft.off),
                  const_cast<int64_t *>(ft.piv), const_cast<int64_t *>(ft.soff), wofs, k0, kb, info, mp,
                  pv) != cudaSuccess)
    return D3M_ECUDA;
  const int steps = (p + NB - 2) / (NB - 1);
  const int cs = panel_cluster_size(p, sizeof(cx<double>));
  cx<double> *arena = reinterpret_cast<cx<double> *>(A);
  int2 *swp = reinterpret_cast<int2 *>(base + Lo.swp);
  int2 *snap = reinterpret_cast<int2 *>(base + Lo.snap);
  for (int stp = 0; stp < steps; ++stp) {
    if (launch_panel<double>(cs, p, m, batch, lvl, ft, wofs, arena, W, pv, dd, dof, ps, k0, kb, info, mp, nullptr,
                             swp, snap, s) != cudaSuccess)
      return D3M_ECUDA;
    int cmin = std::min(p, (stp + 1) * (NB - 1));
    int nt = (m + UT - 1) / UT - cmin / UT;
    dim3 g(std::max(1, nt * (nt + 1) / 2), batch);
    if (launch_prio(k_update<double>, g, dim3(256), 0, s, 0, (const int32_t *)lvl, ft, (const int64_t *)wofs, arena,
                    (const cx<double> *)W, (const int2 *)snap, 0) != cudaSuccess)
      return D3M_ECUDA;
  }
  const dim3 go((unsigned)std::min<int64_t>(((int64_t)batch * m + 255) / 256, 4096));
  if (launch_prio(k_noalloc_out, go, dim3(256), 0, s, 0, m, p, batch, (const int32_t *)pv, (const double2 *)dd,
                  (const double2 *)dof, (const int8_t *)ps, perm, dinv) != cudaSuccess)
    return D3M_ECUDA;
  // asynchronous: the results are complete when `s` reaches this point
  return D3M_OK;
}

}  // namespace d3m

// ============================================================ C ABI (device part)
extern "C" int d3m_dense_ldlt_noalloc(int32_t m, int32_t p, int32_t batch, double *A, int32_t *perm, double *dinv,
                                      int32_t *info, void *stream) {
  if (m <= 0 || p < 0 || p > m || batch <= 0 || !A || !perm || !dinv || !info) return D3M_EINVAL;
  return d3m::dense_ldlt_noalloc(m, p, batch, A, perm, dinv, info, stream);
}

extern "C" int d3m_set_profile(d3m_ctx *h, int32_t on) {
  if (!h) return D3M_EINVAL;
  h->c.opt.profile = on != 0;
  if (h->c.dev) h->c.dev->prof.on = on != 0;
  return D3M_OK;
}

extern "C" int d3m_factor(d3m_ctx *h) {
  if (!h) return D3M_EINVAL;
  d3m::NvtxRange range("d3m_factor");
  try {
    return d3m::dev_factor(h->c);
  } catch (const std::bad_alloc &) {
    h->c.err = "d3m_factor: host allocation failed";
    return D3M_ENOMEM;
  }
}

extern "C" int d3m_solve(d3m_ctx *h, const double *rhs, int64_t ldb, double *x, int64_t ldx, int32_t nrhs,
                         d3m_solve_info *info) {
  if (!h || !rhs || !x || nrhs <= 0 || ldb < h->c.plan.n_edges || ldx < h->c.plan.n_edges) return D3M_EINVAL;
  d3m::NvtxRange range("d3m_solve");
  return d3m::dev_solve(h->c, rhs, ldb, x, ldx, nrhs, info, false);
}

extern "C" int d3m_solve_host(d3m_ctx *h, const double *rhs, int64_t ldb, double *x, int64_t ldx, int32_t nrhs,
                              d3m_solve_info *info) {
  if (!h || !rhs || !x || nrhs <= 0 || ldb < h->c.plan.n_edges || ldx < h->c.plan.n_edges) return D3M_EINVAL;
  d3m::NvtxRange range("d3m_solve_host");
  return d3m::dev_solve(h->c, rhs, ldb, x, ldx, nrhs, info, true);
}

extern "C" int d3m_export_front(d3m_ctx *h, int64_t front, int32_t *m_out, int32_t *p_out, double *F,
                                int32_t *perm, double *dinv) {
  if (!h || front < 0 || front >= (int64_t)h->c.plan.sn_start.size()) return D3M_EINVAL;
  d3m::Ctx &c = h->c;
  const d3m::Plan &P = c.plan;
  int64_t p = P.sn_end[front] - P.sn_start[front];
  int64_t m = p + P.struct_ptr[front + 1] - P.struct_ptr[front];
  if (m_out) *m_out = (int32_t)m;
  if (p_out) *p_out = (int32_t)p;
  if (!F && !perm && !dinv) return D3M_OK;
  if (!c.factored || !c.dev) {
    c.err = "d3m_export_front: no factorisation";
    return D3M_ESTATE;
  }
  d3m::DeviceState *d = c.dev;
  cudaError_t e = cudaSuccess;
  if (F) {
    if (d->precision == D3M_FP64) {
      e = cudaMemcpy(F, (d3m::cx<double> *)d->arena + P.front_off[front], m * m * 16, cudaMemcpyDeviceToHost);
    } else {
      std::vector<float> tmp(2 * m * m);
      e = cudaMemcpy(tmp.data(), (d3m::cx<float> *)d->arena + P.front_off[front], m * m * 8, cudaMemcpyDeviceToHost);
      for (int64_t i = 0; i < 2 * m * m; ++i) F[i] = tmp[i];
    }
  }
  if (e == cudaSuccess && perm) e = cudaMemcpy(perm, d->perm + P.piv_off[front], p * 4, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && dinv) {
    std::vector<double2> dd(p), dof(p);
    std::vector<int8_t> ps(p);
    e = cudaMemcpy(dd.data(), d->dinv_d + P.piv_off[front], p * 16, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(dof.data(), d->dinv_o + P.piv_off[front], p * 16, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(ps.data(), d->psize + P.piv_off[front], p, cudaMemcpyDeviceToHost);
    for (int64_t i = 0; i < p; ++i) {
      dinv[6 * i] = dd[i].x;
      dinv[6 * i + 1] = dd[i].y;
      dinv[6 * i + 2] = dof[i].x;
      dinv[6 * i + 3] = dof[i].y;
      dinv[6 * i + 4] = ps[i];
      dinv[6 * i + 5] = 0;
    }
  }
  if (e != cudaSuccess) {
    c.err = cudaGetErrorString(e);
    return D3M_ECUDA;
  }
  return D3M_OK;
}

extern "C" int d3m_solve_adjoint(d3m_ctx *h, const double *rhs, int64_t ldb, double *y, int64_t ldy,
                                 int32_t nrhs, d3m_solve_info *info) {
  if (!h || !rhs || !y || nrhs <= 0 || ldb < h->c.plan.n_edges || ldy < h->c.plan.n_edges) return D3M_EINVAL;
  d3m::NvtxRange range("d3m_solve_adjoint");
  return d3m::dev_solve(h->c, rhs, ldb, y, ldy, nrhs, info, false, true);
}

extern "C" int d3m_grad_eps(d3m_ctx *h, const double *x, int64_t ldx, const double *y, int64_t ldy, int32_t nrhs,
                            double *grad) {
  if (!h || !x || !y || !grad || nrhs <= 0 || ldx < h->c.plan.n_edges || ldy < h->c.plan.n_edges) return D3M_EINVAL;
  if (h->c.plan.cell_ne > d3m::MAX_CELL_NE) {  // the per-cell table's bound (not reached by any element kind)
    h->c.err = "d3m_grad_eps: more dofs per cell than the gradient's per-cell table holds";
    return D3M_EINVAL;
  }
  d3m::NvtxRange range("d3m_grad_eps");
  return d3m::dev_grad_eps(h->c, x, ldx, y, ldy, nrhs, grad);
}

extern "C" int d3m_dense_ldlt(int32_t m, int32_t p, int32_t batch, double *A, int32_t *perm, double *dinv,
                              int32_t *info, void *stream, int32_t panel_kernel) {
  if (m <= 0 || p < 0 || p > m || batch <= 0 || !A || !perm || !dinv || !info) return D3M_EINVAL;
  std::string err;
  int rc = d3m::dense_ldlt(m, p, batch, A, perm, dinv, info, stream, panel_kernel, err);
  if (rc) fprintf(stderr, "d3m_dense_ldlt: %s\n", err.c_str());
  return rc;
}

