// Kernels of GMRES-based iterative refinement (included by engine.cu).
//
// The mixed path refines x with fp64 residuals r = f - A x.  Plain
// refinement adds M^{-1} r (M^{-1}: the complex64 factors).  GMRES-IR instead
// solves each correction equation A d = r by flexible GMRES in fp64, right
// preconditioned by M^{-1}: Arnoldi on z_k = M^{-1} v_k, w = A z_k, with the
// new direction orthogonalised against the basis by classical Gram-Schmidt
// applied twice (two passes of V^H w and w -= V h; as accurate as modified
// Gram-Schmidt and made of batched reductions), the small Hessenberg
// least-squares problem solved with Givens rotations on the host, and
// d = Z y.  All vectors are edge-space, fp64 complex, row-major n x r (RHS
// fastest), one Krylov space per right-hand side; rows of removed (PEC)
// edges carry no equation and are kept at zero.

// w = A z (fp64), A = Ar + j Ai as in k_residual; rows without entries
// (removed edges) give 0.  One warp per row, lanes over the right-hand sides.
__global__ void __launch_bounds__(256)
    k_spmv(int64_t n, const int64_t *__restrict__ ptr, const int32_t *__restrict__ col,
           const double *__restrict__ vre, const int64_t *__restrict__ iptr, const int32_t *__restrict__ icol,
           const double *__restrict__ vim, const double2 *__restrict__ z, double2 *__restrict__ w, int r) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t row = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); row < n; row += nw) {
    const int64_t a = ptr[row], b = ptr[row + 1];
    for (int c = lane; c < r; c += 32) {
      double2 acc = make_double2(0.0, 0.0);
      for (int64_t q = a; q < b; ++q) {
        const double av = vre[q];
        const double2 xv = z[(int64_t)col[q] * r + c];
        acc.x += av * xv.x;
        acc.y += av * xv.y;
      }
      for (int64_t q = iptr[row]; q < iptr[row + 1]; ++q) {  // j * imaginary part
        const double av = vim[q];
        const double2 xv = z[(int64_t)icol[q] * r + c];
        acc.x -= av * xv.y;
        acc.y += av * xv.x;
      }
      w[row * r + c] = acc;
    }
  }
}

// out[i][c] += sum_rows conj(V_i[row, c]) w[row, c] for i < nv (vector i at
// V + i * vst); out as (re, im) double pairs, accumulated with atomics.
// 256 threads per block: with r <= 256, thread t takes column t % r and
// every (256 / r)-th row of the block's row range; else columns t, t + 256, ...
__global__ void __launch_bounds__(256)
    k_dots(int64_t n, int r, int nv, const double2 *__restrict__ V, int64_t vst, const double2 *__restrict__ w,
           double *__restrict__ out) {
  __shared__ double2 red[256];
  const int tid = threadIdx.x;
  const bool narrow = r <= 256;
  const int nq = narrow ? 256 / r : 1;
  const int q = narrow ? tid / r : 0;
  const int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
  const int64_t r0 = (int64_t)blockIdx.x * chunk, r1 = min(n, r0 + chunk);
  for (int i = 0; i < nv; ++i) {
    const double2 *Vi = V + (int64_t)i * vst;
    for (int cb = 0; cb < (narrow ? 1 : r); cb += 256) {
      const int c = narrow ? tid % r : cb + tid;
      double2 acc = make_double2(0.0, 0.0);
      if (q < nq && c < r)
        for (int64_t row = r0 + q; row < r1; row += nq) {
          const double2 v = Vi[row * r + c], x = w[row * r + c];
          acc.x += v.x * x.x + v.y * x.y;  // conj(v) x
          acc.y += v.x * x.y - v.y * x.x;
        }
      if (narrow) {
        red[tid] = acc;
        __syncthreads();
        if (tid < r) {
          for (int u = 1; u < nq; ++u) {
            acc.x += red[tid + u * r].x;
            acc.y += red[tid + u * r].y;
          }
          atomicAdd(out + 2 * ((int64_t)i * r + c), acc.x);
          atomicAdd(out + 2 * ((int64_t)i * r + c) + 1, acc.y);
        }
        __syncthreads();
      } else if (c < r) {
        atomicAdd(out + 2 * ((int64_t)i * r + c), acc.x);
        atomicAdd(out + 2 * ((int64_t)i * r + c) + 1, acc.y);
      }
    }
  }
}

// w[row, c] -= sum_{i < nv} h[i][c] V_i[row, c]
__global__ void k_sub_many(int64_t n, int r, int nv, const double2 *__restrict__ V, int64_t vst,
                           const double2 *__restrict__ h, double2 *__restrict__ w) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * r; e += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(e % r);
    double2 acc = w[e];
    for (int i = 0; i < nv; ++i) {
      const double2 hv = h[(int64_t)i * r + c], v = V[(int64_t)i * vst + e];
      acc.x -= hv.x * v.x - hv.y * v.y;
      acc.y -= hv.x * v.y + hv.y * v.x;
    }
    w[e] = acc;
  }
}

// out[row, c] = w[row, c] * s[c]
__global__ void k_scale_cols(int64_t n, int r, const double2 *__restrict__ w, const double *__restrict__ s,
                             double2 *__restrict__ out) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * r; e += (int64_t)gridDim.x * blockDim.x) {
    const double sc = s[e % r];
    out[e] = make_double2(w[e].x * sc, w[e].y * sc);
  }
}

// x[row, c] += sum_{j < nz} y[j][c] Z_j[row, c]
__global__ void k_add_combo(int64_t n, int r, int nz, const double2 *__restrict__ Z, int64_t zst,
                            const double2 *__restrict__ y, double2 *__restrict__ x) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * r; e += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(e % r);
    double2 acc = x[e];
    for (int j = 0; j < nz; ++j) {
      const double2 yv = y[(int64_t)j * r + c], v = Z[(int64_t)j * zst + e];
      acc.x += yv.x * v.x - yv.y * v.y;
      acc.y += yv.x * v.y + yv.y * v.x;
    }
    x[e] = acc;
  }
}

// zero the rows of removed (PEC) edges
__global__ void k_mask_rows(int64_t n, int r, const uint8_t *__restrict__ pec, double2 *__restrict__ v) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * r; e += (int64_t)gridDim.x * blockDim.x)
    if (pec[e / r]) v[e] = make_double2(0.0, 0.0);
}
