// Deferred Schur-complement products of the mixed-precision factorisation
// on the 5th-generation tensor cores (included by engine.cu).
//
// Once the restricted Bunch-Kaufman panels of a front have factored its pivot
// block, P F11 P^T = L11 D L11^T, and the update rows have been solved for
// (L21 and W21 = L21 D, Algorithm 1's triangular-solve step), what remains of
// Algorithm 1's update K_ik -= L_ij X_kj^T on the front is one dense product
// with inner dimension p (the pivot-block order):
//   C = F22 - L21 W21^T          (the contribution block: Schur complement
//                                 of an interior front, -K_D of an interface
//                                 front, the update of the fronts of K)
// It runs as complex fp32 on tcgen05 with BF16x3 split operands: every fp32
// value is x = h + m + l + e with h, m, l in bf16 (8 significant bits each:
// h = bf16(x), m = bf16(x - h), l = bf16(x - h - m)) and |e| about 2^-25 |x|,
// and A B^T ~ Ah Bh^T + Ah Bm^T + Am Bh^T + Ah Bl^T + Al Bh^T + Am Bm^T (the
// dropped terms are below 2^-25 too) with fp32 accumulation in TMEM, which
// keeps fp32 accuracy.  Complex arithmetic is four real products per
// accumulator:  Re += Ar Br^T - Ai Bi^T,   Im += Ar Bi^T + Ai Br^T, the minus
// through the A-negate bit of the instruction descriptor.
//
// Operands are first split into six bf16 planes (Re h/m/l, Im h/m/l) in
// global memory, K-major (each operand row holds its K values contiguously),
// every front's block padded to 128 rows and its K to a multiple of 32 with
// zeros.  The GEMM kernel streams 128-row x 32-k tiles of the planes into
// shared memory with TMA (cp.async.bulk.tensor.3d, 64-byte swizzle, one
// tensor map per operand and tree level) through a 2-stage mbarrier
// pipeline: one thread issues the loads, one thread issues tcgen05.mma
// (kind::f16 with bf16 inputs, M = 128, N = 128, K = 16) into four TMEM
// accumulators (Re and Im of the leading h.h products, Re and Im of the
// correction products), and the four warps read their 32 TMEM lanes back
// with tcgen05.ld for the epilogue.  Every mbarrier
// wait is bounded: on expiry the kernel raises an error flag, stops issuing
// work, waits (bounded) for the loads and MMAs it has issued, frees its TMEM
// and returns.

constexpr int G_BM = 128, G_BN = 128, G_BK = 32, G_STAGES = 2, G_NPL = 6;
constexpr int G_PLANE = G_BM * G_BK * 2;                 // bytes of one plane tile (8 KB; G_BN == G_BM)
constexpr int G_STAGE_BYTES = 2 * G_NPL * G_PLANE;       // 6 A planes + 6 B planes
constexpr int G_SMEM = G_STAGES * G_STAGE_BYTES + 1024 + 128;  // + alignment + barriers
constexpr int G_KPAD = 32;                               // K padding of a front's plane block
constexpr int G_TMEM_COLS = 512;  // Re, Im of the h.h products; Re, Im of the correction products

// One output tile of a batched product.
struct TcTile {
  int32_t arow, brow;  // first row of the tile's A / B rows in the plane buffers
  int32_t M, N;        // valid rows / columns (<= 128)
  int32_t nk;          // number of G_BK-wide k chunks (bf16 elements)
  int32_t mode;        // 0: W = acc (fp32 complex, column-major); 1: C -= acc (front, complex64)
  int32_t diag;        // mode 1: tile on the diagonal of the Schur block (keep column <= row)
  int32_t ldc;
  int64_t c_off;       // element offset of the tile's (0, 0) in the output buffer
};

// One 32 x 32 block of a plane-split pass: rows [r0, r0 + 32) and k values
// [k0, k0 + 32) of the operand of front `f` (see k_tc_split).
struct TcSplit {
  int32_t f;           // front (M-order supernode id)
  int32_t r0, k0;
  int32_t rows, cols;  // valid extent of the operand (rows, K)
  int32_t drow;        // destination row of operand row 0 in the plane buffer
  int64_t src;         // element offset of operand (0, 0) in the source buffer
  int32_t ld;          // source column stride (column-major source)
  int32_t gather;      // 1: operand column k is source column perm[k] (pivot order)
};

// BF16x3 split of an fp32 value (round to nearest even at every step; each
// remainder is exact in fp32)
__device__ __forceinline__ void bf16x3_split(float x, uint16_t &h, uint16_t &m, uint16_t &l) {
  const __nv_bfloat16 bh = __float2bfloat16_rn(x);
  const float r1 = x - __bfloat162float(bh);
  const __nv_bfloat16 bm = __float2bfloat16_rn(r1);
  const float r2 = r1 - __bfloat162float(bm);
  const __nv_bfloat16 bl = __float2bfloat16_rn(r2);
  h = __bfloat16_as_ushort(bh);
  m = __bfloat16_as_ushort(bm);
  l = __bfloat16_as_ushort(bl);
}
// the six planes of a complex value at element o of plane 0 (plane stride ps)
__device__ __forceinline__ void put_planes(uint16_t *pl, int64_t o, int64_t ps, cx<float> v) {
  uint16_t h, m, l;
  bf16x3_split(v.re, h, m, l);
  pl[o] = h;
  pl[o + ps] = m;
  pl[o + 2 * ps] = l;
  bf16x3_split(v.im, h, m, l);
  pl[o + 3 * ps] = h;
  pl[o + 4 * ps] = m;
  pl[o + 5 * ps] = l;
}

// Shared-memory matrix descriptor of a K-major operand tile with 64-byte
// swizzle: rows of 32 bf16 (64 bytes), 8-row groups 512 bytes apart.
__device__ __forceinline__ uint64_t g_desc(uint32_t saddr) {
  return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)1 << 16) | ((uint64_t)(512 >> 4) << 32) | (1ull << 46) |
         (4ull << 61);
}
// Instruction descriptor of kind::f16: D f32, A/B bf16, both K-major,
// N = 128, M = 128.
__device__ __forceinline__ uint32_t g_idesc(int negA) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)negA << 13) | ((uint32_t)(G_BN >> 3) << 17) |
         ((uint32_t)(G_BM >> 4) << 24);
}
// D (TMEM) (+)= A B^T, bf16 operands (acc = 0 overwrites D)
__device__ __forceinline__ void bf_mma(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap *tm, int x, int y, int z,
                                            uint32_t mbar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];" ::"r"(dst),
      "l"(tm), "r"(x), "r"(y), "r"(z), "r"(mbar)
      : "memory");
}
__device__ __forceinline__ void mbar_init(uint32_t mbar, int count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mbar), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t mbar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void tc_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
               : "memory");
}
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,"
      "%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
        "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
        "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
        "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
      : "r"(taddr));
}

// The batched complex product on tcgen05.  One CTA (4 warps) per output tile.
// wait_cap bounds the first attempt of every mbarrier wait (the clean-up
// waits after an expiry always use the full bound).
__global__ void __launch_bounds__(128, 1)
    k_tc_gemm(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
              const TcTile *__restrict__ tiles, cx<float> *__restrict__ front, float2 *__restrict__ wout,
              int32_t *__restrict__ err, int wait_cap) {
  constexpr int FULL_CAP = 1 << 22;
  extern __shared__ __align__(16) unsigned char g_raw[];
  // stage tiles start on a 1024-byte boundary of the shared window (swizzle atoms)
  unsigned char *sm = g_raw + ((1024u - (smem_u32(g_raw) & 1023u)) & 1023u);
  uint64_t *full = reinterpret_cast<uint64_t *>(sm + G_STAGES * G_STAGE_BYTES);
  uint64_t *empty = full + G_STAGES;
  uint64_t *done = empty + G_STAGES;
  uint32_t *taddr_s = reinterpret_cast<uint32_t *>(done + 1);
  volatile int *abort_s = reinterpret_cast<volatile int *>(taddr_s + 1);
  int *issued_s = const_cast<int *>(abort_s + 1);
  const TcTile t = tiles[blockIdx.x];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(taddr_s)),
                 "r"(G_TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    for (int s = 0; s < G_STAGES; ++s) {
      mbar_init(smem_u32(full + s), 1);
      mbar_init(smem_u32(empty + s), 1);
    }
    mbar_init(smem_u32(done), 1);
    *abort_s = 0;
    *issued_s = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *taddr_s;
  const uint32_t sbase = smem_u32(sm);
  if (tid == 0) {
    // ---- producer: TMA loads of the 4 + 4 plane tiles of every k chunk
    int kc = 0;
    for (; kc < t.nk; ++kc) {
      const int s = kc % G_STAGES;
      if (kc >= G_STAGES &&
          !mbar_wait_bounded(smem_u32(empty + s), (uint32_t)((kc / G_STAGES - 1) & 1), wait_cap)) {
        *abort_s = 1;
        break;
      }
      if (*abort_s) break;
      const uint32_t st = sbase + s * G_STAGE_BYTES, fb = smem_u32(full + s);
      mbar_expect_tx(fb, G_STAGE_BYTES);
      for (int q = 0; q < G_NPL; ++q) {
        tma_load_3d(st + q * G_PLANE, &tmA, kc * G_BK, t.arow, q, fb);
        tma_load_3d(st + (G_NPL + q) * G_PLANE, &tmB, kc * G_BK, t.brow, q, fb);
      }
    }
    *issued_s = kc;
  } else if (tid == 32) {
    // ---- MMA issuer: 2 k-steps of 16 per chunk, 24 bf16 MMAs per k-step
    // (pieces h, m, l = 0, 1, 2).  The leading products h.h go to their own
    // accumulators (Re: TMEM columns 0-127, Im: 128-255) and the five
    // correction products h.m, m.h, h.l, l.h, m.m, about 2^-8 smaller, to a
    // second pair (256-383, 384-511): the fp32 rounding of the many small
    // additions then stays relative to the small sum, and the two sums meet
    // once, in the epilogue.
    const uint32_t id_pos = g_idesc(0), id_neg = g_idesc(1);
    constexpr int PA[6] = {0, 0, 1, 0, 2, 1}, PB[6] = {0, 1, 0, 2, 0, 1};
    for (int kc = 0; kc < t.nk; ++kc) {
      const int s = kc % G_STAGES;
      if (*abort_s || !mbar_wait_bounded(smem_u32(full + s), (uint32_t)((kc / G_STAGES) & 1), wait_cap)) {
        *abort_s = 1;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t st = sbase + s * G_STAGE_BYTES;
      for (int kk = 0; kk < G_BK / 16; ++kk) {
        const uint32_t ko = (uint32_t)kk * 32;  // 16 bf16 = 32 bytes along the swizzled row
        const uint32_t first = (kc == 0 && kk == 0) ? 0u : 1u;
#pragma unroll
        for (int u = 0; u < 6; ++u) {
          const uint64_t Ar = g_desc(st + PA[u] * G_PLANE + ko), Ai = g_desc(st + (3 + PA[u]) * G_PLANE + ko);
          const uint64_t Br = g_desc(st + (G_NPL + PB[u]) * G_PLANE + ko);
          const uint64_t Bi = g_desc(st + (G_NPL + 3 + PB[u]) * G_PLANE + ko);
          const uint32_t dre = tmem + (u == 0 ? 0 : 2 * G_BN), dim = dre + G_BN;
          const uint32_t acc = (u <= 1) ? first : 1u;  // u = 0 opens the leading pair, u = 1 the correction pair
          bf_mma(dre, Ar, Br, id_pos, acc);
          bf_mma(dre, Ai, Bi, id_neg, 1u);
          bf_mma(dim, Ar, Bi, id_pos, acc);
          bf_mma(dim, Ai, Br, id_pos, 1u);
        }
      }
      tc_commit(smem_u32(empty + s));  // the stage is free once these MMAs have read it
    }
    tc_commit(smem_u32(done));  // completes when every MMA issued above has completed
  }
  // ---- epilogue: wait for the accumulators
  bool ok = mbar_wait_bounded(smem_u32(done), 0, wait_cap);
  if (!ok) mbar_wait_bounded(smem_u32(done), 0, FULL_CAP);  // never release TMEM under running MMAs
  ok = __syncthreads_and(ok) && !*abort_s;
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (ok && t.nk > 0) {
    const int r = warp * 32 + lane;
    const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
    for (int c0 = 0; c0 < G_BN; c0 += 32) {
      uint32_t vr[32], vi[32], cr[32], ci[32];
      tmem_ld32(tmem + lane_base + (uint32_t)c0, vr);
      tmem_ld32(tmem + lane_base + (uint32_t)(G_BN + c0), vi);
      tmem_ld32(tmem + lane_base + (uint32_t)(2 * G_BN + c0), cr);
      tmem_ld32(tmem + lane_base + (uint32_t)(3 * G_BN + c0), ci);
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (r < t.M) {
        if (t.mode == 0) {
          float2 *W = wout + t.c_off + r;
#pragma unroll
          for (int q = 0; q < 32; ++q)
            if (c0 + q < t.N)
              W[(int64_t)(c0 + q) * t.ldc] = make_float2(__uint_as_float(vr[q]) + __uint_as_float(cr[q]),
                                                         __uint_as_float(vi[q]) + __uint_as_float(ci[q]));
        } else {
          // every old value is loaded before the first store (one round of
          // loads in flight instead of 32 load-store round trips)
          cx<float> *C = front + t.c_off + r;
          const int cmax = t.diag ? min(t.N, r + 1) : t.N;
          cx<float> old[32];
#pragma unroll
          for (int q = 0; q < 32; ++q)
            old[q] = c0 + q < cmax ? C[(int64_t)(c0 + q) * t.ldc] : mk<float>(0.f, 0.f);
#pragma unroll
          for (int q = 0; q < 32; ++q)
            if (c0 + q < cmax)
              C[(int64_t)(c0 + q) * t.ldc] =
                  mk<float>(old[q].re - (__uint_as_float(vr[q]) + __uint_as_float(cr[q])),
                            old[q].im - (__uint_as_float(vi[q]) + __uint_as_float(ci[q])));
        }
      }
    }
  } else if (t.nk > 0 && tid == 0) {
    atomicExch(err, 1);
  }
  // loads still in flight after an expiry land before the CTA's shared memory
  // is released: wait (bounded) for the last phase of every stage used
  if (tid == 0) {
    const int n = *issued_s;
    for (int kc = max(0, n - G_STAGES); kc < n; ++kc)
      mbar_wait_bounded(smem_u32(full + kc % G_STAGES), (uint32_t)((kc / G_STAGES) & 1), FULL_CAP);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(G_TMEM_COLS));
}

// Plane split of an operand (complex64, column-major, optionally with its
// columns gathered through the front's pivot order) into the six bf16
// planes, K-major: plane q, row drow + r, column k at
// ((q * rows_total) + drow + r) * kpitch + k.  32 x 32 blocks through shared
// memory (coalesced reads along rows, writes along k); entries outside the
// operand (padding rows and k) are written as zeros.
__global__ void __launch_bounds__(256)
    k_tc_split(const TcSplit *__restrict__ blocks, const cx<float> *__restrict__ src,
               const int32_t *__restrict__ perm, const int64_t *__restrict__ piv_off, uint16_t *__restrict__ planes,
               int64_t rows_total, int kpitch) {
  const TcSplit b = blocks[blockIdx.x];
  __shared__ cx<float> tile[32][33];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
  const int32_t *pv = perm + piv_off[b.f];
  for (int kk = ty; kk < 32; kk += 8) {  // read: column k0 + kk, rows r0 + tx
    const int k = b.k0 + kk, r = b.r0 + tx;
    cx<float> v = mk<float>(0.f, 0.f);
    if (k < b.cols && r < b.rows) {
      const int64_t col = b.gather ? (int64_t)pv[k] : (int64_t)k;
      v = src[b.src + r + col * b.ld];
    }
    tile[kk][tx] = v;
  }
  __syncthreads();
  for (int rr = ty; rr < 32; rr += 8)  // write: row r0 + rr, k0 + tx
    put_planes(planes, (int64_t)(b.drow + b.r0 + rr) * kpitch + b.k0 + tx, rows_total * (int64_t)kpitch,
               tile[tx][rr]);
}
