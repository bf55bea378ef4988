// Batched complex products of the mixed-precision substitution on the
// 5th-generation tensor cores (included by engine.cu after k_cgemm).
//
// The forward and backward sweeps (Algorithm 2's substitutions, one level of
// the elimination tree per launch) multiply the static blocks of the
// factors -- L11^{-1}, its transpose, L21 and L21^T -- by the block of
// right-hand sides of the level: C = alpha op(A) B (+ C), item for item the
// products k_cgemm computes.  With tens of right-hand sides these are
// compute-bound in fp32 FMA; here they run as complex BF16x3 on tcgen05,
// with the split and the accumulation of k_tc_gemm (every fp32 value
// x = h + m + l in bf16, six bf16 products per real product, the leading h.h
// products and the five correction products in separate TMEM accumulators,
// the minus of Re = Ar Br - Ai Bi through the A-negate bit).
//
// The A operands do not change between the factorisation and the solves,
// so they are split once, right after each tree level is factored
// (k_tc_presplit, on the inverse stream): every 128-row x 32-k block of
// every A operand becomes one 48 KB image of its six bf16 planes in exactly
// the K-major, 64-byte-swizzled shared-memory layout the MMA descriptors
// read.  The product kernel then moves A with one bulk copy per k chunk
// (cp.async.bulk, mbarrier transaction count), three stages deep, and its
// producer warps only split the small right-hand-side block B.
//
// k_tc_cgemm: one CTA per 128 x 64 output tile, 320 threads.  Warps 0-7
// load the tile's B chunks (32 x 64 complex64, rows optionally gathered),
// two chunks ahead in registers, split them and store their planes; one
// thread of warp 8 issues the A bulk copies (the first three before the
// programmatic wait for the preceding kernel of the sweep, since A is
// static); one thread of warp 9 issues the MMAs (M = 128, N = 64, K = 16;
// 24 per k-step of 16).  The epilogue stages
// the accumulators through shared memory and writes C one row at a time,
// coalesced along the right-hand sides.  Every mbarrier wait is bounded: on
// expiry the tile raises `err`, stops, waits (bounded) for its MMAs and bulk
// copies in flight, frees its TMEM and writes nothing.

constexpr int Q_BM = 128, Q_BN = 64, Q_BK = 32, Q_STAGES = 3, Q_NPROD = 256, Q_THREADS = 320;
constexpr int Q_APL = Q_BM * Q_BK * 2;                    // bytes of one A plane tile (8 KB)
constexpr int Q_BPL = Q_BN * Q_BK * 2;                    // bytes of one B plane tile (4 KB)
constexpr int Q_ABLK = G_NPL * Q_APL;                     // one pre-split A block (48 KB)
constexpr int Q_STAGE_BYTES = Q_ABLK + G_NPL * Q_BPL;     // 72 KB
constexpr int Q_CPITCH = Q_BN + 1;                        // epilogue staging row pitch (complex)
constexpr int Q_SMEM = Q_STAGES * Q_STAGE_BYTES + 1024 + 256;
constexpr int Q_TMEM_COLS = 256;  // Re, Im of the h.h products; Re, Im of the corrections (64 each)
static_assert(Q_BM * Q_CPITCH * 8 <= Q_STAGES * Q_STAGE_BYTES, "the epilogue staging reuses the stages");
static_assert(Q_SMEM <= 227 * 1024, "shared memory per CTA");

// One 128 x 32 block of an A operand to pre-split: rows [r0, r0 + 128) and
// k [k0, k0 + 32) of the operand at `src` in buffer `abuf` (element (i, k) at
// src + i a_rs + k a_cs, M x K), written as block `blk` of the plane buffer.
struct QPre {
  int64_t src, blk;
  int32_t a_rs, a_cs, abuf, M, K, r0, k0;
};

// First block of row tile tm of a pre-split operand with nkc k chunks, minus
// the tile's first stored chunk: mode 0 stores every chunk of every row tile;
// mode 1 (lower triangular) chunks [0, min(nkc, 4 (tm + 1))); mode 3 (upper)
// chunks [4 tm, nkc) -- the chunks a 128-row tile's k range can reach.
__host__ __device__ inline int64_t q_rowbase(int mode, int nkc, int tm) {
  constexpr int R = Q_BM / Q_BK;
  if (mode != 1 && mode != 3) return (int64_t)tm * nkc;
  int64_t r = 0;
  for (int t = 0; t < tm; ++t) r += mode == 1 ? (nkc < R * (t + 1) ? nkc : R * (t + 1)) : nkc - R * t;
  return mode == 3 ? r - (int64_t)R * tm : r;
}

// Byte offset of 16-byte chunk c (8 bf16 along k) of row `row` in a K-major
// plane tile of 64-byte rows with the 64-byte swizzle: the chunk index is
// XORed with bits 1-2 of the row (address bits 4-5 with bits 7-8).
__device__ __forceinline__ uint32_t q_swz(int row, int c) {
  return (uint32_t)(row * 64 + ((c ^ ((row >> 1) & 3)) << 4));
}
// Instruction descriptor of kind::f16: D f32, A/B bf16, both K-major,
// N = 64, M = 128.
__device__ __forceinline__ uint32_t q_idesc(int negA) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)negA << 13) | ((uint32_t)(Q_BN >> 3) << 17) |
         ((uint32_t)(Q_BM >> 4) << 24);
}
// The six planes (Re h, m, l, Im h, m, l) of 8 consecutive-k complex values,
// each as one 16-byte chunk (element e in bits 16 (e % 2) of word e / 2).
__device__ __forceinline__ void q_split8(const cx<float> *v, uint4 (&out)[6]) {
  uint32_t w[6][4];
#pragma unroll
  for (int e = 0; e < 8; e += 2) {
    uint16_t h0, m0, l0, h1, m1, l1;
    bf16x3_split(v[e].re, h0, m0, l0);
    bf16x3_split(v[e + 1].re, h1, m1, l1);
    w[0][e / 2] = (uint32_t)h0 | ((uint32_t)h1 << 16);
    w[1][e / 2] = (uint32_t)m0 | ((uint32_t)m1 << 16);
    w[2][e / 2] = (uint32_t)l0 | ((uint32_t)l1 << 16);
    bf16x3_split(v[e].im, h0, m0, l0);
    bf16x3_split(v[e + 1].im, h1, m1, l1);
    w[3][e / 2] = (uint32_t)h0 | ((uint32_t)h1 << 16);
    w[4][e / 2] = (uint32_t)m0 | ((uint32_t)m1 << 16);
    w[5][e / 2] = (uint32_t)l0 | ((uint32_t)l1 << 16);
  }
#pragma unroll
  for (int q = 0; q < 6; ++q) out[q] = make_uint4(w[q][0], w[q][1], w[q][2], w[q][3]);
}
__device__ __forceinline__ void mbar_arrive(uint32_t mbar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(mbar) : "memory");
}
__device__ __forceinline__ void bulk_load(uint32_t dst, const void *src, uint32_t bytes, uint32_t mbar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(mbar)
               : "memory");
}

// Pre-split of A blocks (one CTA of 256 threads per block): thread ->
// (row, 16 consecutive k), the fast thread index along the operand's
// contiguous dimension; entries outside the operand are written as zeros.
__global__ void __launch_bounds__(256)
    k_tc_presplit(const QPre *__restrict__ jobs, CgBufs<float> bufs, uint16_t *__restrict__ qpl) {
  const QPre j = jobs[blockIdx.x];
  const cx<float> *A = cg_buf(bufs, j.abuf) + j.src;
  const int tid = threadIdx.x;
  const bool afast = j.a_rs == 1;
  const int ax = afast ? (tid & 127) : (tid >> 1), akh = afast ? (tid >> 7) : (tid & 1);
  const int i = j.r0 + ax;
  const cx<float> *Arow = A + (int64_t)i * j.a_rs;
  cx<float> v[16];
#pragma unroll
  for (int e = 0; e < 16; ++e) {
    const int k = j.k0 + akh * 16 + e;
    v[e] = (i < j.M && k < j.K) ? Arow[(int64_t)k * j.a_cs] : mk<float>(0.f, 0.f);
  }
  unsigned char *dst = reinterpret_cast<unsigned char *>(qpl) + j.blk * (int64_t)Q_ABLK;
  uint4 pl[6];
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    q_split8(v + 8 * h, pl);
    const uint32_t o = q_swz(ax, akh * 2 + h);
#pragma unroll
    for (int q = 0; q < 6; ++q) *reinterpret_cast<uint4 *>(dst + q * Q_APL + o) = pl[q];
  }
}

__global__ void __launch_bounds__(Q_THREADS, 1)
    k_tc_cgemm(const CgItem *__restrict__ items, int nitems, int ntiles, CgBufs<float> bufs,
               const int64_t *__restrict__ gidx, const int32_t *__restrict__ tmap,
               const uint16_t *__restrict__ qpl, int32_t *__restrict__ err, int wait_cap) {
  constexpr int FULL_CAP = 1 << 22;
  extern __shared__ __align__(16) unsigned char q_raw[];
  const int t = blockIdx.x;
  if (t >= ntiles) return;
  // stage tiles start on a 1024-byte boundary of the shared window (swizzle atoms)
  unsigned char *sm = q_raw + ((1024u - (smem_u32(q_raw) & 1023u)) & 1023u);
  uint64_t *afull = reinterpret_cast<uint64_t *>(sm + Q_STAGES * Q_STAGE_BYTES);
  uint64_t *bfull = afull + Q_STAGES;
  uint64_t *empty = bfull + Q_STAGES;
  uint64_t *done = empty + Q_STAGES;
  uint32_t *taddr_s = reinterpret_cast<uint32_t *>(done + 1);
  volatile int *abort_s = reinterpret_cast<volatile int *>(taddr_s + 1);
  volatile int *issued_s = abort_s + 1;   // k chunks whose MMAs were issued
  volatile int *issuedA_s = abort_s + 2;  // k chunks whose A bulk copies were issued
  const CgItem it = items[cg_item_of(items, nitems, t, tmap)];
  const int ntm = (it.M + Q_BM - 1) / Q_BM;
  const int ti = t - it.tile0, tm = ti % ntm, tn = ti / ntm;
  const int i0 = tm * Q_BM, j0 = tn * Q_BN;
  // k range of the tile (triangular operands); klo is a multiple of Q_BK
  int klo = 0, khi = it.K;
  if (it.mode == 1) khi = min(it.K, i0 + Q_BM - it.koff);
  if (it.mode == 3) klo = max(0, i0 - it.koff);
  const int nk = khi > klo ? (khi - klo + Q_BK - 1) / Q_BK : 0;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // B producers (threads < Q_NPROD): thread -> (B column, 8 consecutive k),
  // the fast thread index along B's contiguous dimension (coalesced loads);
  // two chunks in flight in registers, the first two issued before the set-up
  const cx<float> *B = cg_buf(bufs, it.bbuf) + it.b;
  const int64_t *G = it.gath >= 0 ? gidx + it.gath : nullptr;
  const bool bfast = it.b_cs == 1;
  const int bn = bfast ? (tid & 63) : (tid >> 2), bkq = bfast ? (tid >> 6) : (tid & 3);
  const int bj = j0 + bn;
  const uint32_t ob = q_swz(bn, bkq);
  auto load = [&](cx<float>(&rb)[8], int kc) {
    const int k0 = klo + kc * Q_BK + bkq * 8;
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int k = k0 + e;
      cx<float> v = mk<float>(0.f, 0.f);
      if (bj < it.N && k < khi) {
        const int64_t kr = G ? G[k] : (int64_t)k;
        v = B[kr * it.b_rs + (int64_t)bj * it.b_cs];
      }
      rb[e] = v;
    }
  };
  cx<float> r0[8], r1[8];
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(taddr_s)),
                 "r"(Q_TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    for (int s = 0; s < Q_STAGES; ++s) {
      mbar_init(smem_u32(afull + s), 1);
      mbar_init(smem_u32(bfull + s), Q_NPROD);
      mbar_init(smem_u32(empty + s), 1);
    }
    mbar_init(smem_u32(done), 1);
    *abort_s = 0;
    *issued_s = 0;
    *issuedA_s = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *taddr_s;
  const uint32_t sbase = smem_u32(sm);
  // the A blocks are static (written by the factorisation): the first stages
  // are requested before waiting for the predecessor in the sweep
  const uint16_t *asrc = qpl + (it.qa + q_rowbase(it.mode, it.qnk, tm) + klo / Q_BK) * (int64_t)(Q_ABLK / 2);
  const int kpre = min(nk, Q_STAGES);
  if (tid == Q_NPROD)
    for (int kc = 0; kc < kpre; ++kc) {
      const uint32_t fa = smem_u32(afull + kc);
      mbar_expect_tx(fa, Q_ABLK);
      bulk_load(sbase + kc * Q_STAGE_BYTES, asrc + (int64_t)kc * (Q_ABLK / 2), Q_ABLK, fa);
    }
  pdl_wait();  // B and C are written by the preceding kernels of the sweep
  pdl_trigger();
  if (tid < Q_NPROD) {
    // ---- B producers
    if (nk > 0) load(r0, 0);
    if (nk > 1) load(r1, 1);
    auto produce = [&](const cx<float>(&rb)[8], int kc) -> bool {
      const int s = kc % Q_STAGES;
      if (kc >= Q_STAGES &&
          !mbar_wait_bounded(smem_u32(empty + s), (uint32_t)((kc / Q_STAGES - 1) & 1), wait_cap)) {
        *abort_s = 1;
        return false;
      }
      if (*abort_s) return false;
      unsigned char *st = sm + s * Q_STAGE_BYTES + Q_ABLK;
      uint4 pl[6];
      q_split8(rb, pl);
#pragma unroll
      for (int q = 0; q < 6; ++q) *reinterpret_cast<uint4 *>(st + q * Q_BPL + ob) = pl[q];
      // the generic-proxy stores become visible to the tensor cores (async proxy)
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      mbar_arrive(smem_u32(bfull + s));
      return true;
    };
    for (int kc = 0; kc < nk; kc += 2) {
      if (!produce(r0, kc)) break;
      if (kc + 2 < nk) load(r0, kc + 2);
      if (kc + 1 < nk) {
        if (!produce(r1, kc + 1)) break;
        if (kc + 3 < nk) load(r1, kc + 3);
      }
    }
  } else if (tid == Q_NPROD) {
    // ---- A loader: one bulk copy of a pre-split 48 KB block per k chunk
    // (the first kpre were issued before the wait)
    int kc = kpre;
    for (; kc < nk; ++kc) {
      const int s = kc % Q_STAGES;
      if (kc >= Q_STAGES &&
          !mbar_wait_bounded(smem_u32(empty + s), (uint32_t)((kc / Q_STAGES - 1) & 1), wait_cap)) {
        *abort_s = 1;
        break;
      }
      if (*abort_s) break;
      const uint32_t fa = smem_u32(afull + s);
      mbar_expect_tx(fa, Q_ABLK);
      bulk_load(sbase + s * Q_STAGE_BYTES, asrc + (int64_t)kc * (Q_ABLK / 2), Q_ABLK, fa);
    }
    *issuedA_s = kc;
  } else if (tid == Q_NPROD + 32) {
    // ---- MMA issuer: 2 k-steps of 16 per chunk, 24 bf16 MMAs per k-step
    // (pieces h, m, l = 0, 1, 2); leading products to TMEM columns 0-127
    // (Re, Im), the correction products to 128-255
    const uint32_t id_pos = q_idesc(0), id_neg = q_idesc(1);
    constexpr int PA[6] = {0, 0, 1, 0, 2, 1}, PB[6] = {0, 1, 0, 2, 0, 1};
    int kc = 0;
    for (; kc < nk; ++kc) {
      const int s = kc % Q_STAGES;
      const uint32_t ph = (uint32_t)((kc / Q_STAGES) & 1);
      if (*abort_s || !mbar_wait_bounded(smem_u32(afull + s), ph, wait_cap) ||
          !mbar_wait_bounded(smem_u32(bfull + s), ph, wait_cap)) {
        *abort_s = 1;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t st = sbase + s * Q_STAGE_BYTES, sb = st + Q_ABLK;
#pragma unroll
      for (int kk = 0; kk < Q_BK / 16; ++kk) {
        const uint32_t ko = (uint32_t)kk * 32;  // 16 bf16 = 32 bytes along the swizzled row
        const uint32_t first = (kc == 0 && kk == 0) ? 0u : 1u;
#pragma unroll
        for (int u = 0; u < 6; ++u) {
          const uint64_t Ar = g_desc(st + PA[u] * Q_APL + ko), Ai = g_desc(st + (3 + PA[u]) * Q_APL + ko);
          const uint64_t Br = g_desc(sb + PB[u] * Q_BPL + ko), Bi = g_desc(sb + (3 + PB[u]) * Q_BPL + ko);
          const uint32_t dre = tmem + (u == 0 ? 0 : 2 * Q_BN), dim = dre + Q_BN;
          const uint32_t acc = (u <= 1) ? first : 1u;
          bf_mma(dre, Ar, Br, id_pos, acc);
          bf_mma(dre, Ai, Bi, id_neg, 1u);
          bf_mma(dim, Ar, Bi, id_pos, acc);
          bf_mma(dim, Ai, Br, id_pos, 1u);
        }
      }
      tc_commit(smem_u32(empty + s));  // the stage is free once these MMAs have read it
    }
    *issued_s = kc;
    if (kc > 0) tc_commit(smem_u32(done));  // completes when every MMA issued above has completed
  }
  // ---- epilogue: wait for the accumulators (when any MMA was issued)
  __syncthreads();
  bool ok = true;
  if (*issued_s > 0) {
    ok = mbar_wait_bounded(smem_u32(done), 0, wait_cap);
    if (!ok) mbar_wait_bounded(smem_u32(done), 0, FULL_CAP);  // never release TMEM under running MMAs
  }
  ok = __syncthreads_and(ok) && !*abort_s;
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  float2 *stg = reinterpret_cast<float2 *>(sm);
  if (ok && warp < 8) {
    // warp w reads TMEM lanes 32 (w % 4) .. + 31 (its rows), columns 32 (w / 4) .. + 31
    const int r = (warp & 3) * 32 + lane, c0 = (warp >> 2) * 32;
    uint32_t vr[32], vi[32], cr[32], ci[32];
    if (nk > 0) {
      const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;
      tmem_ld32(tmem + lane_base + (uint32_t)c0, vr);
      tmem_ld32(tmem + lane_base + (uint32_t)(Q_BN + c0), vi);
      tmem_ld32(tmem + lane_base + (uint32_t)(2 * Q_BN + c0), cr);
      tmem_ld32(tmem + lane_base + (uint32_t)(3 * Q_BN + c0), ci);
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    } else {
#pragma unroll
      for (int q = 0; q < 32; ++q) vr[q] = vi[q] = cr[q] = ci[q] = 0u;
    }
#pragma unroll
    for (int q = 0; q < 32; ++q)
      stg[r * Q_CPITCH + c0 + q] = make_float2(__uint_as_float(vr[q]) + __uint_as_float(cr[q]),
                                               __uint_as_float(vi[q]) + __uint_as_float(ci[q]));
  }
  __syncthreads();
  if (ok) {
    // thread -> columns lane, lane + 32 of rows warp, warp + 10, ...; with
    // beta every old value of C is loaded before the first store, so the
    // loads are in flight together
    constexpr int NW = Q_THREADS / 32, RPW = (Q_BM + NW - 1) / NW;
    cx<float> *C = cg_buf(bufs, it.cbuf) + it.c;
    const float al = it.alpha;
    cx<float> old[RPW][2];
#pragma unroll
    for (int q = 0; q < RPW; ++q)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int row = warp + NW * q, i = i0 + row, j = j0 + lane + 32 * h;
        old[q][h] = (it.beta && row < Q_BM && i < it.M && j < it.N)
                        ? C[(int64_t)i * it.c_rs + (int64_t)j * it.c_cs]
                        : mk<float>(0.f, 0.f);
      }
#pragma unroll
    for (int q = 0; q < RPW; ++q)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int row = warp + NW * q, i = i0 + row, cc = lane + 32 * h, j = j0 + cc;
        if (row < Q_BM && i < it.M && j < it.N) {
          const float2 a = stg[row * Q_CPITCH + cc];
          C[(int64_t)i * it.c_rs + (int64_t)j * it.c_cs] =
              mk<float>(al * a.x + old[q][h].re, al * a.y + old[q][h].im);
        }
      }
  } else if (tid == 0) {
    atomicExch(err, 1);
  }
  // bulk copies still in flight after an expiry land before the CTA's shared
  // memory is released: wait (bounded) for the last phase of every stage used
  if (tid == Q_NPROD) {
    const int n = *issuedA_s;
    for (int kc = max(0, n - Q_STAGES); kc < n; ++kc)
      mbar_wait_bounded(smem_u32(afull + kc % Q_STAGES), (uint32_t)((kc / Q_STAGES) & 1), FULL_CAP);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(Q_TMEM_COLS));
}
