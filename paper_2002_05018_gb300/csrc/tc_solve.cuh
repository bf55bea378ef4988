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
// One CTA per 128 x 64 output tile, 288 threads.  Warps 0-7 load the tile's
// A (128 x 32) and B (32 x 64) chunks of complex64 from global memory with
// the item's strides (B's rows optionally gathered), split them into the six
// bf16 planes in registers and store them to shared memory in the K-major
// layout with the 64-byte swizzle that the MMA descriptors read (the layout
// TMA's SWIZZLE_64B writes), two stages deep; the global loads of the next
// chunk are in flight while the current one is split and stored.  One thread
// of warp 8 issues the MMAs (M = 128, N = 64, K = 16; 24 per k-step of 16).
// The epilogue stages the accumulators through shared memory and writes C
// one row at a time, coalesced along the right-hand sides.  Every mbarrier
// wait is bounded as in k_tc_gemm: on expiry the tile raises `err`, stops,
// waits (bounded) for the MMAs it has issued, frees its TMEM and writes
// nothing.

constexpr int Q_BM = 128, Q_BN = 64, Q_BK = 32, Q_STAGES = 2, Q_NPROD = 256, Q_THREADS = 288;
constexpr int Q_APL = Q_BM * Q_BK * 2;                    // bytes of one A plane tile (8 KB)
constexpr int Q_BPL = Q_BN * Q_BK * 2;                    // bytes of one B plane tile (4 KB)
constexpr int Q_STAGE_BYTES = G_NPL * (Q_APL + Q_BPL);    // 72 KB
constexpr int Q_CPITCH = Q_BN + 1;                        // epilogue staging row pitch (complex)
constexpr int Q_SMEM = Q_STAGES * Q_STAGE_BYTES + 1024 + 128;
constexpr int Q_TMEM_COLS = 256;  // Re, Im of the h.h products; Re, Im of the corrections (64 each)
static_assert(Q_BM * Q_CPITCH * 8 <= Q_STAGES * Q_STAGE_BYTES, "the epilogue staging reuses the stages");

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

__global__ void __launch_bounds__(Q_THREADS, 1)
    k_tc_cgemm(const CgItem *__restrict__ items, int nitems, int ntiles, CgBufs<float> bufs,
               const int64_t *__restrict__ gidx, int32_t *__restrict__ err, int wait_cap) {
  constexpr int FULL_CAP = 1 << 22;
  extern __shared__ __align__(16) unsigned char q_raw[];
  const int t = blockIdx.x;
  if (t >= ntiles) return;
  // stage tiles start on a 1024-byte boundary of the shared window (swizzle atoms)
  unsigned char *sm = q_raw + ((1024u - (smem_u32(q_raw) & 1023u)) & 1023u);
  uint64_t *full = reinterpret_cast<uint64_t *>(sm + Q_STAGES * Q_STAGE_BYTES);
  uint64_t *empty = full + Q_STAGES;
  uint64_t *done = empty + Q_STAGES;
  uint32_t *taddr_s = reinterpret_cast<uint32_t *>(done + 1);
  volatile int *abort_s = reinterpret_cast<volatile int *>(taddr_s + 1);
  volatile int *issued_s = abort_s + 1;  // k chunks whose MMAs were issued
  int lo = 0, hi = nitems - 1;  // last item with tile0 <= t
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (items[mid].tile0 <= t) lo = mid;
    else hi = mid - 1;
  }
  const CgItem it = items[lo];
  const int ntm = (it.M + Q_BM - 1) / Q_BM;
  const int ti = t - it.tile0, tm = ti % ntm, tn = ti / ntm;
  const int i0 = tm * Q_BM, j0 = tn * Q_BN;
  int klo = 0, khi = it.K;
  if (it.mode == 1) khi = min(it.K, i0 + Q_BM - it.koff);
  if (it.mode == 2) klo = max(0, j0 - it.koff);
  if (it.mode == 3) klo = max(0, i0 - it.koff);
  const int nk = khi > klo ? (khi - klo + Q_BK - 1) / Q_BK : 0;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(taddr_s)),
                 "r"(Q_TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    for (int s = 0; s < Q_STAGES; ++s) {
      mbar_init(smem_u32(full + s), Q_NPROD);
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
  if (tid < Q_NPROD) {
    // ---- producers: thread -> (A row, 16 consecutive k) and (B column, 8
    // consecutive k), the fast thread index along each operand's contiguous
    // dimension so that every warp-wide load is coalesced
    const cx<float> *A = bufs.p[it.abuf] + it.a;
    const cx<float> *B = bufs.p[it.bbuf] + it.b;
    const int64_t *G = it.gath >= 0 ? gidx + it.gath : nullptr;
    const bool afast = it.a_rs == 1, bfast = it.b_cs == 1;
    const int ax = afast ? (tid & 127) : (tid >> 1), akh = afast ? (tid >> 7) : (tid & 1);
    const int bn = bfast ? (tid & 63) : (tid >> 2), bkq = bfast ? (tid >> 6) : (tid & 3);
    const int ai = i0 + ax, bj = j0 + bn;
    const cx<float> *Arow = A + (int64_t)ai * it.a_rs;
    cx<float> ra[16], rb[8];
    auto load = [&](int k0) {
#pragma unroll
      for (int e = 0; e < 16; ++e) {
        const int k = k0 + akh * 16 + e;
        ra[e] = (ai < it.M && k < khi) ? Arow[(int64_t)k * it.a_cs] : mk<float>(0.f, 0.f);
      }
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const int k = k0 + bkq * 8 + e;
        cx<float> v = mk<float>(0.f, 0.f);
        if (bj < it.N && k < khi) {
          const int64_t kr = G ? G[k] : (int64_t)k;
          v = B[kr * it.b_rs + (int64_t)bj * it.b_cs];
        }
        rb[e] = v;
      }
    };
    if (nk > 0) load(klo);
    for (int kc = 0; kc < nk; ++kc) {
      const int s = kc & 1;
      if (kc >= Q_STAGES &&
          !mbar_wait_bounded(smem_u32(empty + s), (uint32_t)(((kc >> 1) - 1) & 1), wait_cap)) {
        *abort_s = 1;
        break;
      }
      if (*abort_s) break;
      unsigned char *st = sm + s * Q_STAGE_BYTES;
      uint4 pl[6];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        q_split8(ra + 8 * h, pl);
        const uint32_t o = q_swz(ax, akh * 2 + h);
#pragma unroll
        for (int q = 0; q < 6; ++q) *reinterpret_cast<uint4 *>(st + q * Q_APL + o) = pl[q];
      }
      q_split8(rb, pl);
      const uint32_t ob = q_swz(bn, bkq);
#pragma unroll
      for (int q = 0; q < 6; ++q) *reinterpret_cast<uint4 *>(st + G_NPL * Q_APL + q * Q_BPL + ob) = pl[q];
      // the generic-proxy stores become visible to the tensor cores (async proxy)
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      mbar_arrive(smem_u32(full + s));
      if (kc + 1 < nk) load(klo + (kc + 1) * Q_BK);
    }
  } else if (tid == Q_NPROD) {
    // ---- MMA issuer: 2 k-steps of 16 per chunk, 24 bf16 MMAs per k-step
    // (pieces h, m, l = 0, 1, 2); leading products to TMEM columns 0-127
    // (Re, Im), the correction products to 128-255
    const uint32_t id_pos = q_idesc(0), id_neg = q_idesc(1);
    constexpr int PA[6] = {0, 0, 1, 0, 2, 1}, PB[6] = {0, 1, 0, 2, 0, 1};
    int kc = 0;
    for (; kc < nk; ++kc) {
      const int s = kc & 1;
      if (*abort_s || !mbar_wait_bounded(smem_u32(full + s), (uint32_t)((kc >> 1) & 1), wait_cap)) {
        *abort_s = 1;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t st = sbase + s * Q_STAGE_BYTES, sb = st + G_NPL * Q_APL;
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
    cx<float> *C = bufs.p[it.cbuf] + it.c;
    const float al = it.alpha;
    for (int row = warp; row < Q_BM; row += Q_THREADS / 32) {
      const int i = i0 + row;
      if (i >= it.M) continue;
      for (int cc = lane; cc < Q_BN; cc += 32) {
        const int j = j0 + cc;
        if (j >= it.N) continue;
        const float2 a = stg[row * Q_CPITCH + cc];
        cx<float> *d = C + (int64_t)i * it.c_rs + (int64_t)j * it.c_cs;
        cx<float> v = mk<float>(al * a.x, al * a.y);
        if (it.beta) {
          const cx<float> o = *d;
          v.re += o.re;
          v.im += o.im;
        }
        *d = v;
      }
    }
  } else if (tid == 0) {
    atomicExch(err, 1);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(Q_TMEM_COLS));
}
