// Exact-split BF16 products of float-pair matrices on the fifth-generation
// tensor cores (tcgen05.mma, accumulators in tensor memory, operands staged in
// shared memory by tiled tensor copies).  Included by dqmc_device.cuh inside its
// namespace, after the float-pair arithmetic.
//
// Scheme (Ozaki, Ogita, Oishi & Rump, Numer. Algorithms 59, 2012, on BF16
// digits): every row i of op(A) and column j of op(B) is scaled by a power of
// two so that its entries satisfy |x| < 2^(e-1), then cut into kUmmaDig
// balanced 8-bit digits,
//     x = 2^(e-8) sum_t q_t 2^(-8t),   q_t integer, |q_t| <= 128.
// The digit planes hold q_t 2^(-8t) as BF16 (exact: eight significant bits and
// a power-of-two scale), so the product of digits t and u carries the weight of
// its diagonal d = t + u:
//     (op(A) op(B))_ij = 2^(eA_i + eB_j - 16) sum_{t,u} sum_k qA_t qB_u 2^(-8(t+u)).
// Diagonals 0..3 are accumulated in FP32 tensor-memory accumulators of their
// own: their terms are multiples of 2^(-8d) below 2^(14-8d), and (d+1) K 2^14 <=
// 2^24 keeps every partial sum exact for K <= 256 (the segment length
// kUmmaKSeg).  Diagonals 4..6 share one accumulator whose FP32 rounding is
// 2^-24 of a term already 2^-32 below the result.  Pairs with t + u > 6
// (weight < 2^-56) are dropped.  The five accumulators are summed in float
// pairs, scaled, and stored (or added) into C.
//
// Tiles: UM = 64 rows (one MMA M) x NT = 48 columns (MMA N), K in chunks of 16
// (one MMA K).  A chunk stages all digits of an A tile and a B tile: the digit
// planes are laid out in global memory (per-chain scratch, L2-resident; the
// constant propagators' planes are prepared once per model) in the order
// (tile, k chunk, digit) with each 16-wide block in the canonical K-major layout
// without swizzle.  The host describes each plane buffer by a tensor map, a 4D
// view [blocks][7 digits][rows][16 k] whose box is one whole block, so one chunk
// is two tiled tensor copies (cp.async.bulk.tensor) of 14 KB and 10.5 KB that
// reproduce the blocks byte for byte in shared memory.  The chunks of
// all tiles form one sequence streamed through three stages: while the 28 MMAs
// of chunk g run, the copies of chunks g+1 and g+2 are in flight, across tile
// boundaries too.  One thread issues the copies and the MMAs; completion is
// tracked with mbarriers whose waits give up after ~1 s (the chain's error
// word records it).
#pragma once

constexpr int kUmmaDig = 7;                 // digits per operand
constexpr int kUmmaSlots = 5;               // accumulators: diagonals 0, 1, 2, 3 and 4..6
constexpr int kUmmaM = 64;                  // tile rows (MMA M)
constexpr int kUmmaNT = 48;                 // tile columns (MMA N)
constexpr int kUmmaK = 16;                  // MMA K and staged chunk
static_assert(kUmmaDig == kPlaneDigits && kUmmaM == kPlaneRowsA && kUmmaNT == kPlaneRowsB && kUmmaK == kPlaneK,
              "the host's tensor maps describe these plane blocks");
constexpr int kUmmaKSeg = 256;              // k per exactly accumulated segment
constexpr int kUmmaCols = 256;              // tensor-memory columns allocated per CTA
constexpr int kUmmaBlockA = kUmmaM * kUmmaK * 2;    // bytes of one digit block of A
constexpr int kUmmaBlockB = kUmmaNT * kUmmaK * 2;   // ... of B
constexpr int kUmmaStageBytes = kUmmaDig * (kUmmaBlockA + kUmmaBlockB);
constexpr int kUmmaStages = 3;                             // copy pipeline depth
constexpr long long kUmmaWaitCycles = 2000000000LL;        // default wait limit, ~1 s

__host__ __device__ inline int umma_pad(int n, int q) { return (n + q - 1) / q * q; }
// bf16 elements of the digit planes of one CTA for products up to n x n x kmax
__host__ __device__ inline size_t umma_plane_elems(int n, int kmax) {
  const size_t kp = (size_t)umma_pad(kmax, kUmmaK);
  return (size_t)kUmmaDig * ((size_t)umma_pad(n, kUmmaM) + (size_t)umma_pad(n, kUmmaNT)) * kp;
}

// State of the tensor-core products of one CTA.  Nothing in it is indexed at
// run time (that would push the kernel's whole shared-memory descriptor into
// local memory): the stages are found by umma_stage, and thread 0's
// bookkeeping lives in the 128-byte shared barrier area.
struct Umma {
  const CUtensorMap* tmA; // tensor maps of the scratch planes as left / right operand
  const CUtensorMap* tmB;
  size_t boff;            // elements from the scratch planes to the right operand's planes
  unsigned char* stage0;  // first staging buffer (kUmmaStageBytes, the GEMM region)
  unsigned char* stage1;  // second; the third follows it
  uint64_t* bar;          // shared, 128 bytes: [0, 48) the 2 kUmmaStages mbarriers (copies landed
                          // per stage, then MMAs done per stage); [48, 96) thread 0's counters
                          // of copies and MMA commits issued and waited per stage; [96, 100)
                          // the TMEM slot; [100, 104) thread 0's count of products; [104, 112)
                          // a barrier that nothing arrives on (the test_stall hook)
  uint32_t* tmem_slot;    // tcgen05.alloc writes the accumulator base here
  int* err;               // chain error word (nonzero: a wait gave up)
  long long limit;        // SM cycles after which a wait gives up
  int stall;              // test hook: the first wait of a product waits on the barrier at
                          // [104, 112), which gives up after `limit`
  int* where;             // [6] or null: the first wait that gave up (kind, chunk, chunks,
                          // product ordinal, barrier word)
};

__device__ __forceinline__ unsigned char* umma_stage(const Umma& U, int st) {
  return st == 0 ? U.stage0 : U.stage1 + (size_t)(st - 1) * kUmmaStageBytes;
}
// thread 0's counters (shared): copies issued / waited, commits issued / waited, per stage
__device__ __forceinline__ uint32_t* umma_book(const Umma& U) { return reinterpret_cast<uint32_t*>(U.bar + 2 * kUmmaStages); }
__device__ __forceinline__ uint32_t* umma_calls(const Umma& U) { return U.tmem_slot + 1; }
__device__ __forceinline__ uint64_t* umma_never(const Umma& U) { return U.bar + 2 * kUmmaStages + 7; }

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor: K-major operand without swizzle; lbo = byte
// distance of core matrices adjacent in K, sbo = in M / N.
__device__ __forceinline__ uint64_t umma_sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version of this architecture
  return d;
}
// Instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both K-major.
__host__ __device__ constexpr uint32_t umma_idesc(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
// Wait for the phase of the given parity to complete; false if it gave up
// after `limit` SM cycles.  Polls with the non-blocking test_wait, so that the
// limit holds however short it is.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, long long limit) {
  const uint32_t a = smem_u32(bar);
  const long long t0 = clock64();
  while (true) {
    uint32_t done;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
    if (clock64() - t0 > limit) return false;
  }
}
// One block of digit planes (all seven digits of a tile x 16-wide K chunk)
// into shared memory: a tiled tensor copy of box (16, rows, 7, 1) at block
// coordinate `block` of the 4D view [blocks][7][rows][16] the map describes.
__device__ __forceinline__ void tma_load_block(void* dst, const CUtensorMap* tm, int block, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
      "[%6];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(tm)), "r"(0), "r"(0), "r"(0), "r"(block), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void umma_bf16(uint32_t dtm, uint64_t ad, uint64_t bd, uint32_t id, uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtm),
      "l"(ad), "l"(bd), "r"(id), "r"(acc));
}
__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float* v) {
  uint32_t r[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
#pragma unroll
  for (int q = 0; q < 8; ++q) v[q] = __uint_as_float(r[q]);
}
__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Tensor memory of the CTA: warp 0 allocates kUmmaCols columns (at most two
// CTAs of a product kernel share an SM, so the 512 columns of an SM never run
// out) and gives up the right to allocate more; the base goes to *slot.
__device__ inline void umma_alloc(const Umma& U) {
  if ((threadIdx.x >> 5) == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(U.tmem_slot)),
                 "r"(kUmmaCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  // the copy and MMA barriers live for the whole kernel: initialised once here,
  // never re-initialised while an arrival could still be on its way
  if (threadIdx.x == 0) {
    for (int q = 0; q < 2 * kUmmaStages; ++q) mbar_init(U.bar + q);
    mbar_init(umma_never(U));
    uint32_t* book = umma_book(U);
    for (int q = 0; q < 4 * kUmmaStages; ++q) book[q] = 0u;
    *umma_calls(U) = 0u;
  }
  // tiled tensor copies need 128-byte aligned shared destinations: a staging
  // buffer that is not marks the products void (they are then skipped and the
  // call reports it) instead of issuing a copy the hardware would reject
  if (threadIdx.x == 0 && (((smem_u32(U.stage0) | smem_u32(U.stage1)) & 127u) != 0u)) {
    if (U.where && U.where[0] == 0) U.where[0] = 9;
    if (U.err) atomicOr(U.err, 2);
  }
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
}
// Every path out of a kernel that allocated calls this (all threads).
__device__ inline void umma_free(const Umma& U) {
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if ((threadIdx.x >> 5) == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(*U.tmem_slot), "r"(kUmmaCols)
                 : "memory");
}

// Offset (elements) of (r, k) inside a digit block of 16 k: core matrices of 8
// rows x 8 k (128 bytes, rows 16 bytes apart), k groups 128 bytes apart, row
// groups 256 bytes apart.
__device__ __forceinline__ int umma_core_off(int r, int k) { return (r >> 3) * 128 + (k >> 3) * 64 + (r & 7) * 8 + (k & 7); }

// Eight consecutive k of one row (or column) cut into digits: writes one
// 16-byte core row per digit, blocks `bstride` elements apart.
__device__ __forceinline__ void umma_split8(const dd* x, int e, __nv_bfloat16* out, size_t bstride) {
  float h[8], l[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    h[q] = ldexpf(x[q].hi, -e);
    l[q] = ldexpf(x[q].lo, -e);
  }
#pragma unroll
  for (int t = 0; t < kUmmaDig; ++t) {
    float dg[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      h[q] *= 256.f;
      l[q] *= 256.f;
      const float qt = rintf(h[q]);
      dg[q] = ldexpf(qt, -8 * t);
      const dd r = two_sum(h[q] - qt, l[q]);
      h[q] = r.hi;
      l[q] = r.lo;
    }
    uint32_t w[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const __nv_bfloat162 p2 = __floats2bfloat162_rn(dg[2 * q], dg[2 * q + 1]);  // exact: 8-bit digits
      w[q] = *reinterpret_cast<const uint32_t*>(&p2);
    }
    *reinterpret_cast<uint4*>(out + (size_t)t * bstride) = make_uint4(w[0], w[1], w[2], w[3]);
  }
}

// Exponents of the logical rows of an operand (R x Kd, padded to Rp rows):
// |x| < 2^(e-1) for every entry of the row (0 for an all-zero or padding row).
// TR: logical row r is column r of X (X[k * ldx + r]); else row r.
template <bool TR>
__device__ void umma_row_exponents(int R, int Kd, const dd* X, int ldx, int Rp, int* ex) {
  const int tid = threadIdx.x, warp_id = tid >> 5, lane_id = tid & 31;
  auto expo = [](float amax) { return amax > 0.f ? ilogbf(amax) + 2 : 0; };
  if (!TR) {
    for (int r = warp_id; r < Rp; r += kThreads / 32) {
      float amax = 0.f;
      if (r < R)
        for (int k = lane_id; k < Kd; k += 32) amax = fmaxf(amax, fabsf(X[(size_t)r * ldx + k].hi));
#pragma unroll
      for (int o = 16; o; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
      if (lane_id == 0) ex[r] = expo(amax);
    }
  } else {
    for (int r = tid; r < Rp; r += kThreads) {
      float amax = 0.f;
      if (r < R)
        for (int k = 0; k < Kd; ++k) amax = fmaxf(amax, fabsf(X[(size_t)k * ldx + r].hi));
      ex[r] = expo(amax);
    }
  }
}

// A split operand prepared once (the constant propagators e^-+dtau K): its digit
// planes in the product's layout and its row exponents; null planes: split the
// operand inside the product.
struct UmmaOperand {
  const __nv_bfloat16* planes;
  const int* ex;
  const CUtensorMap* tm;  // its tensor map (the 4D block view of `planes`)
};

// Digit planes of op(A) (rows of tile height UM) or of op(B)^T (rows = columns
// of op(B), tile height NT): P[(tile * nkc + kc) * kUmmaDig + t] is a block of
// `tile_rows` x 16.  TR: the logical row r of the operand is column r of X
// (X[k * ldx + r]); else row r (X[r * ldx + k]).
template <bool TR>
__device__ void umma_planes(int R, int Kd, const dd* X, int ldx, int Rp, int Kp, int tile_rows, const int* ex,
                            __nv_bfloat16* P) {
  const int nkc = Kp / kUmmaK, kg8 = Kp / 8;
  const size_t blk = (size_t)tile_rows * kUmmaK;
  const int items = Rp * kg8;
  for (int e = threadIdx.x; e < items; e += kThreads) {
    int r, g;
    if (TR) { g = e / Rp; r = e - g * Rp; } else { r = e / kg8; g = e - r * kg8; }
    const int k0 = 8 * g;
    dd x[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int k = k0 + q;
      x[q] = (r < R && k < Kd) ? (TR ? X[(size_t)k * ldx + r] : X[(size_t)r * ldx + k]) : dd{0.f, 0.f};
    }
    const int tile = r / tile_rows, rr = r - tile * tile_rows, kc = k0 / kUmmaK;
    __nv_bfloat16* out = P + ((size_t)tile * nkc + kc) * kUmmaDig * blk + umma_core_off(rr, k0 - kc * kUmmaK);
    umma_split8(x, ex[r], out, blk);
  }
}

// TMEM lane of tile row r for an M = 64 accumulator: rows 16q..16q+15 sit in
// lanes 32q..32q+15 (the four 32-lane sub-partitions, first half each).
__device__ __forceinline__ int umma_lane_of_row64(int r) { return ((r >> 4) << 5) + (r & 15); }

// C (+)= op(A) op(B), M x Nc, inner dimension Kd, float-pair operands (global
// or L2-resident), on the tensor cores.  All threads of the CTA call it.
// planes: the chain's scratch (left operand's planes at the start, the right
// operand's at U.boff; U.tmA / U.tmB their tensor maps); expA, expB: shared
// [roundup(M,64)], [roundup(Nc,48)] ints.  C must not alias A or B.
template <bool TA, bool TB, bool ACC>
__device__ void gemm_umma(int M, int Nc, int Kd, const dd* __restrict__ A, int lda, const dd* __restrict__ B, int ldb,
                          dd* __restrict__ C, int ldc, __nv_bfloat16* planes, int* expA_s, int* expB_s, const Umma U,
                          UmmaOperand cA = {nullptr, nullptr, nullptr}, UmmaOperand cB = {nullptr, nullptr, nullptr}) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int Mp = umma_pad(M, kUmmaM), Np = umma_pad(Nc, kUmmaNT), Kp = umma_pad(Kd, kUmmaK);
  const int nmt = Mp / kUmmaM, nnt = Np / kUmmaNT, nkc = Kp / kUmmaK;
  // after a wait gave up (in this or an earlier product of the kernel) the
  // products are skipped: the results are void and the host reports it
  // (the chain's error word is shared with the peer flavor's CTA: thread 0
  // reads it once for the whole CTA)
  if (tid == 0) *umma_calls(U) += 1u;
  if (__syncthreads_or(tid == 0 && U.err && (*(volatile int*)U.err & 2))) return;
  // earlier generic writes of the staging area (other products) before the
  // copies of this one
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  const CUtensorMap* tmA = cA.planes ? cA.tm : U.tmA;
  const CUtensorMap* tmB = cB.planes ? cB.tm : U.tmB;
  const int* expA = cA.planes ? cA.ex : expA_s;
  const int* expB = cB.planes ? cB.ex : expB_s;
  if (!cA.planes) umma_row_exponents<TA>(M, Kd, A, lda, Mp, expA_s);
  if (!cB.planes) umma_row_exponents<!TB>(Nc, Kd, B, ldb, Np, expB_s);
  __syncthreads();
  if (!cA.planes) {
    umma_planes<TA>(M, Kd, A, lda, Mp, Kp, kUmmaM, expA_s, planes);
  }
  if (!cB.planes) {
    __nv_bfloat16* pb = planes + U.boff;
    umma_planes<!TB>(Nc, Kd, B, ldb, Np, Kp, kUmmaNT, expB_s, pb);
  }
  // the planes are read by the bulk copies (async proxy)
  asm volatile("fence.proxy.async.global;" ::: "memory");
  __syncthreads();
  const uint32_t tmem = *U.tmem_slot;
  constexpr uint32_t idesc = umma_idesc(kUmmaM, kUmmaNT);
  // chunk sequence: tiles (mt, nt) in order, within a tile its k chunks; a tile's
  // chunks are accumulated in segments of kUmmaKSeg
  const int segc = kUmmaKSeg / kUmmaK;
  const int nch = nmt * nnt * nkc;
  // Thread 0's bookkeeping (U.cpy_*, U.mma_*: copies and MMA commits issued and
  // waited per stage, continued across the products of the kernel).  Every
  // barrier has at most one phase in flight when it is waited on (a stage is
  // refilled only after its MMAs are done, its MMAs issued only after its copy
  // landed, and every product ends with all of them waited), so parity waits are
  // sound.  live: no wait has given up; once one has, nothing more is issued and
  // the end of the product drains what is in flight before the tensor memory and
  // the staging buffers are used again.
  uint32_t* cpy_n = umma_book(U);
  uint32_t* cpy_w = cpy_n + kUmmaStages;
  uint32_t* mma_n = cpy_n + 2 * kUmmaStages;
  uint32_t* mma_w = cpy_n + 3 * kUmmaStages;
  bool live = true;
  auto gave_up = [&](int kind, int g) {
    if (live && U.where && U.where[0] == 0) {
      const int st = g % kUmmaStages;
      unsigned long long w = 0;
      asm volatile("ld.shared.b64 %0, [%1];" : "=l"(w) : "r"(smem_u32(U.bar + (kind == 1 ? st : kUmmaStages + st))));
      U.where[0] = kind;
      U.where[1] = g;
      U.where[2] = nch;
      U.where[3] = (int)*umma_calls(U);
      U.where[4] = (int)(w & 0xffffffffu);
      U.where[5] = (int)(w >> 32);
    }
    live = false;
  };
  uint64_t* bar_full = U.bar;
  uint64_t* bar_mma = U.bar + kUmmaStages;
  auto wait_mma = [&](int st, long long lim) {
    if (mma_w[st] == mma_n[st]) return true;
    if (!mbar_wait(bar_mma + st, (mma_n[st] - 1) & 1, lim)) return false;
    mma_w[st] = mma_n[st];
    return true;
  };
  auto wait_copy = [&](int st, long long lim) {
    if (cpy_w[st] == cpy_n[st]) return true;
    if (!mbar_wait(bar_full + st, (cpy_n[st] - 1) & 1, lim)) return false;
    cpy_w[st] = cpy_n[st];
    return true;
  };
  auto issue_copy = [&](int g) {  // thread 0: chunk g into stage g % kUmmaStages
    if (!live || g >= nch) return;
    const int st = g % kUmmaStages;
    if (!wait_mma(st, U.limit)) { gave_up(2, g); return; }
    const int tile = g / nkc, kc = g - tile * nkc, mt = tile / nnt, nt = tile - mt * nnt;
    mbar_expect_tx(bar_full + st, kUmmaStageBytes);
    unsigned char* dst = umma_stage(U, st);
    tma_load_block(dst, tmA, mt * nkc + kc, bar_full + st);
    tma_load_block(dst + kUmmaDig * kUmmaBlockA, tmB, nt * nkc + kc, bar_full + st);
    ++cpy_n[st];
  };
  if (tid == 0)
    for (int g = 0; g < kUmmaStages - 1; ++g) issue_copy(g);
  uint32_t written = 0u;
  for (int g = 0; g < nch; ++g) {
    const int st = g % kUmmaStages;
    const int tile = g / nkc, kc = g - tile * nkc, mt = tile / nnt, nt = tile - mt * nnt;
    if (kc % segc == 0) written = 0u;
    if (tid == 0 && live) {
      bool landed = wait_copy(st, U.limit);
      // test hook: a wait that cannot end (its barrier's phase 0 never completes)
      if (landed && U.stall && g == 0) landed = mbar_wait(umma_never(U), 0u, U.limit);
      if (!landed) {
        gave_up(1, g);
      } else {
        tc_fence_after();
        const uint32_t sa = smem_u32(umma_stage(U, st));
        const uint32_t sb = sa + kUmmaDig * kUmmaBlockA;
#pragma unroll
        for (int t = 0; t < kUmmaDig; ++t)
#pragma unroll
          for (int u = 0; t + u < kUmmaDig; ++u) {
            const int d = (t + u < kUmmaSlots - 1) ? t + u : kUmmaSlots - 1;
            const uint64_t ad = umma_sdesc(sa + t * kUmmaBlockA, 128, 256);
            const uint64_t bd = umma_sdesc(sb + u * kUmmaBlockB, 128, 256);
            umma_bf16(tmem + d * kUmmaNT, ad, bd, idesc, (written >> d) & 1u);
            written |= 1u << d;
          }
        umma_commit(bar_mma + st);
        ++mma_n[st];
      }
    }
    // keep two chunks in flight: chunk g+2 goes where chunk g-1 was, whose MMAs
    // were issued before chunk g's (waiting for them does not drain the pipe)
    if (tid == 0) issue_copy(g + kUmmaStages - 1);
    const bool seg_end = (kc + 1 == nkc) || ((kc + 1) % segc == 0);
    if (!seg_end) continue;
    // epilogue of a tile segment: all its MMAs done (the last commit covers
    // every MMA issued before it); thread 0 waits, then releases the CTA
    if (tid == 0 && live && !wait_mma(st, U.limit)) gave_up(3, g);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const int ks = kc - kc % segc;
    // warp w reads sub-partition w % 4 (rows 16 (w % 4) .. + 15 in its lanes
    // 0..15) and the column half w / 4 of the tile
    const int rloc = (warp & 3) * 16 + (lane & 15);
    const int row = mt * kUmmaM + rloc;
    const bool live_row = (lane < 16) && row < M;
    const int eA = live_row ? expA[row] : 0;
    const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;
    for (int c0 = (warp >> 2) * (kUmmaNT / 2); c0 < (warp >> 2) * (kUmmaNT / 2) + kUmmaNT / 2; c0 += 8) {
      float v[kUmmaSlots][8];
#pragma unroll
      for (int d = 0; d < kUmmaSlots; ++d) tmem_ld8(tmem + lane_base + d * kUmmaNT + c0, v[d]);
      tmem_ld_wait();
      if (live_row) {
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int col = nt * kUmmaNT + c0 + q;
          if (col < Nc) {
            dd sum = {v[kUmmaSlots - 1][q], 0.f};
#pragma unroll
            for (int d = kUmmaSlots - 2; d >= 0; --d) sum = dd_add(sum, {v[d][q], 0.f});
            const int e = eA + expB[col] - 16;
            sum.hi = ldexpf(sum.hi, e);
            sum.lo = ldexpf(sum.lo, e);
            dd* cp = C + (size_t)row * ldc + col;
            *cp = (ACC || ks > 0) ? dd_add(*cp, sum) : sum;
          }
        }
      }
    }
    // the accumulators are overwritten by the next segment's first MMAs
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
  }
  if (tid == 0) {
    // every copy and every MMA commit of the product waited for (all complete
    // already unless a wait gave up: then with the default limit, a drain)
    for (int st = 0; st < kUmmaStages; ++st) {
      const long long lim = live ? U.limit : kUmmaWaitCycles;
      if (!wait_copy(st, lim) && live) gave_up(4, st);
      if (!wait_mma(st, lim) && live) gave_up(5, st);
    }
  }
  const bool ok = live;
  // the staging buffers are reused by generic loads and stores after the product
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  if (!ok && U.err) atomicOr(U.err, 2);
  __syncthreads();
}
