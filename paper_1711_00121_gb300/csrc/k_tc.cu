// Tensor-core (tcgen05) symmetric rank-update of S, used by the deferred and
// per-update S passes and by the one-shot batch form:
//   S[I,J] += D_IJ,  S[J,I] += D_IJ^T  (I <= J),   D = A B^T,
// where row a of A is [xi terms | eta terms] and row a of B is the same row
// with its two halves swapped, so A B^T = Xi H^T + H Xi^T (Alg 1's
// S + M + M^T for every pending term; the proof of Thm 2, Eq. 23-28, for all
// sinks of a batch).  FP32 accuracy from a 3-term split x = hi + lo of the
// operands:
//   D = A_hi B_hi^T + A_hi B_lo^T + A_lo B_hi^T,  accumulated in FP32 (TMEM),
// with hi and lo in TF32 (kind::tf32) or, at twice the tensor rate, in FP16
// (kind::f16) after a power-of-two scaling of each term (exact, see the pack).
//
// k_s_update_tc: one CTA per SM, persistent over the tile-pair list.  Warp 0
// issues TMA loads (128 rows x 128 bytes boxes, 128-byte swizzle) into a
// 2- or 3-stage ring; warp 1 owns two TMEM accumulators (128 lanes x 128
// columns each) and issues tcgen05.mma (M = 128, N = 128, K = 32 bytes) for
// tile t + 1 while warps 2-9 drain tile t, either through a shared copy of
// the accumulator with coalesced 16-byte accesses of S[I,J] (and S[J,I] when
// both triangles are kept) or straight from registers (wide operands).
// k_s_update_tc_pair (upper tiles, wide operands): jobs of two tile pairs
// (I, J), (I, J+1) sharing A(I), one M = 128, N = 256 product per split term
// into a 256-column accumulator.
// Every mbarrier wait is bounded and every stop decision of the epilogue
// warps is taken by all of them: on timeout the kernel records a status word,
// skips the remaining work and still frees its TMEM.
#include <cuda.h>

#include <type_traits>

#include "sr_internal.h"

namespace sr {

namespace {

constexpr int TM = 128;             // rows of an S tile (M)
constexpr int TN = 128;             // columns of an S tile (N)
constexpr int KB = 128;             // bytes of K per stage (one 128-byte swizzle row)
constexpr int STAGES_STAGED = 2;  // stages when the epilogue stages D in shared memory
constexpr int STAGES_DIRECT = 3;  // stages when it adds D to S straight from registers
constexpr int OPB = TM * KB;        // bytes of one operand box: 16 KB
constexpr int STAGE_BYTES = 4 * OPB;
constexpr int TC_THREADS = 320;       // 10 warps: TMA, MMA, 8 epilogue
constexpr uint32_t TMEM_COLS = 256;   // two 128-column accumulators
constexpr int EP = TN + 1;            // row pitch of the shared accumulator copy

// tcgen05 instruction descriptors: D = F32, A and B of the same type, both
// K-major, N = 128, M = 128; kind::tf32 (type code 2) or kind::f16 (F16 = 0).
constexpr uint32_t IDESC_TF32 = (1u << 4) | (2u << 7) | (2u << 10) |
                                ((uint32_t)(TN >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);
constexpr uint32_t IDESC_F16 = (1u << 4) | (0u << 7) | (0u << 10) |
                               ((uint32_t)(TN >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);
// the same with N = 256 (two column tiles side by side)
constexpr uint32_t IDESC_TF32_N256 = (1u << 4) | (2u << 7) | (2u << 10) |
                                     ((uint32_t)(256 >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);
constexpr uint32_t IDESC_F16_N256 = (1u << 4) | (0u << 7) | (0u << 10) |
                                    ((uint32_t)(256 >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// Bounded wait for the phase of `parity` to complete.  Returns false on timeout.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, long long limit,
                                          volatile int* abort_flag) {
  for (long long it = 0; it < limit; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.b32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    if (ok) return true;
    if ((it & 1023) == 1023 && *abort_flag) return false;
  }
  return false;
}

// Wait with a fixed bound of its own, for draining copies and MMAs in flight
// after a stop (their completion does not depend on any other thread).
__device__ __forceinline__ void mbar_drain_wait(uint32_t bar, uint32_t parity) {
  for (long long it = 0; it < (1ll << 24); ++it) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.b32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    if (ok) return;
  }
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y,
                                            uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
      "l"((uint64_t)map), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 bytes apart (SBO), descriptor version 1.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFFu) >> 4);
  d |= (uint64_t)(16u >> 4) << 16;
  d |= (uint64_t)(1024u >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

template <bool F16>
__device__ __forceinline__ void mma_k32b(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc,
                                         uint32_t accumulate) {
  if (F16) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(IDESC_F16), "r"(accumulate)
        : "memory");
  } else {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(IDESC_TF32), "r"(accumulate)
        : "memory");
  }
}

// One MMA with a run-time instruction descriptor (N = 128 or 256).
template <bool F16>
__device__ __forceinline__ void mma_k32b_d(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc,
                                           uint32_t idesc, uint32_t accumulate) {
  if (F16) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
  } else {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
  }
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   bar)
               : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
      "%12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, "
      "%30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int q = 0; q < 32; ++q) v[q] = __uint_as_float(r[q]);
}

// true on all 256 epilogue threads iff pred is true on all of them (barrier 1)
__device__ __forceinline__ bool ep_all(bool pred) {
  uint32_t r;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.and.pred q, 1, 256, p;\n"
      " selp.u32 %0, 1, 0, q;\n}\n"
      : "=r"(r)
      : "r"((uint32_t)pred)
      : "memory");
  return r != 0;
}
__device__ __forceinline__ void ep_sync() { asm volatile("bar.sync 1, 256;" ::: "memory"); }

// One tile pair of the pass: where its S lives, the rows of its two operand
// tiles, and whether S[J, I] is kept as well.
struct TcRef {
  float* S;
  int64_t ld;
  int I, J, rowI, rowJ, n;
  bool mirror;
};

// Tile pairs of one graph: tiles[t] = I << 16 | J (band order); a pair is
// skipped when use_masks and its mask words show no active cross term.
struct TcOneGraph {
  const uint32_t* tiles;
  int nt;
  const uint64_t* mX;
  const uint64_t* mE;
  int use_masks;
  float* S;
  int64_t ld;
  int n, mirror;
  __device__ __forceinline__ int count() const { return nt; }
  __device__ __forceinline__ bool get(int t, TcRef& r) const {
    const uint32_t pr = tiles[t];
    r.I = (int)(pr >> 16);
    r.J = (int)(pr & 0xffffu);
    if (use_masks && ((mX[r.I] & mE[r.J]) | (mE[r.I] & mX[r.J])) == 0ull) return false;
    r.S = S;
    r.ld = ld;
    r.rowI = r.I * TM;
    r.rowJ = r.J * TN;
    r.n = n;
    r.mirror = mirror != 0;
    return true;
  }
};

// Tile pairs of many graphs: tiles[t] = g << 32 | I << 16 | J, *ntiles of
// them; graph g's operand rows start at descs[g].row_off.
struct TcManyGraphs {
  const uint64_t* tiles;
  const int* ntiles;
  const MultiGraphDesc* d;
  __device__ __forceinline__ int count() const { return *ntiles; }
  __device__ __forceinline__ bool get(int t, TcRef& r) const {
    const uint64_t e = tiles[t];
    const MultiGraphDesc& q = d[(int)(e >> 32)];
    r.I = (int)((e >> 16) & 0xffffu);
    r.J = (int)(e & 0xffffu);
    r.S = (float*)q.S;
    r.ld = q.ld;
    r.rowI = (int)q.row_off + r.I * TM;
    r.rowJ = (int)q.row_off + r.J * TN;
    r.n = q.n;
    r.mirror = q.upper == 0;
    return true;
  }
};

// STAGED: the epilogue copies D into shared memory and streams S with
// coalesced 512-byte row segments (2 TMA stages); it also adds D^T to S[J, I]
// when both triangles are kept (MIRROR).  SW (staged, upper tiles only): D is
// staged as four 128 x 32 boxes in the 128-byte swizzle, so that both the
// TMEM-row writes and the row-segment reads are free of bank conflicts, and
// each warp's 16 rows of S[I, J] are fetched before the accumulator wait.
// Otherwise (wide operands: the pass is bound by the tensor cores) each
// epilogue thread adds its row's 64 values of D to S straight from the TMEM
// load, with those S values fetched before the accumulator is ready, and the
// TMA ring has 3 stages.
template <bool F16, bool STAGED, bool MIRROR, bool SW, typename Src>
__global__ void __launch_bounds__(TC_THREADS, 1)
    k_s_update_tc(const __grid_constant__ CUtensorMap tm_hi,
                  const __grid_constant__ CUtensorMap tm_lo,
                  const __grid_constant__ CUtensorMap tm_bhi,
                  const __grid_constant__ CUtensorMap tm_blo, Src src, int nkb, int bswap,
                  long long wait_limit, unsigned long long* __restrict__ counters) {
  static_assert(STAGED || !MIRROR, "the transposed write needs the staged epilogue");
  static_assert(!SW || (STAGED && !MIRROR), "the swizzled epilogue keeps upper tiles only");
  constexpr int STAGES = STAGED ? STAGES_STAGED : STAGES_DIRECT;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bar_full[STAGES], bar_empty[STAGES];
  __shared__ __align__(8) uint64_t bar_acc_full[2], bar_acc_empty[2];
  // the MMA warp hands each active pair (I < 0: no more) to the epilogue with
  // its accumulator slot, so that the epilogue's S loads wait on no list or
  // mask reads of its own
  __shared__ TcRef ep_ref[2];
  __shared__ __align__(8) uint64_t bar_ref[2];
  __shared__ uint32_t tmem_base;
  __shared__ volatile int abort_flag;
  __shared__ __align__(8) uint64_t bar_drain;  // MMAs still in flight after a stop
  uint32_t it_issued = 0;                    // stages the TMA thread has loaded

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t base = (smem_u32(smem_raw) + 1023u) & ~1023u;
  float* sD = reinterpret_cast<float*>(smem_raw + (base - smem_u32(smem_raw)) +
                                       (size_t)STAGES * STAGE_BYTES);
  const int half = nkb / 2;  // bswap: B row = A row with its halves swapped
  const int nt = src.count();

  if (threadIdx.x == 0) {
    abort_flag = 0;
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(smem_u32(&bar_full[s]), 1);
      mbar_init(smem_u32(&bar_empty[s]), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(smem_u32(&bar_acc_full[b]), 1);
      mbar_init(smem_u32(&bar_acc_empty[b]), 256);
      mbar_init(smem_u32(&bar_ref[b]), 1);
    }
    mbar_init(smem_u32(&bar_drain), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_base)),
                 "r"(TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;
  bool ok = true;

  if (warp == 0) {
    // ---------------- TMA producer
    if (lane == 0) {
      uint32_t it = 0;
      for (int t = blockIdx.x; t < nt && ok; t += gridDim.x) {
        TcRef r;
        if (!src.get(t, r)) continue;
        for (int kb = 0; kb < nkb && ok; ++kb, ++it) {
          const int s = it % STAGES;
          const uint32_t ph = (it / STAGES) & 1u;
          if (!mbar_wait(smem_u32(&bar_empty[s]), ph ^ 1u, wait_limit, &abort_flag)) {
            ok = false;
            break;
          }
          const uint32_t st = base + s * STAGE_BYTES;
          const uint32_t fb = smem_u32(&bar_full[s]);
          mbar_expect_tx(fb, STAGE_BYTES);
          const int kb_b = !bswap ? kb : kb < half ? kb + half : kb - half;
          constexpr int KCH = F16 ? KB / 2 : KB / 4;  // elements of K per stage
          tma_load_2d(st + 0 * OPB, &tm_hi, kb * KCH, r.rowI, fb);
          tma_load_2d(st + 1 * OPB, &tm_lo, kb * KCH, r.rowI, fb);
          tma_load_2d(st + 2 * OPB, &tm_bhi, kb_b * KCH, r.rowJ, fb);
          tma_load_2d(st + 3 * OPB, &tm_blo, kb_b * KCH, r.rowJ, fb);
        }
      }
      it_issued = it;
      if (!ok) abort_flag = 1;
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer: tile tl accumulates in TMEM columns (tl & 1) * 128
    if (lane == 0) {
      uint32_t it = 0, tl = 0;
      for (int t = blockIdx.x; t < nt && ok; t += gridDim.x) {
        TcRef r;
        if (!src.get(t, r)) continue;
        const uint32_t b = tl & 1u;
        const uint32_t eph = ((tl >> 1) & 1u) ^ 1u;
        ++tl;
        if (!mbar_wait(smem_u32(&bar_acc_empty[b]), eph, wait_limit, &abort_flag)) {
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        ep_ref[b] = r;
        mbar_arrive(smem_u32(&bar_ref[b]));
        const uint32_t acc = tmem + b * (uint32_t)TN;
        for (int kb = 0; kb < nkb; ++kb, ++it) {
          const int s = it % STAGES;
          const uint32_t ph = (it / STAGES) & 1u;
          if (!mbar_wait(smem_u32(&bar_full[s]), ph, wait_limit, &abort_flag)) {
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t st = base + s * STAGE_BYTES;
          const uint64_t a_hi = smem_desc(st + 0 * OPB), a_lo = smem_desc(st + 1 * OPB);
          const uint64_t b_hi = smem_desc(st + 2 * OPB), b_lo = smem_desc(st + 3 * OPB);
#pragma unroll
          for (int kk = 0; kk < KB / 32; ++kk) {
            // one MMA covers 32 bytes of K: 8 TF32 or 16 FP16 elements
            const uint64_t adv = (uint64_t)(kk * 32) >> 4;
            const uint32_t first = (kb == 0 && kk == 0) ? 0u : 1u;
            mma_k32b<F16>(acc, a_hi + adv, b_hi + adv, first);
            mma_k32b<F16>(acc, a_hi + adv, b_lo + adv, 1u);
            mma_k32b<F16>(acc, a_lo + adv, b_hi + adv, 1u);
          }
          mma_commit(smem_u32(&bar_empty[s]));  // stage reusable once these MMAs finish
        }
        if (!ok) break;
        mma_commit(smem_u32(&bar_acc_full[b]));
      }
      if (ok) {
        // end of the list, in the next slot once the epilogue has left it
        const uint32_t b = tl & 1u;
        if (!mbar_wait(smem_u32(&bar_acc_empty[b]), ((tl >> 1) & 1u) ^ 1u, wait_limit,
                       &abort_flag)) {
          ok = false;
        } else {
          ep_ref[b].I = -1;
          mbar_arrive(smem_u32(&bar_ref[b]));
        }
      }
      if (!ok) abort_flag = 1;
    }
  } else {
    // ---------------- epilogue: warps 2..9 (256 threads)
    const int et = threadIdx.x - 64;     // 0..255
    const int ew = et >> 5;              // epilogue warp 0..7
    const int quarter = warp & 3;        // TMEM lanes this warp may read
    const int chalf = (ew >> 2) * 64;    // columns [chalf, chalf + 64) of the accumulator
    uint32_t tl = 0;
    unsigned long long my_tiles = 0, my_bytes = 0;
    for (;;) {
      const uint32_t b = tl & 1u;
      const uint32_t tph = (tl >> 1) & 1u;
      // each warp reads the posted pair on its own and fetches its S rows;
      // one barrier per pair (tile_go) then agrees on going on, on the end of
      // the list, or on a stop
      const bool posted =
          __all_sync(0xffffffffu, mbar_wait(smem_u32(&bar_ref[b]), tph, wait_limit, &abort_flag));
      TcRef r = {};
      if (posted) r = ep_ref[b];
      const bool go = posted && r.I >= 0;
      const bool at_end = posted && r.I < 0;
      auto tile_go = [&]() -> bool {
        const bool got =
            go ? mbar_wait(smem_u32(&bar_acc_full[b]), tph, wait_limit, &abort_flag) : at_end;
        if (ep_all(go && got)) return true;
        if (!ep_all(at_end)) ok = false;
        return false;
      };
      ++tl;
      float* __restrict__ S = r.S;
      const int64_t ld = r.ld;
      const int I = r.I, J = r.J, n = r.n;
      const bool mirror = MIRROR;
      const int row = quarter * 32 + lane;
      if (!STAGED) {
        // this thread's 64 values of S[I, J] (row `row`, columns chalf ..),
        // fetched while the tensor cores still work on the tile
        float* srow = S + (int64_t)(I * TM + row) * ld + (int64_t)J * TN + chalf;
        float4 sv[16];
        if (go) {
#pragma unroll
          for (int q = 0; q < 16; ++q) sv[q] = *reinterpret_cast<const float4*>(srow + 4 * q);
        }
        if (!tile_go()) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          float v[32];
          tmem_ld32(tmem + b * (uint32_t)TN + ((uint32_t)(quarter * 32) << 16) +
                        (uint32_t)(chalf + 32 * h),
                    v);
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            sv[8 * h + q].x += v[4 * q + 0];
            sv[8 * h + q].y += v[4 * q + 1];
            sv[8 * h + q].z += v[4 * q + 2];
            sv[8 * h + q].w += v[4 * q + 3];
          }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        mbar_arrive(smem_u32(&bar_acc_empty[b]));  // the MMA warp may refill this accumulator
#pragma unroll
        for (int q = 0; q < 16; ++q) *reinterpret_cast<float4*>(srow + 4 * q) = sv[q];
      } else {
      if (SW) {
        constexpr int NQ = TM / 8;  // rows ew + 8 q of the tile; lane l: columns 4 l .. 4 l + 3
        // this warp's rows of S[I, J], in flight while the tile is multiplied
        float4 sv[NQ];
        if (go) {
#pragma unroll
          for (int q = 0; q < NQ; ++q)
            sv[q] = *reinterpret_cast<const float4*>(S + (int64_t)(I * TM + ew + 8 * q) * ld +
                                                     (int64_t)J * TN + lane * 4);
        }
        if (!tile_go()) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        ep_sync();  // every thread is done with the previous tile's shared copy
        // accumulator -> shared tile, one 32-column box at a time: box c / 32
        // holds columns [c, c + 32); row `row` is 128 bytes at row * 128, its
        // 16-byte chunk k stored at chunk k ^ (row & 7)
        const uint32_t ta =
            tmem + b * (uint32_t)TN + ((uint32_t)(quarter * 32) << 16) + (uint32_t)chalf;
#pragma unroll 1
        for (int h = 0; h < 2; ++h) {
          float v[32];
          tmem_ld32(ta + 32u * h, v);
          float* box = sD + (chalf / 32 + h) * (TM * 32) + row * 32;
#pragma unroll
          for (int k = 0; k < 8; ++k)
            *reinterpret_cast<float4*>(box + (k ^ (row & 7)) * 4) =
                make_float4(v[4 * k], v[4 * k + 1], v[4 * k + 2], v[4 * k + 3]);
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        mbar_arrive(smem_u32(&bar_acc_empty[b]));  // the MMA warp may refill this accumulator
        ep_sync();
        // a warp covers one 512-byte row segment per access: lane l takes
        // chunk l & 7 of box l >> 3
        const float* bsrc = sD + (lane >> 3) * (TM * 32);
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
          const int tr = ew + 8 * q;
          const float4 d =
              *reinterpret_cast<const float4*>(bsrc + tr * 32 + (((lane & 7) ^ (tr & 7)) * 4));
          sv[q].x += d.x;
          sv[q].y += d.y;
          sv[q].z += d.z;
          sv[q].w += d.w;
          *reinterpret_cast<float4*>(S + (int64_t)(I * TM + tr) * ld + (int64_t)J * TN +
                                     lane * 4) = sv[q];
        }
      } else {
      if (!tile_go()) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      // accumulator -> shared tile (row = TMEM lane)
#pragma unroll 1
      for (int c0 = chalf; c0 < chalf + 64; c0 += 32) {
        float v[32];
        tmem_ld32(tmem + b * (uint32_t)TN + ((uint32_t)(quarter * 32) << 16) + (uint32_t)c0, v);
#pragma unroll
        for (int q = 0; q < 32; ++q) sD[row * EP + c0 + q] = v[q];
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      mbar_arrive(smem_u32(&bar_acc_empty[b]));  // the MMA warp may refill this accumulator
      ep_sync();
      // S[I, J] += D: a warp covers one 512-byte row segment per access
      constexpr int NQ = TM / 8;
      {
        float4 v[NQ];
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
          const int tr = ew + 8 * q;
          v[q] = *reinterpret_cast<const float4*>(S + (int64_t)(I * TM + tr) * ld + (int64_t)J * TN + lane * 4);
        }
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
          const int tr = ew + 8 * q;
          const float* d = sD + tr * EP + lane * 4;
          v[q].x += d[0];
          v[q].y += d[1];
          v[q].z += d[2];
          v[q].w += d[3];
          *reinterpret_cast<float4*>(S + (int64_t)(I * TM + tr) * ld + (int64_t)J * TN + lane * 4) = v[q];
        }
      }
      if (MIRROR && I != J) {
        // S[J, I] += D^T
        float4 v[NQ];
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
          const int c = ew + 8 * q;
          v[q] = *reinterpret_cast<const float4*>(S + (int64_t)(J * TN + c) * ld + (int64_t)I * TM + lane * 4);
        }
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
          const int c = ew + 8 * q;
          v[q].x += sD[(lane * 4 + 0) * EP + c];
          v[q].y += sD[(lane * 4 + 1) * EP + c];
          v[q].z += sD[(lane * 4 + 2) * EP + c];
          v[q].w += sD[(lane * 4 + 3) * EP + c];
          *reinterpret_cast<float4*>(S + (int64_t)(J * TN + c) * ld + (int64_t)I * TM + lane * 4) = v[q];
        }
      }
      ep_sync();  // the shared tile is free for the next accumulator
      }
      }
      if (et == 0) {
        const long long vr = max(0, min(TM, n - I * TM)), vc = max(0, min(TN, n - J * TN));
        my_tiles += 1;
        my_bytes += (unsigned long long)(vr * vc) * 8ull * ((I == J || !mirror) ? 1ull : 2ull);
      }
    }
    if (!ok) abort_flag = 1;
    if (et == 0 && my_tiles) {
      atomicAdd(&counters[CNT_TILES_TOUCHED], my_tiles);
      atomicAdd(&counters[CNT_S_BYTES], my_bytes);
    }
  }

  __syncthreads();
  if (abort_flag) {
    // a stop on timeout can leave TMA loads and MMAs of this CTA in flight:
    // wait for them (bounded on their own) before shared memory and TMEM go
    if (warp == 0 && lane == 0) {
      const uint32_t from = it_issued > (uint32_t)STAGES ? it_issued - (uint32_t)STAGES : 0u;
      for (uint32_t i = from; i < it_issued; ++i)
        mbar_drain_wait(smem_u32(&bar_full[i % STAGES]), (i / STAGES) & 1u);
    }
    if (warp == 1 && lane == 0) {
      mma_commit(smem_u32(&bar_drain));
      mbar_drain_wait(smem_u32(&bar_drain), 0u);
    }
  }
  if (threadIdx.x == 0 && abort_flag) atomicExch(&counters[CNT_STATUS], (unsigned long long)SR_ERR_TIMEOUT);
  if (warp == 1) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(TMEM_COLS));
  }
}

// Jobs of two tile pairs that share their row tile I: job = I << 32 | J1 << 16
// | J2 (J2 = 0xffff: one pair).  A pair whose AFF mask words show no active
// cross term is dropped; get() returns the active pairs (0, 1 or 2), the
// active column tiles first.
struct TcJobs {
  const uint64_t* jobs;
  int nj;
  const uint64_t* mX;
  const uint64_t* mE;
  int use_masks;
  float* S;
  int64_t ld;
  int n;
  __device__ __forceinline__ int get(int q, int& I, int& J1, int& J2) const {
    const uint64_t e = jobs[q];
    I = (int)((e >> 32) & 0xffffu);
    J1 = (int)((e >> 16) & 0xffffu);
    J2 = (int)(e & 0xffffu);
    bool a1 = true, a2 = J2 != 0xffff;
    if (use_masks) {
      a1 = ((mX[I] & mE[J1]) | (mE[I] & mX[J1])) != 0ull;
      if (a2) a2 = ((mX[I] & mE[J2]) | (mE[I] & mX[J2])) != 0ull;
    }
    if (!a1) {
      J1 = J2;
      a1 = a2;
      a2 = false;
    }
    return a1 ? (a2 ? 2 : 1) : 0;
  }
};

constexpr int STAGES_PAIR = 2;
constexpr int PAIR_STAGE_BYTES = 6 * OPB;  // A hi, A lo, B1 hi, B2 hi, B1 lo, B2 lo
constexpr uint32_t TMEM_COLS_PAIR = 512;   // two jobs in flight x 256 accumulator columns

// The S pass over jobs of two tile pairs (I, J1), (I, J2) sharing A(I): B(J1)
// and B(J2) sit side by side in shared memory as one 256-row operand, so a job
// is one M = 128, N = 256 product per split term (half the shared-memory
// operand reads per flop of two N = 128 products).  Upper tiles only (no
// transposed write); register epilogue as in k_s_update_tc.
template <bool F16>
__global__ void __launch_bounds__(TC_THREADS, 1)
    k_s_update_tc_pair(const __grid_constant__ CUtensorMap tm_hi,
                       const __grid_constant__ CUtensorMap tm_lo, TcJobs src, int nkb,
                       long long wait_limit, unsigned long long* __restrict__ counters) {
  constexpr int STAGES = STAGES_PAIR;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bar_full[STAGES], bar_empty[STAGES];
  __shared__ __align__(8) uint64_t bar_acc_full[2], bar_acc_empty[2];
  __shared__ uint32_t tmem_base;
  __shared__ volatile int abort_flag;
  __shared__ __align__(8) uint64_t bar_drain;  // MMAs still in flight after a stop
  uint32_t it_issued = 0;                    // stages the TMA thread has loaded

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t base = (smem_u32(smem_raw) + 1023u) & ~1023u;
  const int half = nkb / 2;  // B row = A row with its halves swapped
  const int nj = src.nj;

  if (threadIdx.x == 0) {
    abort_flag = 0;
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(smem_u32(&bar_full[s]), 1);
      mbar_init(smem_u32(&bar_empty[s]), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(smem_u32(&bar_acc_full[b]), 1);
      mbar_init(smem_u32(&bar_acc_empty[b]), 256);
    }
    mbar_init(smem_u32(&bar_drain), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_base)),
                 "r"(TMEM_COLS_PAIR));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;
  bool ok = true;

  if (warp == 0) {
    // ---------------- TMA producer
    if (lane == 0) {
      uint32_t it = 0;
      for (int q = blockIdx.x; q < nj && ok; q += gridDim.x) {
        int I, J1, J2;
        const int cnt = src.get(q, I, J1, J2);
        if (cnt == 0) continue;
        for (int kb = 0; kb < nkb && ok; ++kb, ++it) {
          const int s = it % STAGES;
          const uint32_t ph = (it / STAGES) & 1u;
          if (!mbar_wait(smem_u32(&bar_empty[s]), ph ^ 1u, wait_limit, &abort_flag)) {
            ok = false;
            break;
          }
          const uint32_t st = base + s * PAIR_STAGE_BYTES;
          const uint32_t fb = smem_u32(&bar_full[s]);
          mbar_expect_tx(fb, (uint32_t)(cnt == 2 ? 6 : 4) * OPB);
          const int kb_b = kb < half ? kb + half : kb - half;
          constexpr int KCH = F16 ? KB / 2 : KB / 4;  // elements of K per stage
          tma_load_2d(st + 0 * OPB, &tm_hi, kb * KCH, I * TM, fb);
          tma_load_2d(st + 1 * OPB, &tm_lo, kb * KCH, I * TM, fb);
          tma_load_2d(st + 2 * OPB, &tm_hi, kb_b * KCH, J1 * TN, fb);
          tma_load_2d(st + 4 * OPB, &tm_lo, kb_b * KCH, J1 * TN, fb);
          if (cnt == 2) {
            tma_load_2d(st + 3 * OPB, &tm_hi, kb_b * KCH, J2 * TN, fb);
            tma_load_2d(st + 5 * OPB, &tm_lo, kb_b * KCH, J2 * TN, fb);
          }
        }
      }
      it_issued = it;
      if (!ok) abort_flag = 1;
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer: job jl accumulates in TMEM columns (jl & 1) * 256 + [0, 256)
    if (lane == 0) {
      uint32_t it = 0, jl = 0;
      for (int q = blockIdx.x; q < nj && ok; q += gridDim.x) {
        int I, J1, J2;
        const int cnt = src.get(q, I, J1, J2);
        if (cnt == 0) continue;
        const uint32_t idesc = cnt == 2 ? (F16 ? IDESC_F16_N256 : IDESC_TF32_N256)
                                        : (F16 ? IDESC_F16 : IDESC_TF32);
        const uint32_t b = jl & 1u;
        const uint32_t eph = ((jl >> 1) & 1u) ^ 1u;
        ++jl;
        if (!mbar_wait(smem_u32(&bar_acc_empty[b]), eph, wait_limit, &abort_flag)) {
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t acc = tmem + b * 256u;
        for (int kb = 0; kb < nkb; ++kb, ++it) {
          const int s = it % STAGES;
          const uint32_t ph = (it / STAGES) & 1u;
          if (!mbar_wait(smem_u32(&bar_full[s]), ph, wait_limit, &abort_flag)) {
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t st = base + s * PAIR_STAGE_BYTES;
          // B hi (and B lo): rows of B(J1) then B(J2), one 256-row operand
          const uint64_t ah = smem_desc(st + 0 * OPB), al = smem_desc(st + 1 * OPB);
          const uint64_t bh = smem_desc(st + 2 * OPB), bl = smem_desc(st + 4 * OPB);
#pragma unroll
          for (int kk = 0; kk < KB / 32; ++kk) {
            const uint64_t adv = (uint64_t)(kk * 32) >> 4;
            const uint32_t first = (kb == 0 && kk == 0) ? 0u : 1u;
            mma_k32b_d<F16>(acc, ah + adv, bh + adv, idesc, first);
            mma_k32b_d<F16>(acc, ah + adv, bl + adv, idesc, 1u);
            mma_k32b_d<F16>(acc, al + adv, bh + adv, idesc, 1u);
          }
          mma_commit(smem_u32(&bar_empty[s]));  // stage reusable once these MMAs finish
        }
        if (!ok) break;
        mma_commit(smem_u32(&bar_acc_full[b]));
      }
      if (!ok) abort_flag = 1;
    }
  } else {
    // ---------------- epilogue: warps 2..9 (256 threads); S[I, J] += D per active pair
    const int et = threadIdx.x - 64;   // 0..255
    const int ew = et >> 5;            // epilogue warp 0..7
    const int quarter = warp & 3;      // TMEM lanes this warp may read
    const int chalf = (ew >> 2) * 64;  // columns [chalf, chalf + 64) of an accumulator
    const int row = quarter * 32 + lane;
    float* __restrict__ S = src.S;
    const int64_t ld = src.ld;
    const int n = src.n;
    uint32_t jl = 0;
    unsigned long long my_tiles = 0, my_bytes = 0;
    for (int q = blockIdx.x; q < nj; q += gridDim.x) {
      int I, J1, J2;
      const int cnt = src.get(q, I, J1, J2);
      if (cnt == 0) continue;
      const uint32_t b = jl & 1u;
      const uint32_t tph = (jl >> 1) & 1u;
      ++jl;
      for (int u = 0; u < cnt; ++u) {
        const int J = u ? J2 : J1;
        // this thread's 64 values of S[I, J], fetched before the accumulator is read
        float* srow = S + (int64_t)(I * TM + row) * ld + (int64_t)J * TN + chalf;
        float4 sv[16];
#pragma unroll
        for (int c = 0; c < 16; ++c) sv[c] = *reinterpret_cast<const float4*>(srow + 4 * c);
        if (u == 0) {
          const bool got = mbar_wait(smem_u32(&bar_acc_full[b]), tph, wait_limit, &abort_flag);
          if (!ep_all(got)) {
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        }
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          float v[32];
          tmem_ld32(tmem + b * 256u + (uint32_t)(u * 128) + ((uint32_t)(quarter * 32) << 16) +
                        (uint32_t)(chalf + 32 * h),
                    v);
#pragma unroll
          for (int c = 0; c < 8; ++c) {
            sv[8 * h + c].x += v[4 * c + 0];
            sv[8 * h + c].y += v[4 * c + 1];
            sv[8 * h + c].z += v[4 * c + 2];
            sv[8 * h + c].w += v[4 * c + 3];
          }
        }
        if (u == cnt - 1) {
          asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
          mbar_arrive(smem_u32(&bar_acc_empty[b]));  // both accumulators of the job are read
        }
#pragma unroll
        for (int c = 0; c < 16; ++c) *reinterpret_cast<float4*>(srow + 4 * c) = sv[c];
        if (et == 0) {
          const long long vr = max(0, min(TM, n - I * TM)), vc = max(0, min(TN, n - J * TN));
          my_tiles += 1;
          my_bytes += (unsigned long long)(vr * vc) * 8ull;
        }
      }
      if (!ok) break;
    }
    if (!ok) abort_flag = 1;
    if (et == 0 && my_tiles) {
      atomicAdd(&counters[CNT_TILES_TOUCHED], my_tiles);
      atomicAdd(&counters[CNT_S_BYTES], my_bytes);
    }
  }

  __syncthreads();
  if (abort_flag) {
    // a stop on timeout can leave TMA loads and MMAs of this CTA in flight:
    // wait for them (bounded on their own) before shared memory and TMEM go
    if (warp == 0 && lane == 0) {
      const uint32_t from = it_issued > (uint32_t)STAGES ? it_issued - (uint32_t)STAGES : 0u;
      for (uint32_t i = from; i < it_issued; ++i)
        mbar_drain_wait(smem_u32(&bar_full[i % STAGES]), (i / STAGES) & 1u);
    }
    if (warp == 1 && lane == 0) {
      mma_commit(smem_u32(&bar_drain));
      mbar_drain_wait(smem_u32(&bar_drain), 0u);
    }
  }
  if (threadIdx.x == 0 && abort_flag) atomicExch(&counters[CNT_STATUS], (unsigned long long)SR_ERR_TIMEOUT);
  if (warp == 1) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(TMEM_COLS_PAIR));
  }
}

using EncodeFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                              const cuuint64_t*, const cuuint32_t*, const cuuint32_t*,
                              CUtensorMapInterleave, CUtensorMapSwizzle, CUtensorMapL2promotion,
                              CUtensorMapFloatOOBfill);

EncodeFn encode_fn() {
  static EncodeFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeFn)p;
  }
  return fn;
}

// Row-major [rows][kd] operand of 4-byte (FP32/TF32) or 2-byte (FP16)
// elements; boxes of 128 rows x 128 bytes.
bool make_map(CUtensorMap* m, const void* ptr, int64_t rows, int64_t kd, int eb) {
  EncodeFn f = encode_fn();
  if (!f) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)kd, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)kd * eb};
  const cuuint32_t box[2] = {(cuuint32_t)(KB / eb), (cuuint32_t)TM};
  const cuuint32_t estr[2] = {1, 1};
  return f(m, eb == 2 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
           const_cast<void*>(ptr), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
           CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

// Tensor maps of the operands: A (hi, lo) and B (hi, lo); bswap: B is A
// with its halves swapped, read by box.
struct TcMaps {
  CUtensorMap hi, lo, bhi, blo;
  int bswap;
};

template <bool F16, bool STAGED, bool MIRROR, bool SW, typename Src>
int launch_tc_t(const TcMaps& m, const Src& src, int nkb, int grid, long long wait_limit,
                cudaStream_t st, int64_t* counters) {
  const size_t tile = SW ? (size_t)TM * TN * 4 : (size_t)TM * EP * 4;
  const size_t smem = (size_t)(STAGED ? STAGES_STAGED : STAGES_DIRECT) * STAGE_BYTES +
                      (STAGED ? tile : 0) + 1024;
  const void* fn = (const void*)k_s_update_tc<F16, STAGED, MIRROR, SW, Src>;
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
      cudaSuccess)
    return 1;
  k_s_update_tc<F16, STAGED, MIRROR, SW, Src><<<grid, TC_THREADS, smem, st>>>(
      m.hi, m.lo, m.bhi, m.blo, src, nkb, m.bswap, wait_limit, (unsigned long long*)counters);
  return 0;
}

// Wide operands (at least 1 KB of K per row) make the pass tensor-bound:
// register epilogue and 3 stages; narrow ones leave it bound by the S stream:
// staged, coalesced epilogue (swizzled, with S fetched early, for upper tiles).
constexpr int64_t WIDE_K_BYTES = TC_WIDE_K_BYTES;

template <bool F16, typename Src>
int launch_tc_f(const TcMaps& m, const Src& src, int nkb, int64_t kd_bytes, int grid,
                long long wait_limit, cudaStream_t st, int mirror, int64_t* counters) {
  if (mirror)
    return launch_tc_t<F16, true, true, false>(m, src, nkb, grid, wait_limit, st, counters);
  if (kd_bytes >= WIDE_K_BYTES)
    return launch_tc_t<F16, false, false, false>(m, src, nkb, grid, wait_limit, st, counters);
  // the swizzled epilogue for one graph's passes; many small graphs measured
  // faster with the padded staging tile
  return launch_tc_t<F16, true, false, std::is_same<Src, TcOneGraph>::value>(m, src, nkb, grid,
                                                                              wait_limit, st,
                                                                              counters);
}

// Bhi / Blo: B on its own, or null (B = A with its halves swapped).
template <typename Src>
int launch_tc(const void* Ahi, const void* Alo, int64_t n_rows, int64_t kd, const Src& src,
              int grid, long long wait_limit, cudaStream_t st, int f16, int mirror,
              int64_t* counters, const void* Bhi = nullptr, const void* Blo = nullptr) {
  const int eb = f16 ? 2 : 4;
  const int kch = KB / eb;
  const bool bswap = Bhi == nullptr;
  if (kd % ((bswap ? 2 : 1) * kch) != 0 || n_rows % TM != 0 || bswap != (Blo == nullptr))
    return 1;
  TcMaps m;
  m.bswap = bswap ? 1 : 0;
  if (!make_map(&m.hi, Ahi, n_rows, kd, eb)) return 2;
  if (!make_map(&m.lo, Alo, n_rows, kd, eb)) return 2;
  if (bswap) {
    m.bhi = m.hi;
    m.blo = m.lo;
  } else {
    if (!make_map(&m.bhi, Bhi, n_rows, kd, eb)) return 2;
    if (!make_map(&m.blo, Blo, n_rows, kd, eb)) return 2;
  }
  const int nkb = (int)(kd / kch);
  if (f16) return launch_tc_f<true>(m, src, nkb, kd * eb, grid, wait_limit, st, mirror, counters);
  return launch_tc_f<false>(m, src, nkb, kd * eb, grid, wait_limit, st, mirror, counters);
}

// A_hi / A_lo: row-major [n_rows][kd], FP32 holding TF32 values (f16 = 0) or
// FP16 (f16 = 1); the B operand is A with its two column halves swapped, read
// from A by box (kd a multiple of 2 * (128 bytes / element size)) or from
// B_hi / B_lo when given (kd a multiple of 128 bytes / element size).
int launch_s_update_tc(float* S, int64_t ld, const void* Ahi, const void* Alo, int64_t n_rows,
                       int64_t kd, const uint32_t* tiles, int nt, const uint64_t* jobs, int nj,
                       const uint64_t* mX, const uint64_t* mE, int use_masks, int n,
                       int64_t* counters, int grid, long long wait_limit, cudaStream_t st,
                       int upper, int f16, const void* Bhi, const void* Blo) {
  const int eb = f16 ? 2 : 4;
  if (jobs && upper && kd * eb >= WIDE_K_BYTES && !Bhi) {
    // wide operands, upper tiles: jobs of two tile pairs sharing their column tile
    const int kch = KB / eb;
    if (kd % (2 * kch) != 0 || n_rows % TM != 0) return 1;
    CUtensorMap mhi, mlo;
    if (!make_map(&mhi, Ahi, n_rows, kd, eb)) return 2;
    if (!make_map(&mlo, Alo, n_rows, kd, eb)) return 2;
    const int nkb = (int)(kd / kch);
    TcJobs src{jobs, nj, mX, mE, use_masks, S, ld, n};
    const size_t smem = (size_t)STAGES_PAIR * PAIR_STAGE_BYTES + 1024;
    const void* fn = f16 ? (const void*)k_s_update_tc_pair<true> : (const void*)k_s_update_tc_pair<false>;
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
      return 1;
    if (f16)
      k_s_update_tc_pair<true><<<grid, TC_THREADS, smem, st>>>(mhi, mlo, src, nkb, wait_limit,
                                                               (unsigned long long*)counters);
    else
      k_s_update_tc_pair<false><<<grid, TC_THREADS, smem, st>>>(mhi, mlo, src, nkb, wait_limit,
                                                                (unsigned long long*)counters);
    return 0;
  }
  TcOneGraph src{tiles, nt, mX, mE, use_masks, S, ld, n, upper ? 0 : 1};
  return launch_tc(Ahi, Alo, n_rows, kd, src, grid, wait_limit, st, f16, upper ? 0 : 1, counters,
                   Bhi, Blo);
}

int launch_s_update_tc_multi(const void* Ahi, const void* Alo, int64_t rows, int64_t kd,
                             const MultiGraphDesc* descs, const uint64_t* tiles, const int* ntiles,
                             int64_t* counters, int grid, long long wait_limit, cudaStream_t st,
                             int f16, int upper) {
  TcManyGraphs src{tiles, ntiles, descs};
  return launch_tc(Ahi, Alo, rows, kd, src, grid, wait_limit, st, f16, upper ? 0 : 1, counters);
}

}  // namespace sr
