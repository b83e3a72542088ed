// FP8 e4m3 GEMM with FP32 scales per 128 x 128 block, FP32 accumulation and
// output, and the block quantiser that produces its operands.  (The paper
// measures BF16 only; this is the precision variant of the same NN GEMM.)
//
//   A ~ qA (M x K e4m3, row-major) with sA[M/128][K/128],
//   B ~ qB (K x N e4m3, row-major) with sB[K/128][N/128],
//   C[i][j] = sum_kb sA[i/128][kb] * sB[kb][j/128] * sum_{k in kb} qA[i][k] qB[k][j].
//
// Kernel (one CTA per SM, persistent over (128 x BN output tile, K split)
// units; BN = 256 or 128; split S = 1, 2, 4 or 8):
//   warp 0     TMA producer: A block 128 x 128 bytes (K-major) and B block 128 K-rows
//              x BN bytes (N-major, 128-byte-wide column boxes), 128-byte swizzle.
//   warp 1     one thread issues tcgen05.mma kind::f8f6f4 (M = 128, N = BN, K = 32) into
//              one of 512 / BN TMEM buffers, a fresh accumulator per 128-deep K block,
//              and commits once per K block to the buffer's full barrier.
//   warps 2-3  idle: they complete warpgroup 0, whose registers go to the promotion warps.
//   warps 4-11 promotion and epilogue (224 registers each), two warps per TMEM lane
//              quarter, each owning one half of the tile's columns: per K block, tcgen05.ld
//              the block product 64 columns per wait, multiply by sA * sB (one scalar per
//              warp and K block) and add into FP32 registers; after the unit's last block,
//              128B-swizzled staging and a TMA store (beta = 0) or reduce-add (beta = 1).
//              With S > 1 the unit's partial goes to the split-K workspace instead, and the
//              last arriving split of a (tile, warp) sums the S partials in the fixed order
//              0..S-1.  Their release of a buffer (and, through warp 4, of the K block's
//              operand stage) is what lets the producer and the MMA thread reuse it.
// The 256 x 256 tile also runs as a tcgen05 cta_group::2 pair (gemm_fp8_2sm_kernel):
// each CTA of a 2-CTA cluster loads its 128 rows of A and 128 columns of B, the even
// CTA issues the M = 256 MMAs, and each CTA promotes and stores its own 128 rows.
// Padding is never materialised: tensor maps carry the logical extents, reads
// past them are zero-filled, stores clipped, and scales outside the logical
// blocks read as 0.  Every mbarrier wait is bounded; on expiry the kernel
// records an error code, lets its in-flight copies land, releases TMEM and returns.
#include <cuda.h>
#include <cuda_fp8.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <climits>
#include <mutex>
#include <cstring>
#include <string>
#include <vector>

#include "ptx.cuh"
#include "rg_internal.h"

namespace rg {

namespace fp8 {

constexpr int kEpiWarps = 8;                  // two promotion warps per TMEM lane quarter
constexpr int kEpiWarp0 = 4;                  // the promotion warps are warpgroups 1 and 2
constexpr int kThreads = 32 * (kEpiWarp0 + kEpiWarps);
// Register split.  Three warps per SM sub-partition launch with 168 registers each;
// warpgroup 0 (producer, MMA issuer and two idle warps) then shrinks to 56 and the
// promotion warpgroups grow to 224 (setmaxnreg), which holds a thread's BN / 2
// accumulators plus 64 columns of a K block's product.  The shares add up to the
// launch's registers, per CTA and per sub-partition (one warp of each warpgroup).
constexpr int kLaunchRegs = 168, kRegsLow = 56, kRegsHigh = 224;
static_assert(4 * kRegsLow + kEpiWarps * kRegsHigh == (kThreads / 32) * kLaunchRegs, "register split");
static_assert(kRegsLow + 2 * kRegsHigh == 3 * kLaunchRegs, "register split per sub-partition");
constexpr int BM = 128, BK = 128;             // BK: one 128-byte swizzle row of e4m3 = one scale block
constexpr int SB = 128;                       // scale block edge
constexpr int STAGING_PER_WARP = 2 * 4096;
constexpr long long kDrainCycles = 1LL << 30;
constexpr uint32_t FULL = 0xffffffffu;

// PAIR: a cta_group::2 pair computes a 256 x BN tile; each CTA loads its 128 rows of A
// and BN / 2 columns of B and holds its 128 output rows x BN columns in its own TMEM.
template <int BN, bool PAIR = false>
struct Cfg {
  static constexpr int CTAS = PAIR ? 2 : 1;
  static constexpr int STAGES = PAIR ? 5 : BN == 256 ? 3 : 4;
  static constexpr int A_BYTES = BM * BK;
  static constexpr int B_BYTES = BK * BN / CTAS;  // (BN / CTAS) / 128 N-major column boxes of BK rows
  static constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
  static constexpr int NACC = 512 / BN;       // TMEM accumulator buffers of BN columns: all 512 columns
  static constexpr int TMEM_COLS = NACC * BN;
  static constexpr int STAGING_OFF = STAGES * STAGE_BYTES;
  static constexpr int BAR_OFF = STAGING_OFF + kEpiWarps * STAGING_PER_WARP;
  static constexpr int SMEM_BYTES = 1024 + BAR_OFF + 256;
  static constexpr int HALF = BN / 2;         // columns per promotion warp
  static constexpr int LDG = 64;              // columns of a K block's product read per TMEM wait
  // E4M3 x E4M3, A K-major, B MN-major; M = 256 across a pair
  static constexpr uint32_t IDESC = instr_desc(0, 0, 0, 1, 128 * CTAS, BN);
  static_assert(SMEM_BYTES <= 232448, "shared memory budget");
  static_assert(BN == 128 || BN == 256, "tile width");
  static_assert(!PAIR || BN == 256, "pair tile");
  static_assert((2 * STAGES + 2 * NACC + 1) * 8 + 8 <= 256, "barrier block");
};

template <uint32_t N>
__device__ __forceinline__ void setmaxnreg_inc() {
  asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(N));
}
template <uint32_t N>
__device__ __forceinline__ void setmaxnreg_dec() {
  asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(N));
}

// Arrive on an mbarrier given by its shared::cluster address with relaxed semantics: the pair's
// "accumulator buffer read" signal publishes no memory (the TMEM reads it covers have completed,
// tcgen05.wait::ld), so it needs none of the membar a release at cluster scope costs on every K block.
__device__ __forceinline__ void mbar_arrive_cluster_relaxed(uint32_t cluster_addr) {
  asm volatile("mbarrier.arrive.relaxed.cluster.shared::cluster.b64 _, [%0];" ::"r"(cluster_addr) : "memory");
}

// D (+)= A * B across a CTA pair (cta_group::2, M = 256 per instruction), e4m3 inputs, F32 accumulator.
__device__ __forceinline__ void mma_f8_pair(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                            uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::2.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

struct Args {
  int32_t M, N;            // logical output extents
  int32_t tiles_m, tiles_n;  // tiles of the (padded) launch
  int32_t kblocks;         // K blocks of the (padded) launch
  int32_t splits;
  int32_t beta;
  int32_t mb_valid, kb_valid, nb_valid;  // logical scale blocks (reads beyond them are 0)
  int32_t sa_ld, sb_ld;    // leading dimensions of the scale arrays (blocks)
  const float* sA;
  const float* sB;
  float* ws;               // split-K partials [split][tile][BM] x BN
  int32_t* tickets;        // [tile][8], zero between launches
  int32_t* err;
  long long timeout;
};

__device__ __forceinline__ void st_shared_v4(uint32_t addr, float a, float b, float c, float d) {
  asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "f"(a), "f"(b), "f"(c), "f"(d) : "memory");
}

// One warp writes a 32 x 32 FP32 block (lane = row) through swizzled staging
// with a TMA store, or a TMA reduce-add when add is set.
__device__ __forceinline__ void put_block(const CUtensorMap* map, const float* v, int row0, int col0, bool add,
                                          uint32_t stg0, int& sbuf, int lane) {
  if (lane == 0) bulk_wait_read<1>();
  __syncwarp();
  const uint32_t buf = stg0 + sbuf * 4096;
#pragma unroll
  for (int j = 0; j < 8; ++j)
    st_shared_v4(buf + lane * 128 + ((j ^ (lane & 7)) << 4), v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
  fence_proxy_async_smem();
  __syncwarp();
  if (lane == 0) {
    if (add)
      tma_reduce_add_2d(map, buf, col0, row0);
    else
      tma_store_2d(map, buf, col0, row0);
    bulk_commit();
  }
  sbuf ^= 1;
}

// The kernel body.  SPLIT = false: the instance for S = 1 (no workspace path, so its
// promotion loop, which holds BN / 2 accumulators per thread, carries no split-K
// state).  PAIR: one CTA of a cta_group::2 pair (launched as 2-CTA clusters): units
// are (256-row pair tile, split); both CTAs load their operand halves, the even
// CTA's lane issues the pair MMAs, and each CTA promotes and stores its own 128
// rows; tiles, tickets and workspace rows count 128-row tiles (tiles_m is even).
template <int BN, bool SPLIT, bool PAIR>
__device__ __forceinline__ void fp8_body(const CUtensorMap& tmA, const CUtensorMap& tmB, const CUtensorMap& tmC,
                                         const CUtensorMap& tmW, const Args& args) {
  using C = Cfg<BN, PAIR>;
  // Coupled ring (as many stages as accumulator buffers, one CTA: the 128x128 tile): K block kb
  // uses stage kb % STAGES and buffer kb % NACC, the same index.  The producer refills a stage
  // only once the promotion warps have released its buffer, which they do after the block's
  // MMAs completed, so a landed stage also means a free buffer: the MMA thread waits on one
  // barrier and commits to one per K block.
  constexpr bool COUPLED = C::NACC == C::STAGES && !PAIR;
  // Otherwise the MMA thread commits only to the accumulator-full barrier, and the first
  // promotion warp of each CTA frees the K block's stage once it has seen that barrier (the
  // block's MMAs, which read the stage, have completed): one commit per K block, not two.
  constexpr bool STAGE_BY_PROMOTION = !COUPLED;
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw_s = smem_u32(smem_raw);
  uint8_t* smem = smem_raw + ((1024u - (raw_s & 1023u)) & 1023u);
  const uint32_t sbase = smem_u32(smem);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + C::BAR_OFF);
  const uint32_t bar0 = smem_u32(bars);
  auto full_bar = [&](int i) { return bar0 + 8u * i; };
  auto empty_bar = [&](int i) { return bar0 + 8u * (C::STAGES + i); };
  auto tfull_bar = [&](int b) { return bar0 + 8u * (2 * C::STAGES + b); };
  auto tempty_bar = [&](int b) { return bar0 + 8u * (2 * C::STAGES + C::NACC + b); };
  const uint32_t drain_bar = bar0 + 8u * (2 * C::STAGES + 2 * C::NACC);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * C::STAGES + 2 * C::NACC + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  int never = 0;
  volatile int* no_abort = &never;

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const int ntiles = args.tiles_m * args.tiles_n;  // 128-row tiles
  const int S = SPLIT ? args.splits : 1;
  const int rank = PAIR ? static_cast<int>(cluster_ctarank()) : 0;
  const int cid = PAIR ? static_cast<int>(blockIdx.x) / 2 : static_cast<int>(blockIdx.x);
  const int ncl = PAIR ? static_cast<int>(gridDim.x) / 2 : static_cast<int>(gridDim.x);
  const int total = (PAIR ? ntiles / 2 : ntiles) * S;
  // unit u = ((pair) tile u / S, split u % S) runs K blocks [s * kblocks / S, (s + 1) * kblocks / S)
  auto kb_lo = [&](int s) { return S == 1 ? 0 : s * args.kblocks / S; };
  // this CTA's 128-row tile of unit u: tile index (tickets, workspace) and coordinates
  auto tile_of = [&](int u, int& tm, int& tn) {
    const int t = u / S;
    if constexpr (PAIR) {
      tm = 2 * (t / args.tiles_n) + rank;
      tn = t % args.tiles_n;
    } else {
      tm = t / args.tiles_n;
      tn = t % args.tiles_n;
    }
    return tm * args.tiles_n + tn;
  };

  if (threadIdx.x == 0) {
    prefetch_tmap(&tmA);
    prefetch_tmap(&tmB);
    prefetch_tmap(&tmC);
    for (int i = 0; i < C::STAGES; ++i) {
      mbar_init(full_bar(i), 1);
      mbar_init(empty_bar(i), 1);
    }
    for (int b = 0; b < C::NACC; ++b) {
      mbar_init(tfull_bar(b), 1);
      mbar_init(tempty_bar(b), PAIR ? 2 * kEpiWarps : kEpiWarps);  // pair: both CTAs' warps, on the even CTA
    }
    mbar_init(drain_bar, 1);
    *abort_flag = 0;
    fence_mbar_init();
  }
  if (warp == 1) {
    if constexpr (PAIR) {  // collective with the partner's warp 1: the same columns in both CTAs
      tmem_alloc_pair(smem_u32(tmem_slot), C::TMEM_COLS);
      tmem_relinquish_pair();
    } else {
      tmem_alloc(smem_u32(tmem_slot), C::TMEM_COLS);
      tmem_relinquish();
    }
  }
  tc_fence_before();
  __syncthreads();
  if constexpr (PAIR) cluster_sync();  // the partner's barriers are initialised
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;
  grid_dependency_wait();
  grid_launch_dependents();
  // Role branches; each warpgroup first resizes its registers (setmaxnreg acts on whole
  // warpgroups, so warps 0-3 take the same instruction before they part).
  if (warp < kEpiWarp0) {
    setmaxnreg_dec<kRegsLow>();
    if (warp == 0) {
      if (lane == 0) {
        int stage = 0, fills = 0;
        uint32_t ph = 0, issued_mask = 0, issued_ph = 0;
        bool ok = true;
        for (int u = cid; ok && u < total; u += ncl) {
          const int s = u % S;
          int tm, tn;
          tile_of(u, tm, tn);
          const int kb1 = s + 1 == S ? args.kblocks : kb_lo(s + 1);
          for (int kb = kb_lo(s); kb < kb1; ++kb) {
            if (fills >= C::STAGES &&
                !mbar_wait(COUPLED ? tempty_bar(stage) : empty_bar(stage), ph ^ 1u, args.timeout, abort_flag)) {
              ok = false;
              break;
            }
            ++fills;
            const uint32_t sa = sbase + stage * C::STAGE_BYTES;
            if constexpr (PAIR) {
              // both CTAs' loads complete on the even CTA's full barrier, which expects both halves
              if (rank == 0) mbar_arrive_expect_tx(full_bar(stage), 2 * C::STAGE_BYTES);
              const uint32_t fb = mapa_shared(full_bar(stage), 0);
              tma_load_2d_pair(sa, &tmA, fb, kb * BK, tm * BM);
              tma_load_2d_pair(sa + C::A_BYTES, &tmB, fb, tn * BN + rank * (BN / 2), kb * BK);
            } else {
              mbar_arrive_expect_tx(full_bar(stage), C::STAGE_BYTES);
              tma_load_2d(sa, &tmA, full_bar(stage), kb * BK, tm * BM);
#pragma unroll
              for (int j = 0; j < BN / 128; ++j)
                tma_load_2d(sa + C::A_BYTES + j * (BK * 128), &tmB, full_bar(stage), tn * BN + j * 128, kb * BK);
            }
            issued_mask |= 1u << stage;
            issued_ph = (issued_ph & ~(1u << stage)) | (ph << stage);
            if (++stage == C::STAGES) {
              stage = 0;
              ph ^= 1u;
            }
          }
        }
        if (!ok) {
          atomicExch(args.err, 1);
          *abort_flag = 1;
        }
        // no TMA write may still be landing when the CTA exits
        if (!PAIR || rank == 0) {
          for (int i = 0; i < C::STAGES; ++i)
            if (issued_mask & (1u << i)) mbar_wait(full_bar(i), (issued_ph >> i) & 1u, kDrainCycles, no_abort);
        } else if (!ok) {
          // the odd CTA's loads complete on its partner's barriers; after an abort it gives
          // them a bounded time to land (normally every one of them was consumed)
          const long long t0 = clock64();
          while (clock64() - t0 < (kDrainCycles >> 6)) {
          }
        }
      }
    } else if (warp == 1) {
      // Lane 0 alone issues the MMAs and commits (no per-K-block warp vote); a pair's
      // odd CTA issues nothing: the even CTA's MMAs read and write both.
      if (lane == 0 && (!PAIR || rank == 0)) {
        int stage = 0, acc = 0;
        uint32_t ph = 0, aph = 0;
        bool ok = true;
        for (int u = cid; ok && u < total; u += ncl) {
          const int s = u % S;
          const int kb1 = s + 1 == S ? args.kblocks : kb_lo(s + 1);
          for (int kb = kb_lo(s); kb < kb1; ++kb) {
            if constexpr (!COUPLED) {
              ok = mbar_wait(tempty_bar(acc), aph ^ 1u, args.timeout, abort_flag);
              if (!ok) break;
            }
            ok = mbar_wait(full_bar(stage), ph, args.timeout, abort_flag);
            if (!ok) break;
            tc_fence_after();
            const uint32_t sa = sbase + stage * C::STAGE_BYTES;
            const uint32_t sb = sa + C::A_BYTES;
            const uint32_t d = tmem_base + static_cast<uint32_t>(acc * BN);
            // K steps differ only in the descriptors' start address field (address >> 4)
            const uint64_t adesc0 = smem_desc_sw128(sa, 16, 1024);
            const uint64_t bdesc0 = smem_desc_sw128(sb, BK * 128, 1024);  // column boxes BK*128 apart
#pragma unroll
            for (int k = 0; k < BK / 32; ++k) {
              const uint64_t ad = adesc0 + static_cast<uint64_t>((k * 32) >> 4);
              const uint64_t bd = bdesc0 + static_cast<uint64_t>((k * (32 * 128)) >> 4);
              if constexpr (PAIR)
                mma_f8_pair(d, ad, bd, C::IDESC, k > 0 ? 1u : 0u);
              else
                mma_f8(d, ad, bd, C::IDESC, k > 0 ? 1u : 0u);
            }
            if constexpr (PAIR) {
              if constexpr (!STAGE_BY_PROMOTION) mma_commit_pair_multicast(empty_bar(stage), 3);
              mma_commit_pair_multicast(tfull_bar(acc), 3);    // both CTAs' rows of the product are ready
            } else {
              if constexpr (!COUPLED && !STAGE_BY_PROMOTION) mma_commit(empty_bar(stage));
              mma_commit(tfull_bar(acc));
            }
            if (++stage == C::STAGES) {
              stage = 0;
              ph ^= 1u;
            }
            if (++acc == C::NACC) {
              acc = 0;
              aph ^= 1u;
            }
          }
        }
        if (!ok) {
          atomicExch(args.err, 2);
          *abort_flag = 1;
          if constexpr (PAIR)
            mma_commit_pair(drain_bar);
          else
            mma_commit(drain_bar);  // completes once every issued MMA has finished
          mbar_wait(drain_bar, 0, kDrainCycles, no_abort);
        }
      }
      __syncwarp();
    }
  } else {
    setmaxnreg_inc<kRegsHigh>();
    // promotion warps 4..11: lane quarter q (the TMEM lanes this warp may read), column half hc
    const int e = warp - kEpiWarp0;
    const int q = warp & 3;
    const int hc = e / 4;
    const uint32_t stg0 = sbase + C::STAGING_OFF + e * STAGING_PER_WARP;
    int acc = 0, sbuf = 0, pstage = 0;  // pstage: the operand stage of the current K block
    uint32_t aph = 0;
    bool ok = true;
    for (int u = cid; ok && u < total; u += ncl) {
      const int s = u % S;
      int tm, tn;
      const int tile = tile_of(u, tm, tn);
      const int kb1 = s + 1 == S ? args.kblocks : kb_lo(s + 1);
      const int nb = (tn * BN + hc * C::HALF) / SB;  // this half's scale block column
      // scale rows and the last K block with real scales (0 outside the logical blocks: padding)
      const int kbv = (tm < args.mb_valid && nb < args.nb_valid) ? args.kb_valid : 0;
      float r[C::HALF];
#pragma unroll
      for (int i = 0; i < C::HALF; ++i) r[i] = 0.f;
      // The K blocks' scale products, 32 at a time, one per lane: lane l holds that of K block
      // kb0 + 32 j + l.  A load per K block would put its global-memory latency on the promotion's
      // critical path whenever the block's product is already waiting in TMEM.
      float sc_lane = 0.f;
      for (int kb = kb_lo(s); kb < kb1; ++kb) {
        const int rel = kb - kb_lo(s);
        if ((rel & 31) == 0) {
          // (scale pointers are recomputed from the kernel parameters: registers are scarce here)
          const int k = kb + lane;
          sc_lane = (k < kb1 && k < kbv) ? args.sA[static_cast<size_t>(tm) * args.sa_ld + k] *
                                               args.sB[static_cast<size_t>(k) * args.sb_ld + nb]
                                         : 0.f;
        }
        const float sc = __shfl_sync(FULL, sc_lane, rel & 31);
        ok = __all_sync(FULL, mbar_wait(tfull_bar(acc), aph, args.timeout, abort_flag));
        if (!ok) break;
        if constexpr (STAGE_BY_PROMOTION) {
          if (e == 0 && lane == 0) mbar_arrive(empty_bar(pstage));  // this CTA's copy of the stage is free
          if (++pstage == C::STAGES) pstage = 0;
        }
        tc_fence_after();
        const uint32_t t = tmem_base + (static_cast<uint32_t>(q * 32) << 16) +
                           static_cast<uint32_t>(acc * BN + hc * C::HALF);
#pragma unroll
        for (int c = 0; c < C::HALF / C::LDG; ++c) {
          uint32_t p[C::LDG / 32][32];
#pragma unroll
          for (int j = 0; j < C::LDG / 32; ++j) tmem_ld_32x32b_x32(t + c * C::LDG + j * 32, p[j]);
          tmem_ld_wait();
#pragma unroll
          for (int j = 0; j < C::LDG / 32; ++j)
#pragma unroll
            for (int i = 0; i < 32; ++i) {
              float& acc_v = r[c * C::LDG + j * 32 + i];
              acc_v = fmaf(sc, __uint_as_float(p[j][i]), acc_v);
            }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) {
          if constexpr (PAIR)
            mbar_arrive_cluster_relaxed(mapa_shared(tempty_bar(acc), 0));  // the even CTA's MMA reuses it
          else
            mbar_arrive(tempty_bar(acc));
        }
        if (++acc == C::NACC) {
          acc = 0;
          aph ^= 1u;
        }
      }
      if (!ok) break;
      const int row0 = tm * BM + q * 32;
      if constexpr (!SPLIT) {
#pragma unroll
        for (int c = 0; c < C::HALF / 32; ++c) {
          const int col0 = tn * BN + hc * C::HALF + c * 32;
          if (row0 < args.M && col0 < args.N) put_block(&tmC, r + c * 32, row0, col0, args.beta != 0, stg0, sbuf, lane);
        }
        continue;
      }
      // One store loop for both cases: C itself (S = 1) or this split's slot of
      // the workspace (S > 1), which the last arriving split then reduces.
      const bool direct = !SPLIT || S == 1;
      const CUtensorMap* dst = direct ? &tmC : &tmW;
      const int drow = direct ? row0 : (s * ntiles + tile) * BM + q * 32;
      const int dcol = direct ? tn * BN + hc * C::HALF : hc * C::HALF;
      const bool dadd = direct && args.beta != 0;
#pragma unroll
      for (int c = 0; c < C::HALF / 32; ++c)
        if (!direct || (row0 < args.M && dcol + c * 32 < args.N))
          put_block(dst, r + c * 32, drow, dcol + c * 32, dadd, stg0, sbuf, lane);
      if (direct) continue;
      if constexpr (SPLIT) {
      // Split-K: wait for this split's stores, fence them against the generic
      // proxy and take the (tile, warp) ticket.
      if (lane == 0) {
        bulk_wait<0>();
        fence_proxy_async_global();
      }
      __syncwarp();
      int last = 0;
      if (lane == 0) {
        int32_t* tk = args.tickets + static_cast<size_t>(tile) * kEpiWarps + e;
        const int old = atom_add_acq_rel_gpu(tk, 1);
        last = (old == S - 1);
        if (last) *tk = 0;
      }
      last = __shfl_sync(FULL, last, 0);
      if (!last) continue;
      // The last arriver sums the S partials of its rows in the fixed order 0..S-1,
      // its own included (it was stored and fenced above), so the accumulators are
      // no longer live; lane l reads row l of the warp's 32 rows.
#pragma unroll 1
      for (int c = 0; c < C::HALF / 32; ++c) {
        float sum[32];
        for (int tb = 0; tb < S; ++tb) {  // sum = ((p_0 + p_1) + p_2) + ...
          const float4* src = reinterpret_cast<const float4*>(
              args.ws + static_cast<size_t>((tb * ntiles + tile) * BM + q * 32 + lane) * BN + hc * C::HALF + c * 32);
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const float4 v4 = __ldcg(src + j);
            if (tb == 0) {
              sum[4 * j] = v4.x;
              sum[4 * j + 1] = v4.y;
              sum[4 * j + 2] = v4.z;
              sum[4 * j + 3] = v4.w;
            } else {
              sum[4 * j] += v4.x;
              sum[4 * j + 1] += v4.y;
              sum[4 * j + 2] += v4.z;
              sum[4 * j + 3] += v4.w;
            }
          }
        }
        const int col0 = tn * BN + hc * C::HALF + c * 32;
        if (row0 < args.M && col0 < args.N) put_block(&tmC, sum, row0, col0, args.beta != 0, stg0, sbuf, lane);
      }
      }
    }
    if (!ok && lane == 0) {
      atomicExch(args.err, 3);
      *abort_flag = 1;
    }
    // the staging buffers must have been read before the CTA exits; the global writes
    // themselves complete with the grid (a dependent grid's griddepcontrol.wait sees them)
    if (lane == 0) bulk_wait_read<0>();
    __syncwarp();
  }
  __syncthreads();
  // no CTA of a pair exits while its partner may still arrive on its barriers or run
  // MMAs on its shared memory and TMEM
  if constexpr (PAIR) cluster_sync();
  if (warp == 1) {
    tc_fence_after();
    if constexpr (PAIR)
      tmem_dealloc_pair(tmem_base, C::TMEM_COLS);
    else
      tmem_dealloc(tmem_base, C::TMEM_COLS);
  }
}

template <int BN, bool SPLIT>
__global__ void __launch_bounds__(kThreads, 1)
    gemm_fp8_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                    const __grid_constant__ CUtensorMap tmC, const __grid_constant__ CUtensorMap tmW,
                    const Args args) {
  fp8_body<BN, SPLIT, false>(tmA, tmB, tmC, tmW, args);
}

// The 256 x 256 tile as a cta_group::2 pair (grid: 2 CTAs per cluster).
template <bool SPLIT>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(kThreads, 1)
    gemm_fp8_2sm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                        const __grid_constant__ CUtensorMap tmC, const __grid_constant__ CUtensorMap tmW,
                        const Args args) {
  fp8_body<256, SPLIT, true>(tmA, tmB, tmC, tmW, args);
}

// One CTA per 128 x 128 block: amax, scale = amax / 448 (1 for an all-zero
// block), codes = e4m3(x / scale) rounded to nearest even with saturation.
__global__ void __launch_bounds__(256) quantize_kernel(const float* __restrict__ X, int64_t rows, int64_t cols,
                                                       int64_t ldx, uint8_t* __restrict__ Q, int64_t ldq,
                                                       float* __restrict__ scales, int64_t s_ld) {
  __shared__ float red[8];
  const int64_t r0 = static_cast<int64_t>(blockIdx.y) * 128, c0 = static_cast<int64_t>(blockIdx.x) * 128;
  const int tid = threadIdx.x;
  float amax = 0.f;
  for (int i = tid; i < 128 * 128; i += 256) {
    const int64_t r = r0 + i / 128, c = c0 + i % 128;
    if (r < rows && c < cols) amax = fmaxf(amax, fabsf(X[r * ldx + c]));
  }
  for (int o = 16; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
  if ((tid & 31) == 0) red[tid >> 5] = amax;
  __syncthreads();
  float m = red[0];
  for (int w = 1; w < 8; ++w) m = fmaxf(m, red[w]);
  const float s = m > 0.f ? __fdiv_rn(m, 448.0f) : 1.0f;
  if (tid == 0) scales[static_cast<int64_t>(blockIdx.y) * s_ld + blockIdx.x] = s;
  for (int i = tid; i < 128 * 128; i += 256) {
    const int64_t r = r0 + i / 128, c = c0 + i % 128;
    if (r < rows && c < cols) {
      const float v = __fdiv_rn(X[r * ldx + c], s);
      Q[r * ldq + c] = static_cast<uint8_t>(__nv_cvt_float_to_fp8(v, __NV_SATFINITE, __NV_E4M3));
    }
  }
}

}  // namespace fp8

int fp8_make_map(CUtensorMap* m, CUtensorMapDataType dt, const void* base, uint64_t inner, uint64_t outer,
                 uint64_t row_bytes, uint32_t box_inner, uint32_t box_outer);
cudaError_t fp8_launch_pdl(const void* fn, dim3 grid, int threads, int smem, cudaStream_t st, void** params);

namespace fp8 {

using KernFn = void (*)(const CUtensorMap, const CUtensorMap, const CUtensorMap, const CUtensorMap, const Args);
struct TileInfo {
  KernFn fn;        // S = 1
  KernFn fn_split;  // S > 1
  int bn, smem;
  bool pair;        // cta_group::2: 256 x bn tiles on 2-CTA clusters
};
// FP8 tiles: 0 = 128 x 256, 1 = 128 x 128, 2 = 256 x 256 as a cta_group::2 pair.
static TileInfo tile_info(int tile) {
  switch (tile) {
    case 0:
      return TileInfo{gemm_fp8_kernel<256, false>, gemm_fp8_kernel<256, true>, 256, Cfg<256>::SMEM_BYTES, false};
    case 1:
      return TileInfo{gemm_fp8_kernel<128, false>, gemm_fp8_kernel<128, true>, 128, Cfg<128>::SMEM_BYTES, false};
    default:
      return TileInfo{gemm_fp8_2sm_kernel<false>, gemm_fp8_2sm_kernel<true>, 256, Cfg<256, true>::SMEM_BYTES, true};
  }
}

// The kernels' shared-memory limit, once per device.
static int kernels_ready() {
  static std::mutex mu;
  static bool done[64] = {false};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(RG_ERR_CUDA, std::string("FP8: cudaGetDevice: ") + cudaGetErrorString(e));
  std::lock_guard<std::mutex> lk(mu);
  if (dev >= 0 && dev < 64 && done[dev]) return RG_OK;
  for (int t = 0; t < RG_FP8_NUM_TILES; ++t) {
    const TileInfo ti = tile_info(t);
    for (KernFn fn : {ti.fn, ti.fn_split}) {
      e = cudaFuncSetAttribute(reinterpret_cast<const void*>(fn), cudaFuncAttributeMaxDynamicSharedMemorySize, ti.smem);
      if (e != cudaSuccess) return fail(RG_ERR_CUDA, "FP8: shared-memory attribute");
      // The register split grows the promotion warps to what warpgroup 0 gives back, so it
      // holds only if every thread launches with exactly kLaunchRegs registers: a kernel built
      // with fewer would wait forever in setmaxnreg.inc, and is never launched.
      cudaFuncAttributes fa{};
      e = cudaFuncGetAttributes(&fa, reinterpret_cast<const void*>(fn));
      if (e != cudaSuccess) return fail(RG_ERR_CUDA, "FP8: kernel attributes");
      if (fa.numRegs != kLaunchRegs)
        return fail(RG_ERR_CUDA, "FP8: kernel built with " + std::to_string(fa.numRegs) +
                                     " registers per thread; its register split needs " +
                                     std::to_string(kLaunchRegs));
    }
  }
  if (dev >= 0 && dev < 64) done[dev] = true;
  return RG_OK;
}

struct Launch {
  KernFn fn = nullptr;
  CUtensorMap a, b, c, w;
  Args args{};
  dim3 grid;
  int smem = 0;
  bool noop = false, zero_only = false;
  float* C = nullptr;
  int64_t M = 0, N = 0, ldc = 0;
};

// Checks one FP8 GEMM launch and builds its tensor maps and arguments.
static int prepare(const Fp8CtxInfo& info, int64_t M, int64_t N, int64_t K, const uint8_t* qA, int64_t lda,
                   const float* sA, int64_t lds_a, const uint8_t* qB, int64_t ldb, const float* sB, int64_t lds_b,
                   float* C, int64_t ldc, int32_t variant, int32_t beta, int64_t pm, int64_t pn, int64_t pk,
                   Launch* L) {
  if (!variant_fp8(variant)) return fail(RG_ERR_INVALID, "FP8 GEMM: not an FP8 variant id");
  if (M < 0 || N < 0 || K < 0) return fail(RG_ERR_INVALID, "FP8 GEMM: negative size");
  if (beta != 0 && beta != 1) return fail(RG_ERR_INVALID, "FP8 GEMM: beta must be 0 or 1");
  if (pm == 0) pm = M;
  if (pn == 0) pn = N;
  if (pk == 0) pk = K;
  if (pm < M || pn < N || pk < K) return fail(RG_ERR_INVALID, "FP8 GEMM: padded extents smaller than the problem");
  if (pm > (1 << 30) || pn > (1 << 30) || pk > (1 << 30)) return fail(RG_ERR_SHAPE, "FP8 GEMM: size beyond 2^30");
  *L = Launch{};
  if (M == 0 || N == 0) {
    L->noop = true;
    return RG_OK;
  }
  if (!C) return fail(RG_ERR_INVALID, "FP8 GEMM: null C");
  if (ldc < N) return fail(RG_ERR_INVALID, "FP8 GEMM: ldc < N");
  if ((reinterpret_cast<uintptr_t>(C) & 15) || (ldc % 4)) return fail(RG_ERR_ALIGN, "FP8 GEMM: C 16-byte aligned, ldc % 4");
  if (K == 0) {
    L->zero_only = beta == 0;
    L->noop = beta != 0;
    L->C = C;
    L->M = M;
    L->N = N;
    L->ldc = ldc;
    return RG_OK;
  }
  if (!qA || !qB || !sA || !sB) return fail(RG_ERR_INVALID, "FP8 GEMM: null operand");
  const int64_t kb_valid = (K + BK - 1) / BK, nb_valid = (N + SB - 1) / SB, mb_valid = (M + SB - 1) / SB;
  if (lda < K || ldb < N || lds_a < kb_valid || lds_b < nb_valid)
    return fail(RG_ERR_INVALID, "FP8 GEMM: leading dimensions");
  if ((reinterpret_cast<uintptr_t>(qA) & 15) || (reinterpret_cast<uintptr_t>(qB) & 15) || (lda % 16) || (ldb % 16))
    return fail(RG_ERR_ALIGN, "FP8 GEMM: 16-byte aligned operands, lda and ldb multiples of 16");
  const int tile = (variant - RG_FP8_VARIANT_BASE) / RG_NUM_SPLITS;
  const int splits = 1 << ((variant - RG_FP8_VARIANT_BASE) % RG_NUM_SPLITS);
  const TileInfo ti = tile_info(tile);
  int64_t tiles_m = (pm + BM - 1) / BM;
  if (ti.pair) tiles_m += tiles_m & 1;  // whole 256-row pair tiles (an odd CTA past M loads zeros, stores nothing)
  const int64_t tiles_n = (pn + ti.bn - 1) / ti.bn, kblocks = (pk + BK - 1) / BK;
  const int64_t ntiles = tiles_m * tiles_n;
  if (splits > 1 && (splits * ntiles * BM * ti.bn * 4 > info.ws_bytes || ntiles * kEpiWarps > info.max_tickets))
    return fail(RG_ERR_SHAPE, "FP8 GEMM: split-K workspace too small for this shape");
  if (ntiles * splits > (1LL << 30)) return fail(RG_ERR_SHAPE, "FP8 GEMM: too many work units");
  int rc = fp8_make_map(&L->a, CU_TENSOR_MAP_DATA_TYPE_UINT8, qA, K, M, lda, BK, BM);
  if (rc == RG_OK) rc = fp8_make_map(&L->b, CU_TENSOR_MAP_DATA_TYPE_UINT8, qB, N, K, ldb, 128, BK);
  if (rc == RG_OK) rc = fp8_make_map(&L->c, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, C, N, M, ldc * 4, 32, 32);
  if (rc == RG_OK) {
    if (splits > 1)
      rc = fp8_make_map(&L->w, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, info.ws, ti.bn,
                        static_cast<uint64_t>(splits * ntiles * BM), static_cast<uint64_t>(ti.bn) * 4, 32, 32);
    else
      L->w = L->c;  // unused without split-K
  }
  if (rc != RG_OK) return rc;
  Args& g = L->args;
  g.M = static_cast<int32_t>(M);
  g.N = static_cast<int32_t>(N);
  g.tiles_m = static_cast<int32_t>(tiles_m);
  g.tiles_n = static_cast<int32_t>(tiles_n);
  g.kblocks = static_cast<int32_t>(kblocks);
  g.splits = splits;
  g.beta = beta;
  g.mb_valid = static_cast<int32_t>(mb_valid);
  g.kb_valid = static_cast<int32_t>(kb_valid);
  g.nb_valid = static_cast<int32_t>(nb_valid);
  g.sa_ld = static_cast<int32_t>(lds_a);
  g.sb_ld = static_cast<int32_t>(lds_b);
  g.sA = sA;
  g.sB = sB;
  g.ws = info.ws;
  g.tickets = info.tickets;
  g.err = info.err;
  g.timeout = info.timeout;
  L->fn = splits > 1 ? ti.fn_split : ti.fn;
  L->smem = ti.smem;
  L->grid = ti.pair ? dim3(static_cast<unsigned>(2 * std::min<int64_t>(ntiles / 2 * splits, info.sms / 2)))
                    : dim3(static_cast<unsigned>(std::min<int64_t>(ntiles * splits, info.sms)));
  return RG_OK;
}

static cudaError_t launch(const Launch& L, cudaStream_t st) {
  if (L.noop) return cudaSuccess;
  if (L.zero_only) return cudaMemset2DAsync(L.C, L.ldc * 4, 0, L.N * 4, L.M, st);
  void* params[5] = {const_cast<CUtensorMap*>(&L.a), const_cast<CUtensorMap*>(&L.b), const_cast<CUtensorMap*>(&L.c),
                     const_cast<CUtensorMap*>(&L.w), const_cast<Args*>(&L.args)};
  return fp8_launch_pdl(reinterpret_cast<const void*>(L.fn), L.grid, kThreads, L.smem, st, params);
}

// The leaves of an FP8 plan's cell covering (M, N, K), clipped to the problem, on sub-views.
static int plan_launches(const Fp8CtxInfo& info, const rg_plan* plan, int64_t M, int64_t N, int64_t K,
                         const uint8_t* qA, int64_t lda, const float* sA, int64_t lds_a, const uint8_t* qB,
                         int64_t ldb, const float* sB, int64_t lds_b, float* C, int64_t ldc, std::vector<Launch>& out) {
  out.clear();
  if (!plan) return fail(RG_ERR_INVALID, "FP8 plan: null plan");
  if (M <= 0 || N <= 0 || K <= 0) return fail(RG_ERR_INVALID, "FP8 plan: sizes must be positive");
  const Plan& P = plan->p;
  if (P.variant_ids.empty() || !variant_fp8(P.variant_ids[0]))
    return fail(RG_ERR_INVALID, "FP8 plan: a BF16 plan runs through rg_gemm_plan");
  int64_t cell = 0;
  if (plan_cell(P, M, N, K, &cell) != RG_OK) return fail(RG_ERR_SHAPE, "FP8 plan: shape beyond the plan grid");
  for (int64_t i = P.leaf_off[cell]; i < P.leaf_off[cell + 1]; ++i) {
    const rg_leaf& lf = P.leaves[i];
    if (lf.m0 >= M || lf.n0 >= N || lf.k0 >= K) continue;  // wholly in the padding
    if ((lf.m0 % SB) || (lf.n0 % SB) || (lf.k0 % SB))
      return fail(RG_ERR_SHAPE, "FP8 plan: a leaf's offsets are not multiples of the 128-element scale block");
    const int64_t m = std::min(lf.m, M - lf.m0), n = std::min(lf.n, N - lf.n0), k = std::min(lf.k, K - lf.k0);
    Launch L;
    const int rc = prepare(info, m, n, k, qA + lf.m0 * lda + lf.k0, lda, sA + (lf.m0 / SB) * lds_a + lf.k0 / SB,
                           lds_a, qB + lf.k0 * ldb + lf.n0, ldb, sB + (lf.k0 / SB) * lds_b + lf.n0 / SB, lds_b,
                           C + lf.m0 * ldc + lf.n0, ldc, lf.variant, lf.beta, lf.pm, lf.pn, lf.pk, &L);
    if (rc != RG_OK) return rc;
    out.push_back(L);
  }
  return RG_OK;
}

}  // namespace fp8

}  // namespace rg

extern "C" int rg_fp8_quantize(rg_ctx* ctx, const float* X, int64_t rows, int64_t cols, int64_t ldx, uint8_t* Q,
                               int64_t ldq, float* scales, void* stream) {
  rg::clear_error();
  if (!ctx) return rg::fail(RG_ERR_INVALID, "rg_fp8_quantize: null context");
  if (rows < 0 || cols < 0 || ldx < cols || ldq < cols) return rg::fail(RG_ERR_INVALID, "rg_fp8_quantize: sizes");
  if (rows == 0 || cols == 0) return RG_OK;
  if (!X || !Q || !scales) return rg::fail(RG_ERR_INVALID, "rg_fp8_quantize: null pointer");
  const int64_t br = (rows + 127) / 128, bc = (cols + 127) / 128;
  if (br > 65535 || bc > (1LL << 31) - 1) return rg::fail(RG_ERR_SHAPE, "rg_fp8_quantize: too many blocks");
  rg::fp8::quantize_kernel<<<dim3(static_cast<unsigned>(bc), static_cast<unsigned>(br)), 256, 0,
                             static_cast<cudaStream_t>(stream)>>>(X, rows, cols, ldx, Q, ldq, scales, bc);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? RG_OK : rg::fail(RG_ERR_CUDA, std::string("rg_fp8_quantize: ") + cudaGetErrorString(e));
}

extern "C" int rg_gemm_fp8_ex(rg_ctx* ctx, int64_t M, int64_t N, int64_t K, const uint8_t* qA, int64_t lda,
                              const float* sA, int64_t lds_a, const uint8_t* qB, int64_t ldb, const float* sB,
                              int64_t lds_b, float* C, int64_t ldc, int32_t variant, int32_t beta, int64_t pm,
                              int64_t pn, int64_t pk, void* stream) {
  rg::clear_error();
  rg::Fp8CtxInfo info{};
  int rc = rg::ctx_fp8_info(ctx, &info);
  if (rc != RG_OK) return rc;
  rg::fp8::Launch L;
  rc = rg::fp8::prepare(info, M, N, K, qA, lda, sA, lds_a, qB, ldb, sB, lds_b, C, ldc, variant, beta, pm, pn, pk, &L);
  if (rc != RG_OK) return rc;
  if (!L.noop && !L.zero_only && (rc = rg::fp8::kernels_ready()) != RG_OK) return rc;
  const cudaError_t e = rg::fp8::launch(L, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return rg::fail(RG_ERR_CUDA, std::string("rg_gemm_fp8: launch: ") + cudaGetErrorString(e));
  if (!L.noop && !L.zero_only) rg::ctx_count_launches(ctx, 1);
  return RG_OK;
}

extern "C" int rg_gemm_fp8(rg_ctx* ctx, int64_t M, int64_t N, int64_t K, const uint8_t* qA, int64_t lda,
                           const float* sA, const uint8_t* qB, int64_t ldb, const float* sB, float* C, int64_t ldc,
                           void* stream) {
  return rg_gemm_fp8_ex(ctx, M, N, K, qA, lda, sA, K > 0 ? (K + 127) / 128 : 1, qB, ldb, sB,
                        N > 0 ? (N + 127) / 128 : 1, C, ldc, RG_FP8_VARIANT(0, 0), 0, 0, 0, 0, stream);
}

extern "C" int rg_gemm_fp8_plan(rg_ctx* ctx, const rg_plan* plan, int64_t M, int64_t N, int64_t K, const uint8_t* qA,
                                int64_t lda, const float* sA, int64_t lds_a, const uint8_t* qB, int64_t ldb,
                                const float* sB, int64_t lds_b, float* C, int64_t ldc, void* stream) {
  rg::clear_error();
  rg::Fp8CtxInfo info{};
  int rc = rg::ctx_fp8_info(ctx, &info);
  if (rc != RG_OK) return rc;
  std::vector<rg::fp8::Launch> ls;
  rc = rg::fp8::plan_launches(info, plan, M, N, K, qA, lda, sA, lds_a, qB, ldb, sB, lds_b, C, ldc, ls);
  if (rc != RG_OK) return rc;
  if ((rc = rg::fp8::kernels_ready()) != RG_OK) return rc;
  for (const auto& L : ls) {
    const cudaError_t e = rg::fp8::launch(L, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return rg::fail(RG_ERR_CUDA, std::string("rg_gemm_fp8_plan: launch: ") + cudaGetErrorString(e));
    if (!L.noop && !L.zero_only) rg::ctx_count_launches(ctx, 1);
  }
  return RG_OK;
}

namespace {
uint64_t splitmix_next_fp8(uint64_t& s) {
  uint64_t z = (s += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
}  // namespace

extern "C" int rg_sweep_fp8(rg_ctx* ctx, const rg_grid* grid, int32_t n_variants, const int32_t* variant_ids,
                            const rg_plan* plan, const uint8_t* qA, const float* sA, const uint8_t* qB,
                            const float* sB, float* C, const rg_sweep_opts* opts, int64_t* t_ns_out,
                            double* tflops_out, double* stats_out, void* stream) {
  rg::clear_error();
  using namespace rg::fp8;
  if (!ctx || !grid || !qA || !sA || !qB || !sB || !C || !t_ns_out)
    return rg::fail(RG_ERR_INVALID, "rg_sweep_fp8: null argument");
  if (!rg::grid_valid(*grid)) return rg::fail(RG_ERR_INVALID, "rg_sweep_fp8: invalid grid");
  if (plan ? n_variants != 1 : (n_variants <= 0 || !variant_ids))
    return rg::fail(RG_ERR_INVALID, "rg_sweep_fp8: variants");
  if (!plan)
    for (int32_t i = 0; i < n_variants; ++i)
      if (!rg::variant_fp8(variant_ids[i])) return rg::fail(RG_ERR_INVALID, "rg_sweep_fp8: not an FP8 variant id");
  rg_sweep_opts o;
  rg_sweep_opts_default(&o);
  if (opts) o = *opts;
  if (o.reps <= 0 || o.warmup < 0 || o.global_warmup < 0 || o.spin_ns < 0)
    return rg::fail(RG_ERR_INVALID, "rg_sweep_fp8: options");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int64_t cells = rg::cells_of(*grid);
  const int64_t nk = grid->k.count, nn = grid->n.count;
  rg::Fp8CtxInfo info{};
  int rc = rg::ctx_fp8_info(ctx, &info);
  if (rc != RG_OK) return rc;
  if ((rc = kernels_ready()) != RG_OK) return rc;
  std::vector<int64_t> order(static_cast<size_t>(cells) * n_variants);
  for (size_t i = 0; i < order.size(); ++i) order[i] = static_cast<int64_t>(i);
  if (o.shuffle) {
    uint64_t s = o.seed;
    for (size_t i = order.size() - 1; i > 0; --i) std::swap(order[i], order[splitmix_next_fp8(s) % (i + 1)]);
  }
  auto dims = [&](int64_t item, int64_t* M, int64_t* N, int64_t* K) {
    const int64_t cell = item % cells;
    *M = rg::axis_value(grid->m, cell / (nn * nk));
    *N = rg::axis_value(grid->n, (cell / nk) % nn);
    *K = rg::axis_value(grid->k, cell % nk);
  };
  // a split is worth timing only where the unsplit tiles leave SMs idle (counting both CTAs of
  // a pair tile), a pair tile only beyond 128 rows
  if (o.prune_splits && !plan) {
    std::vector<int64_t> keep;
    keep.reserve(order.size());
    for (int64_t it : order) {
      const int32_t v = variant_ids[it / cells];
      const int S = 1 << ((v - RG_FP8_VARIANT_BASE) % RG_NUM_SPLITS);
      const TileInfo ti = tile_info((v - RG_FP8_VARIANT_BASE) / RG_NUM_SPLITS);
      int64_t M, N, K;
      dims(it, &M, &N, &K);
      bool pruned = ti.pair && M <= 128;
      if (S > 1 && !pruned) {
        const int64_t rows = ti.pair ? 2 * ((M + 2 * BM - 1) / (2 * BM)) : (M + BM - 1) / BM;
        const int64_t ctas = rows * ((N + ti.bn - 1) / ti.bn);
        pruned = ctas >= info.sms || (K + BK - 1) / BK < 2 * S;
      }
      if (pruned)
        t_ns_out[it] = RG_T_UNMEASURED;
      else
        keep.push_back(it);
    }
    order.swap(keep);
  }
  std::vector<Launch> ls;
  auto prep = [&](int64_t item, int* launches) -> int {
    int64_t M, N, K;
    dims(item, &M, &N, &K);
    if ((K % 16) || (N % 16)) return rg::fail(RG_ERR_ALIGN, "rg_sweep_fp8: grid sizes must be multiples of 16");
    const int64_t lds_a = (K + 127) / 128, lds_b = (N + 127) / 128;
    int r;
    if (plan) {
      r = plan_launches(info, plan, M, N, K, qA, K, sA, lds_a, qB, N, sB, lds_b, C, N, ls);
    } else {
      ls.resize(1);
      r = prepare(info, M, N, K, qA, K, sA, lds_a, qB, N, sB, lds_b, C, N, variant_ids[item / cells], 0, 0, 0, 0,
                  &ls[0]);
    }
    *launches = static_cast<int>(ls.size());
    return r;
  };
  int64_t n_launch = 0;
  auto run = [&]() -> cudaError_t {
    for (const auto& L : ls) {
      const cudaError_t e = launch(L, st);
      if (e != cudaSuccess) return e;
      ++n_launch;
    }
    return cudaSuccess;
  };
  rc = rg::timed_sweep(ctx, order, o, st, t_ns_out, prep, run);
  rg::ctx_count_launches(ctx, n_launch);
  if (rc != RG_OK) return rc;
  rc = rg_check(ctx, stream);
  if (rc != RG_OK) return rc;
  return rg::sweep_surfaces(grid, plan ? 1 : n_variants, t_ns_out, tflops_out, stats_out);
}

// ------------------------------------------------------------------ FP8 requests of the serving engine
namespace rg {

int fp8_request_status(const Fp8Request& r) {
  if (r.M <= 0 || r.N <= 0 || r.K <= 0 || !r.qA || !r.qB || !r.sA || !r.sB) return RG_ERR_INVALID;
  if (r.lda < r.K || r.ldb < r.N || (r.C && r.ldc < r.N) || r.lds_a < (r.K + 127) / 128 || r.lds_b < (r.N + 127) / 128)
    return RG_ERR_INVALID;
  if ((reinterpret_cast<uintptr_t>(r.qA) & 15) || (reinterpret_cast<uintptr_t>(r.qB) & 15) || (r.lda % 16) ||
      (r.ldb % 16))
    return RG_ERR_ALIGN;
  if (r.C && ((reinterpret_cast<uintptr_t>(r.C) & 15) || (r.ldc % 4))) return RG_ERR_ALIGN;
  if (r.M > (1 << 30) || r.N > (1 << 30) || r.K > (1 << 30)) return RG_ERR_SHAPE;
  return RG_OK;
}

int fp8_enqueue_phase(rg_ctx* ctx, const rg_plan* plan, const Fp8Request& r, int32_t phase, float* ws,
                      int64_t ws_bytes, int32_t* tickets, int64_t max_tickets, void* stream, int32_t* max_phase) {
  Fp8CtxInfo info{};
  int rc = ctx_fp8_info(ctx, &info);
  if (rc != RG_OK) return rc;
  info.ws = ws;
  info.ws_bytes = ws_bytes;
  info.tickets = tickets;
  info.max_tickets = max_tickets;
  if ((rc = fp8::kernels_ready()) != RG_OK) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  *max_phase = 0;
  if (!plan) {
    if (phase != 0) return RG_OK;
    fp8::Launch L;
    rc = fp8::prepare(info, r.M, r.N, r.K, r.qA, r.lda, r.sA, r.lds_a, r.qB, r.ldb, r.sB, r.lds_b, r.C, r.ldc,
                      RG_FP8_VARIANT(0, 0), 0, 0, 0, 0, &L);
    if (rc != RG_OK) return rc;
    const cudaError_t e = fp8::launch(L, st);
    if (e != cudaSuccess) return fail(RG_ERR_CUDA, std::string("FP8 serving: launch: ") + cudaGetErrorString(e));
    ctx_count_launches(ctx, 1);
    return RG_OK;
  }
  const Plan& P = plan->p;
  if (P.variant_ids.empty() || !variant_fp8(P.variant_ids[0]))
    return fail(RG_ERR_INVALID, "FP8 serving: the FP8 plan holds BF16 variants");
  int64_t cell = 0;
  if (plan_cell(P, r.M, r.N, r.K, &cell) != RG_OK) return fail(RG_ERR_SHAPE, "FP8 serving: shape beyond the plan grid");
  for (int64_t i = P.leaf_off[cell]; i < P.leaf_off[cell + 1]; ++i) {
    const rg_leaf& lf = P.leaves[i];
    *max_phase = std::max(*max_phase, lf.phase);
    if (lf.phase != phase || lf.m0 >= r.M || lf.n0 >= r.N || lf.k0 >= r.K) continue;
    if ((lf.m0 % fp8::SB) || (lf.n0 % fp8::SB) || (lf.k0 % fp8::SB))
      return fail(RG_ERR_SHAPE, "FP8 serving: a leaf's offsets are not multiples of the scale block");
    const int64_t m = std::min(lf.m, r.M - lf.m0), n = std::min(lf.n, r.N - lf.n0), k = std::min(lf.k, r.K - lf.k0);
    fp8::Launch L;
    rc = fp8::prepare(info, m, n, k, r.qA + lf.m0 * r.lda + lf.k0, r.lda, r.sA + (lf.m0 / fp8::SB) * r.lds_a + lf.k0 / fp8::SB,
                      r.lds_a, r.qB + lf.k0 * r.ldb + lf.n0, r.ldb, r.sB + (lf.k0 / fp8::SB) * r.lds_b + lf.n0 / fp8::SB,
                      r.lds_b, r.C + lf.m0 * r.ldc + lf.n0, r.ldc, lf.variant, lf.beta, lf.pm, lf.pn, lf.pk, &L);
    if (rc != RG_OK) return rc;
    const cudaError_t e = fp8::launch(L, st);
    if (e != cudaSuccess) return fail(RG_ERR_CUDA, std::string("FP8 serving: launch: ") + cudaGetErrorString(e));
    if (!L.noop && !L.zero_only) ctx_count_launches(ctx, 1);
  }
  return RG_OK;
}

}  // namespace rg
