// FP8 e4m3 GEMM with FP32 scales per 128 x 128 block, FP32 accumulation and
// output, and the block quantiser that produces its operands.  (The paper
// measures BF16 only; this is the precision variant of the same NN GEMM.)
//
//   A ~ qA (M x K e4m3, row-major) with sA[M/128][K/128],
//   B ~ qB (K x N e4m3, row-major) with sB[K/128][N/128],
//   C[i][j] = sum_kb sA[i/128][kb] * sB[kb][j/128] * sum_{k in kb} qA[i][k] qB[k][j].
//
// Kernel (one CTA per SM, persistent over 128 x 256 output tiles):
//   warp 0     TMA producer: A block 128 x 128 bytes (K-major) and B block 128 K-rows
//              x 256 bytes (N-major, two 128-byte-wide halves), 128-byte swizzle.
//   warp 1     one thread issues tcgen05.mma kind::f8f6f4 (M = 128, N = 256, K = 32) into
//              one of two TMEM buffers, a fresh accumulator per 128-deep K block.
//   warps 2-9  promotion and epilogue, two warps per TMEM lane quarter, each owning one
//              128-column half (= one scale block column): per K block, tcgen05.ld the
//              block product, multiply by sA * sB (one scalar per warp and K block) and
//              add into FP32 registers (half a row per thread); after the last block,
//              128B-swizzled staging and TMA store.
// Every mbarrier wait is bounded; on expiry the kernel records an error code,
// lets its in-flight copies land, releases TMEM and returns.
#include <cuda.h>
#include <cuda_fp8.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <string>

#include "ptx.cuh"
#include "rg_internal.h"

namespace rg {

namespace fp8 {

constexpr int kEpiWarps = 8;                  // two promotion warps per TMEM lane quarter
constexpr int kThreads = 32 * (2 + kEpiWarps);
constexpr int BM = 128, BN = 256, BK = 128;  // BK: one 128-byte swizzle row of e4m3 = one scale block
constexpr int SB = 128;                      // scale block edge
constexpr int STAGES = 3;
constexpr int A_BYTES = BM * BK;
constexpr int B_BYTES = BK * BN;             // two 128-column N-major halves of BK rows
constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
constexpr int NACC = 2;                       // TMEM buffers of BN columns
constexpr int TMEM_COLS = 512;
constexpr int STAGING_PER_WARP = 2 * 4096;
constexpr int STAGING_OFF = STAGES * STAGE_BYTES;
constexpr int BAR_OFF = STAGING_OFF + kEpiWarps * STAGING_PER_WARP;
constexpr int SMEM_BYTES = 1024 + BAR_OFF + 256;
constexpr uint32_t IDESC = instr_desc(0, 0, 0, 1, 128, BN);  // E4M3 x E4M3, A K-major, B MN-major
constexpr long long kDrainCycles = 1LL << 30;
constexpr uint32_t FULL = 0xffffffffu;
static_assert(SMEM_BYTES <= 232448, "shared memory budget");

struct Args {
  int32_t M, N;
  int32_t tiles_m, tiles_n;
  int32_t kblocks;
  int32_t sa_ld, sb_ld;  // leading dimensions of the scale arrays (blocks)
  const float* sA;
  const float* sB;
  int32_t* err;
  long long timeout;
};

__device__ __forceinline__ void st_shared_v4(uint32_t addr, float a, float b, float c, float d) {
  asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "f"(a), "f"(b), "f"(c), "f"(d) : "memory");
}

__global__ void __launch_bounds__(kThreads, 1)
    gemm_fp8_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                    const __grid_constant__ CUtensorMap tmC, const Args args) {
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw_s = smem_u32(smem_raw);
  uint8_t* smem = smem_raw + ((1024u - (raw_s & 1023u)) & 1023u);
  const uint32_t sbase = smem_u32(smem);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + BAR_OFF);
  const uint32_t bar0 = smem_u32(bars);
  auto full_bar = [&](int i) { return bar0 + 8u * i; };
  auto empty_bar = [&](int i) { return bar0 + 8u * (STAGES + i); };
  auto tfull_bar = [&](int b) { return bar0 + 8u * (2 * STAGES + b); };
  auto tempty_bar = [&](int b) { return bar0 + 8u * (2 * STAGES + NACC + b); };
  const uint32_t drain_bar = bar0 + 8u * (2 * STAGES + 2 * NACC);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * STAGES + 2 * NACC + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  int never = 0;
  volatile int* no_abort = &never;

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const int total = args.tiles_m * args.tiles_n;

  if (threadIdx.x == 0) {
    prefetch_tmap(&tmA);
    prefetch_tmap(&tmB);
    prefetch_tmap(&tmC);
    for (int i = 0; i < STAGES; ++i) {
      mbar_init(full_bar(i), 1);
      mbar_init(empty_bar(i), 1);
    }
    for (int b = 0; b < NACC; ++b) {
      mbar_init(tfull_bar(b), 1);
      mbar_init(tempty_bar(b), kEpiWarps);
    }
    mbar_init(drain_bar, 1);
    *abort_flag = 0;
    fence_mbar_init();
  }
  if (warp == 1) {
    tmem_alloc(smem_u32(tmem_slot), TMEM_COLS);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;
  grid_dependency_wait();
  grid_launch_dependents();

  if (warp == 0) {
    if (lane == 0) {
      int stage = 0;
      uint32_t ph = 0, issued_mask = 0, issued_ph = 0;
      bool ok = true;
      for (int u = blockIdx.x; ok && u < total; u += gridDim.x) {
        const int tm = u / args.tiles_n, tn = u % args.tiles_n;
        for (int kb = 0; kb < args.kblocks; ++kb) {
          if (!mbar_wait(empty_bar(stage), ph ^ 1u, args.timeout, abort_flag)) {
            ok = false;
            break;
          }
          const uint32_t sa = sbase + stage * STAGE_BYTES;
          mbar_arrive_expect_tx(full_bar(stage), STAGE_BYTES);
          tma_load_2d(sa, &tmA, full_bar(stage), kb * BK, tm * BM);
#pragma unroll
          for (int j = 0; j < BN / 128; ++j)
            tma_load_2d(sa + A_BYTES + j * (BK * 128), &tmB, full_bar(stage), tn * BN + j * 128, kb * BK);
          issued_mask |= 1u << stage;
          issued_ph = (issued_ph & ~(1u << stage)) | (ph << stage);
          if (++stage == STAGES) {
            stage = 0;
            ph ^= 1u;
          }
        }
      }
      if (!ok) {
        atomicExch(args.err, 1);
        *abort_flag = 1;
      }
      for (int i = 0; i < STAGES; ++i)
        if (issued_mask & (1u << i)) mbar_wait(full_bar(i), (issued_ph >> i) & 1u, kDrainCycles, no_abort);
    }
  } else if (warp == 1) {
    // Lane 0 alone issues the MMAs and commits (no per-K-block warp vote).
    if (lane == 0) {
      int stage = 0, acc = 0;
      uint32_t ph = 0, aph = 0;
      bool ok = true;
      for (int u = blockIdx.x; ok && u < total; u += gridDim.x) {
        for (int kb = 0; kb < args.kblocks; ++kb) {
          ok = mbar_wait(tempty_bar(acc), aph ^ 1u, args.timeout, abort_flag);
          if (!ok) break;
          ok = mbar_wait(full_bar(stage), ph, args.timeout, abort_flag);
          if (!ok) break;
          tc_fence_after();
          const uint32_t sa = sbase + stage * STAGE_BYTES;
          const uint32_t sb = sa + A_BYTES;
          const uint32_t d = tmem_base + static_cast<uint32_t>(acc * BN);
          // K steps differ only in the descriptors' start address field (address >> 4)
          const uint64_t adesc0 = smem_desc_sw128(sa, 16, 1024);
          const uint64_t bdesc0 = smem_desc_sw128(sb, BK * 128, 1024);  // halves BK*128 apart
#pragma unroll
          for (int k = 0; k < BK / 32; ++k)
            mma_f8(d, adesc0 + static_cast<uint64_t>((k * 32) >> 4), bdesc0 + static_cast<uint64_t>((k * (32 * 128)) >> 4),
                   IDESC, k > 0 ? 1u : 0u);
          mma_commit(empty_bar(stage));
          mma_commit(tfull_bar(acc));
          if (++stage == STAGES) {
            stage = 0;
            ph ^= 1u;
          }
          if (++acc == NACC) {
            acc = 0;
            aph ^= 1u;
          }
        }
      }
      if (!ok) {
        atomicExch(args.err, 2);
        *abort_flag = 1;
        mma_commit(drain_bar);
        mbar_wait(drain_bar, 0, kDrainCycles, no_abort);
      }
    }
    __syncwarp();
  } else {
    // promotion warps 2..9: lane quarter q (the TMEM lanes this warp may read), column half hc
    const int e = warp - 2;
    const int q = warp & 3;
    const int hc = e / 4;
    const uint32_t stg0 = sbase + STAGING_OFF + e * STAGING_PER_WARP;
    int acc = 0, sbuf = 0;
    uint32_t aph = 0;
    bool ok = true;
    for (int u = blockIdx.x; ok && u < total; u += gridDim.x) {
      const int tm = u / args.tiles_n, tn = u % args.tiles_n;
      const int nb = tn * (BN / SB) + hc;  // this half's scale block column
      float r[BN / 2];
#pragma unroll
      for (int i = 0; i < BN / 2; ++i) r[i] = 0.f;
      for (int kb = 0; kb < args.kblocks; ++kb) {
        const float s = nb < args.sb_ld ? args.sA[static_cast<size_t>(tm) * args.sa_ld + kb] *
                                              args.sB[static_cast<size_t>(kb) * args.sb_ld + nb]
                                        : 0.f;
        ok = __all_sync(FULL, mbar_wait(tfull_bar(acc), aph, args.timeout, abort_flag));
        if (!ok) break;
        tc_fence_after();
        const uint32_t t = tmem_base + (static_cast<uint32_t>(q * 32) << 16) + static_cast<uint32_t>(acc * BN + hc * 128);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          uint32_t p[32];
          tmem_ld_32x32b_x32(t + c * 32, p);
          tmem_ld_wait();
#pragma unroll
          for (int i = 0; i < 32; ++i) r[c * 32 + i] = fmaf(s, __uint_as_float(p[i]), r[c * 32 + i]);
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(tempty_bar(acc));
        if (++acc == NACC) {
          acc = 0;
          aph ^= 1u;
        }
      }
      if (!ok) break;
      const int row0 = tm * BM + q * 32;
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int col0 = tn * BN + hc * 128 + c * 32;
        if (row0 >= args.M || col0 >= args.N) continue;
        if (lane == 0) bulk_wait_read<1>();
        __syncwarp();
        const uint32_t buf = stg0 + sbuf * 4096;
#pragma unroll
        for (int j = 0; j < 8; ++j)
          st_shared_v4(buf + lane * 128 + ((j ^ (lane & 7)) << 4), r[c * 32 + 4 * j], r[c * 32 + 4 * j + 1],
                       r[c * 32 + 4 * j + 2], r[c * 32 + 4 * j + 3]);
        fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) {
          tma_store_2d(&tmC, buf, col0, row0);
          bulk_commit();
        }
        sbuf ^= 1;
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
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem_base, TMEM_COLS);
  }
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

extern "C" int rg_gemm_fp8(rg_ctx* ctx, int64_t M, int64_t N, int64_t K, const uint8_t* qA, int64_t lda,
                           const float* sA, const uint8_t* qB, int64_t ldb, const float* sB, float* C, int64_t ldc,
                           void* stream) {
  rg::clear_error();
  using namespace rg::fp8;
  if (!ctx) return rg::fail(RG_ERR_INVALID, "rg_gemm_fp8: null context");
  if (M < 0 || N < 0 || K < 0) return rg::fail(RG_ERR_INVALID, "rg_gemm_fp8: negative size");
  if (M == 0 || N == 0) return RG_OK;
  if (K == 0) {
    const cudaError_t e = cudaMemset2DAsync(C, ldc * 4, 0, N * 4, M, static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? RG_OK : rg::fail(RG_ERR_CUDA, "rg_gemm_fp8: memset");
  }
  if (!qA || !qB || !sA || !sB || !C) return rg::fail(RG_ERR_INVALID, "rg_gemm_fp8: null pointer");
  if (lda < K || ldb < N || ldc < N) return rg::fail(RG_ERR_INVALID, "rg_gemm_fp8: leading dimensions");
  if ((reinterpret_cast<uintptr_t>(qA) & 15) || (reinterpret_cast<uintptr_t>(qB) & 15) ||
      (reinterpret_cast<uintptr_t>(C) & 15) || (lda % 16) || (ldb % 16) || (ldc % 4))
    return rg::fail(RG_ERR_ALIGN, "rg_gemm_fp8: 16-byte aligned operands, lda and ldb multiples of 16, ldc of 4");
  if (M > (1 << 30) || N > (1 << 30) || K > (1 << 30)) return rg::fail(RG_ERR_SHAPE, "rg_gemm_fp8: size beyond 2^30");
  rg::Fp8CtxInfo info{};
  int rc = rg::ctx_fp8_info(ctx, &info);
  if (rc != RG_OK) return rc;
  int32_t* err = info.err;
  const long long timeout = info.timeout;
  const int sms = info.sms;
  rg::ctx_count_launches(ctx, 1);
  CUtensorMap a, b, c;
  rc = rg::fp8_make_map(&a, CU_TENSOR_MAP_DATA_TYPE_UINT8, qA, K, M, lda, BK, BM);
  if (rc == RG_OK) rc = rg::fp8_make_map(&b, CU_TENSOR_MAP_DATA_TYPE_UINT8, qB, N, K, ldb, 128, BK);
  if (rc == RG_OK) rc = rg::fp8_make_map(&c, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, C, N, M, ldc * 4, 32, 32);
  if (rc != RG_OK) return rc;
  Args args{};
  args.M = static_cast<int32_t>(M);
  args.N = static_cast<int32_t>(N);
  args.tiles_m = static_cast<int32_t>((M + BM - 1) / BM);
  args.tiles_n = static_cast<int32_t>((N + BN - 1) / BN);
  args.kblocks = static_cast<int32_t>((K + BK - 1) / BK);
  args.sa_ld = args.kblocks;
  args.sb_ld = static_cast<int32_t>((N + SB - 1) / SB);
  args.sA = sA;
  args.sB = sB;
  args.err = err;
  args.timeout = timeout;
  static bool attr_done[64] = {false};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev >= 0 && dev < 64 && !attr_done[dev]) {
    const cudaError_t e = cudaFuncSetAttribute(reinterpret_cast<const void*>(gemm_fp8_kernel),
                                               cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
    if (e != cudaSuccess) return rg::fail(RG_ERR_CUDA, "rg_gemm_fp8: shared-memory attribute");
    attr_done[dev] = true;
  }
  const int64_t units = static_cast<int64_t>(args.tiles_m) * args.tiles_n;
  dim3 grid(static_cast<unsigned>(std::min<int64_t>(units, sms)));
  void* params[4] = {&a, &b, &c, &args};
  const cudaError_t e = rg::fp8_launch_pdl(reinterpret_cast<const void*>(gemm_fp8_kernel), grid, kThreads, SMEM_BYTES,
                                           static_cast<cudaStream_t>(stream), params);
  return e == cudaSuccess ? RG_OK : rg::fail(RG_ERR_CUDA, std::string("rg_gemm_fp8: launch: ") + cudaGetErrorString(e));
}

namespace {
uint64_t splitmix_next_fp8(uint64_t& s) {
  uint64_t z = (s += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
}  // namespace

extern "C" int rg_sweep_fp8(rg_ctx* ctx, const rg_grid* grid, const uint8_t* qA, const float* sA, const uint8_t* qB,
                            const float* sB, float* C, const rg_sweep_opts* opts, int64_t* t_ns_out, void* stream) {
  rg::clear_error();
  using namespace rg::fp8;
  if (!ctx || !grid || !qA || !sA || !qB || !sB || !C || !t_ns_out)
    return rg::fail(RG_ERR_INVALID, "rg_sweep_fp8: null argument");
  if (!rg::grid_valid(*grid)) return rg::fail(RG_ERR_INVALID, "rg_sweep_fp8: invalid grid");
  rg_sweep_opts o;
  rg_sweep_opts_default(&o);
  if (opts) o = *opts;
  if (o.reps <= 0 || o.warmup < 0 || o.global_warmup < 0 || o.spin_ns < 0)
    return rg::fail(RG_ERR_INVALID, "rg_sweep_fp8: options");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int64_t cells = rg::cells_of(*grid);
  const int64_t nk = grid->k.count, nn = grid->n.count;
  std::vector<int64_t> order(static_cast<size_t>(cells));
  for (size_t i = 0; i < order.size(); ++i) order[i] = static_cast<int64_t>(i);
  if (o.shuffle) {
    uint64_t s = o.seed;
    for (size_t i = order.size() - 1; i > 0; --i) std::swap(order[i], order[splitmix_next_fp8(s) % (i + 1)]);
  }
  rg::Fp8CtxInfo info{};
  int rc = rg::ctx_fp8_info(ctx, &info);
  if (rc != RG_OK) return rc;
  int32_t* err = info.err;
  const long long timeout = info.timeout;
  const int sms = info.sms;
  if (cudaFuncSetAttribute(reinterpret_cast<const void*>(gemm_fp8_kernel), cudaFuncAttributeMaxDynamicSharedMemorySize,
                           SMEM_BYTES) != cudaSuccess)
    return rg::fail(RG_ERR_CUDA, "rg_sweep_fp8: shared-memory attribute");
  CUtensorMap ma, mb, mc;
  Args args{};
  dim3 grid_dim;
  auto prep = [&](int64_t cell, int* launches) -> int {
    const int64_t a = cell / (nn * nk), b = (cell / nk) % nn, c = cell % nk;
    const int64_t M = rg::axis_value(grid->m, a), N = rg::axis_value(grid->n, b), K = rg::axis_value(grid->k, c);
    if ((K % 16) || (N % 16)) return rg::fail(RG_ERR_ALIGN, "rg_sweep_fp8: grid sizes must be multiples of 16");
    int r = rg::fp8_make_map(&ma, CU_TENSOR_MAP_DATA_TYPE_UINT8, qA, K, M, K, BK, BM);
    if (r == RG_OK) r = rg::fp8_make_map(&mb, CU_TENSOR_MAP_DATA_TYPE_UINT8, qB, N, K, N, 128, BK);
    if (r == RG_OK) r = rg::fp8_make_map(&mc, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, C, N, M, N * 4, 32, 32);
    if (r != RG_OK) return r;
    args.M = static_cast<int32_t>(M);
    args.N = static_cast<int32_t>(N);
    args.tiles_m = static_cast<int32_t>((M + BM - 1) / BM);
    args.tiles_n = static_cast<int32_t>((N + BN - 1) / BN);
    args.kblocks = static_cast<int32_t>((K + BK - 1) / BK);
    args.sa_ld = args.kblocks;
    args.sb_ld = static_cast<int32_t>((N + SB - 1) / SB);
    args.sA = sA;
    args.sB = sB;
    args.err = err;
    args.timeout = timeout;
    grid_dim = dim3(static_cast<unsigned>(std::min<int64_t>(static_cast<int64_t>(args.tiles_m) * args.tiles_n, sms)));
    *launches = 1;
    return RG_OK;
  };
  auto run = [&]() -> cudaError_t {
    void* params[4] = {&ma, &mb, &mc, &args};
    return rg::fp8_launch_pdl(reinterpret_cast<const void*>(gemm_fp8_kernel), grid_dim, kThreads, SMEM_BYTES, st,
                              params);
  };
  rc = rg::timed_sweep(ctx, order, o, st, t_ns_out, prep, run);
  if (rc != RG_OK) return rc;
  return rg_check(ctx, stream);
}
