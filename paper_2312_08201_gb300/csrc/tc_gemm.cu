// tcgen05 + TMA GEMM for the mixed-precision Cauchy-panel product (see
// tc_gemm.cuh). One CTA computes a 128 x 128 FP32 tile in TMEM:
//   warp 0      TMA producer: 4 tiles per stage (A_hi, A_lo, B_hi, B_lo),
//               128-byte swizzled, completion counted on the stage's
//               "full" mbarrier;
//   warp 1      allocates 128 TMEM columns; one lane issues, per 16-wide K
//               slice, three tcgen05.mma (hi*hi, hi*lo, lo*hi) and commits
//               each stage to its "empty" mbarrier, and the whole tile to
//               the "accum" mbarrier;
//   warps 2..5  read the accumulator with tcgen05.ld (each warp its own
//               32-lane quarter) and store FP32 columns to global memory.
// Every mbarrier wait is bounded by a clock-based timeout; on expiry the
// CTA records an error, waits (bounded) for its copies in flight, releases
// TMEM and returns.
#include <cuda_bf16.h>

#include <cstring>
#include <mutex>

#include "lyap_internal.h"
#include "prof.h"
#include "tc_gemm.cuh"

namespace tc {
namespace {

constexpr uint32_t TILE_A = BM * BK * 2;                  // 16 KiB
constexpr uint32_t TILE_B = BN * BK * 2;                  // 16 KiB
constexpr uint32_t STAGE_BYTES = 2 * TILE_A + 2 * TILE_B;  // 64 KiB
constexpr uint32_t SMEM_BYTES = STAGES * STAGE_BYTES + 1024 + 256;
constexpr uint32_t TMEM_COLS = BN;
constexpr long long WAIT_CYCLES = 4000000000LL;  // about 2 s at 2 GHz

// kind::f16 instruction descriptor: D = F32, A = B = BF16, both K-major,
// N = BN, M = BM.
constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) |
                           ((uint32_t)(BM >> 4) << 24);

__device__ __forceinline__ uint32_t sm_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n"
      ".reg .pred p;\n"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      "selp.u32 %0, 1, 0, p;\n"
      "}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait for the phase of the given parity; false on timeout.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (clock64() - t0 > WAIT_CYCLES) return false;
  }
  return true;
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, uint32_t bar, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(
          dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(bar), "r"(x), "r"(y)
      : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_alloc(uint32_t dst_smem, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst_smem), "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t accumulate) {
  asm volatile(
      "{\n"
      ".reg .pred p;\n"
      "setp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n"
      "}\n" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(IDESC), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void umma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

// Shared-memory matrix descriptor, K-major operand in the canonical 128-byte
// swizzled layout written by TMA: 8-row groups 1024 bytes apart (stride
// byte offset), descriptor version 1, layout type 2 (128-byte swizzle).
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t saddr) {
  uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

__global__ void __launch_bounds__(192, 1)
    k_tc_gemm(const __grid_constant__ CUtensorMap tmAh, const __grid_constant__ CUtensorMap tmAl,
              const __grid_constant__ CUtensorMap tmBh, const __grid_constant__ CUtensorMap tmBl,
              float* __restrict__ D, int ldd, int mrows, int ktiles, const int* __restrict__ count, int col_mult,
              int ncols_host, int* __restrict__ err) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + STAGES * STAGE_BYTES);
  uint64_t* empty = full + STAGES;
  uint64_t* accum = empty + STAGES;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(accum + 1);
  int* ctl = reinterpret_cast<int*>(tmem_slot + 1);  // [0] issued, [1] consumed, [2] failed

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
  const int ncols = count ? (*count) * col_mult : ncols_host;
  if (n0 >= ncols) return;  // uniform for the CTA: nothing initialised yet

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(sm_addr(&full[s]), 1);
      mbar_init(sm_addr(&empty[s]), 1);
    }
    mbar_init(sm_addr(accum), 1);
    ctl[0] = ctl[1] = ctl[2] = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) tmem_alloc(sm_addr(tmem_slot), TMEM_COLS);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t taddr = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      int kt = 0;
      for (; kt < ktiles; ++kt) {
        const int s = kt % STAGES;
        const uint32_t ph = (uint32_t)(kt / STAGES) & 1u;
        if (!mbar_wait(sm_addr(&empty[s]), ph ^ 1u)) {
          atomicExch(err, 1);
          ctl[2] = 1;
          break;
        }
        uint8_t* st = smem + s * STAGE_BYTES;
        const uint32_t fb = sm_addr(&full[s]);
        mbar_expect_tx(fb, STAGE_BYTES);
        tma_load_2d(sm_addr(st), &tmAh, fb, kt * BK, m0);
        tma_load_2d(sm_addr(st + TILE_A), &tmAl, fb, kt * BK, m0);
        tma_load_2d(sm_addr(st + 2 * TILE_A), &tmBh, fb, kt * BK, n0);
        tma_load_2d(sm_addr(st + 2 * TILE_A + TILE_B), &tmBl, fb, kt * BK, n0);
      }
      ctl[0] = kt;
    }
  } else if (warp == 1) {
    if (lane == 0) {
      int kt = 0;
      for (; kt < ktiles; ++kt) {
        const int s = kt % STAGES;
        const uint32_t ph = (uint32_t)(kt / STAGES) & 1u;
        if (!mbar_wait(sm_addr(&full[s]), ph)) {
          atomicExch(err, 2);
          ctl[2] = 1;
          break;
        }
        tc_fence_after();
        const uint32_t a_h = sm_addr(smem + s * STAGE_BYTES);
        const uint32_t a_l = a_h + TILE_A;
        const uint32_t b_h = a_h + 2 * TILE_A;
        const uint32_t b_l = b_h + TILE_B;
#pragma unroll
        for (int kk = 0; kk < BK / 16; ++kk) {
          const uint32_t off = kk * 32;  // 16 BF16 along K inside the 128-byte swizzle row
          const uint64_t dah = sdesc_sw128(a_h + off), dal = sdesc_sw128(a_l + off);
          const uint64_t dbh = sdesc_sw128(b_h + off), dbl = sdesc_sw128(b_l + off);
          umma_bf16(taddr, dah, dbh, (kt > 0 || kk > 0) ? 1u : 0u);
          umma_bf16(taddr, dah, dbl, 1u);
          umma_bf16(taddr, dal, dbh, 1u);
        }
        umma_commit(sm_addr(&empty[s]));
      }
      ctl[1] = kt;
      umma_commit(sm_addr(accum));  // fires once every MMA issued above has completed
    }
  } else {
    const int q = warp & 3;  // lanes this warp may read: 32q .. 32q+31
    const bool ready = __all_sync(0xffffffffu, mbar_wait(sm_addr(accum), 0u));
    if (ready) {
      tc_fence_after();
      const int grow = m0 + q * 32 + lane;
#pragma unroll 1
      for (int c0 = 0; c0 < BN; c0 += 32) {
        float v[32];
        tmem_ld32(taddr + ((uint32_t)(q * 32) << 16) + (uint32_t)c0, v);
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const int col = n0 + c0 + j;
          if (grow < mrows && col < ncols) D[(size_t)col * ldd + grow] = v[j];
        }
      }
    } else {
      atomicExch(err, 3);
    }
  }
  tc_fence_before();
  __syncthreads();
  // On a timeout, wait (bounded) for the stages whose copies were issued but
  // not consumed, so no TMA write lands after the CTA has gone.
  if (threadIdx.x == 0 && ctl[2]) {
    for (int kt = ctl[1]; kt < ctl[0]; ++kt) mbar_wait(sm_addr(&full[kt % STAGES]), (uint32_t)(kt / STAGES) & 1u);
  }
  __syncthreads();
  if (warp == 1) {
    __syncwarp();
    tc_fence_after();
    tmem_dealloc(taddr, TMEM_COLS);
  }
}

using EncodeFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                              const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                              CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeFn encode_fn() {
  static EncodeFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeFn>(p);
  });
  return fn;
}

}  // namespace

int make_map(CUtensorMap* map, const void* base, int rows, int kpad, int box_rows) {
  EncodeFn fn = encode_fn();
  if (!fn) {
    lyap_set_last_error("cuTensorMapEncodeTiled not available from the driver");
    return LYAP_ECUDA;
  }
  if (kpad % BK != 0 || (reinterpret_cast<uintptr_t>(base) & 15u) != 0) return LYAP_EINVAL;
  std::memset(map, 0, sizeof(*map));
  cuuint64_t dims[2] = {(cuuint64_t)kpad, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)kpad * 2};
  cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    lyap_set_last_error("cuTensorMapEncodeTiled failed: " + std::to_string((int)r));
    return LYAP_ECUDA;
  }
  return LYAP_OK;
}

int launch(const Maps& m, float* D, int ldd, int mrows, int mpad, int kpad, const int* count, int col_mult,
           int ncols_host, int ncols_cap, int* err, cudaStream_t st) {
  if (mpad % BM != 0 || kpad % BK != 0 || ncols_cap <= 0) return LYAP_EINVAL;
  static std::once_flag once;
  static cudaError_t attr_rc = cudaSuccess;
  std::call_once(once, [] {
    attr_rc = cudaFuncSetAttribute(k_tc_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_BYTES);
  });
  LY_CUDA(attr_rc);
  dim3 grid(mpad / BM, (ncols_cap + BN - 1) / BN);
  k_tc_gemm<<<grid, 192, SMEM_BYTES, st>>>(m.a_hi, m.a_lo, m.b_hi, m.b_lo, D, ldd, mrows, kpad / BK, count, col_mult,
                                          ncols_host, err);
  lyap_count_launch();
  LY_CUDA(cudaGetLastError());
  return LYAP_OK;
}

}  // namespace tc
