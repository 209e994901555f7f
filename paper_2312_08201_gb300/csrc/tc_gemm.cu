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
// TMEM and returns. With `no_tma` set (the LYAP_INJECT_DEVICE_WAIT test
// hook) the producer issues no copy at all, so the MMA warp's first wait
// runs out after `wait_cycles` with nothing in flight.
#include <cuda_bf16.h>

#include <algorithm>
#include <cstring>
#include <mutex>

#include "lyap_internal.h"
#include "prof.h"
#include "tc_gemm.cuh"
#include "tcgen05_util.cuh"

namespace tc {
namespace {

constexpr uint32_t TILE_A = BM * BK * 2;                  // 16 KiB
constexpr uint32_t TILE_B = BN * BK * 2;                  // 16 KiB
constexpr uint32_t STAGE_BYTES = 2 * TILE_A + 2 * TILE_B;  // 64 KiB
constexpr uint32_t SMEM_BYTES = STAGES * STAGE_BYTES + 1024 + 256;
constexpr uint32_t TMEM_COLS = BN;

// kind::f16 instruction descriptor: D = F32, A = B = BF16, both K-major,
// N = BN, M = BM.
constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) |
                           ((uint32_t)(BM >> 4) << 24);

using namespace tcu;

__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t saddr) { return sdesc(saddr, 1024, 2); }

__global__ void __launch_bounds__(192, 1)
    k_tc_gemm(const __grid_constant__ CUtensorMap tmAh, const __grid_constant__ CUtensorMap tmAl,
              const __grid_constant__ CUtensorMap tmBh, const __grid_constant__ CUtensorMap tmBl,
              float* __restrict__ D, int ldd, int mrows, int ktiles_all, const int* __restrict__ count, int col_mult,
              int ncols_host, int* __restrict__ err, int no_tma, long long wait_cycles, int kt_per,
              size_t split_stride) {
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
  // split K: CTA z takes k-tiles [kt0, kt0 + ktiles) and writes its own
  // partial result at D + z * split_stride (the host makes every split
  // non-empty)
  const int kt0 = blockIdx.z * kt_per;
  const int ktiles = min(kt_per, ktiles_all - kt0);
  D += (size_t)blockIdx.z * split_stride;

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
      for (; kt < ktiles && !no_tma; ++kt) {
        const int s = kt % STAGES;
        const uint32_t ph = (uint32_t)(kt / STAGES) & 1u;
        if (!mbar_wait(sm_addr(&empty[s]), ph ^ 1u, wait_cycles)) {
          atomicExch(err, 1);
          ctl[2] = 1;
          break;
        }
        uint8_t* st = smem + s * STAGE_BYTES;
        const uint32_t fb = sm_addr(&full[s]);
        mbar_expect_tx(fb, STAGE_BYTES);
        const int kx = (kt0 + kt) * BK;
        tma_load_2d(sm_addr(st), &tmAh, fb, kx, m0);
        tma_load_2d(sm_addr(st + TILE_A), &tmAl, fb, kx, m0);
        tma_load_2d(sm_addr(st + 2 * TILE_A), &tmBh, fb, kx, n0);
        tma_load_2d(sm_addr(st + 2 * TILE_A + TILE_B), &tmBl, fb, kx, n0);
      }
      ctl[0] = kt;
    }
  } else if (warp == 1) {
    if (lane == 0) {
      int kt = 0;
      for (; kt < ktiles; ++kt) {
        const int s = kt % STAGES;
        const uint32_t ph = (uint32_t)(kt / STAGES) & 1u;
        if (!mbar_wait(sm_addr(&full[s]), ph, wait_cycles)) {
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
          umma_bf16(taddr, dah, dbh, IDESC, (kt > 0 || kk > 0) ? 1u : 0u);
          umma_bf16(taddr, dah, dbl, IDESC, 1u);
          umma_bf16(taddr, dal, dbh, IDESC, 1u);
        }
        umma_commit(sm_addr(&empty[s]));
      }
      ctl[1] = kt;
      umma_commit(sm_addr(accum));  // fires once every MMA issued above has completed
    }
  } else {
    const int q = warp & 3;  // lanes this warp may read: 32q .. 32q+31
    const bool ready = __all_sync(0xffffffffu, mbar_wait(sm_addr(accum), 0u, wait_cycles));
    if (ready && !no_tma) {
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
    for (int kt = ctl[1]; kt < ctl[0]; ++kt)
      mbar_wait(sm_addr(&full[kt % STAGES]), (uint32_t)(kt / STAGES) & 1u, wait_cycles);
  }
  __syncthreads();
  if (warp == 1) {
    __syncwarp();
    tc_fence_after();
    tmem_dealloc(taddr, TMEM_COLS);
  }
}

}  // namespace

}  // namespace tc

namespace tcu {
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
}  // namespace tcu

namespace tc {

int make_map(CUtensorMap* map, const void* base, int rows, int kpad, int box_rows) {
  tcu::EncodeFn fn = tcu::encode_fn();
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
           int ncols_host, int ncols_cap, int* err, cudaStream_t st, bool inject_no_tma) {
  return launch_split(m, D, ldd, mrows, mpad, kpad, count, col_mult, ncols_host, ncols_cap, 1, 0, err, st,
                      inject_no_tma);
}

int launch_split(const Maps& m, float* D, int ldd, int mrows, int mpad, int kpad, const int* count, int col_mult,
                 int ncols_host, int ncols_cap, int splits, size_t split_stride, int* err, cudaStream_t st,
                 bool inject_no_tma) {
  if (mpad % BM != 0 || kpad % BK != 0 || ncols_cap <= 0 || splits < 1) return LYAP_EINVAL;
  const int ktiles = kpad / BK;
  const int kt_per = (ktiles + splits - 1) / splits;
  if ((splits - 1) * kt_per >= ktiles) return LYAP_EINVAL;  // every split takes at least one k-tile
  LY_TRY(lyap_smem_optin(reinterpret_cast<const void*>(k_tc_gemm), SMEM_BYTES));
  dim3 grid(mpad / BM, (ncols_cap + BN - 1) / BN, splits);
  // the injected wait gives up after about 50 us instead of about 2 s
  const long long wait_cycles = inject_no_tma ? 100000LL : tcu::WAIT_CYCLES;
  k_tc_gemm<<<grid, 192, SMEM_BYTES, st>>>(m.a_hi, m.a_lo, m.b_hi, m.b_lo, D, ldd, mrows, ktiles, count, col_mult,
                                          ncols_host, err, inject_no_tma ? 1 : 0, wait_cycles, kt_per,
                                          split_stride);
  lyap_count_launch();
  LY_CUDA(cudaGetLastError());
  return LYAP_OK;
}

int splits_for(int kpad, int want) {
  const int ktiles = kpad / BK;
  int s = std::max(1, std::min(want, ktiles));
  while (s > 1 && (s - 1) * ((ktiles + s - 1) / s) >= ktiles) --s;
  return s;
}

}  // namespace tc
