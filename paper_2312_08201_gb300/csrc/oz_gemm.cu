// Integer-sliced BF16 tensor-core Cauchy-panel product (see oz_gemm.cuh).
//
// k_oz_gemm computes, for one 128-row x 64-column tile, the NS order
// accumulators ACC_0..ACC_{NS-1} (NS x 64 = 512 TMEM columns):
//   warp 0      TMA producer: per K stage the NS digit tiles of A and of B
//               (64-byte swizzle), completion counted on the stage's "full"
//               mbarrier;
//   warp 1      allocates TMEM; one lane issues, per 16-wide K slice, one
//               tcgen05.mma per digit pair (s, t) with s + t < NS into the
//               accumulator of order s + t, commits each stage to its
//               "empty" mbarrier and the tile to the "accum" mbarrier;
//   warps 2..5  read the NS accumulators with tcgen05.ld, combine them in
//               float-float (sum_d 64^-d ACC_d) and store (hi, lo).
// Every mbarrier wait is bounded by a clock-based timeout; on expiry the CTA
// records an error, waits (bounded) for its copies in flight, releases TMEM
// and returns.
#include <cuda_bf16.h>

#include <algorithm>
#include <cstring>
#include <mutex>

#include "cplx.cuh"
#include "lyap_internal.h"
#include "oz_gemm.cuh"
#include "prof.h"
#include "tcgen05_util.cuh"

namespace oz {
namespace {

using namespace tcu;

constexpr uint32_t TILE_A = BM * BK * 2;                      // 8 KiB per digit
constexpr uint32_t TILE_B = BN * BK * 2;                      // 4 KiB per digit
constexpr uint32_t STAGE_BYTES = NS * (TILE_A + TILE_B);      // 96 KiB
constexpr uint32_t SMEM_BYTES = STAGES * STAGE_BYTES + 1024 + 256;
constexpr uint32_t TMEM_COLS = NS * BN;                        // 512
constexpr uint32_t IDESC = idesc_bf16(BM, BN);
constexpr double PAIRS = NS * (NS + 1) / 2;                   // digit products per K element

__device__ __forceinline__ uint64_t sdesc_sw64(uint32_t saddr) { return sdesc(saddr, 512, 4); }

__device__ __forceinline__ double block_max(double v, double* red) {
  red[threadIdx.x] = v;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + s]);
    __syncthreads();
  }
  const double m = red[0];
  __syncthreads();
  return m;
}

// power-of-two exponent e with max / 2^e < 1/2 (0 for an all-zero row)
__device__ __forceinline__ int scale_exp(double m) { return (m > 0.0 && isfinite(m)) ? ilogb(m) + 2 : 0; }

// NS balanced base-64 digits of x in [-1/2, 1/2]; exact arithmetic in FP64
__device__ __forceinline__ void write_digits(double x, __nv_bfloat16* S, size_t slice_stride) {
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    const double y = x * 64.0;
    const double d = rint(y);
    x = y - d;
    S[(size_t)s * slice_stride] = __float2bfloat16_rn((float)d);
  }
}

__global__ void __launch_bounds__(256) k_slice_A(int n, const double2* __restrict__ lam, int mpad, int kpad, int rs,
                                                 __nv_bfloat16* __restrict__ S, int* __restrict__ eA) {
  __shared__ double red[256];
  const int r = blockIdx.x;
  const int rows = rs * n;
  auto val = [&](int c) -> double {
    if (r >= rows || c >= rows) return 0.0;
    const double2 L = crcp(cadd(lam[r / rs], lam[c / rs]));
    if (rs == 1) return L.x;
    if ((r & 1) == 0) return (c & 1) == 0 ? L.x : -L.y;
    return (c & 1) == 0 ? L.y : L.x;
  };
  double mx = 0.0;
  for (int c = threadIdx.x; c < kpad; c += blockDim.x) mx = fmax(mx, fabs(val(c)));
  const int e = scale_exp(block_max(mx, red));
  if (threadIdx.x == 0) eA[r] = e;
  const double sc = ldexp(1.0, -e);
  for (int c = threadIdx.x; c < kpad; c += blockDim.x)
    write_digits(val(c) * sc, S + (size_t)r * kpad + c, (size_t)mpad * kpad);
}

// NS balanced base-64 digits of q = x 2^48 (|q| <= 2^47), top digit first,
// by integer arithmetic (round to nearest at every digit, as write_digits).
__device__ __forceinline__ void write_digits_int(long long q, __nv_bfloat16* S, size_t slice_stride) {
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    const int b = 6 * (NS - 1 - s);
    const long long d = b > 0 ? ((q + (1LL << (b - 1))) >> b) : q;
    q -= d << b;
    S[(size_t)s * slice_stride] = __float2bfloat16_rn((float)d);
  }
}

// Panel digits of the listed systems: W_b[:, p] o P2[:, t] for (p, t) =
// pt, real-split along K in column slot * k^2 + pt (rs = 2), or its real and
// imaginary parts in columns 2 (slot * k^2 + pt) and 2 (slot * k^2 + pt) + 1
// (rs = 1). The column is formed once in shared memory; its digits come from
// one rounding to 48 bits and integer digit extraction (GB300's FP64 pipe is
// narrow).
__global__ void __launch_bounds__(256) k_slice_B(CapArgs64 a, int ncap, int kpad, int rs,
                                                 __nv_bfloat16* __restrict__ S, int* __restrict__ eB) {
  extern __shared__ double zcol[];  // kpad
  __shared__ double red[256];
  const int nsys = a.count ? *a.count : a.nsys;
  const int slot = blockIdx.x;
  if (slot >= nsys) return;
  const int b = a.list ? a.list[slot] : slot;
  const int n = a.n, k = a.k, kk = k * k, rows = rs * n, cm = 3 - rs;
  const double2* Wb = a.W + (size_t)b * a.ldw;
  for (int q = 0; q < kk * cm; ++q) {
    const int pt = q / cm, h = q % cm;  // h: 1 for the imaginary-part column (rs = 1)
    const int p = pt / k, t = pt % k;
    const int col = slot * kk * cm + q;
    double mx = 0.0;
    for (int c = threadIdx.x; c < kpad; c += blockDim.x) {
      double v = 0.0;
      if (c < rows) {
        const int j = c / rs;
        const double2 z = cmul(Wb[(size_t)p * n + j], a.P2[(size_t)t * n + j]);
        v = (rs == 2 ? (c & 1) : h) ? z.y : z.x;
      }
      zcol[c] = v;
      mx = fmax(mx, fabs(v));
    }
    const int e = scale_exp(block_max(mx, red));  // its barriers also publish zcol
    if (threadIdx.x == 0) eB[col] = e;
    const double sc = ldexp(1.0, 48 - e);
    for (int c = threadIdx.x; c < kpad; c += blockDim.x)
      write_digits_int(__double2ll_rn(zcol[c] * sc), S + (size_t)col * kpad + c, (size_t)ncap * kpad);
    __syncthreads();  // zcol is rewritten by the next column
  }
}

__global__ void __launch_bounds__(192, 1)
    k_oz_gemm(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
              float2* __restrict__ D, int ldd, int mrows, int mpad, int ncap, int kt0, int ktiles, int accumulate,
              const int* __restrict__ count, int col_mult, int ncols_host, int* __restrict__ err) {
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
          atomicExch(err, 11);
          ctl[2] = 1;
          break;
        }
        uint8_t* st = smem + s * STAGE_BYTES;
        const uint32_t fb = sm_addr(&full[s]);
        mbar_expect_tx(fb, STAGE_BYTES);
#pragma unroll 1
        for (int g = 0; g < NS; ++g) {
          tma_load_2d(sm_addr(st + g * TILE_A), &tmA, fb, (kt0 + kt) * BK, g * mpad + m0);
          tma_load_2d(sm_addr(st + NS * TILE_A + g * TILE_B), &tmB, fb, (kt0 + kt) * BK, g * ncap + n0);
        }
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
          atomicExch(err, 12);
          ctl[2] = 1;
          break;
        }
        tc_fence_after();
        const uint32_t a0 = sm_addr(smem + s * STAGE_BYTES);
        const uint32_t b0 = a0 + NS * TILE_A;
#pragma unroll
        for (int kk = 0; kk < BK / 16; ++kk) {
          const uint32_t off = kk * 32;  // 16 BF16 along K inside the 64-byte swizzle row
#pragma unroll
          for (int sa = 0; sa < NS; ++sa) {
            const uint64_t da = sdesc_sw64(a0 + sa * TILE_A + off);
#pragma unroll
            for (int sb = 0; sa + sb < NS; ++sb) {
              const uint64_t db = sdesc_sw64(b0 + sb * TILE_B + off);
              // the order's first product (sa = 0) starts its accumulator
              umma_bf16(taddr + (uint32_t)((sa + sb) * BN), da, db, IDESC, (kt > 0 || kk > 0 || sa > 0) ? 1u : 0u);
            }
          }
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
      const uint32_t lane_base = taddr + ((uint32_t)(q * 32) << 16);
#pragma unroll 1
      for (int c0 = 0; c0 < BN; c0 += 32) {
        float h[32], l[32];
        tmem_ld32(lane_base + (uint32_t)c0, h);
#pragma unroll
        for (int j = 0; j < 32; ++j) l[j] = 0.f;
        float w = 1.f;
#pragma unroll 1
        for (int d = 1; d < NS; ++d) {
          w *= 0.015625f;  // 64^-d, exact
          float v[32];
          tmem_ld32(lane_base + (uint32_t)(d * BN + c0), v);
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            const float x = v[j] * w;  // exact: an integer below 2^24 times a power of two
            const float s2 = h[j] + x;
            const float t2 = s2 - h[j];
            l[j] += (h[j] - (s2 - t2)) + (x - t2);
            h[j] = s2;
          }
        }
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const int col = n0 + c0 + j;
          if (grow < mrows && col < ncols) {
            float2* dp = D + (size_t)col * ldd + grow;
            if (accumulate) {
              // add this K chunk to the earlier ones: exact two-sum of the high
              // words, its error and the low words in the low word
              const float2 o = *dp;
              const float s2 = o.x + h[j];
              const float t2 = s2 - o.x;
              *dp = make_float2(s2, o.y + l[j] + ((o.x - (s2 - t2)) + (h[j] - t2)));
            } else {
              *dp = make_float2(h[j], l[j]);
            }
          }
        }
      }
    } else {
      atomicExch(err, 13);
    }
  }
  tc_fence_before();
  __syncthreads();
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

// T(v) W (or the residual) from the sliced product: S_{p,t}[i] for the
// listed systems, then the same FP64 epilogue as the other residual kernels.
__global__ void __launch_bounds__(128) k_oz_epi(CapArgs64 a, const float2* __restrict__ D, int ldd, int rs,
                                                const int* __restrict__ eA, const int* __restrict__ eB) {
  const int nsys = a.count ? *a.count : a.nsys;
  const int slot = blockIdx.y;
  if (slot >= nsys) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int n = a.n, k = a.k, kk = k * k;
  if (i >= n) return;
  const int b = a.list ? a.list[slot] : slot;
  const double2* Wb = a.W + (size_t)b * a.ldw;
  const int er = rs == 2 ? eA[2 * i] : eA[i], ei = rs == 2 ? eA[2 * i + 1] : eA[i];
  for (int t = 0; t < k; ++t) {
    double2 o = make_double2(0.0, 0.0);
    for (int p = 0; p < k; ++p) {
      const int col = slot * kk + p * k + t;
      // real part: row 2i of column col (rs = 2) or row i of column 2 col (rs = 1)
      const size_t xr = rs == 2 ? (size_t)col * ldd + 2 * i : (size_t)(2 * col) * ldd + i;
      const size_t xi = rs == 2 ? xr + 1 : xr + ldd;
      const int cr = rs == 2 ? col : 2 * col, ci = rs == 2 ? col : 2 * col + 1;
      const float2 dr = D[xr], di = D[xi];
      const double2 S = make_double2(ldexp((double)dr.x + (double)dr.y, er + eB[cr] - 12),
                                     ldexp((double)di.x + (double)di.y, ei + eB[ci] - 12));
      o = cfma(a.P1[(size_t)p * n + i], S, o);
      const size_t gidx = a.gT ? ((size_t)(t * k + p) * n + i) : ((size_t)(p * k + t) * n + i);
      o = cfma(Wb[(size_t)p * n + i], a.Gd[gidx], o);
    }
    double2 y = o;
    if (a.mode != CAP_C0) {
      y = csub(cscale(Wb[(size_t)t * n + i], a.vinv[(size_t)b * k + t]), o);
      if (a.mode == CAP_RESID) y = csub(a.rhs[(size_t)b * a.ldr + (size_t)t * n + i], y);
    }
    a.out[(size_t)b * a.ldo + (size_t)t * n + i] = y;
  }
}

}  // namespace

int slice_A(int n, const double2* lam, int mpad, int kpad, int rs, void* S, int* eA, cudaStream_t st) {
  if (mpad % BM != 0 || kpad % BK != 0 || (rs != 1 && rs != 2)) return LYAP_EINVAL;
  k_slice_A<<<mpad, 256, 0, st>>>(n, lam, mpad, kpad, rs, reinterpret_cast<__nv_bfloat16*>(S), eA);
  lyap_count_launch();
  LY_CUDA(cudaGetLastError());
  return LYAP_OK;
}

int make_map(CUtensorMap* map, const void* base, int rows_total, int kpad, int box_rows) {
  tcu::EncodeFn fn = tcu::encode_fn();
  if (!fn) {
    lyap_set_last_error("cuTensorMapEncodeTiled not available from the driver");
    return LYAP_ECUDA;
  }
  if (kpad % BK != 0 || (reinterpret_cast<uintptr_t>(base) & 15u) != 0) return LYAP_EINVAL;
  std::memset(map, 0, sizeof(*map));
  cuuint64_t dims[2] = {(cuuint64_t)kpad, (cuuint64_t)rows_total};
  cuuint64_t strides[1] = {(cuuint64_t)kpad * 2};
  cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    lyap_set_last_error("cuTensorMapEncodeTiled failed: " + std::to_string((int)r));
    return LYAP_ECUDA;
  }
  return LYAP_OK;
}

int residual(const CapArgs64& a, const CUtensorMap& mapA, const int* eA, int mpad, int kpad, int rs, Panel& pn,
             int* err, cudaStream_t st) {
  if (a.k < 1 || a.k > 8 || (rs != 1 && rs != 2)) return LYAP_EINVAL;
  if (a.nsys <= 0) return LYAP_OK;
  const int cm = 3 - rs;  // panel columns per (system, p, t)
  const int kk = a.k * a.k;
  const int ncols_cap = a.nsys * kk * cm;
  if (ncols_cap > pn.ncap) return LYAP_EINVAL;
  LY_TRY(lyap_smem_optin(reinterpret_cast<const void*>(k_oz_gemm), SMEM_BYTES));
  // one column of kpad doubles in shared memory (51 KB at n = 3200)
  LY_TRY(lyap_smem_optin(reinterpret_cast<const void*>(k_slice_B), sizeof(double) * kpad));
  k_slice_B<<<a.nsys, 256, sizeof(double) * kpad, st>>>(a, pn.ncap, kpad, rs, reinterpret_cast<__nv_bfloat16*>(pn.S),
                                                         pn.eB);
  lyap_count_launch();
  LY_CUDA(cudaGetLastError());
  // tensor work per system: NS (NS + 1) / 2 BF16 products of the (rs n x rs n) x (rs n x cm k^2) GEMM
  const int ph = prof_begin(PK_OZGEMM, st);
  dim3 grid(mpad / BM, (ncols_cap + BN - 1) / BN);
  // K in chunks of at most KCHUNK, each summed exactly in FP32 and added to
  // the previous chunks' float-float results (one chunk for 2n <= KCHUNK)
  for (int k0 = 0; k0 < kpad; k0 += KCHUNK) {
    const int kt = (std::min(KCHUNK, kpad - k0)) / BK;
    k_oz_gemm<<<grid, 192, SMEM_BYTES, st>>>(mapA, pn.mapB, pn.D, mpad, rs * a.n, mpad, pn.ncap, k0 / BK, kt,
                                            k0 > 0 ? 1 : 0, a.count, kk * cm, ncols_cap, err);
    lyap_count_launch();
  }
  prof_end(ph, st, PAIRS * 2.0 * (double)(rs * a.n) * (rs * a.n) * kk * cm, 0.0, a.count ? 0 : a.nsys, a.count);
  LY_CUDA(cudaGetLastError());
  k_oz_epi<<<dim3((a.n + 127) / 128, a.nsys), 128, 0, st>>>(a, pn.D, mpad, rs, eA, pn.eB);
  lyap_count_launch();
  LY_CUDA(cudaGetLastError());
  return LYAP_OK;
}

}  // namespace oz
