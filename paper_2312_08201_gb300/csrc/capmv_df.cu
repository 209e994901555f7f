// FP64-accuracy capacitance residual on the FP32 pipes (mixed path).
//
// Refinement needs r = P - T(v) W to FP64 accuracy, but GB300 runs FP64 at
// 1/57 of its FP32 rate. This kernel evaluates the same Cauchy-panel product
// as the FP64 kernel (capmv64.cu) in float-float arithmetic: every value is
// an unevaluated sum hi + lo of two floats; a product keeps hi*hi exactly
// (FMA residue) plus the two cross terms; accumulation is an exact two-sum
// with the rounding errors gathered in the low word and renormalised after
// every K step. About 48 significant bits survive, so the residual error is
// within a small multiple of FP64 rounding of the terms it cancels.
//
// Range: float has an 8-bit exponent, so the operands are scaled by powers
// of two (exact) before they are split: Lc by the seed's 2^-ilogb(max |Lc|),
// Ub/Vb by the seed's 2^-ilogb(max |Ub|, |Vb|), and each system's W by
// 2^-ilogb(max |W_b|), taken on the device before the product. The FP64
// epilogue undoes the scaling and adds the Gd and D(v)^{-1} terms.
#include <mutex>

#include "capmv.cuh"
#include "cplx.cuh"
#include "lyap_internal.h"
#include "prof.h"

namespace {

constexpr int TI = 64, TNC = 64, TJ = 16, SROW = TNC + 1;
constexpr double kFFInstrPerCmac = 54.0;

struct ff2 {  // complex float-float: re = rh + rl, im = ih + il
  float rh, rl, ih, il;
};

__device__ __forceinline__ ff2 to_ff(double2 a) {
  ff2 r;
  r.rh = (float)a.x;
  r.rl = (float)(a.x - (double)r.rh);
  r.ih = (float)a.y;
  r.il = (float)(a.y - (double)r.ih);
  return r;
}

// (sh, sl) += a * b for float-float a, b: exact hi*hi product by FMA, the two
// cross terms rounded once, exact two-sum into sh with the errors kept in sl.
__device__ __forceinline__ void ff_mac(float ah, float al, float bh, float bl, float& sh, float& sl) {
  const float ph = ah * bh;
  float pl = fmaf(ah, bh, -ph);
  pl = fmaf(ah, bl, pl);
  pl = fmaf(al, bh, pl);
  const float s = sh + ph;
  const float t = s - sh;
  const float e = (sh - (s - t)) + (ph - t);
  sh = s;
  sl += e + pl;
}

__device__ __forceinline__ void ff_norm(float& h, float& l) {
  const float s = h + l;
  l = l - (s - h);
  h = s;
}

struct Acc {
  float rh, rl, ih, il;
};

__device__ __forceinline__ void cmac_ff(const ff2& a, const ff2& b, Acc& c) {
  // re += ar br - ai bi ; im += ar bi + ai br
  ff_mac(a.rh, a.rl, b.rh, b.rl, c.rh, c.rl);
  ff_mac(-a.ih, -a.il, b.ih, b.il, c.rh, c.rl);
  ff_mac(a.rh, a.rl, b.ih, b.il, c.ih, c.il);
  ff_mac(a.ih, a.il, b.rh, b.rl, c.ih, c.il);
}

// Per-system power-of-two scale of W (listed systems): sw[b] = 2^-ilogb(max |W_b|).
__global__ void __launch_bounds__(256) k_sys_scale(CapArgs64 a, double* __restrict__ sw) {
  __shared__ double red[256];
  const int nsys = a.count ? *a.count : a.nsys;
  if ((int)blockIdx.x >= nsys) return;
  const int b = a.list ? a.list[blockIdx.x] : (int)blockIdx.x;
  const size_t N = (size_t)a.n * a.k;
  const double2* W = a.W + (size_t)b * a.ldw;
  double mx = 0.0;
  for (size_t e = threadIdx.x; e < N; e += 256) mx = fmax(mx, fmax(fabs(W[e].x), fabs(W[e].y)));
  red[threadIdx.x] = mx;
  __syncthreads();
  for (int st = 128; st > 0; st >>= 1) {
    if ((int)threadIdx.x < st) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + st]);
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double m = red[0];
    int e = (m > 0.0 && isfinite(m)) ? ilogb(m) : 0;
    e = max(-600, min(600, e));
    sw[b] = ldexp(1.0, -e);
  }
}

__global__ void __launch_bounds__(256) k_capmv_df(CapArgs64 a, const float4* __restrict__ Lff, double sp,
                                                  double inv_lp, const double* __restrict__ sw) {
  extern __shared__ double2 smem[];
  ff2* sA = reinterpret_cast<ff2*>(smem);  // [TJ][TI]
  ff2* sB = sA + TJ * TI;                   // [TJ][TNC]
  const int n = a.n, k = a.k, kk = k * k;
  const int SB = TNC / kk;
  const int ncols = SB * kk;
  const int nsys = a.count ? *a.count : a.nsys;
  const int s0 = blockIdx.y * SB;
  if (s0 >= nsys) return;
  const int i0 = blockIdx.x * TI;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  Acc acc[4][4];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[r][c] = Acc{0.f, 0.f, 0.f, 0.f};

  for (int j0 = 0; j0 < n; j0 += TJ) {
#pragma unroll
    for (int q = 0; q < (TJ * TI) / 256; ++q) {
      const int e = tid + 256 * q;
      const int jj = e / TI, ii = e % TI;
      const int i = i0 + ii, j = j0 + jj;
      ff2 v{0.f, 0.f, 0.f, 0.f};
      if (i < n && j < n) {
        const float4 l = Lff[(size_t)j * n + i];
        v = ff2{l.x, l.y, l.z, l.w};
      }
      sA[jj * TI + ii] = v;
    }
#pragma unroll
    for (int q = 0; q < (TJ * TNC) / 256; ++q) {
      const int e = tid + 256 * q;
      const int jj = e / TNC, cc = e % TNC;
      const int j = j0 + jj;
      ff2 v{0.f, 0.f, 0.f, 0.f};
      const int sl = cc / kk;
      if (cc < ncols && j < n && s0 + sl < nsys) {
        const int pt = cc % kk, p = pt / k, t = pt % k;
        const int b = a.list ? a.list[s0 + sl] : s0 + sl;
        v = to_ff(cmul(cscale(a.W[(size_t)b * a.ldw + (size_t)p * n + j], sw[b]), cscale(a.P2[(size_t)t * n + j], sp)));
      }
      sB[jj * TNC + cc] = v;
    }
    __syncthreads();
#pragma unroll 2
    for (int jj = 0; jj < TJ; ++jj) {
      ff2 av[4], bv[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) av[r] = sA[jj * TI + ty + 16 * r];
#pragma unroll
      for (int c = 0; c < 4; ++c) bv[c] = sB[jj * TNC + tx + 16 * c];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          cmac_ff(av[r], bv[c], acc[r][c]);
          ff_norm(acc[r][c].rh, acc[r][c].rl);
          ff_norm(acc[r][c].ih, acc[r][c].il);
        }
    }
    __syncthreads();
  }

  double2* S = smem;
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const int sl = (tx + 16 * c) / kk;
    double us = 0.0;  // undo the Lc, Ub/Vb and W scales (exact powers of two)
    if (tx + 16 * c < ncols && s0 + sl < nsys) us = inv_lp / sw[a.list ? a.list[s0 + sl] : s0 + sl];
#pragma unroll
    for (int r = 0; r < 4; ++r)
      S[(ty + 16 * r) * SROW + tx + 16 * c] = make_double2(((double)acc[r][c].rh + (double)acc[r][c].rl) * us,
                                                           ((double)acc[r][c].ih + (double)acc[r][c].il) * us);
  }
  __syncthreads();

  const int nout = TI * SB * k;
  for (int e = tid; e < nout; e += 256) {
    const int ii = e % TI, rest = e / TI;
    const int t = rest % k, sl = rest / k;
    const int i = i0 + ii;
    if (i >= n || s0 + sl >= nsys) continue;
    const int b = a.list ? a.list[s0 + sl] : s0 + sl;
    const double2* Wb = a.W + (size_t)b * a.ldw;
    double2 o = make_double2(0.0, 0.0);
    for (int p = 0; p < k; ++p) {
      o = cfma(a.P1[(size_t)p * n + i], S[ii * SROW + (sl * k + p) * k + t], o);
      const size_t gidx = a.gT ? ((size_t)(t * k + p) * n + i) : ((size_t)(p * k + t) * n + i);
      o = cfma(Wb[(size_t)p * n + i], a.Gd[gidx], o);
    }
    double2 y = o;
    if (a.mode != CAP_C0) {
      const double2 wt = Wb[(size_t)t * n + i];
      y = csub(cscale(wt, a.vinv[(size_t)b * k + t]), o);
      if (a.mode == CAP_RESID) y = csub(a.rhs[(size_t)b * a.ldr + (size_t)t * n + i], y);
    }
    a.out[(size_t)b * a.ldo + (size_t)t * n + i] = y;
  }
}

__global__ void k_build_lff(int n, const double2* __restrict__ lam, double sl, float4* __restrict__ Lff) {
  const size_t total = (size_t)n * n;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
    const size_t i = idx % n, j = idx / n;
    const double2 L = cscale(crcp(cadd(lam[i], lam[j])), sl);
    const float rh = (float)L.x, ih = (float)L.y;
    Lff[idx] = make_float4(rh, (float)(L.x - (double)rh), ih, (float)(L.y - (double)ih));
  }
}

}  // namespace

int capmv_df_build_lc(int n, const double2* lam, double lc_scale, float4* Lff, cudaStream_t st) {
  const size_t total = (size_t)n * n;
  const int grid = (int)std::min<size_t>((total + 255) / 256, 8192);
  k_build_lff<<<grid, 256, 0, st>>>(n, lam, lc_scale, Lff);
  lyap_count_launch();
  LY_CUDA(cudaGetLastError());
  return LYAP_OK;
}

int capmv_df_launch(const CapArgs64& a, const float4* Lff, double lc_scale, double p_scale, double* sw,
                    cudaStream_t st) {
  if (a.k < 1 || a.k > 8) return LYAP_EINVAL;
  if (a.nsys <= 0) return LYAP_OK;
  const int kk = a.k * a.k;
  const int SB = TNC / kk;
  const size_t smem = (size_t)TI * SROW * sizeof(double2);
  static std::once_flag once;
  static cudaError_t attr_rc = cudaSuccess;
  std::call_once(once, [&] {
    attr_rc = cudaFuncSetAttribute(k_capmv_df, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  });
  LY_CUDA(attr_rc);
  k_sys_scale<<<a.nsys, 256, 0, st>>>(a, sw);
  lyap_count_launch();
  dim3 grid((a.n + TI - 1) / TI, (a.nsys + SB - 1) / SB);
  // work per system: n^2 k^2 float-float complex multiply-adds of 54 FP32
  // instructions each (4 products of 12, two renormalisations of 3)
  const int ph = prof_begin(PK_CAPMV_FF, st);
  k_capmv_df<<<grid, 256, smem, st>>>(a, Lff, p_scale, 1.0 / (lc_scale * p_scale), sw);
  lyap_count_launch();
  prof_end(ph, st, kFFInstrPerCmac * (double)a.n * a.n * kk, 2.0 * (double)a.n * a.k * sizeof(double2),
           a.count ? 0 : a.nsys, a.count);
  LY_CUDA(cudaGetLastError());
  return LYAP_OK;
}
