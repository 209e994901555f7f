// FP64-accuracy capacitance residual on the FP32 pipes (mixed path).
//
// Refinement needs r = P - T(v) W to FP64 accuracy, but GB300 runs FP64 at
// 1/57 of its FP32 rate. This kernel evaluates the same Cauchy-panel product
// as the FP64 kernel (capmv64.cu) in float-float arithmetic: every value is
// an unevaluated sum hi + lo of two floats; a product keeps hi*hi exactly
// (FMA residue) plus the two cross terms; accumulation is an exact two-sum
// with the rounding errors gathered in the low word and renormalised every
// few K steps. About 48 significant bits survive, so the residual error is
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

constexpr int TI = 64, TNC = 64, TJ = 16, SROW = TNC + 1, SBROW = TNC + 1;
constexpr int NORM_EVERY = 4;
// FP32 instructions per float-float complex multiply-add: 4 products of 12
// and two renormalisations of 3 every NORM_EVERY steps
constexpr double kFFInstrPerCmac = 48.0 + 6.0 / NORM_EVERY;

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

// Float-float panel of the listed systems, built once per launch so that the
// product loop runs on FP32 pipes only. Slot s (system b = list[s]) gets
//   sw[b] = 2^-ilogb(max |W_b|),
//   panel[s][p k + t][j] = split((W_b[j, p] sw[b]) (P2[j, t] sp))
// as float4 (re hi, re lo, im hi, im lo).
__global__ void __launch_bounds__(256) k_panel_ff(CapArgs64 a, double sp, double* __restrict__ sw,
                                                  float4* __restrict__ panel) {
  __shared__ double red[256];
  const int nsys = a.count ? *a.count : a.nsys;
  const int slot = blockIdx.x;
  if (slot >= nsys) return;
  const int b = a.list ? a.list[slot] : slot;
  const int n = a.n, k = a.k, kk = k * k;
  const size_t N = (size_t)n * k;
  const double2* W = a.W + (size_t)b * a.ldw;
  double mx = 0.0;
  for (size_t e = threadIdx.x; e < N; e += 256) mx = fmax(mx, fmax(fabs(W[e].x), fabs(W[e].y)));
  red[threadIdx.x] = mx;
  __syncthreads();
  for (int st = 128; st > 0; st >>= 1) {
    if ((int)threadIdx.x < st) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + st]);
    __syncthreads();
  }
  const double m = red[0];
  int ex = (m > 0.0 && isfinite(m)) ? ilogb(m) : 0;
  ex = max(-600, min(600, ex));
  const double sws = ldexp(1.0, -ex);
  if (threadIdx.x == 0) sw[b] = sws;
  float4* out = panel + (size_t)slot * kk * n;
  for (size_t e = threadIdx.x; e < (size_t)kk * n; e += 256) {
    const int pt = (int)(e / n), j = (int)(e % n);
    const int p = pt / k, t = pt % k;
    const ff2 v = to_ff(cmul(cscale(W[(size_t)p * n + j], sws), cscale(a.P2[(size_t)t * n + j], sp)));
    out[e] = make_float4(v.rh, v.rl, v.ih, v.il);
  }
}

__global__ void __launch_bounds__(256, 2) k_capmv_df(CapArgs64 a, const float4* __restrict__ Lff,
                                                     const float4* __restrict__ panel, double inv_lp,
                                                     const double* __restrict__ sw) {
  extern __shared__ double2 smem[];
  ff2* sA = reinterpret_cast<ff2*>(smem);  // [TJ][TI]
  ff2* sB = sA + TJ * TI;                   // [TJ][SBROW]
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
      // 16 consecutive threads read 16 consecutive rows of one panel column
      const int e = tid + 256 * q;
      const int jj = e % TJ, cc = e / TJ;
      const int j = j0 + jj;
      ff2 v{0.f, 0.f, 0.f, 0.f};
      const int sl = cc / kk;
      if (cc < ncols && j < n && s0 + sl < nsys) {
        const float4 f = panel[((size_t)(s0 + sl) * kk + cc % kk) * n + j];
        v = ff2{f.x, f.y, f.z, f.w};
      }
      sB[jj * SBROW + cc] = v;
    }
    __syncthreads();
#pragma unroll 1
    for (int jq = 0; jq < TJ; jq += NORM_EVERY) {
#pragma unroll 1
      for (int jj = jq; jj < jq + NORM_EVERY; ++jj) {
        ff2 bv[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) bv[c] = sB[jj * SBROW + tx + 16 * c];
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          const ff2 av = sA[jj * TI + ty + 16 * r];
#pragma unroll
          for (int c = 0; c < 4; ++c) cmac_ff(av, bv[c], acc[r][c]);
        }
      }
      // fold the low words back every NORM_EVERY steps: between folds each low
      // word gathers 2 NORM_EVERY rounding errors of at most 2^-24 of the sum
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
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
                    float4* panel, cudaStream_t st) {
  if (a.k < 1 || a.k > 8) return LYAP_EINVAL;
  if (a.nsys <= 0) return LYAP_OK;
  const int kk = a.k * a.k;
  const int SB = TNC / kk;
  const size_t smem = (size_t)TI * SROW * sizeof(double2);
  LY_TRY(lyap_smem_optin(reinterpret_cast<const void*>(k_capmv_df), smem));
  k_panel_ff<<<a.nsys, 256, 0, st>>>(a, p_scale, sw, panel);
  lyap_count_launch();
  dim3 grid((a.n + TI - 1) / TI, (a.nsys + SB - 1) / SB);
  // work per system: n^2 k^2 float-float complex multiply-adds of
  // kFFInstrPerCmac FP32 instructions each
  const int ph = prof_begin(PK_CAPMV_FF, st);
  k_capmv_df<<<grid, 256, smem, st>>>(a, Lff, panel, 1.0 / (lc_scale * p_scale), sw);
  lyap_count_launch();
  prof_end(ph, st, kFFInstrPerCmac * (double)a.n * a.n * kk, 2.0 * (double)a.n * a.k * sizeof(double2),
           a.count ? 0 : a.nsys, a.count);
  LY_CUDA(cudaGetLastError());
  return LYAP_OK;
}
