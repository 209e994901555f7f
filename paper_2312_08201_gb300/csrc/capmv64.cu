// FP64 capacitance matvec: the "plain FP64" operator and the residual of the
// mixed path (see capmv.cuh for the algebra).
//
// GB300 runs FP64 at about 1/1800 of its BF16 tensor rate, so this kernel
// is bound by the FP64 FMA pipe: a register-blocked complex GEMM of the
// Cauchy matrix (generated tile by tile from lambda, never stored) with the
// panel W_p o Vb_t (generated on load), 64 x 64 output tile per CTA,
// 4 x 4 complex accumulators per thread, and an epilogue that reduces over
// p inside the tile.
#include "capmv.cuh"
#include "cplx.cuh"
#include "lyap_internal.h"
#include "prof.h"

#include <mutex>

namespace {

constexpr int TI = 64;   // rows per tile
constexpr int TNC = 64;  // panel columns per tile (whole systems: SB * k^2)
constexpr int TJ = 16;   // K step
constexpr int SROW = TNC + 1;

__global__ void __launch_bounds__(256) k_capmv64(CapArgs64 a) {
  extern __shared__ double2 smem[];
  double2* sA = smem;            // [TJ][TI]
  double2* sB = smem + TJ * TI;  // [TJ][TNC]
  const int n = a.n, k = a.k, kk = k * k;
  const int SB = TNC / kk;  // systems per tile (>= 1 since k <= 8)
  const int ncols = SB * kk;
  const int nsys = a.count ? *a.count : a.nsys;
  const int s0 = blockIdx.y * SB;
  if (s0 >= nsys) return;
  const int i0 = blockIdx.x * TI;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;

  // per-column source (system pointer, p, t) for the panel loads
  double2 acc[4][4];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[r][c] = make_double2(0.0, 0.0);

  for (int j0 = 0; j0 < n; j0 += TJ) {
    // Lc tile: sA[jj][ii] = 1/(lam_i + lam_j)
#pragma unroll
    for (int q = 0; q < (TJ * TI) / 256; ++q) {
      int e = tid + 256 * q;
      int jj = e / TI, ii = e % TI;
      int i = i0 + ii, j = j0 + jj;
      double2 v = make_double2(0.0, 0.0);
      if (i < n && j < n) v = crcp(cadd(a.lam[i], a.lam[j]));
      sA[jj * TI + ii] = v;
    }
    // panel tile: sB[jj][cc] = W_b[j, p] * P2[j, t]
#pragma unroll
    for (int q = 0; q < (TJ * TNC) / 256; ++q) {
      int e = tid + 256 * q;
      int jj = e / TNC, cc = e % TNC;
      int j = j0 + jj;
      double2 v = make_double2(0.0, 0.0);
      int sl = cc / kk;
      if (cc < ncols && j < n && s0 + sl < nsys) {
        int pt = cc % kk, p = pt / k, t = pt % k;
        int b = a.list ? a.list[s0 + sl] : s0 + sl;
        v = cmul(a.W[(size_t)b * a.ldw + (size_t)p * n + j], a.P2[(size_t)t * n + j]);
      }
      sB[jj * TNC + cc] = v;
    }
    __syncthreads();
#pragma unroll 4
    for (int jj = 0; jj < TJ; ++jj) {
      double2 av[4], bv[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) av[r] = sA[jj * TI + ty + 16 * r];
#pragma unroll
      for (int c = 0; c < 4; ++c) bv[c] = sB[jj * TNC + tx + 16 * c];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c] = cfma(av[r], bv[c], acc[r][c]);
    }
    __syncthreads();
  }

  // stage the accumulator tile: S[ii][cc]
  double2* S = smem;
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) S[(ty + 16 * r) * SROW + tx + 16 * c] = acc[r][c];
  __syncthreads();

  // epilogue: out_b[i, t] = sum_p P1[i,p] S[i,(sl,p,t)] + sum_p W_b[i,p] Gd(i,p,t), then the mode
  const int nout = TI * SB * k;
  for (int e = tid; e < nout; e += 256) {
    int ii = e % TI, rest = e / TI;
    int t = rest % k, sl = rest / k;
    int i = i0 + ii;
    if (i >= n || s0 + sl >= nsys) continue;
    int b = a.list ? a.list[s0 + sl] : s0 + sl;
    const double2* Wb = a.W + (size_t)b * a.ldw;
    double2 o = make_double2(0.0, 0.0);
    for (int p = 0; p < k; ++p) {
      o = cfma(a.P1[(size_t)p * n + i], S[ii * SROW + (sl * k + p) * k + t], o);
      size_t gidx = a.gT ? ((size_t)(t * k + p) * n + i) : ((size_t)(p * k + t) * n + i);
      o = cfma(Wb[(size_t)p * n + i], a.Gd[gidx], o);
    }
    double2 y = o;
    if (a.mode != CAP_C0) {
      double2 wt = Wb[(size_t)t * n + i];
      y = csub(cscale(wt, a.vinv[(size_t)b * k + t]), o);
      if (a.mode == CAP_RESID) y = csub(a.rhs[(size_t)b * a.ldr + (size_t)t * n + i], y);
    }
    a.out[(size_t)b * a.ldo + (size_t)t * n + i] = y;
  }
}

}  // namespace

int capmv64_launch(const CapArgs64& a, cudaStream_t st) {
  if (a.k < 1 || a.k > 8) return LYAP_EINVAL;
  if (a.nsys <= 0) return LYAP_OK;
  const int kk = a.k * a.k;
  const int SB = TNC / kk;
  const size_t smem = (size_t)TI * SROW * sizeof(double2);  // >= operand tiles
  LY_TRY(lyap_smem_optin(reinterpret_cast<const void*>(k_capmv64), smem));
  dim3 grid((a.n + TI - 1) / TI, (a.nsys + SB - 1) / SB);
  // algorithmic work per system: the Cauchy-panel product, 8 flops per
  // complex MAC over n^2 k^2 MACs, plus the O(n k^2) epilogue
  const int ph = prof_begin(PK_CAPMV64, st);
  k_capmv64<<<grid, 256, smem, st>>>(a);
  lyap_count_launch();
  prof_end(ph, st, 8.0 * (double)a.n * a.n * kk + 16.0 * (double)a.n * kk,
           2.0 * (double)a.n * a.k * sizeof(double2), a.count ? 0 : a.nsys, a.count);
  LY_CUDA(cudaGetLastError());
  return LYAP_OK;
}
