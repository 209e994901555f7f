// Mixed-precision path (an addition to the paper's FP64 method of §2.1):
//  * inner operator T~(v) in FP32 with the Cauchy-panel product on tcgen05
//    tensor cores. The complex product Lc Z is one real GEMM with
//      A[2i][2j] = Re Lc_ij, A[2i][2j+1] = -Im Lc_ij,
//      A[2i+1][2j] = Im Lc_ij, A[2i+1][2j+1] = Re Lc_ij,
//      B[col][2j] = Re Z_j,  B[col][2j+1] = Im Z_j,
//    so D[col][2i], D[col][2i+1] are the real and imaginary parts of (Lc Z)_i.
//    A and B are split into two BF16 terms each (x = hi + lo) and the GEMM
//    accumulates hi*hi + hi*lo + lo*hi in FP32 (about 16 significant bits);
//  * FP32 recycled Krylov inner solves (same batched GCRO-DR, float vectors,
//    FP64 small matrices);
//  * iterative refinement on the capacitance residual r = P - T(v) W,
//    evaluated to FP64 accuracy (integer-sliced product on the BF16 tensor
//    cores, float-float kernel on the FP32 pipes, or the FP64 kernel),
//    W += ||r|| * solve(T~, r/||r||), until
//    ||r|| <= refine_tol ||P||. The trace and the update stay in FP64.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <memory>

#include "cplx.cuh"
#include "krylov.cuh"
#include "mixed.h"
#include "prof.h"
#include "oz_gemm.cuh"
#include "tc_gemm.cuh"
#include "lyap_testing.h"

struct MixedState {
  int mpad = 0, kpad = 0;
  // Layout of the Cauchy products. rs = 2: the complex matrix in real-split
  // form (rows / K entries 2i, 2i+1 = Re, Im of index i), one panel column
  // per (system, p, t). rs = 1 (exactly real eigen-data): the real n x n
  // matrix, and cm = 2 panel columns per (system, p, t), its real and
  // imaginary parts; half the tensor work of the split form.
  int rs = 2, cm = 1;
  DevBuf<__nv_bfloat16> Ahi, Alo;  // mpad x kpad
  DevBuf<float2> Ub32, Vb32, Gd32;
  int ncap = 0;
  DevBuf<__nv_bfloat16> Bhi, Blo;  // ncap x kpad
  DevBuf<float> D;                 // ncap x mpad
  tc::Maps maps;
  DevBuf<int> err;
  bool inject_wait = false;  // LYAP_INJECT_DEVICE_WAIT for the call in progress
  double h_norm = -1.0;      // ||h||, the adjoint right-hand side's norm (set on first use)
  // refinement work
  int bcap = 0;
  DevBuf<double2> R64;
  DevBuf<float2> R32;
  DevBuf<double> norms, vinv_c;
  DevBuf<int> act, cnt;
  DevBuf<float2> wcinv, wpart, wcinv_full;
  WoodState wood;
  // float-float residual operands (capmv_df.cu)
  DevBuf<float4> Lff;  // n x n
  double lc_scale = 1.0, p_scale = 1.0;
  DevBuf<double> sw;   // bcap
  DevBuf<float4> panel_ff;  // bcap x k^2 n
  // integer-sliced tensor-core residual (oz_gemm.cu; K in chunks above 2n = 2046)
  bool oz_ok = false;
  DevBuf<__nv_bfloat16> ozA;  // NS x mpad x kpad digits of the Cauchy matrix
  DevBuf<int> ozEA;           // mpad
  CUtensorMap ozMapA;
  DevBuf<__nv_bfloat16> ozB;  // NS x ncap x kpad digits of the panel
  DevBuf<int> ozEB;           // ncap
  DevBuf<float2> ozD;         // ncap x mpad
  oz::Panel ozPanel;
};

namespace {

__global__ void k_build_A(int n, const double2* __restrict__ lam, int mpad, int kpad, int rs,
                          __nv_bfloat16* __restrict__ Ah, __nv_bfloat16* __restrict__ Al) {
  const size_t total = (size_t)mpad * kpad;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
    const int r = (int)(idx / kpad), c = (int)(idx % kpad);
    const int i = r / rs, j = c / rs;
    double v = 0.0;
    if (i < n && j < n) {
      double2 L = crcp(cadd(lam[i], lam[j]));
      if (rs == 1) v = L.x;
      else if ((r & 1) == 0) v = (c & 1) == 0 ? L.x : -L.y;
      else v = (c & 1) == 0 ? L.y : L.x;
    }
    __nv_bfloat16 hi = __float2bfloat16_rn((float)v);
    __nv_bfloat16 lo = __float2bfloat16_rn((float)(v - (double)__bfloat162float(hi)));
    Ah[idx] = hi;
    Al[idx] = lo;
  }
}

__global__ void k_to_f32(size_t count, const double2* __restrict__ in, float2* __restrict__ out) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x)
    out[i] = make_float2((float)in[i].x, (float)in[i].y);
}

// Panel columns col = slot*k^2 + p*k + t: Z[j] = W_slot[j, p] * P2[j, t],
// stored split (hi, lo); rs = 2: real-split along K (2j, 2j+1) in column
// col; rs = 1: Re Z in column 2 col and Im Z in column 2 col + 1.
template <typename T2>
__global__ void k_panel(int n, int k, const int* __restrict__ list, const int* __restrict__ count, int nsys,
                        const T2* __restrict__ In, size_t in_ss, const float2* __restrict__ P2, int kpad, int rs,
                        __nv_bfloat16* __restrict__ Bh, __nv_bfloat16* __restrict__ Bl) {
  const int slot = blockIdx.y;
  const int ns = count ? *count : nsys;
  if (slot >= ns) return;
  const int b = list ? list[slot] : slot;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const int kk = k * k;
  for (int p = 0; p < k; ++p) {
    const double2 w = to_d2(In[(size_t)b * in_ss + (size_t)p * n + j]);
    const float2 wf = make_float2((float)w.x, (float)w.y);
    for (int t = 0; t < k; ++t) {
      const float2 z = cmul(wf, P2[(size_t)t * n + j]);
      const size_t col = (size_t)(slot * kk + p * k + t);
      const size_t o = rs == 2 ? col * kpad + 2 * j : 2 * col * kpad + j;  // Re of z
      const size_t oi = rs == 2 ? o + 1 : o + kpad;                         // Im of z
      const __nv_bfloat16 hr = __float2bfloat16_rn(z.x), hi = __float2bfloat16_rn(z.y);
      Bh[o] = hr;
      Bh[oi] = hi;
      Bl[o] = __float2bfloat16_rn(z.x - __bfloat162float(hr));
      Bl[oi] = __float2bfloat16_rn(z.y - __bfloat162float(hi));
    }
  }
}

// out[i, t] = sum_p P1[i,p] (Lc Z)[i, (slot,p,t)] + sum_p W[i,p] Gd(i,p,t); then T or C0.
template <typename T2>
__global__ void k_epi(int n, int k, const int* __restrict__ list, const int* __restrict__ count, int nsys,
                      const float* __restrict__ D, int ldd, int rs, const T2* __restrict__ In, size_t in_ss,
                      const float2* __restrict__ P1, const float2* __restrict__ Gd, int gT,
                      const double* __restrict__ vinv, int mode, T2* __restrict__ Out, size_t out_ss) {
  const int slot = blockIdx.y;
  const int ns = count ? *count : nsys;
  if (slot >= ns) return;
  const int b = list ? list[slot] : slot;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int kk = k * k;
  const float2* D2 = reinterpret_cast<const float2*>(D);
  const int ld2 = ldd / 2;
  float2 w[8];
  for (int p = 0; p < k; ++p) w[p] = to_f2(In[(size_t)b * in_ss + (size_t)p * n + i]);
  for (int t = 0; t < k; ++t) {
    float2 o = make_float2(0.f, 0.f);
    for (int p = 0; p < k; ++p) {
      const size_t col = (size_t)(slot * kk + p * k + t);
      const float2 lz = rs == 2 ? D2[col * ld2 + i] : make_float2(D[2 * col * ldd + i], D[(2 * col + 1) * ldd + i]);
      o = cfma(P1[(size_t)p * n + i], lz, o);
      const size_t g = gT ? ((size_t)(t * k + p) * n + i) : ((size_t)(p * k + t) * n + i);
      o = cfma(w[p], Gd[g], o);
    }
    float2 y = o;
    if (mode == CAP_T) y = csub(cscale(w[t], (float)vinv[(size_t)b * k + t]), o);
    Out[(size_t)b * out_ss + (size_t)t * n + i] = from_f2<T2>(y);
  }
}

__global__ void k_gather_r32(int N, int k, const int* __restrict__ act, int nact, const double2* __restrict__ R64,
                             const double* __restrict__ norms, const double* __restrict__ vinv, float2* __restrict__ R32,
                             double* __restrict__ vinv_c) {
  const int c = blockIdx.y;
  if (c >= nact) return;
  const int b = act[c];
  const double s = norms[b] > 0 ? 1.0 / norms[b] : 0.0;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < N; e += gridDim.x * blockDim.x) {
    const double2 r = R64[(size_t)b * N + e];
    R32[(size_t)c * N + e] = make_float2((float)(r.x * s), (float)(r.y * s));
  }
  if (blockIdx.x == 0 && threadIdx.x < k) vinv_c[(size_t)c * k + threadIdx.x] = vinv[(size_t)b * k + threadIdx.x];
}

__global__ void k_scatter_add(int N, const int* __restrict__ act, int nact, const float2* __restrict__ X32,
                              const double* __restrict__ norms, double2* __restrict__ W) {
  const int c = blockIdx.y;
  if (c >= nact) return;
  const int b = act[c];
  const double s = norms[b];
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < N; e += gridDim.x * blockDim.x) {
    const float2 x = X32[(size_t)c * N + e];
    double2 w = W[(size_t)b * N + e];
    w.x += s * (double)x.x;
    w.y += s * (double)x.y;
    W[(size_t)b * N + e] = w;
  }
}

template <typename T2>
__global__ void k_fill_shared(int nsys, size_t N, const double2* __restrict__ src, T2* __restrict__ dst) {
  const int b = blockIdx.y;
  if (b >= nsys) return;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < N; e += (size_t)gridDim.x * blockDim.x)
    dst[(size_t)b * N + e] = from_d2<T2>(src[e]);
}

int gx(size_t N) { return (int)std::max<size_t>(1, std::min<size_t>((N + 255) / 256, 64)); }

int ensure_cols(lyap_seed* sd, int ncols, cudaStream_t st) {
  MixedState& ms = *sd->mixed;
  if (ncols <= ms.ncap) return LYAP_OK;
  const int cap = ((ncols + tc::BN - 1) / tc::BN) * tc::BN;
  LY_TRY(ms.Bhi.alloc((size_t)cap * ms.kpad));
  LY_TRY(ms.Blo.alloc((size_t)cap * ms.kpad));
  LY_TRY(ms.D.alloc((size_t)cap * ms.mpad));
  // on the solve's own stream: a memset on the legacy default stream is not
  // ordered with the context's non-blocking stream and could land after the
  // panel or the product it is meant to precede
  LY_CUDA(cudaMemsetAsync(ms.D.p, 0, ms.D.bytes(), st));      // defined even where a timed-out GEMM wrote nothing
  LY_CUDA(cudaMemsetAsync(ms.Bhi.p, 0, ms.Bhi.bytes(), st));  // K padding stays zero
  LY_CUDA(cudaMemsetAsync(ms.Blo.p, 0, ms.Blo.bytes(), st));
  LY_TRY(tc::make_map(&ms.maps.b_hi, ms.Bhi.p, cap, ms.kpad, tc::BN));
  LY_TRY(tc::make_map(&ms.maps.b_lo, ms.Blo.p, cap, ms.kpad, tc::BN));
  ms.ncap = cap;
  return LYAP_OK;
}

template <typename T2>
int mixed_apply(lyap_seed* sd, bool adjoint, const double* vinv, const int* list, const int* count, int nsys,
                const T2* In, size_t in_ss, T2* Out, size_t out_ss, int mode, cudaStream_t st) {
  MixedState& ms = *sd->mixed;
  const int n = sd->n, k = sd->k, kk = k * k;
  LY_TRY(ensure_cols(sd, nsys * kk * ms.cm, st));
  const float2* P1 = adjoint ? ms.Vb32.p : ms.Ub32.p;
  const float2* P2 = adjoint ? ms.Ub32.p : ms.Vb32.p;
  dim3 g((n + 255) / 256, nsys);
  const int pp = prof_begin(PK_PANEL, st);
  k_panel<T2><<<g, 256, 0, st>>>(n, k, list, count, nsys, In, in_ss, P2, ms.kpad, ms.rs, ms.Bhi.p, ms.Blo.p);
  lyap_count_launch();
  prof_end(pp, st, 0.0, (double)n * k * sizeof(T2) + 8.0 * n * kk, count ? 0 : nsys, count);
  LY_CUDA(cudaGetLastError());
  // tensor work per system: 2 (real) x (rs n)^2 x cm k^2 MACs per product, three products
  const int ph = prof_begin(PK_TCGEMM, st);
  const int cols = kk * ms.cm;
  LY_TRY(tc::launch(ms.maps, ms.D.p, ms.mpad, ms.rs * n, ms.mpad, ms.kpad, count, cols, nsys * cols, nsys * cols,
                    ms.err.p, st, ms.inject_wait));
  prof_end(ph, st, 3.0 * 2.0 * (double)(ms.rs * n) * (ms.rs * n) * cols, 0.0, count ? 0 : nsys, count);
  const int pe = prof_begin(PK_EPI32, st);
  k_epi<T2><<<g, 256, 0, st>>>(n, k, list, count, nsys, ms.D.p, ms.mpad, ms.rs, In, in_ss, P1, ms.Gd32.p, adjoint ? 1 : 0,
                               vinv, mode, Out, out_ss);
  lyap_count_launch();
  prof_end(pe, st, 0.0, (double)kk * n * 8.0 + 4.0 * n * k * sizeof(T2), count ? 0 : nsys, count);
  LY_CUDA(cudaGetLastError());
  return LYAP_OK;
}

int ensure_refine(lyap_seed* sd, int Bc) {
  MixedState& ms = *sd->mixed;
  if (Bc <= ms.bcap) return LYAP_OK;
  const size_t N = (size_t)sd->n * sd->k;
  LY_TRY(ms.R64.alloc((size_t)Bc * N));
  LY_TRY(ms.R32.alloc((size_t)Bc * N));
  LY_TRY(ms.norms.alloc(Bc));
  LY_TRY(ms.vinv_c.alloc((size_t)Bc * sd->k));
  LY_TRY(ms.act.alloc(Bc));
  LY_TRY(ms.cnt.alloc(1));
  LY_TRY(ms.sw.alloc(Bc));
  LY_TRY(ms.panel_ff.alloc((size_t)Bc * sd->k * sd->k * sd->n));
  if (ms.oz_ok) {
    const int ncap = ((Bc * sd->k * sd->k * ms.cm + oz::BN - 1) / oz::BN) * oz::BN;
    LY_TRY(ms.ozB.alloc((size_t)oz::NS * ncap * ms.kpad));
    LY_TRY(ms.ozEB.alloc(ncap));
    LY_TRY(ms.ozD.alloc((size_t)ncap * ms.mpad));
    LY_TRY(oz::make_map(&ms.ozPanel.mapB, ms.ozB.p, oz::NS * ncap, ms.kpad, oz::BN));
    ms.ozPanel.S = ms.ozB.p;
    ms.ozPanel.eB = ms.ozEB.p;
    ms.ozPanel.D = ms.ozD.p;
    ms.ozPanel.ncap = ncap;
  }
  ms.bcap = Bc;
  return LYAP_OK;
}

// Refinement for one right-hand side (shared by all systems): W (Bc x N FP64).
int refine(lyap_seed* sd, int Bc, const double* vinv, const double2* rhs, double rhs_norm, bool adjoint,
           Recycle<float2>& rec, const lyap_opts& o, const SolveParams& prm, cudaStream_t st, KrylovWS<float2>& ws,
           double2* W, std::vector<int>& iters, std::vector<int>& status, std::vector<int>& rsteps) {
  MixedState& ms = *sd->mixed;
  const int n = sd->n, k = sd->k;
  const int N = n * k;
  LY_TRY(ensure_refine(sd, Bc));
  LY_CUDA(cudaMemsetAsync(W, 0, sizeof(double2) * (size_t)Bc * N, st));
  std::vector<int> act(Bc);
  for (int b = 0; b < Bc; ++b) act[b] = b;
  std::vector<double> nrm(Bc, rhs_norm);
  SolveParams pin = prm;
  pin.tol = o.inner_tol;
  const int max_refine = std::max(1, o.max_refine);
  std::vector<int> it, stt;
  for (int step = 0;; ++step) {
    const int nact = (int)act.size();
    LY_CUDA(cudaMemcpyAsync(ms.act.p, act.data(), sizeof(int) * nact, cudaMemcpyHostToDevice, st));
    LY_CUDA(cudaMemcpyAsync(ms.cnt.p, &nact, sizeof(int), cudaMemcpyHostToDevice, st));
    if (step == 0) {
      k_fill_shared<double2><<<dim3(gx(N), Bc), 256, 0, st>>>(Bc, N, rhs, ms.R64.p);
      lyap_count_launch();
      LY_CUDA(cudaMemcpyAsync(ms.norms.p, nrm.data(), sizeof(double) * Bc, cudaMemcpyHostToDevice, st));
    } else {
      CapArgs64 a{};
      a.n = n;
      a.k = k;
      a.lam = sd->lam.p;
      a.P1 = adjoint ? sd->Vb.p : sd->Ub.p;
      a.P2 = adjoint ? sd->Ub.p : sd->Vb.p;
      a.Gd = sd->Gd.p;
      a.gT = adjoint ? 1 : 0;
      a.W = W;
      a.ldw = N;
      a.vinv = vinv;
      a.rhs = rhs;
      a.ldr = 0;
      a.out = ms.R64.p;
      a.ldo = N;
      a.mode = CAP_RESID;
      a.list = ms.act.p;
      a.count = ms.cnt.p;
      a.nsys = nact;
      if (o.residual == LYAP_RESID_FP64) LY_TRY(capmv64_launch(a, st));
      else if (o.residual == LYAP_RESID_TC && ms.oz_ok)
        LY_TRY(oz::residual(a, ms.ozMapA, ms.ozEA.p, ms.mpad, ms.kpad, ms.rs, ms.ozPanel, ms.err.p, st));
      else LY_TRY(capmv_df_launch(a, ms.Lff.p, ms.lc_scale, ms.p_scale, ms.sw.p, ms.panel_ff.p, st));
      kry::k_norms<double2><<<Bc, kry::NT, 0, st>>>(N, Bc, ms.R64.p, N, ms.norms.p);
      lyap_count_launch();
      LY_CUDA(cudaGetLastError());
      LY_CUDA(cudaMemcpyAsync(nrm.data(), ms.norms.p, sizeof(double) * Bc, cudaMemcpyDeviceToHost, st));
      int herr_step = 0;
      LY_CUDA(cudaMemcpyAsync(&herr_step, ms.err.p, sizeof(int), cudaMemcpyDeviceToHost, st));
      LY_CUDA(cudaStreamSynchronize(st));
      if (herr_step) {
        // a bounded wait of a tensor-core kernel ran out: stop at the first sync
        lyap_set_last_error("tensor-core GEMM wait timed out (code " + std::to_string(herr_step) + ")");
        LY_CUDA(cudaMemsetAsync(ms.err.p, 0, sizeof(int), st));
        return LYAP_EDEVICE_TIMEOUT;
      }
      std::vector<int> keep;
      for (int b : act) {
        rsteps[b] = step;
        const double rel = rhs_norm > 0 ? nrm[b] / rhs_norm : nrm[b];
        if (!std::isfinite(rel)) status[b] = LYAP_ENONFINITE;
        else if (rel <= o.refine_tol) status[b] = LYAP_OK;
        else if (step >= max_refine) status[b] = LYAP_ENOCONV;
        else keep.push_back(b);
      }
      act.swap(keep);
      if (act.empty()) break;
      const int na = (int)act.size();
      LY_CUDA(cudaMemcpyAsync(ms.act.p, act.data(), sizeof(int) * na, cudaMemcpyHostToDevice, st));
    }
    const int na = (int)act.size();
    k_gather_r32<<<dim3(gx(N), na), 256, 0, st>>>(N, k, ms.act.p, na, ms.R64.p, ms.norms.p, vinv, ms.R32.p,
                                                  ms.vinv_c.p);
    lyap_count_launch();
    LY_CUDA(cudaGetLastError());
    SysOp<float2> op;
    op.sd = sd;
    op.adjoint = adjoint;
    op.vinv = ms.vinv_c.p;
    if (o.pbar > 0 && sd->tsvd_r > 0) {
      const int r = std::min(o.pbar, sd->tsvd_r);
      if (ms.wcinv.count < (size_t)na * r * r) LY_TRY(ms.wcinv.alloc((size_t)Bc * r * r));
      if (ms.wpart.count < wood_part_count(sd->n, k, na, r)) LY_TRY(ms.wpart.alloc(wood_part_count(sd->n, k, Bc, r)));
      ms.wood.cinv = ms.wcinv.p;
      ms.wood.cpart = ms.wpart.p;
      ms.wood.err = ms.err.p;
      // Cap(v)^{-1} of every chunk system was built once by lyap_mixed_chunk
      LY_TRY(wood_bind(sd, r, na, ms.wcinv_full.p, ms.act.p, ms.wood, st));
      op.wood = &ms.wood;
    }
    LY_TRY(gcrodr_chunk<float2>(op, na, ms.R32.p, (size_t)N, rec, pin, ws, it, stt, st));
    k_scatter_add<<<dim3(gx(N), na), 256, 0, st>>>(N, ms.act.p, na, ws.X.p, ms.norms.p, W);
    lyap_count_launch();
    LY_CUDA(cudaGetLastError());
    for (int c = 0; c < na; ++c) iters[act[c]] += it[c];
  }
  int herr = 0;
  LY_CUDA(cudaMemcpyAsync(&herr, ms.err.p, sizeof(int), cudaMemcpyDeviceToHost, st));
  LY_CUDA(cudaStreamSynchronize(st));
  if (herr) {
    lyap_set_last_error("tensor-core GEMM wait timed out (code " + std::to_string(herr) + ")");
    LY_CUDA(cudaMemsetAsync(ms.err.p, 0, sizeof(int), st));
    return LYAP_EDEVICE_TIMEOUT;
  }
  return LYAP_OK;
}

}  // namespace

void lyap_mixed_free(lyap_seed* sd) {
  delete sd->mixed;
  sd->mixed = nullptr;
}

int lyap_mixed_prepare(lyap_seed* sd, cudaStream_t st) {
  std::unique_ptr<MixedState> ms(new MixedState());
  const int n = sd->n, k = sd->k;
  ms->rs = sd->real_arith ? 1 : 2;
  ms->cm = sd->real_arith ? 2 : 1;
  ms->mpad = ((ms->rs * n + tc::BM - 1) / tc::BM) * tc::BM;
  ms->kpad = ((ms->rs * n + tc::BK - 1) / tc::BK) * tc::BK;
  LY_TRY(ms->Ahi.alloc((size_t)ms->mpad * ms->kpad));
  LY_TRY(ms->Alo.alloc((size_t)ms->mpad * ms->kpad));
  k_build_A<<<gx((size_t)ms->mpad * ms->kpad) * 16, 256, 0, st>>>(n, sd->lam.p, ms->mpad, ms->kpad, ms->rs, ms->Ahi.p,
                                                                  ms->Alo.p);
  lyap_count_launch();
  LY_CUDA(cudaGetLastError());
  LY_TRY(ms->Ub32.alloc((size_t)n * k));
  LY_TRY(ms->Vb32.alloc((size_t)n * k));
  LY_TRY(ms->Gd32.alloc((size_t)n * k * k));
  k_to_f32<<<gx((size_t)n * k), 256, 0, st>>>((size_t)n * k, sd->Ub.p, ms->Ub32.p);
  k_to_f32<<<gx((size_t)n * k), 256, 0, st>>>((size_t)n * k, sd->Vb.p, ms->Vb32.p);
  k_to_f32<<<gx((size_t)n * k * k), 256, 0, st>>>((size_t)n * k * k, sd->Gd.p, ms->Gd32.p);
  lyap_count_launch(3);
  LY_CUDA(cudaGetLastError());
  {
    // power-of-two scales that bring Lc and Ub/Vb to magnitudes near 1 for the
    // float-float residual (max |Lc| = 1 / min |lam_i + lam_j|)
    std::vector<double2> hu((size_t)n * k), hv((size_t)n * k);
    LY_CUDA(cudaMemcpyAsync(hu.data(), sd->Ub.p, sizeof(double2) * hu.size(), cudaMemcpyDeviceToHost, st));
    LY_CUDA(cudaMemcpyAsync(hv.data(), sd->Vb.p, sizeof(double2) * hv.size(), cudaMemcpyDeviceToHost, st));
    LY_CUDA(cudaStreamSynchronize(st));
    double pm = 0.0;
    for (size_t e = 0; e < hu.size(); ++e)
      pm = std::max({pm, std::fabs(hu[e].x), std::fabs(hu[e].y), std::fabs(hv[e].x), std::fabs(hv[e].y)});
    const auto pow2_inv = [](double m) {
      const int e = (m > 0.0 && std::isfinite(m)) ? std::max(-600, std::min(600, std::ilogb(m))) : 0;
      return std::ldexp(1.0, -e);
    };
    ms->p_scale = pow2_inv(pm);
    ms->lc_scale = pow2_inv(sd->min_sum > 0.0 ? 1.0 / sd->min_sum : 1.0);
    LY_TRY(ms->Lff.alloc((size_t)n * n));
    LY_TRY(capmv_df_build_lc(n, sd->lam.p, ms->lc_scale, ms->Lff.p, st));
  }
  {
    LY_TRY(ms->ozA.alloc((size_t)oz::NS * ms->mpad * ms->kpad));
    LY_TRY(ms->ozEA.alloc(ms->mpad));
    LY_TRY(oz::slice_A(n, sd->lam.p, ms->mpad, ms->kpad, ms->rs, ms->ozA.p, ms->ozEA.p, st));
    LY_TRY(oz::make_map(&ms->ozMapA, ms->ozA.p, oz::NS * ms->mpad, ms->kpad, oz::BM));
    ms->oz_ok = true;
  }
  LY_TRY(tc::make_map(&ms->maps.a_hi, ms->Ahi.p, ms->mpad, ms->kpad, tc::BM));
  LY_TRY(tc::make_map(&ms->maps.a_lo, ms->Alo.p, ms->mpad, ms->kpad, tc::BM));
  LY_TRY(ms->err.alloc(1));
  LY_CUDA(cudaMemsetAsync(ms->err.p, 0, sizeof(int), st));
  LY_CUDA(cudaStreamSynchronize(st));
  sd->resident_bytes += ms->Ahi.bytes() + ms->Alo.bytes() + ms->Ub32.bytes() + ms->Vb32.bytes() + ms->Gd32.bytes() +
                        ms->Lff.bytes() + ms->ozA.bytes() + ms->ozEA.bytes();
  sd->mixed = ms.release();
  return LYAP_OK;
}

// After a device timeout the FP32 recycle spaces may hold vectors built with
// an incomplete operator: wait for the work in flight and forget them, so the
// next call starts its recycling afresh.
static void drop_recycle(lyap_seed* sd, KrylovWS<float2>& ws, cudaStream_t st) {
  cudaStreamSynchronize(st);
  if (ws.side) cudaStreamSynchronize(ws.side);
  for (Recycle<float2>* r : {&sd->rec32, &sd->rec32_adj}) {
    r->pending = false;
    r->s = 0;
    r->c0_valid = false;
  }
}

int lyap_mixed_chunk(lyap_seed* sd, int Bc, const double* vinv, const lyap_opts& o, const SolveParams& prm,
                     cudaStream_t st, KrylovWS<float2>& ws, KrylovWS<float2>& wsadj, double2* Wp_out,
                     double2* Zadj_out, double2* Rres_out, std::vector<int>& iters, std::vector<int>& status,
                     std::vector<int>& rsteps) {
  if (!sd->mixed) return LYAP_EINVAL;
  iters.assign(Bc, 0);
  status.assign(Bc, LYAP_OK);
  rsteps.assign(Bc, 0);
  MixedState& ms = *sd->mixed;
  ms.inject_wait = (o.inject & LYAP_INJECT_DEVICE_WAIT) != 0;
  struct ClearInject {
    MixedState& m;
    ~ClearInject() { m.inject_wait = false; }
  } clear_inject{ms};
  if (o.pbar > 0 && sd->tsvd_r > 0) {
    // Cap(v_b)^{-1} for the whole chunk, shared by every refinement step and
    // by the adjoint solves (which apply its transpose)
    const int r = std::min(o.pbar, sd->tsvd_r);
    if (ms.wcinv_full.count < (size_t)Bc * r * r) LY_TRY(ms.wcinv_full.alloc((size_t)Bc * r * r));
    WoodState full;
    full.cinv = ms.wcinv_full.p;
    LY_TRY(wood_prepare(sd, r, Bc, vinv, false, full, st));
  }
  {
    const int rc = refine(sd, Bc, vinv, sd->Ph.p, sd->ph_norm, false, sd->rec32, o, prm, st, ws, Wp_out, iters, status,
                          rsteps);
    if (rc == LYAP_EDEVICE_TIMEOUT) drop_recycle(sd, ws, st);
    if (rc != LYAP_OK) return rc;
  }
  // every system's final residual was evaluated (and kept) by its last refinement step
  if (Rres_out)
    LY_CUDA(cudaMemcpyAsync(Rres_out, sd->mixed->R64.p, sizeof(double2) * (size_t)Bc * sd->n * sd->k,
                            cudaMemcpyDeviceToDevice, st));
  if (Zadj_out) {
    double hn = 0;
    {
      // ||h|| once per seed (a v-independent scalar)
      if (ms.h_norm < 0) {
        kry::k_norms<double2><<<1, kry::NT, 0, st>>>(sd->n * sd->k, 1, sd->h.p, 0, ms.norms.p);
        lyap_count_launch();
        LY_CUDA(cudaMemcpyAsync(&ms.h_norm, ms.norms.p, sizeof(double), cudaMemcpyDeviceToHost, st));
        LY_CUDA(cudaStreamSynchronize(st));
      }
      hn = ms.h_norm;
    }
    std::vector<int> ita(Bc, 0), sta(Bc, LYAP_OK), rsa(Bc, 0);
    {
      const int rc = refine(sd, Bc, vinv, sd->h.p, hn, true, sd->rec32_adj, o, prm, st, wsadj, Zadj_out, ita, sta, rsa);
      if (rc == LYAP_EDEVICE_TIMEOUT) drop_recycle(sd, wsadj, st);
      if (rc != LYAP_OK) return rc;
    }
    for (int b = 0; b < Bc; ++b) {
      iters[b] += ita[b];
      rsteps[b] += rsa[b];
      if (status[b] == LYAP_OK) status[b] = sta[b];
    }
  }
  return LYAP_OK;
}

// ------------------------------------------- continuous-batching engine
namespace {

// new systems: vinv_c[c] = 1 / v[c] (compact), vinv[slot] = vinv_c[c], W[slot] = 0
__global__ void k_engine_join(int nj, int k, size_t N, const int* __restrict__ slots, const double* __restrict__ v,
                              double* __restrict__ vinv_c, double* __restrict__ vinv, double2* __restrict__ W) {
  const int c = blockIdx.y;
  if (c >= nj) return;
  const int s = slots[c];
  if (blockIdx.x == 0 && threadIdx.x < k) {
    const double x = 1.0 / v[(size_t)c * k + threadIdx.x];
    vinv_c[(size_t)c * k + threadIdx.x] = x;
    vinv[(size_t)s * k + threadIdx.x] = x;
  }
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < N; e += (size_t)gridDim.x * blockDim.x)
    W[(size_t)s * N + e] = make_double2(0.0, 0.0);
}

// cinv[slot] = staged[c] (r x r per system)
__global__ void k_engine_cinv(int nj, int rr, const int* __restrict__ slots, const float2* __restrict__ staged,
                              float2* __restrict__ cinv) {
  const int c = blockIdx.y;
  if (c >= nj) return;
  for (int e = threadIdx.x; e < rr; e += blockDim.x) cinv[(size_t)slots[c] * rr + e] = staged[(size_t)c * rr + e];
}

// R[slot] = rhs for the listed slots
__global__ void k_engine_fill(size_t N, const int* __restrict__ slots, int ns, const double2* __restrict__ rhs,
                              double2* __restrict__ R) {
  const int c = blockIdx.y;
  if (c >= ns) return;
  const int s = slots[c];
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < N; e += (size_t)gridDim.x * blockDim.x)
    R[(size_t)s * N + e] = rhs[e];
}

// out[c] = ||R[slot_c]|| for the listed slots
__global__ void __launch_bounds__(kry::NT) k_engine_norms(int N, const int* __restrict__ slots, int ns,
                                                          const double2* __restrict__ R, double* __restrict__ out) {
  __shared__ double red[32];
  const int c = blockIdx.x;
  if (c >= ns) return;
  const double2* r = R + (size_t)slots[c] * N;
  double acc[1] = {0.0};
  for (int e = threadIdx.x; e < N; e += kry::NT) acc[0] += cabs2(r[e]);
  kry::block_sum<1>(acc, red);
  if (threadIdx.x == 0) out[c] = sqrt(acc[0]);
}

// f[c] = Re <h, A[slot_c]> for the listed slots
__global__ void __launch_bounds__(kry::NT) k_engine_dot_h(int N, const int* __restrict__ slots, int ns,
                                                          const double2* __restrict__ A, const double2* __restrict__ h,
                                                          double* __restrict__ out) {
  __shared__ double red[32];
  const int c = blockIdx.x;
  if (c >= ns) return;
  const double2* a = A + (size_t)slots[c] * N;
  double acc[1] = {0.0};
  for (int e = threadIdx.x; e < N; e += kry::NT) acc[0] += cmul(a[e], h[e]).x;
  kry::block_sum<1>(acc, red);
  if (threadIdx.x == 0) out[c] = acc[0];
}

}  // namespace

struct MixedEngine {
  int cap = 0, r = 0;
  DevBuf<double2> W;      // cap x N: FP64 solution of every slot
  DevBuf<double> vinv;    // cap x k
  DevBuf<float2> cinv;    // cap x r x r: Cap(v)^{-1} of every slot
  DevBuf<double> vstage, vinv_c, fout, rout, eout;
  DevBuf<float2> cstage, cpart_stage;
  DevBuf<int> slots, slots2;
  DevBuf<double2> delta;  // cap x N: P^{-1} r of retiring slots (error estimate)
  std::vector<int> steps, iters;  // per slot; steps < 0: free
  KrylovWS<float2> ws;
};

int lyap_engine_create(lyap_seed* sd, int cap, const lyap_opts& o, MixedEngine** out) {
  *out = nullptr;
  if (!sd->mixed || cap < 1) return LYAP_EINVAL;
  std::unique_ptr<MixedEngine> e(new MixedEngine());
  const size_t N = (size_t)sd->n * sd->k;
  const int k = sd->k;
  e->cap = cap;
  e->r = (o.pbar > 0 && sd->tsvd_r > 0) ? std::min(o.pbar, sd->tsvd_r) : 0;
  LY_TRY(e->W.alloc((size_t)cap * N));
  LY_TRY(e->vinv.alloc((size_t)cap * k));
  LY_TRY(e->vstage.alloc((size_t)cap * k));
  LY_TRY(e->vinv_c.alloc((size_t)cap * k));
  LY_TRY(e->fout.alloc(cap));
  LY_TRY(e->rout.alloc(cap));
  LY_TRY(e->eout.alloc(cap));
  LY_TRY(e->slots.alloc(cap));
  LY_TRY(e->slots2.alloc(cap));
  LY_TRY(e->delta.alloc((size_t)cap * N));
  if (e->r > 0) {
    LY_TRY(e->cinv.alloc((size_t)cap * e->r * e->r));
    LY_TRY(e->cstage.alloc((size_t)cap * e->r * e->r));
  }
  e->steps.assign(cap, -1);
  e->iters.assign(cap, 0);
  *out = e.release();
  return LYAP_OK;
}

void lyap_engine_free(lyap_seed* sd, MixedEngine* e) {
  if (!e) return;
  // a recycle hand-over still pending on the engine's side stream is
  // resolved before that stream and its event go away
  Recycle<float2>& rec = sd->rec32;
  if (e->ws.side) {
    cudaEventSynchronize(e->ws.side_done);
    if (rec.pending && rec.ready == e->ws.side_done) {
      rec.pending = false;
      if (*rec.ok_host) {
        rec.s = rec.pending_s;
        rec.c0_valid = true;
      }
    }
  }
  delete e;
}

int lyap_engine_free_slots(const MixedEngine* e) {
  int c = 0;
  for (int s : e->steps) c += s < 0 ? 1 : 0;
  return c;
}

// One refinement step of every occupied slot: systems join (fresh W = 0)
// and retire here, so a system waits at most one step to enter the
// lockstep set. Each step is the refinement of lyap_mixed_chunk: the
// FP64-accurate residual, the decision per system, and one recycled FP32
// inner solve for those that go on.
int lyap_engine_step(lyap_seed* sd, MixedEngine& e, const lyap_opts& o, cudaStream_t st,
                     const std::vector<EngineJoin>& joins, std::vector<EngineDone>& done) {
  done.clear();
  MixedState& ms = *sd->mixed;
  const int n = sd->n, k = sd->k;
  const int N = n * k;
  SolveParams prm;
  LY_TRY(lyap_params_from_opts(o, prm));
  SolveParams pin = prm;
  pin.tol = o.inner_tol;
  LY_TRY(ensure_refine(sd, e.cap));
  // ---- joins
  const int nj = (int)joins.size();
  if (nj > 0) {
    std::vector<int> js(nj);
    std::vector<double> vs((size_t)nj * k);
    for (int c = 0; c < nj; ++c) {
      js[c] = joins[c].slot;
      if (e.steps[js[c]] >= 0) return LYAP_EINVAL;
      std::memcpy(vs.data() + (size_t)c * k, joins[c].v, sizeof(double) * k);
    }
    LY_CUDA(cudaMemcpyAsync(e.slots.p, js.data(), sizeof(int) * nj, cudaMemcpyHostToDevice, st));
    LY_CUDA(cudaMemcpyAsync(e.vstage.p, vs.data(), sizeof(double) * vs.size(), cudaMemcpyHostToDevice, st));
    k_engine_join<<<dim3(gx(N), nj), 256, 0, st>>>(nj, k, (size_t)N, e.slots.p, e.vstage.p, e.vinv_c.p, e.vinv.p,
                                                   e.W.p);
    lyap_count_launch();
    LY_CUDA(cudaGetLastError());
    if (e.r > 0) {
      WoodState tmp;
      tmp.cinv = e.cstage.p;
      LY_TRY(wood_prepare(sd, e.r, nj, e.vinv_c.p, false, tmp, st));
      k_engine_cinv<<<dim3(1, nj), 256, 0, st>>>(nj, e.r * e.r, e.slots.p, e.cstage.p, e.cinv.p);
      lyap_count_launch();
      LY_CUDA(cudaGetLastError());
    }
    for (int c = 0; c < nj; ++c) {
      e.steps[js[c]] = 0;
      e.iters[js[c]] = 0;
    }
  }
  // ---- residuals: fresh systems start from r = P, the others are evaluated
  std::vector<int> fresh, old;
  for (int s = 0; s < e.cap; ++s) {
    if (e.steps[s] == 0) fresh.push_back(s);
    else if (e.steps[s] > 0) old.push_back(s);
  }
  if (fresh.empty() && old.empty()) return LYAP_OK;
  std::vector<double> nrm_old(old.size());
  if (!fresh.empty()) {
    LY_CUDA(cudaMemcpyAsync(e.slots2.p, fresh.data(), sizeof(int) * fresh.size(), cudaMemcpyHostToDevice, st));
    k_engine_fill<<<dim3(gx(N), (int)fresh.size()), 256, 0, st>>>((size_t)N, e.slots2.p, (int)fresh.size(),
                                                                   sd->Ph.p, ms.R64.p);
    lyap_count_launch();
  }
  if (!old.empty()) {
    const int no = (int)old.size();
    LY_CUDA(cudaMemcpyAsync(ms.act.p, old.data(), sizeof(int) * no, cudaMemcpyHostToDevice, st));
    LY_CUDA(cudaMemcpyAsync(ms.cnt.p, &no, sizeof(int), cudaMemcpyHostToDevice, st));
    CapArgs64 a{};
    a.n = n;
    a.k = k;
    a.lam = sd->lam.p;
    a.P1 = sd->Ub.p;
    a.P2 = sd->Vb.p;
    a.Gd = sd->Gd.p;
    a.W = e.W.p;
    a.ldw = N;
    a.vinv = e.vinv.p;
    a.rhs = sd->Ph.p;
    a.ldr = 0;
    a.out = ms.R64.p;
    a.ldo = N;
    a.mode = CAP_RESID;
    a.list = ms.act.p;
    a.count = ms.cnt.p;
    a.nsys = no;
    if (o.residual == LYAP_RESID_FP64) LY_TRY(capmv64_launch(a, st));
    else if (o.residual == LYAP_RESID_TC && ms.oz_ok)
      LY_TRY(oz::residual(a, ms.ozMapA, ms.ozEA.p, ms.mpad, ms.kpad, ms.rs, ms.ozPanel, ms.err.p, st));
    else LY_TRY(capmv_df_launch(a, ms.Lff.p, ms.lc_scale, ms.p_scale, ms.sw.p, ms.panel_ff.p, st));
    k_engine_norms<<<no, kry::NT, 0, st>>>(N, ms.act.p, no, ms.R64.p, e.rout.p);
    lyap_count_launch();
    LY_CUDA(cudaGetLastError());
    LY_CUDA(cudaMemcpyAsync(nrm_old.data(), e.rout.p, sizeof(double) * no, cudaMemcpyDeviceToHost, st));
  }
  int herr = 0;
  LY_CUDA(cudaMemcpyAsync(&herr, ms.err.p, sizeof(int), cudaMemcpyDeviceToHost, st));
  LY_CUDA(cudaStreamSynchronize(st));
  if (herr) {
    LY_CUDA(cudaMemsetAsync(ms.err.p, 0, sizeof(int), st));
    lyap_set_last_error("tensor-core GEMM wait timed out (code " + std::to_string(herr) + ")");
    return LYAP_EDEVICE_TIMEOUT;
  }
  // ---- decisions
  const double pn = sd->ph_norm;
  std::vector<int> go, fin, fin_status;
  std::vector<double> norms_go, fin_rel;
  for (int s : fresh) {
    go.push_back(s);
    norms_go.push_back(pn);
  }
  for (size_t c = 0; c < old.size(); ++c) {
    const int s = old[c];
    const double rel = pn > 0 ? nrm_old[c] / pn : nrm_old[c];
    int stt = 1;  // 1: continue
    if (!std::isfinite(rel)) stt = LYAP_ENONFINITE;
    else if (rel <= o.refine_tol) stt = LYAP_OK;
    else if (e.steps[s] >= std::max(1, o.max_refine)) stt = LYAP_ENOCONV;
    if (stt == 1) {
      go.push_back(s);
      norms_go.push_back(nrm_old[c]);
    } else {
      fin.push_back(s);
      fin_status.push_back(stt);
      fin_rel.push_back(rel);
    }
  }
  // ---- retire: trace and error estimate (block-Jacobi proxy, as lyap_trace_EX)
  if (!fin.empty()) {
    const int nf = (int)fin.size();
    LY_CUDA(cudaMemcpyAsync(e.slots2.p, fin.data(), sizeof(int) * nf, cudaMemcpyHostToDevice, st));
    LY_CUDA(cudaMemcpyAsync(ms.cnt.p, &nf, sizeof(int), cudaMemcpyHostToDevice, st));
    k_engine_dot_h<<<nf, kry::NT, 0, st>>>(N, e.slots2.p, nf, e.W.p, sd->h.p, e.fout.p);
    lyap_count_launch();
    LY_TRY(prec_apply<double2>(sd, nullptr, false, e.vinv.p, e.slots2.p, ms.cnt.p, nf, ms.R64.p, (size_t)N,
                               e.delta.p, (size_t)N, st));
    k_engine_dot_h<<<nf, kry::NT, 0, st>>>(N, e.slots2.p, nf, e.delta.p, sd->h.p, e.eout.p);
    lyap_count_launch();
    LY_CUDA(cudaGetLastError());
    std::vector<double> fh(nf), eh(nf);
    LY_CUDA(cudaMemcpyAsync(fh.data(), e.fout.p, sizeof(double) * nf, cudaMemcpyDeviceToHost, st));
    LY_CUDA(cudaMemcpyAsync(eh.data(), e.eout.p, sizeof(double) * nf, cudaMemcpyDeviceToHost, st));
    LY_CUDA(cudaStreamSynchronize(st));
    for (int c = 0; c < nf; ++c) {
      const int s = fin[c];
      EngineDone d;
      d.slot = s;
      d.f = sd->f0 + fh[c];
      d.info.iters = e.iters[s];
      d.info.refine_steps = e.steps[s];
      d.info.status = fin_status[c];
      d.info.rel_resid = fin_rel[c];
      d.info.err_est = d.f != 0 ? std::fabs(eh[c]) / std::fabs(d.f) : std::fabs(eh[c]);
      done.push_back(d);
      e.steps[s] = -1;
    }
  }
  if (go.empty()) return LYAP_OK;
  // ---- one inner solve of every continuing system
  const int na = (int)go.size();
  LY_CUDA(cudaMemcpyAsync(ms.act.p, go.data(), sizeof(int) * na, cudaMemcpyHostToDevice, st));
  // ms.norms is indexed by slot in k_gather_r32 / k_scatter_add
  {
    std::vector<double> nfull(e.cap, 0.0);
    for (int c = 0; c < na; ++c) nfull[go[c]] = norms_go[c];
    LY_CUDA(cudaMemcpyAsync(ms.norms.p, nfull.data(), sizeof(double) * e.cap, cudaMemcpyHostToDevice, st));
    k_gather_r32<<<dim3(gx(N), na), 256, 0, st>>>(N, k, ms.act.p, na, ms.R64.p, ms.norms.p, e.vinv.p, ms.R32.p,
                                                  ms.vinv_c.p);
    lyap_count_launch();
    LY_CUDA(cudaGetLastError());
    SysOp<float2> op;
    op.sd = sd;
    op.vinv = ms.vinv_c.p;
    if (e.r > 0) {
      if (ms.wcinv.count < (size_t)na * e.r * e.r) LY_TRY(ms.wcinv.alloc((size_t)e.cap * e.r * e.r));
      if (ms.wpart.count < wood_part_count(n, k, na, e.r)) LY_TRY(ms.wpart.alloc(wood_part_count(n, k, e.cap, e.r)));
      ms.wood.cinv = ms.wcinv.p;
      ms.wood.cpart = ms.wpart.p;
      ms.wood.err = ms.err.p;
      LY_TRY(wood_bind(sd, e.r, na, e.cinv.p, ms.act.p, ms.wood, st));
      op.wood = &ms.wood;
    }
    std::vector<int> it, stt;
    LY_TRY(gcrodr_chunk<float2>(op, na, ms.R32.p, (size_t)N, sd->rec32, pin, e.ws, it, stt, st));
    k_scatter_add<<<dim3(gx(N), na), 256, 0, st>>>(N, ms.act.p, na, e.ws.X.p, ms.norms.p, e.W.p);
    lyap_count_launch();
    LY_CUDA(cudaGetLastError());
    for (int c = 0; c < na; ++c) {
      e.iters[go[c]] += it[c];
      e.steps[go[c]] += 1;
    }
  }
  return LYAP_OK;
}

// ------------------------------------------------------------ SysOp<float2>
template <>
int SysOp<float2>::apply(const int* list, const int* count, int B, const float2* In, size_t in_ss, float2* Out,
                         size_t out_ss, cudaStream_t st) const {
  return mixed_apply<float2>(sd, adjoint, vinv, list, count, B, In, in_ss, Out, out_ss, CAP_T, st);
}
template <>
int SysOp<float2>::apply_c0(int nvec, const float2* In, float2* Out, cudaStream_t st) const {
  const size_t N = (size_t)sd->n * sd->k;
  return mixed_apply<float2>(sd, adjoint, nullptr, nullptr, nullptr, nvec, In, N, Out, N, CAP_C0, st);
}
template <>
int SysOp<float2>::precond(const int* list, const int* count, int B, const float2* In, size_t in_ss, float2* Out,
                           size_t out_ss, cudaStream_t st) const {
  return prec_apply<float2>(sd, wood, adjoint, vinv, list, count, B, In, in_ss, Out, out_ss, st);
}

// ------------------------------------------------------------ testing hooks
extern "C" int lyap_test_apply(lyap_seed* sd, int nsys, const double* v, const double* w, int precision, int adjoint,
                               double* out) {
  if (!sd || nsys <= 0 || !v || !w || !out) return LYAP_EINVAL;
  (void)cudaGetLastError();
  LY_CUDA(cudaSetDevice(sd->device));
  cudaStream_t st = sd->ctx->stream;
  const int k = sd->k;
  const size_t N = (size_t)sd->n * k;
  DevBuf<double> vinv;
  LY_TRY(vinv.alloc((size_t)nsys * k));
  std::vector<double> hv((size_t)nsys * k);
  LY_CUDA(cudaMemcpyAsync(hv.data(), v, sizeof(double) * hv.size(), cudaMemcpyDeviceToHost, st));
  LY_CUDA(cudaStreamSynchronize(st));
  for (double& x : hv) x = 1.0 / x;
  LY_CUDA(cudaMemcpyAsync(vinv.p, hv.data(), sizeof(double) * hv.size(), cudaMemcpyHostToDevice, st));
  if (precision == LYAP_FP64 || precision == LYAP_TEST_FF || precision == LYAP_TEST_TC) {
    CapArgs64 a{};
    a.n = sd->n;
    a.k = k;
    a.lam = sd->lam.p;
    a.P1 = adjoint ? sd->Vb.p : sd->Ub.p;
    a.P2 = adjoint ? sd->Ub.p : sd->Vb.p;
    a.Gd = sd->Gd.p;
    a.gT = adjoint ? 1 : 0;
    a.W = reinterpret_cast<const double2*>(w);
    a.ldw = N;
    a.vinv = vinv.p;
    a.out = reinterpret_cast<double2*>(out);
    a.ldo = N;
    a.mode = CAP_T;
    a.nsys = nsys;
    if (precision == LYAP_FP64) {
      LY_TRY(capmv64_launch(a, st));
    } else if (precision == LYAP_TEST_TC) {
      MixedState& ms = *sd->mixed;
      if (!ms.oz_ok) return LYAP_EINVAL;
      const int ncap = ((nsys * k * k * ms.cm + oz::BN - 1) / oz::BN) * oz::BN;
      DevBuf<__nv_bfloat16> Bd;
      DevBuf<int> eB;
      DevBuf<float2> Dd;
      LY_TRY(Bd.alloc((size_t)oz::NS * ncap * ms.kpad));
      LY_TRY(eB.alloc(ncap));
      LY_TRY(Dd.alloc((size_t)ncap * ms.mpad));
      oz::Panel pn;
      pn.S = Bd.p;
      pn.eB = eB.p;
      pn.D = Dd.p;
      pn.ncap = ncap;
      LY_TRY(oz::make_map(&pn.mapB, Bd.p, oz::NS * ncap, ms.kpad, oz::BN));
      LY_TRY(oz::residual(a, ms.ozMapA, ms.ozEA.p, ms.mpad, ms.kpad, ms.rs, pn, ms.err.p, st));
      LY_CUDA(cudaStreamSynchronize(st));
    } else {
      DevBuf<double> sw;
      DevBuf<float4> panel;
      LY_TRY(sw.alloc(nsys));
      LY_TRY(panel.alloc((size_t)nsys * k * k * sd->n));
      LY_TRY(capmv_df_launch(a, sd->mixed->Lff.p, sd->mixed->lc_scale, sd->mixed->p_scale, sw.p, panel.p, st));
      LY_CUDA(cudaStreamSynchronize(st));
    }
  } else {
    LY_TRY(mixed_apply<double2>(sd, adjoint != 0, vinv.p, nullptr, nullptr, nsys, reinterpret_cast<const double2*>(w),
                                N, reinterpret_cast<double2*>(out), N, CAP_T, st));
  }
  LY_CUDA(cudaStreamSynchronize(st));
  int herr = 0;
  if (sd->mixed) LY_CUDA(cudaMemcpy(&herr, sd->mixed->err.p, sizeof(int), cudaMemcpyDeviceToHost));
  return herr ? LYAP_EDEVICE_TIMEOUT : LYAP_OK;
}

namespace {
__global__ void k_split_rows(int rows, int cols, int kpad, const float* __restrict__ X, __nv_bfloat16* __restrict__ H,
                             __nv_bfloat16* __restrict__ L) {
  const size_t total = (size_t)rows * kpad;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
    const int r = (int)(idx / kpad), c = (int)(idx % kpad);
    const float x = c < cols ? X[(size_t)r * cols + c] : 0.f;
    const __nv_bfloat16 h = __float2bfloat16_rn(x);
    H[idx] = h;
    L[idx] = __float2bfloat16_rn(x - __bfloat162float(h));
  }
}
}  // namespace

extern "C" int lyap_test_tc_gemm(int M, int N, int K, const float* A, const float* B, float* D) {
  if (M <= 0 || N <= 0 || K <= 0 || !A || !B || !D) return LYAP_EINVAL;
  const int mpad = ((M + tc::BM - 1) / tc::BM) * tc::BM;
  const int kpad = ((K + tc::BK - 1) / tc::BK) * tc::BK;
  const int ncap = ((N + tc::BN - 1) / tc::BN) * tc::BN;
  DevBuf<__nv_bfloat16> ah, al, bh, bl;
  DevBuf<float> Dp;
  DevBuf<int> err;
  LY_TRY(ah.alloc((size_t)mpad * kpad));
  LY_TRY(al.alloc((size_t)mpad * kpad));
  LY_TRY(bh.alloc((size_t)ncap * kpad));
  LY_TRY(bl.alloc((size_t)ncap * kpad));
  LY_TRY(Dp.alloc((size_t)ncap * mpad));
  LY_TRY(err.alloc(1));
  LY_CUDA(cudaMemset(ah.p, 0, ah.bytes()));
  LY_CUDA(cudaMemset(al.p, 0, al.bytes()));
  LY_CUDA(cudaMemset(bh.p, 0, bh.bytes()));
  LY_CUDA(cudaMemset(bl.p, 0, bl.bytes()));
  LY_CUDA(cudaMemset(err.p, 0, sizeof(int)));
  k_split_rows<<<1024, 256>>>(M, K, kpad, A, ah.p, al.p);
  k_split_rows<<<1024, 256>>>(N, K, kpad, B, bh.p, bl.p);
  lyap_count_launch(2);
  LY_CUDA(cudaGetLastError());
  tc::Maps m;
  LY_TRY(tc::make_map(&m.a_hi, ah.p, mpad, kpad, tc::BM));
  LY_TRY(tc::make_map(&m.a_lo, al.p, mpad, kpad, tc::BM));
  LY_TRY(tc::make_map(&m.b_hi, bh.p, ncap, kpad, tc::BN));
  LY_TRY(tc::make_map(&m.b_lo, bl.p, ncap, kpad, tc::BN));
  LY_TRY(tc::launch(m, Dp.p, mpad, M, mpad, kpad, nullptr, 1, N, N, err.p, 0));
  LY_CUDA(cudaDeviceSynchronize());
  int herr = 0;
  LY_CUDA(cudaMemcpy(&herr, err.p, sizeof(int), cudaMemcpyDeviceToHost));
  LY_CUDA(cudaMemcpy2D(D, sizeof(float) * M, Dp.p, sizeof(float) * mpad, sizeof(float) * M, N, cudaMemcpyDeviceToDevice));
  return herr ? LYAP_EDEVICE_TIMEOUT : LYAP_OK;
}
