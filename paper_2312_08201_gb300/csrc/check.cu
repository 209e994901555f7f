// Independent check of capacitance solutions through the explicit Lyapunov
// solution (a verification tool, O(n^3) per parameter vector, FP64 on
// cuBLAS).
//
// From the seed's eigen-decomposition A0^T = Qp diag(lam) Qp^{-1} and a
// shifted capacitance solution W' (lyap_param_solve),
//     X(v) = X0 + Qp (Lc o (W' Ub^T + Ub W'^T)) Qp^T,
//     X0   = Qp (-Lc o (Gh Gh^T)) Qp^T,   Gh = Qp^{-1} G,   Lc_ij = 1/(lam_i + lam_j)
// (eqs. (splitXv), (seedLE) and (Xsmalllastline) of §2.1 with the shift
// W' = W + P D(v)). The check then evaluates, in FP64, the true residual of
// the equation itself,
//     R = A(v)^T X + X A(v) + G G^T,   A(v) = A0 - U diag(v) V^T,
// and its backward error ||R||_F / (2 ||A(v)||_F ||X||_F + ||G G^T||_F) (the
// form of the backward error proposition of §2.2), together with
// trace(E X). None of it goes through the capacitance operator the solver
// used, so an error in the seed precompute, the operator or the trace
// vector shows up here.
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "cplx.cuh"
#include "lyap_internal.h"
#include "prof.h"

namespace {

int gsz(size_t count) { return (int)std::max<size_t>(1, std::min<size_t>((count + 255) / 256, 4096)); }

// M[i,j] *= s / (lam_i + lam_j)
__global__ void k_chk_cauchy(int n, const double2* __restrict__ lam, double2* __restrict__ M, double s) {
  const size_t total = (size_t)n * n;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const size_t i = e % n, j = e / n;
    M[e] = cscale(cmul(M[e], crcp(cadd(lam[i], lam[j]))), s);
  }
}

// out = Re(in) (+ add)
__global__ void k_chk_real(size_t count, const double2* __restrict__ in, const double* __restrict__ add,
                           double* __restrict__ out) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < count; e += (size_t)gridDim.x * blockDim.x)
    out[e] = in[e].x + (add ? add[e] : 0.0);
}

__global__ void k_chk_complex(size_t count, const double* __restrict__ in, double2* __restrict__ out) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < count; e += (size_t)gridDim.x * blockDim.x)
    out[e] = make_double2(in[e], 0.0);
}

// R = T + T^T - M - M^T + GG  (n x n, column-major)
__global__ void k_chk_resid(int n, const double* __restrict__ T, const double* __restrict__ M,
                            const double* __restrict__ GG, double* __restrict__ R) {
  const size_t total = (size_t)n * n;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const size_t i = e % n, j = e / n, t = j + i * (size_t)n;
    R[e] = T[e] + T[t] - M[e] - M[t] + GG[e];
  }
}

// D = A - U diag(v) V^T
__global__ void k_chk_av(int n, int k, const double* __restrict__ A, const double* __restrict__ U,
                         const double* __restrict__ V, const double* __restrict__ v, double* __restrict__ D) {
  const size_t total = (size_t)n * n;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const size_t i = e % n, j = e / n;
    double s = A[e];
    for (int t = 0; t < k; ++t) s -= U[i + (size_t)t * n] * v[t] * V[j + (size_t)t * n];
    D[e] = s;
  }
}

int zgemm(cublasHandle_t h, cublasOperation_t ta, cublasOperation_t tb, int m, int n, int k, const double2* A,
          int lda, const double2* B, int ldb, double2* C, int ldc) {
  const cuDoubleComplex one = make_cuDoubleComplex(1.0, 0.0), zero = make_cuDoubleComplex(0.0, 0.0);
  LY_BLAS(cublasZgemm(h, ta, tb, m, n, k, &one, reinterpret_cast<const cuDoubleComplex*>(A), lda,
                      reinterpret_cast<const cuDoubleComplex*>(B), ldb, &zero, reinterpret_cast<cuDoubleComplex*>(C),
                      ldc));
  return LYAP_OK;
}

int dgemm(cublasHandle_t h, cublasOperation_t ta, cublasOperation_t tb, int m, int n, int k, double alpha,
          const double* A, int lda, const double* B, int ldb, double beta, double* C, int ldc) {
  LY_BLAS(cublasDgemm(h, ta, tb, m, n, k, &alpha, A, lda, B, ldb, &beta, C, ldc));
  return LYAP_OK;
}

double fro(cublasHandle_t h, const double* A, size_t count) {
  double r = 0.0;
  if (cublasDnrm2(h, (int)count, A, 1, &r) != CUBLAS_STATUS_SUCCESS) return NAN;
  return r;
}

}  // namespace

extern "C" int lyap_check_explicit(lyap_seed* sd, int nv, const double* v, const double* w, const double* A0,
                                   const double* U, const double* V, const double* G, int g, const double* E,
                                   int mem_kind, double* backward_err_out, double* trace_out) {
  if (!sd || nv < 0 || g < 1 || (nv > 0 && (!v || !w || !A0 || !U || !V || !G || !backward_err_out || !trace_out)))
    return LYAP_EINVAL;
  if (mem_kind != LYAP_MEM_HOST && mem_kind != LYAP_MEM_DEVICE) return LYAP_EINVAL;
  if (nv == 0) return LYAP_OK;
  (void)cudaGetLastError();
  LY_CUDA(cudaSetDevice(sd->device));
  lyap_ctx* ctx = sd->ctx;
  cudaStream_t st = ctx->stream;
  const int n = sd->n, k = sd->k;
  const size_t nn = (size_t)n * n, N = (size_t)n * k;
  std::vector<double> hv((size_t)nv * k);
  const cudaMemcpyKind kind = mem_kind == LYAP_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  // on the context's stream, like every other input of the call
  LY_CUDA(cudaMemcpyAsync(hv.data(), v, sizeof(double) * hv.size(),
                          mem_kind == LYAP_MEM_HOST ? cudaMemcpyHostToHost : cudaMemcpyDeviceToHost, st));
  LY_CUDA(cudaStreamSynchronize(st));
  DevBuf<double> dA, dU, dV, dG, dE, dv, GG, Xr, X0r, T, M, K1, R, Av;
  DevBuf<double2> Gc, Gh, Z1, Z2, WU, UW, Wd;
  LY_TRY(dA.alloc(nn));
  LY_TRY(dU.alloc(N));
  LY_TRY(dV.alloc(N));
  LY_TRY(dG.alloc((size_t)n * g));
  LY_TRY(dv.alloc(k));
  LY_CUDA(cudaMemcpyAsync(dA.p, A0, sizeof(double) * nn, kind, st));
  LY_CUDA(cudaMemcpyAsync(dU.p, U, sizeof(double) * N, kind, st));
  LY_CUDA(cudaMemcpyAsync(dV.p, V, sizeof(double) * N, kind, st));
  LY_CUDA(cudaMemcpyAsync(dG.p, G, sizeof(double) * n * g, kind, st));
  if (E) {
    LY_TRY(dE.alloc(nn));
    LY_CUDA(cudaMemcpyAsync(dE.p, E, sizeof(double) * nn, kind, st));
  }
  LY_TRY(GG.alloc(nn));
  LY_TRY(Xr.alloc(nn));
  LY_TRY(X0r.alloc(nn));
  LY_TRY(T.alloc(nn));
  LY_TRY(M.alloc(nn));
  LY_TRY(K1.alloc(N));
  LY_TRY(R.alloc(nn));
  LY_TRY(Av.alloc(nn));
  LY_TRY(Gc.alloc((size_t)n * g));
  LY_TRY(Gh.alloc((size_t)n * g));
  LY_TRY(Z1.alloc(nn));
  LY_TRY(Z2.alloc(nn));
  LY_TRY(WU.alloc(2 * N));
  LY_TRY(UW.alloc(2 * N));
  LY_TRY(Wd.alloc(N));
  std::lock_guard<std::mutex> lk(ctx->handle_mu);
  cublasHandle_t bl = ctx->blas;
  LY_BLAS(cublasSetStream(bl, st));
  // G G^T and X0 = Qp (-Lc o (Gh Gh^T)) Qp^T
  LY_TRY(dgemm(bl, CUBLAS_OP_N, CUBLAS_OP_T, n, n, g, 1.0, dG.p, n, dG.p, n, 0.0, GG.p, n));
  k_chk_complex<<<gsz((size_t)n * g), 256, 0, st>>>((size_t)n * g, dG.p, Gc.p);
  lyap_count_launch();
  LY_TRY(zgemm(bl, CUBLAS_OP_N, CUBLAS_OP_N, n, g, n, sd->Qi.p, n, Gc.p, n, Gh.p, n));
  LY_TRY(zgemm(bl, CUBLAS_OP_N, CUBLAS_OP_T, n, n, g, Gh.p, n, Gh.p, n, Z1.p, n));
  k_chk_cauchy<<<gsz(nn), 256, 0, st>>>(n, sd->lam.p, Z1.p, -1.0);
  lyap_count_launch();
  LY_TRY(zgemm(bl, CUBLAS_OP_N, CUBLAS_OP_N, n, n, n, sd->Qp.p, n, Z1.p, n, Z2.p, n));
  LY_TRY(zgemm(bl, CUBLAS_OP_N, CUBLAS_OP_T, n, n, n, Z2.p, n, sd->Qp.p, n, Z1.p, n));
  k_chk_real<<<gsz(nn), 256, 0, st>>>(nn, Z1.p, nullptr, X0r.p);
  lyap_count_launch();
  LY_CUDA(cudaGetLastError());
  const double ngg = fro(bl, GG.p, nn);
  for (int b = 0; b < nv; ++b) {
    // Xd = Qp (Lc o ([W' Ub] [Ub W']^T)) Qp^T
    const double2* wb = reinterpret_cast<const double2*>(w) + (size_t)b * N;
    if (mem_kind == LYAP_MEM_HOST) {
      LY_CUDA(cudaMemcpyAsync(Wd.p, wb, sizeof(double2) * N, cudaMemcpyHostToDevice, st));
      wb = Wd.p;
    }
    LY_CUDA(cudaMemcpyAsync(WU.p, wb, sizeof(double2) * N, cudaMemcpyDeviceToDevice, st));
    LY_CUDA(cudaMemcpyAsync(WU.p + N, sd->Ub.p, sizeof(double2) * N, cudaMemcpyDeviceToDevice, st));
    LY_CUDA(cudaMemcpyAsync(UW.p, sd->Ub.p, sizeof(double2) * N, cudaMemcpyDeviceToDevice, st));
    LY_CUDA(cudaMemcpyAsync(UW.p + N, wb, sizeof(double2) * N, cudaMemcpyDeviceToDevice, st));
    LY_TRY(zgemm(bl, CUBLAS_OP_N, CUBLAS_OP_T, n, n, 2 * k, WU.p, n, UW.p, n, Z1.p, n));
    k_chk_cauchy<<<gsz(nn), 256, 0, st>>>(n, sd->lam.p, Z1.p, 1.0);
    lyap_count_launch();
    LY_TRY(zgemm(bl, CUBLAS_OP_N, CUBLAS_OP_N, n, n, n, sd->Qp.p, n, Z1.p, n, Z2.p, n));
    LY_TRY(zgemm(bl, CUBLAS_OP_N, CUBLAS_OP_T, n, n, n, Z2.p, n, sd->Qp.p, n, Z1.p, n));
    k_chk_real<<<gsz(nn), 256, 0, st>>>(nn, Z1.p, X0r.p, Xr.p);  // X = X0 + Re(Xd)
    lyap_count_launch();
    // R = A0^T X + X A0 - V D (U^T X) - (V D (U^T X))^T + G G^T   (X symmetric)
    LY_CUDA(cudaMemcpyAsync(dv.p, hv.data() + (size_t)b * k, sizeof(double) * k, cudaMemcpyHostToDevice, st));
    LY_TRY(dgemm(bl, CUBLAS_OP_T, CUBLAS_OP_N, n, n, n, 1.0, dA.p, n, Xr.p, n, 0.0, T.p, n));
    LY_TRY(dgemm(bl, CUBLAS_OP_T, CUBLAS_OP_N, k, n, n, 1.0, dU.p, n, Xr.p, n, 0.0, K1.p, k));  // U^T X
    LY_CUDA(cudaMemcpyAsync(Av.p, dV.p, sizeof(double) * N, cudaMemcpyDeviceToDevice, st));
    for (int t = 0; t < k; ++t) LY_BLAS(cublasDscal(bl, n, hv.data() + (size_t)b * k + t, Av.p + (size_t)t * n, 1));
    LY_TRY(dgemm(bl, CUBLAS_OP_N, CUBLAS_OP_N, n, n, k, 1.0, Av.p, n, K1.p, k, 0.0, M.p, n));  // V D U^T X
    k_chk_resid<<<gsz(nn), 256, 0, st>>>(n, T.p, M.p, GG.p, R.p);
    k_chk_av<<<gsz(nn), 256, 0, st>>>(n, k, dA.p, dU.p, dV.p, dv.p, Av.p);  // A(v)
    lyap_count_launch(2);
    LY_CUDA(cudaGetLastError());
    const double nr = fro(bl, R.p, nn), nx = fro(bl, Xr.p, nn), na = fro(bl, Av.p, nn);
    backward_err_out[b] = nr / (2.0 * na * nx + ngg);
    double tr = 0.0;
    if (E) {
      LY_BLAS(cublasDdot(bl, (int)nn, dE.p, 1, Xr.p, 1, &tr));  // E symmetric: trace(E X) = sum E o X
    } else {
      std::vector<double> diag(n);
      LY_CUDA(cudaMemcpy2DAsync(diag.data(), sizeof(double), Xr.p, sizeof(double) * (n + 1), sizeof(double), n,
                                cudaMemcpyDeviceToHost, st));
      LY_CUDA(cudaStreamSynchronize(st));
      for (int i = 0; i < n; ++i) tr += diag[i];
    }
    trace_out[b] = tr;
  }
  LY_CUDA(cudaStreamSynchronize(st));
  return LYAP_OK;
}
