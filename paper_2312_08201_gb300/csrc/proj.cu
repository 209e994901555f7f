// Projection framework for large parametrized Lyapunov sequences (paper
// §2.2: eqs. (EK_def), (param_projected), the backward error proposition,
// Algorithm 1), on the device.
//
// Convention of §2.2: A_p(v) = A0p - B_l D(v) B_r^T with A0p = A0^T,
// B_l = V, B_r = U (the API's A(v) = A0 - U diag(v) V^T), and the change
// X_d(v) = X(v) - X0 solving
//     A_p(v) X_d + X_d A_p(v)^T = P (I2 (x) D(v)) P^T,   P = [X0 B_r, B_l].
//
// Offline (once per projection object, cuBLAS/cuSOLVER in FP64):
//   * the LU factors of A0 (Assumption 3); solves with A0p use them
//     transposed;
//   * one orthonormal basis of EK_m(A0p, P) for every v, one block per
//     expansion: block 1 spans [P, A0p^{-1} P] (so P = V_1 G), block j+1 is
//     [A0p V_j^(1), A0p^{-1} V_j^(2)] orthogonalised against all blocks by
//     block classical Gram-Schmidt, twice; directions below 1e-13 of their
//     candidate's size are dropped (the deflation the paper points to), the
//     two halves of a block deflate separately, an empty block ends the
//     space;
//   * A0p V_m, kept next to V_m, gives T_m = V_m^T A0p V_m and the block
//     row E_m^T underline(T)_m = V_{m+1-block}^T A0p V_m of the Arnoldi
//     relation;
//   * the n-sized scalars of the backward error: ||A0||_F,
//     (B_r^T B_l) o (B_r^T B_l), a = diag(B_r^T A0p B_l), and P^T P.
// For each m (Algorithm 1), the projected equation (param_projected) is a
// parametrized Lyapunov equation of order d = dim V_m whose right-hand side
// factor is [V_m^T X0 B_r, B_{l,m}]: it is solved by the library's own
// small-scale path (§2.1: eigen-decomposition of T_m, SMW capacitance
// systems, recycled GCRO-DR) for all remaining v in one lockstep batch, as
// §2.2 suggests. From each capacitance solution W' the projected solution
//     Y_m(v) = Qp (Lc o (W' Ub^T + Ub W'^T)) Qp^T
// is formed by batched GEMMs, and the backward error of the proposition
//     Delta = sqrt(2) ||E_m^T underline(T)_m Y|| /
//             (2 sqrt(||A0||^2 + v^T H v - 2 a^T v) ||Y|| + ||G (I2 (x) D) G^T||)
// needs no n-sized work per v. f(v) = f(X0) + trace(V_m^T E V_m Y_m(v)).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <memory>
#include <mutex>
#include <vector>

#include "cplx.cuh"
#include "krylov.cuh"
#include "lyap_internal.h"
#include "prof.h"

namespace {

constexpr double kRankTol = 1e-13;  // deflation threshold, relative to the candidate block's largest column

// Ls_b[i,j] = Lc_ij (sum_t W_b[i,t] Ub[j,t] + Ub[i,t] W_b[j,t]),  Lc_ij = 1/(lam_i + lam_j)
__global__ void k_proj_hadamard(int d, int k, int nsys, const double2* __restrict__ lam,
                                const double2* __restrict__ Ub, const double2* __restrict__ W,
                                double2* __restrict__ L) {
  const int b = blockIdx.y;
  if (b >= nsys) return;
  const size_t dd = (size_t)d * d;
  const double2* Wb = W + (size_t)b * d * k;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < dd; idx += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(idx % d), j = (int)(idx / d);
    double2 s = make_double2(0.0, 0.0);
    for (int t = 0; t < k; ++t) {
      s = cadd(s, cmul(Wb[(size_t)t * d + i], Ub[(size_t)t * d + j]));
      s = cadd(s, cmul(Ub[(size_t)t * d + i], Wb[(size_t)t * d + j]));
    }
    L[(size_t)b * dd + idx] = cmul(s, crcp(cadd(lam[i], lam[j])));
  }
}

// Yr_b = Re(Y_b), nrm[b] = ||Y_b||_F^2 (the imaginary part is rounding)
__global__ void __launch_bounds__(kry::NT) k_proj_real(int d, int nsys, const double2* __restrict__ Y,
                                                       double* __restrict__ Yr, double* __restrict__ nrm) {
  __shared__ double red[32];
  const int b = blockIdx.x;
  if (b >= nsys) return;
  const size_t dd = (size_t)d * d;
  double acc[1] = {0.0};
  for (size_t e = threadIdx.x; e < dd; e += kry::NT) {
    const double y = Y[(size_t)b * dd + e].x;
    Yr[(size_t)b * dd + e] = y;
    acc[0] += y * y;
  }
  kry::block_sum<1>(acc, red);
  if (threadIdx.x == 0) nrm[b] = acc[0];
}

__global__ void __launch_bounds__(kry::NT) k_proj_sqnorm(size_t len, int nsys, const double* __restrict__ A,
                                                         double* __restrict__ out) {
  __shared__ double red[32];
  const int b = blockIdx.x;
  if (b >= nsys) return;
  double acc[1] = {0.0};
  for (size_t e = threadIdx.x; e < len; e += kry::NT) {
    const double x = A[(size_t)b * len + e];
    acc[0] += x * x;
  }
  kry::block_sum<1>(acc, red);
  if (threadIdx.x == 0) out[b] = acc[0];
}

int gridsz(size_t count) { return (int)std::max<size_t>(1, std::min<size_t>((count + 255) / 256, 4096)); }

int dgemm(cublasHandle_t h, cublasOperation_t ta, cublasOperation_t tb, int m, int n, int k, double alpha,
          const double* A, int lda, const double* B, int ldb, double beta, double* C, int ldc) {
  if (m <= 0 || n <= 0) return LYAP_OK;
  LY_BLAS(cublasDgemm(h, ta, tb, m, n, k, &alpha, A, lda, B, ldb, &beta, C, ldc));
  return LYAP_OK;
}

}  // namespace

struct lyap_proj {
  lyap_ctx* ctx = nullptr;
  int device = 0;
  int n = 0, k = 0;
  bool has_E = false;
  DevBuf<double> A0, LU, U, V, E, XBr, P;
  DevBuf<int> ipiv, info;
  double f0 = 0.0, normA0 = 0.0;
  std::vector<double> H, a, PtP;  // k x k, k, 2k x 2k (host, column-major)
  // basis V_m and A0p V_m, n x cap each; block b holds columns [off[b], off[b+1])
  DevBuf<double> Vm, AVm;
  int cap = 0, dim = 0;
  std::vector<int> off{0}, split;
  bool exhausted = false;
  DevBuf<double> work;  // n x 2k candidates and scratch
  // cusolver gesvd scratch
  DevBuf<double> svd_s, svd_u, svd_work;
  int svd_lwork = 0;
  // the projected seed of the last m (kept between calls)
  lyap_seed* small = nullptr;
  int small_m = -1;
  int small_prec = -1, small_pbar = -1;
  ~lyap_proj() {
    if (small) lyap_seed_free(small);
  }
};

namespace {

int ensure_cap(lyap_proj* pj, int need, cudaStream_t st) {
  if (need <= pj->cap) return LYAP_OK;
  const int ncap = std::max(need, std::max(2 * pj->cap, 8 * pj->k));
  const size_t n = pj->n;
  DevBuf<double> nv, nav;
  LY_TRY(nv.alloc(n * ncap));
  LY_TRY(nav.alloc(n * ncap));
  if (pj->dim > 0) {
    LY_CUDA(cudaMemcpyAsync(nv.p, pj->Vm.p, sizeof(double) * n * pj->dim, cudaMemcpyDeviceToDevice, st));
    LY_CUDA(cudaMemcpyAsync(nav.p, pj->AVm.p, sizeof(double) * n * pj->dim, cudaMemcpyDeviceToDevice, st));
    LY_CUDA(cudaStreamSynchronize(st));  // the old buffers are freed below
  }
  pj->Vm = std::move(nv);
  pj->AVm = std::move(nav);
  pj->cap = ncap;
  return LYAP_OK;
}

// Append the orthonormal directions of Range(W) (n x w, overwritten) that
// are new to the current basis: block classical Gram-Schmidt against the
// basis, twice, then a thin SVD; singular values below kRankTol times the
// largest candidate column norm are dropped. Returns the count appended.
int append_directions(lyap_proj* pj, double* W, int w, cudaStream_t st, int* added) {
  *added = 0;
  if (w == 0) return LYAP_OK;
  const int n = pj->n;
  cublasHandle_t bl = pj->ctx->blas;
  double ref = 0.0;
  for (int c = 0; c < w; ++c) {
    double nc = 0.0;
    LY_BLAS(cublasDnrm2(bl, n, W + (size_t)c * n, 1, &nc));  // host result: synchronises
    ref = std::max(ref, nc);
  }
  if (!(ref > 0.0)) return LYAP_OK;
  DevBuf<double> C;
  if (pj->dim > 0) LY_TRY(C.alloc((size_t)pj->dim * w));
  for (int pass = 0; pass < 2 && pj->dim > 0; ++pass) {
    LY_TRY(dgemm(bl, CUBLAS_OP_T, CUBLAS_OP_N, pj->dim, w, n, 1.0, pj->Vm.p, n, W, n, 0.0, C.p, pj->dim));
    LY_TRY(dgemm(bl, CUBLAS_OP_N, CUBLAS_OP_N, n, w, pj->dim, -1.0, pj->Vm.p, n, C.p, pj->dim, 1.0, W, n));
  }
  // thin SVD W = Us S Vt (m = n >= w columns)
  if (pj->svd_s.count < (size_t)w) LY_TRY(pj->svd_s.alloc(2 * pj->k + 2));
  if (pj->svd_u.count < (size_t)n * w) LY_TRY(pj->svd_u.alloc((size_t)n * (2 * pj->k + 2)));
  int lwork = 0;
  LY_SOLVER(cusolverDnDgesvd_bufferSize(pj->ctx->solver, n, w, &lwork));
  if (lwork > pj->svd_lwork) {
    LY_TRY(pj->svd_work.alloc(lwork));
    pj->svd_lwork = lwork;
  }
  DevBuf<double> vt, rwork;
  LY_TRY(vt.alloc((size_t)w * w));
  LY_TRY(rwork.alloc((size_t)w));
  LY_SOLVER(cusolverDnDgesvd(pj->ctx->solver, 'S', 'N', n, w, W, n, pj->svd_s.p, pj->svd_u.p, n, vt.p, w,
                             pj->svd_work.p, lwork, rwork.p, pj->info.p));
  std::vector<double> sv(w);
  int hinfo = 0;
  LY_CUDA(cudaMemcpyAsync(sv.data(), pj->svd_s.p, sizeof(double) * w, cudaMemcpyDeviceToHost, st));
  LY_CUDA(cudaMemcpyAsync(&hinfo, pj->info.p, sizeof(int), cudaMemcpyDeviceToHost, st));
  LY_CUDA(cudaStreamSynchronize(st));
  if (hinfo != 0) {
    lyap_set_last_error("gesvd info = " + std::to_string(hinfo));
    return LYAP_ESOLVER;
  }
  int r = 0;
  while (r < w && sv[r] > kRankTol * ref) ++r;
  if (r == 0) return LYAP_OK;
  LY_TRY(ensure_cap(pj, pj->dim + r, st));
  LY_CUDA(cudaMemcpyAsync(pj->Vm.p + (size_t)pj->dim * n, pj->svd_u.p, sizeof(double) * n * r,
                          cudaMemcpyDeviceToDevice, st));
  // A0p times the new columns: A0^T Q
  LY_TRY(dgemm(bl, CUBLAS_OP_T, CUBLAS_OP_N, n, r, n, 1.0, pj->A0.p, n, pj->Vm.p + (size_t)pj->dim * n, n, 0.0,
               pj->AVm.p + (size_t)pj->dim * n, n));
  pj->dim += r;
  *added = r;
  return LYAP_OK;
}

// W = A0p^{-1} W (n x w) with the stored LU of A0: A0^T x = b
int solve_A0p(lyap_proj* pj, double* W, int w, cudaStream_t st) {
  if (w == 0) return LYAP_OK;
  LY_SOLVER(cusolverDnDgetrs(pj->ctx->solver, CUBLAS_OP_T, pj->n, w, pj->LU.p, pj->n, pj->ipiv.p, W, pj->n,
                             pj->info.p));
  int hinfo = 0;
  LY_CUDA(cudaMemcpyAsync(&hinfo, pj->info.p, sizeof(int), cudaMemcpyDeviceToHost, st));
  LY_CUDA(cudaStreamSynchronize(st));
  if (hinfo != 0) {
    lyap_set_last_error("getrs info = " + std::to_string(hinfo));
    return LYAP_ESOLVER;
  }
  return LYAP_OK;
}

// Block 1: [P, A0p^{-1} P] (eq. (EK_def) with m = 1).
int first_block(lyap_proj* pj, cudaStream_t st) {
  const int n = pj->n, w = 2 * pj->k;
  double* W = pj->work.p;
  LY_CUDA(cudaMemcpyAsync(W, pj->P.p, sizeof(double) * n * w, cudaMemcpyDeviceToDevice, st));
  int r1 = 0, r2 = 0;
  LY_TRY(append_directions(pj, W, w, st, &r1));
  LY_CUDA(cudaMemcpyAsync(W, pj->P.p, sizeof(double) * n * w, cudaMemcpyDeviceToDevice, st));
  LY_TRY(solve_A0p(pj, W, w, st));
  LY_TRY(append_directions(pj, W, w, st, &r2));
  pj->off.push_back(pj->dim);
  pj->split.push_back(r1);
  return LYAP_OK;
}

// Block j+1 from [A0p V_j^(1), A0p^{-1} V_j^(2)].
int expand(lyap_proj* pj, cudaStream_t st) {
  const int n = pj->n;
  const int nb = (int)pj->split.size();
  const int o = pj->off[nb - 1], sz = pj->off[nb] - o, sp = pj->split[nb - 1];
  double* W = pj->work.p;
  int r1 = 0, r2 = 0;
  if (sp > 0) {
    LY_TRY(dgemm(pj->ctx->blas, CUBLAS_OP_T, CUBLAS_OP_N, n, sp, n, 1.0, pj->A0.p, n, pj->Vm.p + (size_t)o * n, n,
                 0.0, W, n));
    LY_TRY(append_directions(pj, W, sp, st, &r1));
  }
  if (sz - sp > 0) {
    LY_CUDA(cudaMemcpyAsync(W, pj->Vm.p + (size_t)(o + sp) * n, sizeof(double) * n * (sz - sp),
                            cudaMemcpyDeviceToDevice, st));
    LY_TRY(solve_A0p(pj, W, sz - sp, st));
    LY_TRY(append_directions(pj, W, sz - sp, st, &r2));
  }
  pj->off.push_back(pj->dim);
  pj->split.push_back(r1);
  if (r1 + r2 == 0) pj->exhausted = true;
  return LYAP_OK;
}

// Blocks up to m + 1 exist (or the space has ended).
int ensure_blocks(lyap_proj* pj, int m, cudaStream_t st) {
  if (pj->split.empty()) LY_TRY(first_block(pj, st));
  while ((int)pj->split.size() < m + 1 && !pj->exhausted) LY_TRY(expand(pj, st));
  return LYAP_OK;
}

// The projected seed of V_m (m blocks): A0 = T_m^T, U = B_{r,m}, V = B_{l,m},
// right-hand side block V_m^T X0 B_r, E = V_m^T E V_m.
int build_small(lyap_proj* pj, int m, const lyap_opts& o, cudaStream_t st) {
  const int mm = std::min(m, (int)pj->split.size());
  if (pj->small && pj->small_m == mm && pj->small_prec == o.precision && pj->small_pbar == o.pbar)
    return LYAP_OK;
  if (pj->small) {
    lyap_seed_free(pj->small);
    pj->small = nullptr;
  }
  const int n = pj->n, k = pj->k, d = pj->off[mm];
  cublasHandle_t bl = pj->ctx->blas;
  std::unique_lock<std::mutex> lk(pj->ctx->handle_mu);  // released before the preconditioner set-up takes it
  LY_BLAS(cublasSetStream(bl, st));
  LY_SOLVER(cusolverDnSetStream(pj->ctx->solver, st));
  DevBuf<double> At, Us, Vs, P1s, Es;
  LY_TRY(At.alloc((size_t)d * d));
  LY_TRY(Us.alloc((size_t)d * k));
  LY_TRY(Vs.alloc((size_t)d * k));
  LY_TRY(P1s.alloc((size_t)d * k));
  // T_m^T = (V_m^T A0p V_m)^T = (A0p V_m)^T V_m
  LY_TRY(dgemm(bl, CUBLAS_OP_T, CUBLAS_OP_N, d, d, n, 1.0, pj->AVm.p, n, pj->Vm.p, n, 0.0, At.p, d));
  LY_TRY(dgemm(bl, CUBLAS_OP_T, CUBLAS_OP_N, d, k, n, 1.0, pj->Vm.p, n, pj->U.p, n, 0.0, Us.p, d));
  LY_TRY(dgemm(bl, CUBLAS_OP_T, CUBLAS_OP_N, d, k, n, 1.0, pj->Vm.p, n, pj->V.p, n, 0.0, Vs.p, d));
  LY_TRY(dgemm(bl, CUBLAS_OP_T, CUBLAS_OP_N, d, k, n, 1.0, pj->Vm.p, n, pj->XBr.p, n, 0.0, P1s.p, d));
  if (pj->has_E) {
    DevBuf<double> EV;
    LY_TRY(EV.alloc((size_t)n * d));
    LY_TRY(Es.alloc((size_t)d * d));
    LY_TRY(dgemm(bl, CUBLAS_OP_N, CUBLAS_OP_N, n, d, n, 1.0, pj->E.p, n, pj->Vm.p, n, 0.0, EV.p, n));
    LY_TRY(dgemm(bl, CUBLAS_OP_T, CUBLAS_OP_N, d, d, n, 1.0, pj->Vm.p, n, EV.p, n, 0.0, Es.p, d));
  }
  std::unique_ptr<lyap_seed> sd(new lyap_seed());
  sd->ctx = pj->ctx;
  sd->device = pj->device;
  sd->n = d;
  sd->k = k;
  sd->g = 0;
  LY_TRY(lyap_seed_build(pj->ctx, sd.get(), At.p, Us.p, Vs.p, nullptr, pj->has_E ? Es.p : nullptr, st, P1s.p));
  lk.unlock();
  LY_TRY(lyap_seed_finish(sd.get(), std::min(o.pbar, d * k), o.precision == LYAP_BF16_IR, st));
  pj->small = sd.release();
  pj->small_m = mm;
  pj->small_prec = o.precision;
  pj->small_pbar = o.pbar;
  return LYAP_OK;
}

}  // namespace

extern "C" int lyap_proj_create(lyap_ctx* ctx, int n, int k, int g, const double* A0, const double* U,
                                const double* V, const double* G, const double* E, const double* XBr, double fX0,
                                int mem_kind, const lyap_opts* opts, lyap_proj** out) {
  if (!ctx || !out || !A0 || !U || !V || n < 1 || k < 1 || k > 8 || 2 * k > n) return LYAP_EINVAL;
  if (!XBr && (!G || g < 1)) return LYAP_EINVAL;
  if (mem_kind != LYAP_MEM_HOST && mem_kind != LYAP_MEM_DEVICE) return LYAP_EINVAL;
  *out = nullptr;
  lyap_opts o;
  lyap_opts_default(&o);
  if (opts) o = *opts;
  (void)cudaGetLastError();
  LY_CUDA(cudaSetDevice(ctx->device));
  cudaStream_t st = o.stream ? static_cast<cudaStream_t>(o.stream) : ctx->stream;
  std::lock_guard<std::mutex> lk(ctx->handle_mu);
  LY_BLAS(cublasSetStream(ctx->blas, st));
  LY_SOLVER(cusolverDnSetStream(ctx->solver, st));
  std::unique_ptr<lyap_proj> pj(new lyap_proj());
  pj->ctx = ctx;
  pj->device = ctx->device;
  pj->n = n;
  pj->k = k;
  pj->has_E = E != nullptr;
  const size_t nn = (size_t)n * n;
  const cudaMemcpyKind kind = mem_kind == LYAP_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  LY_TRY(pj->A0.alloc(nn));
  LY_TRY(pj->U.alloc((size_t)n * k));
  LY_TRY(pj->V.alloc((size_t)n * k));
  LY_TRY(pj->XBr.alloc((size_t)n * k));
  LY_TRY(pj->P.alloc((size_t)n * 2 * k));
  LY_TRY(pj->work.alloc((size_t)n * 2 * k));
  LY_TRY(pj->info.alloc(1));
  LY_CUDA(cudaMemcpyAsync(pj->A0.p, A0, nn * sizeof(double), kind, st));
  LY_CUDA(cudaMemcpyAsync(pj->U.p, U, (size_t)n * k * sizeof(double), kind, st));
  LY_CUDA(cudaMemcpyAsync(pj->V.p, V, (size_t)n * k * sizeof(double), kind, st));
  if (E) {
    LY_TRY(pj->E.alloc(nn));
    LY_CUDA(cudaMemcpyAsync(pj->E.p, E, nn * sizeof(double), kind, st));
  }
  if (XBr) {
    LY_CUDA(cudaMemcpyAsync(pj->XBr.p, XBr, (size_t)n * k * sizeof(double), kind, st));
    pj->f0 = fX0;
  } else {
    // X0 B_r and f(X0) from the small-scale seed factorisation (FP64):
    // X0 B_r = Qp (X0h Vb) = Qp Ph
    DevBuf<double> dG;
    const double* pG = G;
    if (mem_kind == LYAP_MEM_HOST) {
      LY_TRY(dG.alloc((size_t)n * g));
      LY_CUDA(cudaMemcpyAsync(dG.p, G, (size_t)n * g * sizeof(double), cudaMemcpyHostToDevice, st));
      pG = dG.p;
    }
    lyap_seed tmp;
    tmp.ctx = ctx;
    tmp.device = ctx->device;
    tmp.n = n;
    tmp.k = k;
    tmp.g = g;
    LY_TRY(lyap_seed_build(ctx, &tmp, pj->A0.p, pj->U.p, pj->V.p, pG, pj->has_E ? pj->E.p : nullptr, st));
    DevBuf<double2> xb;
    LY_TRY(xb.alloc((size_t)n * k));
    const cuDoubleComplex one = make_cuDoubleComplex(1.0, 0.0), zero = make_cuDoubleComplex(0.0, 0.0);
    LY_BLAS(cublasZgemm(ctx->blas, CUBLAS_OP_N, CUBLAS_OP_N, n, k, n, &one,
                        reinterpret_cast<const cuDoubleComplex*>(tmp.Qp.p), n,
                        reinterpret_cast<const cuDoubleComplex*>(tmp.Ph.p), n, &zero,
                        reinterpret_cast<cuDoubleComplex*>(xb.p), n));
    // real part (the imaginary part is rounding for a real A0)
    LY_BLAS(cublasDcopy(ctx->blas, n * k, reinterpret_cast<const double*>(xb.p), 2, pj->XBr.p, 1));
    pj->f0 = tmp.f0;
  }
  // P = [X0 B_r, B_l]
  LY_CUDA(cudaMemcpyAsync(pj->P.p, pj->XBr.p, (size_t)n * k * sizeof(double), cudaMemcpyDeviceToDevice, st));
  LY_CUDA(cudaMemcpyAsync(pj->P.p + (size_t)n * k, pj->V.p, (size_t)n * k * sizeof(double), cudaMemcpyDeviceToDevice,
                          st));
  // offline scalars of the backward error
  {
    LY_BLAS(cublasDnrm2(ctx->blas, (int)std::min<size_t>(nn, 0x7fffffff), pj->A0.p, 1, &pj->normA0));
    DevBuf<double> BB, AV, BAB, PP;
    LY_TRY(BB.alloc((size_t)k * k));
    LY_TRY(AV.alloc((size_t)n * k));
    LY_TRY(BAB.alloc((size_t)k * k));
    LY_TRY(PP.alloc((size_t)4 * k * k));
    // B_r^T B_l = U^T V; B_r^T A0p B_l = U^T A0^T V
    LY_TRY(dgemm(ctx->blas, CUBLAS_OP_T, CUBLAS_OP_N, k, k, n, 1.0, pj->U.p, n, pj->V.p, n, 0.0, BB.p, k));
    LY_TRY(dgemm(ctx->blas, CUBLAS_OP_T, CUBLAS_OP_N, n, k, n, 1.0, pj->A0.p, n, pj->V.p, n, 0.0, AV.p, n));
    LY_TRY(dgemm(ctx->blas, CUBLAS_OP_T, CUBLAS_OP_N, k, k, n, 1.0, pj->U.p, n, AV.p, n, 0.0, BAB.p, k));
    LY_TRY(dgemm(ctx->blas, CUBLAS_OP_T, CUBLAS_OP_N, 2 * k, 2 * k, n, 1.0, pj->P.p, n, pj->P.p, n, 0.0, PP.p, 2 * k));
    std::vector<double> hbb((size_t)k * k), hbab((size_t)k * k);
    pj->PtP.resize((size_t)4 * k * k);
    LY_CUDA(cudaMemcpyAsync(hbb.data(), BB.p, sizeof(double) * k * k, cudaMemcpyDeviceToHost, st));
    LY_CUDA(cudaMemcpyAsync(hbab.data(), BAB.p, sizeof(double) * k * k, cudaMemcpyDeviceToHost, st));
    LY_CUDA(cudaMemcpyAsync(pj->PtP.data(), PP.p, sizeof(double) * 4 * k * k, cudaMemcpyDeviceToHost, st));
    LY_CUDA(cudaStreamSynchronize(st));
    pj->H.resize((size_t)k * k);
    pj->a.resize(k);
    for (int i = 0; i < k * k; ++i) pj->H[i] = hbb[i] * hbb[i];
    for (int i = 0; i < k; ++i) pj->a[i] = hbab[(size_t)i * k + i];
  }
  // LU of A0 (Assumption 3)
  {
    LY_TRY(pj->LU.alloc(nn));
    LY_TRY(pj->ipiv.alloc(n));
    LY_CUDA(cudaMemcpyAsync(pj->LU.p, pj->A0.p, nn * sizeof(double), cudaMemcpyDeviceToDevice, st));
    int lwork = 0;
    LY_SOLVER(cusolverDnDgetrf_bufferSize(ctx->solver, n, n, pj->LU.p, n, &lwork));
    DevBuf<double> wk;
    LY_TRY(wk.alloc(lwork > 0 ? lwork : 1));
    LY_SOLVER(cusolverDnDgetrf(ctx->solver, n, n, pj->LU.p, n, wk.p, pj->ipiv.p, pj->info.p));
    int hinfo = 0;
    LY_CUDA(cudaMemcpyAsync(&hinfo, pj->info.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    LY_CUDA(cudaStreamSynchronize(st));
    if (hinfo != 0) {
      lyap_set_last_error("A0 is singular (getrf info " + std::to_string(hinfo) + ")");
      return LYAP_EUNSTABLE_SEED;
    }
  }
  LY_TRY(first_block(pj.get(), st));
  *out = pj.release();
  return LYAP_OK;
}

extern "C" int lyap_proj_free(lyap_proj* pj) {
  if (!pj) return LYAP_EINVAL;
  cudaSetDevice(pj->device);
  delete pj;
  return LYAP_OK;
}

extern "C" int lyap_proj_dims(const lyap_proj* pj, int* blocks, int* dim) {
  if (!pj) return LYAP_EINVAL;
  if (blocks) *blocks = (int)pj->split.size();
  if (dim) *dim = pj->dim;
  return LYAP_OK;
}

extern "C" int lyap_proj_trace_EX(lyap_proj* pj, int nv, const double* v, int mem_kind, const lyap_opts* opts,
                                  double eps, int m_max, double* trace_out, double* delta_out, int* blocks_out,
                                  lyap_result_info* info) {
  if (!pj || nv < 0 || (nv > 0 && (!v || !trace_out)) || !(eps > 0.0) || m_max < 2) return LYAP_EINVAL;
  if (mem_kind != LYAP_MEM_HOST && mem_kind != LYAP_MEM_DEVICE) return LYAP_EINVAL;
  if (nv == 0) return LYAP_OK;
  lyap_opts o;
  lyap_opts_default(&o);
  if (opts) o = *opts;
  if (o.precision != LYAP_FP64 && o.precision != LYAP_BF16_IR) return LYAP_EINVAL;
  (void)cudaGetLastError();
  LY_CUDA(cudaSetDevice(pj->device));
  cudaStream_t st = o.stream ? static_cast<cudaStream_t>(o.stream) : pj->ctx->stream;
  const int k = pj->k;
  // the algorithm is driven from the host: parameters and results pass through it
  std::vector<double> hv((size_t)nv * k);
  if (mem_kind == LYAP_MEM_HOST) {
    std::memcpy(hv.data(), v, sizeof(double) * hv.size());
  } else {
    LY_CUDA(cudaMemcpyAsync(hv.data(), v, sizeof(double) * hv.size(), cudaMemcpyDeviceToHost, st));
    LY_CUDA(cudaStreamSynchronize(st));
  }
  LY_TRY(lyap_check_v(nv, k, hv.data()));
  std::vector<double> f(nv, NAN), dl(nv, NAN);
  std::vector<int> mused(nv, 0);
  std::vector<lyap_result_info> inf(nv);
  for (auto& x : inf) {
    x.iters = 0;
    x.refine_steps = 0;
    x.status = LYAP_ENOCONV;
    x.rel_resid = NAN;
    x.err_est = NAN;
  }
  std::vector<int> remaining(nv);
  for (int i = 0; i < nv; ++i) remaining[i] = i;
  const int chunk = 512;
  DevBuf<double> dv, Wd, R, Yr, RY, nY, nRY, fs;
  DevBuf<double2> L1, L2;
  lyap_opts os = o;
  os.stream = st;
  for (int m = 1; m < m_max && !remaining.empty(); ++m) {
    {
      std::lock_guard<std::mutex> lk(pj->ctx->handle_mu);
      LY_BLAS(cublasSetStream(pj->ctx->blas, st));
      LY_SOLVER(cusolverDnSetStream(pj->ctx->solver, st));
      LY_TRY(ensure_blocks(pj, m, st));
    }
    LY_TRY(build_small(pj, m, o, st));
    const int mm = pj->small_m;
    const int d = pj->off[mm];
    const bool last_block = mm >= (int)pj->split.size();  // no next block: the space has ended
    const int r = last_block ? 0 : pj->off[mm + 1] - d;
    lyap_seed* sd = pj->small;
    const size_t dd = (size_t)d * d;
    // E_m^T underline(T)_m = V_{next}^T (A0p V_m)   (r x d)
    if (r > 0) {
      if (R.count < (size_t)r * d) LY_TRY(R.alloc((size_t)r * d));
      std::lock_guard<std::mutex> lk(pj->ctx->handle_mu);
      LY_BLAS(cublasSetStream(pj->ctx->blas, st));
      LY_TRY(dgemm(pj->ctx->blas, CUBLAS_OP_T, CUBLAS_OP_N, r, d, pj->n, 1.0, pj->Vm.p + (size_t)d * pj->n, pj->n,
                   pj->AVm.p, pj->n, 0.0, R.p, r));
    }
    std::vector<int> keep;
    for (size_t c0 = 0; c0 < remaining.size(); c0 += chunk) {
      const int nb = (int)std::min<size_t>(chunk, remaining.size() - c0);
      std::vector<double> vb((size_t)nb * k);
      for (int b = 0; b < nb; ++b)
        std::memcpy(vb.data() + (size_t)b * k, hv.data() + (size_t)remaining[c0 + b] * k, sizeof(double) * k);
      if (dv.count < (size_t)nb * k) LY_TRY(dv.alloc((size_t)chunk * k));
      if (Wd.count < (size_t)nb * d * k * 2) LY_TRY(Wd.alloc((size_t)chunk * d * k * 2));
      if (L1.count < (size_t)nb * dd) {
        LY_TRY(L1.alloc((size_t)nb * dd));
        LY_TRY(L2.alloc((size_t)nb * dd));
        LY_TRY(Yr.alloc((size_t)nb * dd));
      }
      if (RY.count < (size_t)nb * std::max(r, 1) * d) LY_TRY(RY.alloc((size_t)nb * std::max(r, 1) * d));
      if (nY.count < (size_t)nb) {
        LY_TRY(nY.alloc(chunk));
        LY_TRY(nRY.alloc(chunk));
        LY_TRY(fs.alloc(chunk));
      }
      LY_CUDA(cudaMemcpyAsync(dv.p, vb.data(), sizeof(double) * vb.size(), cudaMemcpyHostToDevice, st));
      std::vector<lyap_result_info> si(nb);
      LY_TRY(lyap_param_solve(sd, nb, dv.p, LYAP_MEM_DEVICE, &os, Wd.p, si.data()));
      const double2* W2 = reinterpret_cast<const double2*>(Wd.p);
      // f_small = <h, W'>; Y = Qp (Lc o (W' Ub^T + Ub W'^T)) Qp^T
      kry::k_dot_h<double2><<<nb, kry::NT, 0, st>>>(d * k, nb, W2, (size_t)d * k, sd->h.p, fs.p, nullptr);
      lyap_count_launch();
      k_proj_hadamard<<<dim3(gridsz(dd), nb), 256, 0, st>>>(d, k, nb, sd->lam.p, sd->Ub.p, W2, L1.p);
      lyap_count_launch();
      LY_CUDA(cudaGetLastError());
      {
        std::lock_guard<std::mutex> lk(pj->ctx->handle_mu);
        cublasHandle_t bl = pj->ctx->blas;
        LY_BLAS(cublasSetStream(bl, st));
        const cuDoubleComplex one = make_cuDoubleComplex(1.0, 0.0), zero = make_cuDoubleComplex(0.0, 0.0);
        LY_BLAS(cublasZgemmStridedBatched(bl, CUBLAS_OP_N, CUBLAS_OP_N, d, d, d, &one,
                                          reinterpret_cast<const cuDoubleComplex*>(sd->Qp.p), d, 0,
                                          reinterpret_cast<const cuDoubleComplex*>(L1.p), d, dd, &zero,
                                          reinterpret_cast<cuDoubleComplex*>(L2.p), d, dd, nb));
        LY_BLAS(cublasZgemmStridedBatched(bl, CUBLAS_OP_N, CUBLAS_OP_T, d, d, d, &one,
                                          reinterpret_cast<const cuDoubleComplex*>(L2.p), d, dd,
                                          reinterpret_cast<const cuDoubleComplex*>(sd->Qp.p), d, 0, &zero,
                                          reinterpret_cast<cuDoubleComplex*>(L1.p), d, dd, nb));
        k_proj_real<<<nb, kry::NT, 0, st>>>(d, nb, L1.p, Yr.p, nY.p);
        lyap_count_launch();
        if (r > 0) {
          const double alpha = 1.0, beta = 0.0;
          LY_BLAS(cublasDgemmStridedBatched(bl, CUBLAS_OP_N, CUBLAS_OP_N, r, d, d, &alpha, R.p, r, 0, Yr.p, d, dd,
                                            &beta, RY.p, r, (long long)r * d, nb));
          k_proj_sqnorm<<<nb, kry::NT, 0, st>>>((size_t)r * d, nb, RY.p, nRY.p);
          lyap_count_launch();
        } else {
          LY_CUDA(cudaMemsetAsync(nRY.p, 0, sizeof(double) * nb, st));
        }
        LY_CUDA(cudaGetLastError());
      }
      std::vector<double> hy(nb), hry(nb), hf(nb);
      LY_CUDA(cudaMemcpyAsync(hy.data(), nY.p, sizeof(double) * nb, cudaMemcpyDeviceToHost, st));
      LY_CUDA(cudaMemcpyAsync(hry.data(), nRY.p, sizeof(double) * nb, cudaMemcpyDeviceToHost, st));
      LY_CUDA(cudaMemcpyAsync(hf.data(), fs.p, sizeof(double) * nb, cudaMemcpyDeviceToHost, st));
      LY_CUDA(cudaStreamSynchronize(st));
      for (int b = 0; b < nb; ++b) {
        const int i = remaining[c0 + b];
        const double* x = hv.data() + (size_t)i * k;
        // ||A(v)||_F^2 = ||A0||^2 + v^T H v - 2 a^T v
        double na2 = pj->normA0 * pj->normA0;
        for (int p = 0; p < k; ++p) {
          na2 -= 2.0 * pj->a[p] * x[p];
          for (int q = 0; q < k; ++q) na2 += x[p] * pj->H[(size_t)q * k + p] * x[q];
        }
        // ||P (I2 (x) D) P^T||_F^2 = trace(M PtP M PtP), M = I2 (x) D
        const int k2 = 2 * k;
        std::vector<double> MG((size_t)k2 * k2);  // M * PtP
        for (int row = 0; row < k2; ++row) {
          const int src = row < k ? row + k : row - k;  // M swaps the halves and scales by v
          const double s = x[row < k ? row : row - k];
          for (int col = 0; col < k2; ++col) MG[(size_t)col * k2 + row] = s * pj->PtP[(size_t)col * k2 + src];
        }
        double rhs2 = 0.0;
        for (int p = 0; p < k2; ++p)
          for (int q = 0; q < k2; ++q) rhs2 += MG[(size_t)q * k2 + p] * MG[(size_t)p * k2 + q];
        const double den = 2.0 * std::sqrt(std::max(na2, 0.0)) * std::sqrt(hy[b]) + std::sqrt(std::max(rhs2, 0.0));
        const double delta = den > 0 ? std::sqrt(2.0) * std::sqrt(hry[b]) / den : 0.0;
        f[i] = pj->f0 + hf[b];
        dl[i] = delta;
        mused[i] = mm;
        inf[i].iters += si[b].iters;
        inf[i].refine_steps += si[b].refine_steps;
        inf[i].rel_resid = si[b].rel_resid;
        inf[i].err_est = delta;
        const bool solved = si[b].status == LYAP_OK;
        if (solved && (delta <= eps || last_block)) {
          inf[i].status = LYAP_OK;
        } else {
          inf[i].status = solved ? LYAP_ENOCONV : si[b].status;
          keep.push_back(i);
        }
      }
    }
    remaining.swap(keep);
    if (pj->exhausted && mm >= (int)pj->split.size()) break;
  }
  if (info) std::memcpy(info, inf.data(), sizeof(lyap_result_info) * nv);
  if (delta_out) std::memcpy(delta_out, dl.data(), sizeof(double) * nv);
  if (blocks_out) std::memcpy(blocks_out, mused.data(), sizeof(int) * nv);
  if (mem_kind == LYAP_MEM_HOST) {
    std::memcpy(trace_out, f.data(), sizeof(double) * nv);
  } else {
    LY_CUDA(cudaMemcpyAsync(trace_out, f.data(), sizeof(double) * nv, cudaMemcpyHostToDevice, st));
    LY_CUDA(cudaStreamSynchronize(st));
  }
  return LYAP_OK;
}
