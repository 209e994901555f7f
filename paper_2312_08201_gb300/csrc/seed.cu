// Offline seed factorisation and precomputation (paper §2.1, Table 1
// "offline" column), all on the device in FP64.
//
// In the paper's convention (A_p = A0^T, B_l = V, B_r = U, Q = G G^T):
//   eig:   A_p = Qp diag(lam) Qp^{-1},  Qi = Qp^{-1}                   (§2.1)
//   Lc_ij = 1 / (lam_i + lam_j)                                        (eq. (Z(v)))
//   Ub = Qi B_l,  Vb = Qp^T B_r                                        (M, N of eq. (deltaX_SMW2))
//   seed solution in eigen-coordinates (eq. (seedLE)):
//        X0h = Qi X0 Qi^T = -Lc o (Gh Gh^T),  Gh = Qi G
//   capacitance right-hand side: N^T vec(X0h) = [vec(X0h Vb); vec(Vb^T X0h)];
//        the shifted unknown W' = W + P D(v) satisfies
//        (D(v)^{-1} - N^T L0^{-1} M) w' = N^T vec(X0h), a v-independent
//        right-hand side (derivation in the design notes); only the n x k
//        block Ph = X0h Vb is stored because the solution lies in the
//        subspace W2 = W1^T (the Lyapunov solution is symmetric).
//   trace: f = trace(E X0) + trace(Eh (Lc o (W' Ub^T + Ub W'^T))),
//        Eh = Qp^T sym(E) Qp, so f = f0 + <h, W'> with h = 2 (Eh o Lc) Ub.
//   diagonal blocks of N^T L0^{-1} M (eq. (N1M1)): Gd[:, p, t] = Lc (Ub_p o Vb_t).
#include "cplx.cuh"
#include "lyap_internal.h"
#include "prof.h"

#include <cmath>
#include <vector>

namespace {

__global__ void k_transpose_to_complex(int n, const double* __restrict__ A, double2* __restrict__ out) {
  // out = A^T (column-major), imaginary part zero
  size_t total = (size_t)n * n;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
    size_t i = idx % n, j = idx / n;
    out[idx] = make_double2(A[j + i * (size_t)n], 0.0);
  }
}

// part[blk] = (sum (A - A^T)^2, sum A^2) partial sums, fixed order
__global__ void k_asym_partial(int n, const double* __restrict__ A, double* __restrict__ part) {
  __shared__ double s0[256], s1[256];
  double a = 0.0, b = 0.0;
  const size_t total = (size_t)n * n;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
    const size_t i = idx % n, j = idx / n;
    const double x = A[idx], d = x - A[j + i * (size_t)n];
    a += d * d;
    b += x * x;
  }
  s0[threadIdx.x] = a;
  s1[threadIdx.x] = b;
  __syncthreads();
  for (int st = 128; st > 0; st >>= 1) {
    if (threadIdx.x < st) {
      s0[threadIdx.x] += s0[threadIdx.x + st];
      s1[threadIdx.x] += s1[threadIdx.x + st];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = s0[0];
    part[2 * blockIdx.x + 1] = s1[0];
  }
}

// Orthogonal eigenvectors V (real, n x n): Qp = V, Qi = V^T; lam = w (real).
__global__ void k_from_symmetric(int n, const double* __restrict__ V, const double* __restrict__ w,
                                 double2* __restrict__ Qp, double2* __restrict__ Qi, double2* __restrict__ lam) {
  const size_t total = (size_t)n * n;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
    const size_t i = idx % n, j = idx / n;
    Qp[idx] = make_double2(V[idx], 0.0);
    Qi[idx] = make_double2(V[j + i * (size_t)n], 0.0);
    if (j == 0) lam[i] = make_double2(w[i], 0.0);
  }
}

__global__ void k_real_to_complex(size_t count, const double* __restrict__ in, double2* __restrict__ out) {
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < count; idx += (size_t)gridDim.x * blockDim.x)
    out[idx] = make_double2(in[idx], 0.0);
}

__global__ void k_sym_to_complex(int n, const double* __restrict__ E, double2* __restrict__ out) {
  size_t total = (size_t)n * n;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
    size_t i = idx % n, j = idx / n;
    out[idx] = make_double2(0.5 * (E[idx] + E[j + i * (size_t)n]), 0.0);
  }
}

__global__ void k_identity(int n, double2* __restrict__ out) {
  size_t total = (size_t)n * n;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
    size_t i = idx % n, j = idx / n;
    out[idx] = make_double2(i == j ? 1.0 : 0.0, 0.0);
  }
}

// M[i,j] *= scale / (lam_i + lam_j)
__global__ void k_cauchy_hadamard(int n, const double2* __restrict__ lam, double2* __restrict__ M, double scale) {
  size_t total = (size_t)n * n;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
    size_t i = idx % n, j = idx / n;
    double2 z = cadd(lam[i], lam[j]);
    M[idx] = cscale(cmul(M[idx], crcp(z)), scale);
  }
}

__global__ void k_fill_cauchy(int n, const double2* __restrict__ lam, double2* __restrict__ L) {
  size_t total = (size_t)n * n;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
    size_t i = idx % n, j = idx / n;
    L[idx] = crcp(cadd(lam[i], lam[j]));
  }
}

// out = in rounded to FP32
__global__ void k_round_f32(size_t count, const double2* __restrict__ in, float2* __restrict__ out) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x)
    out[i] = make_float2((float)in[i].x, (float)in[i].y);
}

// Y[:, p*k + t] = Ub[:, p] o Vb[:, t]
__global__ void k_panel_products(int n, int k, const double2* __restrict__ Ub, const double2* __restrict__ Vb,
                                 double2* __restrict__ Y) {
  size_t total = (size_t)n * k * k;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
    size_t i = idx % n, col = idx / n;
    int p = (int)(col / k), t = (int)(col % k);
    Y[idx] = cmul(Ub[i + (size_t)p * n], Vb[i + (size_t)t * n]);
  }
}

// Deterministic block partial sums (fixed grid, fixed tree) of Re(a o b),
// |a|^2 (mode 1), or min/max statistics of lam.
constexpr int RED_THREADS = 256;
constexpr int RED_BLOCKS = 256;

__global__ void k_partial_dot_re(size_t count, const double2* __restrict__ a, const double2* __restrict__ b,
                                 double* __restrict__ part) {
  __shared__ double sm[RED_THREADS];
  double acc = 0.0;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < count; idx += (size_t)gridDim.x * blockDim.x) {
    double2 x = a[idx];
    double2 y = b ? b[idx] : cconj(x);
    acc += x.x * y.x - x.y * y.y;
  }
  sm[threadIdx.x] = acc;
  __syncthreads();
  for (int s = RED_THREADS / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sm[threadIdx.x] += sm[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sm[0];
}

__global__ void k_finish_sum(int count, const double* __restrict__ part, double* __restrict__ out) {
  __shared__ double sm[RED_THREADS];
  double acc = 0.0;
  for (int i = threadIdx.x; i < count; i += blockDim.x) acc += part[i];
  sm[threadIdx.x] = acc;
  __syncthreads();
  for (int s = RED_THREADS / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sm[threadIdx.x] += sm[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = sm[0];
}

// out[0] = max Re lam, out[1] = min |lam_i + lam_j|, out[2] = max |lam|, out[3] = max |Im lam|
__global__ void k_lambda_stats(int n, const double2* __restrict__ lam, double* __restrict__ out) {
  __shared__ double smax[RED_THREADS], smin[RED_THREADS], sabs[RED_THREADS], sim[RED_THREADS];
  double mx = -INFINITY, mn = INFINITY, ab = 0.0, im = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    double2 li = lam[i];
    mx = fmax(mx, li.x);
    ab = fmax(ab, sqrt(cabs2(li)));
    im = fmax(im, fabs(li.y));
    for (int j = 0; j < n; ++j) mn = fmin(mn, cabs2(cadd(li, lam[j])));
  }
  smax[threadIdx.x] = mx;
  smin[threadIdx.x] = mn;
  sabs[threadIdx.x] = ab;
  sim[threadIdx.x] = im;
  __syncthreads();
  for (int s = RED_THREADS / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      smax[threadIdx.x] = fmax(smax[threadIdx.x], smax[threadIdx.x + s]);
      smin[threadIdx.x] = fmin(smin[threadIdx.x], smin[threadIdx.x + s]);
      sabs[threadIdx.x] = fmax(sabs[threadIdx.x], sabs[threadIdx.x + s]);
      sim[threadIdx.x] = fmax(sim[threadIdx.x], sim[threadIdx.x + s]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[0] = smax[0];
    out[1] = sqrt(smin[0]);
    out[2] = sabs[0];
    out[3] = sim[0];
  }
}

int grid_for(size_t count) {
  size_t g = (count + 255) / 256;
  if (g > 4096) g = 4096;
  if (g < 1) g = 1;
  return (int)g;
}

int zgemm(cublasHandle_t h, cublasOperation_t ta, cublasOperation_t tb, int m, int n, int k, double2 alpha,
          const double2* A, int lda, const double2* B, int ldb, double2 beta, double2* C, int ldc) {
  LY_BLAS(cublasZgemm(h, ta, tb, m, n, k, reinterpret_cast<const cuDoubleComplex*>(&alpha),
                      reinterpret_cast<const cuDoubleComplex*>(A), lda, reinterpret_cast<const cuDoubleComplex*>(B),
                      ldb, reinterpret_cast<const cuDoubleComplex*>(&beta), reinterpret_cast<cuDoubleComplex*>(C),
                      ldc));
  return LYAP_OK;
}

int re_dot(const double2* a, const double2* b, size_t count, double* out_host, cudaStream_t st) {
  DevBuf<double> part, res;
  LY_TRY(part.alloc(RED_BLOCKS));
  LY_TRY(res.alloc(1));
  k_partial_dot_re<<<RED_BLOCKS, RED_THREADS, 0, st>>>(count, a, b, part.p); lyap_count_launch();
  k_finish_sum<<<1, RED_THREADS, 0, st>>>(RED_BLOCKS, part.p, res.p); lyap_count_launch();
  LY_CUDA(cudaGetLastError());
  LY_CUDA(cudaMemcpyAsync(out_host, res.p, sizeof(double), cudaMemcpyDeviceToHost, st));
  LY_CUDA(cudaStreamSynchronize(st));
  return LYAP_OK;
}

}  // namespace

int lyap_seed_build(lyap_ctx* ctx, lyap_seed* sd, const double* A0, const double* U, const double* V,
                    const double* G, const double* E, cudaStream_t st, const double* P1) {
  const int n = sd->n, k = sd->k, g = sd->g;
  const size_t nn = (size_t)n * n;
  LY_BLAS(cublasSetStream(ctx->blas, st));
  LY_SOLVER(cusolverDnSetStream(ctx->solver, st));
  const double2 one = make_double2(1.0, 0.0), zero = make_double2(0.0, 0.0);

  LY_TRY(sd->lam.alloc(n));
  LY_TRY(sd->Qp.alloc(nn));
  LY_TRY(sd->Qi.alloc(nn));
  DevBuf<double2> W1, W2;
  LY_TRY(W1.alloc(nn));
  LY_TRY(W2.alloc(nn));

  // ---- symmetric A0: orthogonal eigenvectors from the symmetric solver ----
  bool symmetric = false;
  {
    DevBuf<double> part;
    LY_TRY(part.alloc(2 * RED_BLOCKS));
    k_asym_partial<<<RED_BLOCKS, RED_THREADS, 0, st>>>(n, A0, part.p);
    lyap_count_launch();
    LY_CUDA(cudaGetLastError());
    std::vector<double> hp(2 * RED_BLOCKS);
    LY_CUDA(cudaMemcpyAsync(hp.data(), part.p, sizeof(double) * hp.size(), cudaMemcpyDeviceToHost, st));
    LY_CUDA(cudaStreamSynchronize(st));
    double asym = 0, nrm = 0;
    for (int b = 0; b < RED_BLOCKS; ++b) {
      asym += hp[2 * b];
      nrm += hp[2 * b + 1];
    }
    symmetric = asym <= 1e-28 * nrm;
  }
  if (symmetric) {
    // A_p = A0^T = A0 = V diag(w) V^T: Qp = V, Qp^{-1} = V^T (repeated
    // eigenvalues keep an orthonormal basis, unlike a general eigensolver)
    DevBuf<double> Vr, w, work;
    DevBuf<int> dinfo;
    LY_TRY(Vr.alloc(nn));
    LY_TRY(w.alloc(n));
    LY_TRY(dinfo.alloc(1));
    LY_CUDA(cudaMemcpyAsync(Vr.p, A0, nn * sizeof(double), cudaMemcpyDeviceToDevice, st));
    int lwork = 0;
    LY_SOLVER(cusolverDnDsyevd_bufferSize(ctx->solver, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, n, Vr.p, n,
                                          w.p, &lwork));
    LY_TRY(work.alloc(lwork > 0 ? lwork : 1));
    LY_SOLVER(cusolverDnDsyevd(ctx->solver, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, n, Vr.p, n, w.p, work.p,
                               lwork, dinfo.p));
    int info = 0;
    LY_CUDA(cudaMemcpyAsync(&info, dinfo.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    LY_CUDA(cudaStreamSynchronize(st));
    if (info != 0) {
      lyap_set_last_error("syevd info = " + std::to_string(info));
      return LYAP_ESOLVER;
    }
    k_from_symmetric<<<grid_for(nn), 256, 0, st>>>(n, Vr.p, w.p, sd->Qp.p, sd->Qi.p, sd->lam.p);
    lyap_count_launch();
    LY_CUDA(cudaGetLastError());
    sd->real_arith = 1;
  } else {
    // ---- eig(A_p), A_p = A0^T (complex FP64, right eigenvectors) ----------
    k_transpose_to_complex<<<grid_for(nn), 256, 0, st>>>(n, A0, W1.p); lyap_count_launch();
    LY_CUDA(cudaGetLastError());
    {
      cusolverDnParams_t params;
      LY_SOLVER(cusolverDnCreateParams(&params));
      size_t dws = 0, hws = 0;
      cusolverStatus_t s1 = cusolverDnXgeev_bufferSize(
          ctx->solver, params, CUSOLVER_EIG_MODE_NOVECTOR, CUSOLVER_EIG_MODE_VECTOR, n, CUDA_C_64F, W1.p, n,
          CUDA_C_64F, sd->lam.p, CUDA_C_64F, nullptr, 1, CUDA_C_64F, sd->Qp.p, n, CUDA_C_64F, &dws, &hws);
      if (s1 != CUSOLVER_STATUS_SUCCESS) {
        cusolverDnDestroyParams(params);
        lyap_set_last_error("cusolverDnXgeev_bufferSize failed: " + std::to_string(s1));
        return LYAP_ESOLVER;
      }
      DevBuf<char> dwork;
      DevBuf<int> dinfo;
      int rc = dwork.alloc(dws ? dws : 1);
      if (rc == LYAP_OK) rc = dinfo.alloc(1);
      if (rc != LYAP_OK) {
        cusolverDnDestroyParams(params);
        return rc;
      }
      std::vector<char> hwork(hws ? hws : 1);
      cusolverStatus_t s2 = cusolverDnXgeev(ctx->solver, params, CUSOLVER_EIG_MODE_NOVECTOR, CUSOLVER_EIG_MODE_VECTOR,
                                            n, CUDA_C_64F, W1.p, n, CUDA_C_64F, sd->lam.p, CUDA_C_64F, nullptr, 1,
                                            CUDA_C_64F, sd->Qp.p, n, CUDA_C_64F, dwork.p, dws, hwork.data(), hws,
                                            dinfo.p);
      cusolverDnDestroyParams(params);
      if (s2 != CUSOLVER_STATUS_SUCCESS) {
        lyap_set_last_error("cusolverDnXgeev failed: " + std::to_string(s2));
        return LYAP_ESOLVER;
      }
      int info = 0;
      LY_CUDA(cudaMemcpyAsync(&info, dinfo.p, sizeof(int), cudaMemcpyDeviceToHost, st));
      LY_CUDA(cudaStreamSynchronize(st));
      if (info != 0) {
        lyap_set_last_error("geev info = " + std::to_string(info));
        return LYAP_ESOLVER;
      }
    }

  }
  // ---- stability and uniqueness -----------------------------------------
  {
    DevBuf<double> stats;
    LY_TRY(stats.alloc(4));
    k_lambda_stats<<<1, RED_THREADS, 0, st>>>(n, sd->lam.p, stats.p); lyap_count_launch();
    LY_CUDA(cudaGetLastError());
    double hs[4];
    LY_CUDA(cudaMemcpyAsync(hs, stats.p, sizeof(hs), cudaMemcpyDeviceToHost, st));
    LY_CUDA(cudaStreamSynchronize(st));
    sd->max_re = hs[0];
    sd->min_sum = hs[1];
    sd->real_path = hs[3] <= 1e-14 * hs[2] ? 1 : 0;
    // A seed built from a given right-hand side factor (a projected
    // equation of §2.2) needs only the uniqueness condition
    // lambda_i + lambda_j != 0, not the stability of its own A0.
    if ((!P1 && !(hs[0] < 0.0)) || !(hs[1] > 1e-12 * hs[2])) {
      lyap_set_last_error("seed A0 is not stable (max Re lambda = " + std::to_string(hs[0]) +
                          ", min |lambda_i + lambda_j| = " + std::to_string(hs[1]) + ")");
      return LYAP_EUNSTABLE_SEED;
    }
  }

  // ---- Qi = Qp^{-1} by LU (general case) ------------------------------------
  if (!symmetric) {
    LY_CUDA(cudaMemcpyAsync(W1.p, sd->Qp.p, nn * sizeof(double2), cudaMemcpyDeviceToDevice, st));
    k_identity<<<grid_for(nn), 256, 0, st>>>(n, sd->Qi.p); lyap_count_launch();
    LY_CUDA(cudaGetLastError());
    int lwork = 0;
    LY_SOLVER(cusolverDnZgetrf_bufferSize(ctx->solver, n, n, reinterpret_cast<cuDoubleComplex*>(W1.p), n, &lwork));
    DevBuf<double2> work;
    DevBuf<int> ipiv, dinfo;
    LY_TRY(work.alloc(lwork > 0 ? lwork : 1));
    LY_TRY(ipiv.alloc(n));
    LY_TRY(dinfo.alloc(1));
    LY_SOLVER(cusolverDnZgetrf(ctx->solver, n, n, reinterpret_cast<cuDoubleComplex*>(W1.p), n,
                               reinterpret_cast<cuDoubleComplex*>(work.p), ipiv.p, dinfo.p));
    LY_SOLVER(cusolverDnZgetrs(ctx->solver, CUBLAS_OP_N, n, n, reinterpret_cast<const cuDoubleComplex*>(W1.p), n,
                               ipiv.p, reinterpret_cast<cuDoubleComplex*>(sd->Qi.p), n, dinfo.p));
    int info = 0;
    LY_CUDA(cudaMemcpyAsync(&info, dinfo.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    LY_CUDA(cudaStreamSynchronize(st));
    if (info != 0) {
      lyap_set_last_error("eigenvector matrix is singular (getrf/getrs info " + std::to_string(info) + ")");
      return LYAP_EUNSTABLE_SEED;
    }
  }
  {
    double nq = 0, ni = 0;
    LY_TRY(re_dot(sd->Qp.p, nullptr, nn, &nq, st));
    LY_TRY(re_dot(sd->Qi.p, nullptr, nn, &ni, st));
    sd->cond_Q = std::sqrt(nq) * std::sqrt(ni);
  }

  // ---- projected data ------------------------------------------------------
  DevBuf<double2> Vc, Uc, Gc;
  LY_TRY(Vc.alloc((size_t)n * k));
  LY_TRY(Uc.alloc((size_t)n * k));
  k_real_to_complex<<<grid_for((size_t)n * k), 256, 0, st>>>((size_t)n * k, V, Vc.p); lyap_count_launch();
  k_real_to_complex<<<grid_for((size_t)n * k), 256, 0, st>>>((size_t)n * k, U, Uc.p); lyap_count_launch();
  LY_CUDA(cudaGetLastError());
  LY_TRY(sd->Ub.alloc((size_t)n * k));
  LY_TRY(sd->Vb.alloc((size_t)n * k));
  LY_TRY(zgemm(ctx->blas, CUBLAS_OP_N, CUBLAS_OP_N, n, k, n, one, sd->Qi.p, n, Vc.p, n, zero, sd->Ub.p, n));
  LY_TRY(zgemm(ctx->blas, CUBLAS_OP_T, CUBLAS_OP_N, n, k, n, one, sd->Qp.p, n, Uc.p, n, zero, sd->Vb.p, n));

  LY_TRY(sd->Ph.alloc((size_t)n * k));
  if (P1) {
    // The right-hand side factor's first block is given (P1 = X0 B_r of
    // eq. (rhs_newexpression)): Ph = Qi P1, and f counts only the change
    // X - X0 (f0 = 0). The projected equations of §2.2 are built this way.
    LY_TRY(Gc.alloc((size_t)n * k));
    k_real_to_complex<<<grid_for((size_t)n * k), 256, 0, st>>>((size_t)n * k, P1, Gc.p); lyap_count_launch();
    LY_CUDA(cudaGetLastError());
    LY_TRY(zgemm(ctx->blas, CUBLAS_OP_N, CUBLAS_OP_N, n, k, n, one, sd->Qi.p, n, Gc.p, n, zero, sd->Ph.p, n));
  } else {
    // ---- seed solution in eigen-coordinates: X0h = -Lc o (Gh Gh^T) ---------
    LY_TRY(Gc.alloc((size_t)n * g));
    k_real_to_complex<<<grid_for((size_t)n * g), 256, 0, st>>>((size_t)n * g, G, Gc.p); lyap_count_launch();
    LY_CUDA(cudaGetLastError());
    DevBuf<double2> Gh;
    LY_TRY(Gh.alloc((size_t)n * g));
    LY_TRY(zgemm(ctx->blas, CUBLAS_OP_N, CUBLAS_OP_N, n, g, n, one, sd->Qi.p, n, Gc.p, n, zero, Gh.p, n));
    LY_TRY(zgemm(ctx->blas, CUBLAS_OP_N, CUBLAS_OP_T, n, n, g, one, Gh.p, n, Gh.p, n, zero, W1.p, n));
    k_cauchy_hadamard<<<grid_for(nn), 256, 0, st>>>(n, sd->lam.p, W1.p, -1.0); lyap_count_launch();  // W1 = X0h
    LY_CUDA(cudaGetLastError());
    LY_TRY(zgemm(ctx->blas, CUBLAS_OP_N, CUBLAS_OP_N, n, k, n, one, W1.p, n, sd->Vb.p, n, zero, sd->Ph.p, n));
  }
  {
    double pn = 0;
    LY_TRY(re_dot(sd->Ph.p, nullptr, (size_t)n * k, &pn, st));
    sd->ph_norm = std::sqrt(pn);
  }

  // ---- trace data: Eh = Qp^T sym(E) Qp, f0 = sum Eh o X0h, h = 2 (Eh o Lc) Ub ----
  if (E) {
    k_sym_to_complex<<<grid_for(nn), 256, 0, st>>>(n, E, W2.p); lyap_count_launch();
    LY_CUDA(cudaGetLastError());
    DevBuf<double2> W3;
    LY_TRY(W3.alloc(nn));
    LY_TRY(zgemm(ctx->blas, CUBLAS_OP_N, CUBLAS_OP_N, n, n, n, one, W2.p, n, sd->Qp.p, n, zero, W3.p, n));
    LY_TRY(zgemm(ctx->blas, CUBLAS_OP_T, CUBLAS_OP_N, n, n, n, one, sd->Qp.p, n, W3.p, n, zero, W2.p, n));
  } else {
    LY_TRY(zgemm(ctx->blas, CUBLAS_OP_T, CUBLAS_OP_N, n, n, n, one, sd->Qp.p, n, sd->Qp.p, n, zero, W2.p, n));
  }
  if (P1) sd->f0 = 0.0;
  else LY_TRY(re_dot(W2.p, W1.p, nn, &sd->f0, st));  // Eh, X0h symmetric: trace(Eh X0h) = sum Eh o X0h
  k_cauchy_hadamard<<<grid_for(nn), 256, 0, st>>>(n, sd->lam.p, W2.p, 2.0); lyap_count_launch();  // W2 = 2 Eh o Lc
  LY_CUDA(cudaGetLastError());
  LY_TRY(sd->h.alloc((size_t)n * k));
  LY_TRY(zgemm(ctx->blas, CUBLAS_OP_N, CUBLAS_OP_N, n, k, n, one, W2.p, n, sd->Ub.p, n, zero, sd->h.p, n));

  // ---- diagonal blocks Gd[:, p, t] = Lc (Ub_p o Vb_t) ------------------------
  {
    DevBuf<double2> Y;
    LY_TRY(Y.alloc((size_t)n * k * k));
    k_panel_products<<<grid_for((size_t)n * k * k), 256, 0, st>>>(n, k, sd->Ub.p, sd->Vb.p, Y.p); lyap_count_launch();
    k_fill_cauchy<<<grid_for(nn), 256, 0, st>>>(n, sd->lam.p, W1.p); lyap_count_launch();
    LY_CUDA(cudaGetLastError());
    LY_TRY(sd->Gd.alloc((size_t)n * k * k));
    LY_TRY(zgemm(ctx->blas, CUBLAS_OP_N, CUBLAS_OP_N, n, k * k, n, one, W1.p, n, Y.p, n, zero, sd->Gd.p, n));
    LY_TRY(sd->Gdf.alloc((size_t)n * k * k));
    k_round_f32<<<grid_for((size_t)n * k * k), 256, 0, st>>>((size_t)n * k * k, sd->Gd.p, sd->Gdf.p);
    lyap_count_launch();
    LY_CUDA(cudaGetLastError());
  }
  LY_CUDA(cudaStreamSynchronize(st));
  sd->resident_bytes = sd->lam.bytes() + sd->Qp.bytes() + sd->Qi.bytes() + sd->Ub.bytes() + sd->Vb.bytes() +
                       sd->Gd.bytes() + sd->Gdf.bytes() + sd->Ph.bytes() + sd->h.bytes();
  return LYAP_OK;
}
