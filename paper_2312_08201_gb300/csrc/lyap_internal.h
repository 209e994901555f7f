// Internal declarations of liblyap (not part of the public C ABI).
#pragma once

#include <cuda_runtime.h>
#include <cublas_v2.h>
#include <cusolverDn.h>

#include <cstdint>
#include <cstdio>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/lyap.h"

// ------------------------------------------------------------------ errors
// Every internal routine returns an int status (LYAP_OK or a negative code);
// these macros turn CUDA/cuBLAS/cuSOLVER failures into codes without
// throwing across the C ABI.
#define LY_CUDA(call)                                                                     \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess) {                                                              \
      lyap_set_last_error(std::string(#call) + ": " + cudaGetErrorString(e_));            \
      return e_ == cudaErrorMemoryAllocation ? LYAP_ENOMEM : LYAP_ECUDA;                 \
    }                                                                                     \
  } while (0)
#define LY_BLAS(call)                                                                     \
  do {                                                                                    \
    cublasStatus_t s_ = (call);                                                           \
    if (s_ != CUBLAS_STATUS_SUCCESS) {                                                    \
      lyap_set_last_error(std::string(#call) + ": cublas status " + std::to_string(s_)); \
      return LYAP_ESOLVER;                                                                \
    }                                                                                     \
  } while (0)
#define LY_SOLVER(call)                                                                     \
  do {                                                                                      \
    cusolverStatus_t s_ = (call);                                                           \
    if (s_ != CUSOLVER_STATUS_SUCCESS) {                                                    \
      lyap_set_last_error(std::string(#call) + ": cusolver status " + std::to_string(s_)); \
      return LYAP_ESOLVER;                                                                  \
    }                                                                                       \
  } while (0)
#define LY_TRY(expr)              \
  do {                            \
    int rc_ = (expr);             \
    if (rc_ != LYAP_OK) return rc_; \
  } while (0)

void lyap_set_last_error(const std::string& msg);

// Raise the dynamic shared-memory limit of kernel `func` to at least `bytes`
// on the current device. The setting belongs to the device's context, so it
// is made once per (device, kernel) and again only for a larger size.
int lyap_smem_optin(const void* func, size_t bytes);

// ------------------------------------------------------------ device memory
// Owning device buffer (no exceptions; allocation reports a status code).
template <typename T>
struct DevBuf {
  T* p = nullptr;
  size_t count = 0;
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  DevBuf(DevBuf&& o) noexcept : p(o.p), count(o.count) { o.p = nullptr; o.count = 0; }
  DevBuf& operator=(DevBuf&& o) noexcept {
    if (this != &o) { release(); p = o.p; count = o.count; o.p = nullptr; o.count = 0; }
    return *this;
  }
  ~DevBuf() { release(); }
  int alloc(size_t n) {
    release();
    if (n == 0) return LYAP_OK;
    cudaError_t e = cudaMalloc(&p, n * sizeof(T));
    if (e != cudaSuccess) {
      p = nullptr;
      lyap_set_last_error(std::string("cudaMalloc: ") + cudaGetErrorString(e));
      return LYAP_ENOMEM;
    }
    count = n;
    return LYAP_OK;
  }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    count = 0;
  }
  size_t bytes() const { return count * sizeof(T); }
};

// ------------------------------------------------------------------ handles
struct lyap_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  cublasHandle_t blas = nullptr;
  cusolverDnHandle_t solver = nullptr;
  unsigned inject_pending = 0;  // host-side fault injection consumed by the next call
  std::mutex handle_mu;         // serialises use of blas/solver across host threads
};

// Recycled subspace kept across calls (and across the parameter sequence):
// Ut (N x s, complex) spans approximate eigenvectors of T(v) for the
// smallest |theta|; C0Ut = C0 * Ut is v-independent, so T(v) Ut =
// Ut D(v)^{-1} - C0Ut costs O(N s) for a new v.
template <typename R2>
struct Recycle {
  DevBuf<R2> Ut;
  DevBuf<R2> C0Ut;
  int s = 0;     // columns held (0 = none yet)
  bool c0_valid = false;
  // An update still running on the producing workspace's side stream: the
  // solver resolves it (ready, then *ok_host) before the next use.
  bool pending = false;
  int pending_s = 0;
  cudaEvent_t ready = nullptr;
  const volatile int* ok_host = nullptr;
};

struct lyap_seed {
  lyap_ctx* ctx = nullptr;
  int device = 0;  // kept here so the seed can be released after its context
  int n = 0, k = 0, g = 0;
  int real_path = 0;
  // 1 when the eigen-decomposition is exactly real (symmetric A0): lam, Qp,
  // Qi and every projected factor have zero imaginary parts, so the mixed
  // path's Cauchy products use the real n x n matrix, with the real and
  // imaginary parts of each panel column as two columns.
  int real_arith = 0;
  double cond_Q = 0, f0 = 0, max_re = 0, min_sum = 0;
  // Eigen-data (P convention): A0^T = Qp diag(lam) Qp^{-1}.
  DevBuf<double2> lam;  // n
  DevBuf<double2> Qp;   // n x n
  DevBuf<double2> Qi;   // n x n
  // Projected data (n x k each, column-major): Ub = Qi V, Vb = Qp^T U.
  DevBuf<double2> Ub, Vb;
  // Gd[(p*k + t)*n + i] = [Lc (Ub_p o Vb_t)]_i: diagonal blocks of N^T L0^{-1} M.
  DevBuf<double2> Gd;
  DevBuf<float2> Gdf;  // FP32 copy of Gd: the preconditioner's block solves run in FP32
  // Capacitance right-hand side of the shifted system T(v) W' = Ph (n x k).
  DevBuf<double2> Ph;
  // Trace vector: f(v) = f0 + Re sum(h o W').
  DevBuf<double2> h;
  double ph_norm = 0;  // ||Ph||_F
  // Mixed path: Lc in two bf16 terms, real-split (see tc_gemm.cu).
  DevBuf<uint16_t> Lhi, Llo;
  int lc_ld = 0;  // padded leading dimension of the split operand
  // Truncated SVD of the v-independent coupling operator (eq. (prec)):
  // O ~ tsvd_N tsvd_M^T, nk x tsvd_r each (FP32), built on first use.
  DevBuf<float2> tsvd_N, tsvd_M;
  int tsvd_r = 0;
  int tsvd_gen = 0;  // counts rebuilds of tsvd_N / tsvd_M
  DevBuf<float2> cap_work;  // K(v)^{-1} Nl of a chunk of systems while Cap(v)^{-1} is built
  // Recycle spaces: primal/adjoint x FP64/FP32-inner.
  Recycle<double2> rec64, rec64_adj;
  Recycle<float2> rec32, rec32_adj;
  size_t resident_bytes = 0;
  // Solver workspaces cached across calls (owned; freed with the seed).
  struct SeedWork* work = nullptr;
  // Mixed-path operands and buffers (owned; freed with the seed).
  struct MixedState* mixed = nullptr;
  // Tensor-core operands and panels of the FP32 Woodbury apply (owned).
  struct PrecTcState* prec_tc = nullptr;
};

// ------------------------------------------------------------------ helpers
int lyap_validate_opts(const lyap_opts* in, lyap_opts* out);
int lyap_check_v(int nv, int k, const double* v_host);

// Seed factor (seed.cu)
// Operands of the mixed path (mixed = true), the truncated SVD of the
// preconditioner (pbar > 0) and the solver's workspace cache, after
// lyap_seed_build.
int lyap_seed_finish(lyap_seed* seed, int pbar, bool mixed, cudaStream_t st);
// P1 (device n x k, may be null): the first block X0 B_r of the right-hand
// side factor of eq. (rhs_newexpression), given instead of G; the seed's
// traces then count only X(v) - X0 (f0 = 0).
int lyap_seed_build(lyap_ctx* ctx, lyap_seed* seed, const double* A0, const double* U,
                    const double* V, const double* G, const double* E, cudaStream_t st,
                    const double* P1 = nullptr);
