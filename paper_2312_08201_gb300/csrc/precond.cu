// Truncated-SVD coupling of the preconditioner (eq. (prec)); see precond.cuh.
#include <algorithm>
#include <cmath>
#include <mutex>
#include <vector>

#include "cplx.cuh"
#include "krylov.cuh"
#include "lyap_internal.h"
#include "precond.cuh"
#include "prof.h"

namespace {

constexpr int WT = 256;
constexpr int RMAX = 64;

// O[(t*n+i), (p*n+j)] = Ub[i,p] Lc_ij Vb[j,t]  (N x N, column-major)
__global__ void k_build_O(int n, int k, const double2* __restrict__ lam, const double2* __restrict__ Ub,
                          const double2* __restrict__ Vb, double2* __restrict__ O) {
  const size_t N = (size_t)n * k;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < N * N; idx += (size_t)gridDim.x * blockDim.x) {
    const size_t row = idx % N, col = idx / N;
    const int t = (int)(row / n), i = (int)(row % n), p = (int)(col / n), j = (int)(col % n);
    const double2 L = crcp(cadd(lam[i], lam[j]));
    O[idx] = cmul(cmul(Ub[i + (size_t)p * n], L), Vb[j + (size_t)t * n]);
  }
}

// Deterministic test matrix for the randomized range finder (splitmix64 hash
// of the index to a uniform complex number in the unit square).
__global__ void k_sketch(size_t count, double2* __restrict__ out) {
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < count; idx += (size_t)gridDim.x * blockDim.x) {
    unsigned long long z = (idx + 1) * 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    z ^= z >> 31;
    const double a = (double)(z & 0xFFFFFFFFULL) / 4294967296.0 - 0.5;
    const double b = (double)(z >> 32) / 4294967296.0 - 0.5;
    out[idx] = make_double2(a, b);
  }
}

__global__ void k_scale_cols_tof32(size_t rows, int cols, const double2* __restrict__ X, size_t ldx,
                                   const double* __restrict__ scale, int transpose_from_rows, float2* __restrict__ out) {
  // out (rows x cols, column-major) = X[:, c] * scale[c]  or  X^T (X given as cols x rows) * scale
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < rows * cols; idx += (size_t)gridDim.x * blockDim.x) {
    const size_t r = idx % rows;
    const int c = (int)(idx / rows);
    const double2 v = transpose_from_rows ? X[c + r * ldx] : X[r + (size_t)c * ldx];
    const double s = scale[c];
    out[idx] = make_float2((float)(v.x * s), (float)(v.y * s));
  }
}

int gridn(size_t n) { return (int)std::max<size_t>(1, std::min<size_t>((n + 255) / 256, 8192)); }

int zgemm(cublasHandle_t h, cublasOperation_t ta, cublasOperation_t tb, int m, int n, int k, const double2* A,
          int lda, const double2* B, int ldb, double2* C, int ldc) {
  const cuDoubleComplex one = make_cuDoubleComplex(1.0, 0.0), zero = make_cuDoubleComplex(0.0, 0.0);
  LY_BLAS(cublasZgemm(h, ta, tb, m, n, k, &one, reinterpret_cast<const cuDoubleComplex*>(A), lda,
                      reinterpret_cast<const cuDoubleComplex*>(B), ldb, &zero, reinterpret_cast<cuDoubleComplex*>(C),
                      ldc));
  return LYAP_OK;
}

// Orthonormalise the columns of Y (m x L) in place (Householder QR).
int orth(cusolverDnHandle_t sol, int m, int L, double2* Y, cudaStream_t st) {
  int lw1 = 0, lw2 = 0;
  LY_SOLVER(cusolverDnZgeqrf_bufferSize(sol, m, L, reinterpret_cast<cuDoubleComplex*>(Y), m, &lw1));
  DevBuf<double2> tau, work;
  DevBuf<int> info;
  LY_TRY(tau.alloc(L));
  LY_TRY(info.alloc(1));
  LY_TRY(work.alloc(std::max(lw1, 1)));
  LY_SOLVER(cusolverDnZgeqrf(sol, m, L, reinterpret_cast<cuDoubleComplex*>(Y), m,
                             reinterpret_cast<cuDoubleComplex*>(tau.p), reinterpret_cast<cuDoubleComplex*>(work.p), lw1,
                             info.p));
  LY_SOLVER(cusolverDnZungqr_bufferSize(sol, m, L, L, reinterpret_cast<cuDoubleComplex*>(Y), m,
                                        reinterpret_cast<cuDoubleComplex*>(tau.p), &lw2));
  if (lw2 > lw1) LY_TRY(work.alloc(lw2));
  LY_SOLVER(cusolverDnZungqr(sol, m, L, L, reinterpret_cast<cuDoubleComplex*>(Y), m,
                             reinterpret_cast<cuDoubleComplex*>(tau.p), reinterpret_cast<cuDoubleComplex*>(work.p),
                             std::max(lw1, lw2), info.p));
  return LYAP_OK;
}

// Solve the k x k system K_j x = rhs (K_j[t][p] = delta/v_t - Gd[j,p,t],
// transposed when gT) by Gaussian elimination with partial pivoting.
__device__ __forceinline__ void solve_block(int n, int k, int j, const double2* __restrict__ Gd, int gT,
                                            const double* __restrict__ vinv_b, float2 (&x)[8]) {
  float2 K[8][9];
  for (int t = 0; t < k; ++t) {
    for (int p = 0; p < k; ++p) {
      const size_t gi = gT ? ((size_t)(t * k + p) * n + j) : ((size_t)(p * k + t) * n + j);
      double2 v = cscale(Gd[gi], -1.0);
      if (t == p) v.x += vinv_b[t];
      K[t][p] = make_float2((float)v.x, (float)v.y);
    }
    K[t][k] = x[t];
  }
  for (int c = 0; c < k; ++c) {
    int piv = c;
    float best = cabs2(K[c][c]);
    for (int r = c + 1; r < k; ++r) {
      const float a = cabs2(K[r][c]);
      if (a > best) {
        best = a;
        piv = r;
      }
    }
    if (piv != c)
      for (int q = 0; q <= k; ++q) {
        const float2 tmp = K[c][q];
        K[c][q] = K[piv][q];
        K[piv][q] = tmp;
      }
    const float2 inv = best > 0.f ? cscale(cconj(K[c][c]), 1.f / best) : make_float2(0.f, 0.f);
    for (int r = c + 1; r < k; ++r) {
      const float2 f = cmul(K[r][c], inv);
      for (int q = c; q <= k; ++q) K[r][q] = csub(K[r][q], cmul(f, K[c][q]));
    }
  }
  for (int c = k - 1; c >= 0; --c) {
    float2 s = K[c][k];
    for (int q = c + 1; q < k; ++q) s = csub(s, cmul(K[c][q], x[q]));
    const float d = cabs2(K[c][c]);
    x[c] = d > 0.f ? cscale(cmul(s, cconj(K[c][c])), 1.f / d) : make_float2(0.f, 0.f);
  }
}

// Cap_b = I - Ml^T K_b^{-1} Nl (r x r), then its LU with partial pivoting
// (one CTA per system; warp 0 factors).
__global__ void __launch_bounds__(WT) k_cap_build(int n, int k, int r, const double2* __restrict__ Gd,
                                                  const double* __restrict__ vinv, const float2* __restrict__ Nl,
                                                  const float2* __restrict__ Ml, int ldr, float2* __restrict__ lu,
                                                  int* __restrict__ piv) {
  extern __shared__ float2 sw[];  // [J x k x r] K^{-1} Nl rows, [J x k x r] Ml rows; then r x r
  constexpr int J = 8;
  float2* sm = sw + (size_t)J * k * r;
  const int b = blockIdx.x;
  const double* vb = vinv + (size_t)b * k;
  const int nout = r * r;
  float2 acc[16];
#pragma unroll
  for (int u = 0; u < 16; ++u) acc[u] = make_float2(0.f, 0.f);
  for (int j0 = 0; j0 < n; j0 += J) {
    // W_j = K_j^{-1} Nl[(., j), l]  for j in the chunk, all l
    for (int e = threadIdx.x; e < J * r; e += WT) {
      const int jj = e / r, l = e % r, j = j0 + jj;
      float2 x[8];
      if (j < n) {
        for (int t = 0; t < k; ++t) x[t] = Nl[(size_t)t * n + j + (size_t)l * ldr];
        solve_block(n, k, j, Gd, 0, vb, x);
      }
      for (int t = 0; t < k; ++t) {
        sw[((size_t)jj * k + t) * r + l] = j < n ? x[t] : make_float2(0.f, 0.f);
        sm[((size_t)jj * k + t) * r + l] = j < n ? Ml[(size_t)t * n + j + (size_t)l * ldr] : make_float2(0.f, 0.f);
      }
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < 16; ++u) {
      const int o = threadIdx.x + u * WT;
      if (o < nout) {
        const int l = o % r, l2 = o / r;
        float2 a = acc[u];
        for (int q = 0; q < J * k; ++q) a = cfma(sm[(size_t)q * r + l], sw[(size_t)q * r + l2], a);
        acc[u] = a;
      }
    }
    __syncthreads();
  }
  float2* C = sw;  // r x r, column-major
#pragma unroll
  for (int u = 0; u < 16; ++u) {
    const int o = threadIdx.x + u * WT;
    if (o < nout) {
      const int l = o % r, l2 = o / r;
      C[o] = make_float2((l == l2 ? 1.f : 0.f) - acc[u].x, -acc[u].y);
    }
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    int* pv = piv + (size_t)b * r;
    for (int c = 0; c < r; ++c) {
      int p = c;
      float best = cabs2(C[c + c * r]);
      for (int i = c + 1; i < r; ++i) {
        const float a = cabs2(C[i + c * r]);
        if (a > best) {
          best = a;
          p = i;
        }
      }
      __syncwarp();
      if (p != c)
        for (int q = lane; q < r; q += 32) {
          const float2 tmp = C[c + q * r];
          C[c + q * r] = C[p + q * r];
          C[p + q * r] = tmp;
        }
      if (lane == 0) pv[c] = p;
      __syncwarp();
      const float2 d = C[c + c * r];
      const float dd = cabs2(d);
      const float2 inv = dd > 0.f ? cscale(cconj(d), 1.f / dd) : make_float2(0.f, 0.f);
      for (int i = c + 1 + lane; i < r; i += 32) C[i + c * r] = cmul(C[i + c * r], inv);
      __syncwarp();
      for (int q = c + 1 + lane; q < r; q += 32) {
        const float2 cq = C[c + q * r];
        for (int i = c + 1; i < r; ++i) C[i + q * r] = csub(C[i + q * r], cmul(C[i + c * r], cq));
      }
      __syncwarp();
    }
  }
  __syncthreads();
  for (int o = threadIdx.x; o < nout; o += WT) lu[(size_t)b * nout + o] = C[o];
}

// z_b += K^{-1} A Cap^{-1} B^T z_b  (primal: A = Nl, B = Ml; adjoint:
// A = Ml, B = Nl, K and Cap transposed).
template <typename T2>
__global__ void __launch_bounds__(WT) k_wood_apply(int n, int k, int r, const int* __restrict__ list,
                                                   const int* __restrict__ count, const double2* __restrict__ Gd,
                                                   int adjoint, const double* __restrict__ vinv,
                                                   const float2* __restrict__ Aop, const float2* __restrict__ Bop,
                                                   int ldr, const float2* __restrict__ lu, const int* __restrict__ piv,
                                                   T2* __restrict__ Z, size_t z_ss) {
  __shared__ float red[32 * 32];
  __shared__ float2 c[RMAX], y[RMAX];
  const int slot = blockIdx.x;
  if (slot >= *count) return;
  const int b = list[slot];
  const int N = n * k;
  T2* z = Z + (size_t)b * z_ss;
  for (int l0 = 0; l0 < r; l0 += 16) {
    float acc[32];
#pragma unroll
    for (int u = 0; u < 32; ++u) acc[u] = 0.f;
    for (int e = threadIdx.x; e < N; e += WT) {
      const double2 zd = to_d2(z[e]);
      const float2 ze = make_float2((float)zd.x, (float)zd.y);
#pragma unroll
      for (int u = 0; u < 16; ++u) {
        if (l0 + u < r) {
          const float2 m = Bop[e + (size_t)(l0 + u) * ldr];
          acc[2 * u] += m.x * ze.x - m.y * ze.y;
          acc[2 * u + 1] += m.x * ze.y + m.y * ze.x;
        }
      }
    }
    kry::block_sum<32, float>(acc, red);
    if (threadIdx.x < 16 && l0 + threadIdx.x < r) c[l0 + threadIdx.x] = make_float2(acc[2 * threadIdx.x], acc[2 * threadIdx.x + 1]);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    // y = Cap^{-1} c (P Cap = L U) or y = Cap^{-T} c (Cap^T = U^T L^T P)
    const float2* C = lu + (size_t)b * r * r;
    const int* pv = piv + (size_t)b * r;
    if (!adjoint) {
      for (int i = 0; i < r; ++i) y[i] = c[i];
      for (int i = 0; i < r; ++i) {
        const int p = pv[i];
        if (p != i) {
          const float2 t = y[i];
          y[i] = y[p];
          y[p] = t;
        }
      }
      for (int i = 0; i < r; ++i)
        for (int q = 0; q < i; ++q) y[i] = csub(y[i], cmul(C[i + q * r], y[q]));
      for (int i = r - 1; i >= 0; --i) {
        float2 s = y[i];
        for (int q = i + 1; q < r; ++q) s = csub(s, cmul(C[i + q * r], y[q]));
        const float2 d = C[i + i * r];
        const float dd = cabs2(d);
        y[i] = dd > 0.f ? cscale(cmul(s, cconj(d)), 1.f / dd) : make_float2(0.f, 0.f);
      }
    } else {
      // U^T w = c (forward), L^T y' = w (backward, unit), y = P^T y'
      for (int i = 0; i < r; ++i) {
        float2 s = c[i];
        for (int q = 0; q < i; ++q) s = csub(s, cmul(C[q + i * r], y[q]));
        const float2 d = C[i + i * r];
        const float dd = cabs2(d);
        y[i] = dd > 0.f ? cscale(cmul(s, cconj(d)), 1.f / dd) : make_float2(0.f, 0.f);
      }
      for (int i = r - 1; i >= 0; --i)
        for (int q = i + 1; q < r; ++q) y[i] = csub(y[i], cmul(C[q + i * r], y[q]));
      for (int i = r - 1; i >= 0; --i) {
        const int p = pv[i];
        if (p != i) {
          const float2 t = y[i];
          y[i] = y[p];
          y[p] = t;
        }
      }
    }
  }
  __syncthreads();
  const double* vb = vinv + (size_t)b * k;
  for (int j = threadIdx.x; j < n; j += WT) {
    float2 x[8];
    for (int t = 0; t < k; ++t) {
      float2 s = make_float2(0.f, 0.f);
      for (int l = 0; l < r; ++l) s = cfma(Aop[(size_t)t * n + j + (size_t)l * ldr], y[l], s);
      x[t] = s;
    }
    solve_block(n, k, j, Gd, adjoint, vb, x);
    for (int t = 0; t < k; ++t) {
      const size_t e = (size_t)t * n + j;
      const double2 zd = to_d2(z[e]);
      z[e] = from_d2<T2>(make_double2(zd.x + x[t].x, zd.y + x[t].y));
    }
  }
}

}  // namespace

int lyap_tsvd_prepare(lyap_seed* sd, int r, cudaStream_t st) {
  const int n = sd->n, k = sd->k;
  const int N = n * k;
  r = std::min(r, std::min(RMAX, N - 1));
  if (r <= 0) return LYAP_OK;
  lyap_ctx* ctx = sd->ctx;
  std::lock_guard<std::mutex> lk(ctx->handle_mu);  // library handles are shared by the context's users
  if (sd->tsvd_r >= r) return LYAP_OK;
  LY_BLAS(cublasSetStream(ctx->blas, st));
  LY_SOLVER(cusolverDnSetStream(ctx->solver, st));
  const int L = std::min(N, r + 10);
  DevBuf<double2> O, Y, Z, Bs, G;
  LY_TRY(O.alloc((size_t)N * N));
  LY_TRY(Y.alloc((size_t)N * L));
  LY_TRY(Z.alloc((size_t)N * L));
  LY_TRY(Bs.alloc((size_t)L * N));
  LY_TRY(G.alloc((size_t)L * L));
  k_build_O<<<gridn((size_t)N * N), 256, 0, st>>>(n, k, sd->lam.p, sd->Ub.p, sd->Vb.p, O.p);
  k_sketch<<<gridn((size_t)N * L), 256, 0, st>>>((size_t)N * L, Z.p);
  lyap_count_launch(2);
  LY_CUDA(cudaGetLastError());
  LY_TRY(zgemm(ctx->blas, CUBLAS_OP_N, CUBLAS_OP_N, N, L, N, O.p, N, Z.p, N, Y.p, N));
  for (int it = 0; it < 2; ++it) {  // power iterations sharpen the dominant subspace
    LY_TRY(orth(ctx->solver, N, L, Y.p, st));
    LY_TRY(zgemm(ctx->blas, CUBLAS_OP_C, CUBLAS_OP_N, N, L, N, O.p, N, Y.p, N, Z.p, N));
    LY_TRY(orth(ctx->solver, N, L, Z.p, st));
    LY_TRY(zgemm(ctx->blas, CUBLAS_OP_N, CUBLAS_OP_N, N, L, N, O.p, N, Z.p, N, Y.p, N));
  }
  LY_TRY(orth(ctx->solver, N, L, Y.p, st));                                             // Q
  LY_TRY(zgemm(ctx->blas, CUBLAS_OP_C, CUBLAS_OP_N, L, N, N, Y.p, N, O.p, N, Bs.p, L));  // Q^H O
  LY_TRY(zgemm(ctx->blas, CUBLAS_OP_N, CUBLAS_OP_C, L, L, N, Bs.p, L, Bs.p, L, G.p, L));  // Bs Bs^H
  DevBuf<double> w;
  DevBuf<int> info;
  LY_TRY(w.alloc(L));
  LY_TRY(info.alloc(1));
  int lw = 0;
  LY_SOLVER(cusolverDnZheevd_bufferSize(ctx->solver, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, L,
                                        reinterpret_cast<cuDoubleComplex*>(G.p), L, w.p, &lw));
  DevBuf<double2> work;
  LY_TRY(work.alloc(std::max(lw, 1)));
  LY_SOLVER(cusolverDnZheevd(ctx->solver, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, L,
                             reinterpret_cast<cuDoubleComplex*>(G.p), L, w.p,
                             reinterpret_cast<cuDoubleComplex*>(work.p), lw, info.p));
  // top r eigenpairs (ascending order from heevd): sigma_l = sqrt(w), u_l
  std::vector<double> wh(L);
  LY_CUDA(cudaMemcpyAsync(wh.data(), w.p, sizeof(double) * L, cudaMemcpyDeviceToHost, st));
  LY_CUDA(cudaStreamSynchronize(st));
  DevBuf<double2> Ur, QU, VH;
  LY_TRY(Ur.alloc((size_t)L * r));
  for (int l = 0; l < r; ++l)
    LY_CUDA(cudaMemcpyAsync(Ur.p + (size_t)l * L, G.p + (size_t)(L - 1 - l) * L, sizeof(double2) * L,
                            cudaMemcpyDeviceToDevice, st));
  std::vector<double> sig(r), isig(r);
  for (int l = 0; l < r; ++l) {
    sig[l] = std::sqrt(std::max(0.0, wh[L - 1 - l]));
    isig[l] = sig[l] > 0 ? 1.0 / sig[l] : 0.0;
  }
  DevBuf<double> dsig, disig;
  LY_TRY(dsig.alloc(r));
  LY_TRY(disig.alloc(r));
  LY_CUDA(cudaMemcpyAsync(dsig.p, sig.data(), sizeof(double) * r, cudaMemcpyHostToDevice, st));
  LY_CUDA(cudaMemcpyAsync(disig.p, isig.data(), sizeof(double) * r, cudaMemcpyHostToDevice, st));
  LY_TRY(QU.alloc((size_t)N * r));
  LY_TRY(VH.alloc((size_t)r * N));
  LY_TRY(zgemm(ctx->blas, CUBLAS_OP_N, CUBLAS_OP_N, N, r, L, Y.p, N, Ur.p, L, QU.p, N));  // Q U_r
  LY_TRY(zgemm(ctx->blas, CUBLAS_OP_C, CUBLAS_OP_N, r, N, L, Ur.p, L, Bs.p, L, VH.p, r));  // U_r^H Bs = S V^H
  LY_TRY(sd->tsvd_N.alloc((size_t)N * r));
  LY_TRY(sd->tsvd_M.alloc((size_t)N * r));
  // Nl = Q U_r S ; Ml = (S^{-1} U_r^H Bs)^T = (V^H)^T, so O ~ Nl Ml^T
  k_scale_cols_tof32<<<gridn((size_t)N * r), 256, 0, st>>>(N, r, QU.p, N, dsig.p, 0, sd->tsvd_N.p);
  k_scale_cols_tof32<<<gridn((size_t)N * r), 256, 0, st>>>(N, r, VH.p, r, disig.p, 1, sd->tsvd_M.p);
  lyap_count_launch(2);
  LY_CUDA(cudaGetLastError());
  LY_CUDA(cudaStreamSynchronize(st));
  sd->tsvd_r = r;
  sd->resident_bytes += sd->tsvd_N.bytes() + sd->tsvd_M.bytes();
  return LYAP_OK;
}

int wood_prepare(lyap_seed* sd, int r, int B, const double* vinv, bool /*adjoint*/, WoodState& ws, cudaStream_t st) {
  r = std::min(r, sd->tsvd_r);
  ws.r = r;
  ws.B = B;
  ws.Nl = sd->tsvd_N.p;
  ws.Ml = sd->tsvd_M.p;
  ws.ldr = sd->n * sd->k;
  if (r <= 0 || B <= 0) return LYAP_OK;
  const size_t smem = std::max(sizeof(float2) * 2 * 8 * sd->k * r, sizeof(float2) * r * r);
  static std::once_flag once;
  static cudaError_t attr_rc = cudaSuccess;
  std::call_once(once, [] {
    attr_rc = cudaFuncSetAttribute(k_cap_build, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)(sizeof(float2) * 2 * 8 * 8 * RMAX));
  });
  LY_CUDA(attr_rc);
  const int ph = prof_begin(PK_PRECOND, st);
  k_cap_build<<<B, WT, smem, st>>>(sd->n, sd->k, r, sd->Gd.p, vinv, ws.Nl, ws.Ml, ws.ldr, ws.lu, ws.piv);
  lyap_count_launch();
  prof_end(ph, st, 8.0 * sd->n * sd->k * r * r, 0.0, B, nullptr);
  LY_CUDA(cudaGetLastError());
  return LYAP_OK;
}

template <typename T2>
int wood_apply(lyap_seed* sd, const WoodState& ws, bool adjoint, const double* vinv, const int* list,
               const int* count, int B, T2* Z, size_t z_ss, cudaStream_t st) {
  if (ws.r <= 0) return LYAP_OK;
  const float2* A = adjoint ? ws.Ml : ws.Nl;
  const float2* Bm = adjoint ? ws.Nl : ws.Ml;
  k_wood_apply<T2><<<B, WT, 0, st>>>(sd->n, sd->k, ws.r, list, count, sd->Gd.p, adjoint ? 1 : 0, vinv, A, Bm, ws.ldr,
                                     ws.lu, ws.piv, Z, z_ss);
  lyap_count_launch();
  LY_CUDA(cudaGetLastError());
  return LYAP_OK;
}

template int wood_apply<double2>(lyap_seed*, const WoodState&, bool, const double*, const int*, const int*, int,
                                 double2*, size_t, cudaStream_t);
template int wood_apply<float2>(lyap_seed*, const WoodState&, bool, const double*, const int*, const int*, int,
                                float2*, size_t, cudaStream_t);
