// Truncated-SVD coupling of the preconditioner (eq. (prec)); see precond.cuh.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <mutex>
#include <type_traits>
#include <vector>

#include "cplx.cuh"
#include "krylov.cuh"
#include "lyap_internal.h"
#include "precond.cuh"
#include "prof.h"
#include "tc_gemm.cuh"

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

// Solve K_j x = x in place for the k x k block of row j,
//   K_j[t][p] = delta_tp / v_t - Gd[j, p, t]   (transposed when gT),
// in FP32 throughout (Gd: the seed's FP32 copy, 1/v_t rounded to FP32),
// by Gaussian elimination with partial pivoting. k is a template argument and
// each elimination step is its own instantiation (Elim<K, C>), so every index
// is a compile-time constant and the block stays in registers; rows are
// exchanged by selects.
template <int K, int C>
struct Elim {
  static __device__ __forceinline__ void run(float (&Ar)[K][K], float (&Ai)[K][K], float2 (&x)[K]) {
    float best = Ar[C][C] * Ar[C][C] + Ai[C][C] * Ai[C][C];
    int piv = C;
#pragma unroll
    for (int r = C + 1; r < K; ++r) {
      const float a = Ar[r][C] * Ar[r][C] + Ai[r][C] * Ai[r][C];
      if (a > best) {
        best = a;
        piv = r;
      }
    }
#pragma unroll
    for (int r = C + 1; r < K; ++r) {
      const bool sw = r == piv;
#pragma unroll
      for (int q = C; q < K; ++q) {
        const float ar = Ar[C][q], ai = Ai[C][q], br = Ar[r][q], bi = Ai[r][q];
        Ar[C][q] = sw ? br : ar;
        Ai[C][q] = sw ? bi : ai;
        Ar[r][q] = sw ? ar : br;
        Ai[r][q] = sw ? ai : bi;
      }
      const float2 a = x[C], b = x[r];
      x[C] = sw ? b : a;
      x[r] = sw ? a : b;
    }
    // 1 / pivot = conj(pivot) / |pivot|^2
    const float2 inv = best > 0.f ? make_float2(Ar[C][C] / best, -Ai[C][C] / best) : make_float2(0.f, 0.f);
#pragma unroll
    for (int r = C + 1; r < K; ++r) {
      const float2 f = cmul(make_float2(Ar[r][C], Ai[r][C]), inv);
#pragma unroll
      for (int q = C + 1; q < K; ++q) {
        const float2 v = csub(make_float2(Ar[r][q], Ai[r][q]), cmul(f, make_float2(Ar[C][q], Ai[C][q])));
        Ar[r][q] = v.x;
        Ai[r][q] = v.y;
      }
      x[r] = csub(x[r], cmul(f, x[C]));
    }
    Elim<K, C + 1>::run(Ar, Ai, x);
  }
};
template <int K>
struct Elim<K, K> {
  static __device__ __forceinline__ void run(float (&)[K][K], float (&)[K][K], float2 (&)[K]) {}
};

// LU factorisation with partial pivoting of the k x k block, kept in
// registers: U on and above the diagonal, the multipliers of each step
// below it, and the pivot row of each step in piv (at step C, columns >= C
// of rows C and piv[C] are swapped; lu_solve replays the swaps in order).
template <int K, int C>
struct Lu {
  static __device__ __forceinline__ void run(float (&Ar)[K][K], float (&Ai)[K][K], int (&piv)[K]) {
    float best = Ar[C][C] * Ar[C][C] + Ai[C][C] * Ai[C][C];
    int p = C;
#pragma unroll
    for (int r = C + 1; r < K; ++r) {
      const float a = Ar[r][C] * Ar[r][C] + Ai[r][C] * Ai[r][C];
      if (a > best) {
        best = a;
        p = r;
      }
    }
    piv[C] = p;
#pragma unroll
    for (int r = C + 1; r < K; ++r) {
      const bool sw = r == p;
#pragma unroll
      for (int q = C; q < K; ++q) {  // earlier multipliers stay: lu_solve swaps x step by step
        const float ar = Ar[C][q], ai = Ai[C][q], br = Ar[r][q], bi = Ai[r][q];
        Ar[C][q] = sw ? br : ar;
        Ai[C][q] = sw ? bi : ai;
        Ar[r][q] = sw ? ar : br;
        Ai[r][q] = sw ? ai : bi;
      }
    }
    const float2 inv = best > 0.f ? make_float2(Ar[C][C] / best, -Ai[C][C] / best) : make_float2(0.f, 0.f);
#pragma unroll
    for (int r = C + 1; r < K; ++r) {
      const float2 f = cmul(make_float2(Ar[r][C], Ai[r][C]), inv);
#pragma unroll
      for (int q = C + 1; q < K; ++q) {
        const float2 v = csub(make_float2(Ar[r][q], Ai[r][q]), cmul(f, make_float2(Ar[C][q], Ai[C][q])));
        Ar[r][q] = v.x;
        Ai[r][q] = v.y;
      }
      Ar[r][C] = f.x;
      Ai[r][C] = f.y;
    }
    Lu<K, C + 1>::run(Ar, Ai, piv);
  }
};
template <int K>
struct Lu<K, K> {
  static __device__ __forceinline__ void run(float (&)[K][K], float (&)[K][K], int (&)[K]) {}
};

// x <- (P L U)^{-1} x with the factors of Lu
template <int K>
__device__ __forceinline__ void lu_solve(const float (&Ar)[K][K], const float (&Ai)[K][K], const int (&piv)[K],
                                         float2 (&x)[K]) {
#pragma unroll
  for (int c = 0; c < K; ++c) {
#pragma unroll
    for (int r = c + 1; r < K; ++r) {
      const bool sw = r == piv[c];
      const float2 a = x[c], b = x[r];
      x[c] = sw ? b : a;
      x[r] = sw ? a : b;
    }
#pragma unroll
    for (int r = c + 1; r < K; ++r) x[r] = csub(x[r], cmul(make_float2(Ar[r][c], Ai[r][c]), x[c]));
  }
#pragma unroll
  for (int c = K - 1; c >= 0; --c) {
    float2 s = x[c];
#pragma unroll
    for (int q = c + 1; q < K; ++q) s = csub(s, cmul(make_float2(Ar[c][q], Ai[c][q]), x[q]));
    const float d = Ar[c][c] * Ar[c][c] + Ai[c][c] * Ai[c][c];
    x[c] = d > 0.f ? make_float2((s.x * Ar[c][c] + s.y * Ai[c][c]) / d, (s.y * Ar[c][c] - s.x * Ai[c][c]) / d)
                   : make_float2(0.f, 0.f);
  }
}

template <int K>
__device__ __forceinline__ void bsolve(int n, int j, const float2* __restrict__ Gd, int gT, const float (&vb)[K],
                                       float2 (&x)[K]) {
  float Ar[K][K], Ai[K][K];
#pragma unroll
  for (int t = 0; t < K; ++t)
#pragma unroll
    for (int p = 0; p < K; ++p) {
      const size_t gi = gT ? ((size_t)(t * K + p) * n + j) : ((size_t)(p * K + t) * n + j);
      const float2 g = Gd[gi];
      Ar[t][p] = (t == p ? vb[t] : 0.f) - g.x;
      Ai[t][p] = -g.y;
    }
  Elim<K, 0>::run(Ar, Ai, x);
#pragma unroll
  for (int c = K - 1; c >= 0; --c) {
    float2 s = x[c];
#pragma unroll
    for (int q = c + 1; q < K; ++q) s = csub(s, cmul(make_float2(Ar[c][q], Ai[c][q]), x[q]));
    const float d = Ar[c][c] * Ar[c][c] + Ai[c][c] * Ai[c][c];
    x[c] = d > 0.f ? make_float2((s.x * Ar[c][c] + s.y * Ai[c][c]) / d, (s.y * Ar[c][c] - s.x * Ai[c][c]) / d)
                   : make_float2(0.f, 0.f);
  }
}

template <int K>
__device__ __forceinline__ void load_vb(const double* __restrict__ vinv, int b, float (&vb)[K]) {
#pragma unroll
  for (int t = 0; t < K; ++t) vb[t] = (float)vinv[(size_t)b * K + t];
}


// Gauss-Jordan inversion with partial pivoting of the r x r matrix C
// (column-major, shared memory), by the whole CTA; Inv starts as I and
// ends as C^{-1}; C is destroyed.
__device__ void gj_invert(int r, float2* C, float2* Inv, float2* fcol, int* piv_sp) {
  const int nout = r * r;
  int& piv_s = *piv_sp;
  for (int c = 0; c < r; ++c) {
    if (threadIdx.x < 32) {
      float best = -1.f;
      int p = c;
      for (int i = c + threadIdx.x; i < r; i += 32) {
        const float a = cabs2(C[i + c * r]);
        if (a > best) {
          best = a;
          p = i;
        }
      }
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        const float ob = __shfl_xor_sync(0xffffffffu, best, off);
        const int op = __shfl_xor_sync(0xffffffffu, p, off);
        if (ob > best || (ob == best && op < p)) {
          best = ob;
          p = op;
        }
      }
      if (threadIdx.x == 0) piv_s = p;
    }
    __syncthreads();
    const int p = piv_s;
    if (p != c)
      for (int q = threadIdx.x; q < 2 * r; q += WT) {
        float2* M = q < r ? C : Inv;
        const int qq = q < r ? q : q - r;
        const float2 t = M[c + qq * r];
        M[c + qq * r] = M[p + qq * r];
        M[p + qq * r] = t;
      }
    __syncthreads();
    const float2 d = C[c + c * r];
    const float dd = cabs2(d);
    const float2 dinv = dd > 0.f ? cscale(cconj(d), 1.f / dd) : make_float2(0.f, 0.f);
    for (int i = threadIdx.x; i < r; i += WT) fcol[i] = i == c ? make_float2(0.f, 0.f) : C[i + c * r];
    __syncthreads();
    for (int q = threadIdx.x; q < 2 * r; q += WT) {
      float2* M = q < r ? C : Inv;
      const int qq = q < r ? q : q - r;
      M[c + qq * r] = cmul(M[c + qq * r], dinv);
    }
    __syncthreads();
    for (int e = threadIdx.x; e < 2 * nout; e += WT) {
      float2* M = e < nout ? C : Inv;
      const int ee = e < nout ? e : e - nout;
      const int i = ee % r, q = ee / r;
      if (i != c) M[i + q * r] = csub(M[i + q * r], cmul(fcol[i], M[c + q * r]));
    }
    __syncthreads();
  }
}

// Y_b = K_b(v)^{-1} Nl for the systems of a chunk (Y: nsys x nk x r, column-
// major per system). One thread per (row j, system): the k x k block is
// factorised once and its factors solve the r columns.
template <int K>
__global__ void __launch_bounds__(WT) k_kinv_nl(int n, int r, const float2* __restrict__ Gd,
                                                const double* __restrict__ vinv, const float2* __restrict__ Nl,
                                                int ldr, int nsys, float2* __restrict__ Y) {
  const int j = blockIdx.x * WT + threadIdx.x;
  const int b = blockIdx.y;
  if (j >= n || b >= nsys) return;
  float vb[K];
  load_vb<K>(vinv, b, vb);
  float Ar[K][K], Ai[K][K];
#pragma unroll
  for (int t = 0; t < K; ++t)
#pragma unroll
    for (int p = 0; p < K; ++p) {
      const float2 g = Gd[(size_t)(p * K + t) * n + j];
      Ar[t][p] = (t == p ? vb[t] : 0.f) - g.x;
      Ai[t][p] = -g.y;
    }
  int piv[K];
  Lu<K, 0>::run(Ar, Ai, piv);
  const size_t nk = (size_t)n * K;
  float2* Yb = Y + (size_t)b * nk * r;
  for (int l = 0; l < r; ++l) {
    float2 x[K];
#pragma unroll
    for (int t = 0; t < K; ++t) x[t] = Nl[(size_t)t * n + j + (size_t)l * ldr];
    lu_solve<K>(Ar, Ai, piv, x);
#pragma unroll
    for (int t = 0; t < K; ++t) Yb[(size_t)t * n + j + (size_t)l * nk] = x[t];
  }
}

// cinv_b = (I + C_b)^{-1} for C_b = -Ml^T Y_b (r x r, from the batched GEMM)
__global__ void __launch_bounds__(WT) k_cap_inv(int r, const float2* __restrict__ Cin, float2* __restrict__ cinv) {
  extern __shared__ float2 cm[];  // C, Inv (r x r each)
  __shared__ float2 fcol[RMAX];
  __shared__ int piv_s;
  const int b = blockIdx.x;
  const int nout = r * r;
  float2* C = cm;
  float2* Inv = cm + nout;
  for (int e = threadIdx.x; e < nout; e += WT) {
    const int i = e % r, q = e / r;
    float2 c = Cin[(size_t)b * nout + e];
    if (i == q) c.x += 1.f;
    C[e] = c;
    Inv[e] = make_float2(i == q ? 1.f : 0.f, 0.f);
  }
  __syncthreads();
  gj_invert(r, C, Inv, fcol, &piv_s);
  for (int o = threadIdx.x; o < nout; o += WT) cinv[(size_t)b * nout + o] = Inv[o];
}

// Preconditioner apply for the listed systems:
//   z = K^{-1} r, then (rank r > 0) z += K^{-1} A Cap^{-1} B^T z
// with A = Nl, B = Ml (primal) or A = Ml, B = Nl, K^T and Cap^{-T}
// (adjoint). Two kernels over tiles of PRT rows x PST systems (a few hundred
// CTAs for a full batch; every row of A and B read from L2 serves PST
// systems):
//   k_prec_a: z = K^{-1} r for the tile, and the tile's partial sums of
//             c = B^T z, written per row tile (no atomics: deterministic);
//   k_prec_y: c = sum of the partials, y = Cap^{-1} c, one CTA per system,
//             y written over the first row tile's partial;
//   k_prec_b: z += K^{-1} (A y) for the tile.
// FP32 arithmetic; input and output in the Krylov precision.
constexpr int PST = 16;
template <int K>
struct PrecTile {
  static constexpr int RT = K <= 4 ? 64 : 32;
};

template <typename T2, int K>
__global__ void __launch_bounds__(WT) k_prec_a(int n, const int* __restrict__ list, const int* __restrict__ count,
                                               const float2* __restrict__ Gd, int adj,
                                               const double* __restrict__ vinv, const T2* __restrict__ In,
                                               size_t in_ss, T2* __restrict__ Out, size_t out_ss, int r,
                                               const float2* __restrict__ Bop, int ldr, float2* __restrict__ Cp,
                                               int nslots) {
  constexpr int RT = PrecTile<K>::RT;
  __shared__ float2 zs[PST][K][RT + 1];
  const int nact = *count;
  const int s0 = blockIdx.y * PST;
  if (s0 >= nact) return;
  const int j0 = blockIdx.x * RT;
  for (int e = threadIdx.x; e < RT * PST; e += WT) {
    const int row = e % RT, sl = e / RT;
    const int j = j0 + row;
    float2 x[K];
    if (s0 + sl < nact && j < n) {
      const int b = list[s0 + sl];
      float vb[K];
      load_vb<K>(vinv, b, vb);
      const T2* in = In + (size_t)b * in_ss;
#pragma unroll
      for (int t = 0; t < K; ++t) x[t] = to_f2(in[(size_t)t * n + j]);
      bsolve<K>(n, j, Gd, adj, vb, x);
      T2* out = Out + (size_t)b * out_ss;
#pragma unroll
      for (int t = 0; t < K; ++t) out[(size_t)t * n + j] = from_f2<T2>(x[t]);
    } else {
#pragma unroll
      for (int t = 0; t < K; ++t) x[t] = make_float2(0.f, 0.f);
    }
    if (r > 0) {
#pragma unroll
      for (int t = 0; t < K; ++t) zs[sl][t][row] = x[t];
    }
  }
  if (r <= 0) return;
  // c partials: thread (lp, sp) owns ranks 2lp, 2lp+1 of systems 2sp, 2sp+1;
  // QC rows of B at a time are staged in shared memory (coalesced over rows)
  constexpr int QC = 16;
  __shared__ float2 bs[QC][RMAX + 1];  // odd row length: the fill's stores spread over the banks
  const int rows = min(RT, n - j0);
  const int lp = threadIdx.x & 31, sp = threadIdx.x >> 5;
  const int l0 = 2 * lp, sl0 = 2 * sp;
  float2 acc[2][2];
#pragma unroll
  for (int u = 0; u < 2; ++u)
#pragma unroll
    for (int w = 0; w < 2; ++w) acc[u][w] = make_float2(0.f, 0.f);
  for (int t = 0; t < K; ++t)
    for (int q0 = 0; q0 < rows; q0 += QC) {
      __syncthreads();  // the previous chunk is consumed (and, first time, zs is complete)
      for (int e = threadIdx.x; e < QC * r; e += WT) {
        const int qq = e % QC, l = e / QC;
        bs[qq][l] = q0 + qq < rows ? Bop[(size_t)t * n + j0 + q0 + qq + (size_t)l * ldr] : make_float2(0.f, 0.f);
      }
      __syncthreads();
#pragma unroll 4
      for (int qq = 0; qq < QC; ++qq) {
        const float2 b0 = bs[qq][l0], b1 = bs[qq][l0 + 1];
        const float2 z0 = zs[sl0][t][min(q0 + qq, RT - 1)], z1 = zs[sl0 + 1][t][min(q0 + qq, RT - 1)];
        acc[0][0] = cfma(b0, z0, acc[0][0]);
        acc[0][1] = cfma(b0, z1, acc[0][1]);
        acc[1][0] = cfma(b1, z0, acc[1][0]);
        acc[1][1] = cfma(b1, z1, acc[1][1]);
      }
    }
#pragma unroll
  for (int u = 0; u < 2; ++u)
#pragma unroll
    for (int w = 0; w < 2; ++w)
      if (l0 + u < r && s0 + sl0 + w < nact) Cp[((size_t)blockIdx.x * nslots + s0 + sl0 + w) * r + l0 + u] = acc[u][w];
}

// y = Cap^{-1} c (Cap^{-T} c for the adjoint) for the listed systems, c the
// sum of k_prec_a's row-tile partials; one CTA per system slot. Cap^{-1} is
// staged in shared memory with an odd column stride, so both the plain and
// the transposed product read it without bank conflicts.
__global__ void __launch_bounds__(WT) k_prec_y(const int* __restrict__ list, const int* __restrict__ count, int adj,
                                               int r, const float2* __restrict__ cinv, float2* __restrict__ Cp,
                                               int nslots, int ntx) {
  __shared__ float2 Cs[RMAX * (RMAX + 1)];
  __shared__ float2 cs[RMAX];
  __shared__ float2 ys[WT / RMAX][RMAX];
  const int s = blockIdx.x;
  if (s >= *count) return;
  const int rp = r | 1;
  const float2* Ci = cinv + (size_t)list[s] * r * r;
  for (int e = threadIdx.x; e < r * r; e += WT) Cs[(e % r) + (e / r) * rp] = Ci[e];
  for (int l = threadIdx.x; l < r; l += WT) {
    float2 c = make_float2(0.f, 0.f);
    for (int tx = 0; tx < ntx; ++tx) c = cadd(c, Cp[((size_t)tx * nslots + s) * r + l]);
    cs[l] = c;
  }
  __syncthreads();
  // thread (l, g): the terms q = g, g + G, ... of y_l
  constexpr int G = WT / RMAX;
  const int l = threadIdx.x % RMAX, g = threadIdx.x / RMAX;
  float2 y = make_float2(0.f, 0.f);
  if (l < r) {
    if (adj) {
      for (int q = g; q < r; q += G) y = cfma(Cs[q + l * rp], cs[q], y);
    } else {
      for (int q = g; q < r; q += G) y = cfma(Cs[l + q * rp], cs[q], y);
    }
  }
  ys[g][l] = y;
  __syncthreads();
  if (threadIdx.x < r) {
    float2 t = ys[0][threadIdx.x];
#pragma unroll
    for (int u = 1; u < G; ++u) t = cadd(t, ys[u][threadIdx.x]);
    Cp[(size_t)s * r + threadIdx.x] = t;
  }
}

template <typename T2, int K>
__global__ void __launch_bounds__(WT) k_prec_b(int n, const int* __restrict__ list, const int* __restrict__ count,
                                               const float2* __restrict__ Gd, int adj,
                                               const double* __restrict__ vinv, T2* __restrict__ Out, size_t out_ss,
                                               int r, const float2* __restrict__ Aop, int ldr,
                                               const float2* __restrict__ Yp) {
  constexpr int RT = PrecTile<K>::RT;
  __shared__ float2 ys[PST][RMAX + 1];
  const int nact = *count;
  const int s0 = blockIdx.y * PST;
  if (s0 >= nact) return;
  const int j0 = blockIdx.x * RT;
  for (int e = threadIdx.x; e < PST * r; e += WT) {
    const int sl = e / r, l = e % r;
    ys[sl][l] = s0 + sl < nact ? Yp[(size_t)(s0 + sl) * r + l] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  // thread = (row, group of PG systems): each entry of the row of A is
  // loaded once and serves PG systems
  constexpr int PG = K <= 2 ? 4 : (K <= 4 ? 2 : 1);
  for (int e = threadIdx.x; e < RT * (PST / PG); e += WT) {
    const int row = e % RT, g0 = (e / RT) * PG;
    const int j = j0 + row;
    if (j >= n || s0 + g0 >= nact) continue;
    float2 x[PG][K];
#pragma unroll
    for (int u = 0; u < PG; ++u)
#pragma unroll
      for (int t = 0; t < K; ++t) x[u][t] = make_float2(0.f, 0.f);
    for (int l = 0; l < r; ++l) {
      float2 a[K];
#pragma unroll
      for (int t = 0; t < K; ++t) a[t] = Aop[(size_t)t * n + j + (size_t)l * ldr];
#pragma unroll
      for (int u = 0; u < PG; ++u) {
        const float2 y = ys[g0 + u][l];
#pragma unroll
        for (int t = 0; t < K; ++t) x[u][t] = cfma(a[t], y, x[u][t]);
      }
    }
#pragma unroll
    for (int u = 0; u < PG; ++u) {
      if (s0 + g0 + u >= nact) break;
      const int b = list[s0 + g0 + u];
      float vb[K];
      load_vb<K>(vinv, b, vb);
      bsolve<K>(n, j, Gd, adj, vb, x[u]);
      T2* out = Out + (size_t)b * out_ss;
#pragma unroll
      for (int t = 0; t < K; ++t) {
        const size_t e2 = (size_t)t * n + j;
        out[e2] = add_f2(out[e2], x[u][t]);
      }
    }
  }
}

// FP32 Krylov vectors: the two products of the apply run on the tensor cores
// (the tcgen05 BF16x3 GEMM of the inner operator, real-split complex
// operands), over the active systems in slot order:
//   k_prec_z    z = K^{-1} r, stored, and its panel row (BF16 hi/lo, real-split)
//   GEMM 1      c = B^T z, K = 2nk split across CTAs (partial sums per split)
//   k_prec_ytc  y = Cap^{-1} (sum of the partials), and its panel row
//   GEMM 2      d = A y
//   k_prec_dtc  z += K^{-1} d
// BF16x3 keeps about 16 bits of each product (relative error near 2^-16),
// far inside what the preconditioner's convergence needs.

__device__ __forceinline__ void split_bf16(float v, __nv_bfloat16& hi, __nv_bfloat16& lo) {
  hi = __float2bfloat16_rn(v);
  lo = __float2bfloat16_rn(v - __bfloat162float(hi));
}

// Real-split operand of a product with M (nk x r complex, leading dimension
// ld): trans = 1 gives M^T (rows 2l, 2l+1; K entries 2q, 2q+1), trans = 0
// gives M (rows 2q, 2q+1; K entries 2l, 2l+1); each 2 x 2 block is
// [[Re, -Im], [Im, Re]] of the entry. Padding rows and K entries are zero.
__global__ void k_split_op(int nk, int r, const float2* __restrict__ M, int ld, int trans, int mpad, int kpad,
                           __nv_bfloat16* __restrict__ H, __nv_bfloat16* __restrict__ Lo) {
  const size_t total = (size_t)mpad * kpad;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
    const int row = (int)(idx / kpad), col = (int)(idx % kpad);
    const int q = trans ? col >> 1 : row >> 1, l = trans ? row >> 1 : col >> 1;
    float v = 0.f;
    if (q < nk && l < r) {
      const float2 m = M[(size_t)q + (size_t)l * ld];
      const int ri = row & 1, ci = col & 1;
      v = ri == ci ? m.x : (ri == 0 ? -m.y : m.y);
    }
    split_bf16(v, H[idx], Lo[idx]);
  }
}

// z = K^{-1} r for slot s (system list[s]), stored, and panel row s.
template <int K>
__global__ void __launch_bounds__(WT) k_prec_z(int n, const int* __restrict__ list, const int* __restrict__ count,
                                               const float2* __restrict__ Gd, int adj, const double* __restrict__ vinv,
                                               const float2* __restrict__ In, size_t in_ss, float2* __restrict__ Out,
                                               size_t out_ss, int kpad, __nv_bfloat16* __restrict__ Ph,
                                               __nv_bfloat16* __restrict__ Pl) {
  const int j = blockIdx.x * WT + threadIdx.x;
  const int s = blockIdx.y;
  if (j >= n || s >= *count) return;
  const int b = list[s];
  float vb[K];
  load_vb<K>(vinv, b, vb);
  float2 x[K];
  const float2* in = In + (size_t)b * in_ss;
#pragma unroll
  for (int t = 0; t < K; ++t) x[t] = in[(size_t)t * n + j];
  bsolve<K>(n, j, Gd, adj, vb, x);
  float2* out = Out + (size_t)b * out_ss;
#pragma unroll
  for (int t = 0; t < K; ++t) {
    const size_t q = (size_t)t * n + j;
    out[q] = x[t];
    const size_t o = (size_t)s * kpad + 2 * q;
    split_bf16(x[t].x, Ph[o], Pl[o]);
    split_bf16(x[t].y, Ph[o + 1], Pl[o + 1]);
  }
}

// y = Cap^{-1} c (Cap^{-T} c for the adjoint) for slot s, c from the split
// partials of GEMM 1 (rows 2l, 2l+1 of column s, ldd per column, dstride
// per split); y goes to panel row s (K entries 2l, 2l+1). One CTA per slot,
// Cap^{-1} staged as in k_prec_y.
__global__ void __launch_bounds__(WT) k_prec_ytc(const int* __restrict__ list, const int* __restrict__ count, int adj,
                                                 int r, const float2* __restrict__ cinv, const float* __restrict__ D1,
                                                 int ldd, int splits, size_t dstride, int kpad,
                                                 __nv_bfloat16* __restrict__ Ph, __nv_bfloat16* __restrict__ Pl) {
  __shared__ float2 Cs[RMAX * (RMAX + 1)];
  __shared__ float2 cs[RMAX];
  __shared__ float2 ys[WT / RMAX][RMAX];
  const int s = blockIdx.x;
  if (s >= *count) return;
  const int rp = r | 1;
  const float2* Ci = cinv + (size_t)list[s] * r * r;
  for (int e = threadIdx.x; e < r * r; e += WT) Cs[(e % r) + (e / r) * rp] = Ci[e];
  for (int l = threadIdx.x; l < r; l += WT) {
    float2 c = make_float2(0.f, 0.f);
    for (int z = 0; z < splits; ++z) {
      const float* d = D1 + (size_t)z * dstride + (size_t)s * ldd + 2 * l;
      c = cadd(c, make_float2(d[0], d[1]));
    }
    cs[l] = c;
  }
  __syncthreads();
  constexpr int G = WT / RMAX;
  const int l = threadIdx.x % RMAX, g = threadIdx.x / RMAX;
  float2 y = make_float2(0.f, 0.f);
  if (l < r) {
    if (adj) {
      for (int q = g; q < r; q += G) y = cfma(Cs[q + l * rp], cs[q], y);
    } else {
      for (int q = g; q < r; q += G) y = cfma(Cs[l + q * rp], cs[q], y);
    }
  }
  ys[g][l] = y;
  __syncthreads();
  if (threadIdx.x < r) {
    float2 t = ys[0][threadIdx.x];
#pragma unroll
    for (int u = 1; u < G; ++u) t = cadd(t, ys[u][threadIdx.x]);
    const size_t o = (size_t)s * kpad + 2 * threadIdx.x;
    split_bf16(t.x, Ph[o], Pl[o]);
    split_bf16(t.y, Ph[o + 1], Pl[o + 1]);
  }
}

// z += K^{-1} d for slot s, d from GEMM 2 (rows 2q, 2q+1 of column s).
template <int K>
__global__ void __launch_bounds__(WT) k_prec_dtc(int n, const int* __restrict__ list, const int* __restrict__ count,
                                                 const float2* __restrict__ Gd, int adj,
                                                 const double* __restrict__ vinv, const float* __restrict__ D2,
                                                 int ldd, float2* __restrict__ Out, size_t out_ss) {
  const int j = blockIdx.x * WT + threadIdx.x;
  const int s = blockIdx.y;
  if (j >= n || s >= *count) return;
  const int b = list[s];
  float vb[K];
  load_vb<K>(vinv, b, vb);
  float2 x[K];
  const float* d = D2 + (size_t)s * ldd;
#pragma unroll
  for (int t = 0; t < K; ++t) {
    const size_t q = (size_t)t * n + j;
    x[t] = make_float2(d[2 * q], d[2 * q + 1]);
  }
  bsolve<K>(n, j, Gd, adj, vb, x);
  float2* out = Out + (size_t)b * out_ss;
#pragma unroll
  for (int t = 0; t < K; ++t) out[(size_t)t * n + j] = cadd(out[(size_t)t * n + j], x[t]);
}

// Cap(v_b)^{-1} for systems b < B: Y_b = K_b^{-1} Nl (k_kinv_nl), then
// Cap_b - I = -Ml^T Y_b for all systems of a chunk in one strided-batched
// CGEMM (FP32, cuBLAS), then one Gauss-Jordan inversion per system. Chunks
// of systems keep the Y buffer (nk x r per system) within kCapWorkBytes.
constexpr size_t kCapWorkBytes = size_t(1) << 30;

template <int K>
int launch_cap_build(lyap_seed* sd, int r, int B, const double* vinv, const WoodState& ws, cudaStream_t st) {
  const int n = sd->n;
  const size_t nk = (size_t)n * K, per = nk * (size_t)r * sizeof(float2) + (size_t)r * r * sizeof(float2);
  const int chunk = (int)std::max<size_t>(1, std::min<size_t>((size_t)B, kCapWorkBytes / per));
  const size_t need = (size_t)chunk * (nk * r + (size_t)r * r);
  if (sd->cap_work.count < need) LY_TRY(sd->cap_work.alloc(need));
  float2* Y = sd->cap_work.p;
  float2* Cm = Y + (size_t)chunk * nk * r;
  LY_TRY(lyap_smem_optin(reinterpret_cast<const void*>(k_cap_inv), 2 * sizeof(float2) * RMAX * RMAX));
  lyap_ctx* ctx = sd->ctx;
  for (int b0 = 0; b0 < B; b0 += chunk) {
    const int nb = std::min(chunk, B - b0);
    k_kinv_nl<K><<<dim3((n + WT - 1) / WT, nb), WT, 0, st>>>(n, r, sd->Gdf.p, vinv + (size_t)b0 * K, ws.Nl, ws.ldr,
                                                             nb, Y);
    {
      std::lock_guard<std::mutex> lk(ctx->handle_mu);  // library handles are shared by the context's users
      LY_BLAS(cublasSetStream(ctx->blas, st));
      const cuComplex m1 = make_cuComplex(-1.f, 0.f), z = make_cuComplex(0.f, 0.f);
      LY_BLAS(cublasCgemmStridedBatched(ctx->blas, CUBLAS_OP_T, CUBLAS_OP_N, r, r, (int)nk, &m1,
                                        reinterpret_cast<const cuComplex*>(ws.Ml), ws.ldr, 0,
                                        reinterpret_cast<const cuComplex*>(Y), (int)nk, (long long)nk * r, &z,
                                        reinterpret_cast<cuComplex*>(Cm), r, (long long)r * r, nb));
    }
    k_cap_inv<<<nb, WT, 2 * sizeof(float2) * r * r, st>>>(r, Cm, ws.cinv + (size_t)b0 * r * r);
    lyap_count_launch(2);
    LY_CUDA(cudaGetLastError());
  }
  return LYAP_OK;
}

}  // namespace

// Operands of the two products for rank r (both directions) of the seed's
// current truncated SVD, and panels for a batch of systems; rebuilt when the
// rank or the SVD changes, grown with the batch.
struct PrecTcState {
  int r = 0, nk = 0, gen = -1, kpad1 = 0, mpad2 = 0, kpad2 = 0;
  DevBuf<__nv_bfloat16> a1h[2], a1l[2], a2h[2], a2l[2];  // [0] primal, [1] adjoint
  tc::Maps m1[2], m2[2];
  int ncap = 0, splits = 1;
  DevBuf<__nv_bfloat16> b1h, b1l, b2h, b2l;  // ncap x kpad1, ncap x kpad2
  DevBuf<float> d1, d2;                      // splits x ncap x 128, ncap x mpad2
};

void lyap_prec_tc_free(lyap_seed* sd) {
  delete sd->prec_tc;
  sd->prec_tc = nullptr;
}

namespace {

int ensure_prec_tc(lyap_seed* sd, const WoodState& ws, int B, cudaStream_t st, PrecTcState** out) {
  const int nk = sd->n * sd->k, r = ws.r;
  if (!sd->prec_tc) sd->prec_tc = new PrecTcState();
  PrecTcState& P = *sd->prec_tc;
  if (P.r != r || P.nk != nk || P.gen != sd->tsvd_gen) {
    P.r = r;
    P.nk = nk;
    P.gen = sd->tsvd_gen;
    P.kpad1 = ((2 * nk + tc::BK - 1) / tc::BK) * tc::BK;
    P.mpad2 = ((2 * nk + tc::BM - 1) / tc::BM) * tc::BM;
    P.kpad2 = ((2 * r + tc::BK - 1) / tc::BK) * tc::BK;
    for (int dir = 0; dir < 2; ++dir) {
      const float2* Bm = dir ? ws.Nl : ws.Ml;  // c = Bm^T z
      const float2* Am = dir ? ws.Ml : ws.Nl;  // d = Am y
      LY_TRY(P.a1h[dir].alloc((size_t)tc::BM * P.kpad1));
      LY_TRY(P.a1l[dir].alloc((size_t)tc::BM * P.kpad1));
      LY_TRY(P.a2h[dir].alloc((size_t)P.mpad2 * P.kpad2));
      LY_TRY(P.a2l[dir].alloc((size_t)P.mpad2 * P.kpad2));
      k_split_op<<<gridn((size_t)tc::BM * P.kpad1), 256, 0, st>>>(nk, r, Bm, ws.ldr, 1, tc::BM, P.kpad1,
                                                                  P.a1h[dir].p, P.a1l[dir].p);
      k_split_op<<<gridn((size_t)P.mpad2 * P.kpad2), 256, 0, st>>>(nk, r, Am, ws.ldr, 0, P.mpad2, P.kpad2,
                                                                   P.a2h[dir].p, P.a2l[dir].p);
      lyap_count_launch(2);
      LY_CUDA(cudaGetLastError());
      LY_TRY(tc::make_map(&P.m1[dir].a_hi, P.a1h[dir].p, tc::BM, P.kpad1, tc::BM));
      LY_TRY(tc::make_map(&P.m1[dir].a_lo, P.a1l[dir].p, tc::BM, P.kpad1, tc::BM));
      LY_TRY(tc::make_map(&P.m2[dir].a_hi, P.a2h[dir].p, P.mpad2, P.kpad2, tc::BM));
      LY_TRY(tc::make_map(&P.m2[dir].a_lo, P.a2l[dir].p, P.mpad2, P.kpad2, tc::BM));
    }
    P.ncap = 0;  // the panels' K extents changed
  }
  if (B > P.ncap) {
    const int cap = ((B + tc::BN - 1) / tc::BN) * tc::BN;
    // K split of GEMM 1: about one CTA per SM over the batch's column tiles
    const int want = std::max(1, 152 / (cap / tc::BN));
    P.splits = tc::splits_for(P.kpad1, want);
    LY_TRY(P.b1h.alloc((size_t)cap * P.kpad1));
    LY_TRY(P.b1l.alloc((size_t)cap * P.kpad1));
    LY_TRY(P.b2h.alloc((size_t)cap * P.kpad2));
    LY_TRY(P.b2l.alloc((size_t)cap * P.kpad2));
    LY_TRY(P.d1.alloc((size_t)P.splits * cap * tc::BM));
    LY_TRY(P.d2.alloc((size_t)cap * P.mpad2));
    // K padding of the panels stays zero (their rows are written up to 2 nk / 2 r)
    LY_CUDA(cudaMemsetAsync(P.b1h.p, 0, P.b1h.bytes(), st));
    LY_CUDA(cudaMemsetAsync(P.b1l.p, 0, P.b1l.bytes(), st));
    LY_CUDA(cudaMemsetAsync(P.b2h.p, 0, P.b2h.bytes(), st));
    LY_CUDA(cudaMemsetAsync(P.b2l.p, 0, P.b2l.bytes(), st));
    for (int dir = 0; dir < 2; ++dir) {
      LY_TRY(tc::make_map(&P.m1[dir].b_hi, P.b1h.p, cap, P.kpad1, tc::BN));
      LY_TRY(tc::make_map(&P.m1[dir].b_lo, P.b1l.p, cap, P.kpad1, tc::BN));
      LY_TRY(tc::make_map(&P.m2[dir].b_hi, P.b2h.p, cap, P.kpad2, tc::BN));
      LY_TRY(tc::make_map(&P.m2[dir].b_lo, P.b2l.p, cap, P.kpad2, tc::BN));
    }
    P.ncap = cap;
  }
  *out = &P;
  return LYAP_OK;
}

template <typename T2, int K>
int launch_prec(lyap_seed* sd, const WoodState* ws, bool adjoint, const double* vinv, const int* list,
                const int* count, int B, const T2* In, size_t in_ss, T2* Out, size_t out_ss, cudaStream_t st) {
  constexpr int RT = PrecTile<K>::RT;
  const int n = sd->n;
  const int r = ws ? ws->r : 0;
  const int ntx = (n + RT - 1) / RT;
  const dim3 grid(ntx, (B + PST - 1) / PST);
  const float2* A = ws ? (adjoint ? ws->Ml : ws->Nl) : nullptr;
  const float2* Bm = ws ? (adjoint ? ws->Nl : ws->Ml) : nullptr;
  if constexpr (std::is_same<T2, float2>::value) {
    if (r > 0) {
      // each step is its own span of the kernel accounting (the two
      // products under prec_gemm); flops and bytes per system
      if (!ws->err) return LYAP_EINVAL;
      PrecTcState* P = nullptr;
      LY_TRY(ensure_prec_tc(sd, *ws, B, st, &P));
      const int dir = adjoint ? 1 : 0;
      const double N = (double)n * K;
      const dim3 gz((n + WT - 1) / WT, B);
      int ph = prof_begin(PK_PRECOND, st);
      k_prec_z<K><<<gz, WT, 0, st>>>(n, list, count, sd->Gdf.p, dir, vinv, In, in_ss, Out, out_ss, P->kpad1,
                                     P->b1h.p, P->b1l.p);
      prof_end(ph, st, 8.0 * N * K, 16.0 * N + 8.0 * N, 0, count);
      ph = prof_begin(PK_PRECGEMM, st);
      const size_t dstride = (size_t)P->ncap * tc::BM;
      LY_TRY(tc::launch_split(P->m1[dir], P->d1.p, tc::BM, 2 * r, tc::BM, P->kpad1, count, 1, B, B, P->splits, dstride,
                              ws->err, st));
      prof_end(ph, st, 3.0 * 2.0 * (2.0 * r) * (2.0 * N), 0.0, 0, count);
      ph = prof_begin(PK_PRECOND, st);
      k_prec_ytc<<<B, WT, 0, st>>>(list, count, dir, r, ws->cinv, P->d1.p, tc::BM, P->splits, dstride, P->kpad2,
                                   P->b2h.p, P->b2l.p);
      prof_end(ph, st, 8.0 * r * r, 8.0 * r * r + 8.0 * r * P->splits, 0, count);
      ph = prof_begin(PK_PRECGEMM, st);
      LY_TRY(tc::launch(P->m2[dir], P->d2.p, P->mpad2, 2 * n * K, P->mpad2, P->kpad2, count, 1, B, B, ws->err, st));
      prof_end(ph, st, 3.0 * 2.0 * (2.0 * N) * (2.0 * r), 0.0, 0, count);
      ph = prof_begin(PK_PRECOND, st);
      k_prec_dtc<K><<<gz, WT, 0, st>>>(n, list, count, sd->Gdf.p, dir, vinv, P->d2.p, P->mpad2, Out, out_ss);
      prof_end(ph, st, 8.0 * N * K, 24.0 * N, 0, count);
      lyap_count_launch(3);
      LY_CUDA(cudaGetLastError());
      return LYAP_OK;
    }
  }
  k_prec_a<T2, K><<<grid, WT, 0, st>>>(n, list, count, sd->Gdf.p, adjoint ? 1 : 0, vinv, In, in_ss, Out, out_ss, r, Bm,
                                       ws ? ws->ldr : 0, ws ? ws->cpart : nullptr, B);
  lyap_count_launch();
  if (r > 0) {
    k_prec_y<<<B, WT, 0, st>>>(list, count, adjoint ? 1 : 0, r, ws->cinv, ws->cpart, B, ntx);
    k_prec_b<T2, K><<<grid, WT, 0, st>>>(n, list, count, sd->Gdf.p, adjoint ? 1 : 0, vinv, Out, out_ss, r, A, ws->ldr,
                                         ws->cpart);
    lyap_count_launch(2);
  }
  return LYAP_OK;
}


__global__ void k_gather_cinv(const float2* __restrict__ src, const int* __restrict__ idx, int B, int rr,
                              float2* __restrict__ dst) {
  const size_t total = (size_t)B * rr;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const size_t c = e / rr, o = e % rr;
    dst[e] = src[(size_t)idx[c] * rr + o];
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
  ++sd->tsvd_gen;  // operands built from the previous factors are stale
  sd->resident_bytes += sd->tsvd_N.bytes() + sd->tsvd_M.bytes();
  return LYAP_OK;
}

int wood_bind(lyap_seed* sd, int r, int B, const float2* cinv_full, const int* idx, WoodState& ws, cudaStream_t st) {
  r = std::min(r, sd->tsvd_r);
  ws.r = r;
  ws.B = B;
  ws.Nl = sd->tsvd_N.p;
  ws.Ml = sd->tsvd_M.p;
  ws.ldr = sd->n * sd->k;
  if (r <= 0 || B <= 0) return LYAP_OK;
  const size_t total = (size_t)B * r * r;
  k_gather_cinv<<<gridn(total), 256, 0, st>>>(cinv_full, idx, B, r * r, ws.cinv);
  lyap_count_launch();
  LY_CUDA(cudaGetLastError());
  return LYAP_OK;
}

size_t wood_part_count(int n, int k, int B, int r) {
  const int RT = k <= 4 ? PrecTile<1>::RT : PrecTile<8>::RT;
  return (size_t)((n + RT - 1) / RT) * (size_t)B * (size_t)std::max(r, 0);
}

int wood_prepare(lyap_seed* sd, int r, int B, const double* vinv, bool /*adjoint*/, WoodState& ws, cudaStream_t st) {
  r = std::min(r, sd->tsvd_r);
  ws.r = r;
  ws.B = B;
  ws.Nl = sd->tsvd_N.p;
  ws.Ml = sd->tsvd_M.p;
  ws.ldr = sd->n * sd->k;
  if (r <= 0 || B <= 0) return LYAP_OK;
  const int ph = prof_begin(PK_CAPBUILD, st);
  int rc = LYAP_EINVAL;
  switch (sd->k) {
    case 1: rc = launch_cap_build<1>(sd, r, B, vinv, ws, st); break;
    case 2: rc = launch_cap_build<2>(sd, r, B, vinv, ws, st); break;
    case 3: rc = launch_cap_build<3>(sd, r, B, vinv, ws, st); break;
    case 4: rc = launch_cap_build<4>(sd, r, B, vinv, ws, st); break;
    case 5: rc = launch_cap_build<5>(sd, r, B, vinv, ws, st); break;
    case 6: rc = launch_cap_build<6>(sd, r, B, vinv, ws, st); break;
    case 7: rc = launch_cap_build<7>(sd, r, B, vinv, ws, st); break;
    case 8: rc = launch_cap_build<8>(sd, r, B, vinv, ws, st); break;
  }
  if (rc != LYAP_OK) return rc;
  lyap_count_launch();
  prof_end(ph, st, 8.0 * sd->n * sd->k * r * r + 16.0 * r * r * r, 0.0, B, nullptr);
  LY_CUDA(cudaGetLastError());
  return LYAP_OK;
}

template <typename T2>
int prec_apply(lyap_seed* sd, const WoodState* ws, bool adjoint, const double* vinv, const int* list,
               const int* count, int B, const T2* In, size_t in_ss, T2* Out, size_t out_ss, cudaStream_t st) {
  if (ws && ws->r <= 0) ws = nullptr;
  const bool gemm_form = std::is_same<T2, float2>::value && ws;  // accounts its own steps
  const int ph = gemm_form ? -1 : prof_begin(PK_PRECOND, st);
  int rc = LYAP_OK;
  switch (sd->k) {
    case 1: rc = launch_prec<T2, 1>(sd, ws, adjoint, vinv, list, count, B, In, in_ss, Out, out_ss, st); break;
    case 2: rc = launch_prec<T2, 2>(sd, ws, adjoint, vinv, list, count, B, In, in_ss, Out, out_ss, st); break;
    case 3: rc = launch_prec<T2, 3>(sd, ws, adjoint, vinv, list, count, B, In, in_ss, Out, out_ss, st); break;
    case 4: rc = launch_prec<T2, 4>(sd, ws, adjoint, vinv, list, count, B, In, in_ss, Out, out_ss, st); break;
    case 5: rc = launch_prec<T2, 5>(sd, ws, adjoint, vinv, list, count, B, In, in_ss, Out, out_ss, st); break;
    case 6: rc = launch_prec<T2, 6>(sd, ws, adjoint, vinv, list, count, B, In, in_ss, Out, out_ss, st); break;
    case 7: rc = launch_prec<T2, 7>(sd, ws, adjoint, vinv, list, count, B, In, in_ss, Out, out_ss, st); break;
    case 8: rc = launch_prec<T2, 8>(sd, ws, adjoint, vinv, list, count, B, In, in_ss, Out, out_ss, st); break;
    default: return LYAP_EINVAL;
  }
  if (rc != LYAP_OK) return rc;
  // algorithmic bytes per system: read r, write z, read+write z again when r > 0
  const int r = ws ? ws->r : 0;
  const double N = (double)sd->n * sd->k;
  if (!gemm_form)
    prof_end(ph, st, 8.0 * N * sd->k + (r > 0 ? 16.0 * N * r + 8.0 * N * sd->k + 8.0 * r * r : 0.0),
             N * sizeof(T2) * (r > 0 ? 4.0 : 2.0), 0, count);
  LY_CUDA(cudaGetLastError());
  return LYAP_OK;
}

template int prec_apply<double2>(lyap_seed*, const WoodState*, bool, const double*, const int*, const int*, int,
                                 const double2*, size_t, double2*, size_t, cudaStream_t);
template int prec_apply<float2>(lyap_seed*, const WoodState*, bool, const double*, const int*, const int*, int,
                                const float2*, size_t, float2*, size_t, cudaStream_t);
