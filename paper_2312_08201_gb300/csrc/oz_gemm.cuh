// FP64-accuracy Cauchy-panel product on the BF16 tensor cores by exact
// integer slicing (the splitting scheme of Ozaki et al. for error-free
// matrix products), used for the mixed path's refinement residual.
//
// Every row r of the real-split Cauchy matrix A (2n x 2n; for exactly real
// eigenvalues the real n x n matrix, with the real and imaginary parts of a
// panel column as two columns) and every panel column c of B (one
// (system, p, t) column, K = 2n or n) is scaled by a power of
// two so that its entries lie in [-1/2, 1/2], then written as NS = 8
// balanced base-64 digits:
//     A[r][k] = 2^eA[r] sum_s a_s[r][k] 64^-(s+1),   a_s in [-32, 32],
// exact up to 2^-49 of the row's scale (the same for B). The digits are
// small integers, hence exact in BF16, and a digit product is at most 2^10.
// For each order d = s + t <= NS - 1 the tensor cores accumulate
//     ACC_d[r][c] = sum_{s+t=d} sum_k a_s[r][k] b_t[c][k]
// in FP32. Every partial sum is an integer below (d+1) K 2^10 <= NS K 2^10,
// which stays below 2^24 (no rounding) for K <= 2046; longer K runs in
// chunks of KCHUNK whose exact results are added in float-float. The result
//     D[r][c] = 2^(eA[r] + eB[c] - 12) sum_d 64^-d ACC_d[r][c]
// is combined in float-float; dropping the orders d >= NS leaves an error of
// about 2^-47 of |A||B|^T.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "capmv.cuh"

namespace oz {

constexpr int NS = 8;            // digits per operand
constexpr int BM = 128;          // rows of A per CTA (TMEM lanes)
constexpr int BN = 64;           // panel columns per CTA (per order accumulator)
constexpr int BK = 32;           // K per stage: 32 BF16 = one 64-byte swizzle row
constexpr int STAGES = 2;
constexpr int KMAX = 2046;       // largest K with exact FP32 accumulation
constexpr int KCHUNK = 2016;     // K per accumulation chunk (a multiple of BK, at most KMAX)

// Digits of the Cauchy matrix of a seed (rows mpad, K kpad): real-split
// (2n x 2n, rs = 2) or, for exactly real eigenvalues, the real n x n matrix
// (rs = 1). S: NS x mpad x kpad BF16 (slice-major), eA: mpad exponents.
int slice_A(int n, const double2* lam, int mpad, int kpad, int rs, void* S, int* eA, cudaStream_t st);

// Operand maps (64-byte swizzle, box BK x rows) over slice-stacked matrices.
int make_map(CUtensorMap* map, const void* base, int rows_total, int kpad, int box_rows);

struct Panel {
  void* S = nullptr;        // NS x ncap x kpad BF16 digits of B
  int* eB = nullptr;        // ncap exponents
  float2* D = nullptr;      // ncap x mpad float-float results (hi, lo)
  int ncap = 0;             // panel columns the buffers hold (multiple of BN)
  CUtensorMap mapB;
};

// r = rhs - T(v) W (CAP_RESID) or T(v) W (CAP_T) for the listed systems of a
// (n, k, W, P1, P2, Gd, vinv, rhs, out, list, count): digits of the panel,
// the tensor-core product, and the FP64 epilogue. mapA/eA: the seed's
// digits, in the layout rs of slice_A; with rs = 1 every panel column is two
// columns (real and imaginary parts), so pn holds 2 k^2 columns per system;
// err: device flag for an expired bounded wait.
int residual(const CapArgs64& a, const CUtensorMap& mapA, const int* eA, int mpad, int kpad, int rs, Panel& pn,
             int* err, cudaStream_t st);

}  // namespace oz
