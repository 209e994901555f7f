// tcgen05 (5th-generation tensor core) GEMM for the Cauchy-panel product of
// the mixed-precision capacitance operator:
//     D[col][row] = sum_kx A[row][kx] * B[col][kx],
// A = real-split Cauchy matrix (2n x 2n, K-major), B = real-split panel
// (one row of K per panel column, K-major), both given as two BF16 terms
// (x = hi + lo); D accumulates hi*hi + hi*lo + lo*hi in FP32 (TMEM).
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace tc {

constexpr int BM = 128;   // rows of A per CTA (TMEM lanes)
constexpr int BN = 128;   // panel columns per CTA (TMEM columns)
constexpr int BK = 64;    // K per stage: 64 BF16 = one 128-byte swizzle row
constexpr int STAGES = 3;

struct Maps {
  CUtensorMap a_hi, a_lo, b_hi, b_lo;
};

// Encode a 2-D BF16 K-major tensor map (rows x kpad, row stride kpad*2 bytes)
// with a box of box_rows x 64 and 128-byte swizzle.
int make_map(CUtensorMap* map, const void* base, int rows, int kpad, int box_rows);

// D (ldd floats per column) for columns [0, ncols) where ncols = *count *
// col_mult when count != nullptr (device), else ncols_host. Grid covers
// mpad/BM x ceil(ncols_cap/BN); tiles past ncols exit at once. err: device
// int set non-zero if a bounded wait expired. inject_no_tma (test hook of
// LYAP_INJECT_DEVICE_WAIT): no copy is issued, every wait is short, the
// MMA warp's wait runs out, err is set and D is left untouched.
int launch(const Maps& m, float* D, int ldd, int mrows, int mpad, int kpad, const int* count, int col_mult,
           int ncols_host, int ncols_cap, int* err, cudaStream_t st, bool inject_no_tma = false);

// The same product with K split `splits` ways (grid z): split z sums its
// share of the k-tiles and writes its partial D at D + z * split_stride
// (floats); the caller adds the partials. Every split must get at least one
// k-tile (splits_for picks the largest count <= want that does).
int launch_split(const Maps& m, float* D, int ldd, int mrows, int mpad, int kpad, const int* count, int col_mult,
                 int ncols_host, int ncols_cap, int splits, size_t split_stride, int* err, cudaStream_t st,
                 bool inject_no_tma = false);
int splits_for(int kpad, int want);

}  // namespace tc
