// Preconditioner of eq. (prec) with the truncated-SVD coupling (paper §2.1).
//
// In the reduced unknown W (n x k, vec index t*n + i) the capacitance
// operator splits as T(v) = K(v) - O with
//   K(v) W[:, t] = W[:, t] / v_t - sum_p W[:, p] o Gd[:, p, t]  (block diagonal:
//        one k x k matrix per row i, the diagonal blocks of eq. (N1M1)),
//   O(W)[:, t]   = sum_p Ub_p o (Lc (W_p o Vb_t))                (the off-diagonal
//        blocks of eqs. (N2M1), (N1M2), v-independent).
// The paper approximates the off-diagonal blocks by their truncated SVD of
// rank pbar: O ~ Nl Ml^T (Nl, Ml: nk x pbar). Then
//   P(v) = K(v) - Nl Ml^T,
//   P(v)^{-1} r = K^{-1} r + K^{-1} Nl Cap^{-1} Ml^T K^{-1} r,
//   Cap(v) = I - Ml^T K(v)^{-1} Nl                      (pbar x pbar per v),
// the Sherman-Morrison-Woodbury form of the paper's Schur-complement apply
// (restricted to the invariant subspace W2 = W1^T it is the same operator).
// The adjoint operator T^T = K^T - O^T uses O^T ~ Ml Nl^T and Cap^T.
#pragma once
#include <cuda_runtime.h>

struct lyap_seed;

struct WoodState {
  int r = 0;             // rank in use (0: block-Jacobi only)
  int B = 0;             // systems with an inverted Cap
  float2* cinv = nullptr;  // B x r x r: Cap^{-1}, column-major
  float2* cpart = nullptr; // wood_part_count(n, k, B, r) entries: partial sums of the apply
  const float2* Nl = nullptr;  // nk x rmax (seed)
  const float2* Ml = nullptr;
  int ldr = 0;  // leading dimension (rows) of Nl/Ml = nk
  int* err = nullptr;  // device flag for an expired bounded wait (FP32 path's tensor-core products)
};

// Tensor-core operands of the FP32 path's apply (owned by the seed).
void lyap_prec_tc_free(lyap_seed* sd);

// Offline: rank-r truncated SVD of the coupling operator (randomized, two
// power iterations). Builds seed-resident Nl, Ml (FP32) once per rank.
int lyap_tsvd_prepare(lyap_seed* sd, int r, cudaStream_t st);

// Entries of WoodState::cpart that a batch of B systems needs.
size_t wood_part_count(int n, int k, int B, int r);

// Per chunk: invert Cap(v_b) for systems b < B (vinv: B x k) into ws.cinv
// (caller-owned, B r^2 entries). ws must stay alive while the chunk runs.
int wood_prepare(lyap_seed* sd, int r, int B, const double* vinv, bool adjoint, WoodState& ws, cudaStream_t st);

// Per refinement step: ws.cinv[c] = cinv_full[idx[c]] for c < B (Cap(v)
// depends on v only, so the inverses of a chunk are built once).
int wood_bind(lyap_seed* sd, int r, int B, const float2* cinv_full, const int* idx, WoodState& ws, cudaStream_t st);

// Out_b = P(v_b)^{-1} In_b for the listed systems: block-Jacobi K^{-1}, plus
// the Woodbury term K^{-1} Nl Cap^{-1} Ml^T K^{-1} when ws has rank > 0
// (ws == nullptr: block-Jacobi only). Adjoint: P^T.
template <typename T2>
int prec_apply(lyap_seed* sd, const WoodState* ws, bool adjoint, const double* vinv, const int* list,
               const int* count, int B, const T2* In, size_t in_ss, T2* Out, size_t out_ss, cudaStream_t st);
