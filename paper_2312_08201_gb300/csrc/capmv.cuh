// Capacitance operator of the SMW formula (paper §2.1, eq. (SMW_linearsystem)),
// applied matrix-free.
//
// With Lc_ij = 1/(lam_i + lam_j), Ub = Qp^{-1} B_l, Vb = Qp^T B_r, the paper's
// operator N^T L0^{-1} M acts on w = [vec(W1); vec(W2)] as
//     Y = Lc o (W1 Ub^T + Ub W2),   N^T L0^{-1} M w = [vec(Y Vb); vec(Vb^T Y)].
// The right-hand side and the solution stay in the subspace W2 = W1^T
// (symmetric Y), so only the n x k block W = W1 is carried:
//     C0(W)[:, t] = sum_p W_p o Gd[:, p, t] + sum_p Ub_p o (Lc (W_p o Vb_t)),
// with Gd[:, p, t] = Lc (Ub_p o Vb_t) the diagonal blocks of eq. (N1M1). The
// second sum is one product of Lc with an n x k^2 panel per system; over a
// batch of systems it is a GEMM with the shared Cauchy matrix, followed by a
// fused epilogue that multiplies by Ub, adds the Gd term and applies
// T(v) W = W D(v)^{-1} - C0(W).
//
// The transposed operator T(v)^T (adjoint solve for the gradient) is the same
// with Ub and Vb exchanged and Gd[:, p, t] -> Gd[:, t, p].
#pragma once
#include <cuda_runtime.h>

enum CapMode { CAP_C0 = 0, CAP_T = 1, CAP_RESID = 2 };

struct CapArgs64 {
  int n, k;
  const double2* lam;  // n eigenvalues
  const double2* P1;   // n x k: Ub (primal) or Vb (adjoint)
  const double2* P2;   // n x k: Vb (primal) or Ub (adjoint)
  const double2* Gd;   // n x k x k
  int gT;              // 1: use Gd[:, t, p]
  const double2* W;    // inputs, system b at W + b * ldw
  size_t ldw;
  const double* vinv;  // 1/v, system b at vinv + b*k (T and RESID modes)
  const double2* rhs;  // RESID: system b at rhs + b * ldr (ldr = 0: shared)
  size_t ldr;
  double2* out;  // system b at out + b * ldo
  size_t ldo;
  int mode;
  const int* list;   // optional: tile system s -> b = list[s]
  const int* count;  // optional: number of listed systems (device)
  int nsys;          // systems when list == nullptr; upper bound otherwise
};

int capmv64_launch(const CapArgs64& a, cudaStream_t st);

// The same operator in float-float arithmetic on the FP32 pipes (FP64-level
// accuracy; see capmv_df.cu). Lff: n x n pairs (re hi, re lo, im hi, im lo) of
// lc_scale * Lc, built by capmv_df_build_lc; p_scale: power of two applied to
// P2; sw: device scratch indexed by system (>= largest system index + 1),
// overwritten with each listed system's W scale; panel: device scratch of
// nsys k^2 n float4 (the float-float panel of each listed system).
int capmv_df_build_lc(int n, const double2* lam, double lc_scale, float4* Lff, cudaStream_t st);
int capmv_df_launch(const CapArgs64& a, const float4* Lff, double lc_scale, double p_scale, double* sw,
                    float4* panel, cudaStream_t st);
