// Mixed-precision path: FP32 inner solves whose Cauchy GEMM runs on tcgen05
// tensor cores, wrapped in refinement on the FP64 capacitance residual.
#pragma once
#include "lyap_internal.h"
#include "solver.h"

// Build the low-precision Cauchy operands of a seed (called by the factor).
int lyap_mixed_prepare(lyap_seed* sd, cudaStream_t st);
void lyap_mixed_free(lyap_seed* sd);

// Solve the chunk's Bc systems (vinv already in the seed work area) to the
// FP64 residual tolerance; W' (and the adjoint Z when Zadj_out != nullptr)
// are written as FP64 complex, Bc x n*k. Rres_out (Bc x n*k) receives the
// FP64 residual P - T(v) W' of each system's final iterate, as evaluated by
// the refinement's last step.
int lyap_mixed_chunk(lyap_seed* sd, int Bc, const double* vinv, const lyap_opts& o, const SolveParams& prm,
                     cudaStream_t st, KrylovWS<float2>& ws, KrylovWS<float2>& wsadj, double2* Wp_out,
                     double2* Zadj_out, double2* Rres_out, std::vector<int>& iters, std::vector<int>& status,
                     std::vector<int>& rsteps);
