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

// Continuous batching of one seed's mixed-path solves (the server's engine):
// `cap` persistent slots; systems join at a refinement-step boundary and
// retire when their FP64 residual meets refine_tol (or fails).
struct MixedEngine;
struct EngineJoin {
  int slot;         // a free slot
  const double* v;  // k parameters (host)
};
struct EngineDone {
  int slot;
  double f;
  lyap_result_info info;
};
int lyap_engine_create(lyap_seed* sd, int cap, const lyap_opts& o, MixedEngine** out);
void lyap_engine_free(lyap_seed* sd, MixedEngine* e);
int lyap_engine_free_slots(const MixedEngine* e);
int lyap_engine_step(lyap_seed* sd, MixedEngine& e, const lyap_opts& o, cudaStream_t st,
                     const std::vector<EngineJoin>& joins, std::vector<EngineDone>& done);
