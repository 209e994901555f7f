// Kernel accounting: a process-wide launch counter and, when enabled, CUDA
// event pairs around selected kernels together with the algorithmic work
// (flops and bytes the method requires) of each launch. The unit count of
// a launch may live on the device (active-system lists); it is copied to
// pinned host memory after the launch and read when the profile is read.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

enum ProfKernel {
  PK_CAPMV64 = 0,   // FP64 capacitance matvec (Cauchy-panel GEMM)
  PK_TCGEMM = 1,    // tcgen05 Cauchy-panel GEMM (mixed path)
  PK_ORTHO = 2,     // CGS2 Arnoldi orthogonalisation
  PK_PRECOND = 3,   // preconditioner apply (block-Jacobi + Woodbury term)
  PK_GRAM = 4,      // batched Gram matrices (recycle update)
  PK_TSMM = 5,      // batched tall-skinny products
  PK_RITZ = 6,      // harmonic-Ritz small dense problems
  PK_EPI32 = 7,     // FP32 operator epilogue (mixed path)
  PK_LSQ = 8,       // (no launches: the Givens step runs in the orthogonalisation kernel)
  PK_CYCLE = 9,     // cycle start/solve/update kernels
  PK_PANEL = 10,    // panel build for the tensor-core GEMM
  PK_RECSTART = 11, // recycle start (AU, CholQR2, projection)
  PK_CAPMV_FF = 12, // float-float capacitance matvec (mixed-path residual);
                    // its "flops" are FP32 lane instructions
  PK_CAPBUILD = 13, // Woodbury capacitance Cap(v)^{-1} per system
  PK_OZGEMM = 14,   // integer-sliced tensor-core residual product (mixed path)
  PK_PRECGEMM = 15, // the Woodbury apply's two tcgen05 products (FP32 path)
  PK_COUNT = 16
};

void lyap_count_launch(int n = 1);

// Returns a handle (>= 0) or -1 when profiling is off. Units per launch are
// either `units_host` (if units_dev == nullptr) or *units_dev at launch end.
int prof_begin(int kernel, cudaStream_t st);
void prof_end(int handle, cudaStream_t st, double flops_per_unit, double bytes_per_unit, int units_host,
              const int* units_dev);
