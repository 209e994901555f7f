/*
 * Testing hooks of liblyap: direct access to single kernels so that tests can
 * check them against reference products. Not needed to solve anything.
 */
#ifndef LYAP_TESTING_H
#define LYAP_TESTING_H

#include "lyap.h"

#ifdef __cplusplus
extern "C" {
#endif

/* out_b = T(v_b) w_b for nsys systems (the operator of eq. (SMW_linearsystem)
 * in the reduced unknown W = W1, see lyap.h), or T(v_b)^T w_b when adjoint.
 * v: device, nsys x k row-major; w, out: device, nsys x n x k complex128
 * (column-major per system). precision LYAP_FP64 uses the FP64 Cauchy-panel
 * kernel; LYAP_BF16_IR the tensor-core operator of the mixed path (inputs
 * rounded to FP32, BF16-split GEMM, FP32 epilogue); LYAP_TEST_FF the
 * float-float kernel of the mixed path's refinement residual (FP64 in and
 * out, float-float products). Synchronises. Returns LYAP_EDEVICE_TIMEOUT if
 * a bounded device wait expired. */
#define LYAP_TEST_FF 3
/* precision for lyap_test_apply: the integer-sliced tensor-core product of the
 * mixed path's TC residual (FP64 in and out; n <= 1023) */
#define LYAP_TEST_TC 4
int lyap_test_apply(lyap_seed* seed, int nsys, const double* v, const double* w, int precision, int adjoint,
                    double* out);

/* D = A B^T through the tcgen05 kernel with BF16-split operands:
 * A: device M x K row-major float, B: device N x K row-major float,
 * D: device N x M row-major float (D[n*M + m] = sum_k A[m,k] B[n,k]).
 * Allocates temporaries. Synchronises. */
int lyap_test_tc_gemm(int M, int N, int K, const float* A, const float* B, float* D);

#ifdef __cplusplus
}
#endif

#endif /* LYAP_TESTING_H */
