// Mixed-precision path (placeholder until the tensor-core operator lands).
#include "mixed.h"

int lyap_mixed_prepare(lyap_seed*, cudaStream_t) { return LYAP_OK; }

int lyap_mixed_chunk(lyap_seed*, int, const double*, const lyap_opts&, const SolveParams&, cudaStream_t,
                     KrylovWS<float2>&, KrylovWS<float2>&, double2*, double2*, std::vector<int>&,
                     std::vector<int>&, std::vector<int>&) {
  lyap_set_last_error("mixed precision path not available");
  return LYAP_EINVAL;
}

template <>
int SysOp<float2>::apply(const int*, const int*, int, const float2*, size_t, float2*, size_t, cudaStream_t) const {
  return LYAP_EINVAL;
}
template <>
int SysOp<float2>::apply_c0(int, const float2*, float2*, cudaStream_t) const { return LYAP_EINVAL; }
template <>
int SysOp<float2>::precond(const int*, const int*, int, const float2*, size_t, float2*, size_t,
                           cudaStream_t) const {
  return LYAP_EINVAL;
}
