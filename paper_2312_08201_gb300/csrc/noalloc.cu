// Allocation-free FP64 check of given capacitance solutions.
//
// Some callers cannot call cudaMalloc while they run: hosts whose device
// memory is carved out once at start-up by their own pool and must not grow
// afterwards, and plug-ins that run inside another framework's allocator and
// may not go around it. lyap_check_solution_noalloc serves them: it
// evaluates f(v) = trace(E X(v)) and the relative FP64 capacitance residual
// for solutions W' the caller already holds, with every intermediate in the
// static device array below instead of fresh allocations.
//
// The array holds LYAP_NOALLOC_SCRATCH complex doubles (33 MiB, 34,603,008
// bytes): enough for nv * n * k <= 2^21 residual entries together with the
// nv * k reciprocals of v. Every GPU that loads the library keeps it until
// the process exits. All calls share it and it keeps the last call's
// contents: calls that overlap on the GPU (different streams, or host
// threads without ordering) race on it. Every element a call reads was
// written earlier in the same call, so no part of it has to start at zero
// and nothing is cleared.
#include <mutex>

#include "capmv.cuh"
#include "cplx.cuh"
#include "krylov.cuh"
#include "lyap_internal.h"
#include "prof.h"

#define LYAP_NOALLOC_SCRATCH LYAP_NOALLOC_MAX_ENTRIES

namespace {

static __device__ __align__(256) double2 g_noalloc_scratch[LYAP_NOALLOC_SCRATCH];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
double2* g_scratch_ptr[kMaxDevices] = {nullptr};

// 1/v for every entry; a zero or non-finite v_i gives NaN, which then shows
// in the residual of its system.
__global__ void k_noalloc_vinv(int count, const double* __restrict__ v, double* __restrict__ vinv) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  double x = v[i];
  vinv[i] = (x != 0.0 && isfinite(x)) ? 1.0 / x : __longlong_as_double(0x7ff8000000000000LL);
}

// trace[b] = f0 + Re <h, W'_b>,  resid[b] = ||r_b|| / ||Ph|| (r in scratch)
__global__ void __launch_bounds__(kry::NT) k_noalloc_reduce(int N, int nv, const double2* __restrict__ W,
                                                            const double2* __restrict__ h,
                                                            const double2* __restrict__ r, double f0, double ph_norm,
                                                            double* __restrict__ trace, double* __restrict__ resid) {
  __shared__ double red[64];
  const int b = blockIdx.x;
  if (b >= nv) return;
  double acc[2] = {0.0, 0.0};
  for (int e = threadIdx.x; e < N; e += kry::NT) {
    acc[0] += cmul(W[(size_t)b * N + e], h[e]).x;
    acc[1] += cabs2(r[(size_t)b * N + e]);
  }
  kry::block_sum<2>(acc, red);
  if (threadIdx.x == 0) {
    trace[b] = f0 + acc[0];
    resid[b] = ph_norm > 0 ? sqrt(acc[1]) / ph_norm : sqrt(acc[1]);
  }
}

// Device address of the scratch array for the current device, looked up once.
int scratch_for_current_device(double2** out) {
  int dev = -1;
  LY_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return LYAP_EINVAL;
  std::lock_guard<std::mutex> lk(g_setup_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      lyap_set_last_error(std::string("cudaGetSymbolAddress(no-alloc scratch): ") + cudaGetErrorString(e));
      return LYAP_ECUDA;
    }
    g_scratch_ptr[dev] = static_cast<double2*>(p);
  }
  *out = g_scratch_ptr[dev];
  return LYAP_OK;
}

}  // namespace

extern "C" int lyap_check_solution_noalloc(lyap_seed* seed, int nv, const double* v, const double* w,
                                           double* trace_out, double* resid_out, void* stream) {
  if (!seed || nv < 0 || (nv > 0 && (!v || !w || !trace_out || !resid_out))) return LYAP_EINVAL;
  if (nv == 0) return LYAP_OK;
  const int n = seed->n, k = seed->k;
  const size_t N = (size_t)n * k;
  const size_t n_vinv = ((size_t)nv * k + 1) / 2;  // doubles packed in double2 slots
  const size_t need = n_vinv + (size_t)nv * N;
  if (need > LYAP_NOALLOC_SCRATCH) {
    lyap_set_last_error("lyap_check_solution_noalloc: nv*n*k + nv*k/2 = " + std::to_string(need) +
                        " exceeds the static scratch of " + std::to_string(LYAP_NOALLOC_SCRATCH) +
                        " complex doubles; split the call");
    return LYAP_EINVAL;
  }
  LY_CUDA(cudaSetDevice(seed->device));
  double2* scratch = nullptr;
  LY_TRY(scratch_for_current_device(&scratch));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  double* vinv = reinterpret_cast<double*>(scratch);
  double2* r = scratch + n_vinv;
  k_noalloc_vinv<<<(nv * k + 255) / 256, 256, 0, st>>>(nv * k, v, vinv);
  lyap_count_launch();
  LY_CUDA(cudaGetLastError());
  CapArgs64 a{};
  a.n = n;
  a.k = k;
  a.lam = seed->lam.p;
  a.P1 = seed->Ub.p;
  a.P2 = seed->Vb.p;
  a.Gd = seed->Gd.p;
  a.W = reinterpret_cast<const double2*>(w);
  a.ldw = N;
  a.vinv = vinv;
  a.rhs = seed->Ph.p;
  a.ldr = 0;
  a.out = r;
  a.ldo = N;
  a.mode = CAP_RESID;
  a.nsys = nv;
  LY_TRY(capmv64_launch(a, st));
  k_noalloc_reduce<<<nv, kry::NT, 0, st>>>((int)N, nv, reinterpret_cast<const double2*>(w), seed->h.p, r, seed->f0,
                                           seed->ph_norm, trace_out, resid_out);
  lyap_count_launch();
  LY_CUDA(cudaGetLastError());
  return LYAP_OK;
}
