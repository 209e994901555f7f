// C ABI of liblyap (declarations and documentation in include/lyap.h).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>

#include "cplx.cuh"
#include "krylov.cuh"
#include "lyap_internal.h"
#include "prof.h"
#include "mixed.h"
#include "precond.cuh"
#include "solver.h"

// ------------------------------------------------------------- last error
namespace {
thread_local std::string g_last_error;
}
void lyap_set_last_error(const std::string& msg) { g_last_error = msg; }
extern "C" const char* lyap_last_error(void) { return g_last_error.c_str(); }

int lyap_smem_optin(const void* func, size_t bytes) {
  static std::mutex mu;
  static std::map<std::pair<int, const void*>, size_t> done;
  int dev = -1;
  LY_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(mu);
  size_t& have = done[{dev, func}];
  if (have >= bytes) return LYAP_OK;
  LY_CUDA(cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
  have = bytes;
  return LYAP_OK;
}

// Workspaces cached per seed.
struct SeedWork {
  KrylovWS<double2> ws64, ws64adj;
  KrylovWS<float2> ws32, ws32adj;
  DevBuf<double> vinv, vdev;
  DevBuf<double2> Wp, Zadj, Rres, tmp;
  DevBuf<double> red0, red1, red2, red3;
  DevBuf<float2> wcinv, wpart;
  DevBuf<int> lst, cnt;  // system list of the error estimate
  DevBuf<int> vbad;      // device-side count of invalid parameters in the call
  int* vbad_host = nullptr;  // pinned copy, read at the chunk's sync
  WoodState wood;
  ~SeedWork() {
    if (vbad_host) cudaFreeHost(vbad_host);
  }
};

namespace {

// 1/v for every entry. An entry that is zero (excluded by §1) or not finite
// is counted in *bad and gets 1/v = 0, so the solve stays finite; the call
// reports LYAP_EINVAL when it reads the count.
__global__ void k_vinv(int count, const double* __restrict__ v, double* __restrict__ out, int* __restrict__ bad) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  const double x = v[i];
  const bool ok = x != 0.0 && isfinite(x);
  out[i] = ok ? 1.0 / x : 0.0;
  if (!ok) atomicAdd(bad, 1);
}

// f[b] = f0 + tr[b] into the caller's device output
__global__ void k_trace_out(int nsys, double f0, const double* __restrict__ tr, double* __restrict__ f) {
  int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b < nsys) f[b] = f0 + tr[b];
}

// grad[b, i] = v_i^{-2} Re sum_s Z_b[s, i] W_b[s, i]  (pairing without conjugation)
__global__ void k_grad(int n, int k, int nsys, const double2* __restrict__ W, const double2* __restrict__ Z,
                       const double* __restrict__ vinv, double* __restrict__ grad) {
  __shared__ double red[32];
  const int b = blockIdx.x / k, i = blockIdx.x % k;
  if (b >= nsys) return;
  const size_t N = (size_t)n * k;
  double acc[1] = {0.0};
  for (int s = threadIdx.x; s < n; s += blockDim.x) {
    double2 p = cmul(Z[(size_t)b * N + (size_t)i * n + s], W[(size_t)b * N + (size_t)i * n + s]);
    acc[0] += p.x;
  }
  kry::block_sum<1>(acc, red);
  if (threadIdx.x == 0) {
    double vi = vinv[(size_t)b * k + i];
    grad[(size_t)b * k + i] = vi * vi * acc[0];
  }
}

// out[b] = Re sum_e A_b[e] B_b[e]
__global__ void k_dot_pair(int N, int nsys, const double2* __restrict__ A, const double2* __restrict__ Bv,
                           double* __restrict__ out) {
  __shared__ double red[32];
  const int b = blockIdx.x;
  if (b >= nsys) return;
  double acc[1] = {0.0};
  for (int e = threadIdx.x; e < N; e += blockDim.x) acc[0] += cmul(A[(size_t)b * N + e], Bv[(size_t)b * N + e]).x;
  kry::block_sum<1>(acc, red);
  if (threadIdx.x == 0) out[b] = acc[0];
}

int grid_of(size_t n) { return (int)std::max<size_t>(1, std::min<size_t>((n + 255) / 256, 65535)); }

}  // namespace

// ------------------------------------------------------------------ options
extern "C" void lyap_opts_default(lyap_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->tol = 1e-12;
  o->refine_tol = 1e-11;
  o->inner_tol = 1e-3;
  o->maxit = 300;
  o->m = 40;
  o->s = 10;
  o->pbar = 50;
  o->batch = 0;
  o->precision = LYAP_FP64;
  o->max_refine = 10;
  o->hbm_budget = 0;
  o->stream = nullptr;
  o->inject = 0;
  o->residual = LYAP_RESID_TC;
}

extern "C" const char* lyap_strerror(int code) {
  switch (code) {
    case LYAP_OK: return "ok";
    case LYAP_PENDING: return "pending";
    case LYAP_EINVAL: return "invalid argument";
    case LYAP_ENOMEM: return "out of device memory or over budget";
    case LYAP_EUNSTABLE_SEED: return "seed matrix not stable (Lyapunov solution not unique)";
    case LYAP_ECUDA: return "CUDA error";
    case LYAP_ESOLVER: return "cuSOLVER/cuBLAS error";
    case LYAP_ENOCONV: return "no convergence within maxit";
    case LYAP_EBREAKDOWN: return "Krylov breakdown";
    case LYAP_EDEVICE_TIMEOUT: return "device wait timed out";
    case LYAP_ENOTFOUND: return "unknown seed or ticket";
    case LYAP_ENONFINITE: return "non-finite value in solve";
    case LYAP_ECANCELLED: return "cancelled";
    default: return "unknown status";
  }
}

int lyap_check_v(int nv, int k, const double* v) {
  for (size_t i = 0; i < (size_t)nv * k; ++i)
    if (!std::isfinite(v[i]) || v[i] == 0.0) {
      lyap_set_last_error("parameter " + std::to_string(i) + " is zero or not finite");
      return LYAP_EINVAL;
    }
  return LYAP_OK;
}

// ------------------------------------------------------------------ context
extern "C" int lyap_ctx_create(int device, lyap_ctx** out) {
  if (!out) return LYAP_EINVAL;
  *out = nullptr;
  int ndev = 0;
  LY_CUDA(cudaGetDeviceCount(&ndev));
  if (device < 0 || device >= ndev) return LYAP_EINVAL;
  LY_CUDA(cudaSetDevice(device));
  std::unique_ptr<lyap_ctx> c(new lyap_ctx());
  c->device = device;
  LY_CUDA(cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking));
  LY_BLAS(cublasCreate(&c->blas));
  LY_SOLVER(cusolverDnCreate(&c->solver));
  *out = c.release();
  return LYAP_OK;
}

extern "C" void lyap_ctx_destroy(lyap_ctx* c) {
  if (!c) return;
  cudaSetDevice(c->device);
  if (c->solver) cusolverDnDestroy(c->solver);
  if (c->blas) cublasDestroy(c->blas);
  if (c->stream) cudaStreamDestroy(c->stream);
  delete c;
}

static cudaStream_t pick_stream(lyap_ctx* c, const lyap_opts& o) {
  return o.stream ? static_cast<cudaStream_t>(o.stream) : c->stream;
}

// ---------------------------------------------------------------- seed factor
extern "C" int lyap_seed_factor(lyap_ctx* ctx, int n, int k, int g, const double* A0, const double* U,
                                const double* V, const double* G, const double* E, int mem_kind,
                                const lyap_opts* opts, lyap_seed** out, double* cond_Q_out) {
  if (!ctx || !out || !A0 || !U || !V || !G || n < 1 || k < 1 || k > 8 || k > n || g < 1) return LYAP_EINVAL;
  if (mem_kind != LYAP_MEM_HOST && mem_kind != LYAP_MEM_DEVICE) return LYAP_EINVAL;
  *out = nullptr;
  lyap_opts o;
  lyap_opts_default(&o);
  if (opts) o = *opts;
  (void)cudaGetLastError();  // a stale error of an unrelated earlier call is not this call's
  LY_CUDA(cudaSetDevice(ctx->device));
  cudaStream_t st = pick_stream(ctx, o);
  const size_t nn = (size_t)n * n;
  DevBuf<double> dA, dU, dV, dG, dE;
  const double *pA = A0, *pU = U, *pV = V, *pG = G, *pE = E;
  if (mem_kind == LYAP_MEM_HOST) {
    for (size_t i = 0; i < nn; ++i)
      if (!std::isfinite(A0[i]) || (E && !std::isfinite(E[i]))) return LYAP_EINVAL;
    LY_TRY(dA.alloc(nn));
    LY_TRY(dU.alloc((size_t)n * k));
    LY_TRY(dV.alloc((size_t)n * k));
    LY_TRY(dG.alloc((size_t)n * g));
    LY_CUDA(cudaMemcpyAsync(dA.p, A0, nn * sizeof(double), cudaMemcpyHostToDevice, st));
    LY_CUDA(cudaMemcpyAsync(dU.p, U, (size_t)n * k * sizeof(double), cudaMemcpyHostToDevice, st));
    LY_CUDA(cudaMemcpyAsync(dV.p, V, (size_t)n * k * sizeof(double), cudaMemcpyHostToDevice, st));
    LY_CUDA(cudaMemcpyAsync(dG.p, G, (size_t)n * g * sizeof(double), cudaMemcpyHostToDevice, st));
    pA = dA.p;
    pU = dU.p;
    pV = dV.p;
    pG = dG.p;
    if (E) {
      LY_TRY(dE.alloc(nn));
      LY_CUDA(cudaMemcpyAsync(dE.p, E, nn * sizeof(double), cudaMemcpyHostToDevice, st));
      pE = dE.p;
    }
  }
  std::unique_ptr<lyap_seed> sd(new lyap_seed());
  sd->ctx = ctx;
  sd->device = ctx->device;
  sd->n = n;
  sd->k = k;
  sd->g = g;
  LY_TRY(lyap_seed_build(ctx, sd.get(), pA, pU, pV, pG, pE, st));
  LY_TRY(lyap_seed_finish(sd.get(), o.pbar, true, st));
  if (cond_Q_out) *cond_Q_out = sd->cond_Q;
  *out = sd.release();
  return LYAP_OK;
}

int lyap_seed_finish(lyap_seed* sd, int pbar, bool mixed, cudaStream_t st) {
  if (mixed) LY_TRY(lyap_mixed_prepare(sd, st));
  if (pbar > 0) LY_TRY(lyap_tsvd_prepare(sd, pbar, st));
  sd->work = new SeedWork();
  return LYAP_OK;
}

extern "C" int lyap_seed_stats_get(const lyap_seed* sd, lyap_seed_stats* o) {
  if (!sd || !o) return LYAP_EINVAL;
  o->n = sd->n;
  o->k = sd->k;
  o->g = sd->g;
  o->real_path = sd->real_path;
  o->cond_Q = sd->cond_Q;
  o->f0 = sd->f0;
  o->max_re_lambda = sd->max_re;
  o->min_abs_lambda_sum = sd->min_sum;
  o->resident_bytes = sd->resident_bytes;
  return LYAP_OK;
}

extern "C" int lyap_seed_free(lyap_seed* sd) {
  if (!sd) return LYAP_EINVAL;
  cudaSetDevice(sd->device);
  delete sd->work;
  lyap_mixed_free(sd);
  lyap_prec_tc_free(sd);
  delete sd;
  return LYAP_OK;
}

// ------------------------------------------------------------ online solves
namespace {

struct CallIO {
  int nv = 0;
  int mem = LYAP_MEM_HOST;
  const double* v = nullptr;  // nv x k, host or device (mem)
};

// Host parameters are checked here; device parameters are checked by k_vinv
// in stream order, and the result is read at each chunk's sync.
int load_v(lyap_seed* sd, int nv, const double* v, int mem_kind, CallIO& io) {
  if (nv < 0 || (nv > 0 && !v)) return LYAP_EINVAL;
  if (mem_kind != LYAP_MEM_HOST && mem_kind != LYAP_MEM_DEVICE) return LYAP_EINVAL;
  io.nv = nv;
  io.mem = mem_kind;
  io.v = v;
  if (nv == 0 || mem_kind == LYAP_MEM_DEVICE) return LYAP_OK;
  return lyap_check_v(nv, sd->k, v);
}

// Where a chunk's results go: host arrays, or the caller's device arrays
// (written in stream order). Pointers are already offset to the chunk.
struct ChunkOut {
  int mem = LYAP_MEM_HOST;
  double* f = nullptr;
  double* g = nullptr;
  lyap_result_info* info = nullptr;
};

// Final FP64 report for one chunk: trace, residual, error estimate, and
// (with an adjoint solution Zadj) the gradient and the dual-weighted error
// estimate |<z, r>| / |f|. Device outputs are written on the stream; the
// host waits once for the per-result reports and the parameter check.
int report_chunk(lyap_seed* sd, SeedWork& w, int Bc, const double2* Wp, const double2* Zadj, bool have_resid,
                 cudaStream_t st, const ChunkOut& out) {
  const int n = sd->n, k = sd->k;
  const size_t N = (size_t)n * k;
  if (w.Rres.count < (size_t)Bc * N) LY_TRY(w.Rres.alloc((size_t)Bc * N));
  if (w.tmp.count < (size_t)Bc * N) LY_TRY(w.tmp.alloc((size_t)Bc * N));
  for (DevBuf<double>* r : {&w.red0, &w.red1, &w.red2, &w.red3})
    if (r->count < (size_t)Bc * k) LY_TRY(r->alloc((size_t)Bc * k));
  kry::k_dot_h<double2><<<Bc, kry::NT, 0, st>>>((int)N, Bc, Wp, N, sd->h.p, w.red0.p, nullptr); lyap_count_launch();
  // r = Ph - T(v) W' (unless the caller already holds it in w.Rres)
  if (!have_resid) {
  CapArgs64 a{};
  a.n = n;
  a.k = k;
  a.lam = sd->lam.p;
  a.P1 = sd->Ub.p;
  a.P2 = sd->Vb.p;
  a.Gd = sd->Gd.p;
  a.W = Wp;
  a.ldw = N;
  a.vinv = w.vinv.p;
  a.rhs = sd->Ph.p;
  a.ldr = 0;
  a.out = w.Rres.p;
  a.ldo = N;
  a.mode = CAP_RESID;
  a.nsys = Bc;
  LY_TRY(capmv64_launch(a, st));
  }
  kry::k_norms<double2><<<Bc, kry::NT, 0, st>>>((int)N, Bc, w.Rres.p, N, w.red1.p); lyap_count_launch();
  if (Zadj) {
    k_dot_pair<<<Bc, kry::NT, 0, st>>>((int)N, Bc, w.Rres.p, Zadj, w.red2.p); lyap_count_launch();
    k_grad<<<Bc * k, kry::NT, 0, st>>>(n, k, Bc, Wp, Zadj, w.vinv.p, w.red3.p); lyap_count_launch();
  } else {
    // delta = P^{-1} r (block-Jacobi proxy for T^{-1} r); estimate <h, delta>
    SysOp<double2> op;
    op.sd = sd;
    op.vinv = w.vinv.p;
    if (w.lst.count < (size_t)Bc) LY_TRY(w.lst.alloc(Bc));
    if (w.cnt.count < 1) LY_TRY(w.cnt.alloc(1));
    kry::k_iota<<<grid_of(Bc), 256, 0, st>>>(Bc, w.lst.p, w.cnt.p); lyap_count_launch();
    LY_TRY(op.precond(w.lst.p, w.cnt.p, Bc, w.Rres.p, N, w.tmp.p, N, st));
    kry::k_dot_h<double2><<<Bc, kry::NT, 0, st>>>((int)N, Bc, w.tmp.p, N, sd->h.p, w.red2.p, nullptr); lyap_count_launch();
  }
  if (out.mem == LYAP_MEM_DEVICE) {
    if (out.f) {
      k_trace_out<<<grid_of(Bc), 256, 0, st>>>(Bc, sd->f0, w.red0.p, out.f);
      lyap_count_launch();
    }
    if (out.g && Zadj)
      LY_CUDA(cudaMemcpyAsync(out.g, w.red3.p, sizeof(double) * Bc * k, cudaMemcpyDeviceToDevice, st));
  }
  LY_CUDA(cudaGetLastError());
  std::vector<double> tr(Bc), rn(Bc), ee(Bc), gr((size_t)Bc * k);
  LY_CUDA(cudaMemcpyAsync(tr.data(), w.red0.p, sizeof(double) * Bc, cudaMemcpyDeviceToHost, st));
  LY_CUDA(cudaMemcpyAsync(rn.data(), w.red1.p, sizeof(double) * Bc, cudaMemcpyDeviceToHost, st));
  LY_CUDA(cudaMemcpyAsync(ee.data(), w.red2.p, sizeof(double) * Bc, cudaMemcpyDeviceToHost, st));
  if (Zadj && out.mem == LYAP_MEM_HOST && out.g)
    LY_CUDA(cudaMemcpyAsync(gr.data(), w.red3.p, sizeof(double) * Bc * k, cudaMemcpyDeviceToHost, st));
  LY_CUDA(cudaMemcpyAsync(w.vbad_host, w.vbad.p, sizeof(int), cudaMemcpyDeviceToHost, st));
  LY_CUDA(cudaStreamSynchronize(st));
  if (*w.vbad_host) {
    lyap_set_last_error(std::to_string(*w.vbad_host) + " parameter(s) zero or not finite");
    return LYAP_EINVAL;
  }
  for (int b = 0; b < Bc; ++b) {
    const double f = sd->f0 + tr[b];
    if (out.mem == LYAP_MEM_HOST && out.f) out.f[b] = f;
    if (out.info) {
      out.info[b].rel_resid = sd->ph_norm > 0 ? rn[b] / sd->ph_norm : rn[b];
      out.info[b].err_est = f != 0 ? std::fabs(ee[b]) / std::fabs(f) : std::fabs(ee[b]);
    }
    if (out.mem == LYAP_MEM_HOST && out.g && Zadj)
      for (int i = 0; i < k; ++i) out.g[(size_t)b * k + i] = gr[(size_t)b * k + i];
  }
  return LYAP_OK;
}

// Solve all nv systems (FP64 or mixed), primal (and adjoint when want_grad).
int run_sweep(lyap_seed* sd, const CallIO& io, const lyap_opts& o, cudaStream_t st, double* f_out, double* g_out,
              bool want_grad, double* w_out, lyap_result_info* info) {
  const int n = sd->n, k = sd->k, nv = io.nv;
  const size_t N = (size_t)n * k;
  SolveParams prm;
  LY_TRY(lyap_params_from_opts(o, prm));
  if (o.precision != LYAP_FP64 && o.precision != LYAP_BF16_IR) return LYAP_EINVAL;
  SeedWork& w = *sd->work;
  // Default batch: the whole sweep in lockstep (one recycle chain per call),
  // capped so the Krylov workspaces use at most a quarter of free memory.
  int B = o.batch;
  if (B <= 0) {
    size_t freeb = 0, totalb = 0;
    cudaMemGetInfo(&freeb, &totalb);
    const size_t per_sys = (size_t)(2 * o.m + 2 * o.s + 6) * N * (o.precision == LYAP_FP64 ? 16 : 8) +
                           (size_t)((o.m + o.s + 1) * (o.m + o.s + 1) * 8) * 16;
    const size_t cap = std::max<size_t>(1, (freeb / 4) / std::max<size_t>(per_sys, 1));
    B = (int)std::min<size_t>(std::min<size_t>(4096, cap), (size_t)std::max(nv, 1));
  }
  B = std::min(B, std::max(nv, 1));
  if (w.vinv.count < (size_t)B * k) LY_TRY(w.vinv.alloc((size_t)B * k));
  if (io.mem == LYAP_MEM_HOST && w.vdev.count < (size_t)B * k) LY_TRY(w.vdev.alloc((size_t)B * k));
  if (w.Wp.count < (size_t)B * N) LY_TRY(w.Wp.alloc((size_t)B * N));
  if (want_grad && w.Zadj.count < (size_t)B * N) LY_TRY(w.Zadj.alloc((size_t)B * N));
  if (w.Rres.count < (size_t)B * N) LY_TRY(w.Rres.alloc((size_t)B * N));
  if (w.vbad.count < 1) LY_TRY(w.vbad.alloc(1));
  if (!w.vbad_host) LY_CUDA(cudaHostAlloc(reinterpret_cast<void**>(&w.vbad_host), sizeof(int), cudaHostAllocDefault));
  LY_CUDA(cudaMemsetAsync(w.vbad.p, 0, sizeof(int), st));
  if (o.pbar > 0) LY_TRY(lyap_tsvd_prepare(sd, o.pbar, st));
  std::vector<int> it, stt, ita, sta, rsteps;
  for (int c0 = 0; c0 < nv; c0 += B) {
    const int Bc = std::min(B, nv - c0);
    const double* vsrc = io.v + (size_t)c0 * k;
    if (io.mem == LYAP_MEM_HOST) {
      LY_CUDA(cudaMemcpyAsync(w.vdev.p, vsrc, sizeof(double) * Bc * k, cudaMemcpyHostToDevice, st));
      vsrc = w.vdev.p;
    }
    k_vinv<<<grid_of((size_t)Bc * k), 256, 0, st>>>(Bc * k, vsrc, w.vinv.p, w.vbad.p); lyap_count_launch();
    LY_CUDA(cudaGetLastError());
    bool have_resid = false;
    const WoodState* wood = nullptr;
    if (o.precision == LYAP_FP64 && o.pbar > 0 && sd->tsvd_r > 0) {
      const int r = std::min(o.pbar, sd->tsvd_r);
      if (w.wcinv.count < (size_t)Bc * r * r) LY_TRY(w.wcinv.alloc((size_t)B * r * r));
      if (w.wpart.count < wood_part_count(n, k, Bc, r)) LY_TRY(w.wpart.alloc(wood_part_count(n, k, B, r)));
      w.wood.cinv = w.wcinv.p;
      w.wood.cpart = w.wpart.p;
      LY_TRY(wood_prepare(sd, r, Bc, w.vinv.p, false, w.wood, st));
      wood = &w.wood;
    }
    if (o.precision == LYAP_FP64) {
      SysOp<double2> op;
      op.sd = sd;
      op.vinv = w.vinv.p;
      op.wood = wood;
      LY_TRY(gcrodr_chunk(op, Bc, sd->Ph.p, 0, sd->rec64, prm, w.ws64, it, stt, st));
      LY_CUDA(cudaMemcpyAsync(w.Wp.p, w.ws64.X.p, sizeof(double2) * Bc * N, cudaMemcpyDeviceToDevice, st));
      rsteps.assign(Bc, 0);
      if (want_grad) {
        SysOp<double2> opa;
        opa.sd = sd;
        opa.adjoint = true;
        opa.vinv = w.vinv.p;
        opa.wood = wood;
        LY_TRY(gcrodr_chunk(opa, Bc, sd->h.p, 0, sd->rec64_adj, prm, w.ws64adj, ita, sta, st));
        LY_CUDA(cudaMemcpyAsync(w.Zadj.p, w.ws64adj.X.p, sizeof(double2) * Bc * N, cudaMemcpyDeviceToDevice, st));
        for (int b = 0; b < Bc; ++b) {
          it[b] += ita[b];
          if (stt[b] == LYAP_OK) stt[b] = sta[b];
        }
      }
    } else {
      LY_TRY(lyap_mixed_chunk(sd, Bc, w.vinv.p, o, prm, st, w.ws32, w.ws32adj, w.Wp.p, want_grad ? w.Zadj.p : nullptr,
                              w.Rres.p, it, stt, rsteps));
      have_resid = true;
    }
    ChunkOut out;
    out.mem = io.mem;
    out.f = f_out ? f_out + c0 : nullptr;
    out.g = g_out ? g_out + (size_t)c0 * k : nullptr;
    out.info = info ? info + c0 : nullptr;
    LY_TRY(report_chunk(sd, w, Bc, w.Wp.p, want_grad ? w.Zadj.p : nullptr, have_resid, st, out));
    if (out.info)
      for (int b = 0; b < Bc; ++b) {
        out.info[b].iters = it[b];
        out.info[b].status = stt[b];
        out.info[b].refine_steps = rsteps.empty() ? 0 : rsteps[b];
      }
    if (w_out) {
      double* dst = w_out + (size_t)c0 * N * 2;
      LY_CUDA(cudaMemcpyAsync(dst, w.Wp.p, sizeof(double2) * Bc * N,
                              io.mem == LYAP_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, st));
      // the next chunk overwrites Wp
      if (c0 + Bc < nv || io.mem == LYAP_MEM_HOST) LY_CUDA(cudaStreamSynchronize(st));
    }
  }
  // the call's stream waits for the recycle updates still running on the
  // workspaces' side streams, so that work counted after the call includes them
  if (w.ws64.side) LY_CUDA(cudaStreamWaitEvent(st, w.ws64.side_done, 0));
  if (w.ws64adj.side) LY_CUDA(cudaStreamWaitEvent(st, w.ws64adj.side_done, 0));
  if (w.ws32.side) LY_CUDA(cudaStreamWaitEvent(st, w.ws32.side_done, 0));
  if (w.ws32adj.side) LY_CUDA(cudaStreamWaitEvent(st, w.ws32adj.side_done, 0));
  return LYAP_OK;
}

int entry(lyap_seed* sd, int nv, const double* v, int mem_kind, const lyap_opts* opts, double* trace_out,
          double* grad_out, double* w_out, lyap_result_info* info) {
  if (!sd) return LYAP_EINVAL;
  lyap_opts o;
  lyap_opts_default(&o);
  if (opts) o = *opts;
  (void)cudaGetLastError();  // a stale error of an unrelated earlier call is not this call's
  LY_CUDA(cudaSetDevice(sd->device));
  cudaStream_t st = pick_stream(sd->ctx, o);
  CallIO io;
  LY_TRY(load_v(sd, nv, v, mem_kind, io));
  if (nv == 0) return LYAP_OK;
  if (o.inject & LYAP_INJECT_ALLOC_FAIL) {
    lyap_set_last_error("injected allocation failure");
    return LYAP_ENOMEM;
  }
  return run_sweep(sd, io, o, st, trace_out, grad_out, grad_out != nullptr, w_out, info);
}

}  // namespace

extern "C" int lyap_param_solve(lyap_seed* sd, int nv, const double* v, int mem_kind, const lyap_opts* opts,
                                double* w_out, lyap_result_info* info) {
  return entry(sd, nv, v, mem_kind, opts, nullptr, nullptr, w_out, info);
}

extern "C" int lyap_trace_EX(lyap_seed* sd, int nv, const double* v, int mem_kind, const lyap_opts* opts,
                             double* trace_out, lyap_result_info* info) {
  if (!trace_out && nv > 0) return LYAP_EINVAL;
  return entry(sd, nv, v, mem_kind, opts, trace_out, nullptr, nullptr, info);
}

extern "C" int lyap_grad(lyap_seed* sd, int nv, const double* v, int mem_kind, const lyap_opts* opts,
                         double* trace_out, double* grad_out, lyap_result_info* info) {
  if ((!trace_out || !grad_out) && nv > 0) return LYAP_EINVAL;
  return entry(sd, nv, v, mem_kind, opts, trace_out, grad_out, nullptr, info);
}
