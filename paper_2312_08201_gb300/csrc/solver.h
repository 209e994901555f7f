// Batched recycled Krylov solver (host driver) shared by the FP64 path, the
// mixed-precision inner solves, the adjoint solves and the server.
#pragma once
#include "capmv.cuh"
#include "lyap_internal.h"
#include "precond.cuh"

struct SolveParams {
  double tol = 1e-12;
  int maxit = 300;
  int m = 30;
  int s = 10;
  unsigned inject = 0;
};

// T(v) (or T(v)^T) for a batch of systems, with the block-Jacobi
// preconditioner of eq. (prec). T2 = double2: FP64 kernels; T2 = float2:
// tensor-core inner operator (mixed path).
template <typename T2>
struct SysOp {
  lyap_seed* sd = nullptr;
  bool adjoint = false;
  const double* vinv = nullptr;  // B x k, device
  const WoodState* wood = nullptr;  // truncated-SVD coupling (nullptr: block-Jacobi only)
  int apply(const int* list, const int* count, int B, const T2* In, size_t in_ss, T2* Out, size_t out_ss,
            cudaStream_t st) const;
  int apply_c0(int nvec, const T2* In, T2* Out, cudaStream_t st) const;
  int precond(const int* list, const int* count, int B, const T2* In, size_t in_ss, T2* Out, size_t out_ss,
              cudaStream_t st) const;
};

template <typename T2>
struct KrylovWS {
  int B = 0, N = 0, m = 0, smax = 0;
  size_t wstride = 0;
  DevBuf<T2> V, Z, C, U, X, R;
  DevBuf<double2> H, H0, Bk, g, sn, coefY, coefR, F, UU, work, Pu, Qc, Gs, Rinv, Racc, Rtmp;
  DevBuf<double> cs, beta, tolabs, tmpd;
  DevBuf<int> jstop, flag, iters, lists, counts, ok, hasrec, rflag;
  DevBuf<int> kerr;  // set by a kernel whose bounded wait expired
  // The recycle update of a chunk's last cycle (harmonic Ritz of the last
  // system, hand-over to the Recycle) runs on a side stream, overlapping
  // the caller's next work; the next chunk on this workspace waits for it.
  cudaStream_t side = nullptr;
  cudaEvent_t side_start = nullptr, side_done = nullptr;
  int* rec_ok_host = nullptr;  // pinned
  DevBuf<int> rec_ok_dev;
  DevBuf<double> vinv_last;
  // Early exit from an Arnoldi cycle: each step's active count is written to
  // a ring of mapped pinned slots, with an event per step; the host reads
  // the count of a step POLL_LAG steps back before queueing the next one.
  static constexpr int POLL_LAG = 2;
  static constexpr int POLL_RING = POLL_LAG + 1;
  int* poll_host = nullptr;  // POLL_RING ints, pinned and mapped
  int* poll_dev = nullptr;   // device view of poll_host
  cudaEvent_t poll_ev[POLL_RING] = {};
  int ensure(int B, int N, int m, int s, cudaStream_t st);
  int ensure_side();
  int ensure_poll();
  size_t bytes() const;
  KrylovWS() = default;
  KrylovWS(const KrylovWS&) = delete;
  KrylovWS& operator=(const KrylovWS&) = delete;
  ~KrylovWS();
};

// Solve op(v_b) x_b = rhs_b for the B systems of one chunk, starting from
// x = 0 and the recycle space `rec` (updated on return from the chunk's
// last system). rhs_ss = 0: one right-hand side shared by all systems.
// On return ws.X holds the solutions; iters/status (host, size B) report.
template <typename T2>
int gcrodr_chunk(const SysOp<T2>& op, int B, const T2* rhs, size_t rhs_ss, Recycle<T2>& rec,
                 const SolveParams& prm, KrylovWS<T2>& ws, std::vector<int>& iters, std::vector<int>& status,
                 cudaStream_t st);

int lyap_params_from_opts(const lyap_opts& o, SolveParams& p);
