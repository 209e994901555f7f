// Host driver of the batched recycled Krylov solver (GCRO-DR, paper §2.1).
//
// Per chunk of B systems (consecutive parameter vectors of the sequence):
//  1. Recycle start: the shared space Ut from the previous chunk gives
//     T(v_b) Ut = Ut D(v_b)^{-1} - C0 Ut (C0 Ut is v-independent), a
//     CholQR2 factorisation T(v_b) Ut = C_b R_b, U_b = Ut R_b^{-1}, and the
//     projection x_b = U_b C_b^H r_b, r_b -= C_b C_b^H r_b.
//  2. Cycles of m - s Arnoldi steps with (I - C C^H) T P^{-1} (right block-
//     Jacobi preconditioning, kept in a flexible basis Z = P^{-1} V so the
//     recycle space stays in the solution space), CGS2, Givens least squares.
//  3. After each cycle: x += Z y2 - U (Bk y2), r = V (beta e1 - H y2), and
//     the recycle space is replaced by the s harmonic Ritz vectors of
//     smallest |theta| from the cycle's augmented space (the default of the
//     paper's cited GCRO-DR implementation).
//  4. The chunk's last system's U becomes the next chunk's shared Ut; with
//     B = 1 this is the paper's system-to-system recycling.
#include <algorithm>
#include <cmath>
#include <mutex>
#include <type_traits>

#include "cplx.cuh"
#include "krylov.cuh"
#include "krylov_cl.cuh"
#include "solver.h"
#include "prof.h"

namespace {

template <typename T2>
__global__ void k_bcast(int B, size_t N, const T2* __restrict__ src, size_t src_ss, T2* __restrict__ dst,
                        size_t dst_ss) {
  const int b = blockIdx.y;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < N; e += (size_t)gridDim.x * blockDim.x)
    dst[(size_t)b * dst_ss + e] = src[(size_t)b * src_ss + e];
}

template <typename T2>
__global__ void k_zero(size_t count, T2* __restrict__ p) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < count; e += (size_t)gridDim.x * blockDim.x)
    p[e] = from_d2<T2>(make_double2(0.0, 0.0));
}

__global__ void k_init_sys(int B, const double* __restrict__ norms, double tol, double* __restrict__ tolabs,
                           int* __restrict__ iters, int* __restrict__ flag, int* __restrict__ hasrec, int hr) {
  int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  tolabs[b] = tol * norms[b];
  iters[b] = 0;
  flag[b] = 1;
  hasrec[b] = hr;
}

__global__ void k_add_iters(const int* __restrict__ list, const int* __restrict__ count, const int* __restrict__ jstop,
                            int* __restrict__ iters) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= *count) return;
  int b = list[s];
  iters[b] += jstop[b];
}

// ok[b] == 0 in the first recycle update (no previous space): zero C_b, U_b
template <typename T2>
__global__ void k_zero_failed(size_t N, int s, const int* __restrict__ list, const int* __restrict__ count,
                              const int* __restrict__ ok, T2* __restrict__ C, T2* __restrict__ U, size_t ss) {
  const int slot = blockIdx.y;
  if (slot >= *count) return;
  const int b = list[slot];
  if (ok[b]) return;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < N * s; e += (size_t)gridDim.x * blockDim.x) {
    C[(size_t)b * ss + e] = from_d2<T2>(make_double2(0.0, 0.0));
    U[(size_t)b * ss + e] = from_d2<T2>(make_double2(0.0, 0.0));
  }
}

// The recycle space is updated for systems that run another cycle, and for
// the chunk's last system, whose space seeds the next chunk.
__global__ void k_want_ritz(const int* __restrict__ list, const int* __restrict__ count, const int* __restrict__ flag,
                            const int* __restrict__ jstop, int last, int* __restrict__ want) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= *count) return;
  int b = list[s];
  want[b] = (jstop[b] > 0 && (flag[b] > 0 || b == last)) ? 1 : 0;
}

__global__ void k_mark_rec(const int* __restrict__ list, const int* __restrict__ count, const int* __restrict__ ok,
                           int* __restrict__ hasrec) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= *count) return;
  int b = list[s];
  if (ok[b]) hasrec[b] = 1;
}

// C0 U = U D(v)^{-1} - T(v) U = U D^{-1} - C   (relation T U = C)
template <typename T2>
__global__ void k_c0_from_relation(int n, int k, int s, const T2* __restrict__ U, const T2* __restrict__ C,
                                   const double* __restrict__ vinv_b, T2* __restrict__ C0U) {
  const size_t N = (size_t)n * k;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < N * s; e += (size_t)gridDim.x * blockDim.x) {
    int t = (int)((e % N) / n);
    C0U[e] = from_d2<T2>(csub(cscale(to_d2(U[e]), vinv_b[t]), to_d2(C[e])));
  }
}

// Hand-over of the chunk's recycle space, on the device: when the last
// system holds a recycle space (hasrec), Ut = its U and C0Ut from the
// relation T U = C; *ok tells the host whether it happened.
template <typename T2>
__global__ void k_handover(int n, int k, int s, const int* __restrict__ hasrec, int last, const T2* __restrict__ U,
                           const T2* __restrict__ C, const double* __restrict__ vinv_b, T2* __restrict__ Ut,
                           T2* __restrict__ C0U, int* __restrict__ ok) {
  const bool have = hasrec[last] != 0;
  if (blockIdx.x == 0 && threadIdx.x == 0) *ok = have ? 1 : 0;
  if (!have) return;
  const size_t N = (size_t)n * k;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < N * s; e += (size_t)gridDim.x * blockDim.x) {
    const int t = (int)((e % N) / n);
    const double2 u = to_d2(U[e]);
    Ut[e] = U[e];
    C0U[e] = from_d2<T2>(csub(cscale(u, vinv_b[t]), to_d2(C[e])));
  }
}

inline int gx(size_t N) {
  size_t g = (N + kry::NT - 1) / kry::NT;
  if (g > 64) g = 64;
  return (int)std::max<size_t>(g, 1);
}

template <typename T2>
kry::Seg<T2> seg(T2* base, size_t ss, size_t vs, int count) {
  kry::Seg<T2> s;
  s.base = base;
  s.ss = ss;
  s.vs = vs;
  s.count = count;
  s.cdev = nullptr;
  s.cadd = 0;
  return s;
}
template <typename T2>
kry::Seg<T2> segd(T2* base, size_t ss, size_t vs, const int* cdev, int cadd) {
  kry::Seg<T2> s = seg(base, ss, vs, 0);
  s.cdev = cdev;
  s.cadd = cadd;
  return s;
}
template <typename T2>
kry::Seg2<T2> seg2(kry::Seg<T2> a, kry::Seg<T2> b) {
  kry::Seg2<T2> s;
  s.a = a;
  s.b = b;
  return s;
}

}  // namespace

// ------------------------------------------------------------------ options
int lyap_params_from_opts(const lyap_opts& o, SolveParams& p) {
  if (!(o.tol > 0) || o.maxit < 1 || o.m < 4 || o.m > 60 || o.s < 0 || o.s > 16 || o.s >= o.m - 1)
    return LYAP_EINVAL;
  p.tol = o.tol;
  p.maxit = o.maxit;
  p.m = o.m;
  p.s = o.s;
  p.inject = o.inject;
  return LYAP_OK;
}

// --------------------------------------------------------------- workspace
template <typename T2>
int KrylovWS<T2>::ensure_side() {
  if (side) return LYAP_OK;
  LY_CUDA(cudaStreamCreateWithFlags(&side, cudaStreamNonBlocking));
  LY_CUDA(cudaEventCreateWithFlags(&side_start, cudaEventDisableTiming));
  LY_CUDA(cudaEventCreateWithFlags(&side_done, cudaEventDisableTiming));
  LY_CUDA(cudaHostAlloc(reinterpret_cast<void**>(&rec_ok_host), sizeof(int), cudaHostAllocDefault));
  *rec_ok_host = 0;
  LY_TRY(rec_ok_dev.alloc(1));
  LY_TRY(vinv_last.alloc(8));
  return LYAP_OK;
}

template <typename T2>
int KrylovWS<T2>::ensure_poll() {
  if (poll_host) return LYAP_OK;
  for (int i = 0; i < POLL_RING; ++i) LY_CUDA(cudaEventCreateWithFlags(&poll_ev[i], cudaEventDisableTiming));
  LY_CUDA(cudaHostAlloc(reinterpret_cast<void**>(&poll_host), sizeof(int) * POLL_RING, cudaHostAllocMapped));
  for (int i = 0; i < POLL_RING; ++i) poll_host[i] = 1;
  LY_CUDA(cudaHostGetDevicePointer(reinterpret_cast<void**>(&poll_dev), poll_host, 0));
  return LYAP_OK;
}

template <typename T2>
KrylovWS<T2>::~KrylovWS() {
  if (side) {
    cudaStreamSynchronize(side);
    cudaStreamDestroy(side);
  }
  if (side_start) cudaEventDestroy(side_start);
  if (side_done) cudaEventDestroy(side_done);
  if (rec_ok_host) cudaFreeHost(rec_ok_host);
  for (int i = 0; i < POLL_RING; ++i)
    if (poll_ev[i]) cudaEventDestroy(poll_ev[i]);
  if (poll_host) cudaFreeHost(poll_host);
}

template <typename T2>
int KrylovWS<T2>::ensure(int B_, int N_, int m_, int s_, cudaStream_t st) {
  if (B_ <= B && N_ == N && m_ == m && s_ == smax && V.p) return LYAP_OK;
  B = B_;
  N = N_;
  m = m_;
  smax = std::max(s_, 1);
  const size_t Bs = B, Ns = N;
  const int LD = m + smax + 1;
  wstride = (size_t)5 * LD * LD + (size_t)3 * LD * 16 + 256 + 2 * LD + 16;
  LY_TRY(V.alloc(Bs * (m + 1) * Ns));
  LY_TRY(Z.alloc(Bs * m * Ns));
  LY_TRY(C.alloc(Bs * smax * Ns));
  LY_TRY(U.alloc(Bs * smax * Ns));
  LY_TRY(X.alloc(Bs * Ns));
  LY_TRY(R.alloc(Bs * Ns));
  LY_TRY(H.alloc(Bs * (m + 1) * m));
  LY_TRY(H0.alloc(Bs * (m + 1) * m));
  LY_TRY(Bk.alloc(Bs * smax * m));
  LY_TRY(g.alloc(Bs * (m + 1)));
  LY_TRY(sn.alloc(Bs * m));
  LY_TRY(coefY.alloc(Bs * LD));
  LY_TRY(coefR.alloc(Bs * (m + 1)));
  LY_TRY(F.alloc(Bs * LD * LD));
  LY_TRY(UU.alloc(Bs * smax * smax));
  LY_TRY(work.alloc(Bs * wstride));
  LY_TRY(Pu.alloc(Bs * LD * 16));
  LY_TRY(Qc.alloc(Bs * LD * 16));
  LY_TRY(Gs.alloc(Bs * smax * smax));
  LY_TRY(Rinv.alloc(Bs * smax * smax));
  LY_TRY(Racc.alloc(Bs * smax * smax));
  LY_TRY(Rtmp.alloc(Bs * smax * smax));
  LY_TRY(cs.alloc(Bs * m));
  LY_TRY(beta.alloc(Bs));
  LY_TRY(tolabs.alloc(Bs));
  LY_TRY(tmpd.alloc(Bs));
  LY_TRY(jstop.alloc(Bs));
  LY_TRY(flag.alloc(Bs));
  LY_TRY(iters.alloc(Bs));
  LY_TRY(lists.alloc(Bs * 6));
  LY_TRY(counts.alloc(8));
  LY_TRY(ok.alloc(Bs));
  LY_TRY(hasrec.alloc(Bs));
  LY_TRY(rflag.alloc(Bs));
  LY_TRY(kerr.alloc(1));
  LY_CUDA(cudaMemsetAsync(kerr.p, 0, sizeof(int), st));  // ordered with the solve on st
  return LYAP_OK;
}

template <typename T2>
size_t KrylovWS<T2>::bytes() const {
  return V.bytes() + Z.bytes() + C.bytes() + U.bytes() + X.bytes() + R.bytes() + H.bytes() + H0.bytes() +
         Bk.bytes() + g.bytes() + sn.bytes() + coefY.bytes() + coefR.bytes() + F.bytes() + UU.bytes() +
         work.bytes() + Pu.bytes() + Qc.bytes() + Gs.bytes() + Rinv.bytes() + Racc.bytes() + Rtmp.bytes() +
         cs.bytes() + beta.bytes() + tolabs.bytes() + tmpd.bytes() + jstop.bytes() + flag.bytes() + iters.bytes() +
         lists.bytes() + counts.bytes() + ok.bytes() + hasrec.bytes() + rflag.bytes() + kerr.bytes();
}

// --------------------------------------------------------- orthogonalisation
// Shared memory per CTA of the cluster variant; at most kOrthoSmemCap lets
// two CTAs share an SM. Long vectors (nk of several thousand) use clusters
// of 16 CTAs (a non-portable size) and then up to kOrthoSmemBig per CTA.
constexpr size_t kOrthoSmemCap = 100 * 1024;
constexpr size_t kOrthoSmemBig = 200 * 1024;

namespace {
// Clusters of 16 CTAs need an opt-in per device and kernel.
template <typename T2>
int allow_cluster16() {
  static std::mutex mu;
  static std::vector<int> done;
  int dev = 0;
  LY_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(mu);
  if (std::find(done.begin(), done.end(), dev) != done.end()) return LYAP_OK;
  LY_CUDA(cudaFuncSetAttribute(kry::k_ortho_cl<T2>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
  done.push_back(dev);
  return LYAP_OK;
}
}  // namespace

// CGS2 of Arnoldi step j for the listed systems (at most B). The cluster
// kernel stages each system's basis in shared memory over C CTAs: the
// smallest C of 1, 2, 4, 8 whose slices fit kOrthoSmemCap, else 16 CTAs at
// kOrthoSmemCap, else the smallest C up to 16 at kOrthoSmemBig. When none
// fits, the vectors do not start on 16-byte boundaries (bulk copies need
// them) or the cluster cannot be scheduled, the kernel that streams the
// basis from memory runs instead.
template <typename T2>
int launch_ortho(int N, int j, int m, int s_cur, const int* list, const int* count, int B, T2* V, const T2* C,
                 size_t c_ss, double2* H, double2* Bk, int smax, const kry::LsqArgs& la, int* err, cudaStream_t st) {
  const int nb = s_cur + j + 1;
  constexpr int kAlign = 16 / sizeof(T2);  // elements per 16 bytes
  int cl = 0, L = 0;
  auto slice = [&](int c) { return ((N + c - 1) / c + kAlign - 1) / kAlign * kAlign; };
  if (((size_t)N * sizeof(T2)) % 16 == 0 && nb <= kry::OCL_MAXNB) {
    const int tiers[][2] = {{1, 0}, {2, 0}, {4, 0}, {8, 0}, {16, 0}, {1, 1}, {2, 1}, {4, 1}, {8, 1}, {16, 1}};
    for (const auto& t : tiers) {
      const int c = t[0];
      const size_t cap = t[1] ? kOrthoSmemBig : kOrthoSmemCap;
      if (kry::ortho_cl_smem<T2>(nb, slice(c)) <= cap) {
        cl = c;
        L = slice(c);
        break;
      }
    }
  }
  if (cl > 0) {
    const size_t smem = kry::ortho_cl_smem<T2>(nb, L);
    LY_TRY(lyap_smem_optin(reinterpret_cast<const void*>(kry::k_ortho_cl<T2>), smem > kOrthoSmemCap ? kOrthoSmemBig
                                                                                                    : kOrthoSmemCap));
    if (cl > 8) LY_TRY(allow_cluster16<T2>());
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(B * cl, 1, 1);
    cfg.blockDim = dim3(kry::OCT, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cl;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const cudaError_t e = cudaLaunchKernelEx(&cfg, kry::k_ortho_cl<T2>, N, L, j, m, s_cur, list, count, V, C, c_ss,
                                             H, Bk, smax, la, err);
    if (e == cudaSuccess) {
      lyap_count_launch();
      return LYAP_OK;
    }
    (void)cudaGetLastError();  // a cluster shape the device cannot hold: stream instead
  }
  kry::k_ortho<T2><<<B, kry::OT, 0, st>>>(N, j, m, s_cur, list, count, V, C, c_ss, H, Bk, smax, la);
  lyap_count_launch();
  LY_CUDA(cudaGetLastError());
  return LYAP_OK;
}

// ------------------------------------------------------------------ solver
template <typename T2>
int gcrodr_chunk(const SysOp<T2>& op, int B, const T2* rhs, size_t rhs_ss, Recycle<T2>& rec,
                 const SolveParams& prm, KrylovWS<T2>& ws, std::vector<int>& iters, std::vector<int>& status,
                 cudaStream_t st) {
  const int n = op.sd->n, k = op.sd->k;
  const int N = n * k;
  const int m = prm.m, s = prm.s;
  // the previous chunk's recycle update on this workspace (side stream) must be
  // complete before its buffers are reused; it has normally finished long ago
  if (ws.side) LY_CUDA(cudaEventSynchronize(ws.side_done));
  if (rec.pending) {
    LY_CUDA(cudaEventSynchronize(rec.ready));
    rec.pending = false;
    if (*rec.ok_host) {
      rec.s = rec.pending_s;
      rec.c0_valid = true;
    }
  }
  LY_TRY(ws.ensure(B, N, m, s, st));
  const int smax = ws.smax;
  const int LD = m + smax + 1;
  const size_t NS = (size_t)N;
  int* L = ws.lists.p;
  int* Lstart = L;
  int* La = L + B;
  int* Lb = L + 2 * B;
  int* Lchunk = L + 3 * B;
  int* Lritz = L + 4 * B;
  int* cnt = ws.counts.p;
  int* cstart = cnt + 0;
  int* ca = cnt + 1;
  int* cb = cnt + 2;
  int* cchunk = cnt + 3;
  int* critz = cnt + 4;
  const int g1 = (B + 255) / 256;

  // ---- initial state: x = 0, r = rhs ----------------------------------
  kry::k_iota<<<g1, 256, 0, st>>>(B, Lchunk, cchunk); lyap_count_launch();
  k_zero<T2><<<512, 256, 0, st>>>((size_t)B * NS, ws.X.p); lyap_count_launch();
  k_bcast<T2><<<dim3(gx(NS), B), kry::NT, 0, st>>>(B, NS, rhs, rhs_ss, ws.R.p, NS); lyap_count_launch();
  kry::k_norms<T2><<<B, kry::NT, 0, st>>>(N, B, ws.R.p, NS, ws.tmpd.p); lyap_count_launch();
  const bool have_rec = rec.s == s && s > 0 && rec.Ut.p != nullptr;
  k_init_sys<<<g1, 256, 0, st>>>(B, ws.tmpd.p, prm.tol, ws.tolabs.p, ws.iters.p, ws.flag.p, ws.hasrec.p,
                                 have_rec ? 1 : 0); lyap_count_launch();
  LY_CUDA(cudaGetLastError());

  int s_cur = 0;
  if (have_rec) {
    // T(v_b) Ut via the v-independent C0 Ut
    if (!rec.c0_valid) {
      LY_TRY(rec.C0Ut.alloc((size_t)s * NS));
      LY_TRY(op.apply_c0(s, rec.Ut.p, rec.C0Ut.p, st));
      rec.c0_valid = true;
    }
    const size_t ss = (size_t)smax * NS;
    bool fused = false;
    if constexpr (std::is_same<T2, float2>::value) {
      // FP32 solves: the whole recycle start in one kernel while C_b fits in shared memory
      const size_t rsm = kry::recstart32_smem_bytes(s, N);
      if (rsm <= 200 * 1024) {
        LY_TRY(lyap_smem_optin(reinterpret_cast<const void*>(kry::k_recstart32), 200 * 1024));
        const int ph_ = prof_begin(PK_RECSTART, st);
        kry::k_recstart32<<<B, kry::RS_T, rsm, st>>>(n, k, s, Lchunk, cchunk, rec.Ut.p, rec.C0Ut.p, op.vinv, ws.C.p,
                                                     ws.U.p, ss, ws.X.p, ws.R.p, ws.ok.p);
        lyap_count_launch();
        prof_end(ph_, st, 0.0, (4.0 * s + 4.0) * N * sizeof(T2), 0, cchunk);
        LY_CUDA(cudaGetLastError());
        fused = true;
      }
    }
    if (!fused) {
    kry::k_make_AU<T2><<<dim3(gx(NS * s), B), kry::NT, 0, st>>>(n, k, s, Lchunk, cchunk, rec.Ut.p, rec.C0Ut.p,
                                                                 op.vinv, ws.C.p, ss); lyap_count_launch();
    // CholQR2: C = AU R^{-1}, U = Ut R^{-1}
    for (int pass = 0; pass < 2; ++pass) {
      auto cseg = seg2(seg(ws.C.p, ss, NS, s), seg(ws.C.p, ss, NS, 0));
      LY_TRY(kry::launch_gram<T2>(N, Lchunk, cchunk, B, B, cseg, cseg, ws.Gs.p, s, (size_t)smax * smax, st));
      kry::k_chol_rinv<<<(B * 32 + 255) / 256, 256, 0, st>>>(s, Lchunk, cchunk, ws.Gs.p, (size_t)smax * smax,
                                                             ws.Rinv.p, ws.Racc.p, ws.Rtmp.p, pass, ws.ok.p); lyap_count_launch();
      if (pass == 0) {
        // Racc = Rinv
        LY_CUDA(cudaMemcpyAsync(ws.Racc.p, ws.Rinv.p, sizeof(double2) * (size_t)B * s * s,
                                cudaMemcpyDeviceToDevice, st));
      }
      // C := C Rinv (in place: each element column-set is read before written)
      kry::k_tsmm<T2, T2><<<dim3(gx(NS), B), kry::NT, 0, st>>>(N, Lchunk, cchunk, cseg, ws.Rinv.p, s,
                                                               (size_t)s * s, s, ws.C.p, ss, NS, 0); lyap_count_launch();
    }
    // U = Ut Racc (shared input: system stride 0)
    auto useg = seg2(seg(rec.Ut.p, 0, NS, s), seg(rec.Ut.p, 0, NS, 0));
    kry::k_tsmm<T2, T2><<<dim3(gx(NS), B), kry::NT, 0, st>>>(N, Lchunk, cchunk, useg, ws.Racc.p, s,
                                                             (size_t)s * s, s, ws.U.p, ss, NS, 0); lyap_count_launch();
    LY_CUDA(cudaGetLastError());
    }
    std::vector<int> okh(B);
    LY_CUDA(cudaMemcpyAsync(okh.data(), ws.ok.p, sizeof(int) * B, cudaMemcpyDeviceToHost, st));
    LY_CUDA(cudaStreamSynchronize(st));
    bool all_ok = std::all_of(okh.begin(), okh.end(), [](int v) { return v == 1; });
    if (all_ok) {
      if (!fused) {  // the fused kernel has applied the projection already
        const int ph_ = prof_begin(PK_RECSTART, st);
        kry::k_project<T2><<<B, kry::NT, 0, st>>>(N, s, Lchunk, cchunk, ws.C.p, ws.U.p, ss, ws.X.p, ws.R.p); lyap_count_launch();
        prof_end(ph_, st, 0.0, 0.0, 0, nullptr);
      }
      LY_CUDA(cudaGetLastError());
      s_cur = s;
    } else {
      k_init_sys<<<g1, 256, 0, st>>>(B, ws.tmpd.p, prm.tol, ws.tolabs.p, ws.iters.p, ws.flag.p, ws.hasrec.p, 0); lyap_count_launch();
      rec.c0_valid = false;
    }
  }

  const int maxit = (prm.inject & LYAP_INJECT_FORCE_MAXIT) ? 1 : prm.maxit;
  LY_TRY(ws.ensure_poll());
  const size_t css = (size_t)smax * NS;
  int chunk_count = B;
  int guard = 0;
  bool last_async = false;  // the last cycle's recycle update runs on ws.side
  while (chunk_count > 0 && guard++ < 100000) {
    LY_CUDA(cudaMemcpyAsync(Lstart, Lchunk, sizeof(int) * B, cudaMemcpyDeviceToDevice, st));
    LY_CUDA(cudaMemcpyAsync(cstart, cchunk, sizeof(int), cudaMemcpyDeviceToDevice, st));
    {
      const int ph_ = prof_begin(PK_CYCLE, st);
      kry::k_cycle_start<T2><<<B, kry::NT, 0, st>>>(N, m, Lstart, cstart, ws.R.p, ws.V.p, ws.g.p, ws.tolabs.p,
                                                  ws.flag.p, ws.jstop.p, ws.beta.p); lyap_count_launch();
      prof_end(ph_, st, 0.0, 0.0, 0, nullptr);
    }
    kry::k_compact<<<1, 1024, 0, st>>>(Lstart, cstart, ws.flag.p, La, ca); lyap_count_launch();
    LY_CUDA(cudaGetLastError());
    int* Lcur = La;
    int* ccur = ca;
    int* Lnext = Lb;
    int* cnext = cb;
    const int mc = m - s_cur;
    constexpr int LAG = KrylovWS<T2>::POLL_LAG, RING = KrylovWS<T2>::POLL_RING;
    for (int j = 0; j < mc; ++j) {
      if (j >= LAG) {
        // once every system of the chunk has stopped, the cycle's remaining
        // steps would launch on empty lists: stop queueing them
        const int q = (j - LAG) % RING;
        LY_CUDA(cudaEventSynchronize(ws.poll_ev[q]));
        if (*static_cast<volatile int*>(ws.poll_host + q) == 0) break;
      }
      T2* Vj = ws.V.p;  // slot j of each system: V + b*(m+1)*N + j*N
      T2* Zj = ws.Z.p;
      LY_TRY(op.precond(Lcur, ccur, B, Vj + (size_t)j * NS, (size_t)(m + 1) * NS, Zj + (size_t)j * NS,
                        (size_t)m * NS, st));
      LY_TRY(op.apply(Lcur, ccur, B, Zj + (size_t)j * NS, (size_t)m * NS, Vj + (size_t)(j + 1) * NS,
                      (size_t)(m + 1) * NS, st));
      {
        // CGS2's algorithmic traffic: one read of the nb basis vectors, w read
        // and written once (the kernel itself rereads the basis from L2)
        const int nb = s_cur + j + 1;
        const int ph = prof_begin(PK_ORTHO, st);
        // the same kernel applies the Givens least-squares update to the new column
        const kry::LsqArgs la{ws.H0.p, ws.cs.p, ws.sn.p, ws.g.p, ws.tolabs.p, ws.jstop.p, ws.flag.p, ws.iters.p,
                              maxit};
        LY_TRY(launch_ortho<T2>(N, j, m, s_cur, Lcur, ccur, B, ws.V.p, ws.C.p, css, ws.H.p, ws.Bk.p, smax, la,
                                ws.kerr.p, st));
        prof_end(ph, st, 2.0 * 2.0 * 8.0 * nb * N, (nb + 2.0) * N * sizeof(T2), 0, ccur);
      }
      kry::k_compact<<<1, 1024, 0, st>>>(Lcur, ccur, ws.flag.p, Lnext, cnext, ws.poll_dev + j % RING);
      lyap_count_launch();
      LY_CUDA(cudaGetLastError());
      LY_CUDA(cudaEventRecord(ws.poll_ev[j % RING], st));
      std::swap(Lcur, Lnext);
      std::swap(ccur, cnext);
    }
    // ---- cycle end -----------------------------------------------------
    {
      const int ph_ = prof_begin(PK_CYCLE, st);
      // one warp per system
      kry::k_cycle_solve<<<(B + kry::CS_WARPS - 1) / kry::CS_WARPS, 32 * kry::CS_WARPS, 0, st>>>(m, smax, s_cur, Lstart, cstart, ws.H.p, ws.H0.p, ws.Bk.p, ws.g.p,
                                           ws.beta.p, ws.jstop.p, ws.coefY.p, ws.coefR.p); lyap_count_launch();
      prof_end(ph_, st, 0.0, 0.0, 0, nullptr);
    }
    {
      const int ph_ = prof_begin(PK_CYCLE, st);
      kry::k_update_xr<T2><<<dim3(gx(NS), B), kry::NT, 0, st>>>(N, m, smax, s_cur, Lstart, cstart, ws.jstop.p,
                                                              ws.coefY.p, ws.coefR.p, ws.U.p, ws.Z.p, ws.V.p,
                                                              ws.X.p, ws.R.p); lyap_count_launch();
      prof_end(ph_, st, 0.0, 0.0, 0, nullptr);
    }
    k_add_iters<<<g1, 256, 0, st>>>(Lstart, cstart, ws.jstop.p, ws.iters.p); lyap_count_launch();
    LY_CUDA(cudaGetLastError());
    // ---- next cycle: systems still running (flag > 0). The count is read
    // here, before the recycle update, so that the update's launches are
    // sized by it: at most chunk_count + 1 systems (the continuing ones and
    // the chunk's last system) need harmonic-Ritz vectors.
    kry::k_compact<<<1, 1024, 0, st>>>(Lstart, cstart, ws.flag.p, Lchunk, cchunk); lyap_count_launch();
    LY_CUDA(cudaGetLastError());
    LY_CUDA(cudaMemcpyAsync(&chunk_count, cchunk, sizeof(int), cudaMemcpyDeviceToHost, st));
    int kerr_h = 0;
    LY_CUDA(cudaMemcpyAsync(&kerr_h, ws.kerr.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    LY_CUDA(cudaStreamSynchronize(st));
    if (kerr_h) {
      LY_CUDA(cudaMemsetAsync(ws.kerr.p, 0, sizeof(int), st));
      lyap_set_last_error("orthogonalisation copy wait timed out (code " + std::to_string(kerr_h) + ")");
      return LYAP_EDEVICE_TIMEOUT;
    }
    const int Bw = std::min(B, chunk_count + 1);
    // ---- recycle update (harmonic Ritz) ----------------------------------
    // After the chunk's last cycle only the last system is updated, and only
    // the next chunk uses the result: run it on the side stream.
    const bool async_update = s > 0 && chunk_count == 0;
    last_async = async_update;
    cudaStream_t us = st;
    if (async_update) {
      LY_TRY(ws.ensure_side());
      LY_CUDA(cudaMemcpyAsync(ws.vinv_last.p, op.vinv + (size_t)(B - 1) * k, sizeof(double) * k,
                              cudaMemcpyDeviceToDevice, st));
      LY_CUDA(cudaEventRecord(ws.side_start, st));
      LY_CUDA(cudaStreamWaitEvent(ws.side, ws.side_start, 0));
      us = ws.side;
    }
    if (s > 0) {
      auto Vh = seg2(seg(ws.C.p, css, NS, s_cur), segd(ws.V.p, (size_t)(m + 1) * NS, NS, ws.jstop.p, 1));
      auto Wh = seg2(seg(ws.U.p, css, NS, s_cur), segd(ws.Z.p, (size_t)m * NS, NS, ws.jstop.p, 0));
      int* Lwant = L + 5 * B;
      int* cwant = cnt + 5;
      k_want_ritz<<<g1, 256, 0, us>>>(Lstart, cstart, ws.flag.p, ws.jstop.p, B - 1, ws.rflag.p);
      lyap_count_launch();
      kry::k_compact<<<1, 1024, 0, us>>>(Lstart, cstart, ws.rflag.p, Lwant, cwant);
      lyap_count_launch();
      {
        const int ph_ = prof_begin(PK_GRAM, us);
        LY_TRY(kry::launch_gram<T2>(N, Lwant, cwant, Bw, Bw, Vh, Wh, ws.F.p, LD, (size_t)LD * LD, us));
        prof_end(ph_, us, 0.0, 0.0, 0, nullptr);
      }
      if (s_cur > 0) {
        auto Us = seg2(seg(ws.U.p, css, NS, s_cur), seg(ws.U.p, css, NS, 0));
        LY_TRY(kry::launch_gram<T2>(N, Lwant, cwant, Bw, Bw, Us, Us, ws.UU.p, smax, (size_t)smax * smax, us));
      }
      {
        const int ph_ = prof_begin(PK_RITZ, us);
        const size_t rsm = kry::ritz_smem_bytes(m, smax);
      if (rsm > 48 * 1024) {
        // the largest size any call needs (m <= 60, s <= 16)
        LY_TRY(lyap_smem_optin(reinterpret_cast<const void*>(kry::k_ritz), kry::ritz_smem_bytes(60, 16)));
      }
      kry::k_ritz<<<Bw, 32, rsm, us>>>(m, smax, s_cur, s, Lwant, cwant, ws.jstop.p, ws.H0.p,
                                                        ws.Bk.p, ws.F.p, ws.UU.p, ws.work.p, ws.wstride, ws.Pu.p,
                                                        ws.Qc.p, ws.ok.p); lyap_count_launch();
        prof_end(ph_, us, 0.0, 0.0, 0, nullptr);
      }
      // systems whose update succeeded: new U = [U Z] Pu, C = [C V] Qc (in place)
      {
        // list of systems with ok = 1 (flag-like compaction on ok)
        kry::k_compact<<<1, 1024, 0, us>>>(Lwant, cwant, ws.ok.p, Lritz, critz); lyap_count_launch();
        {
          const int ph_ = prof_begin(PK_TSMM, us);
          kry::k_tsmm<T2, T2><<<dim3(gx(NS), Bw), kry::NT, 0, us>>>(N, Lritz, critz, Wh, ws.Pu.p, LD,
                                                                 (size_t)LD * 16, s, ws.U.p, css, NS, 0); lyap_count_launch();
          prof_end(ph_, us, 0.0, 0.0, 0, nullptr);
        }
        {
          const int ph_ = prof_begin(PK_TSMM, us);
          kry::k_tsmm<T2, T2><<<dim3(gx(NS), Bw), kry::NT, 0, us>>>(N, Lritz, critz, Vh, ws.Qc.p, LD,
                                                                 (size_t)LD * 16, s, ws.C.p, css, NS, 0); lyap_count_launch();
          prof_end(ph_, us, 0.0, 0.0, 0, nullptr);
        }
        k_mark_rec<<<g1, 256, 0, us>>>(Lwant, cwant, ws.ok.p, ws.hasrec.p); lyap_count_launch();
        if (s_cur == 0) {
          k_zero_failed<T2><<<dim3(gx(NS * s), Bw), kry::NT, 0, us>>>(NS, s, Lwant, cwant, ws.ok.p, ws.C.p,
                                                                     ws.U.p, css);
          lyap_count_launch();
        }
        LY_CUDA(cudaGetLastError());
      }
      s_cur = s;
    }
  }

  // ---- report and hand the recycle space to the next chunk ----------------
  iters.assign(B, 0);
  status.assign(B, 0);
  std::vector<int> fl(B), hr(B);
  LY_CUDA(cudaMemcpyAsync(iters.data(), ws.iters.p, sizeof(int) * B, cudaMemcpyDeviceToHost, st));
  LY_CUDA(cudaMemcpyAsync(fl.data(), ws.flag.p, sizeof(int) * B, cudaMemcpyDeviceToHost, st));
  if (!last_async) LY_CUDA(cudaMemcpyAsync(hr.data(), ws.hasrec.p, sizeof(int) * B, cudaMemcpyDeviceToHost, st));
  LY_CUDA(cudaStreamSynchronize(st));
  for (int b = 0; b < B; ++b) {
    int f = fl[b];
    int code = f < 0 ? -f : 2;
    status[b] = code == 1 ? LYAP_OK
                : code == 2 ? LYAP_ENOCONV
                : code == 3 ? LYAP_EBREAKDOWN
                            : LYAP_ENONFINITE;
  }
  if (last_async) {
    // hand-over on the side stream, resolved by the next chunk on this workspace
    if (rec.Ut.count < (size_t)s * NS) LY_TRY(rec.Ut.alloc((size_t)s * NS));
    if (rec.C0Ut.count < (size_t)s * NS) LY_TRY(rec.C0Ut.alloc((size_t)s * NS));
    const size_t off = (size_t)(B - 1) * css;
    k_handover<T2><<<gx(NS * s), kry::NT, 0, ws.side>>>(n, k, s, ws.hasrec.p, B - 1, ws.U.p + off, ws.C.p + off,
                                                         ws.vinv_last.p, rec.Ut.p, rec.C0Ut.p, ws.rec_ok_dev.p);
    lyap_count_launch();
    LY_CUDA(cudaGetLastError());
    LY_CUDA(cudaMemcpyAsync(ws.rec_ok_host, ws.rec_ok_dev.p, sizeof(int), cudaMemcpyDeviceToHost, ws.side));
    LY_CUDA(cudaEventRecord(ws.side_done, ws.side));
    rec.pending = true;
    rec.pending_s = s;
    rec.ready = ws.side_done;
    rec.ok_host = ws.rec_ok_host;
    return LYAP_OK;
  }
  if (s > 0 && hr[B - 1]) {
    LY_TRY(rec.Ut.alloc((size_t)s * NS));
    LY_TRY(rec.C0Ut.alloc((size_t)s * NS));
    const size_t off = (size_t)(B - 1) * css;
    LY_CUDA(cudaMemcpyAsync(rec.Ut.p, ws.U.p + off, sizeof(T2) * s * NS, cudaMemcpyDeviceToDevice, st));
    k_c0_from_relation<T2><<<gx(NS * s), kry::NT, 0, st>>>(n, k, s, ws.U.p + off, ws.C.p + off,
                                                            op.vinv + (size_t)(B - 1) * k, rec.C0Ut.p); lyap_count_launch();
    LY_CUDA(cudaGetLastError());
    rec.s = s;
    rec.c0_valid = true;
  }
  return LYAP_OK;
}

namespace kry {
template <typename T2>
int launch_gram(int N, const int* list, const int* count, int B, int expect, const Seg2<T2>& A, const Seg2<T2>& Bm,
                double2* out, int ldo, size_t os, cudaStream_t st) {
  LY_TRY(lyap_smem_optin(reinterpret_cast<const void*>(k_gram<T2>), gram_smem_bytes<T2>()));
  // split each system over a cluster of CTAs only while the systems alone leave SMs idle
  const int split = expect * 4 <= 152 ? GSPLIT : 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(B, split, 1);
  cfg.blockDim = dim3(GT, 1, 1);
  cfg.dynamicSmemBytes = gram_smem_bytes<T2>();
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 1;
  attr[0].val.clusterDim.y = split;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  LY_CUDA(cudaLaunchKernelEx(&cfg, k_gram<T2>, N, list, count, A, Bm, out, ldo, os));
  lyap_count_launch();
  return LYAP_OK;
}
}  // namespace kry

template struct KrylovWS<double2>;
template struct KrylovWS<float2>;
template int gcrodr_chunk<double2>(const SysOp<double2>&, int, const double2*, size_t, Recycle<double2>&,
                                   const SolveParams&, KrylovWS<double2>&, std::vector<int>&, std::vector<int>&,
                                   cudaStream_t);
template int gcrodr_chunk<float2>(const SysOp<float2>&, int, const float2*, size_t, Recycle<float2>&,
                                  const SolveParams&, KrylovWS<float2>&, std::vector<int>&, std::vector<int>&,
                                  cudaStream_t);

// --------------------------------------------------- FP64 operator (SysOp)
template <>
int SysOp<double2>::apply(const int* list, const int* count, int B, const double2* In, size_t in_ss, double2* Out,
                          size_t out_ss, cudaStream_t st) const {
  CapArgs64 a{};
  a.n = sd->n;
  a.k = sd->k;
  a.lam = sd->lam.p;
  a.P1 = adjoint ? sd->Vb.p : sd->Ub.p;
  a.P2 = adjoint ? sd->Ub.p : sd->Vb.p;
  a.Gd = sd->Gd.p;
  a.gT = adjoint ? 1 : 0;
  a.W = In;
  a.ldw = in_ss;
  a.vinv = vinv;
  a.out = Out;
  a.ldo = out_ss;
  a.mode = CAP_T;
  a.list = list;
  a.count = count;
  a.nsys = B;
  return capmv64_launch(a, st);
}

template <>
int SysOp<double2>::apply_c0(int nvec, const double2* In, double2* Out, cudaStream_t st) const {
  CapArgs64 a{};
  a.n = sd->n;
  a.k = sd->k;
  a.lam = sd->lam.p;
  a.P1 = adjoint ? sd->Vb.p : sd->Ub.p;
  a.P2 = adjoint ? sd->Ub.p : sd->Vb.p;
  a.Gd = sd->Gd.p;
  a.gT = adjoint ? 1 : 0;
  a.W = In;
  a.ldw = (size_t)sd->n * sd->k;
  a.out = Out;
  a.ldo = (size_t)sd->n * sd->k;
  a.mode = CAP_C0;
  a.nsys = nvec;
  return capmv64_launch(a, st);
}

template <>
int SysOp<double2>::precond(const int* list, const int* count, int B, const double2* In, size_t in_ss,
                            double2* Out, size_t out_ss, cudaStream_t st) const {
  return prec_apply<double2>(sd, wood, adjoint, vinv, list, count, B, In, in_ss, Out, out_ss, st);
}
