// Batched kernels of the recycled Krylov solver (GCRO-DR, paper §2.1; the
// method is cited there from Parks et al. and restated in the design notes).
//
// B systems run in lockstep; each has its own Arnoldi basis, recycle space
// and small projected matrices. A device-side list of active systems lets
// converged systems drop out mid-cycle without a host round trip. Vector
// storage is complex (T2 = double2 for the FP64 path, float2 for the inner
// solves of the mixed path); every reduction and every small projected
// matrix is FP64 and summed in a fixed order, so results do not depend on
// which other systems share the batch.
#pragma once
#include <cooperative_groups.h>

#include "cplx.cuh"
#include "smalldense.cuh"

namespace kry {

constexpr int NT = 256;  // threads per CTA for vector kernels

// Sum NV doubles over the CTA (fixed shuffle tree, fixed cross-warp order).
template <int NV, typename R = double>
__device__ __forceinline__ void block_sum(R (&v)[NV], R* red /* NV*32 */) {
#pragma unroll
  for (int i = 0; i < NV; ++i)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[i] += __shfl_xor_sync(0xffffffffu, v[i], o);
  const int warp = threadIdx.x >> 5, ln = threadIdx.x & 31, nw = blockDim.x >> 5;
  __syncthreads();
  if (ln == 0)
#pragma unroll
    for (int i = 0; i < NV; ++i) red[i * 32 + warp] = v[i];
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int i = 0; i < NV; ++i) {
      R x = ln < nw ? red[i * 32 + ln] : R(0);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
      if (ln == 0) red[i * 32] = x;
    }
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < NV; ++i) v[i] = red[i * 32];
  __syncthreads();
}

// A strided family of vectors: vector i of system b at base + b*ss + i*vs.
template <typename T2>
struct Seg {
  T2* base;
  size_t ss, vs;
  int count;        // fixed count, or
  const int* cdev;  // per-system count (cdev[b] + cadd) when non-null
  int cadd;
  __device__ __forceinline__ int cnt(int b) const { return cdev ? cdev[b] + cadd : count; }
  __device__ __forceinline__ T2* vec(int b, int i) const { return base + (size_t)b * ss + (size_t)i * vs; }
};

// Two concatenated segments [S0 S1].
template <typename T2>
struct Seg2 {
  Seg<T2> a, b;
  __device__ __forceinline__ int cnt(int s) const { return a.cnt(s) + b.cnt(s); }
  __device__ __forceinline__ T2* vec(int s, int i) const {
    int na = a.cnt(s);
    return i < na ? a.vec(s, i) : b.vec(s, i - na);
  }
};

// ----------------------------------------------------------------- lists
// Rebuild an ordered list of systems: out = [b in in_list : flag[b] > 0].
// host_count (optional, mapped pinned memory) receives a copy of the count
// that the host may read once the kernel has completed.
__global__ void k_compact(const int* __restrict__ in_list, const int* __restrict__ in_count,
                          const int* __restrict__ flag, int* __restrict__ out_list, int* __restrict__ out_count,
                          int* host_count = nullptr);
__global__ void k_iota(int B, int* list, int* count);

// ------------------------------------------------------ Givens least squares
// status codes kept per system
enum { ST_RUN = 0, ST_CONV = 1, ST_MAXIT = 2, ST_BREAK = 3, ST_NONFINITE = 4 };

struct LsqArgs {
  double2* H0;
  double* cs;
  double2* sn;
  double2* g;
  const double* tolabs;
  int* jstop;
  int* flag;
  const int* iters_done;
  int maxit;
};

// Column j of H (rows 0..j+1) is copied to H0 (unrotated, for the residual
// and the harmonic-Ritz problem), rotated by the previous rotations, and a
// new rotation zeroes H[j+1, j]. |g[j+1]| is the residual norm of the
// projected problem; when it reaches tolabs, or H[j+1, j] vanishes
// (breakdown: exact solution in the space), the system stops this cycle.
// Run by one thread per system, right after the column is complete: the
// column (h, j + 2 entries) and the previous rotations (cs_s, sn_s) are in
// shared memory, and gj = g[j], tolabs, iterations done were loaded before
// the column was; only stores go to global memory.
//
// R is the arithmetic of the rotations: the precision of the Krylov vectors.
// With FP32 vectors the column's entries carry FP32 inner products, and a
// serial chain of FP64 operations on one thread (GB300's FP64 rate is 1/64
// of its FP32 rate) would cost more than the rest of the Arnoldi step;
// storage stays FP64 either way.
template <typename R>
__device__ __forceinline__ void lsq_column(int b, int j, int m, double2* __restrict__ H, const double2* h,
                                           const double* cs_s, const double2* sn_s, double2 gj, double tola,
                                           int iters_done, const LsqArgs& L) {
  using C = typename Cplx<R>::T;
  const auto in = [](double2 x) -> C { return C{(R)x.x, (R)x.y}; };
  const auto out = [](C x) -> double2 { return make_double2((double)x.x, (double)x.y); };
  double2* hg = H + (size_t)b * (m + 1) * m + (size_t)j * (m + 1);
  C top = in(h[0]);
  for (int i = 0; i < j; ++i) {
    const C bot = in(h[i + 1]);
    const R ci = (R)cs_s[i];
    const C si = in(sn_s[i]);
    hg[i] = out(cadd(cscale(top, ci), cmul(si, bot)));
    top = csub(cscale(bot, ci), cjmul(si, top));
  }
  const C low = in(h[j + 1]);
  R cj;
  C sj;
  {  // rotation zeroing low under top, scaled so that no square overflows
    const R ax = sqrt(cabs2(top)), ay = sqrt(cabs2(low));
    if (ay == R(0)) {
      cj = R(1);
      sj = C{R(0), R(0)};
    } else if (ax == R(0)) {
      cj = R(0);
      sj = C{R(1), R(0)};
    } else {
      const R mx = ax > ay ? ax : ay;
      const R r = mx * sqrt((ax / mx) * (ax / mx) + (ay / mx) * (ay / mx));
      cj = ax / r;
      sj = cscale(cjmul(low, cscale(top, R(1) / ax)), R(1) / r);  // (top / |top|) conj(low) / r
    }
  }
  const C rho = cadd(cscale(top, cj), cmul(sj, low));
  const double sub = (double)low.x;
  hg[j] = out(rho);
  hg[j + 1] = make_double2(0.0, 0.0);
  L.cs[(size_t)b * m + j] = (double)cj;
  L.sn[(size_t)b * m + j] = out(sj);
  double2* gb = L.g + (size_t)b * (m + 1);
  const C gjc = in(gj);
  gb[j] = out(cscale(gjc, cj));
  const C gn = cscale(cjmul(sj, gjc), R(-1));
  gb[j + 1] = out(gn);
  const double res = sqrt(cabs2(out(gn)));
  const double2 rhod = out(rho);
  int st = ST_RUN;
  if (!isfinite(res) || !isfinite(rhod.x) || !isfinite(rhod.y)) st = ST_NONFINITE;
  else if (res <= tola) st = ST_CONV;
  else if (!(sub > 1e-14 * sqrt(cabs2(rhod)))) st = ST_CONV;  // invariant subspace: exact in the space
  else if (iters_done + j + 1 >= L.maxit) st = ST_MAXIT;
  L.jstop[b] = j + 1;  // provisional when still running (the cycle may end here)
  if (st != ST_RUN) L.flag[b] = -st;  // negative: stopped this cycle with a final status
}

// The serial part of lsq_column on copies in shared memory, for a caller
// that converts in parallel: hr[0..j+1] holds the column in the precision R
// and is rotated in place (hr[0..j] the rotated column, hr[j+1] = 0), csr and
// snr the previous rotations. Only the rotation's own results (cs, sn, g,
// jstop, flag) go to global memory here; the caller stores hr into H.
template <typename R>
__device__ __forceinline__ void lsq_rotate(int b, int j, int m, typename Cplx<R>::T* hr, const R* csr,
                                           const typename Cplx<R>::T* snr, double2 gj, double tola,
                                           int iters_done, const LsqArgs& L) {
  using C = typename Cplx<R>::T;
  C top = hr[0];
  for (int i = 0; i < j; ++i) {
    const C bot = hr[i + 1];
    const R ci = csr[i];
    const C si = snr[i];
    hr[i] = cadd(cscale(top, ci), cmul(si, bot));
    top = csub(cscale(bot, ci), cjmul(si, top));
  }
  const C low = hr[j + 1];
  R cj;
  C sj;
  {  // rotation zeroing low under top, scaled so that no square overflows
    const R ax = sqrt(cabs2(top)), ay = sqrt(cabs2(low));
    if (ay == R(0)) {
      cj = R(1);
      sj = C{R(0), R(0)};
    } else if (ax == R(0)) {
      cj = R(0);
      sj = C{R(1), R(0)};
    } else {
      const R mx = ax > ay ? ax : ay;
      const R r = mx * sqrt((ax / mx) * (ax / mx) + (ay / mx) * (ay / mx));
      cj = ax / r;
      sj = cscale(cjmul(low, cscale(top, R(1) / ax)), R(1) / r);  // (top / |top|) conj(low) / r
    }
  }
  const C rho = cadd(cscale(top, cj), cmul(sj, low));
  hr[j] = rho;
  hr[j + 1] = C{R(0), R(0)};
  const C gjc = C{(R)gj.x, (R)gj.y};
  const C gn = cscale(cjmul(sj, gjc), R(-1));
  const C g0 = cscale(gjc, cj);
  L.cs[(size_t)b * m + j] = (double)cj;
  L.sn[(size_t)b * m + j] = make_double2((double)sj.x, (double)sj.y);
  double2* gb = L.g + (size_t)b * (m + 1);
  gb[j] = make_double2((double)g0.x, (double)g0.y);
  gb[j + 1] = make_double2((double)gn.x, (double)gn.y);
  const R res = sqrt(cabs2(gn));
  const R rr = sqrt(cabs2(rho));
  int st = ST_RUN;
  if (!isfinite(res) || !isfinite(rho.x) || !isfinite(rho.y)) st = ST_NONFINITE;
  else if ((double)res <= tola) st = ST_CONV;
  else if (!((double)low.x > 1e-14 * (double)rr)) st = ST_CONV;  // invariant subspace: exact in the space
  else if (iters_done + j + 1 >= L.maxit) st = ST_MAXIT;
  L.jstop[b] = j + 1;  // provisional when still running (the cycle may end here)
  if (st != ST_RUN) L.flag[b] = -st;  // negative: stopped this cycle with a final status
}

// ----------------------------------------------------------- CGS2 Arnoldi
// Sum 32 per-thread values over a warp: after the call lane l holds, in
// v[0], the warp total of value l (a butterfly that halves the values per
// lane at every step: 31 shuffles instead of 32 x 5).
template <typename R>
__device__ __forceinline__ void warp_reduce_scatter32(R (&v)[32]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int s = 16; s >= 1; s >>= 1) {
    const bool upper = (lane & s) != 0;
#pragma unroll
    for (int i = 0; i < s; ++i) {
      const R send = upper ? v[i] : v[i + s];
      const R keep = upper ? v[i + s] : v[i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, s);
    }
  }
}

constexpr int OT = 512;  // threads per system in the orthogonalisation

// w = V_b[j+1] is orthogonalised against the recycled C_b (s_cur vectors)
// and V_b[0..j] with two classical Gram-Schmidt passes, then normalised, and
// the new column of H enters the Givens least-squares update; the
// summed coefficients of both passes go to Bk (C part) and H (V part) in
// FP64. The first pass's update and the second pass's inner products share
// one sweep over the basis, and the second update computes ||w||: the
// basis is read three times.
template <typename T2>
__global__ void __launch_bounds__(OT, sizeof(T2) == 8 ? 2 : 1) k_ortho(int N, int j, int m, int s_cur, const int* __restrict__ list,
                                             const int* __restrict__ count, T2* __restrict__ V,
                                             const T2* __restrict__ C, size_t c_ss, double2* __restrict__ H,
                                             double2* __restrict__ Bk, int smax, LsqArgs L) {
  using R = typename RealOf<T2>::T;
  constexpr int NW = OT / 32;
  __shared__ R red[NW][32];
  __shared__ T2 coef[2][64];
  __shared__ double2 hcol[64];  // new column of H (m + 1 <= 61 entries)
  __shared__ double cs_s[64];   // previous Givens rotations
  __shared__ double2 sn_s[64];
  const int slot = blockIdx.x;
  if (slot >= *count) return;
  const int b = list[slot];
  T2* Vb = V + (size_t)b * (m + 1) * N;
  T2* w = Vb + (size_t)(j + 1) * N;
  const T2* Cb = C + (size_t)b * c_ss;
  const int nb = s_cur + j + 1;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  auto basis = [&](int q) -> const T2* { return q < s_cur ? Cb + (size_t)q * N : Vb + (size_t)(q - s_cur) * N; };
  // block sum of 16 complex inner products held as 32 reals per thread
  auto reduce16 = [&](R (&acc)[32], T2* out, int q0) {
    warp_reduce_scatter32<R>(acc);
    red[warp][lane] = acc[0];
    __syncthreads();
    if (threadIdx.x < 32) {
      R s = R(0);
#pragma unroll
      for (int w2 = 0; w2 < NW; ++w2) s += red[w2][threadIdx.x];
      const R im = __shfl_xor_sync(0xffffffffu, s, 1);
      const int q = q0 + (threadIdx.x >> 1);
      if ((threadIdx.x & 1) == 0 && q < nb) {
        T2 c;
        c.x = s;
        c.y = im;
        out[q] = c;
      }
    }
    __syncthreads();
  };
  // w -= sum_q basis_q[e] * cf[q], with the basis loads issued eight at a time
  auto update = [&](int e, T2 we, const T2* cf) -> T2 {
    for (int p0 = 0; p0 < nb; p0 += 8) {
      T2 qv[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) qv[u] = p0 + u < nb ? basis(p0 + u)[e] : cvt<T2>(make_double2(0.0, 0.0));
#pragma unroll
      for (int u = 0; u < 8; ++u)
        if (p0 + u < nb) we = csub(we, cmul(qv[u], cf[p0 + u]));
    }
    return we;
  };
  auto accumulate = [&](R (&acc)[32], int e, int q0, T2 we) {
#pragma unroll
    for (int u = 0; u < 16; ++u) {
      if (q0 + u < nb) {
        const T2 qe = basis(q0 + u)[e];
        acc[2 * u] += qe.x * we.x + qe.y * we.y;
        acc[2 * u + 1] += qe.x * we.y - qe.y * we.x;
      }
    }
  };
  // pass 1: inner products
  for (int q0 = 0; q0 < nb; q0 += 16) {
    R acc[32];
#pragma unroll
    for (int u = 0; u < 32; ++u) acc[u] = R(0);
    for (int e = threadIdx.x; e < N; e += OT) accumulate(acc, e, q0, w[e]);
    reduce16(acc, coef[0], q0);
  }
  // pass 1 update, fused with the pass 2 inner products
  for (int q0 = 0; q0 < nb; q0 += 16) {
    R acc[32];
#pragma unroll
    for (int u = 0; u < 32; ++u) acc[u] = R(0);
    for (int e = threadIdx.x; e < N; e += OT) {
      T2 we = w[e];
      if (q0 == 0) {
        we = update(e, we, coef[0]);
        w[e] = we;
      }
      accumulate(acc, e, q0, we);
    }
    reduce16(acc, coef[1], q0);
  }
  // pass 2 update and the norm
  R nr = R(0);
  for (int e = threadIdx.x; e < N; e += OT) {
    const T2 we = update(e, w[e], coef[1]);
    w[e] = we;
    nr += cabs2(we);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) nr += __shfl_xor_sync(0xffffffffu, nr, o);
  if (lane == 0) red[warp][0] = nr;
  __syncthreads();
  R tot = R(0);
#pragma unroll
  for (int w2 = 0; w2 < NW; ++w2) tot += red[w2][0];
  double2* H0c = L.H0 + (size_t)b * (m + 1) * m + (size_t)j * (m + 1);
  double2* Bc = Bk + (size_t)b * smax * m + (size_t)j * smax;
  if (threadIdx.x < nb) {
    const int q = threadIdx.x;
    const double2 cval = cadd(to_d2(coef[0][q]), to_d2(coef[1][q]));
    if (q < s_cur) {
      Bc[q] = cval;
    } else {
      H0c[q - s_cur] = cval;
      hcol[q - s_cur] = cval;
    }
  }
  if (threadIdx.x >= 32 && threadIdx.x < 32 + j) {  // the previous rotations
    cs_s[threadIdx.x - 32] = L.cs[(size_t)b * m + threadIdx.x - 32];
    sn_s[threadIdx.x - 32] = L.sn[(size_t)b * m + threadIdx.x - 32];
  }
  double2 gj = make_double2(0.0, 0.0);
  double tola = 0.0;
  int itd = 0;
  if (threadIdx.x == 0) {
    gj = L.g[(size_t)b * (m + 1) + j];
    tola = L.tolabs[b];
    itd = L.iters_done[b];
    const double nrm = sqrt((double)tot);
    H0c[j + 1] = make_double2(nrm, 0.0);
    hcol[j + 1] = make_double2(nrm, 0.0);
  }
  __syncthreads();
  if (threadIdx.x == 0)  // while the others normalise w
    lsq_column<typename RealOf<T2>::T>(b, j, m, H, hcol, cs_s, sn_s, gj, tola, itd, L);
  const R rn = sqrt(tot);
  const R inv = rn > R(0) ? R(1) / rn : R(0);
  for (int e = threadIdx.x; e < N; e += OT) w[e] = cscale(w[e], inv);
}

// ---------------------------------------------------------------- starts
// beta = ||r_b||, V_b[0] = r_b / beta, g = beta e1; systems already below
// tolabs are flagged done (jstop = 0).
template <typename T2>
__global__ void __launch_bounds__(NT) k_cycle_start(int N, int m, const int* __restrict__ list,
                                                   const int* __restrict__ count, const T2* __restrict__ R,
                                                   T2* __restrict__ V, double2* __restrict__ g,
                                                   const double* __restrict__ tolabs, int* __restrict__ flag,
                                                   int* __restrict__ jstop, double* __restrict__ beta_out) {
  using RT = typename RealOf<T2>::T;
  __shared__ RT red[32];
  const int slot = blockIdx.x;
  if (slot >= *count) return;
  const int b = list[slot];
  const T2* r = R + (size_t)b * N;
  RT s[1] = {RT(0)};
  for (int e = threadIdx.x; e < N; e += NT) s[0] += cabs2(r[e]);
  block_sum<1, RT>(s, red);
  const RT rn = sqrt(s[0]);
  T2* v0 = V + (size_t)b * (m + 1) * N;
  const RT inv = rn > RT(0) ? RT(1) / rn : RT(0);
  for (int e = threadIdx.x; e < N; e += NT) v0[e] = cscale(r[e], inv);
  if (threadIdx.x == 0) {
    const double beta = sqrt((double)s[0]);
    double2* gb = g + (size_t)b * (m + 1);
    gb[0] = make_double2(beta, 0.0);
    beta_out[b] = beta;
    bool done = !(beta > tolabs[b]);
    flag[b] = done ? -1 : 1;  // -1: converged (status code 1)
    jstop[b] = 0;
  }
}

// --------------------------------------------------- cycle end: y, residual
// Solve the rotated triangular system for y2 (length jstop), y1 = -Bk y2,
// and the residual coefficients c = beta e1 - H0 y2 (length jstop + 1).
// Outputs per system: coefY[0..s_cur) = y1, coefY[s_cur..s_cur+jstop) = y2,
// coefR[0..jstop] = c.
constexpr int CS_WARPS = 4;  // systems (warps) per CTA of k_cycle_solve
__global__ void k_cycle_solve(int m, int smax, int s_cur, const int* __restrict__ list,
                              const int* __restrict__ count, const double2* __restrict__ H,
                              const double2* __restrict__ H0, const double2* __restrict__ Bk,
                              const double2* __restrict__ g, const double* __restrict__ beta,
                              const int* __restrict__ jstop, double2* __restrict__ coefY, double2* __restrict__ coefR);

// x_b += [U_b Z_b] coefY,  r_b = V_b[0..jstop] coefR
template <typename T2>
__global__ void __launch_bounds__(NT) k_update_xr(int N, int m, int smax, int s_cur, const int* __restrict__ list,
                                                 const int* __restrict__ count, const int* __restrict__ jstop,
                                                 const double2* __restrict__ coefY,
                                                 const double2* __restrict__ coefR, const T2* __restrict__ U,
                                                 const T2* __restrict__ Z, const T2* __restrict__ V,
                                                 T2* __restrict__ X, T2* __restrict__ R) {
  __shared__ T2 cy[128], cr[128];
  const int slot = blockIdx.y;
  if (slot >= *count) return;
  const int b = list[slot];
  const int js = jstop[b];
  if (js <= 0) return;
  for (int q = threadIdx.x; q < s_cur + js; q += NT) cy[q] = cvt<T2>(coefY[(size_t)b * (m + smax + 1) + q]);
  for (int q = threadIdx.x; q <= js; q += NT) cr[q] = cvt<T2>(coefR[(size_t)b * (m + 1) + q]);
  __syncthreads();
  const T2* Ub = U + (size_t)b * smax * N;
  const T2* Zb = Z + (size_t)b * m * N;
  const T2* Vb = V + (size_t)b * (m + 1) * N;
  for (int e = blockIdx.x * NT + threadIdx.x; e < N; e += gridDim.x * NT) {
    T2 x = X[(size_t)b * N + e];
    for (int q = 0; q < s_cur; ++q) x = cfma(Ub[(size_t)q * N + e], cy[q], x);
    for (int q = 0; q < js; ++q) x = cfma(Zb[(size_t)q * N + e], cy[s_cur + q], x);
    X[(size_t)b * N + e] = x;
    T2 r = cvt<T2>(make_double2(0.0, 0.0));
    for (int q = 0; q <= js; ++q) r = cfma(Vb[(size_t)q * N + e], cr[q], r);
    R[(size_t)b * N + e] = r;
  }
}

// ------------------------------------------------- batched Gram: A^H B
// out_b (na x nb, ld = ldo, system stride os) = [A segs]^H [B segs],
// na, nb <= 64. Each system is served by a cluster of gridDim.y CTAs (GT
// threads each; 1 for full batches, GSPLIT when few systems need a Gram)
// that split the vector length: CTA r sums elements
// [r N / gridDim.y, (r+1) N / gridDim.y), and CTA 0 adds the partial Grams of
// the cluster in rank order through distributed shared memory
// (deterministic).
// Within a CTA, K tiles are staged with consecutive threads reading one
// vector (coalesced); the tile length grows when the matrices are narrow.
// Outputs are 2 x 2 tiles; when there are fewer tiles than threads, Q
// consecutive threads share a tile and split each K tile (their partial
// sums meet through shuffles). Each K tile is summed in the vector precision
// and accumulated in FP64.
constexpr int GT = 256, GSPLIT = 8, GK_ELEMS = 2048;  // staged elements per operand

// dynamic shared memory of k_gram: two staging buffers, reused for the na x nb partial Gram
template <typename T2>
__host__ __device__ constexpr size_t gram_smem_bytes() {
  return (2 * GK_ELEMS * sizeof(T2) > 64 * 64 * sizeof(double2)) ? 2 * GK_ELEMS * sizeof(T2)
                                                                  : 64 * 64 * sizeof(double2);
}

template <typename T2>
__global__ void __launch_bounds__(GT)
    k_gram(int N, const int* __restrict__ list, const int* __restrict__ count, Seg2<T2> A, Seg2<T2> Bm,
           double2* __restrict__ out, int ldo, size_t os) {
  namespace cg = cooperative_groups;
  extern __shared__ __align__(16) unsigned char gsm[];
  T2* sa = reinterpret_cast<T2*>(gsm);
  T2* sb = sa + GK_ELEMS;
  double2* part = reinterpret_cast<double2*>(gsm);  // after the K loop
  cg::cluster_group cluster = cg::this_cluster();
  const int slot = blockIdx.x;
  if (slot >= *count) return;  // uniform over the cluster (same slot)
  const int rank = (int)cluster.block_rank();
  const int nsplit = (int)gridDim.y;  // the launch makes the cluster span gridDim.y
  const int b = list[slot];
  const int na = A.cnt(b), nbb = Bm.cnt(b);
  const int ta = (na + 1) / 2, tb = (nbb + 1) / 2, ntile = ta * tb;  // <= 1024 = 4 GT
  int Q = 1;
  while (Q < 32 && ntile * Q * 2 <= GT) Q *= 2;
  const int q = threadIdx.x % Q, tslot = threadIdx.x / Q, tstride = GT / Q;
  const int cmax = max(2 * ta, 2 * tb);
  const int ld = cmax + 1;  // padded row of a staged K element
  int tk = GK_ELEMS / ld;
  if (tk >= 32) tk -= tk % 32;
  const int e_beg = (int)((long long)N * rank / nsplit), e_end = (int)((long long)N * (rank + 1) / nsplit);
  const T2 z = cvt<T2>(make_double2(0.0, 0.0));
  double2 acc[4][4];
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) acc[u][v] = make_double2(0.0, 0.0);
  for (int e0 = e_beg; e0 < e_end; e0 += tk) {
    for (int e = threadIdx.x; e < tk * cmax; e += GT) {
      const int c = e / tk, l = e % tk;
      const int ee = e0 + l;
      sa[l * ld + c] = (c < na && ee < e_end) ? A.vec(b, c)[ee] : z;
      sb[l * ld + c] = (c < nbb && ee < e_end) ? Bm.vec(b, c)[ee] : z;
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int tile = tslot + u * tstride;
      if (tile < ntile) {
        const int i0 = 2 * (tile % ta), j0 = 2 * (tile / ta);
        T2 t00 = z, t01 = z, t10 = z, t11 = z;
        for (int l = q; l < tk; l += Q) {
          const T2* ra = sa + l * ld;
          const T2* rb = sb + l * ld;
          const T2 a0 = ra[i0], a1 = ra[i0 + 1], b0 = rb[j0], b1 = rb[j0 + 1];
          t00 = cadd(t00, cjmul(a0, b0));
          t10 = cadd(t10, cjmul(a1, b0));
          t01 = cadd(t01, cjmul(a0, b1));
          t11 = cadd(t11, cjmul(a1, b1));
        }
        acc[u][0] = cadd(acc[u][0], to_d2(t00));
        acc[u][1] = cadd(acc[u][1], to_d2(t10));
        acc[u][2] = cadd(acc[u][2], to_d2(t01));
        acc[u][3] = cadd(acc[u][3], to_d2(t11));
      }
    }
    __syncthreads();
  }
  // partial sums of the Q threads of a tile (consecutive lanes of one warp)
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v)
      for (int o = Q / 2; o > 0; o >>= 1) {
        acc[u][v].x += __shfl_xor_sync(0xffffffffu, acc[u][v].x, o);
        acc[u][v].y += __shfl_xor_sync(0xffffffffu, acc[u][v].y, o);
      }
  // this CTA's partial Gram into its shared memory (the staging buffers are free)
  if (q == 0) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int tile = tslot + u * tstride;
      if (tile < ntile) {
        const int i0 = 2 * (tile % ta), j0 = 2 * (tile / ta);
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          const int i = i0 + (v & 1), jj = j0 + (v >> 1);
          if (i < na && jj < nbb) part[i + jj * na] = acc[u][v];
        }
      }
    }
  }
  cluster.sync();
  if (rank == 0) {
    for (int e = threadIdx.x; e < na * nbb; e += GT) {
      double2 sum = make_double2(0.0, 0.0);
      for (int r = 0; r < nsplit; ++r) sum = cadd(sum, cluster.map_shared_rank(part, r)[e]);
      out[(size_t)b * os + (e % na) + (size_t)(e / na) * ldo] = sum;
    }
  }
  cluster.sync();  // keep every CTA's shared memory alive until rank 0 has read it
}

// Launch of k_gram for up to B listed systems, of which about `expect` are
// listed; clusters of GSPLIT CTAs per system when that leaves the GPU
// underfilled (sets the shared-memory limit once).
template <typename T2>
int launch_gram(int N, const int* list, const int* count, int B, int expect, const Seg2<T2>& A,
                const Seg2<T2>& Bm, double2* out, int ldo, size_t os, cudaStream_t st);

// ------------------------------------- batched tall-skinny times small matrix
// Out_b[:, c] = sum_i In_b[i] M_b[i, c],  c < ncols (<= 16), i < In.cnt(b).
// M_b at Msmall + b*ms (ld = ldm); with shared_in the input segments ignore b.
template <typename T2, typename TO2>
__global__ void __launch_bounds__(NT) k_tsmm(int N, const int* __restrict__ list, const int* __restrict__ count,
                                            Seg2<T2> In, const double2* __restrict__ Msmall, int ldm, size_t ms,
                                            int ncols, TO2* __restrict__ Out, size_t o_ss, size_t o_vs,
                                            int accumulate) {
  __shared__ T2 sm[64 * 16];
  const int slot = blockIdx.y;
  if (slot >= *count) return;
  const int b = list[slot];
  const int ni = In.cnt(b);
  for (int q = threadIdx.x; q < ni * ncols; q += NT) {
    int i = q % ni, c = q / ni;
    sm[i * 16 + c] = cvt<T2>(Msmall[(size_t)b * ms + i + (size_t)c * ldm]);
  }
  __syncthreads();
  for (int e = blockIdx.x * NT + threadIdx.x; e < N; e += gridDim.x * NT) {
    T2 acc[16];
#pragma unroll
    for (int c = 0; c < 16; ++c) acc[c] = cvt<T2>(make_double2(0.0, 0.0));
    for (int i = 0; i < ni; ++i) {
      const T2 x = In.vec(b, i)[e];
#pragma unroll
      for (int c = 0; c < 16; ++c)
        if (c < ncols) acc[c] = cfma(x, sm[i * 16 + c], acc[c]);
    }
#pragma unroll
    for (int c = 0; c < 16; ++c) {
      if (c < ncols) {
        TO2* o = Out + (size_t)b * o_ss + (size_t)c * o_vs + e;
        double2 v = to_d2(acc[c]);
        if (accumulate) v = cadd(to_d2(*o), v);
        *o = from_d2<TO2>(v);
      }
    }
  }
}

// ------------------------------------------------ harmonic-Ritz recycle update
// For each system (one warp): with Ghat = [[D, Bk], [0, H0]] (rows s+js+1,
// cols s+js), F = [C V]^H [U Z] (columns of U scaled by D = 1/||U_i||),
// solve Ghat^H Ghat z = theta Ghat^H F z for the s smallest |theta|
// (Cholesky Ghat^H Ghat = L L^H turns it into the standard problem
// K y = mu y, K = L^{-1} Ghat^H F L^{-H}, mu = 1/theta: largest |mu|);
// P = L^{-H} Y_sel; QR: Ghat P = Qc R. Outputs Pu = diag(D, I) P R^{-1}
// (new U = [U Z] Pu) and Qc (new C = [C V] Qc); ok[b] = 1 on success.
__global__ void k_ritz(int m, int smax, int s_cur, int s_new, const int* __restrict__ list,
                       const int* __restrict__ count, const int* __restrict__ jstop, const double2* __restrict__ H0,
                       const double2* __restrict__ Bk, const double2* __restrict__ F, const double2* __restrict__ UU,
                       double2* __restrict__ work, size_t wstride, double2* __restrict__ Pu,
                       double2* __restrict__ Qc, int* __restrict__ ok);
// Dynamic shared memory of k_ritz (launched with 32 threads per CTA, one CTA per system).
size_t ritz_smem_bytes(int m, int smax);

// ------------------------------------------------------- recycle start (CholQR2)
// Given Gram G (s x s) of the current C block, Rinv = L^{-H} (upper), with
// G = L L^H; Racc := Racc * Rinv when accumulate. ok[b] = 0 on failure.
__global__ void k_chol_rinv(int s, const int* __restrict__ list, const int* __restrict__ count,
                            double2* __restrict__ G, size_t gs, double2* __restrict__ Rinv,
                            double2* __restrict__ Racc, double2* __restrict__ tmp, int accumulate,
                            int* __restrict__ ok);

// Recycle start of the FP32 solves, fused into one CTA per listed system
// (the FP64 path runs the same steps as separate kernels):
//   C = T(v_b) Ut = Ut D(v_b)^{-1} - C0Ut,
//   two CholQR passes (G = C^H C = L L^H, C := C L^{-H}; the 16 x 16 factor
//   and its inverse in one warp's registers), Ra = product of the L^{-H}
//   factors, C written out, U = Ut Ra,
//   c = C^H r, x += U c, r -= C c.
// C_b stays in shared memory between the steps. ok[b] = 0 when a Cholesky
// factor fails (the projection is then not applied to that system).
constexpr int RS_T = 512;
__global__ void k_recstart32(int n, int k, int s, const int* __restrict__ list, const int* __restrict__ count,
                             const float2* __restrict__ Ut, const float2* __restrict__ C0Ut,
                             const double* __restrict__ vinv, float2* __restrict__ C, float2* __restrict__ U,
                             size_t ss, float2* __restrict__ X, float2* __restrict__ R, int* __restrict__ ok);
size_t recstart32_smem_bytes(int s, int N);

// AU_b[c] = Ut[c] o (1/v_b per column block) - C0Ut[c]
template <typename T2>
__global__ void __launch_bounds__(NT) k_make_AU(int n, int k, int s, const int* __restrict__ list,
                                               const int* __restrict__ count, const T2* __restrict__ Ut,
                                               const T2* __restrict__ C0Ut, const double* __restrict__ vinv,
                                               T2* __restrict__ AU, size_t au_ss) {
  const int slot = blockIdx.y;
  if (slot >= *count) return;
  const int b = list[slot];
  const int N = n * k;
  for (int e = blockIdx.x * NT + threadIdx.x; e < N * s; e += gridDim.x * NT) {
    int t = (e % N) / n;
    double2 u = to_d2(Ut[e]);
    double2 cu = to_d2(C0Ut[e]);
    AU[(size_t)b * au_ss + e] = from_d2<T2>(csub(cscale(u, vinv[(size_t)b * k + t]), cu));
  }
}

// c = C_b^H r_b (s values): x_b += U_b c, r_b -= C_b c
template <typename T2>
__global__ void __launch_bounds__(NT) k_project(int N, int s, const int* __restrict__ list,
                                               const int* __restrict__ count, const T2* __restrict__ C,
                                               const T2* __restrict__ U, size_t ss, T2* __restrict__ X,
                                               T2* __restrict__ R) {
  using RT = typename RealOf<T2>::T;
  __shared__ RT red[32 * 32];
  __shared__ T2 coef[16];
  const int slot = blockIdx.x;
  if (slot >= *count) return;
  const int b = list[slot];
  const T2* Cb = C + (size_t)b * ss;
  const T2* Ub = U + (size_t)b * ss;
  T2* x = X + (size_t)b * N;
  T2* r = R + (size_t)b * N;
  RT acc[32];
#pragma unroll
  for (int u = 0; u < 32; ++u) acc[u] = RT(0);
  for (int e = threadIdx.x; e < N; e += NT) {
    const T2 re = r[e];
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      if (q < s) {
        const T2 ce = Cb[(size_t)q * N + e];
        acc[2 * q] += ce.x * re.x + ce.y * re.y;
        acc[2 * q + 1] += ce.x * re.y - ce.y * re.x;
      }
    }
  }
  block_sum<32, RT>(acc, red);
  if (threadIdx.x < 16) {
    T2 c;
    c.x = acc[2 * threadIdx.x];
    c.y = acc[2 * threadIdx.x + 1];
    coef[threadIdx.x] = c;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < N; e += NT) {
    T2 xe = x[e], re = r[e];
    for (int q = 0; q < s; ++q) {
      xe = cfma(Ub[(size_t)q * N + e], coef[q], xe);
      re = csub(re, cmul(Cb[(size_t)q * N + e], coef[q]));
    }
    x[e] = xe;
    r[e] = re;
  }
}

// ------------------------------------------------------------- reductions
// out[b] = Re sum_e a_b[e] * h[e] (h shared) ; used for the trace <h, W'>
template <typename T2>
__global__ void __launch_bounds__(NT) k_dot_h(int N, int nsys, const T2* __restrict__ A, size_t ss,
                                             const double2* __restrict__ h, double* __restrict__ re_out,
                                             double* __restrict__ im_out) {
  __shared__ double red[64];
  const int b = blockIdx.x;
  if (b >= nsys) return;
  double acc[2] = {0.0, 0.0};
  for (int e = threadIdx.x; e < N; e += NT) {
    double2 p = cmul(to_d2(A[(size_t)b * ss + e]), h[e]);
    acc[0] += p.x;
    acc[1] += p.y;
  }
  block_sum<2>(acc, red);
  if (threadIdx.x == 0) {
    re_out[b] = acc[0];
    if (im_out) im_out[b] = acc[1];
  }
}

// out[b] = ||a_b||_2
template <typename T2>
__global__ void __launch_bounds__(NT) k_norms(int N, int nsys, const T2* __restrict__ A, size_t ss,
                                             double* __restrict__ out) {
  using RT = typename RealOf<T2>::T;
  __shared__ RT red[32];
  const int b = blockIdx.x;
  if (b >= nsys) return;
  RT acc[1] = {RT(0)};
  for (int e = threadIdx.x; e < N; e += NT) acc[0] += cabs2(A[(size_t)b * ss + e]);
  block_sum<1, RT>(acc, red);
  if (threadIdx.x == 0) out[b] = sqrt((double)acc[0]);
}

}  // namespace kry
