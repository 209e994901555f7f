// Non-template kernels of the batched recycled Krylov solver (see krylov.cuh).
#include "krylov.cuh"

namespace kry {

__global__ void k_iota(int B, int* list, int* count) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < B; i += gridDim.x * blockDim.x) list[i] = i;
  if (blockIdx.x == 0 && threadIdx.x == 0) *count = B;
}

// single CTA of 1024 threads; order-preserving
__global__ void k_compact(const int* __restrict__ in_list, const int* __restrict__ in_count,
                          const int* __restrict__ flag, int* __restrict__ out_list, int* __restrict__ out_count) {
  __shared__ int sc[1024];
  const int n = *in_count;
  const int per = (n + blockDim.x - 1) / blockDim.x;
  const int beg = threadIdx.x * per;
  const int end = min(n, beg + per);
  int c = 0;
  for (int i = beg; i < end; ++i) c += flag[in_list[i]] > 0;
  sc[threadIdx.x] = c;
  __syncthreads();
  for (int off = 1; off < (int)blockDim.x; off <<= 1) {
    int v = (int)threadIdx.x >= off ? sc[threadIdx.x - off] : 0;
    __syncthreads();
    sc[threadIdx.x] += v;
    __syncthreads();
  }
  int pos = sc[threadIdx.x] - c;
  for (int i = beg; i < end; ++i) {
    int b = in_list[i];
    if (flag[b] > 0) out_list[pos++] = b;
  }
  if (threadIdx.x == blockDim.x - 1) *out_count = sc[threadIdx.x];
}

__global__ void k_cycle_solve(int m, int smax, int s_cur, const int* __restrict__ list,
                              const int* __restrict__ count, const double2* __restrict__ H,
                              const double2* __restrict__ H0, const double2* __restrict__ Bk,
                              const double2* __restrict__ g, const double* __restrict__ beta,
                              const int* __restrict__ jstop, double2* __restrict__ coefY, double2* __restrict__ coefR) {
  const int slot = blockIdx.x * blockDim.x + threadIdx.x;
  if (slot >= *count) return;
  const int b = list[slot];
  const int js = jstop[b];
  const double2* Hb = H + (size_t)b * (m + 1) * m;
  const double2* H0b = H0 + (size_t)b * (m + 1) * m;
  const double2* gb = g + (size_t)b * (m + 1);
  double2* cy = coefY + (size_t)b * (m + smax + 1);
  double2* cr = coefR + (size_t)b * (m + 1);
  double2* y2 = cy + s_cur;
  for (int i = js - 1; i >= 0; --i) {
    double2 x = gb[i];
    for (int l = i + 1; l < js; ++l) x = csub(x, cmul(Hb[i + (size_t)l * (m + 1)], y2[l]));
    double2 d = Hb[i + (size_t)i * (m + 1)];
    y2[i] = cabs2(d) > 0 ? cdiv(x, d) : make_double2(0.0, 0.0);
  }
  const double2* Bb = Bk + (size_t)b * smax * m;
  for (int q = 0; q < s_cur; ++q) {
    double2 x = make_double2(0.0, 0.0);
    for (int l = 0; l < js; ++l) x = cfma(Bb[q + (size_t)l * smax], y2[l], x);
    cy[q] = cscale(x, -1.0);
  }
  for (int i = 0; i <= js; ++i) {
    double2 x = make_double2(i == 0 ? beta[b] : 0.0, 0.0);
    for (int l = 0; l < js; ++l) {
      if (i <= l + 1) x = csub(x, cmul(H0b[i + (size_t)l * (m + 1)], y2[l]));
    }
    cr[i] = x;
  }
}

// One warp (one CTA of 32 threads) per system. The generalized problem
// Ghat^H Ghat z = theta Ghat^H Fhat z is reduced through a Householder QR
// Ghat = Qg Rg (no normal equations): Rg z = theta (Qg^H Fhat) z, i.e.
// K z = mu z with K = Rg^{-1} (Qg^H Fhat) and mu = 1/theta; the s largest |mu|
// (smallest |theta|) are kept. The eigen-decomposition runs in FP32 in
// shared memory; it only selects the recycle subspace. The part that keeps
// the relation T U = C exact (Y = Ghat P, Y = Qc R, Pu = diag(D, I) P R^{-1})
// runs in FP64.
__global__ void __launch_bounds__(32) k_ritz(int m, int smax, int s_cur, int s_new, const int* __restrict__ list,
                                           const int* __restrict__ count, const int* __restrict__ jstop,
                                           const double2* __restrict__ H0, const double2* __restrict__ Bk,
                                           const double2* __restrict__ F, const double2* __restrict__ UU,
                                           double2* __restrict__ work, size_t wstride, double2* __restrict__ Pu,
                                           double2* __restrict__ Qc, int* __restrict__ ok) {
  const int slot = blockIdx.x;
  if (slot >= *count) return;
  const int b = list[slot];
  const int js = jstop[b];
  const int me = s_cur + js, re = me + 1;
  const int LD = m + smax + 1;
  if (me < s_new || js <= 0) {
    if (sd::lane() == 0) ok[b] = 0;
    return;
  }
  // shared matrices use leading dimension LS = m + 1 >= re (re x me at most).
  // K is formed in place of Qg^H Fhat, and Q takes the space of Gf once its
  // triangular factor has been used.
  const int LS = m + 1;
  extern __shared__ float2 smf[];
  float2* Gf = smf;                          // LS x LS
  float2* Ff = Gf + (size_t)LS * LS;         // LS x LS -> Qg^H Fhat -> K
  float2* K = Ff;
  float2* Q = Gf;                            // after the triangular solve
  float2* vt = Ff + (size_t)LS * LS;         // LS
  float2* Yz = vt + LS;                      // LS x 16
  float2* Xf = Yz + (size_t)LS * 16;         // LS x 16
  int* sel = reinterpret_cast<int*>(Xf + (size_t)LS * 16);  // 16
  double2* w = work + (size_t)b * wstride;
  double2* Gh = w;                           // LD x LD (FP64)
  double2* P = Gh + (size_t)LD * LD;         // LD x 16
  double2* Y = P + (size_t)LD * 16;          // LD x 16
  double2* Yq = Y + (size_t)LD * 16;         // LD x 16
  double2* R = Yq + (size_t)LD * 16;         // 16 x 16
  double2* coef = R + 256;                   // LD
  double D[16];
  const double2* UUb = UU + (size_t)b * smax * smax;
  for (int q = 0; q < s_cur; ++q) {
    const double nn = UUb[q + (size_t)q * smax].x;
    D[q] = nn > 0 ? 1.0 / sqrt(nn) : 1.0;
  }
  const double2* H0b = H0 + (size_t)b * (m + 1) * m;
  const double2* Bb = Bk + (size_t)b * smax * m;
  const double2* Fb = F + (size_t)b * LD * LD;
  for (int e = sd::lane(); e < re * me; e += 32) {
    const int i = e % re, c = e / re;
    double2 v = make_double2(0.0, 0.0);
    if (i < s_cur && c < s_cur) {
      if (i == c) v = make_double2(D[i], 0.0);
    } else if (i < s_cur) {
      v = Bb[i + (size_t)(c - s_cur) * smax];
    } else if (c >= s_cur) {
      const int ii = i - s_cur, cc = c - s_cur;
      if (ii <= cc + 1) v = H0b[ii + (size_t)cc * (m + 1)];
    }
    Gh[i + (size_t)c * LD] = v;
    Gf[i + (size_t)c * LS] = make_float2((float)v.x, (float)v.y);
    double2 f = Fb[i + (size_t)c * LD];
    if (c < s_cur) f = cscale(f, D[c]);
    Ff[i + (size_t)c * LS] = make_float2((float)f.x, (float)f.y);
  }
  sd::wsync();
  sd::householder_qr_apply<float2>(re, me, Gf, LS, Ff, LS, me, vt);
  sd::trsm_upper_left<float2>(me, me, Gf, LS, K, LS);  // K = Rg^{-1} (Qg^H Fhat), in place
  bool fin = true;
  for (int e = sd::lane(); e < me * me; e += 32) {
    const float2 v = K[(e % me) + (size_t)(e / me) * LS];
    fin &= isfinite(v.x) && isfinite(v.y);
  }
  if (!__all_sync(0xffffffffu, fin)) {
    if (sd::lane() == 0) ok[b] = 0;
    return;
  }
  sd::hessenberg<float2>(me, K, LS, Q, LS, vt);
  if (sd::hqr<float2>(me, K, LS, Q, LS, 60 * me)) {
    if (sd::lane() == 0) ok[b] = 0;
    return;
  }
  if (sd::lane() == 0) {
    for (int c = 0; c < s_new; ++c) {
      int best = -1;
      float bv = -1.f;
      for (int i = 0; i < me; ++i) {
        bool used = false;
        for (int q = 0; q < c; ++q) used |= sel[q] == i;
        if (used) continue;
        const float a = cabs2(K[i + (size_t)i * LS]);
        if (a > bv) {
          bv = a;
          best = i;
        }
      }
      sel[c] = best;
    }
  }
  sd::wsync();
  sd::schur_vectors<float2>(me, K, LS, Q, LS, sel, s_new, Yz, LS, Xf, LS);
  for (int e = sd::lane(); e < me * s_new; e += 32) {
    const float2 x = Xf[(e % me) + (size_t)(e / me) * LS];
    P[(e % me) + (size_t)(e / me) * LD] = make_double2(x.x, x.y);
  }
  sd::wsync();
  sd::gemm_nn(re, s_new, me, Gh, LD, P, LD, Y, LD);
  if (sd::qr_cgs2(re, s_new, Y, LD, Yq, LD, R, 16, coef)) {
    if (sd::lane() == 0) ok[b] = 0;
    return;
  }
  for (int e = sd::lane(); e < s_cur * s_new; e += 32) {
    const int i = e % s_cur, c = e / s_cur;
    P[i + (size_t)c * LD] = cscale(P[i + (size_t)c * LD], D[i]);
  }
  sd::wsync();
  sd::trsm_right_upper(me, s_new, R, 16, P, LD);
  bool finite = true;
  for (int e = sd::lane(); e < me * s_new; e += 32) {
    const double2 v = P[(e % me) + (size_t)(e / me) * LD];
    finite &= isfinite(v.x) && isfinite(v.y);
  }
  if (!__all_sync(0xffffffffu, finite)) {
    if (sd::lane() == 0) ok[b] = 0;
    return;
  }
  double2* Pub = Pu + (size_t)b * LD * 16;
  double2* Qcb = Qc + (size_t)b * LD * 16;
  for (int e = sd::lane(); e < me * s_new; e += 32)
    Pub[(e % me) + (size_t)(e / me) * LD] = P[(e % me) + (size_t)(e / me) * LD];
  for (int e = sd::lane(); e < re * s_new; e += 32)
    Qcb[(e % re) + (size_t)(e / re) * LD] = Yq[(e % re) + (size_t)(e / re) * LD];
  if (sd::lane() == 0) ok[b] = 1;
}

size_t ritz_smem_bytes(int m, int /*smax*/) {
  const int LS = m + 1;
  return sizeof(float2) * ((size_t)2 * LS * LS + LS + (size_t)2 * LS * 16) + 16 * sizeof(int);
}

__global__ void k_chol_rinv(int s, const int* __restrict__ list, const int* __restrict__ count,
                            double2* __restrict__ G, size_t gs, double2* __restrict__ Rinv,
                            double2* __restrict__ Racc, double2* __restrict__ tmp, int accumulate,
                            int* __restrict__ ok) {
  const int wg = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (wg >= *count) return;
  const int b = list[wg];
  double2* Gb = G + (size_t)b * gs;
  if (sd::cholesky(s, Gb, s)) {
    if (sd::lane() == 0) ok[b] = 0;
    return;
  }
  double2* Ri = Rinv + (size_t)b * s * s;
  for (int e = sd::lane(); e < s * s; e += 32) Ri[e] = make_double2((e % s) == (e / s) ? 1.0 : 0.0, 0.0);
  sd::wsync();
  sd::trsm_lower_h_left(s, s, Gb, s, Ri, s);  // Ri = L^{-H}
  if (accumulate) {
    double2* Ra = Racc + (size_t)b * s * s;
    double2* T = tmp + (size_t)b * s * s;
    sd::gemm_nn(s, s, s, Ra, s, Ri, s, T, s);
    for (int e = sd::lane(); e < s * s; e += 32) Ra[e] = T[e];
    sd::wsync();
  }
  if (sd::lane() == 0) ok[b] = 1;
}

}  // namespace kry
