// Non-template kernels of the batched recycled Krylov solver (see krylov.cuh).
#include "krylov.cuh"

namespace kry {

__global__ void k_iota(int B, int* list, int* count) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < B; i += gridDim.x * blockDim.x) list[i] = i;
  if (blockIdx.x == 0 && threadIdx.x == 0) *count = B;
}

// single CTA of 1024 threads; order-preserving
__global__ void k_compact(const int* __restrict__ in_list, const int* __restrict__ in_count,
                          const int* __restrict__ flag, int* __restrict__ out_list, int* __restrict__ out_count,
                          int* host_count) {
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
  if (threadIdx.x == blockDim.x - 1) {
    *out_count = sc[threadIdx.x];
    if (host_count) *host_count = sc[threadIdx.x];
  }
}

// One warp per system (CS_WARPS warps per CTA). Back substitution
// R y2 = g (R = the rotated Hessenberg H, js x js upper triangular) by
// columns: lane i keeps x_i for rows i and i + 32; once y2[l] is final, every
// row above it subtracts H[i, l] y2[l] in parallel. Then
// cy = -Bk y2 (the recycled part) and cr = beta e1 - H0 y2 (the coefficients
// of the new residual in [C V]).
__global__ void __launch_bounds__(32 * CS_WARPS) k_cycle_solve(
    int m, int smax, int s_cur, const int* __restrict__ list, const int* __restrict__ count,
    const double2* __restrict__ H, const double2* __restrict__ H0, const double2* __restrict__ Bk,
    const double2* __restrict__ g, const double* __restrict__ beta, const int* __restrict__ jstop,
    double2* __restrict__ coefY, double2* __restrict__ coefR) {
  __shared__ double2 ys[CS_WARPS][64];
  const int wi = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int slot = blockIdx.x * CS_WARPS + wi;
  if (slot >= *count) return;  // whole warp
  const int b = list[slot];
  const int js = jstop[b];
  const size_t ldh = (size_t)(m + 1);
  const double2* Hb = H + (size_t)b * (m + 1) * m;
  const double2* H0b = H0 + (size_t)b * (m + 1) * m;
  const double2* gb = g + (size_t)b * (m + 1);
  double2* cy = coefY + (size_t)b * (m + smax + 1);
  double2* cr = coefR + (size_t)b * (m + 1);
  double2* y2 = cy + s_cur;
  double2* y = ys[wi];
  const double2 zero = make_double2(0.0, 0.0);
  double2 x0 = lane < js ? gb[lane] : zero, x1 = lane + 32 < js ? gb[lane + 32] : zero;
  for (int l = js - 1; l >= 0; --l) {
    if (lane == (l & 31)) {
      const double2 xl = l < 32 ? x0 : x1;
      const double2 d = Hb[l + l * ldh];
      y[l] = cabs2(d) > 0 ? cdiv(xl, d) : zero;
    }
    __syncwarp();
    const double2 yl = y[l];
    if (lane < l) x0 = csub(x0, cmul(Hb[lane + l * ldh], yl));
    if (lane + 32 < l) x1 = csub(x1, cmul(Hb[lane + 32 + l * ldh], yl));
  }
  __syncwarp();
  for (int l = lane; l < js; l += 32) y2[l] = y[l];
  const double2* Bb = Bk + (size_t)b * smax * m;
  for (int q = lane; q < s_cur; q += 32) {
    double2 x = zero;
    for (int l = 0; l < js; ++l) x = cfma(Bb[q + (size_t)l * smax], y[l], x);
    cy[q] = cscale(x, -1.0);
  }
  for (int i = lane; i <= js; i += 32) {
    double2 x = make_double2(i == 0 ? beta[b] : 0.0, 0.0);
    for (int l = (i > 0 ? i - 1 : 0); l < js; ++l) x = csub(x, cmul(H0b[i + l * ldh], y[l]));
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

// Recycle start of the FP32 solves in one CTA per system (see krylov.cuh).
// Everything runs in FP32: the Gram matrices of C are those of nearly
// orthonormal columns (C = T(v) Ut with T(v') Ut orthonormal for the
// previous v'), and the second CholQR pass removes what the first leaves.
// Shared memory: 16 x 16 Gram, Cholesky factor, this pass's L^{-H} and the
// accumulated product (column-major, ld 16), reduction scratch, D(v)^{-1},
// then C_b (s rows of N, row stride N + 1).

// Lower Cholesky factor L of the leading s x s block of the Hermitian matrix
// Gf (16 x 16, column-major, ld 16; identity beyond the block) in one warp,
// in shared memory: at step j lane i >= j forms L(i, j), then the lanes
// update the trailing block, a pair (i, q) with j < q <= i per lane per
// round. Writes L to Lf (identity beyond the block, zero above the diagonal)
// and 1 / L(j, j) to rdiag; Gf is overwritten. Returns nonzero when a pivot
// is not positive. Loops run over s, not 16, and keep nothing in register
// arrays (a register-array form of the same factorisation ran about 7x
// slower inside the recycle-start kernel than on its own).
__device__ __forceinline__ int chol16_warp(int s, float2* Gf, float2* Lf, float* rdiag) {
  const int lane = threadIdx.x & 31;
  for (int e = lane; e < 256; e += 32) {
    const int i = e & 15, c = e >> 4;
    Lf[e] = (i >= s || c >= s) ? make_float2(i == c ? 1.f : 0.f, 0.f) : make_float2(0.f, 0.f);
  }
  if (lane < 16 && lane >= s) rdiag[lane] = 1.f;
  __syncwarp();
  int bad = 0;
  for (int j = 0; j < s; ++j) {
    const float d = Gf[j + j * 16].x;
    bad |= !(d > 0.f) || !isfinite(d);
    const float rs = rsqrtf(d);
    if (lane >= j && lane < s) Lf[lane + j * 16] = lane == j ? make_float2(d * rs, 0.f) : cscale(Gf[lane + j * 16], rs);
    if (lane == 0) rdiag[j] = rs;
    __syncwarp();
    // trailing update G(i, q) -= L(i, j) conj(L(q, j)) for j < q <= i < s
    const int t = s - 1 - j;  // trailing order
    for (int e = lane; e < t * (t + 1) / 2; e += 32) {
      int q = 0, rem = e;  // e -> (i, q) with q <= i, both counted from j + 1
      while (rem > q) {
        rem -= q + 1;
        ++q;
      }
      const int ii = j + 1 + q, qq = j + 1 + rem;  // rem <= q
      const float2 upd = cmul(Lf[ii + j * 16], cconj(Lf[qq + j * 16]));
      Gf[ii + qq * 16] = csub(Gf[ii + qq * 16], upd);
    }
    __syncwarp();
  }
  return bad;
}

// Rf = L^{-H} (upper triangular; identity beyond the s x s block): lane c
// solves L x = e_c by forward substitution, in shared memory (Xs, 16 x 16),
// and writes conj(x) as row c of Rf.
__device__ __forceinline__ void linvh16_warp(int s, const float2* Lf, const float* rdiag, float2* Xs, float2* Rf) {
  const int lane = threadIdx.x & 31;
  for (int e = lane; e < 256; e += 32) {
    const int i = e & 15, c = e >> 4;
    Rf[e] = (i >= s || c >= s) ? make_float2(i == c ? 1.f : 0.f, 0.f) : make_float2(0.f, 0.f);
  }
  __syncwarp();
  if (lane < s) {
    const int c = lane;
    for (int i = c; i < s; ++i) {
      float2 acc = make_float2(i == c ? 1.f : 0.f, 0.f);
      for (int p = c; p < i; ++p) acc = csub(acc, cmul(Lf[i + p * 16], Xs[p + c * 16]));
      const float r = rdiag[i];
      const float2 x = make_float2(acc.x * r, acc.y * r);
      Xs[i + c * 16] = x;
      Rf[c + i * 16] = cconj(x);
    }
  }
  __syncwarp();
}

__global__ void __launch_bounds__(RS_T) k_recstart32(int n, int k, int s, const int* __restrict__ list,
                                                    const int* __restrict__ count, const float2* __restrict__ Ut,
                                                    const float2* __restrict__ C0Ut, const double* __restrict__ vinv,
                                                    float2* __restrict__ C, float2* __restrict__ U, size_t ss,
                                                    float2* __restrict__ X, float2* __restrict__ R,
                                                    int* __restrict__ ok) {
  extern __shared__ __align__(16) unsigned char rsm[];
  float2* Gf = reinterpret_cast<float2*>(rsm);                           // 16 x 16
  float2* Lf = Gf + 256;                                                 // 16 x 16
  float2* Rf = Lf + 256;                                                 // 16 x 16, this pass's L^{-H}
  float2* Raf = Rf + 256;                                                // 16 x 16, product of the L^{-H}
  float* red = reinterpret_cast<float*>(Raf + 256);                      // (RS_T / 32) x 32
  float2* coef = reinterpret_cast<float2*>(red + (RS_T / 32) * 32);      // 16
  float* vf = reinterpret_cast<float*>(coef + 16);                       // 16: D(v_b)^{-1}
  float* rdiag = vf + 16;                                                // 16
  int* fail = reinterpret_cast<int*>(rdiag + 16);                        // 4 ints (keeps 16-byte alignment)
  float2* Cs = reinterpret_cast<float2*>(fail + 4);                      // s x N
  const int slot = blockIdx.x;
  if (slot >= *count) return;
  const int b = list[slot];
  const int N = n * k;
  const int LDC = N + 1;  // padded row of C in shared memory
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid < k) vf[tid] = (float)vinv[(size_t)b * k + tid];
  if (tid == 0) fail[0] = 0;
  __syncthreads();
  // C = Ut D(v)^{-1} - C0 Ut = T(v) Ut
  for (int e = tid; e < N; e += RS_T) {
    const float vi = vf[e / n];
    for (int c = 0; c < s; ++c) {
      const float2 u = Ut[(size_t)c * N + e], cu = C0Ut[(size_t)c * N + e];
      Cs[(size_t)c * LDC + e] = make_float2(u.x * vi - cu.x, u.y * vi - cu.y);
    }
  }
  __syncthreads();
  const int npair = s * (s + 1) / 2;
  int Q = 1;
  while (Q < 32 && npair * Q * 2 <= RS_T) Q *= 2;
  for (int pass = 0; pass < 2; ++pass) {
    // Gram G = C^H C (upper pairs i <= j, Q threads per pair over a strided
    // share of the elements)
    {
      const int p = tid / Q, q = tid % Q;
      float2 acc = make_float2(0.f, 0.f);
      int i = 0, j = 0;
      if (p < npair) {
        int rem = p;
        while (rem >= s - i) {
          rem -= s - i;
          ++i;
        }
        j = i + rem;
        const float2* ci = Cs + (size_t)i * LDC;
        const float2* cj = Cs + (size_t)j * LDC;
        for (int e = q; e < N; e += Q) acc = cadd(acc, cjmul(ci[e], cj[e]));
      }
      for (int o = Q / 2; o > 0; o >>= 1) {
        acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
        acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
      }
      if (p < npair && q == 0) {  // G[i][j] = sum conj(C_i) C_j (column-major, ld 16); Hermitian
        if (i == j) acc.y = 0.f;
        Gf[i + j * 16] = acc;
        Gf[j + i * 16] = cconj(acc);
      }
    }
    __syncthreads();
    // G = L L^H, Rf = L^{-H} (the Gram's space is free once L is formed)
    if (warp == 0) {
      const int bad = chol16_warp(s, Gf, Lf, rdiag);
      linvh16_warp(s, Lf, rdiag, Gf, Rf);
      if (bad && lane == 0) fail[0] = 1;
    }
    __syncthreads();
    if (fail[0]) {
      if (tid == 0) ok[b] = 0;
      return;
    }
    // Ra := Rf (first pass) or Ra Rf (second); both upper triangular
    float2 ra = make_float2(0.f, 0.f);
    if (tid < 256) {
      const int ri = tid & 15, rj = tid >> 4;
      if (pass == 0) {
        ra = Rf[tid];
      } else {
#pragma unroll
        for (int p = 0; p < 16; ++p) ra = cfma(Raf[ri + p * 16], Rf[p + rj * 16], ra);
      }
    }
    // C := C Rf, element by element (all s values of an element in registers)
    for (int e = tid; e < N; e += RS_T) {
      float2 v[16];
#pragma unroll
      for (int c = 0; c < 16; ++c) v[c] = c < s ? Cs[(size_t)c * LDC + e] : make_float2(0.f, 0.f);
#pragma unroll
      for (int jj = 0; jj < 16; ++jj) {
        if (jj < s) {
          float2 o = make_float2(0.f, 0.f);
#pragma unroll
          for (int c = 0; c < 16; ++c)
            if (c <= jj) o = cfma(v[c], Rf[c + jj * 16], o);  // Rf is upper triangular
          Cs[(size_t)jj * LDC + e] = o;
        }
      }
    }
    __syncthreads();
    if (tid < 256) Raf[tid] = ra;
  }
  // write C; coef = C^H r
  float acc[32];
#pragma unroll
  for (int u = 0; u < 32; ++u) acc[u] = 0.f;
  for (int e = tid; e < N; e += RS_T) {
    const float2 re = R[(size_t)b * N + e];
#pragma unroll
    for (int c = 0; c < 16; ++c) {
      if (c < s) {
        const float2 ce = Cs[(size_t)c * LDC + e];
        C[(size_t)b * ss + (size_t)c * N + e] = ce;
        acc[2 * c] += ce.x * re.x + ce.y * re.y;
        acc[2 * c + 1] += ce.x * re.y - ce.y * re.x;
      }
    }
  }
  warp_reduce_scatter32<float>(acc);
  red[warp * 32 + lane] = acc[0];
  __syncthreads();
  if (tid < 32) {
    float v = 0.f;
#pragma unroll
    for (int w = 0; w < RS_T / 32; ++w) v += red[w * 32 + tid];
    const float im = __shfl_xor_sync(0xffffffffu, v, 1);
    if ((tid & 1) == 0 && (tid >> 1) < s) coef[tid >> 1] = make_float2(v, im);
  }
  __syncthreads();
  // U = Ut Ra;  x += U coef;  r -= C coef
  for (int e = tid; e < N; e += RS_T) {
    float2 ut[16];
#pragma unroll
    for (int c = 0; c < 16; ++c) ut[c] = c < s ? Ut[(size_t)c * N + e] : make_float2(0.f, 0.f);
    float2 xs = X[(size_t)b * N + e], rs = R[(size_t)b * N + e];
#pragma unroll
    for (int jj = 0; jj < 16; ++jj) {
      if (jj < s) {
        float2 uj = make_float2(0.f, 0.f);
#pragma unroll
        for (int c = 0; c < 16; ++c)
          if (c <= jj) uj = cfma(ut[c], Raf[c + jj * 16], uj);  // Ra is upper triangular
        U[(size_t)b * ss + (size_t)jj * N + e] = uj;
        xs = cfma(uj, coef[jj], xs);
        rs = csub(rs, cmul(Cs[(size_t)jj * LDC + e], coef[jj]));
      }
    }
    X[(size_t)b * N + e] = xs;
    R[(size_t)b * N + e] = rs;
  }
  if (tid == 0) ok[b] = 1;
}

size_t recstart32_smem_bytes(int s, int N) {
  return sizeof(float2) * 4 * 256 + sizeof(float) * (RS_T / 32) * 32 + sizeof(float2) * 16 + sizeof(float) * 32 +
         sizeof(int) * 4 + sizeof(float2) * (size_t)s * (N + 1);
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
