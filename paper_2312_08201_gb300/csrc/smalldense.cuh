// Small dense complex FP64 routines run by one warp per system (matrices of
// order <= ~64 in global memory, column-major). Used by the recycled Krylov
// solver for the harmonic-Ritz recycle update (GCRO-DR, paper §2.1: keep the
// s approximate eigenvectors with eigenvalues of smallest magnitude).
//
// Every lane computes the same scalar control values from memory that all
// lanes can see, so lanes agree on branches without extra communication;
// vector loops are split over lanes and separated by __syncwarp().
#pragma once
#include "cplx.cuh"

namespace sd {

__device__ __forceinline__ int lane() { return threadIdx.x & 31; }
__device__ __forceinline__ void wsync() { __syncwarp(); }
__device__ __forceinline__ double cabs_(double2 z) { return sqrt(cabs2(z)); }
__device__ __forceinline__ float cabs_(float2 z) { return sqrtf(cabs2(z)); }
template <typename T2>
__device__ __forceinline__ T2 zero2() {
  T2 z;
  z.x = 0;
  z.y = 0;
  return z;
}
template <typename T2>
__device__ __forceinline__ T2 re2(typename RealOf<T2>::T x) {
  T2 z;
  z.x = x;
  z.y = 0;
  return z;
}
template <typename R>
__device__ __forceinline__ R eps_of();
template <>
__device__ __forceinline__ double eps_of<double>() {
  return 2.220446049250313e-16;
}
template <>
__device__ __forceinline__ float eps_of<float>() {
  return 1.1920929e-7f;
}

// C (m x n) = A^H B, A: K x m (lda), B: K x n (ldb)
__device__ inline void gemm_hn(int m, int n, int K, const double2* A, int lda, const double2* B, int ldb,
                               double2* C, int ldc) {
  for (int e = lane(); e < m * n; e += 32) {
    int i = e % m, j = e / m;
    double2 acc = mk(0.0, 0.0);
    for (int l = 0; l < K; ++l) acc = cadd(acc, cjmul(A[l + (size_t)i * lda], B[l + (size_t)j * ldb]));
    C[i + (size_t)j * ldc] = acc;
  }
  wsync();
}

// C (m x n) = A B, A: m x K, B: K x n
__device__ inline void gemm_nn(int m, int n, int K, const double2* A, int lda, const double2* B, int ldb,
                               double2* C, int ldc) {
  for (int e = lane(); e < m * n; e += 32) {
    int i = e % m, j = e / m;
    double2 acc = mk(0.0, 0.0);
    for (int l = 0; l < K; ++l) acc = cfma(A[i + (size_t)l * lda], B[l + (size_t)j * ldb], acc);
    C[i + (size_t)j * ldc] = acc;
  }
  wsync();
}

// In-place lower Cholesky of a Hermitian positive definite matrix.
// Returns 0 on success, 1 if a pivot is not positive.
__device__ inline int cholesky(int m, double2* A, int lda) {
  for (int j = 0; j < m; ++j) {
    double d = A[j + (size_t)j * lda].x;
    for (int p = 0; p < j; ++p) d -= cabs2(A[j + (size_t)p * lda]);
    if (!(d > 0.0) || !isfinite(d)) return 1;
    d = sqrt(d);
    wsync();
    for (int i = j + 1 + lane(); i < m; i += 32) {
      double2 x = A[i + (size_t)j * lda];
      for (int p = 0; p < j; ++p) x = csub(x, cmul(A[i + (size_t)p * lda], cconj(A[j + (size_t)p * lda])));
      A[i + (size_t)j * lda] = cscale(x, 1.0 / d);
    }
    wsync();
    if (lane() == 0) A[j + (size_t)j * lda] = mk(d, 0.0);
    wsync();
  }
  for (int e = lane(); e < m * m; e += 32) {
    int i = e % m, j = e / m;
    if (i < j) A[i + (size_t)j * lda] = mk(0.0, 0.0);
  }
  wsync();
  return 0;
}

// B := L^{-1} B (L lower m x m, B m x n); lanes over columns
__device__ inline void trsm_lower_left(int m, int n, const double2* L, int ldl, double2* B, int ldb) {
  for (int c = lane(); c < n; c += 32) {
    for (int i = 0; i < m; ++i) {
      double2 x = B[i + (size_t)c * ldb];
      for (int p = 0; p < i; ++p) x = csub(x, cmul(L[i + (size_t)p * ldl], B[p + (size_t)c * ldb]));
      B[i + (size_t)c * ldb] = cdiv(x, L[i + (size_t)i * ldl]);
    }
  }
  wsync();
}

// B := B L^{-H} (B r x m): row x solves x L^H = b, i.e. L conj(x) = conj(b)
__device__ inline void trsm_right_lower_h(int r, int m, const double2* L, int ldl, double2* B, int ldb) {
  for (int row = lane(); row < r; row += 32) {
    for (int i = 0; i < m; ++i) {
      double2 x = cconj(B[row + (size_t)i * ldb]);
      for (int p = 0; p < i; ++p) x = csub(x, cmul(L[i + (size_t)p * ldl], cconj(B[row + (size_t)p * ldb])));
      B[row + (size_t)i * ldb] = cconj(cdiv(x, L[i + (size_t)i * ldl]));
    }
  }
  wsync();
}

// X := L^{-H} X (X m x n): solve L^H y = x by backward substitution; lanes over columns
__device__ inline void trsm_lower_h_left(int m, int n, const double2* L, int ldl, double2* X, int ldx) {
  for (int c = lane(); c < n; c += 32) {
    for (int i = m - 1; i >= 0; --i) {
      double2 x = X[i + (size_t)c * ldx];
      for (int p = i + 1; p < m; ++p) x = csub(x, cmul(cconj(L[p + (size_t)i * ldl]), X[p + (size_t)c * ldx]));
      X[i + (size_t)c * ldx] = cdiv(x, cconj(L[i + (size_t)i * ldl]));
    }
  }
  wsync();
}

// Householder reduction to upper Hessenberg form, A := Q^H A Q, Q accumulated
// (Q initialised to I here). v: scratch of length m.
template <typename T2>
__device__ inline void hessenberg(int m, T2* A, int lda, T2* Q, int ldq, T2* v) {
  using R = typename RealOf<T2>::T;
  for (int e = lane(); e < m * m; e += 32) {
    int i = e % m, j = e / m;
    Q[i + (size_t)j * ldq] = re2<T2>(i == j ? R(1) : R(0));
  }
  wsync();
  for (int c = 0; c + 2 < m; ++c) {
    const int len = m - c - 1;
    R xn2 = 0;
    for (int i = 0; i < len; ++i) xn2 += cabs2(A[c + 1 + i + (size_t)c * lda]);
    T2 x0 = A[c + 1 + (size_t)c * lda];
    R alpha = sqrt(xn2);
    R ax0 = cabs_(x0);
    if (alpha == R(0) || xn2 - ax0 * ax0 <= xn2 * eps_of<R>() * eps_of<R>()) {
      wsync();
      continue;  // already in Hessenberg form in this column
    }
    T2 ph = ax0 > R(0) ? cscale(x0, R(1) / ax0) : re2<T2>(R(1));
    T2 v0 = cadd(x0, cscale(ph, alpha));
    R vn2 = xn2 - ax0 * ax0 + cabs2(v0);
    R beta = R(2) / vn2;
    wsync();
    for (int i = lane(); i < len; i += 32) v[i] = i == 0 ? v0 : A[c + 1 + i + (size_t)c * lda];
    wsync();
    // left: A[c+1:, j] -= beta v (v^H A[c+1:, j]) for j >= c
    for (int j = c + lane(); j < m; j += 32) {
      T2 s = zero2<T2>();
      for (int i = 0; i < len; ++i) s = cadd(s, cjmul(v[i], A[c + 1 + i + (size_t)j * lda]));
      s = cscale(s, beta);
      for (int i = 0; i < len; ++i) A[c + 1 + i + (size_t)j * lda] = csub(A[c + 1 + i + (size_t)j * lda], cmul(v[i], s));
    }
    wsync();
    // right: A[i, c+1:] -= beta (A[i, c+1:] v) v^H for all i; same for Q
    for (int i = lane(); i < m; i += 32) {
      T2 s = zero2<T2>(), sq = zero2<T2>();
      for (int l = 0; l < len; ++l) {
        s = cfma(A[i + (size_t)(c + 1 + l) * lda], v[l], s);
        sq = cfma(Q[i + (size_t)(c + 1 + l) * ldq], v[l], sq);
      }
      s = cscale(s, beta);
      sq = cscale(sq, beta);
      for (int l = 0; l < len; ++l) {
        A[i + (size_t)(c + 1 + l) * lda] = csub(A[i + (size_t)(c + 1 + l) * lda], cmul(s, cconj(v[l])));
        Q[i + (size_t)(c + 1 + l) * ldq] = csub(Q[i + (size_t)(c + 1 + l) * ldq], cmul(sq, cconj(v[l])));
      }
    }
    wsync();
    for (int i = c + 2 + lane(); i < m; i += 32) A[i + (size_t)c * lda] = zero2<T2>();
    wsync();
  }
}

// Givens rotation G = [[c, s], [-conj(s), c]] with G [x; y] = [rho; 0].
template <typename T2, typename R>
__device__ inline void givens(T2 x, T2 y, R& c, T2& s) {
  R ax = cabs_(x), ay = cabs_(y);
  if (ay == R(0)) {
    c = R(1);
    s = zero2<T2>();
  } else if (ax == R(0)) {
    c = R(0);
    s = re2<T2>(R(1));
  } else {
    R r = sqrt(ax * ax + ay * ay);
    T2 al = cscale(x, R(1) / ax);
    c = ax / r;
    s = cscale(cjmul(y, al), R(1) / r);  // al * conj(y) / r
  }
}

// Complex single-shift QR iteration on an upper Hessenberg matrix H
// (Wilkinson shift, exceptional shift every 10 iterations, deflation on
// negligible subdiagonals), accumulating Q. On return H is upper triangular
// (Schur form) and A_original = Q H Q^H. Returns 0 on success.
template <typename T2>
__device__ inline int hqr(int m, T2* H, int ldh, T2* Q, int ldq, int maxit) {
  using R = typename RealOf<T2>::T;
  const R eps = eps_of<R>();
  int hi = m - 1, its = 0, total = 0;
  while (hi > 0) {
    int l = hi;
    while (l > 0) {
      R sc = cabs_(H[l - 1 + (size_t)(l - 1) * ldh]) + cabs_(H[l + (size_t)l * ldh]);
      if (sc == R(0)) sc = R(1e-30);
      if (cabs_(H[l + (size_t)(l - 1) * ldh]) <= eps * sc) break;
      --l;
    }
    if (l == hi) {
      wsync();
      if (lane() == 0) H[hi + (size_t)(hi - 1) * ldh] = zero2<T2>();
      wsync();
      --hi;
      its = 0;
      continue;
    }
    if (++total > maxit) return 1;
    ++its;
    T2 mu;
    T2 d = H[hi + (size_t)hi * ldh];
    if (its % 10 == 0) {
      mu = cadd(d, re2<T2>(cabs_(H[hi + (size_t)(hi - 1) * ldh])));
    } else {
      T2 a = H[hi - 1 + (size_t)(hi - 1) * ldh], b = H[hi - 1 + (size_t)hi * ldh];
      T2 c = H[hi + (size_t)(hi - 1) * ldh];
      T2 half = cscale(csub(a, d), R(0.5));
      T2 disc2 = cadd(cmul(half, half), cmul(b, c));
      // principal complex square root
      R r = cabs_(disc2);
      R sr = sqrt(R(0.5) * (r + disc2.x));
      R si = sqrt(fmax(R(0), R(0.5) * (r - disc2.x)));
      if (disc2.y < 0) si = -si;
      T2 disc;
      disc.x = sr;
      disc.y = si;
      T2 tr2 = cscale(cadd(a, d), R(0.5));
      T2 m1 = cadd(tr2, disc), m2 = csub(tr2, disc);
      mu = cabs2(csub(m1, d)) <= cabs2(csub(m2, d)) ? m1 : m2;
    }
    T2 x = csub(H[l + (size_t)l * ldh], mu);
    T2 y = H[l + 1 + (size_t)l * ldh];
    for (int kk = l; kk < hi; ++kk) {
      if (kk > l) {
        x = H[kk + (size_t)(kk - 1) * ldh];
        y = H[kk + 1 + (size_t)(kk - 1) * ldh];
      }
      R c;
      T2 s;
      givens(x, y, c, s);
      wsync();
      int j0 = kk > l ? kk - 1 : kk;
      for (int j = j0 + lane(); j < m; j += 32) {
        T2 top = H[kk + (size_t)j * ldh], bot = H[kk + 1 + (size_t)j * ldh];
        H[kk + (size_t)j * ldh] = cadd(cscale(top, c), cmul(s, bot));
        // the rotation annihilates the bulge H[kk+1, kk-1]: store the exact zero
        H[kk + 1 + (size_t)j * ldh] = (kk > l && j == kk - 1) ? zero2<T2>() : csub(cscale(bot, c), cjmul(s, top));
      }
      wsync();
      int imax = kk + 2 < hi ? kk + 2 : hi;
      for (int i = lane(); i < m; i += 32) {
        if (i <= imax) {
          T2 lft = H[i + (size_t)kk * ldh], rgt = H[i + (size_t)(kk + 1) * ldh];
          H[i + (size_t)kk * ldh] = cadd(cscale(lft, c), cmul(cconj(s), rgt));
          H[i + (size_t)(kk + 1) * ldh] = csub(cscale(rgt, c), cmul(s, lft));
        }
        T2 lft = Q[i + (size_t)kk * ldq], rgt = Q[i + (size_t)(kk + 1) * ldq];
        Q[i + (size_t)kk * ldq] = cadd(cscale(lft, c), cmul(cconj(s), rgt));
        Q[i + (size_t)(kk + 1) * ldq] = csub(cscale(rgt, c), cmul(s, lft));
      }
      wsync();
    }
  }
  return 0;
}

// Eigenvectors of the triangular Schur form T for the selected indices,
// back-transformed by Q: X[:, c] = Q y_c with (T - T_qq I) y_c = 0,
// y_c[q] = 1, normalised to unit 2-norm. One lane per selected vector.
template <typename T2>
__device__ inline void schur_vectors(int m, const T2* T, int ldt, const T2* Q, int ldq, const int* sel, int ns, T2* Y,
                                     int ldy, T2* X, int ldx) {
  using R = typename RealOf<T2>::T;
  for (int c = lane(); c < ns; c += 32) {
    int q = sel[c];
    T2 mu = T[q + (size_t)q * ldt];
    T2* y = Y + (size_t)c * ldy;
    for (int i = 0; i < m; ++i) y[i] = zero2<T2>();
    y[q] = re2<T2>(R(1));
    R tnorm = 0;
    for (int i = 0; i <= q; ++i) tnorm = fmax(tnorm, cabs_(T[i + (size_t)i * ldt]));
    R floor_d = R(64) * eps_of<R>() * (tnorm > R(0) ? tnorm : R(1));
    for (int i = q - 1; i >= 0; --i) {
      T2 sum = zero2<T2>();
      for (int j = i + 1; j <= q; ++j) sum = cfma(T[i + (size_t)j * ldt], y[j], sum);
      T2 den = csub(T[i + (size_t)i * ldt], mu);
      if (cabs_(den) < floor_d) den = re2<T2>(floor_d);
      y[i] = cscale(cdiv(sum, den), R(-1));
      if (!(cabs2(y[i]) < R(1e30))) y[i] = zero2<T2>();
    }
  }
  wsync();
  for (int e = lane(); e < m * ns; e += 32) {
    int r = e % m, c = e / m;
    int q = sel[c];
    T2 acc = zero2<T2>();
    for (int i = 0; i <= q; ++i) acc = cfma(Q[r + (size_t)i * ldq], Y[i + (size_t)c * ldy], acc);
    X[r + (size_t)c * ldx] = acc;
  }
  wsync();
  for (int c = lane(); c < ns; c += 32) {
    R nrm = 0;
    for (int r = 0; r < m; ++r) nrm += cabs2(X[r + (size_t)c * ldx]);
    nrm = nrm > R(0) ? R(1) / sqrt(nrm) : R(1);
    for (int r = 0; r < m; ++r) X[r + (size_t)c * ldx] = cscale(X[r + (size_t)c * ldx], nrm);
  }
  wsync();
}

// Householder QR of G (r x c, r >= c) in place; the reflectors are also
// applied to F (r x nf): on return the upper triangle of G holds R and the
// first c rows of F hold Q^H F. v: scratch of length r.
template <typename T2>
__device__ inline void householder_qr_apply(int r, int c, T2* G, int ldg, T2* F, int ldf, int nf, T2* v) {
  using R = typename RealOf<T2>::T;
  for (int k = 0; k < c; ++k) {
    const int len = r - k;
    R xn2 = 0;
    for (int i = 0; i < len; ++i) xn2 += cabs2(G[k + i + (size_t)k * ldg]);
    const T2 x0 = G[k + (size_t)k * ldg];
    const R alpha = sqrt(xn2);
    const R ax0 = cabs_(x0);
    wsync();
    if (!(alpha > R(0))) continue;
    const T2 ph = ax0 > R(0) ? cscale(x0, R(1) / ax0) : re2<T2>(R(1));
    const T2 v0 = cadd(x0, cscale(ph, alpha));
    const R vn2 = xn2 - ax0 * ax0 + cabs2(v0);
    const R beta = R(2) / vn2;
    for (int i = lane(); i < len; i += 32) v[i] = i == 0 ? v0 : G[k + i + (size_t)k * ldg];
    wsync();
    for (int j = k + lane(); j < c + nf; j += 32) {
      T2* col = j < c ? G + (size_t)j * ldg : F + (size_t)(j - c) * ldf;
      T2 s = zero2<T2>();
      for (int i = 0; i < len; ++i) s = cadd(s, cjmul(v[i], col[k + i]));
      s = cscale(s, beta);
      for (int i = 0; i < len; ++i) col[k + i] = csub(col[k + i], cmul(v[i], s));
    }
    wsync();
  }
}

// X := R^{-1} X (R upper c x c, X c x n); lanes over columns
template <typename T2>
__device__ inline void trsm_upper_left(int c, int n, const T2* Rm, int ldr, T2* X, int ldx) {
  for (int j = lane(); j < n; j += 32) {
    for (int i = c - 1; i >= 0; --i) {
      T2 x = X[i + (size_t)j * ldx];
      for (int l = i + 1; l < c; ++l) x = csub(x, cmul(Rm[i + (size_t)l * ldr], X[l + (size_t)j * ldx]));
      X[i + (size_t)j * ldx] = cdiv(x, Rm[i + (size_t)i * ldr]);
    }
  }
  wsync();
}

// Thin QR by classical Gram-Schmidt with one re-orthogonalisation:
// A (r x n) -> Qm (r x n, orthonormal columns), R (n x n upper).
// Returns 0 on success, 1 if a column is numerically dependent.
__device__ inline int qr_cgs2(int r, int n, const double2* A, int lda, double2* Qm, int ldq, double2* R, int ldr,
                              double2* coef) {
  for (int e = lane(); e < n * n; e += 32) R[(e % n) + (size_t)(e / n) * ldr] = mk(0.0, 0.0);
  wsync();
  for (int j = 0; j < n; ++j) {
    for (int i = lane(); i < r; i += 32) Qm[i + (size_t)j * ldq] = A[i + (size_t)j * lda];
    wsync();
    for (int pass = 0; pass < 2; ++pass) {
      for (int q = lane(); q < j; q += 32) {
        double2 acc = mk(0.0, 0.0);
        for (int i = 0; i < r; ++i) acc = cadd(acc, cjmul(Qm[i + (size_t)q * ldq], Qm[i + (size_t)j * ldq]));
        coef[q] = acc;
      }
      wsync();
      for (int i = lane(); i < r; i += 32) {
        double2 x = Qm[i + (size_t)j * ldq];
        for (int q = 0; q < j; ++q) x = csub(x, cmul(Qm[i + (size_t)q * ldq], coef[q]));
        Qm[i + (size_t)j * ldq] = x;
      }
      for (int q = lane(); q < j; q += 32) R[q + (size_t)j * ldr] = cadd(R[q + (size_t)j * ldr], coef[q]);
      wsync();
    }
    double nrm = 0.0, anrm = 0.0;
    for (int i = 0; i < r; ++i) {
      nrm += cabs2(Qm[i + (size_t)j * ldq]);
      anrm += cabs2(A[i + (size_t)j * lda]);
    }
    nrm = sqrt(nrm);
    if (!(nrm > 1e-13 * sqrt(anrm)) || !isfinite(nrm)) return 1;
    wsync();
    for (int i = lane(); i < r; i += 32) Qm[i + (size_t)j * ldq] = cscale(Qm[i + (size_t)j * ldq], 1.0 / nrm);
    if (lane() == 0) R[j + (size_t)j * ldr] = mk(nrm, 0.0);
    wsync();
  }
  return 0;
}

// X := X R^{-1} (X r x n, R n x n upper): row x solves x R = b
__device__ inline void trsm_right_upper(int r, int n, const double2* R, int ldr, double2* X, int ldx) {
  for (int row = lane(); row < r; row += 32) {
    for (int j = 0; j < n; ++j) {
      double2 x = X[row + (size_t)j * ldx];
      for (int i = 0; i < j; ++i) x = csub(x, cmul(X[row + (size_t)i * ldx], R[i + (size_t)j * ldr]));
      X[row + (size_t)j * ldx] = cdiv(x, R[j + (size_t)j * ldr]);
    }
  }
  wsync();
}

}  // namespace sd
