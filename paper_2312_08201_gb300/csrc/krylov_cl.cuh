// CGS2 orthogonalisation of the Arnoldi step with the basis staged in
// shared memory across a thread-block cluster (the GCRO-DR step of paper
// §2.1, same arithmetic as kry::k_ortho).
//
// One cluster of C CTAs serves one system; CTA r owns the element slice
// [r L, min((r+1) L, N)) of every vector. Its thread 0 issues one bulk copy
// (cp.async.bulk, completion counted on an mbarrier) per basis vector and
// one for w, so the whole slice of the basis is read from memory once per
// step; both Gram-Schmidt passes, the norm and the scaling then run from
// shared memory. The partial inner products of the CTAs meet through
// distributed shared memory, summed in rank order by every CTA, so all CTAs
// apply identical coefficients and the result does not depend on timing.
// CTA 0 writes the new column of H (and Bk) and runs the Givens update.
//
// Every wait is bounded; on expiry the CTA sets *err, still takes part in
// every cluster barrier, waits (bounded) for its copies in flight and
// returns, so no CTA of the cluster is left waiting.
#pragma once
#include <cooperative_groups.h>

#include "krylov.cuh"
#include "tcgen05_util.cuh"

namespace kry {

constexpr int OCT = 256;          // threads per CTA of k_ortho_cl
// Norm of the orthogonalised vector from the second pass's coefficients:
// ||w2||^2 = ||w1||^2 - ||h2||^2 (w1 - w2 = V h2 with V orthonormal), with
// ||w1||^2 reduced together with the second pass's inner products, so the
// step needs two cluster reductions instead of three.
constexpr bool kFoldNorm = true;
constexpr int OCL_MAXNB = 64;     // basis vectors (s_cur + j + 1 <= m + 1 <= 61)
constexpr int OCL_MAXC = 16;      // CTAs per cluster (the launcher's largest tier)

__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}

// Dynamic shared memory of k_ortho_cl: the mbarrier, three sets of partial
// sums and two coefficient vectors, then (nb + 1) slices of L elements.
template <typename T2>
__host__ __device__ constexpr size_t ortho_cl_header() {
  return ((16 + 3 * 2 * OCL_MAXNB * sizeof(typename RealOf<T2>::T) + 2 * OCL_MAXNB * sizeof(T2)) + 127) / 128 * 128;
}
template <typename T2>
__host__ __device__ constexpr size_t ortho_cl_smem(int nb, int L) {
  return ortho_cl_header<T2>() + (size_t)(nb + 1) * L * sizeof(T2);
}

template <typename T2>
__global__ void __launch_bounds__(OCT) k_ortho_cl(int N, int L, int j, int m, int s_cur,
                                                 const int* __restrict__ list, const int* __restrict__ count,
                                                 T2* __restrict__ V, const T2* __restrict__ C, size_t c_ss,
                                                 double2* __restrict__ H, double2* __restrict__ Bk, int smax,
                                                 LsqArgs Ls, int* __restrict__ err) {
  using R = typename RealOf<T2>::T;
  namespace cg = cooperative_groups;
  constexpr int NW = OCT / 32;
  extern __shared__ __align__(128) unsigned char osm[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(osm);             // [0, 8)
  R* part = reinterpret_cast<R*>(osm + 16);                      // 3 x 2 x OCL_MAXNB partial sums
  T2* coef = reinterpret_cast<T2*>(osm + 16 + 3 * 2 * OCL_MAXNB * sizeof(R));  // 2 x OCL_MAXNB
  T2* data = reinterpret_cast<T2*>(osm + ortho_cl_header<T2>());  // (nb + 1) slices of L elements
  using C2 = typename Cplx<R>::T;
  __shared__ C2 hr[66];   // column j of H in the vectors' precision (rank 0)
  __shared__ R csr[64];   // previous rotations
  __shared__ C2 snr[64];
  __shared__ R red[NW];
  __shared__ int failed;

  cg::cluster_group cl = cg::this_cluster();
  const int ncta = (int)cl.num_blocks();
  const int rank = (int)cl.block_rank();
  const int slot = blockIdx.x / ncta;
  if (slot >= *count) return;  // uniform over the cluster
  const int b = list[slot];
  const int nb = s_cur + j + 1;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int e0 = rank * L;
  const int len = max(0, min(L, N - e0));
  T2* Vb = V + (size_t)b * (m + 1) * N;
  T2* w = Vb + (size_t)(j + 1) * N;
  const T2* Cb = C + (size_t)b * c_ss;
  auto gbasis = [&](int q) -> const T2* { return q < s_cur ? Cb + (size_t)q * N : Vb + (size_t)(q - s_cur) * N; };
  T2* sw = data + (size_t)nb * L;
  const uint32_t mb = tcu::sm_addr(bar);

  if (tid == 0) {
    failed = 0;
    tcu::mbar_init(mb, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (tid == 0 && len > 0) {
    const uint32_t bytes = (uint32_t)(len * sizeof(T2));
    tcu::mbar_expect_tx(mb, bytes * (uint32_t)(nb + 1));
    for (int q = 0; q < nb; ++q) bulk_g2s(tcu::sm_addr(data + (size_t)q * L), gbasis(q) + e0, bytes, mb);
    bulk_g2s(tcu::sm_addr(sw), w + e0, bytes, mb);
  }
  if (len > 0 && !tcu::mbar_wait(mb, 0)) {
    if (lane == 0) failed = 1;
  }
  __syncthreads();
  const bool ok = failed == 0;
  if (!ok && tid == 0) atomicExch(err, 21);

  // partial inner products conj(basis_q) . x over this CTA's slice, one warp per vector
  // Two basis vectors per warp and pass over x (x is read once for both);
  // two independent accumulators per product, so the loads overlap.
  auto partial_dots = [&](const T2* x, R* out) {
    for (int q = warp; q < nb; q += 2 * NW) {
      const int q2 = q + NW < nb ? q + NW : q;  // a lone last vector is paired with itself
      R ax = R(0), ay = R(0), cx = R(0), cy = R(0);
      if (ok) {
        const T2* va = data + (size_t)q * L;
        const T2* vb = data + (size_t)q2 * L;
        R p[8] = {R(0), R(0), R(0), R(0), R(0), R(0), R(0), R(0)};
        int e = lane;
        for (; e + 32 < len; e += 64) {
#pragma unroll
          for (int u = 0; u < 2; ++u) {
            const T2 c = x[e + 32 * u], a = va[e + 32 * u], d = vb[e + 32 * u];
            p[4 * u + 0] += a.x * c.x + a.y * c.y;
            p[4 * u + 1] += a.x * c.y - a.y * c.x;
            p[4 * u + 2] += d.x * c.x + d.y * c.y;
            p[4 * u + 3] += d.x * c.y - d.y * c.x;
          }
        }
        if (e < len) {
          const T2 c = x[e], a = va[e], d = vb[e];
          p[0] += a.x * c.x + a.y * c.y;
          p[1] += a.x * c.y - a.y * c.x;
          p[2] += d.x * c.x + d.y * c.y;
          p[3] += d.x * c.y - d.y * c.x;
        }
        ax = p[0] + p[4];
        ay = p[1] + p[5];
        cx = p[2] + p[6];
        cy = p[3] + p[7];
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        ax += __shfl_xor_sync(0xffffffffu, ax, o);
        ay += __shfl_xor_sync(0xffffffffu, ay, o);
        cx += __shfl_xor_sync(0xffffffffu, cx, o);
        cy += __shfl_xor_sync(0xffffffffu, cy, o);
      }
      if (lane == 0) {
        out[2 * q] = ax;
        out[2 * q + 1] = ay;
        if (q2 != q) {
          out[2 * q2] = cx;
          out[2 * q2 + 1] = cy;
        }
      }
    }
  };
  // coefficients: the cluster's partial sums added in rank order; the remote
  // loads are all issued before the first add (ranks past ncta add zero)
  auto gather = [&](R* in, T2* cf, int extra) {
    cl.sync();
    if (tid < 2 * nb + extra) {
      R v[OCL_MAXC];
#pragma unroll
      for (int r = 0; r < OCL_MAXC; ++r) v[r] = r < ncta ? cl.map_shared_rank(in, r)[tid] : R(0);
      R s = R(0);
#pragma unroll
      for (int r = 0; r < OCL_MAXC; ++r) s += v[r];
      reinterpret_cast<R*>(cf)[tid] = s;
    }
    __syncthreads();
  };
  // x -= sum_q basis_q coef_q over the slice; returns this thread's sum of |x|^2
  auto update = [&](const T2* cf) -> R {
    R nr = R(0);
    if (!ok) return nr;
    for (int e = tid; e < len; e += OCT) {
      // two partial sums over the basis, so consecutive loads are independent
      T2 s0 = sw[e], s1 = T2{R(0), R(0)};
      int q = 0;
      for (; q + 1 < nb; q += 2) {
        s0 = csub(s0, cmul(data[(size_t)q * L + e], cf[q]));
        s1 = csub(s1, cmul(data[(size_t)(q + 1) * L + e], cf[q + 1]));
      }
      if (q < nb) s0 = csub(s0, cmul(data[(size_t)q * L + e], cf[q]));
      const T2 we = cadd(s0, s1);
      sw[e] = we;
      nr += cabs2(we);
    }
    return nr;
  };

  auto block_total = [&](R x) -> R {  // sum over the CTA, on thread 0
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if (lane == 0) red[warp] = x;
    __syncthreads();
    R t = R(0);
    if (tid == 0)
      for (int w2 = 0; w2 < NW; ++w2) t += red[w2];
    return t;
  };
  // pass 1
  partial_dots(sw, part);
  gather(part, coef, 0);
  const R n1 = update(coef);
  __syncthreads();
  R tot = R(0);
  if (kFoldNorm) {
    // pass 2 with ||w1||^2 in the same reduction
    R* p2 = part + 2 * OCL_MAXNB;
    const R t1 = block_total(n1);
    if (tid == 0) p2[2 * nb] = t1;
    partial_dots(sw, p2);
    gather(p2, coef + OCL_MAXNB, 1);
    update(coef + OCL_MAXNB);
    const R* c2 = reinterpret_cast<const R*>(coef + OCL_MAXNB);
    tot = c2[2 * nb];
    for (int q = 0; q < 2 * nb; ++q) tot -= c2[q] * c2[q];
    tot = tot > R(0) ? tot : R(0);
  } else {
    // pass 2
    partial_dots(sw, part + 2 * OCL_MAXNB);
    gather(part + 2 * OCL_MAXNB, coef + OCL_MAXNB, 0);
    const R nr = update(coef + OCL_MAXNB);
    // norm of the orthogonalised w
    R* pn = part + 4 * OCL_MAXNB;
    const R t2 = block_total(nr);
    if (tid == 0) pn[0] = t2;
    cl.sync();
    for (int r = 0; r < ncta; ++r) tot += cl.map_shared_rank(pn, r)[0];
  }
  // scale and store this CTA's slice of the new basis vector
  const R rn = sqrt(tot);
  const R inv = rn > R(0) ? R(1) / rn : R(0);
  if (ok)
    for (int e = tid; e < len; e += OCT) w[e0 + e] = cscale(sw[e], inv);
  double2 gj = make_double2(0.0, 0.0);
  double tola = 0.0;
  int itd = 0;
  if (rank == 0 && ok) {
    // the column and the previous rotations, converted in parallel
    double2* H0c = Ls.H0 + (size_t)b * (m + 1) * m + (size_t)j * (m + 1);
    double2* Bc = Bk + (size_t)b * smax * m + (size_t)j * smax;
    if (tid < nb) {
      const int q = tid;
      const double2 cval = cadd(to_d2(coef[q]), to_d2(coef[OCL_MAXNB + q]));
      if (q < s_cur) {
        Bc[q] = cval;
      } else {
        H0c[q - s_cur] = cval;
        hr[q - s_cur] = C2{(R)cval.x, (R)cval.y};
      }
    }
    if (tid >= 64 && tid < 64 + j) {
      const double2 sn = Ls.sn[(size_t)b * m + tid - 64];
      csr[tid - 64] = (R)Ls.cs[(size_t)b * m + tid - 64];
      snr[tid - 64] = C2{(R)sn.x, (R)sn.y};
    }
    if (tid == 0) {
      gj = Ls.g[(size_t)b * (m + 1) + j];
      tola = Ls.tolabs[b];
      itd = Ls.iters_done[b];
      H0c[j + 1] = make_double2((double)rn, 0.0);
      hr[j + 1] = C2{rn, R(0)};
    }
    __syncthreads();
  }
  if (!ok && tid == 0 && len > 0) tcu::mbar_wait(mb, 0);  // no copy may land after the CTA has gone
  cl.sync();  // every CTA's partial sums stay readable until all have read them
  // the serial Givens update reads only rank 0's own shared memory, so the
  // other CTAs of the cluster are already free; its results are stored in
  // parallel
  if (rank == 0) {
    if (ok && tid == 0) lsq_rotate<R>(b, j, m, hr, csr, snr, gj, tola, itd, Ls);
    __syncthreads();
    if (ok && tid <= j + 1) {
      double2* hg = H + (size_t)b * (m + 1) * m + (size_t)j * (m + 1);
      hg[tid] = make_double2((double)hr[tid].x, (double)hr[tid].y);
    }
  }
}

}  // namespace kry
