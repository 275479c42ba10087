// Truncated SVD of one gate's M' inside one thread block (Eq. 9 of the paper).
//
// Route: Householder bidiagonalisation of the tall orientation of M' (the paper's
// own SVD also starts from a bidiagonal reduction), then the singular values of the
// real bidiagonal B from Sturm counts of its Golub-Kahan tridiagonal
// TGK = [[0, B], [B^T, 0]] (multisection bisection), singular vectors of B from a
// twisted factorisation of TGK - sigma I, re-orthonormalisation (block classical
// Gram-Schmidt twice with Cholesky QR inside each block of 8, in descending sigma
// order), and back-transformation by the stored Householder reflectors.
//
// Conventions: the reflector H = I - tau v v^H (v_0 = 1) satisfies H^H x = beta e_1
// with beta real. T (r x p, r >= p, column-major, leading dimension ld) is reduced
// to T = Q B P^H with Q = H_0 H_1 ... and P = G_0 G_1 ...; reflector k's tail is
// (unscaled tail stored in T) x (scale stored over its pivot), see bidiagonalize.
#pragma once
#include <cfloat>
#include "cx.cuh"

namespace mpsvqe {

template <class R>
__device__ __forceinline__ R rabs(R x) {
  return x < R(0) ? -x : x;
}
// Division inside Sturm recurrences: a correctly rounded quotient is not needed there
// (the counts and twisted factorisations tolerate a few ulps per step).
__device__ __forceinline__ float qdiv(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double qdiv(double a, double b) { return a / b; }

// LAPACK-style reflector for x = (alpha, tail) with ||tail||^2 = xn2. A vector whose
// squared norm is within 16x of the smallest normal number counts as zero: the squares
// that make up that norm have lost their bits to underflow (entries below ~5e-19 in
// FP32, ~6e-154 in FP64), so the norm could come out as 0 while alpha is not, and
// 1 / (alpha - beta) would be a division by zero. The identity is taken there and the
// entries (absolutely that small) are dropped from the bidiagonal.
template <class R>
__device__ __forceinline__ void make_reflector(Cx<R> alpha, R xn2, Cx<R>* tau, R* beta, Cx<R>* scale) {
  constexpr R kTiny2 = R(16) * (sizeof(R) == 4 ? R(FLT_MIN) : R(DBL_MIN));
  const R n2 = alpha.x * alpha.x + alpha.y * alpha.y + xn2;
  if ((xn2 == R(0) && alpha.y == R(0)) || !(n2 > kTiny2)) {
    *tau = cx<R>(0, 0);
    *beta = alpha.x;
    *scale = cx<R>(0, 0);
    return;
  }
  const R nrm = sqrt(n2);
  const R b = alpha.x >= R(0) ? -nrm : nrm;
  *beta = b;
  *tau = cx<R>((b - alpha.x) / b, -alpha.y / b);
  // scale = 1 / (alpha - beta)
  const Cx<R> den = cx<R>(alpha.x - b, alpha.y);
  const R dn = den.x * den.x + den.y * den.y;
  *scale = cx<R>(den.x / dn, -den.y / dn);
}

// Householder bidiagonalisation, NT threads, T in shared (or global) memory. dd[k]
// (diagonal) and ee[k] (superdiagonal) receive the real entries, tauL/tauR the
// reflector factors. Each step is two block-wide half steps with one barrier after
// each: every warp recomputes the reflector from the column (left) or row (right) it
// acts on, which that half step does not modify, so no single-warp section sits
// between the updates. The reflector tails stay unscaled in T (left: column k below
// the diagonal; right: row k right of the superdiagonal). Their scale factors
// 1/(alpha - beta) are written over the consumed pivots T[k][k] (left) and
// T[k+1][k] (right) one half step later, when no thread reads those entries.
// Left update: 16 lanes per column, EA entries per lane (rows k + lane + 16 e).
// Right update: G lanes per row, EB entries per lane (columns k + 1 + g + G e),
// 32 / G consecutive rows per warp. With a leading dimension of 2 (mod 16)
// complex<float> entries (G = 8) or an odd one for complex<double> (G = 16) both
// walks are free of shared-memory bank conflicts.
template <class R>
__device__ __forceinline__ R warp_sum_norm2(const Cx<R>* x, int i0, int i1, int stride) {
  R s = 0;
  for (int i = i0 + (int)(threadIdx.x & 31); i < i1; i += 32) s += norm2(x[(size_t)i * stride]);
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  return s;
}

template <class R, int NT, int EA>
__device__ __forceinline__ void bidiag_left_update(Cx<R>* T, int ld, int k, int r, int p, Cx<R> ct,
                                                   Cx<R> sc) {
  const int tid = threadIdx.x, l = tid & 15, grp = tid >> 4, wcol = (tid >> 5) << 1;
  const int nr = r - k;
  const Cx<R>* tk = T + (size_t)k * ld + k;
  Cx<R> v[EA];
#pragma unroll
  for (int e = 0; e < EA; ++e) {
    const int off = l + 16 * e;
    v[e] = off == 0 ? cx<R>(1, 0) : (off < nr ? tk[off] * sc : cx<R>(0, 0));
  }
  // the loop test is uniform over a warp (its two columns are cbase + wcol, + 1)
  for (int cbase = k + 1; cbase + wcol < p; cbase += NT / 16) {
    const int col = cbase + grp;
    const bool act = col < p;
    Cx<R>* tc = T + (size_t)(act ? col : k) * ld + k;
    Cx<R> x[EA];
    Cx<R> s = cx<R>(0, 0);
#pragma unroll
    for (int e = 0; e < EA; ++e) {
      const int off = l + 16 * e;
      x[e] = (act && off < nr) ? tc[off] : cx<R>(0, 0);
      cmac_conj(s, v[e], x[e]);
    }
#pragma unroll
    for (int o = 1; o < 16; o <<= 1) {
      s.x += __shfl_xor_sync(0xffffffffu, s.x, o, 16);
      s.y += __shfl_xor_sync(0xffffffffu, s.y, o, 16);
    }
    const Cx<R> f = ct * s;
#pragma unroll
    for (int e = 0; e < EA; ++e) {
      const int off = l + 16 * e;
      if (act && off < nr) tc[off] = x[e] - f * v[e];
    }
  }
}

template <class R, int NT, int G, int EB>
__device__ __forceinline__ void bidiag_right_update(Cx<R>* T, int ld, int k, int r, int p, Cx<R> t,
                                                    Cx<R> sc) {
  const int tid = threadIdx.x, g = tid & (G - 1), rw = tid / G, wrow = (tid >> 5) * (32 / G);
  const int nc = p - k - 1;
  Cx<R> w[EB];
#pragma unroll
  for (int e = 0; e < EB; ++e) {
    const int off = g + G * e;
    w[e] = off == 0 ? cx<R>(1, 0)
                    : (off < nc ? conj(T[(size_t)(k + 1 + off) * ld + k]) * sc : cx<R>(0, 0));
  }
  Cx<R>* t1 = T + (size_t)(k + 1) * ld;
  for (int rbase = k + 1; rbase + wrow < r; rbase += NT / G) {
    const int row = rbase + rw;
    const bool act = row < r;
    Cx<R> x[EB];
    Cx<R> s = cx<R>(0, 0);
#pragma unroll
    for (int e = 0; e < EB; ++e) {
      const int off = g + G * e;
      x[e] = (act && off < nc) ? t1[(size_t)off * ld + row] : cx<R>(0, 0);
      cmac(s, x[e], w[e]);
    }
#pragma unroll
    for (int o = 1; o < G; o <<= 1) {
      s.x += __shfl_xor_sync(0xffffffffu, s.x, o, G);
      s.y += __shfl_xor_sync(0xffffffffu, s.y, o, G);
    }
    const Cx<R> f = t * s;
#pragma unroll
    for (int e = 0; e < EB; ++e) {
      const int off = g + G * e;
      if (act && off < nc) t1[(size_t)off * ld + row] = x[e] - f * conj(w[e]);
    }
  }
}

// r <= 256 rows, p <= r columns.
template <class R, int NT>
__device__ void bidiagonalize(Cx<R>* T, int ld, int r, int p, R* dd, R* ee, Cx<R>* tauL, Cx<R>* tauR) {
  Cx<R> pend_r = cx<R>(0, 0);   // thread 0: scale of the last right reflector
  for (int k = 0; k < p; ++k) {
    // --- left half step: reflector of column k (rows k..r-1), applied to columns k+1..p-1
    Cx<R>* ck = T + (size_t)k * ld;
    Cx<R> tau, sc;
    R beta;
    make_reflector(ck[k], warp_sum_norm2(ck, k + 1, r, 1), &tau, &beta, &sc);
    if (threadIdx.x == 0) {
      dd[k] = beta;
      tauL[k] = tau;
      if (k > 0) ck[k - 1] = pend_r;   // T[k][k-1]: pivot of right reflector k-1
    }
    const Cx<R> sc_l = sc;
    if (k + 1 < p) {
      const int nr = r - k;
      const Cx<R> ct = conj(tau);
      if (nr <= 16) bidiag_left_update<R, NT, 1>(T, ld, k, r, p, ct, sc);
      else if (nr <= 32) bidiag_left_update<R, NT, 2>(T, ld, k, r, p, ct, sc);
      else if (nr <= 64) bidiag_left_update<R, NT, 4>(T, ld, k, r, p, ct, sc);
      else if (nr <= 128) bidiag_left_update<R, NT, 8>(T, ld, k, r, p, ct, sc);
      else bidiag_left_update<R, NT, 16>(T, ld, k, r, p, ct, sc);
    }
    __syncthreads();
    if (k + 1 >= p) {
      if (threadIdx.x == 0) ck[k] = sc_l;
      break;
    }
    // --- right half step: reflector of conj(row k) (columns k+1..p-1), applied to
    //     rows k+1..r-1
    make_reflector(conj(T[(size_t)(k + 1) * ld + k]), warp_sum_norm2(T + k, k + 2, p, ld), &tau, &beta,
                   &sc);
    if (threadIdx.x == 0) {
      ee[k] = beta;
      tauR[k] = tau;
      ck[k] = sc_l;   // T[k][k]: pivot of left reflector k
      pend_r = sc;
    }
    {
      // 8 lanes per row for complex<float>, 16 for complex<double> (register budget)
      constexpr int G = sizeof(R) == 4 ? 8 : 16;
      const int nc = p - k - 1;
      if (nc <= G) bidiag_right_update<R, NT, G, 1>(T, ld, k, r, p, tau, sc);
      else if (nc <= 2 * G) bidiag_right_update<R, NT, G, 2>(T, ld, k, r, p, tau, sc);
      else if (nc <= 4 * G) bidiag_right_update<R, NT, G, 4>(T, ld, k, r, p, tau, sc);
      else if (nc <= 8 * G) bidiag_right_update<R, NT, G, 8>(T, ld, k, r, p, tau, sc);
      else if (nc <= 16 * G) bidiag_right_update<R, NT, G, 16>(T, ld, k, r, p, tau, sc);
      else bidiag_right_update<R, NT, 16, 16>(T, ld, k, r, p, tau, sc);
    }
    __syncthreads();
  }
  __syncthreads();
}

// Number of singular values of B that are >= x, from the negative count of the
// LDL^T factorisation of TGK - x I (b2 = squared off-diagonal of TGK, length N-1).
template <class R>
__device__ __forceinline__ int count_ge(const R* b2, int p, R x, R tiny) {
  const int N = 2 * p;
  R q = -x;
  int neg = q < R(0);
#pragma unroll 8
  for (int i = 1; i < N; ++i) {
    if (rabs(q) < tiny) q = -tiny;
    q = -x - qdiv(b2[i - 1], q);
    neg += q < R(0);
  }
  return N - neg;
}

// Same count restricted to TGK indices [s, e) (one unreduced block after splitting).
template <class R>
__device__ __forceinline__ int count_ge_block(const R* b2, int s, int e, R x, R tiny) {
  R q = -x;
  int neg = q < R(0);
#pragma unroll 4
  for (int i = s + 1; i < e; ++i) {
    if (rabs(q) < tiny) q = -tiny;
    q = -x - qdiv(b2[i - 1], q);
    neg += q < R(0);
  }
  return (e - s) - neg;
}

// All kk largest singular values (descending) into sig[0..kk), NT threads.
// scratch: lo[kk], hi[kk], cnt[NT], xs[NT].
template <class R, int NT>
__device__ void bisect_singular_values(const R* b2, int p, R smax, int kk, int iters, R* sig, R* lo, R* hi,
                                       int* cnt, R* xs, const R* grid) {
  const int tid = threadIdx.x;
  const R tiny = smax * R(1e-30) + R(1e-37);
  // grid pass: NT log-spaced shifts smax * grid[t] (grid computed once per launch)
  {
    const R x = smax * grid[tid];
    xs[tid] = x;
    cnt[tid] = count_ge(b2, p, x, tiny);
  }
  __syncthreads();
  for (int i = tid; i < kk; i += NT) {
    // largest grid index with cnt >= i+1 (cnt is non-increasing in the index)
    int a = -1, b = NT;
    while (b - a > 1) {
      const int mid = (a + b) >> 1;
      if (cnt[mid] >= i + 1) a = mid; else b = mid;
    }
    lo[i] = a >= 0 ? xs[a] : R(0);
    hi[i] = (a + 1 < NT) ? xs[a + 1] : smax * R(1.001) + tiny;
  }
  __syncthreads();
  const int per = max(1, NT / max(kk, 1));
  for (int it = 0; it < iters; ++it) {
    const int i = tid / per, j = tid - i * per;
    const bool act = i < kk;
    R x = 0;
    int c = 0;
    if (act) {
      x = lo[i] + (hi[i] - lo[i]) * (R)(j + 1) / (R)(per + 1);
      c = count_ge(b2, p, x, tiny);
    }
    xs[tid] = x;
    cnt[tid] = c;
    __syncthreads();
    if (act && j == 0) {
      R nlo = lo[i], nhi = hi[i];
      for (int q = 0; q < per; ++q) {
        const R xq = xs[tid + q];
        if (cnt[tid + q] >= i + 1) nlo = fmax(nlo, xq); else nhi = fmin(nhi, xq);
      }
      lo[i] = nlo;
      hi[i] = nhi;
    }
    __syncthreads();
  }
  for (int i = tid; i < kk; i += NT) sig[i] = R(0.5) * (lo[i] + hi[i]);
  __syncthreads();
}

// Eigenvector of the TGK block [s0, e0) (zero diagonal, off-diagonal b) for eigenvalue
// lam by a twisted factorisation; writes the half selected by `odd` (0: even TGK
// indices = right singular vector of B; 1: odd indices = left singular vector),
// normalised, into w[0..p). dp, dm: per-thread scratch of at least 2p entries.
template <class R>
__device__ void twisted_vector(const R* b, int p, int s0, int e0, R lam, R tiny, R* dp, R* dm, int stride, int odd,
                               R* w) {
  // dp, dm: this thread's scratch, entry i at [i * stride] (threads interleaved, so a
  // group of threads stepping through i touches consecutive addresses)
  dp[(size_t)s0 * stride] = -lam;
  R prev = -lam;
  for (int i = s0 + 1; i < e0; ++i) {
    if (rabs(prev) < tiny) prev = -tiny;
    prev = -lam - qdiv(b[i - 1] * b[i - 1], prev);
    dp[(size_t)i * stride] = prev;
  }
  // backward pass fused with the twist search: gamma_i = dp_i + dm_i + lam. The scratch
  // lives in global memory, so its reads are issued 8 at a time ahead of their use.
  constexpr int PF = 8;
  int rr = e0 - 1;
  R nxt = -lam;
  dm[(size_t)(e0 - 1) * stride] = nxt;
  R best = rabs(dp[(size_t)(e0 - 1) * stride] + nxt + lam);
  for (int i0 = e0 - 2; i0 >= s0; i0 -= PF) {
    R dpv[PF];
#pragma unroll
    for (int u = 0; u < PF; ++u) dpv[u] = i0 - u >= s0 ? dp[(size_t)(i0 - u) * stride] : R(0);
#pragma unroll
    for (int u = 0; u < PF; ++u) {
      const int i = i0 - u;
      if (i >= s0) {
        R q = nxt;
        if (rabs(q) < tiny) q = -tiny;
        nxt = -lam - qdiv(b[i] * b[i], q);
        dm[(size_t)i * stride] = nxt;
        const R g = rabs(dpv[u] + nxt + lam);
        if (g < best) {
          best = g;
          rr = i;
        }
      }
    }
  }
  // z_rr = 1; z_i = -(b_i / dp_i) z_{i+1} below, z_i = -(b_{i-1} / dm_i) z_{i-1} above
  for (int q = 0; q < p; ++q) w[q] = R(0);
  R z = 1;
  if ((rr & 1) == odd) w[rr >> 1] = z;
  for (int i0 = rr - 1; i0 >= s0; i0 -= PF) {
    R dv[PF];
#pragma unroll
    for (int u = 0; u < PF; ++u) dv[u] = i0 - u >= s0 ? dp[(size_t)(i0 - u) * stride] : R(1);
#pragma unroll
    for (int u = 0; u < PF; ++u) {
      const int i = i0 - u;
      if (i >= s0) {
        R d = dv[u];
        if (rabs(d) < tiny) d = -tiny;
        z = -qdiv(b[i], d) * z;
        if ((i & 1) == odd) w[i >> 1] = z;
      }
    }
  }
  z = 1;
  for (int i0 = rr + 1; i0 < e0; i0 += PF) {
    R dv[PF];
#pragma unroll
    for (int u = 0; u < PF; ++u) dv[u] = i0 + u < e0 ? dm[(size_t)(i0 + u) * stride] : R(1);
#pragma unroll
    for (int u = 0; u < PF; ++u) {
      const int i = i0 + u;
      if (i < e0) {
        R d = dv[u];
        if (rabs(d) < tiny) d = -tiny;
        z = -qdiv(b[i - 1], d) * z;
        if ((i & 1) == odd) w[i >> 1] = z;
      }
    }
  }
  R nrm = 0;
  for (int q = 0; q < p; ++q) nrm += w[q] * w[q];
  const R inv = nrm > R(0) ? R(1) / sqrt(nrm) : R(0);
  for (int q = 0; q < p; ++q) w[q] *= inv;
}

// Block [s, e) of the split TGK that owns target t: the (m+1)-th eigenvalue inside the
// window (lam - delta, lam + delta] scanning blocks in index order, where m counts the
// earlier targets that fall in the same window (exactly degenerate values of different
// blocks get different blocks).
template <class R>
__device__ void owning_block(const R* b2, int N, const R* sig, int t, R delta, R tiny, int* s_out, int* e_out) {
  const R lam = sig[t];
  int m = 0;
  for (int u = 0; u < t; ++u) m += rabs(sig[u] - lam) <= delta;
  int occ = 0, bs = 0;
  *s_out = 0;
  *e_out = N;
  for (int i = 0; i < N; ++i) {
    const bool end = (i == N - 1) || (b2[i] == R(0));
    if (!end) continue;
    const int e = i + 1;
    const int inwin = count_ge_block(b2, bs, e, lam - delta, tiny) - count_ge_block(b2, bs, e, lam + delta, tiny);
    if (inwin > 0 && occ + inwin > m) {
      *s_out = bs;
      *e_out = e;
      return;
    }
    occ += inwin;
    bs = e;
  }
}

// Block classical Gram-Schmidt twice (BCGS2) over the rows of W (k x p, row stride
// ldw), in blocks of 8 rows. Each of the two repetitions projects the block out of all
// earlier rows and then orthonormalises it internally by Cholesky QR (G = W_b W_b^T =
// L L^T, W_b <- L^{-1} W_b). Row t of the result depends only on rows 0..t, so the
// leading singular vectors keep their directions. A Cholesky pivot below 1e-6 of its
// diagonal (a row that is numerically a combination of earlier rows) counts as a
// collapse. coef: >= 8 k shared scratch (used once k > 8); small: >= 128 shared.
template <class R, int NT>
__device__ void orthonormalize_rows_block(R* W, int ldw, int k, int p, R* coef, R* small, int* collapsed) {
  const int tid = threadIdx.x;
  for (int b0 = 0; b0 < k; b0 += 8) {
    const int nb = min(8, k - b0);
    for (int rep = 0; rep < 2; ++rep) {
      if (b0 > 0) {
        // coef[u * 8 + j] = <w_u, w_{b0+j}>, 8 lanes per dot
        const int nd = b0 * nb;
        for (int base = 0; base < nd * 8; base += NT) {
          const int d = (base + tid) >> 3, l = tid & 7;
          const bool act = d < nd;
          const int u = act ? d / nb : 0, j = act ? d - u * nb : 0;
          R acc = 0;
          if (act)
            for (int q = l; q < p; q += 8) acc += W[(size_t)u * ldw + q] * W[(size_t)(b0 + j) * ldw + q];
          for (int o = 1; o < 8; o <<= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
          if (act && l == 0) coef[u * 8 + j] = acc;
        }
        __syncthreads();
        for (int it = tid; it < nb * p; it += NT) {
          const int j = it / p, q = it - j * p;
          R v = W[(size_t)(b0 + j) * ldw + q];
          for (int u = 0; u < b0; ++u) v -= coef[u * 8 + j] * W[(size_t)u * ldw + q];
          W[(size_t)(b0 + j) * ldw + q] = v;
        }
        __syncthreads();
      }
      // Gram matrix of the block (lower triangle): small[i * 8 + j], j <= i
      const int ng = nb * (nb + 1) / 2;
      for (int base = 0; base < ng * 8; base += NT) {
        const int d = (base + tid) >> 3, l = tid & 7;
        const bool act = d < ng;
        int i = 0;
        while ((i + 1) * (i + 2) / 2 <= d && i < 7) ++i;
        const int j = d - i * (i + 1) / 2;
        R acc = 0;
        if (act)
          for (int q = l; q < p; q += 8) acc += W[(size_t)(b0 + i) * ldw + q] * W[(size_t)(b0 + j) * ldw + q];
        for (int o = 1; o < 8; o <<= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (act && l == 0) small[i * 8 + j] = acc;
      }
      __syncthreads();
      // Cholesky factor L and its inverse X = L^{-1} (written to small + 64); one thread,
      // the 8 x 8 factor kept in registers (all indices compile-time)
      if (tid == 0) {
        R Lm[8][8], Xm[8][8];
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            Lm[i][j] = (j <= i && i < nb) ? small[i * 8 + j] : R(0);
            Xm[i][j] = R(0);
          }
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          if (j < nb) {
            const R gjj = Lm[j][j];
            R d = gjj;
#pragma unroll
            for (int u = 0; u < j; ++u) d -= Lm[j][u] * Lm[j][u];
            if (!(d > R(1e-6) * gjj)) {
              ++*collapsed;
              d = gjj > R(0) ? gjj * R(1e-30) : R(1e-30);
            }
            const R ljj = sqrt(d), inv = R(1) / ljj;
            Lm[j][j] = ljj;
#pragma unroll
            for (int i = j + 1; i < 8; ++i) {
              R v = Lm[i][j];
#pragma unroll
              for (int u = 0; u < j; ++u) v -= Lm[i][u] * Lm[j][u];
              Lm[i][j] = v * inv;
            }
          }
        }
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          Xm[j][j] = R(1) / Lm[j][j];
#pragma unroll
          for (int i = j + 1; i < 8; ++i) {
            R v = 0;
#pragma unroll
            for (int u = j; u < i; ++u) v += Lm[i][u] * Xm[u][j];
            Xm[i][j] = -v / Lm[i][i];
          }
        }
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
          for (int j = 0; j < 8; ++j) small[64 + i * 8 + j] = Xm[i][j];
      }
      __syncthreads();
      // W_b <- X W_b, one thread per column
      for (int q = tid; q < p; q += NT) {
        R x[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) x[i] = i < nb ? W[(size_t)(b0 + i) * ldw + q] : R(0);
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          if (i < nb) {
            R y = 0;
#pragma unroll
            for (int u = 0; u <= i; ++u) y += small[64 + i * 8 + u] * x[u];
            W[(size_t)(b0 + i) * ldw + q] = y;
          }
        }
      }
      __syncthreads();
    }
  }
}

// One-sided (Hestenes) Jacobi on the `ncols` columns of X (each of length `len`,
// column stride ldx), used when the bidiagonal route reports a collapsed vector
// (numerically degenerate singular values without a split). Columns converge to
// sigma_p times a singular vector; columns below sqrt(zero2) are numerically zero.
template <class R, int NT, int MAXE>
__device__ void jacobi_columns(Cx<R>* X, int ldx, int ncols, int len, double zero2, int max_sweeps,
                               int* noconv) {
  int G = 1;
  while (G < 32 && G * MAXE < len) G <<= 1;
  const int npairs = (ncols + 1) >> 1;
  while (G < 32 && G < len && (NT / (2 * G)) >= npairs) G <<= 1;
  const int ept = (len + G - 1) / G;
  const int ngroups = NT / G, grp = threadIdx.x / G, lane = threadIdx.x - grp * G;
  const R tol = R(2) * (sizeof(R) == 8 ? R(2.220446049250313e-16) : R(1.1920929e-7)) * sqrt((R)len);
  const int mm = ncols + (ncols & 1);  // even number of players; index ncols is a dummy
  bool converged = ncols <= 1;
  int sweep = 0;
  for (; sweep < max_sweeps && !converged; ++sweep) {
    int rotated = 0;
    for (int r = 0; r < mm - 1; ++r) {
      for (int base = 0; base < mm / 2; base += ngroups) {
        const int pi = base + grp;
        int p = 0, q = 1;
        if (pi == 0) {
          p = r;
          q = mm - 1;
        } else if (pi < mm / 2) {
          p = (r + pi) % (mm - 1);
          q = (r - pi + (mm - 1)) % (mm - 1);
        }
        const bool active = pi < mm / 2 && p < ncols && q < ncols;
        Cx<R>* xp = X + (size_t)p * ldx;
        Cx<R>* xq = X + (size_t)q * ldx;
        Cx<R> vp[MAXE], vq[MAXE];
        R al = 0, be = 0;
        Cx<R> ga = cx<R>(0, 0);
#pragma unroll
        for (int e = 0; e < MAXE; ++e) {
          const int idx = lane + e * G;
          if (active && e < ept && idx < len) {
            vp[e] = xp[idx];
            vq[e] = xq[idx];
          } else {
            vp[e] = cx<R>(0, 0);
            vq[e] = cx<R>(0, 0);
          }
          al += norm2(vp[e]);
          be += norm2(vq[e]);
          cmac_conj(ga, vp[e], vq[e]);
        }
        for (int o = G >> 1; o > 0; o >>= 1) {
          al += __shfl_xor_sync(0xffffffffu, al, o, G);
          be += __shfl_xor_sync(0xffffffffu, be, o, G);
          ga.x += __shfl_xor_sync(0xffffffffu, ga.x, o, G);
          ga.y += __shfl_xor_sync(0xffffffffu, ga.y, o, G);
        }
        const R ag = sqrt(norm2(ga));
        if (active && ag > R(0) && (double)fmin(al, be) > zero2 && ag > tol * sqrt(al) * sqrt(be)) {
          const R zeta = (be - al) / (R(2) * ag);
          const R az = rabs(zeta);
          const R t = az > R(1e15) ? R(0.5) / zeta : copysign(R(1), zeta) / (az + sqrt(R(1) + zeta * zeta));
          if (t != R(0)) {
            const R cs = R(1) / sqrt(R(1) + t * t), sn = cs * t;
            const Cx<R> sph = cx<R>(sn * ga.x / ag, sn * ga.y / ag);
#pragma unroll
            for (int e = 0; e < MAXE; ++e) {
              const int idx = lane + e * G;
              if (e < ept && idx < len) {
                const Cx<R> a = vp[e], b = vq[e];
                xp[idx] = cs * a - conj(sph) * b;
                xq[idx] = sph * a + cs * b;
              }
            }
            rotated = 1;
          }
        }
      }
      __syncthreads();
    }
    converged = !__syncthreads_or(rotated);
  }
  if (threadIdx.x == 0 && !converged) ++*noconv;
}

}  // namespace mpsvqe
