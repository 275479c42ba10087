// Truncated SVD of one gate's M' inside one thread block (Eq. 9 of the paper).
//
// Route: Householder bidiagonalisation of the tall orientation of M' (the paper's
// own SVD also starts from a bidiagonal reduction), then the singular values of the
// real bidiagonal B from Sturm counts of its Golub-Kahan tridiagonal
// TGK = [[0, B], [B^T, 0]] (multisection bisection), singular vectors of B from a
// twisted factorisation of TGK - sigma I, re-orthonormalisation (classical
// Gram-Schmidt twice, in descending sigma order), and back-transformation by the
// stored Householder reflectors.
//
// Conventions: the reflector H = I - tau v v^H (v_0 = 1) satisfies H^H x = beta e_1
// with beta real. T (r x p, r >= p, column-major, leading dimension ld) is reduced
// to T = Q B P^H with Q = H_0 H_1 ... (left reflectors stored below the diagonal),
// P = G_0 G_1 ... (right reflectors stored right of the superdiagonal).
#pragma once
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

// LAPACK-style reflector for x = (alpha, tail) with ||tail||^2 = xn2.
template <class R>
__device__ __forceinline__ void make_reflector(Cx<R> alpha, R xn2, Cx<R>* tau, R* beta, Cx<R>* scale) {
  if (xn2 == R(0) && alpha.y == R(0)) {
    *tau = cx<R>(0, 0);
    *beta = alpha.x;
    *scale = cx<R>(0, 0);
    return;
  }
  const R nrm = sqrt(alpha.x * alpha.x + alpha.y * alpha.y + xn2);
  const R b = alpha.x >= R(0) ? -nrm : nrm;
  *beta = b;
  *tau = cx<R>((b - alpha.x) / b, -alpha.y / b);
  // scale = 1 / (alpha - beta)
  const Cx<R> den = cx<R>(alpha.x - b, alpha.y);
  const R dn = den.x * den.x + den.y * den.y;
  *scale = cx<R>(den.x / dn, -den.y / dn);
}

// Householder bidiagonalisation, NT threads, T in shared (or global) memory. dd[k]
// (diagonal) and ee[k] (superdiagonal) receive the real entries; tauL/tauR the
// reflector factors. Each column (left update) or row (right update) is handled by 8
// lanes that keep their 16 entries in registers between the dot product and the
// rank-1 update, so every element is read and written once per half step.
// vb, wb: shared scratch of >= r and >= p complex entries (reflector vectors).
template <class R, int NT>
__device__ void bidiagonalize(Cx<R>* T, int ld, int r, int p, R* dd, R* ee, Cx<R>* tauL, Cx<R>* tauR,
                              Cx<R>* vb, Cx<R>* wb, unsigned long long* sub = nullptr) {
  long long tm = clock64();
  auto mark = [&](int i) {
    if (sub && threadIdx.x == 0) {
      const long long now = clock64();
      sub[i] += (unsigned long long)(now - tm);
      tm = now;
    }
  };
  constexpr int EPL = sizeof(R) == 4 ? 16 : 8;   // entries per lane
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int k = 0; k < p; ++k) {
    // --- left reflector on column k, rows k..r-1 (warp 0)
    if (warp == 0) {
      R xn2 = 0;
      for (int i = k + 1 + lane; i < r; i += 32) xn2 += norm2(T[(size_t)k * ld + i]);
      for (int o = 16; o > 0; o >>= 1) xn2 += __shfl_xor_sync(0xffffffffu, xn2, o);
      Cx<R> tau, sc;
      R beta;
      make_reflector(T[(size_t)k * ld + k], xn2, &tau, &beta, &sc);
      for (int i = k + 1 + lane; i < r; i += 32) {
        const Cx<R> v = T[(size_t)k * ld + i] * sc;
        T[(size_t)k * ld + i] = v;
        vb[i] = v;
      }
      if (lane == 0) {
        T[(size_t)k * ld + k] = cx<R>(beta, 0);
        vb[k] = cx<R>(1, 0);
        dd[k] = beta;
        tauL[k] = tau;
      }
    }
    __syncthreads();
    mark(0);
    // --- apply H^H = I - conj(tau) v v^H to columns k+1..p-1
    {
      const Cx<R> ct = conj(tauL[k]);
      const int nr = r - k;
      // lanes per column for this step: the fewest that cover the live rows
      int lg = 0;
      while (lg < 5 && (EPL << lg) < nr) ++lg;
      const int LPC = 1 << lg, grp = tid >> lg, l8 = tid & (LPC - 1);
      Cx<R> v[EPL];
#pragma unroll
      for (int e = 0; e < EPL; ++e) {
        const int i = k + l8 + LPC * e;
        v[e] = (l8 + LPC * e < nr) ? vb[i] : cx<R>(0, 0);
      }
      for (int cbase = k + 1; cbase < p; cbase += NT / LPC) {
        const int col = cbase + grp;
        const bool act = col < p;
        Cx<R>* tc = T + (size_t)(act ? col : k) * ld;
        Cx<R> x[EPL];
        Cx<R> s = cx<R>(0, 0);
#pragma unroll
        for (int e = 0; e < EPL; ++e) {
          const int off = l8 + LPC * e;
          x[e] = (act && off < nr) ? tc[k + off] : cx<R>(0, 0);
          cmac_conj(s, v[e], x[e]);
        }
        for (int o = 1; o < LPC; o <<= 1) {
          s.x += __shfl_xor_sync(0xffffffffu, s.x, o, LPC);
          s.y += __shfl_xor_sync(0xffffffffu, s.y, o, LPC);
        }
        const Cx<R> f = ct * s;
#pragma unroll
        for (int e = 0; e < EPL; ++e) {
          const int off = l8 + LPC * e;
          if (act && off < nr) tc[k + off] = x[e] - f * v[e];
        }
      }
    }
    __syncthreads();
    mark(1);
    if (k >= p - 1) break;
    // --- right reflector on row k, columns k+1..p-1 (warp 0), acting on conj(row)
    if (warp == 0) {
      R xn2 = 0;
      for (int j = k + 2 + lane; j < p; j += 32) xn2 += norm2(T[(size_t)j * ld + k]);
      for (int o = 16; o > 0; o >>= 1) xn2 += __shfl_xor_sync(0xffffffffu, xn2, o);
      Cx<R> tau, sc;
      R beta;
      make_reflector(conj(T[(size_t)(k + 1) * ld + k]), xn2, &tau, &beta, &sc);
      for (int j = k + 2 + lane; j < p; j += 32) {
        const Cx<R> w = conj(T[(size_t)j * ld + k]) * sc;
        T[(size_t)j * ld + k] = w;
        wb[j] = w;
      }
      if (lane == 0) {
        T[(size_t)(k + 1) * ld + k] = cx<R>(beta, 0);
        wb[k + 1] = cx<R>(1, 0);
        ee[k] = beta;
        tauR[k] = tau;
      }
    }
    __syncthreads();
    mark(2);
    // --- apply G = I - tau w w^H from the right to rows k+1..r-1, columns k+1..p-1
    {
      const Cx<R> t = tauR[k];
      const int nc = p - k - 1;
      int lg = 0;
      while (lg < 5 && (EPL << lg) < nc) ++lg;
      const int LPC = 1 << lg, grp = tid >> lg, l8 = tid & (LPC - 1);
      Cx<R> w[EPL];
#pragma unroll
      for (int e = 0; e < EPL; ++e) {
        const int off = l8 + LPC * e;
        w[e] = (off < nc) ? wb[k + 1 + off] : cx<R>(0, 0);
      }
      for (int rbase = k + 1; rbase < r; rbase += NT / LPC) {
        const int row = rbase + grp;
        const bool act = row < r;
        const int rr = act ? row : k;
        Cx<R> x[EPL];
        Cx<R> s = cx<R>(0, 0);
#pragma unroll
        for (int e = 0; e < EPL; ++e) {
          const int off = l8 + LPC * e;
          x[e] = (act && off < nc) ? T[(size_t)(k + 1 + off) * ld + rr] : cx<R>(0, 0);
          cmac(s, x[e], w[e]);
        }
        for (int o = 1; o < LPC; o <<= 1) {
          s.x += __shfl_xor_sync(0xffffffffu, s.x, o, LPC);
          s.y += __shfl_xor_sync(0xffffffffu, s.y, o, LPC);
        }
        const Cx<R> f = t * s;
#pragma unroll
        for (int e = 0; e < EPL; ++e) {
          const int off = l8 + LPC * e;
          if (act && off < nc) T[(size_t)(k + 1 + off) * ld + rr] = x[e] - f * conj(w[e]);
        }
      }
    }
    __syncthreads();
    mark(3);
  }
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
  // backward pass fused with the twist search: gamma_i = dp_i + dm_i + lam
  int rr = e0 - 1;
  R nxt = -lam;
  dm[(size_t)(e0 - 1) * stride] = nxt;
  R best = rabs(dp[(size_t)(e0 - 1) * stride] + nxt + lam);
  for (int i = e0 - 2; i >= s0; --i) {
    R q = nxt;
    if (rabs(q) < tiny) q = -tiny;
    nxt = -lam - qdiv(b[i] * b[i], q);
    dm[(size_t)i * stride] = nxt;
    const R g = rabs(dp[(size_t)i * stride] + nxt + lam);
    if (g < best) {
      best = g;
      rr = i;
    }
  }
  // z_rr = 1; z_i = -(b_i / dp_i) z_{i+1} below, z_i = -(b_{i-1} / dm_i) z_{i-1} above
  for (int q = 0; q < p; ++q) w[q] = R(0);
  R z = 1;
  if ((rr & 1) == odd) w[rr >> 1] = z;
  for (int i = rr - 1; i >= s0; --i) {
    R d = dp[(size_t)i * stride];
    if (rabs(d) < tiny) d = -tiny;
    z = -qdiv(b[i], d) * z;
    if ((i & 1) == odd) w[i >> 1] = z;
  }
  z = 1;
  for (int i = rr + 1; i < e0; ++i) {
    R d = dm[(size_t)i * stride];
    if (rabs(d) < tiny) d = -tiny;
    z = -qdiv(b[i - 1], d) * z;
    if ((i & 1) == odd) w[i >> 1] = z;
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

// Cholesky-QR twice over the rows of W (k x p, row stride ldw): G = W W^T, G = L L^T,
// W <- L^{-1} W. Row t of the result depends only on rows 0..t (Gram-Schmidt order),
// so the leading singular vectors are kept as computed. A pivot below 1e-6 of its
// diagonal (a row that is numerically a combination of earlier rows) counts as a
// collapse. G: k x k shared scratch.
template <class R, int NT>
__device__ void orthonormalize_rows_chol(R* W, int ldw, int k, int p, R* G, int* collapsed) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int pass = 0; pass < 2; ++pass) {
    // G = W W^T (lower triangle)
    for (int e = tid; e < k * k; e += NT) {
      const int a = e / k, b = e - a * k;
      if (b > a) continue;
      R acc = 0;
      const R* wa = W + (size_t)a * ldw;
      const R* wb = W + (size_t)b * ldw;
#pragma unroll 4
      for (int q = 0; q < p; ++q) acc += wa[q] * wb[q];
      G[a * k + b] = acc;
    }
    __syncthreads();
    // in-place Cholesky (lower), one warp
    if (warp == 0) {
      for (int j = 0; j < k; ++j) {
        R d = G[j * k + j];
        for (int u = lane; u < j; u += 32) {
          const R l = G[j * k + u];
          d -= l * l;  // partial, reduced below
        }
        // reduce the partial subtraction across lanes
        R part = G[j * k + j] - d;
        for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
        const R diag = G[j * k + j];
        R piv = diag - part;
        if (lane == 0 && !(piv > R(1e-6) * diag)) {
          ++*collapsed;
        }
        if (!(piv > R(0))) piv = diag > R(0) ? diag * R(1e-30) : R(1e-30);
        const R ljj = sqrt(piv);
        __syncwarp();
        for (int i = j + 1 + lane; i < k; i += 32) {
          R v = G[i * k + j];
          for (int u = 0; u < j; ++u) v -= G[i * k + u] * G[j * k + u];
          G[i * k + j] = v / ljj;
        }
        __syncwarp();
        if (lane == 0) G[j * k + j] = ljj;
        __syncwarp();
      }
    }
    __syncthreads();
    // W <- L^{-1} W, one thread per column
    for (int q = tid; q < p; q += NT) {
      for (int t = 0; t < k; ++t) {
        R v = W[(size_t)t * ldw + q];
        for (int u = 0; u < t; ++u) v -= G[t * k + u] * W[(size_t)u * ldw + q];
        W[(size_t)t * ldw + q] = v / G[t * k + t];
      }
    }
    __syncthreads();
  }
}

// Block classical Gram-Schmidt (twice) over the rows of W (k x p, row stride ldw), in
// blocks of 8 rows: each block is projected out of all earlier rows in two passes, then
// orthonormalised internally by one warp (modified Gram-Schmidt). Row t of the result
// depends only on rows 0..t, so the leading singular vectors keep their directions. A
// row whose remainder falls below 1e-3 of its norm counts as a collapse.
// coef: >= 8 k shared scratch.
template <class R, int NT>
__device__ void orthonormalize_rows_block(R* W, int ldw, int k, int p, R* coef, int* collapsed) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int b0 = 0; b0 < k; b0 += 8) {
    const int nb = min(8, k - b0);
    for (int pass = 0; pass < 2 && b0 > 0; ++pass) {
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
    if (warp == 0) {
      for (int j = 0; j < nb; ++j) {
        R* wj = W + (size_t)(b0 + j) * ldw;
        R n0 = 0;
        for (int q = lane; q < p; q += 32) n0 += wj[q] * wj[q];
        for (int o = 16; o > 0; o >>= 1) n0 += __shfl_xor_sync(0xffffffffu, n0, o);
        for (int rep = 0; rep < 2; ++rep)
          for (int i = 0; i < j; ++i) {
            const R* wi = W + (size_t)(b0 + i) * ldw;
            R d = 0;
            for (int q = lane; q < p; q += 32) d += wi[q] * wj[q];
            for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
            for (int q = lane; q < p; q += 32) wj[q] -= d * wi[q];
            __syncwarp();
          }
        R nr = 0;
        for (int q = lane; q < p; q += 32) nr += wj[q] * wj[q];
        for (int o = 16; o > 0; o >>= 1) nr += __shfl_xor_sync(0xffffffffu, nr, o);
        if (lane == 0 && !(nr > R(1e-6) * n0)) ++*collapsed;
        const R inv = nr > R(0) ? R(1) / sqrt(nr) : R(0);
        for (int q = lane; q < p; q += 32) wj[q] *= inv;
        __syncwarp();
      }
    }
    __syncthreads();
  }
}

// Classical Gram-Schmidt twice over the rows of W (k x p, row stride ldw), in order.
template <class R, int NT>
__device__ void orthonormalize_rows(R* W, int ldw, int k, int p, R* coef, int* collapsed) {
  const int tid = threadIdx.x;
  for (int t = 0; t < k; ++t) {
    for (int pass = 0; pass < 2; ++pass) {
      // coef[s] = <w_s, w_t> for s < t, 8 threads per dot
      const int s = tid >> 3, l8 = tid & 7;
      for (int sb = s; ; sb += NT / 8) {
        const bool act = sb < t;
        if (!__any_sync(0xffffffffu, act)) break;
        R acc = 0;
        if (act)
          for (int q = l8; q < p; q += 8) acc += W[(size_t)sb * ldw + q] * W[(size_t)t * ldw + q];
        for (int o = 1; o < 8; o <<= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (act && l8 == 0) coef[sb] = acc;
      }
      __syncthreads();
      for (int q = tid; q < p; q += NT) {
        R v = W[(size_t)t * ldw + q];
        for (int u = 0; u < t; ++u) v -= coef[u] * W[(size_t)u * ldw + q];
        W[(size_t)t * ldw + q] = v;
      }
      __syncthreads();
    }
    // normalise row t (warp 0)
    if ((tid >> 5) == 0) {
      R acc = 0;
      for (int q = tid; q < p; q += 32) acc += W[(size_t)t * ldw + q] * W[(size_t)t * ldw + q];
      for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
      const R inv = acc > R(0) ? R(1) / sqrt(acc) : R(0);
      if (tid == 0 && acc < R(1e-6)) ++*collapsed;
      for (int q = tid; q < p; q += 32) W[(size_t)t * ldw + q] *= inv;
    }
    __syncthreads();
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
