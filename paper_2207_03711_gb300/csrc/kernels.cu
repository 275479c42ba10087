// CUDA kernels of the MPS-VQE hot path for sm_103a (GB300).
//
//  k_reset        product-state reference (Sec. III-D: X gates on the occupied qubits).
//  k_circuit      persistent per-slot gate engine: for each two-site gate,
//                 Eq. (7) contraction, Eq. (8) row scaling by lambda_{n-1}, Eq. (9)
//                 truncated SVD by one-sided (Hestenes) Jacobi, Eq. (10) updates.
//  k_right_envs   right identity environments R_k and B^_k = B_k R_{k+1}.
//  k_level_T/child/close   one level of the Pauli-string prefix trie (Eq. 11 generalised).
//  k_energy_sum   E = sum_i a_i <P_i> (Eq. 2) with Neumaier compensation in FP64.
#include <cfloat>

#include "cx.cuh"
#include "kernels.cuh"

namespace mpsvqe {

template <class R>
struct Eps;
template <>
struct Eps<double> {
  static constexpr double v = 2.220446049250313e-16;
};
template <>
struct Eps<float> {
  static constexpr float v = 1.1920929e-7f;
};

template <class R>
__device__ __forceinline__ R shfl_x(R v, int o, int w) {
  return __shfl_xor_sync(0xffffffffu, v, o, w);
}

// ------------------------------------------------------------------------- reset
template <class R>
__global__ void k_reset(DevMPS m, int slot0, const uint8_t* occ) {
  const int s = slot0 + blockIdx.x;
  Cx<R>* B = (Cx<R>*)m.B + (size_t)s * m.slot_elems;
  int* rank = m.rank + (size_t)s * (m.n + 1);
  double* lam = m.lam + (size_t)s * (m.n - 1) * m.chi;
  for (int k = threadIdx.x; k < m.n; k += blockDim.x) {
    const uint8_t o = occ[(size_t)blockIdx.x * m.n + k];
    Cx<R>* b = B + m.site_off[k];
    b[0] = cx<R>(o ? R(0) : R(1), R(0));
    b[1] = cx<R>(o ? R(1) : R(0), R(0));
  }
  for (int b = threadIdx.x; b <= m.n; b += blockDim.x) rank[b] = 1;
  for (int b = threadIdx.x; b < m.n - 1; b += blockDim.x) lam[(size_t)b * m.chi] = 1.0;
  if (threadIdx.x == 0) m.dw[s] = 0.0;
  if (threadIdx.x < 4) m.stat[s * 4 + threadIdx.x] = (threadIdx.x == 2) ? 1 : 0;
}

cudaError_t launch_reset(const DevMPS& m, int prec, int slot0, int count, const uint8_t* occ,
                         cudaStream_t st) {
  if (prec == MPS_PREC_FP64)
    k_reset<double><<<count, 128, 0, st>>>(m, slot0, occ);
  else
    k_reset<float><<<count, 128, 0, st>>>(m, slot0, occ);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- gate engine

struct CircSmem {
  __host__ __device__ static constexpr size_t head(int mmax, int nt) {
    return ((16 * 16 /*U double*/ + 16 * 16 /*U in R, padded*/ + (size_t)mmax * 8 + (size_t)mmax * 4 +
             64 + (size_t)(nt / 32) * 16) +
            255) &
           ~(size_t)255;
  }
};

template <class R, int NT, int MAXE>
__global__ void __launch_bounds__(NT) k_circuit(DevMPS m, CircDev c, int64_t g0, int64_t g1,
                                                int slot0, const double* theta, double cutoff,
                                                int max_sweeps, int x_in_smem) {
  extern __shared__ __align__(256) unsigned char smem[];
  const int s = slot0 + blockIdx.x;
  const int n = m.n, chi = m.chi, mmax = 2 * chi;
  Cx<R>* Bslot = (Cx<R>*)m.B + (size_t)s * m.slot_elems;
  double* lam = m.lam + (size_t)s * (n - 1) * chi;
  int* rank = m.rank + (size_t)s * (n + 1);
  Cx<R>* W = (Cx<R>*)m.work_M + (size_t)s * mmax * mmax;

  Cx<double>* U = (Cx<double>*)smem;
  Cx<R>* Uf = (Cx<R>*)(smem + 256);
  double* sig2 = (double*)(smem + 512);
  int* order = (int*)(sig2 + mmax);
  int* misc = order + mmax;
  Cx<R>* X = x_in_smem ? (Cx<R>*)(smem + CircSmem::head(mmax, NT))
                       : (Cx<R>*)m.work_X + (size_t)s * mmax * (mmax + 1);
  const double* th = theta + (size_t)blockIdx.x * c.n_params;

  int st_max_sweeps = 0, st_noconv = 0, st_max_rank = 1;
  double dw_acc = 0.0;

  for (int64_t g = g0; g < g1; ++g) {
    const GateRec gr = c.gates[g];
    // (1) the 4x4 gate: fixed, or mats[m1] . Rz(phi) on one site . mats[m0]
    if (threadIdx.x < 16) {
      const int i = threadIdx.x >> 2, j = threadIdx.x & 3;
      const Cx<double>* A = (const Cx<double>*)c.mats + 16 * (size_t)gr.m0;
      Cx<double> u;
      if (gr.param < 0) {
        u = A[threadIdx.x];
      } else {
        const Cx<double>* P = (const Cx<double>*)c.mats + 16 * (size_t)gr.m1;
        const double half = 0.5 * gr.scale * th[gr.param];
        double sn, cs;
        sincos(half, &sn, &cs);
        u = cx(0.0, 0.0);
        for (int k = 0; k < 4; ++k) {
          const int bit = gr.rz_site == 0 ? ((k >> 1) & 1) : (k & 1);
          const Cx<double> ph = cx(cs, bit ? sn : -sn);  // Rz = diag(e^{-i phi/2}, e^{i phi/2})
          u = u + (P[i * 4 + k] * ph) * A[k * 4 + j];
        }
      }
      U[threadIdx.x] = u;
      Uf[threadIdx.x] = cx<R>((R)u.x, (R)u.y);
    }
    const int bond = gr.bond;
    const int rl = rank[bond], rm = rank[bond + 1], rr = rank[bond + 2];
    const int mrows = 2 * rl, ncol = 2 * rr, ldx = ncol + 1;
    Cx<R>* Bn = Bslot + m.site_off[bond];
    Cx<R>* Bn1 = Bslot + m.site_off[bond + 1];
    const double* laml = bond > 0 ? lam + (size_t)(bond - 1) * chi : nullptr;
    __syncthreads();

    // (2) Eq. (7): M[(a,i),(j,c)] = sum_{i'j'} U[ij,i'j'] sum_b B_n[a,i',b] B_{n+1}[b,j',c];
    //     W <- M; Eq. (8): column (a,i) of X <- conj(lambda_{n-1}[a] M[(a,i),:]).
    for (int it = threadIdx.x; it < rl * rr; it += NT) {
      const int a = it / rr, cc = it - a * rr;
      Cx<R> t00 = cx<R>(0, 0), t01 = t00, t10 = t00, t11 = t00;
      const Cx<R>* x0p = Bn + (size_t)(2 * a) * rm;
      const Cx<R>* x1p = x0p + rm;
      for (int b = 0; b < rm; ++b) {
        const Cx<R> x0 = x0p[b], x1 = x1p[b];
        const Cx<R> y0 = Bn1[(size_t)(2 * b) * rr + cc], y1 = Bn1[(size_t)(2 * b + 1) * rr + cc];
        cmac(t00, x0, y0);
        cmac(t01, x0, y1);
        cmac(t10, x1, y0);
        cmac(t11, x1, y1);
      }
      const Cx<R> th4[4] = {t00, t01, t10, t11};
      const R la = laml ? (R)laml[a] : R(1);
#pragma unroll
      for (int ij = 0; ij < 4; ++ij) {
        Cx<R> v = cx<R>(0, 0);
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) cmac(v, Uf[ij * 4 + kk], th4[kk]);
        const int row = 2 * a + (ij >> 1), col = (ij & 1) * rr + cc;
        W[(size_t)row * ncol + col] = v;
        X[(size_t)row * ldx + col] = conj(la * v);
      }
    }
    __syncthreads();

    // (3) Eq. (9): one-sided Jacobi on the mrows columns of X (length ncol). The
    // columns converge to sigma_p v_p^* (conjugated right singular vectors of M').
    int G = 1;
    while (G < 32 && G * MAXE < ncol) G <<= 1;
    const int npairs = mrows >> 1;
    while (G < 32 && G < ncol && (NT / (2 * G)) >= npairs) G <<= 1;
    const int ept = (ncol + G - 1) / G;
    const int ngroups = NT / G, grp = threadIdx.x / G, lane = threadIdx.x - grp * G;
    const R tol = R(2) * Eps<R>::v * sqrt((R)ncol);
    int sweep = 0;
    bool converged = (mrows <= 1);
    for (; sweep < max_sweeps && !converged; ++sweep) {
      int rotated = 0;
      for (int r = 0; r < mrows - 1; ++r) {
        // every lane of a warp runs the same trip count (group shuffles need full warps)
        for (int base = 0; base < npairs; base += ngroups) {
          const int pi = base + grp;
          const bool active = pi < npairs;
          int p = 0, q = 1;
          if (pi == 0) {
            p = r;
            q = mrows - 1;
          } else if (active) {
            p = (r + pi) % (mrows - 1);
            q = (r - pi + (mrows - 1)) % (mrows - 1);
          }
          Cx<R>* xp = X + (size_t)p * ldx;
          Cx<R>* xq = X + (size_t)q * ldx;
          Cx<R> vp[MAXE], vq[MAXE];
          R al = 0, be = 0;
          Cx<R> ga = cx<R>(0, 0);
#pragma unroll
          for (int e = 0; e < MAXE; ++e) {
            const int idx = lane + e * G;
            if (active && e < ept && idx < ncol) {
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
            al += shfl_x(al, o, G);
            be += shfl_x(be, o, G);
            ga.x += shfl_x(ga.x, o, G);
            ga.y += shfl_x(ga.y, o, G);
          }
          const R ag = sqrt(norm2(ga));
          if (active && ag > R(0) && ag > tol * sqrt(al) * sqrt(be)) {
            const R zeta = (be - al) / (R(2) * ag);
            const R az = fabs(zeta);
            const R t = az > R(1e15) ? R(0.5) / zeta
                                     : copysign(R(1), zeta) / (az + sqrt(R(1) + zeta * zeta));
            if (t != R(0)) {
              const R cs = R(1) / sqrt(R(1) + t * t), sn = cs * t;
              const Cx<R> ph = cx<R>(ga.x / ag, ga.y / ag);  // e^{i phi} = gamma / |gamma|
              const Cx<R> sph = cx<R>(sn * ph.x, sn * ph.y);
#pragma unroll
              for (int e = 0; e < MAXE; ++e) {
                const int idx = lane + e * G;
                if (e < ept && idx < ncol) {
                  const Cx<R> a = vp[e], b = vq[e];
                  // xp' = c xp - s e^{-i phi} xq ; xq' = s e^{i phi} xp + c xq
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
    if (!converged) ++st_noconv;
    st_max_sweeps = max(st_max_sweeps, sweep);

    // (4) squared column norms (FP64 accumulation), descending order, truncation
    for (int base = 0; base < mrows; base += ngroups) {
      const int p = base + grp;
      double acc = 0.0;
      if (p < mrows)
        for (int idx = lane; idx < ncol; idx += G) acc += (double)norm2(X[(size_t)p * ldx + idx]);
      for (int o = G >> 1; o > 0; o >>= 1) acc += shfl_x(acc, o, G);
      if (lane == 0 && p < mrows) sig2[p] = acc;
    }
    __syncthreads();
    for (int p = threadIdx.x; p < mrows; p += NT) {
      const double v = sig2[p];
      int rk = 0;
      for (int q = 0; q < mrows; ++q) {
        const double w = sig2[q];
        rk += (w > v) || (w == v && q < p);
      }
      order[rk] = p;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      const double s0 = sig2[order[0]];
      const int kmax = min(chi, min(mrows, ncol));
      int k = 0;
      while (k < kmax && sig2[order[k]] > cutoff * cutoff * s0) ++k;
      if (k == 0) k = 1;
      double total = 0.0, dropped = 0.0;
      for (int t = 0; t < mrows; ++t) total += sig2[order[t]];
      for (int t = k; t < mrows; ++t) dropped += sig2[order[t]];
      if (total > 0.0) dw_acc += dropped / total;
      misc[0] = k;
      st_max_rank = max(st_max_rank, k);
    }
    __syncthreads();
    const int k = misc[0];

    // (5) Eq. (10): B_{n+1} <- V (rows v_t = conj(column)/sigma), lambda_n <- sigma,
    //     B_n <- M V^+ i.e. B_n[(a,i),t] = sum_q M[(a,i),q] X[p_t][q] / sigma_t.
    for (int idx = threadIdx.x; idx < k * ncol; idx += NT) {
      const int t = idx / ncol, q = idx - t * ncol;
      const int p = order[t];
      const R inv = (R)(1.0 / sqrt(sig2[p]));
      Bn1[idx] = conj(inv * X[(size_t)p * ldx + q]);
    }
    for (int idx = threadIdx.x; idx < mrows * k; idx += NT) {
      const int t = idx / mrows, row = idx - t * mrows;
      const int p = order[t];
      const Cx<R>* xr = X + (size_t)p * ldx;
      const Cx<R>* wr = W + (size_t)row * ncol;
      Cx<R> acc = cx<R>(0, 0);
      for (int q = 0; q < ncol; ++q) cmac(acc, wr[q], xr[q]);
      const R inv = (R)(1.0 / sqrt(sig2[p]));
      Bn[(size_t)row * k + t] = inv * acc;
    }
    for (int t = threadIdx.x; t < k; t += NT) lam[(size_t)bond * chi + t] = sqrt(sig2[order[t]]);
    if (threadIdx.x == 0) rank[bond + 1] = k;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    m.dw[s] += dw_acc;
    int* stt = m.stat + s * 4;
    stt[0] = max(stt[0], st_max_sweeps);
    stt[1] += st_noconv;
    stt[2] = max(stt[2], st_max_rank);
  }
}

template <class R, int NT, int MAXE>
static cudaError_t launch_circ_t(const DevMPS& m, const CircDev& c, int64_t g0, int64_t g1,
                                 int slot0, int count, const double* theta, double cutoff,
                                 int max_sweeps, cudaStream_t st) {
  const int mmax = 2 * m.chi;
  const size_t head = CircSmem::head(mmax, NT);
  const size_t xbytes = (size_t)mmax * (mmax + 1) * sizeof(Cx<R>);
  const int x_in_smem = (head + xbytes) <= 200 * 1024;
  const size_t smem = head + (x_in_smem ? xbytes : 0);
  cudaError_t e = cudaFuncSetAttribute(k_circuit<R, NT, MAXE>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_circuit<R, NT, MAXE><<<count, NT, smem, st>>>(m, c, g0, g1, slot0, theta, cutoff, max_sweeps,
                                                  x_in_smem);
  return cudaGetLastError();
}

cudaError_t launch_circuit(const DevMPS& m, int prec, const CircDev& c, int64_t g0, int64_t g1,
                           int slot0, int count, const double* theta, double cutoff,
                           int max_sweeps, cudaStream_t st) {
  const bool big = 2 * m.chi > 256;
  if (prec == MPS_PREC_FP64)
    return big ? launch_circ_t<double, 256, 16>(m, c, g0, g1, slot0, count, theta, cutoff, max_sweeps, st)
               : launch_circ_t<double, 256, 8>(m, c, g0, g1, slot0, count, theta, cutoff, max_sweeps, st);
  return big ? launch_circ_t<float, 512, 16>(m, c, g0, g1, slot0, count, theta, cutoff, max_sweeps, st)
             : launch_circ_t<float, 512, 8>(m, c, g0, g1, slot0, count, theta, cutoff, max_sweeps, st);
}

// ------------------------------------------------------------ small tiled GEMM
// C (Mdim x Ndim, ldc) = sum_t s_t opA_t(A_t) B_t with 256 threads and 64x64 tiles.
// opA: A stored Mdim x K (lda) when conjT = false, or K x Mdim (lda) used as A^+.
template <class R>
struct GemmTerm {
  const Cx<R>* A;
  int lda;
  bool conjT;
  const Cx<R>* B;
  int ldb;
  Cx<R> s;
};

template <class R>
__device__ void block_gemm(int Mdim, int Ndim, int K, const GemmTerm<R>* terms, int nterm, Cx<R>* C,
                           int ldc, Cx<R> (*As)[17], Cx<R> (*Bs)[65]) {
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  for (int m0 = 0; m0 < Mdim; m0 += 64)
    for (int n0 = 0; n0 < Ndim; n0 += 64) {
      Cx<R> acc[4][4];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = cx<R>(0, 0);
      for (int t = 0; t < nterm; ++t) {
        const GemmTerm<R> T = terms[t];
        for (int k0 = 0; k0 < K; k0 += 16) {
          for (int e = threadIdx.x; e < 64 * 16; e += 256) {
            const int r = e >> 4, cc = e & 15;
            const int gm = m0 + r, gk = k0 + cc;
            Cx<R> v = cx<R>(0, 0);
            if (gm < Mdim && gk < K) v = T.conjT ? conj(T.A[(size_t)gk * T.lda + gm]) : T.A[(size_t)gm * T.lda + gk];
            As[r][cc] = T.s * v;
          }
          for (int e = threadIdx.x; e < 16 * 64; e += 256) {
            const int r = e >> 6, cc = e & 63;
            const int gk = k0 + r, gn = n0 + cc;
            Bs[r][cc] = (gk < K && gn < Ndim) ? T.B[(size_t)gk * T.ldb + gn] : cx<R>(0, 0);
          }
          __syncthreads();
#pragma unroll 4
          for (int kk = 0; kk < 16; ++kk) {
            Cx<R> a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[ty + 16 * i][kk];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
              for (int j = 0; j < 4; ++j) cmac(acc[i][j], a[i], b[j]);
          }
          __syncthreads();
        }
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int gm = m0 + ty + 16 * i, gn = n0 + tx + 16 * j;
          if (gm < Mdim && gn < Ndim) C[(size_t)gm * ldc + gn] = acc[i][j];
        }
    }
}

// --------------------------------------------------------- right environments
// R_n = [1]; R_k = sum_i B_k^i R_{k+1} B_k^{i+}; Bhat_k^i = B_k^i R_{k+1} (same layout as B_k).
template <class R>
__global__ void __launch_bounds__(256) k_right_envs(DevMPS m, int slot, Cx<R>* Renv, Cx<R>* Bhat) {
  __shared__ Cx<R> As[64][17];
  __shared__ Cx<R> Bs[16][65];
  const int n = m.n, chi2 = m.chi * m.chi;
  const Cx<R>* Bslot = (const Cx<R>*)m.B + (size_t)slot * m.slot_elems;
  const int* rank = m.rank + (size_t)slot * (n + 1);
  if (threadIdx.x == 0) Renv[(size_t)n * chi2] = cx<R>(1, 0);
  __syncthreads();
  for (int k = n - 1; k >= 0; --k) {
    const int Dl = rank[k], Dr = rank[k + 1];
    const Cx<R>* Bk = Bslot + m.site_off[k];
    Cx<R>* Bh = Bhat + m.site_off[k];
    const Cx<R>* Rn = Renv + (size_t)(k + 1) * chi2;
    for (int i = 0; i < 2; ++i) {  // Bhat^i = B^i R_{k+1}: (Dl x Dr)(Dr x Dr)
      GemmTerm<R> t{Bk + i * Dr, 2 * Dr, false, Rn, Dr, cx<R>(1, 0)};
      block_gemm<R>(Dl, Dr, Dr, &t, 1, Bh + i * Dr, 2 * Dr, As, Bs);
      __syncthreads();
    }
    // R_k = sum_i Bhat^i (B^i)^+ : (Dl x Dr)(Dr x Dl). As a product with A = Bhat^i and
    // B = (B^i)^+ we use C^T-free form: R_k[a][a'] = sum_b Bhat[a][b] conj(B[a'][b]).
    Cx<R>* Rk = Renv + (size_t)k * chi2;
    for (int e = threadIdx.x; e < Dl * Dl; e += 256) {
      const int a = e / Dl, ap = e - a * Dl;
      Cx<R> acc = cx<R>(0, 0);
      for (int i = 0; i < 2; ++i) {
        const Cx<R>* hr = Bh + (size_t)(2 * a + i) * Dr;
        const Cx<R>* br = Bk + (size_t)(2 * ap + i) * Dr;
        for (int b = 0; b < Dr; ++b) cmac(acc, hr[b], conj(br[b]));
      }
      Rk[e] = acc;
    }
    __syncthreads();
  }
}

cudaError_t launch_right_envs(const DevMPS& m, int prec, int slot, MeasDev& w, cudaStream_t st) {
  if (prec == MPS_PREC_FP64)
    k_right_envs<double><<<1, 256, 0, st>>>(m, slot, (Cx<double>*)w.R, (Cx<double>*)w.Bhat);
  else
    k_right_envs<float><<<1, 256, 0, st>>>(m, slot, (Cx<float>*)w.R, (Cx<float>*)w.Bhat);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ trie level
// Pauli letter -> the two (i, j, sigma_ij) entries of its 2x2 matrix.
template <class R>
__device__ __forceinline__ void letter_entries(uint8_t l, int* ii, int* jj, Cx<R>* s) {
  switch (l) {
    case 0: ii[0] = 0; jj[0] = 0; s[0] = cx<R>(1, 0); ii[1] = 1; jj[1] = 1; s[1] = cx<R>(1, 0); break;
    case 1: ii[0] = 0; jj[0] = 1; s[0] = cx<R>(1, 0); ii[1] = 1; jj[1] = 0; s[1] = cx<R>(1, 0); break;
    case 2: ii[0] = 0; jj[0] = 1; s[0] = cx<R>(0, -1); ii[1] = 1; jj[1] = 0; s[1] = cx<R>(0, 1); break;
    default: ii[0] = 0; jj[0] = 0; s[0] = cx<R>(1, 0); ii[1] = 1; jj[1] = 1; s[1] = cx<R>(-1, 0); break;
  }
}

// T_j[u] = L_k[u] B_k^j  (Dk x Dk)(Dk x Dk1), grid (nodes, 2)
template <class R>
__global__ void __launch_bounds__(256) k_level_T(DevMPS m, int slot, int k, const Cx<R>* Lin, Cx<R>* T) {
  __shared__ Cx<R> As[64][17];
  __shared__ Cx<R> Bs[16][65];
  const int u = blockIdx.x, j = blockIdx.y;
  const int chi2 = m.chi * m.chi;
  const int* rank = m.rank + (size_t)slot * (m.n + 1);
  const int Dk = rank[k], Dk1 = rank[k + 1];
  const Cx<R>* Bk = (const Cx<R>*)m.B + (size_t)slot * m.slot_elems + m.site_off[k];
  GemmTerm<R> t{Lin + (size_t)u * chi2, Dk, false, Bk + j * Dk1, 2 * Dk1, cx<R>(1, 0)};
  block_gemm<R>(Dk, Dk1, Dk, &t, 1, T + ((size_t)u * 2 + j) * chi2, Dk1, As, Bs);
}

// L_{k+1}[c] = sum_ij sigma_ij (B_k^i)^+ T_j[parent(c)]
template <class R>
__global__ void __launch_bounds__(256) k_level_child(DevMPS m, int slot, int k, const int32_t* parent,
                                                     const uint8_t* edge, const Cx<R>* T, Cx<R>* Lout) {
  __shared__ Cx<R> As[64][17];
  __shared__ Cx<R> Bs[16][65];
  const int c = blockIdx.x;
  const int chi2 = m.chi * m.chi;
  const int* rank = m.rank + (size_t)slot * (m.n + 1);
  const int Dk = rank[k], Dk1 = rank[k + 1];
  const Cx<R>* Bk = (const Cx<R>*)m.B + (size_t)slot * m.slot_elems + m.site_off[k];
  const int u = parent[c];
  int ii[2], jj[2];
  Cx<R> sg[2];
  letter_entries<R>(edge[c], ii, jj, sg);
  GemmTerm<R> t[2];
  for (int e = 0; e < 2; ++e)
    t[e] = GemmTerm<R>{Bk + ii[e] * Dk1, 2 * Dk1, true, T + ((size_t)u * 2 + jj[e]) * chi2, Dk1, sg[e]};
  block_gemm<R>(Dk1, Dk1, Dk, t, 2, Lout + (size_t)c * chi2, Dk1, As, Bs);
}

// <P> (unnormalised) = sum_ij sigma_ij <Bhat_k^i, T_j[node]>_F, FP64 accumulation
template <class R>
__global__ void __launch_bounds__(256) k_level_close(DevMPS m, int slot, int k, const int32_t* cnode,
                                                     const uint8_t* cletter, const int32_t* cterm,
                                                     const Cx<R>* T, const Cx<R>* Bhat, double* vals) {
  __shared__ double red[2][8];
  const int c = blockIdx.x;
  const int chi2 = m.chi * m.chi;
  const int* rank = m.rank + (size_t)slot * (m.n + 1);
  const int Dk = rank[k], Dk1 = rank[k + 1];
  const Cx<R>* Bh = Bhat + m.site_off[k];
  const int u = cnode[c];
  int ii[2], jj[2];
  Cx<R> sg[2];
  letter_entries<R>(cletter[c], ii, jj, sg);
  double re = 0.0, im = 0.0;
  for (int e = 0; e < 2; ++e) {
    const Cx<R>* Tj = T + ((size_t)u * 2 + jj[e]) * chi2;
    double pr = 0.0, pi = 0.0;
    for (int idx = threadIdx.x; idx < Dk * Dk1; idx += 256) {
      const int a = idx / Dk1, b = idx - a * Dk1;
      const Cx<R> h = Bh[(size_t)(2 * a + ii[e]) * Dk1 + b];
      const Cx<R> tv = Tj[idx];
      // conj(h) * tv
      pr += (double)h.x * tv.x + (double)h.y * tv.y;
      pi += (double)h.x * tv.y - (double)h.y * tv.x;
    }
    re += (double)sg[e].x * pr - (double)sg[e].y * pi;
    im += (double)sg[e].x * pi + (double)sg[e].y * pr;
  }
  for (int o = 16; o > 0; o >>= 1) {
    re += __shfl_xor_sync(0xffffffffu, re, o);
    im += __shfl_xor_sync(0xffffffffu, im, o);
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = re;
    red[1][threadIdx.x >> 5] = im;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0, b = 0;
    for (int w = 0; w < 8; ++w) {
      a += red[0][w];
      b += red[1][w];
    }
    vals[2 * (size_t)cterm[c]] = a;
    vals[2 * (size_t)cterm[c] + 1] = b;
  }
}

template <class R>
static cudaError_t launch_level_t(const DevMPS& m, int slot, MeasDev& w, int k, const TrieLevelDev& lv,
                                  int parity, cudaStream_t st, int* launches) {
  const Cx<R>* Lin = (const Cx<R>*)w.L[parity];
  Cx<R>* Lout = (Cx<R>*)w.L[parity ^ 1];
  Cx<R>* T = (Cx<R>*)w.T;
  if (lv.n_nodes > 0) {
    k_level_T<R><<<dim3(lv.n_nodes, 2), 256, 0, st>>>(m, slot, k, Lin, T);
    ++*launches;
  }
  if (lv.n_closes > 0) {
    k_level_close<R><<<lv.n_closes, 256, 0, st>>>(m, slot, k, lv.close_node, lv.close_letter, lv.close_term,
                                                   T, (const Cx<R>*)w.Bhat, w.vals);
    ++*launches;
  }
  if (lv.n_children > 0) {
    k_level_child<R><<<lv.n_children, 256, 0, st>>>(m, slot, k, lv.parent, lv.edge, T, Lout);
    ++*launches;
  }
  return cudaGetLastError();
}

cudaError_t launch_level(const DevMPS& m, int prec, int slot, MeasDev& w, int k, const TrieLevelDev& lv,
                         int parity, cudaStream_t st, int* launches) {
  if (prec == MPS_PREC_FP64) return launch_level_t<double>(m, slot, w, k, lv, parity, st, launches);
  return launch_level_t<float>(m, slot, w, k, lv, parity, st, launches);
}

// ------------------------------------------------------------------ energy sum
__device__ __forceinline__ void neumaier_add(double& s, double& c, double v) {
  const double t = s + v;
  if (fabs(s) >= fabs(v))
    c += (s - t) + v;
  else
    c += (v - t) + s;
  s = t;
}

template <class R>
__global__ void __launch_bounds__(1024) k_energy_sum(int64_t n_terms, const double* coeff, const double* vals,
                                                     const Cx<R>* R0, double id_coeff, int64_t id_term,
                                                     double* out) {
  __shared__ double ps[1024], pc[1024];
  const double norm = (double)R0[0].x;
  const int64_t chunk = (n_terms + 1023) / 1024;
  const int64_t b = (int64_t)threadIdx.x * chunk, e = min(n_terms, b + chunk);
  double s = 0.0, c = 0.0;
  for (int64_t t = b; t < e; ++t) {
    double re, im;
    if (t == id_term) {
      re = 1.0;
      im = 0.0;
    } else {
      re = vals[2 * t] / norm;
      im = vals[2 * t + 1] / norm;
      neumaier_add(s, c, coeff[t] * re);
    }
    out[4 + 2 * t] = re;
    out[5 + 2 * t] = im;
  }
  ps[threadIdx.x] = s;
  pc[threadIdx.x] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    double S = 0.0, Cc = 0.0;
    for (int i = 0; i < 1024; ++i) {
      neumaier_add(S, Cc, ps[i]);
      neumaier_add(S, Cc, pc[i]);
    }
    neumaier_add(S, Cc, id_coeff);
    out[0] = S + Cc;
    out[1] = norm;
  }
}

cudaError_t launch_energy_sum(const DevMPS& m, int prec, int slot, MeasDev& w, int64_t n_terms,
                              const double* coeff_dev, double id_coeff, int64_t id_term, cudaStream_t st) {
  (void)m;
  (void)slot;
  if (prec == MPS_PREC_FP64)
    k_energy_sum<double><<<1, 1024, 0, st>>>(n_terms, coeff_dev, w.vals, (const Cx<double>*)w.R, id_coeff,
                                             id_term, w.out);
  else
    k_energy_sum<float><<<1, 1024, 0, st>>>(n_terms, coeff_dev, w.vals, (const Cx<float>*)w.R, id_coeff,
                                            id_term, w.out);
  return cudaGetLastError();
}

}  // namespace mpsvqe
