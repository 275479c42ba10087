// CUDA kernels of the MPS-VQE hot path for sm_103a (GB300).
//
//  k_reset        product-state reference (Sec. III-D: X gates on the occupied qubits).
//  k_circuit      persistent per-slot gate engine: for each two-site gate,
//                 Eq. (7) contraction, Eq. (8) row scaling by lambda_{n-1}, Eq. (9)
//                 truncated SVD (bidiagonal route of svd.cuh, one-sided Jacobi for
//                 spectra that stay degenerate), Eq. (10) updates.
//  k_right_envs   right identity environments R_k and B^_k = B_k R_{k+1}.
//  k_level_T/child/close   one level of the Pauli-string prefix trie (Eq. 11 generalised).
//  k_energy_sum   E = sum_i a_i <P_i> (Eq. 2) with Neumaier compensation in FP64.
#include <cfloat>
#include <cmath>
#include <cstdint>
#include <mutex>

#include "cx.cuh"
#include "kernels.cuh"
#include "svd.cuh"

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
  if (threadIdx.x < kStatWords) m.stat[s * kStatWords + threadIdx.x] = (threadIdx.x == 2) ? 1 : 0;
}

cudaError_t launch_reset(const DevMPS& m, int prec, int slot0, int count, const uint8_t* occ,
                         cudaStream_t st) {
  if (prec == MPS_PREC_FP64)
    k_reset<double><<<count, 128, 0, st>>>(m, slot0, occ);
  else
    k_reset<float><<<count, 128, 0, st>>>(m, slot0, occ);
  return cudaGetLastError();
}

// ------------------------------------------------------------ small tiled GEMM
// C (Mdim x Ndim, ldc) = sum_t s_t opA_t(A_t) opB_t(B_t) with NTH threads (256 or 512)
// and 64x64 tiles. opA: A stored Mdim x K (lda), or K x Mdim used as A^H (conjT).
// opB: B stored K x Ndim (ldb), or Ndim x K used as B^T (transB); conjB conjugates the
// entries of B as they are loaded.
template <class R>
struct GemmTerm {
  const Cx<R>* A;
  int lda;
  bool conjT;
  const Cx<R>* B;
  int ldb;
  Cx<R> s;
  bool transB;
  bool conjB = false;
};

// One 64 x 64 output tile at (m0, n0).
template <class R, int NTH>
__device__ void gemm_tile(int m0, int n0, int Mdim, int Ndim, int K, const GemmTerm<R>* terms, int nterm, Cx<R>* C,
                          int ldc, Cx<R> (*As)[17], Cx<R> (*Bs)[65]) {
  constexpr int TY = NTH / 16, RPT = 64 / TY;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  Cx<R> acc[RPT][4];
#pragma unroll
  for (int i = 0; i < RPT; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = cx<R>(0, 0);
  for (int t = 0; t < nterm; ++t) {
    const GemmTerm<R> T = terms[t];
    for (int k0 = 0; k0 < K; k0 += 16) {
      for (int e = threadIdx.x; e < 64 * 16; e += NTH) {
        const int r = e >> 4, cc = e & 15;
        const int gm = m0 + r, gk = k0 + cc;
        Cx<R> v = cx<R>(0, 0);
        if (gm < Mdim && gk < K) v = T.conjT ? conj(T.A[(size_t)gk * T.lda + gm]) : T.A[(size_t)gm * T.lda + gk];
        As[r][cc] = T.s * v;
      }
      for (int e = threadIdx.x; e < 16 * 64; e += NTH) {
        const int r = T.transB ? (e & 15) : (e >> 6), cc = T.transB ? (e >> 4) : (e & 63);
        const int gk = k0 + r, gn = n0 + cc;
        Cx<R> v = cx<R>(0, 0);
        if (gk < K && gn < Ndim) v = T.transB ? T.B[(size_t)gn * T.ldb + gk] : T.B[(size_t)gk * T.ldb + gn];
        Bs[r][cc] = T.conjB ? conj(v) : v;
      }
      __syncthreads();
#pragma unroll 4
      for (int kk = 0; kk < 16; ++kk) {
        Cx<R> a[RPT], b[4];
#pragma unroll
        for (int i = 0; i < RPT; ++i) a[i] = As[ty + TY * i][kk];
#pragma unroll
        for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
        for (int i = 0; i < RPT; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) cmac(acc[i][j], a[i], b[j]);
      }
      __syncthreads();
    }
  }
#pragma unroll
  for (int i = 0; i < RPT; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gm = m0 + ty + TY * i, gn = n0 + tx + 16 * j;
      if (gm < Mdim && gn < Ndim) C[(size_t)gm * ldc + gn] = acc[i][j];
    }
}

template <class R, int NTH>
__device__ void block_gemm(int Mdim, int Ndim, int K, const GemmTerm<R>* terms, int nterm, Cx<R>* C, int ldc,
                           Cx<R> (*As)[17], Cx<R> (*Bs)[65]) {
  for (int m0 = 0; m0 < Mdim; m0 += 64)
    for (int n0 = 0; n0 < Ndim; n0 += 64) gemm_tile<R, NTH>(m0, n0, Mdim, Ndim, K, terms, nterm, C, ldc, As, Bs);
}

// The same product spread over a grid: one 64 x 64 tile per thread block, blockIdx.z
// selecting one of up to four independent products.
template <class R>
struct GridGemm {
  GemmTerm<R> t[4][2];
  int nterm;
  Cx<R>* C[4];
  int ldc, M, N, K;
};

template <class R>
__global__ void __launch_bounds__(256) k_cgemm_grid(GridGemm<R> g) {
  __shared__ Cx<R> As[64][17];
  __shared__ Cx<R> Bs[16][65];
  const int z = blockIdx.z;
  gemm_tile<R, 256>(blockIdx.y * 64, blockIdx.x * 64, g.M, g.N, g.K, g.t[z], g.nterm, g.C[z], g.ldc, As, Bs);
}

// ------------------------------------------------ compensated re-orthonormalisation
// Error-free transformations in FP32: TwoSum (Knuth) and the FMA form of TwoProd, the
// building blocks of the compensated dot product "Dot2" (Ogita, Rump and Oishi, 2005),
// which returns a dot product as accurate as if it were accumulated in twice the
// working precision. The _rn intrinsics keep the compiler from contracting the
// products into the sums, which would break the error-free transformations.
__device__ __forceinline__ void dot2_acc(float a, float b, float& s, float& c) {
  const float p = __fmul_rn(a, b);
  const float ep = fmaf(a, b, -p);
  const float t = __fadd_rn(s, p);
  const float bv = __fsub_rn(t, s);
  const float et = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bv)), __fsub_rn(p, bv));
  s = t;
  c = __fadd_rn(c, __fadd_rn(ep, et));
}

// Rows x_0..x_{k-1} (length len, row stride ldx) of X are close to orthonormal; one
// Newton-Schulz step X <- X - (1/2) E X with E = X X^H - I pulls them to
// orthonormality up to the rounding of the update. E is tiny (a few 1e-7 after the
// FP32 back-transformation), so it is only useful if the Gram matrix is accurate far
// below FP32 resolution: each entry is a Dot2 sum. Xs (k x ldx) and Es (k x k) are
// staging areas; the result is written to out (row stride len).
template <int NT>
__device__ void newton_schulz_rows(const Cx<float>* X, int k, int len, Cx<float>* Xs, int ldx, Cx<float>* Es,
                                   Cx<float>* out) {
  const int tid = threadIdx.x;
  for (int idx = tid; idx < k * len; idx += NT) {
    const int i = idx / len, q = idx - i * len;
    Xs[(size_t)i * ldx + q] = X[idx];
  }
  __syncthreads();
  const int npair = k * (k + 1) / 2;
  for (int e = tid; e < npair; e += NT) {
    // e -> (i, j), i <= j, rows of the upper triangle in order
    int i = (int)((2.0f * k + 1.0f - sqrtf((2.0f * k + 1.0f) * (2.0f * k + 1.0f) - 8.0f * e)) * 0.5f);
    while (i > 0 && i * k - i * (i - 1) / 2 > e) --i;
    while ((i + 1) * k - (i + 1) * i / 2 <= e) ++i;
    const int j = i + (e - (i * k - i * (i - 1) / 2));
    const Cx<float>* xi = Xs + (size_t)i * ldx;
    const Cx<float>* xj = Xs + (size_t)j * ldx;
    float sr = 0.f, cr = 0.f, si = 0.f, ci = 0.f;
    for (int q = 0; q < len; ++q) {
      const Cx<float> a = xi[q], b = xj[q];
      // G_ij = sum_q a conj(b)
      dot2_acc(a.x, b.x, sr, cr);
      dot2_acc(a.y, b.y, sr, cr);
      dot2_acc(a.y, b.x, si, ci);
      dot2_acc(-a.x, b.y, si, ci);
    }
    // the diagonal is within 1e-6 of 1, so sr - 1 is exact (Sterbenz)
    const float er = __fadd_rn(i == j ? __fsub_rn(sr, 1.0f) : sr, cr);
    const float ei = i == j ? 0.0f : __fadd_rn(si, ci);
    Es[(size_t)i * k + j] = cx<float>(er, ei);
    Es[(size_t)j * k + i] = cx<float>(er, -ei);
  }
  __syncthreads();
  for (int idx = tid; idx < k * len; idx += NT) {
    const int i = idx / len, q = idx - i * len;
    Cx<float> acc = cx<float>(0.f, 0.f);
    for (int j = 0; j < k; ++j) cmac(acc, Es[(size_t)i * k + j], Xs[(size_t)j * ldx + q]);
    const Cx<float> x = Xs[(size_t)i * ldx + q];
    out[idx] = cx<float>(x.x - 0.5f * acc.x, x.y - 0.5f * acc.y);
  }
  __syncthreads();
}

// ---------------------------------------------------------------- gate engine
//
// Shared-memory plan of k_circuit for bond cap chi (mmax = 2 chi), NT threads:
//   [head]  U (16 complex double), U in R, FP64 reduction slots, misc ints
//   [svd]   dd, ee, b (2 mmax), b2 (2 mmax), tauL, tauR, sig, lo, hi, coef (mmax each),
//           cnt, xs, bisection grid (NT each), iteration table (chi)
//   [W]     chi rows of real singular vectors of the bidiagonal (stride ldw) and a
//           chi x chi Gram area
//   [T]     (mmax + 16) x mmax complex: the tall orientation of M', later the tiles of
//           the site-update GEMM
// When W and T do not both fit they live in the slot's global workspace (L2
// resident) and only the GEMM tiles stay in shared memory.
// Algorithmic real flops of one gate step, counted as the textbook dense algorithms:
// contraction theta = B_n B_{n+1} (2 rl x rm x 2 rr complex MACs), the 4x4 gate on
// (i, j), Golub-Reinsch SVD of the (m x n) complex M' computing singular values and
// right vectors (4 (4 m n^2 + 8 n^3) real flops for m >= n, roles swapped otherwise),
// and the site update B_n = M V^H (2 rl x 2 rr x k complex MACs). A complex MAC is 8.
__device__ __forceinline__ double flops_per_gate(int rl, int rm, int rr, int k) {
  const double m = 2.0 * rl, n = 2.0 * rr;
  const double big = m >= n ? m : n, small = m >= n ? n : m;
  const double contract = 8.0 * m * rm * n + 8.0 * 4.0 * m * n;
  const double svd = 4.0 * (4.0 * big * small * small + 8.0 * small * small * small);
  const double update = 8.0 * m * n * k;
  return contract + svd + update;
}

// Capacity of bond b (b = -1 and b = n-1 are the trivial outer bonds): the largest rank
// an n-site MPS with bond cap chi can have there, min(chi, 2^min(b+1, n-1-b)).
__device__ __forceinline__ int bond_cap(int b, int n, int chi) {
  if (b < 0 || b >= n - 1) return 1;
  const int e = min(min(b + 1, n - 1 - b), 30);
  return min(chi, 1 << e);
}

template <class R>
struct EngineLayout {
  size_t head, svd, ldw, w_off, w_bytes, t_off, t_bytes, g_bytes, total;
  bool w_smem, t_smem;
  __host__ __device__ EngineLayout(int chi, int nt) {
    const size_t mmax = 2 * (size_t)chi;
    head = 256 + 256 + (size_t)(nt / 32 + 2) * 8 + 64;
    head = (head + 255) & ~(size_t)255;
    svd = sizeof(R) * (2 * mmax + 4 * mmax + 5 * mmax) + sizeof(Cx<R>) * 2 * mmax + (sizeof(R) + 4) * nt +
          (8 + 4) * mmax + 16 + sizeof(R) * nt + 4 * (size_t)chi + 16;
    svd = (svd + 255) & ~(size_t)255;
    // singular-vector rows: stride = 8 (mod 32) entries, so that the 8-lane dot products
    // of four rows in one warp start in four different bank groups
    ldw = mmax + 1;
    ldw += (8 + 32 - (ldw & 31)) & 31;
    w_bytes = sizeof(R) * ((size_t)chi * ldw + (size_t)chi * chi);   // W rows + Gram
    w_bytes = (w_bytes + 255) & ~(size_t)255;
    t_bytes = sizeof(Cx<R>) * (mmax + 16) * mmax;
    // the site-update GEMM tiles (64x17 + 16x65 complex) reuse the T area (T is dead by
    // then) or take their own area when T lives in global memory
    g_bytes = sizeof(Cx<R>) * (64 * 17 + 16 * 65);
    const size_t cap = 227 * 1024 - 1024;
    w_off = head + svd;
    // W goes to shared memory only if the GEMM tiles still fit behind it
    w_smem = w_off + w_bytes + g_bytes <= cap;
    t_off = w_off + (w_smem ? w_bytes : 0);
    const size_t t_area = t_bytes > g_bytes ? t_bytes : g_bytes;
    t_smem = w_smem && t_off + t_area <= cap;
    total = t_off + (t_smem ? t_area : g_bytes);
  }
};

// TS: the singular-vector area and T live in shared memory (the layout decides on the
// host); a compile-time placement lets the compiler use shared-memory instructions.
template <class R, int NT, bool RAW = false, bool TS = true>
__global__ void __launch_bounds__(NT) k_circuit(DevMPS m, CircDev c, int64_t g0, int64_t g1,
                                                int slot0, const double* theta, double cutoff,
                                                int max_sweeps) {
  extern __shared__ __align__(256) unsigned char smem[];
  const EngineLayout<R> L(m.chi, NT);
  const int s = slot0 + blockIdx.x;
  const int n = m.n, chi = m.chi, mmax = 2 * chi;
  Cx<R>* Bslot = (Cx<R>*)m.B + (size_t)s * m.slot_elems;
  double* lam = m.lam + (size_t)s * (n - 1) * chi;
  int* rank = m.rank + (size_t)s * (n + 1);
  Cx<R>* W = (Cx<R>*)m.work_M + (size_t)s * mmax * mmax;
  R* scratch = (R*)((double*)m.work_S + (size_t)s * 16 * chi * chi);  // twisted-factorisation rows

  Cx<double>* U = (Cx<double>*)smem;
  Cx<R>* Uf = (Cx<R>*)(smem + 256);
  double* red = (double*)(smem + 512);
  int* misc = (int*)(red + NT / 32 + 2);
  R* dd = (R*)(smem + L.head);
  R* ee = dd + mmax;
  R* bb = ee + mmax;          // 2 mmax
  R* b2 = bb + 2 * mmax;      // 2 mmax
  R* sig = b2 + 2 * mmax;
  R* lo = sig + mmax;
  R* hi = lo + mmax;
  R* coef = hi + mmax;
  R* xs = coef + mmax;        // NT
  Cx<R>* tauL = (Cx<R>*)(xs + NT);
  Cx<R>* tauR = tauL + mmax;
  int* cnt = (int*)(tauR + mmax);
  double* sig2d = (double*)(((uintptr_t)(cnt + NT) + 15) & ~(uintptr_t)15);
  int* order = (int*)(sig2d + mmax);
  R* grid = (R*)(order + mmax);              // NT log-spaced bisection shifts / smax
  int* iters_of = (int*)(grid + NT);         // bisection passes for kk = 1..chi
  Cx<R>(*gA)[17] = reinterpret_cast<Cx<R>(*)[17]>(smem + L.t_off);
  Cx<R>(*gB)[65] = reinterpret_cast<Cx<R>(*)[65]>(smem + L.t_off + sizeof(Cx<R>) * 64 * 17);
  const int ldw = (int)L.ldw;
  R* Wv = TS ? (R*)(smem + L.w_off) : (R*)((double*)m.work_S + (size_t)s * 16 * chi * chi + 8 * chi * chi);
  Cx<R>* T = TS ? (Cx<R>*)(smem + L.t_off) : (Cx<R>*)m.work_X + (size_t)s * mmax * (mmax + 16);
  const double* th = theta + (size_t)blockIdx.x * c.n_params;

  int st_max_iters = 0, st_max_rank = 1, st_bad = 0, st_nonfinite = 0, st_badarg = 0;
  if (threadIdx.x == 0) misc[2] = 0;
  {
    // per-launch tables: grid shifts over [10^-decades, 1] and, for kk targets, the
    // number of (NT/kk + 1)-fold refinement passes that reach the working precision
    constexpr bool kF64 = sizeof(R) == 8;
    const double decades = kF64 ? 15.0 : 8.0;
    grid[threadIdx.x] = (R)exp10(decades * (double)((int)threadIdx.x - (NT - 1)) / (double)(NT - 1));
    const double w0 = decades * 2.302585092994046 / (NT - 1);
    for (int kk = 1 + threadIdx.x; kk <= chi; kk += NT) {
      const int per = max(1, NT / kk);
      iters_of[kk - 1] = (int)ceil(log(w0 / (kF64 ? 2e-16 : 6e-8)) / log((double)(per + 1))) + 1;
    }
  }
  __syncthreads();
  unsigned long long ph[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  double alg_flops = 0.0;  // algorithmic real flops of the gate steps (see flops_per_gate)
  long long t_mark = clock64();
#define PHASE(i)                                   \
  do {                                             \
    if (threadIdx.x == 0) {                        \
      const long long now_ = clock64();            \
      ph[i] += (unsigned long long)(now_ - t_mark); \
      t_mark = now_;                               \
    }                                              \
  } while (0)
  double dw_acc = 0.0;

  const int64_t g_first = c.start_gate ? max(g0, c.start_gate[blockIdx.x]) : g0;
  const int64_t g_shift = c.shift_gate ? c.shift_gate[blockIdx.x] : -1;
  const double phi_shift = c.shift_phi ? c.shift_phi[blockIdx.x] : 0.0;
  for (int64_t g = g_first; g < g1; ++g) {
    GateRec gr;
    if constexpr (RAW) {
      gr.bond = c.raw_bond[g];
      gr.param = -1;
      gr.m0 = (int32_t)g;
    } else {
      gr = c.gates[g];
    }
    // (1) the 4x4 gate: fixed, or mats[m1] . Rz(phi) on one site . mats[m0]
    if (threadIdx.x < 16) {
      const int i = threadIdx.x >> 2, j = threadIdx.x & 3;
      const Cx<double>* A = (const Cx<double>*)c.mats + 16 * (size_t)gr.m0;
      Cx<double> u;
      if (gr.param < 0) {
        u = A[threadIdx.x];
      } else {
        const Cx<double>* P = (const Cx<double>*)c.mats + 16 * (size_t)gr.m1;
        const double half = 0.5 * (gr.scale * th[gr.param] + (g == g_shift ? phi_shift : 0.0));
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
    if constexpr (RAW) {
      // caller-owned device arrays: the bond and the three ranks it touches must lie
      // inside the site capacities before anything is indexed (uniform over the block)
      bool ok = bond >= 0 && bond <= n - 2;
      if (ok) {
        const int r0 = rank[bond], r1 = rank[bond + 1], r2 = rank[bond + 2];
        ok = r0 >= 1 && r0 <= bond_cap(bond - 1, n, chi) && r1 >= 1 && r1 <= bond_cap(bond, n, chi) && r2 >= 1 &&
             r2 <= bond_cap(bond + 1, n, chi);
      }
      if (!ok) {
        if (threadIdx.x == 0) st_badarg = 1;
        break;
      }
    }
    const int rl = rank[bond], rm = rank[bond + 1], rr = rank[bond + 2];
    const int mrows = 2 * rl, ncol = 2 * rr;
    const bool tall = mrows >= ncol;
    const int tr = tall ? mrows : ncol, tp = tall ? ncol : mrows;
    // leading dimension: 2 (mod 16) complex<float> entries, so that 16-lane column
    // walks and 8-column x 2-row walks of a half warp hit 16 distinct bank pairs;
    // odd for complex<double>, so that 8 consecutive columns of one row do too
    const int ld = sizeof(R) == 4 ? tr + ((18 - (tr & 15)) & 15) : tr + ((17 - (tr & 15)) & 15);
    Cx<R>* Bn = Bslot + m.site_off[bond];
    Cx<R>* Bn1 = Bslot + m.site_off[bond + 1];
    const double* laml = bond > 0 ? lam + (size_t)(bond - 1) * chi : nullptr;
    __syncthreads();

    // (2) Eq. (7): M[(a,i),(j,c)] = sum_{i'j'} U[ij,i'j'] sum_b B_n[a,i',b] B_{n+1}[b,j',c];
    //     W <- M; Eq. (8): M' = lambda_{n-1}[a] M, stored tall in T (M' or M'^H).
    //     Theta = B_n (2 r_l x r_m) . B_{n+1} (r_m x 2 r_r) by the tiled GEMM into W, then
    //     the gate on each (i, j) quad in place
    {
      GemmTerm<R> gt{Bn, rm, false, Bn1, 2 * rr, cx<R>(1, 0), false};
      block_gemm<R, NT>(mrows, ncol, rm, &gt, 1, W, ncol, gA, gB);
    }
    __syncthreads();
    double fro = 0.0;
    for (int it = threadIdx.x; it < rl * rr; it += NT) {
      const int a = it / rr, cc = it - a * rr;
      Cx<R>* w0 = W + (size_t)(2 * a) * ncol + cc;
      Cx<R>* w1 = w0 + ncol;
      const Cx<R> th4[4] = {w0[0], w0[rr], w1[0], w1[rr]};
      const R la = laml ? (R)laml[a] : R(1);
#pragma unroll
      for (int ij = 0; ij < 4; ++ij) {
        Cx<R> v = cx<R>(0, 0);
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) cmac(v, Uf[ij * 4 + kk], th4[kk]);
        const int row = 2 * a + (ij >> 1), col = (ij & 1) * rr + cc;
        W[(size_t)row * ncol + col] = v;
        const Cx<R> mv = la * v;
        if (tall)
          T[(size_t)col * ld + row] = mv;
        else
          T[(size_t)row * ld + col] = conj(mv);
        fro += (double)norm2(mv);
      }
    }
    for (int o = 16; o > 0; o >>= 1) fro += __shfl_xor_sync(0xffffffffu, fro, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = fro;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int w = 0; w < NT / 32; ++w) t += red[w];
      red[NT / 32] = t;
    }

    __syncthreads();
    // a NaN or Inf in M' (from corrupted inputs) would run through every later stage:
    // the gate is skipped, the state left as it was, and the host reports the count
    if (!(red[NT / 32] <= DBL_MAX)) {
      if (threadIdx.x == 0) ++st_nonfinite;
      continue;
    }
    PHASE(0);
    // (3) Eq. (9): bidiagonalise T = Q B P^H (B real); the reflector vectors are staged
    //     in the (not yet used) singular-vector buffer
    bidiagonalize<R, NT>(T, ld, tr, tp, dd, ee, tauL, tauR);
    PHASE(1);
    // Golub-Kahan tridiagonal off-diagonal b = (d0, e0, d1, e1, ..., d_{p-1})
    for (int i = threadIdx.x; i < 2 * tp - 1; i += NT) {
      const R v = (i & 1) ? ee[i >> 1] : dd[i >> 1];
      bb[i] = v;
      b2[i] = v * v;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
      R smax = 0;
      for (int i = threadIdx.x; i < 2 * tp; i += 32) {
        const R left = i > 0 ? rabs(bb[i - 1]) : R(0), right = i < 2 * tp - 1 ? rabs(bb[i]) : R(0);
        smax = fmax(smax, left + right);
      }
      for (int o = 16; o > 0; o >>= 1) smax = fmax(smax, __shfl_xor_sync(0xffffffffu, smax, o));
      if (threadIdx.x == 0) coef[0] = smax;
    }
    __syncthreads();
    const R smax = coef[0];
    // split the TGK where an off-diagonal is negligible (exact degeneracies live in
    // different blocks after this; the perturbation is below 4 eps ||B||)
    for (int i = threadIdx.x; i < 2 * tp - 1; i += NT)
      if (rabs(bb[i]) <= R(4) * Eps<R>::v * smax) {
        bb[i] = R(0);
        b2[i] = R(0);
      }
    __syncthreads();
    const int kk = min(chi, tp);
    const bool fp64 = sizeof(R) == 8;
    const int iters = iters_of[kk - 1];
    bisect_singular_values<R, NT>(b2, tp, smax, kk, iters, sig, lo, hi, cnt, xs, grid);
    if (threadIdx.x < 32) {
      // sig is descending: k = number of leading values above cutoff * sig_0
      const R s0 = sig[0];
      int cntk = 0;
      for (int t = threadIdx.x; t < kk; t += 32) cntk += (sig[t] > (R)cutoff * s0 && sig[t] > R(0));
      for (int o = 16; o > 0; o >>= 1) cntk += __shfl_xor_sync(0xffffffffu, cntk, o);
      if (threadIdx.x == 0) {
        const int k = cntk > 0 ? cntk : 1;
        misc[0] = k;
        st_max_rank = max(st_max_rank, k);
        st_max_iters = max(st_max_iters, iters);
      }
    }
    __syncthreads();
    const int k = misc[0];
    PHASE(2);

    // (4) singular vectors of B from twisted factorisations, then CGS2
    const R tiny = smax * (fp64 ? R(1e-300) : R(1e-30)) + (fp64 ? R(1e-300) : R(1e-37));
    for (int t = threadIdx.x; t < k; t += NT) {
      // scratch rows interleaved over the k threads: dp at [i k + t], dm after 2p k entries
      R* dp = scratch + t;
      int s0, e0;
      const R delta = R(8) * (hi[t] - lo[t]) + R(4) * Eps<R>::v * smax;
      owning_block<R>(b2, 2 * tp, sig, t, delta, tiny, &s0, &e0);
      twisted_vector<R>(bb, tp, s0, e0, sig[t], tiny, dp, dp + (size_t)2 * tp * k, k, tall ? 0 : 1,
                        Wv + (size_t)t * ldw);
    }
    if (threadIdx.x == 0) misc[1] = 0;
    __syncthreads();
    PHASE(3);
    orthonormalize_rows_block<R, NT>(Wv, ldw, k, tp, Wv + (size_t)chi * ldw, xs, &misc[1]);
    PHASE(4);
    Cx<R>* xout = (Cx<R>*)scratch;               // k x ncol right singular vectors v_t
    int kf = k;                                  // kept count of the path taken
    if (misc[1] == 0) {
      // (5) back-transformation: x_t = P w_t (tall) or Q [w_t; 0] (wide) is the right
      //     singular vector v_t of M' (length ncol); 16 entries per thread. First the
      //     stored reflectors are turned into their vectors in place (tail times scale,
      //     conjugated for the right reflectors; 1 at the start), which the unused
      //     factor array of the other side holds meanwhile.
      const int nref = tall ? tp - 1 : tp;
      Cx<R>* scl = tall ? tauL : tauR;
      for (int jr = threadIdx.x; jr < nref; jr += NT)
        scl[jr] = tall ? T[(size_t)(jr + 1) * ld + jr] : T[(size_t)jr * ld + jr];
      __syncthreads();
      for (int idx = threadIdx.x; idx < nref * ncol; idx += NT) {
        // consecutive threads walk consecutive shared-memory entries
        const int jr = tall ? idx % nref : idx / ncol, q = tall ? idx / nref : idx % ncol;
        const int start = tall ? jr + 1 : jr;
        if (q < start) continue;
        Cx<R>& e = tall ? T[(size_t)q * ld + jr] : T[(size_t)jr * ld + q];
        e = q == start ? cx<R>(1, 0) : (tall ? conj(e) * scl[jr] : e * scl[jr]);
      }
      __syncthreads();
      int LV = 8;
      while (LV < 32 && LV * 16 < ncol) LV <<= 1;
      const int vpp = NT / LV;
      const int grp = threadIdx.x / LV, l = threadIdx.x - grp * LV;
      for (int vb = 0; vb < k; vb += vpp) {
        const int t = vb + grp;
        const bool act = t < k;
        Cx<R> x[16];
#pragma unroll
        for (int e = 0; e < 16; ++e) {
          const int q = l + e * LV;
          R val = R(0);
          if (act && q < tp) val = Wv[(size_t)t * ldw + q];
          x[e] = cx<R>(val, R(0));
        }
        for (int jr = nref - 1; jr >= 0; --jr) {
          const int start = tall ? jr + 1 : jr;
          const Cx<R> tau = tall ? tauR[jr] : tauL[jr];
          // every entry is processed (zeros above the start): skipping the leading
          // entries with a block-uniform test was measured slower than the work saved
          Cx<R> hv[16];
          Cx<R> sdot = cx<R>(0, 0);
#pragma unroll
          for (int e = 0; e < 16; ++e) {
            const int q = l + e * LV;
            hv[e] = (q >= start && q < ncol) ? (tall ? T[(size_t)q * ld + jr] : T[(size_t)jr * ld + q])
                                             : cx<R>(0, 0);
            cmac_conj(sdot, hv[e], x[e]);
          }
          for (int o = 1; o < LV; o <<= 1) {
            sdot.x += __shfl_xor_sync(0xffffffffu, sdot.x, o, LV);
            sdot.y += __shfl_xor_sync(0xffffffffu, sdot.y, o, LV);
          }
          const Cx<R> f = tau * sdot;
#pragma unroll
          for (int e = 0; e < 16; ++e) x[e] = x[e] - f * hv[e];
        }
        if (act) {
#pragma unroll
          for (int e = 0; e < 16; ++e) {
            const int q = l + e * LV;
            if (q < ncol) xout[(size_t)t * ncol + q] = x[e];
          }
        }
      }
      if (threadIdx.x == 0) {
        double kept = 0.0;
        for (int t = 0; t < k; ++t) kept += (double)sig[t] * (double)sig[t];
        const double total = red[NT / 32];
        if (total > 0.0) dw_acc += fmax(0.0, total - kept) / total;
      }
      __syncthreads();
    } else {
      // (5') degenerate spectrum without a split: one-sided Jacobi on the columns
      //      X = conj rows of M' (rebuilt from W and lambda_{n-1}) in the T buffer
      ++st_bad;
      const int ldx = ncol + 1;
      Cx<R>* X = T;
      for (int idx = threadIdx.x; idx < mrows * ncol; idx += NT) {
        const int row = idx / ncol, q = idx - row * ncol;
        const R la = laml ? (R)laml[row >> 1] : R(1);
        X[(size_t)row * ldx + q] = conj(la * W[(size_t)row * ncol + q]);
      }
      __syncthreads();
      const double zero2 = (double)Eps<R>::v * Eps<R>::v * 16.0 * red[NT / 32];
      jacobi_columns<R, NT, 8>(X, ldx, mrows, ncol, zero2, max_sweeps, &misc[2]);
      for (int p = threadIdx.x; p < mrows; p += NT) {
        double acc = 0.0;
        for (int q = 0; q < ncol; ++q) acc += (double)norm2(X[(size_t)p * ldx + q]);
        sig2d[p] = acc;
      }
      __syncthreads();
      for (int p = threadIdx.x; p < mrows; p += NT) {
        const double v = sig2d[p];
        int rk = 0;
        for (int q = 0; q < mrows; ++q) {
          const double w = sig2d[q];
          rk += (w > v) || (w == v && q < p);
        }
        order[rk] = p;
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        const double s0 = sig2d[order[0]];
        const int kmax = min(chi, min(mrows, ncol));
        int kk2 = 0;
        while (kk2 < kmax && sig2d[order[kk2]] > cutoff * cutoff * s0) ++kk2;
        if (kk2 == 0) kk2 = 1;
        double total = 0.0, dropped = 0.0;
        for (int t = 0; t < mrows; ++t) total += sig2d[order[t]];
        for (int t = kk2; t < mrows; ++t) dropped += sig2d[order[t]];
        if (total > 0.0) dw_acc += dropped / total;
        misc[0] = kk2;
        st_max_rank = max(st_max_rank, kk2);
      }
      __syncthreads();
      kf = misc[0];
      for (int t = threadIdx.x; t < kf; t += NT) sig[t] = (R)sqrt(sig2d[order[t]]);
      for (int idx = threadIdx.x; idx < kf * ncol; idx += NT) {
        const int t = idx / ncol, q = idx - t * ncol;
        const int p = order[t];
        const R inv = (R)(1.0 / sqrt(sig2d[p]));
        xout[idx] = inv * X[(size_t)p * ldx + q];   // column p of X = sigma * v_t
      }
      __syncthreads();
    }
    if constexpr (sizeof(R) == 4) {
      // (5b) mixed precision: the FP32 back-transformation leaves the rows of V
      //      orthonormal only to a few 1e-7; over a long circuit that defect, not the
      //      rounding of the stored tensors, dominates the energy error. One compensated
      //      Newton-Schulz step brings it down to the storage rounding. T is dead here
      //      and stages V and E = V V^H - I.
      const int ldx = ncol + 1;
      newton_schulz_rows<NT>(xout, kf, ncol, T, ldx, T + (size_t)kf * ldx, xout);
    }
    PHASE(5);
    // (6) Eq. (10): B_{n+1} <- V (row t = v_t^H), B_n <- M V^H (column t = M v_t),
    //     lambda_n <- sigma
    for (int idx = threadIdx.x; idx < kf * ncol; idx += NT) Bn1[idx] = conj(xout[idx]);
    {
      GemmTerm<R> gt{W, ncol, false, xout, ncol, cx<R>(1, 0), true};
      block_gemm<R, NT>(mrows, kf, ncol, &gt, 1, Bn, kf, gA, gB);
    }
    for (int t = threadIdx.x; t < kf; t += NT) lam[(size_t)bond * chi + t] = (double)sig[t];
    if (threadIdx.x == 0) rank[bond + 1] = kf;
    __syncthreads();
    PHASE(6);
    if (threadIdx.x == 0) alg_flops += flops_per_gate(rl, rm, rr, kf);
  }
#undef PHASE
  if (threadIdx.x == 0) {
    for (int i = 0; i < 7; ++i) m.prof[s * 8 + i] += ph[i];
    m.prof[s * 8 + 7] = __double_as_longlong(__longlong_as_double(m.prof[s * 8 + 7]) + alg_flops);
    m.dw[s] += dw_acc;
    int* stt = m.stat + s * kStatWords;
    stt[0] = max(stt[0], st_max_iters);
    stt[1] += misc[2];
    stt[3] += st_bad;
    stt[2] = max(stt[2], st_max_rank);
    stt[4] += st_nonfinite;
    stt[5] |= st_badarg;
  }
}

// The dynamic shared-memory limit of a kernel is process-wide state: handles of
// different chi launch the same instantiation from several threads, so the limit is
// raised once to the device's opt-in maximum and never lowered.
template <auto Kernel>
static cudaError_t raise_smem_limit() {
  static std::once_flag once[64];
  static cudaError_t status[64];
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::call_once(once[dev], [dev] {
    int optin = 0;
    status[dev] = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (status[dev] == cudaSuccess)
      status[dev] = cudaFuncSetAttribute(Kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
  });
  return status[dev];
}

template <class R, int NT>
static cudaError_t launch_circ_t(const DevMPS& m, const CircDev& c, int64_t g0, int64_t g1,
                                 int slot0, int count, const double* theta, double cutoff,
                                 int max_sweeps, cudaStream_t st) {
  const EngineLayout<R> L(m.chi, NT);
  if (L.w_smem && L.t_smem) {
    cudaError_t e = raise_smem_limit<k_circuit<R, NT, false, true>>();
    if (e != cudaSuccess) return e;
    k_circuit<R, NT, false, true><<<count, NT, L.total, st>>>(m, c, g0, g1, slot0, theta, cutoff, max_sweeps);
  } else {
    cudaError_t e = raise_smem_limit<k_circuit<R, NT, false, false>>();
    if (e != cudaSuccess) return e;
    k_circuit<R, NT, false, false><<<count, NT, L.total, st>>>(m, c, g0, g1, slot0, theta, cutoff, max_sweeps);
  }
  return cudaGetLastError();
}

cudaError_t launch_circuit(const DevMPS& m, int prec, const CircDev& c, int64_t g0, int64_t g1,
                           int slot0, int count, const double* theta, double cutoff,
                           int max_sweeps, cudaStream_t st) {
  if (prec == MPS_PREC_FP64)
    return launch_circ_t<double, 512>(m, c, g0, g1, slot0, count, theta, cutoff, max_sweeps, st);
  return launch_circ_t<float, 512>(m, c, g0, g1, slot0, count, theta, cutoff, max_sweeps, st);
}

// --------------------------------------------------------- right environments
// R_n = [1]; R_k = sum_i Bhat_k^i (B_k^i)^+ with Bhat_k^i = B_k^i R_{k+1} (same layout as
// B_k). Per site two grid launches (the two Bhat^i products side by side, then R_k), so
// large bond dimensions use many SMs. ranks: the slot's bond ranks on the host
// (ranks[k] = left dimension of site k).
template <class R>
static cudaError_t right_envs_t(const DevMPS& m, int slot, const int* ranks, const int64_t* site_off, Cx<R>* Renv,
                                Cx<R>* Bhat, Cx<R>* Q, cudaStream_t st) {
  const int n = m.n;
  const size_t chi2 = (size_t)m.chi * m.chi;
  const Cx<R>* Bslot = (const Cx<R>*)m.B + (size_t)slot * m.slot_elems;
  static const Cx<R> one = cx<R>(1, 0);
  cudaError_t e = cudaMemcpyAsync(Renv + (size_t)n * chi2, &one, sizeof(Cx<R>), cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return e;
  for (int k = n - 1; k >= 0; --k) {
    const int Dl = ranks[k], Dr = ranks[k + 1];
    const Cx<R>* Bk = Bslot + site_off[k];
    Cx<R>* Bh = Bhat + site_off[k];
    const Cx<R>* Rn = Renv + (size_t)(k + 1) * chi2;
    GridGemm<R> g{};
    g.nterm = 1;
    g.ldc = 2 * Dr;
    g.M = Dl;
    g.N = Dr;
    g.K = Dr;
    for (int i = 0; i < 2; ++i) {   // Bhat^i = B^i R_{k+1}: (Dl x Dr)(Dr x Dr)
      g.t[i][0] = GemmTerm<R>{Bk + i * Dr, 2 * Dr, false, Rn, Dr, cx<R>(1, 0), false};
      g.C[i] = Bh + i * Dr;
    }
    k_cgemm_grid<R><<<dim3((Dr + 63) / 64, (Dl + 63) / 64, 2), 256, 0, st>>>(g);
    // R_k = sum_i Bhat^i (B^i)^+: B^i read as (Dl x Dr) transposed and conjugated
    GridGemm<R> h{};
    h.nterm = 2;
    h.ldc = Dl;
    h.M = Dl;
    h.N = Dl;
    h.K = Dr;
    for (int i = 0; i < 2; ++i) h.t[0][i] = GemmTerm<R>{Bh + i * Dr, 2 * Dr, false, Bk + i * Dr, 2 * Dr, cx<R>(1, 0), true, true};
    h.C[0] = Renv + (size_t)k * chi2;
    k_cgemm_grid<R><<<dim3((Dl + 63) / 64, (Dl + 63) / 64, 1), 256, 0, st>>>(h);
    // Q_k^P = sum over the letter's two entries (i, j, s) of conj(s) Bhat^i (B^j)^+, one
    // product per letter I, X, Y, Z: a string closing at site k with letter P has
    // <P> = sum_ab L[a][b] conj(Q_k^P[a][b]) (Eq. 11 with the right part contracted)
    GridGemm<R> q{};
    q.nterm = 2;
    q.ldc = Dl;
    q.M = Dl;
    q.N = Dl;
    q.K = Dr;
    for (int l = 0; l < 4; ++l) {
      const int ii[4][2] = {{0, 1}, {0, 1}, {0, 1}, {0, 1}};
      const int jj[4][2] = {{0, 1}, {1, 0}, {1, 0}, {0, 1}};
      // conj of the letter's entries: I (1, 1), X (1, 1), Y (-i, i) -> (i, -i), Z (1, -1)
      const Cx<R> cs[4][2] = {{cx<R>(1, 0), cx<R>(1, 0)},
                              {cx<R>(1, 0), cx<R>(1, 0)},
                              {cx<R>(0, 1), cx<R>(0, -1)},
                              {cx<R>(1, 0), cx<R>(-1, 0)}};
      for (int e = 0; e < 2; ++e)
        q.t[l][e] = GemmTerm<R>{Bh + ii[l][e] * Dr, 2 * Dr, false, Bk + jj[l][e] * Dr, 2 * Dr, cs[l][e], true, true};
      q.C[l] = Q + ((size_t)k * 4 + l) * chi2;
    }
    k_cgemm_grid<R><<<dim3((Dl + 63) / 64, (Dl + 63) / 64, 4), 256, 0, st>>>(q);
  }
  return cudaGetLastError();
}

cudaError_t launch_right_envs(const DevMPS& m, int prec, int slot, const int* ranks, const int64_t* site_off,
                              MeasDev& w, cudaStream_t st, int* launches) {
  *launches += 3 * m.n;
  if (prec == MPS_PREC_FP64)
    return right_envs_t<double>(m, slot, ranks, site_off, (Cx<double>*)w.R, (Cx<double>*)w.Bhat, (Cx<double>*)w.Q,
                                st);
  return right_envs_t<float>(m, slot, ranks, site_off, (Cx<float>*)w.R, (Cx<float>*)w.Bhat, (Cx<float>*)w.Q, st);
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

// Level buffers are dense: node u of level k holds L at u Dk^2 (leading dimension Dk)
// and, on the CUDA-core route, T_j at (2u + j) Dk Dk1 (leading dimension Dk1).
// T_j[u] = L_k[u] B_k^j  (Dk x Dk)(Dk x Dk1), grid (nodes, 2)
template <class R>
__global__ void __launch_bounds__(256) k_level_T(DevMPS m, int slot, int k, const Cx<R>* Lin, Cx<R>* T) {
  __shared__ Cx<R> As[64][17];
  __shared__ Cx<R> Bs[16][65];
  const int u = blockIdx.x, j = blockIdx.y;
  const int* rank = m.rank + (size_t)slot * (m.n + 1);
  const int Dk = rank[k], Dk1 = rank[k + 1];
  const Cx<R>* Bk = (const Cx<R>*)m.B + (size_t)slot * m.slot_elems + m.site_off[k];
  GemmTerm<R> t{Lin + (size_t)u * Dk * Dk, Dk, false, Bk + j * Dk1, 2 * Dk1, cx<R>(1, 0), false};
  block_gemm<R, 256>(Dk, Dk1, Dk, &t, 1, T + ((size_t)u * 2 + j) * Dk * Dk1, Dk1, As, Bs);
}

// L_{k+1}[c] = sum_ij sigma_ij (B_k^i)^+ T_j[parent(c)]
template <class R>
__global__ void __launch_bounds__(256) k_level_child(DevMPS m, int slot, int k, const int32_t* parent,
                                                     const uint8_t* edge, const Cx<R>* T, Cx<R>* Lout,
                                                     int node_base) {
  __shared__ Cx<R> As[64][17];
  __shared__ Cx<R> Bs[16][65];
  const int c = blockIdx.x;
  const int* rank = m.rank + (size_t)slot * (m.n + 1);
  const int Dk = rank[k], Dk1 = rank[k + 1];
  const Cx<R>* Bk = (const Cx<R>*)m.B + (size_t)slot * m.slot_elems + m.site_off[k];
  const int u = parent[c] - node_base;
  int ii[2], jj[2];
  Cx<R> sg[2];
  letter_entries<R>(edge[c], ii, jj, sg);
  GemmTerm<R> t[2];
  for (int e = 0; e < 2; ++e)
    t[e] = GemmTerm<R>{Bk + ii[e] * Dk1, 2 * Dk1, true, T + ((size_t)u * 2 + jj[e]) * Dk * Dk1, Dk1, sg[e], false};
  block_gemm<R, 256>(Dk1, Dk1, Dk, t, 2, Lout + (size_t)c * Dk1 * Dk1, Dk1, As, Bs);
}

// <P> (unnormalised) of a string closing at site k with letter P on node u:
// sum_ab L[u][a][b] conj(Q_k^P[a][b]), Q_k^P = sum_ij conj(P_ij) Bhat_k^i (B_k^j)^+ from the
// right-environment pass. This equals sum_ij P_ij <Bhat_k^i, L[u] B_k^j>_F (Eq. 11 with
// the right part contracted first) and reads one D x D block of the node instead of the
// two D x D' blocks of T. Both blocks are contiguous with leading dimension D.
template <class R>
__global__ void __launch_bounds__(256) k_level_close(DevMPS m, int slot, int k, const int32_t* cnode,
                                                     const uint8_t* cletter, const int32_t* cterm,
                                                     const Cx<R>* L, const Cx<R>* Q, double* vals,
                                                     int node_base) {
  __shared__ double red[2][8];
  const int c = blockIdx.x;
  const int chi2 = m.chi * m.chi;
  const int* rank = m.rank + (size_t)slot * (m.n + 1);
  const int Dk = rank[k];
  const Cx<R>* Lu = L + (size_t)(cnode[c] - node_base) * Dk * Dk;
  const Cx<R>* Qp = Q + ((size_t)k * 4 + (cletter[c] & 3)) * chi2;
  const int n = Dk * Dk;
  double re = 0.0, im = 0.0;
  // R = float: FP32 products summed in FP32 over runs of 8 entries, the runs summed in
  // FP64. GB300's FP64 (and FP32 -> FP64 conversion) throughput is a small fraction of
  // its FP32 rate; one FP64 step per entry made the close a third of a chi = 256
  // measurement. A run's FP32 sum is off by at most ~8 ulps of its magnitudes, below the
  // ~2^-21 relative error of the tensor-core environments. R = double: FP64.
  int idx = threadIdx.x;
  for (; idx + 7 * 256 < n; idx += 8 * 256) {
    // a full run: its 16 loads are issued before the products that use them
    Cx<R> q[8], l[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      q[t] = Qp[idx + t * 256];
      l[t] = Lu[idx + t * 256];
    }
    R sr = 0, si = 0;
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      // conj(q) * l
      sr += q[t].x * l[t].x + q[t].y * l[t].y;
      si += q[t].x * l[t].y - q[t].y * l[t].x;
    }
    re += (double)sr;
    im += (double)si;
  }
  if (idx < n) {
    R sr = 0, si = 0;
    for (; idx < n; idx += 256) {
      const Cx<R> q = Qp[idx], l = Lu[idx];
      sr += q.x * l.x + q.y * l.y;
      si += q.x * l.y - q.y * l.x;
    }
    re += (double)sr;
    im += (double)si;
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

cudaError_t launch_env_T(const DevMPS& m, int prec, int slot, int k, const void* L, void* T, int n_nodes,
                         cudaStream_t st) {
  if (n_nodes <= 0) return cudaSuccess;
  if (prec == MPS_PREC_FP64)
    k_level_T<double><<<dim3(n_nodes, 2), 256, 0, st>>>(m, slot, k, (const Cx<double>*)L, (Cx<double>*)T);
  else
    k_level_T<float><<<dim3(n_nodes, 2), 256, 0, st>>>(m, slot, k, (const Cx<float>*)L, (Cx<float>*)T);
  return cudaGetLastError();
}

cudaError_t launch_env_close(const DevMPS& m, int prec, int slot, int k, const void* L, const void* Q,
                             const int32_t* cnode, const uint8_t* cletter, const int32_t* cterm, int n_closes,
                             int node_base, double* vals, cudaStream_t st) {
  if (n_closes <= 0) return cudaSuccess;
  if (prec == MPS_PREC_FP64)
    k_level_close<double><<<n_closes, 256, 0, st>>>(m, slot, k, cnode, cletter, cterm, (const Cx<double>*)L,
                                                     (const Cx<double>*)Q, vals, node_base);
  else
    k_level_close<float><<<n_closes, 256, 0, st>>>(m, slot, k, cnode, cletter, cterm, (const Cx<float>*)L,
                                                    (const Cx<float>*)Q, vals, node_base);
  return cudaGetLastError();
}

cudaError_t launch_env_child(const DevMPS& m, int prec, int slot, int k, const void* T, const int32_t* parent,
                             const uint8_t* edge, int n_children, int node_base, void* Lout, cudaStream_t st) {
  if (n_children <= 0) return cudaSuccess;
  if (prec == MPS_PREC_FP64)
    k_level_child<double><<<n_children, 256, 0, st>>>(m, slot, k, parent, edge, (const Cx<double>*)T,
                                                       (Cx<double>*)Lout, node_base);
  else
    k_level_child<float><<<n_children, 256, 0, st>>>(m, slot, k, parent, edge, (const Cx<float>*)T,
                                                      (Cx<float>*)Lout, node_base);
  return cudaGetLastError();
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

// ------------------------------------------------------------------------------
// Allocation-free variant of the gate engine for callers that cannot allocate device
// memory themselves or through this library (the paper has no counterpart; see the
// declaration of mps_apply_gates_noalloc in include/mpsvqe.h). Its workspace lives in
// the file-scope array below, which every GPU that loads the library keeps until the
// process exits; all calls share it.
namespace mpsvqe {
namespace {
constexpr size_t kNoAllocScratchBytes = size_t(1) << 20;   // 1 MiB
constexpr int kNoAllocMaxChi = 64;
}  // namespace
}  // namespace mpsvqe

static __device__ __align__(256) unsigned char g_noalloc_scratch[mpsvqe::kNoAllocScratchBytes];

#include <cstring>
#include <mutex>
#include "../../include/mpsvqe.h"

namespace {
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[64] = {nullptr};
}  // namespace

extern "C" int mps_apply_gates_noalloc(int n_qubits, int chi, void* site_tensors, const int64_t* site_offsets,
                                       double* lambdas, int32_t* ranks, int64_t n_gates, const int32_t* bonds,
                                       const double* gates, void* cuda_stream, double* discarded_weight) {
  using namespace mpsvqe;
  if (!site_tensors || !site_offsets || !lambdas || !ranks || (n_gates > 0 && (!bonds || !gates))) {
    set_error_message("mps_apply_gates_noalloc: null device pointer");
    return MPS_EINVAL;
  }
  if (n_qubits < 2 || n_qubits > kMaxQubits || chi < 1 || chi > kNoAllocMaxChi || n_gates < 0) {
    set_error_message("mps_apply_gates_noalloc: needs 2 <= n_qubits <= 128, 1 <= chi <= 64 and n_gates >= 0 "
                      "(the fixed 1 MiB device workspace holds one chi <= 64 gate step)");
    return MPS_EINVAL;
  }
  const size_t mm = 2 * (size_t)chi;
  const size_t off_M = 0;
  const size_t off_X = off_M + ((mm * mm * 8 + 255) & ~(size_t)255);
  const size_t off_S = off_X + ((mm * (mm + 16) * 8 + 255) & ~(size_t)255);
  const size_t off_dw = off_S + ((16 * (size_t)chi * chi * 8 + 255) & ~(size_t)255);
  const size_t off_end = off_dw + 256;
  if (off_end > kNoAllocScratchBytes) {
    set_error_message("mps_apply_gates_noalloc: workspace larger than the 1 MiB device array");
    return MPS_EINVAL;
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    set_error_message("mps_apply_gates_noalloc: no current CUDA device");
    return MPS_ECUDA;
  }
  unsigned char* base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
        set_error_message("mps_apply_gates_noalloc: cudaGetSymbolAddress of the device workspace failed");
        return MPS_ECUDA;
      }
      g_noalloc_ptr[dev] = p;
    }
    base = (unsigned char*)g_noalloc_ptr[dev];
  }
  cudaStream_t st = (cudaStream_t)cuda_stream;
  DevMPS d{};
  d.n = n_qubits;
  d.chi = chi;
  d.n_slots = 1;
  d.slot_elems = 0;
  d.site_off = site_offsets;
  d.B = site_tensors;
  d.lam = lambdas;
  d.rank = ranks;
  d.work_M = base + off_M;
  d.work_X = base + off_X;
  d.work_S = base + off_S;
  d.dw = (double*)(base + off_dw);
  d.stat = (int*)(base + off_dw + 8);
  d.prof = (unsigned long long*)(base + off_dw + 64);
  // the shared array keeps the previous call's contents: clear the accumulators
  if (cudaMemsetAsync(base + off_dw, 0, 256, st) != cudaSuccess) return MPS_ECUDA;
  CircDev c{};
  c.gates = nullptr;
  c.n_gates = n_gates;
  c.mats = gates;
  c.n_params = 1;
  c.raw_bond = bonds;
  const EngineLayout<float> L(chi, 512);
  if (!(L.w_smem && L.t_smem)) {   // holds for every chi <= 64 in complex64
    set_error_message("mps_apply_gates_noalloc: gate workspace does not fit in shared memory");
    return MPS_EINVAL;
  }
  if (raise_smem_limit<k_circuit<float, 512, true, true>>() != cudaSuccess) return MPS_ECUDA;
  const double* theta = (const double*)(base + off_dw + 128);   // never read: every gate is fixed
  for (int64_t g0 = 0; g0 < n_gates; g0 += 16384) {
    const int64_t g1 = g0 + 16384 < n_gates ? g0 + 16384 : n_gates;
    k_circuit<float, 512, true, true><<<1, 512, L.total, st>>>(d, c, g0, g1, 0, theta, std::ldexp(1.0, -20), 60);
    if (cudaGetLastError() != cudaSuccess) return MPS_ECUDA;
  }
  if (discarded_weight) {
    // the discarded weight and the status words sit next to each other in the array:
    // one copy brings both back
    unsigned char host[8 + 4 * kStatWords];
    if (cudaMemcpyAsync(host, d.dw, sizeof(host), cudaMemcpyDeviceToHost, st) != cudaSuccess) return MPS_ECUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return MPS_ECUDA;
    int stat[kStatWords];
    std::memcpy(discarded_weight, host, 8);
    std::memcpy(stat, host + 8, sizeof(stat));
    if (stat[5]) {
      set_error_message("mps_apply_gates_noalloc: a bond outside [0, n-2] or a rank outside its capacity "
                        "reached the device; gates from there on were not applied");
      return MPS_EINVAL;
    }
    if (stat[4] > 0) {
      set_error_message("mps_apply_gates_noalloc: a gate's M' held a NaN or Inf; the gate was skipped");
      return MPS_ENONFINITE;
    }
    if (stat[1] > 0) {
      set_error_message("mps_apply_gates_noalloc: a Jacobi SVD fallback reached its sweep cap");
      return MPS_ENOCONV;
    }
  }
  return MPS_OK;
}
