// Environment contractions of the trie measurement on the tensor cores (mixed precision).
//
// One trie level k (site k, left bond D = D_k, right bond D' = D_{k+1}) does two dense
// complex contractions per node (Eq. 11 generalised to Pauli strings, Sec. III-C):
//   T_j[u] = L[u] B^j                         (D x D)(D x D'),  j = 0, 1
//   C_ij[u] = (B^i)^+ T_j[u]                  (D' x D)(D x D'), i, j = 0, 1
// and a child with letter P on its edge takes L[child] = sum_ij P_ij C_ij[parent]. Over
// a chunk of U nodes both become single real GEMMs with a shared operand built from the
// site tensor (split-complex: real and imaginary planes side by side along K):
//   GEMM-T: rows (u, a) of [Re L | Im L]  (U D x 2D)  times  BT (4D' x 2D)^T
//           BT row (j, re, c) = [ Re B^j[:, c], -Im B^j[:, c] ],
//           BT row (j, im, c) = [ Im B^j[:, c],  Re B^j[:, c] ]
//   GEMM-C: AC (4D' x 2D) times rows (u, j, c) of [Re T_j[u][:, c] | Im T_j[u][:, c]]^T
//           AC row (i, re, c') = [ Re B^i[:, c'],  Im B^i[:, c'] ],
//           AC row (i, im, c') = [-Im B^i[:, c'],  Re B^i[:, c'] ]
// Both run on tc::launch_gemm_tf32x3 (tcgen05, compensated TF32 splits made inside the
// GEMM from the FP32 tiles it loads). The kernels here build the FP32 operand planes and
// move results between the GEMM layouts and
// the complex environment buffers that the rest of the measurement uses (L: node u at
// u chi^2, leading dimension D; T: T_j[u] at (2u + j) chi^2, leading dimension D').
#include <cstdint>

#include "cx.cuh"
#include "env_tc.cuh"
#include "tc_gemm.cuh"

namespace mpsvqe {

__host__ __device__ inline int64_t round4(int64_t x) { return (x + 3) & ~(int64_t)3; }

// ---------------------------------------------------------------- operand planes
// [Re L[u][a][:] | Im L[u][a][:]] for rows (u, a), leading dimension ldk.
__global__ void k_tc_pack_L(const Cx<float>* L, int64_t chi2, int U, int D, float* out, int64_t ldk) {
  const int64_t total = (int64_t)U * D * ldk;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = i / ldk, col = i - row * ldk;
    const int u = (int)(row / D), a = (int)(row - (int64_t)u * D);
    float v = 0.f;
    if (col < 2 * D) {
      const Cx<float> z = L[(size_t)u * chi2 + (size_t)a * D + (col < D ? col : col - D)];
      v = col < D ? z.x : z.y;
    }
    out[i] = v;
  }
}

// BT (4D' x ldk) and AC (4D' x ldk) from site k (B[b][j][c] at (b 2 + j) D' + c).
__global__ void k_tc_site_operands(const Cx<float>* Bk, int D, int Dp, int64_t ldk, float* bt, float* ac) {
  const int64_t total = (int64_t)4 * Dp * ldk;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = i / ldk;
    const int col = (int)(i - row * ldk);
    const int j = (int)(row / (2 * Dp)), ro = (int)((row / Dp) & 1), c = (int)(row % Dp);
    float vt = 0.f, va = 0.f;
    if (col < 2 * D) {
      const int ri = col >= D, b = ri ? col - D : col;
      const Cx<float> z = Bk[((size_t)b * 2 + j) * Dp + c];   // B^j[b][c] (also B^i[a][c'] with i = j)
      // BT: re row [Br, -Bi], im row [Bi, Br]
      vt = ro == 0 ? (ri == 0 ? z.x : -z.y) : (ri == 0 ? z.y : z.x);
      // AC: re row [Br, Bi], im row [-Bi, Br]
      va = ro == 0 ? (ri == 0 ? z.x : z.y) : (ri == 0 ? -z.y : z.x);
    }
    bt[i] = vt;
    ac[i] = va;
  }
}

// C_T (U D x 4D', rows (u, a), columns (j, re/im, c)) -> T_j[u][a][c] complex.
__global__ void k_tc_scatter_T(const float* CT, int U, int D, int Dp, Cx<float>* T, int64_t chi2) {
  const int64_t total = (int64_t)U * 2 * D * Dp;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(i % Dp);
    int64_t r = i / Dp;
    const int a = (int)(r % D);
    r /= D;
    const int j = (int)(r & 1);
    const int u = (int)(r >> 1);
    const float* row = CT + ((int64_t)u * D + a) * 4 * Dp;
    T[((size_t)u * 2 + j) * chi2 + (size_t)a * Dp + c] = cx<float>(row[(2 * j) * Dp + c], row[(2 * j + 1) * Dp + c]);
  }
}

// Rows (u - pa, j, c) of [Re T_j[u][:, c] | Im T_j[u][:, c]] for parents u in [pa, pb):
// a transpose of each D x D' block through 32 x 32 shared-memory tiles.
__global__ void k_tc_pack_TT(const Cx<float>* T, int64_t chi2, int pa, int D, int Dp, float* out, int64_t ldk) {
  __shared__ Cx<float> tile[32][33];
  const int blk = blockIdx.z;               // (u - pa) * 2 + j
  const int u = pa + (blk >> 1), j = blk & 1;
  const int a0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
  const Cx<float>* Tj = T + ((size_t)u * 2 + j) * chi2;
  for (int y = threadIdx.y; y < 32; y += blockDim.y) {
    const int a = a0 + y, c = c0 + threadIdx.x;
    tile[y][threadIdx.x] = (a < D && c < Dp) ? Tj[(size_t)a * Dp + c] : cx<float>(0.f, 0.f);
  }
  __syncthreads();
  for (int y = threadIdx.y; y < 32; y += blockDim.y) {
    const int c = c0 + y, a = a0 + threadIdx.x;
    if (c < Dp && a < D) {
      const Cx<float> z = tile[threadIdx.x][y];
      const int64_t row = ((int64_t)blk * Dp + c) * ldk;
      out[row + a] = z.x;
      out[row + D + a] = z.y;
    }
  }
  // zero padding columns 2D..ldk-1 of the rows this block owns (first a-tile only)
  if (blockIdx.y == 0) {
    for (int y = threadIdx.y; y < 32; y += blockDim.y) {
      const int c = c0 + y;
      if (c < Dp)
        for (int col = 2 * D + threadIdx.x; col < ldk; col += 32) {
          const int64_t row = ((int64_t)blk * Dp + c) * ldk;
          out[row + col] = 0.f;
        }
    }
  }
}

// Children [0, nc): L[child][c'][c] = sum_e s_e C_{i_e j_e}[parent][c'][c], with
// C_L (4D' x ldc), rows (i, re/im, c'), columns ((u - pa), j, c).
__global__ void k_tc_combine(const float* CL, int64_t ldc, int Dp, const int32_t* parent, const uint8_t* edge,
                             int nc, int node_base, int pa, Cx<float>* Lout, int64_t chi2) {
  const int64_t total = (int64_t)nc * Dp * Dp;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(i % Dp);
    const int64_t r = i / Dp;
    const int cp = (int)(r % Dp);
    const int ch = (int)(r / Dp);
    const int u = parent[ch] - node_base - pa;
    const uint8_t lt = edge[ch];
    // letter -> (i, j, s) pairs: I: (0,0,1)(1,1,1); X: (0,1,1)(1,0,1); Y: (0,1,-i)(1,0,i); Z: (0,0,1)(1,1,-1)
    int ii[2], jj[2];
    Cx<float> sg[2];
    switch (lt) {
      case 0: ii[0] = 0; jj[0] = 0; sg[0] = cx<float>(1, 0); ii[1] = 1; jj[1] = 1; sg[1] = cx<float>(1, 0); break;
      case 1: ii[0] = 0; jj[0] = 1; sg[0] = cx<float>(1, 0); ii[1] = 1; jj[1] = 0; sg[1] = cx<float>(1, 0); break;
      case 2: ii[0] = 0; jj[0] = 1; sg[0] = cx<float>(0, -1); ii[1] = 1; jj[1] = 0; sg[1] = cx<float>(0, 1); break;
      default: ii[0] = 0; jj[0] = 0; sg[0] = cx<float>(1, 0); ii[1] = 1; jj[1] = 1; sg[1] = cx<float>(-1, 0); break;
    }
    Cx<float> acc = cx<float>(0.f, 0.f);
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const int64_t col = ((int64_t)u * 2 + jj[e]) * Dp + c;
      const float re = CL[((int64_t)(2 * ii[e]) * Dp + cp) * ldc + col];
      const float im = CL[((int64_t)(2 * ii[e] + 1) * Dp + cp) * ldc + col];
      acc = acc + sg[e] * cx<float>(re, im);
    }
    Lout[(size_t)ch * chi2 + (size_t)cp * Dp + c] = acc;
  }
}

static inline int grid_for(int64_t total) {
  const int64_t b = (total + 255) / 256;
  return (int)(b < 152 * 32 ? (b > 0 ? b : 1) : 152 * 32);
}

size_t env_tc_scratch_floats(int chi, int max_nodes) {
  const int64_t D = chi, Dp = chi, U = max_nodes, ldk = round4(2 * D);
  const int64_t lplane = U * D * ldk;               // [Re L | Im L]
  const int64_t site = 2 * 4 * Dp * ldk;            // BT, AC
  const int64_t ct = U * D * 4 * Dp;                // GEMM-T output
  const int64_t tt = U * 2 * Dp * ldk;              // [Re T^T | Im T^T]
  const int64_t cl = 4 * Dp * U * 2 * Dp;           // GEMM-C output
  const int64_t pad = 64;                           // 16-byte alignment of each part
  return (size_t)(lplane + site + ct + tt + cl + 8 * pad);
}

namespace {
struct Parts {
  float *lp, *bt, *ac, *ct, *tt, *cl;
};
Parts carve(float* base, int chi, int max_nodes) {
  const int64_t D = chi, Dp = chi, U = max_nodes, ldk = round4(2 * D);
  auto take = [&](int64_t n) {
    float* p = base;
    base += (n + 63) & ~(int64_t)63;
    return p;
  };
  Parts p;
  p.lp = take(U * D * ldk);
  p.bt = take(4 * Dp * ldk);
  p.ac = take(4 * Dp * ldk);
  p.ct = take(U * D * 4 * Dp);
  p.tt = take(U * 2 * Dp * ldk);
  p.cl = take(4 * Dp * U * 2 * Dp);
  return p;
}
}  // namespace

cudaError_t env_tc_site(const EnvTc& s, const Cx<float>* Bk, int D, int Dp, cudaStream_t st) {
  const Parts p = carve(s.scratch, s.chi, s.max_nodes);
  const int64_t ldk = round4(2 * D);
  k_tc_site_operands<<<grid_for(4 * Dp * ldk), 256, 0, st>>>(Bk, D, Dp, ldk, p.bt, p.ac);
  return cudaGetLastError();
}

cudaError_t env_tc_T(const EnvTc& s, const Cx<float>* L, Cx<float>* T, int U, int D, int Dp, cudaStream_t st,
                     cudaEvent_t e0, cudaEvent_t e1) {
  if (U <= 0) return cudaSuccess;
  const Parts p = carve(s.scratch, s.chi, s.max_nodes);
  const int64_t ldk = round4(2 * D), chi2 = (int64_t)s.chi * s.chi;
  k_tc_pack_L<<<grid_for((int64_t)U * D * ldk), 256, 0, st>>>(L, chi2, U, D, p.lp, ldk);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (e0 && (e = cudaEventRecord(e0, st)) != cudaSuccess) return e;
  e = tc::launch_gemm_tf32x3(tc::Plane{p.lp, ldk}, tc::Plane{p.bt, ldk}, U * D, 4 * Dp, 2 * D, p.ct, 4 * Dp, s.err,
                             st);
  if (e != cudaSuccess) return e;
  if (e1 && (e = cudaEventRecord(e1, st)) != cudaSuccess) return e;
  k_tc_scatter_T<<<grid_for((int64_t)U * 2 * D * Dp), 256, 0, st>>>(p.ct, U, D, Dp, T, chi2);
  return cudaGetLastError();
}

cudaError_t env_tc_children(const EnvTc& s, const Cx<float>* T, int pa, int pb, int D, int Dp,
                            const int32_t* parent, const uint8_t* edge, int nc, int node_base, Cx<float>* Lout,
                            cudaStream_t st, cudaEvent_t e0, cudaEvent_t e1) {
  if (nc <= 0 || pb <= pa) return cudaSuccess;
  const Parts p = carve(s.scratch, s.chi, s.max_nodes);
  const int64_t ldk = round4(2 * D), chi2 = (int64_t)s.chi * s.chi;
  const int np = pb - pa;
  k_tc_pack_TT<<<dim3((Dp + 31) / 32, (D + 31) / 32, np * 2), dim3(32, 8), 0, st>>>(T, chi2, pa, D, Dp, p.tt, ldk);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int64_t N = (int64_t)np * 2 * Dp;
  if (e0 && (e = cudaEventRecord(e0, st)) != cudaSuccess) return e;
  e = tc::launch_gemm_tf32x3(tc::Plane{p.ac, ldk}, tc::Plane{p.tt, ldk}, 4 * Dp, (int)N, 2 * D, p.cl, N, s.err, st);
  if (e != cudaSuccess) return e;
  if (e1 && (e = cudaEventRecord(e1, st)) != cudaSuccess) return e;
  k_tc_combine<<<grid_for((int64_t)nc * Dp * Dp), 256, 0, st>>>(p.cl, N, Dp, parent, edge, nc, node_base, pa, Lout,
                                                                chi2);
  return cudaGetLastError();
}

}  // namespace mpsvqe
