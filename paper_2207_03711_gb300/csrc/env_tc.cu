// Environment contractions of the trie measurement on the tensor cores (mixed precision).
//
// One trie level k (site k, left bond D = D_k, right bond D' = D_{k+1}) does two dense
// complex contractions (Eq. 11 generalised to Pauli strings, Sec. III-C):
//   T_j[u] = L[u] B^j                               (D x D)(D x D'),  j = 0, 1
//   L[child] = sum_ij P_ij (B^i)^+ T_j[u]          P = the edge letter of the child
// The second is formed per child, not per parent: with W_i = sum_j P_ij T_j[u] (for
// I: (T_0, T_1); X: (T_1, T_0); Y: (-i T_1, i T_0); Z: (T_0, -T_1)) it is one product
// sum_i (B^i)^+ W_i with the i sum stacked along K. In a Jordan-Wigner trie almost every
// parent has a single child (the next letter of a Z chain), and computing the four
// C_ij = (B^i)^+ T_j of every parent, as a per-parent form would, doubles that work.
// Over a chunk both become single real GEMMs with a shared operand built from the site
// tensor:
//   GEMM-T: rows (u, a) of L[u] read as interleaved floats (re, im per entry; U D x 2D),
//           the level buffer itself, times BT (4D' x 2D)^T with
//           BT row (j, c, re) = [ Re B^j[b, c], -Im B^j[b, c] ]_b   (interleaved per b),
//           BT row (j, c, im) = [ Im B^j[b, c],  Re B^j[b, c] ]_b,
//           so that output row (u, a) is [T_0[u][a][:] | T_1[u][a][:]] as interleaved
//           complex: the GEMM writes the level's T buffer directly.
//   GEMM-C: A2 (2D' x 4D) times rows (child, c) of
//           [Re W_0[:, c] | Im W_0[:, c] | Re W_1[:, c] | Im W_1[:, c]]^T
//           A2 row (re, c') = [ Re B^0[:, c'],  Im B^0[:, c'],  Re B^1[:, c'],  Im B^1[:, c'] ],
//           A2 row (im, c') = [-Im B^0[:, c'],  Re B^0[:, c'], -Im B^1[:, c'],  Re B^1[:, c'] ]
// Both run on tc::launch_gemm_tf32x3 (tcgen05, compensated TF32 splits made inside the
// GEMM from the FP32 tiles it loads). Level buffers are dense: L[u] at u D^2 (leading
// dimension D); on this route T_j[u][a][c] at ((u D + a) 2 + j) D' + c. The kernels here
// build the site operands and the W rows and place the children's environments.
#include <cstdint>

#include "cx.cuh"
#include "env_tc.cuh"
#include "tc_gemm.cuh"

namespace mpsvqe {

// ---------------------------------------------------------------- operand planes
// BT (4D' x 2D) and A2 (2D' x 4D) from site k (B[b][j][c] at (b 2 + j) D' + c).
__global__ void k_tc_site_operands(const Cx<float>* Bk, int D, int Dp, float* bt, float* a2) {
  const int64_t nbt = (int64_t)4 * Dp * 2 * D, na2 = (int64_t)2 * Dp * 4 * D;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nbt + na2;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (i < nbt) {
      const int64_t row = i / (2 * D);
      const int col = (int)(i - row * 2 * D);
      const int ro = (int)(row & 1), c = (int)((row >> 1) % Dp), j = (int)((row >> 1) / Dp);
      const int b = col >> 1, ri = col & 1;
      const Cx<float> z = Bk[((size_t)b * 2 + j) * Dp + c];   // B^j[b][c]
      // re row: (Br, -Bi) per b; im row: (Bi, Br) per b
      bt[i] = ro == 0 ? (ri == 0 ? z.x : -z.y) : (ri == 0 ? z.y : z.x);
    } else {
      const int64_t e = i - nbt, row = e / (4 * D);
      const int col = (int)(e - row * 4 * D);
      const int ro = (int)(row / Dp), cp = (int)(row % Dp);
      const int ii = col / (2 * D), ri = (col / D) & 1, a = col % D;
      const Cx<float> z = Bk[((size_t)a * 2 + ii) * Dp + cp];   // B^i[a][c']
      // re row [Br, Bi] per i, im row [-Bi, Br] per i
      a2[e] = ro == 0 ? (ri == 0 ? z.x : z.y) : (ri == 0 ? -z.y : z.x);
    }
  }
}

// Rows (child, c) of [Re W_0[:, c] | Im W_0[:, c] | Re W_1[:, c] | Im W_1[:, c]] (leading
// dimension 4D) for children [0, nc), W_i = sum_j P_ij T_j[parent] with P the child's
// edge letter: a transpose of the parent's two D x D' blocks through 32 x 32 shared-memory
// tiles, mixed per letter on the way out.
__global__ void k_tc_pack_W(const Cx<float>* T, const int32_t* parent, const uint8_t* edge, int node_base, int D,
                            int Dp, float* out) {
  __shared__ Cx<float> t0[32][33];
  __shared__ Cx<float> t1[32][33];
  const int ch = blockIdx.z;
  const int u = parent[ch] - node_base;
  const uint8_t lt = edge[ch];
  const int a0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
  const Cx<float>* Tu = T + (size_t)u * 2 * D * Dp;   // row a: [T_0[u][a][:] | T_1[u][a][:]]
  for (int y = threadIdx.y; y < 32; y += blockDim.y) {
    const int a = a0 + y, c = c0 + threadIdx.x;
    const bool in = a < D && c < Dp;
    t0[y][threadIdx.x] = in ? Tu[(size_t)a * 2 * Dp + c] : cx<float>(0.f, 0.f);
    t1[y][threadIdx.x] = in ? Tu[(size_t)a * 2 * Dp + Dp + c] : cx<float>(0.f, 0.f);
  }
  __syncthreads();
  const int64_t ldk = 4 * (int64_t)D;
  for (int y = threadIdx.y; y < 32; y += blockDim.y) {
    const int c = c0 + y, a = a0 + threadIdx.x;
    if (c < Dp && a < D) {
      const Cx<float> x0 = t0[threadIdx.x][y], x1 = t1[threadIdx.x][y];
      Cx<float> w0, w1;
      switch (lt) {
        case 0: w0 = x0; w1 = x1; break;                                        // I
        case 1: w0 = x1; w1 = x0; break;                                        // X
        case 2: w0 = cx<float>(x1.y, -x1.x); w1 = cx<float>(-x0.y, x0.x); break;  // Y: -i T_1, i T_0
        default: w0 = x0; w1 = cx<float>(-x1.x, -x1.y); break;                  // Z
      }
      float* row = out + ((int64_t)ch * Dp + c) * ldk;
      row[a] = w0.x;
      row[D + a] = w0.y;
      row[2 * D + a] = w1.x;
      row[3 * D + a] = w1.y;
    }
  }
}

// Children [0, nc): L[child][c'][c] from C_L (2D' x nc D'), rows (re/im, c'), columns
// (child, c).
__global__ void k_tc_place(const float* CL, int Dp, int nc, Cx<float>* Lout) {
  const int64_t total = (int64_t)nc * Dp * Dp, N = (int64_t)nc * Dp;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(i % Dp);
    const int64_t r = i / Dp;
    const int cp = (int)(r % Dp);
    const int ch = (int)(r / Dp);
    const int64_t col = (int64_t)ch * Dp + c;
    Lout[((size_t)ch * Dp + cp) * Dp + c] = cx<float>(CL[(int64_t)cp * N + col], CL[(int64_t)(Dp + cp) * N + col]);
  }
}

static inline int grid_for(int64_t total) {
  const int64_t b = (total + 255) / 256;
  return (int)(b < 152 * 32 ? (b > 0 ? b : 1) : 152 * 32);
}

size_t env_tc_scratch_floats(int chi, int max_nodes) {
  const int64_t D = chi, Dp = chi, U = max_nodes;
  const int64_t site = 4 * Dp * 2 * D + 2 * Dp * 4 * D;   // BT, A2
  const int64_t w = U * Dp * 4 * D;                       // W rows of up to U children
  const int64_t cl = 2 * Dp * U * Dp;                     // GEMM-C output
  const int64_t pad = 64;                                 // 256-byte alignment of each part
  return (size_t)(site + w + cl + 4 * pad);
}

namespace {
struct Parts {
  float *bt, *a2, *w, *cl;
};
Parts carve(float* base, int chi, int max_nodes) {
  const int64_t D = chi, Dp = chi, U = max_nodes;
  auto take = [&](int64_t n) {
    float* p = base;
    base += (n + 63) & ~(int64_t)63;
    return p;
  };
  Parts p;
  p.bt = take(4 * Dp * 2 * D);
  p.a2 = take(2 * Dp * 4 * D);
  p.w = take(U * Dp * 4 * D);
  p.cl = take(2 * Dp * U * Dp);
  return p;
}
}  // namespace

cudaError_t env_tc_site(const EnvTc& s, const Cx<float>* Bk, int D, int Dp, cudaStream_t st) {
  const Parts p = carve(s.scratch, s.chi, s.max_nodes);
  k_tc_site_operands<<<grid_for(16 * (int64_t)Dp * D), 256, 0, st>>>(Bk, D, Dp, p.bt, p.a2);
  return cudaGetLastError();
}

cudaError_t env_tc_T(const EnvTc& s, const Cx<float>* L, Cx<float>* T, int U, int D, int Dp, cudaStream_t st,
                     cudaEvent_t e0, cudaEvent_t e1) {
  if (U <= 0) return cudaSuccess;
  const Parts p = carve(s.scratch, s.chi, s.max_nodes);
  cudaError_t e;
  if (e0 && (e = cudaEventRecord(e0, st)) != cudaSuccess) return e;
  e = tc::launch_gemm_tf32x3(tc::Plane{(const float*)L, 2 * (int64_t)D}, tc::Plane{p.bt, 2 * (int64_t)D}, U * D,
                             4 * Dp, 2 * D, (float*)T, 4 * (int64_t)Dp, s.err, st);
  if (e != cudaSuccess) return e;
  if (e1 && (e = cudaEventRecord(e1, st)) != cudaSuccess) return e;
  return cudaSuccess;
}

cudaError_t env_tc_children(const EnvTc& s, const Cx<float>* T, const int32_t* parent, const uint8_t* edge, int nc,
                            int node_base, int D, int Dp, Cx<float>* Lout, cudaStream_t st, cudaEvent_t e0,
                            cudaEvent_t e1) {
  if (nc <= 0) return cudaSuccess;
  const Parts p = carve(s.scratch, s.chi, s.max_nodes);
  k_tc_pack_W<<<dim3((Dp + 31) / 32, (D + 31) / 32, nc), dim3(32, 8), 0, st>>>(T, parent, edge, node_base, D, Dp,
                                                                               p.w);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int64_t N = (int64_t)nc * Dp;
  if (e0 && (e = cudaEventRecord(e0, st)) != cudaSuccess) return e;
  e = tc::launch_gemm_tf32x3(tc::Plane{p.a2, 4 * (int64_t)D}, tc::Plane{p.w, 4 * (int64_t)D}, 2 * Dp, (int)N, 4 * D,
                             p.cl, N, s.err, st);
  if (e != cudaSuccess) return e;
  if (e1 && (e = cudaEventRecord(e1, st)) != cudaSuccess) return e;
  k_tc_place<<<grid_for((int64_t)nc * Dp * Dp), 256, 0, st>>>(p.cl, Dp, nc, Lout);
  return cudaGetLastError();
}

}  // namespace mpsvqe
