// Environment contractions of the trie measurement on the tensor cores (mixed
// precision); see env_tc.cu for the GEMM formulation.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

#include "cx.cuh"

namespace mpsvqe {

// Scratch of one handle for chunks of up to max_nodes children at bond cap chi.
struct EnvTc {
  float* scratch = nullptr;   // env_tc_scratch_floats(chi, max_nodes) floats, 256-byte aligned
  int* err = nullptr;         // device int: set by a tensor-core pipeline wait that ran out
  int chi = 0;
  int max_nodes = 0;
};

size_t env_tc_scratch_floats(int chi, int max_nodes);

// Shared operands of site k (D = left bond, Dp = right bond), once per level chunk.
cudaError_t env_tc_site(const EnvTc& s, const Cx<float>* Bk, int D, int Dp, cudaStream_t st);
// T_j[u] = L[u] B^j for the U nodes of a dense level chunk (L[u] at u D^2; T written as
// T_j[u][a][c] at ((u D + a) 2 + j) D' + c; both 16-byte aligned, D and D' even).
// e0 / e1 (optional) are recorded on st right before and after the tensor-core GEMM.
cudaError_t env_tc_T(const EnvTc& s, const Cx<float>* L, Cx<float>* T, int U, int D, int Dp, cudaStream_t st,
                     cudaEvent_t e0 = nullptr, cudaEvent_t e1 = nullptr);
// L[child] = sum_ij P_ij (B^i)^+ T_j[parent] for nc <= max_nodes children (parent: trie
// node indices, node_base = the trie index of T's entry 0; edge: the letters P), written
// densely (child c at c D'^2).
cudaError_t env_tc_children(const EnvTc& s, const Cx<float>* T, const int32_t* parent, const uint8_t* edge, int nc,
                            int node_base, int D, int Dp, Cx<float>* Lout, cudaStream_t st,
                            cudaEvent_t e0 = nullptr, cudaEvent_t e1 = nullptr);

}  // namespace mpsvqe
