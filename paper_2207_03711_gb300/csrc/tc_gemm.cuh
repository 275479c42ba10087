// Tensor-core (tcgen05) GEMM with compensated TF32 splits: the contraction primitive of
// the environment sweeps in mixed precision (see tc_gemm.cu).
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

namespace mpsvqe {
namespace tc {

// An FP32 operand held as two planes, hi = tf32(x) and lo = tf32(x - hi), row-major
// with K contiguous and leading dimension ld (floats, a multiple of 4; both planes
// 16-byte aligned).
struct SplitPlane {
  const float* hi;
  const float* lo;
  int64_t ld;
};

// hi/lo split of an M x K row-major plane (leading dimension ld_in) into planes of
// leading dimension ld_out; columns K..ld_out-1 become zero.
cudaError_t launch_split_tf32(const float* x, int64_t ld_in, int M, int K, float* hi, float* lo, int64_t ld_out,
                              cudaStream_t st);

// C (M x N, leading dimension ldc) = A (M x K) . B (N x K)^T on the tensor cores as
// A_hi B_hi + A_hi B_lo + A_lo B_hi with FP32 accumulation. *err (device int) receives a
// non-zero code if a bounded pipeline wait ran out. Returns cudaErrorInvalidValue for
// misaligned planes.
cudaError_t launch_gemm_tf32x3(const SplitPlane& A, const SplitPlane& B, int M, int N, int K, float* C, int64_t ldc,
                               int* err, cudaStream_t st);

}  // namespace tc
}  // namespace mpsvqe
