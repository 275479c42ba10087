// Tensor-core (tcgen05) GEMM with compensated TF32 splits: the contraction primitive of
// the environment sweeps in mixed precision (see tc_gemm.cu).
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

namespace mpsvqe {
namespace tc {

// An FP32 operand, row-major with K contiguous and leading dimension ld (floats, a
// multiple of 4), 16-byte aligned.
struct Plane {
  const float* p;
  int64_t ld;
};

// Copy of an M x K row-major plane (leading dimension ld_in) into one of leading
// dimension ld_out; columns K..ld_out-1 become zero.
cudaError_t launch_pad_rows(const float* x, int64_t ld_in, int M, int K, float* out, int64_t ld_out,
                            cudaStream_t st);

// C (M x N, leading dimension ldc) = A (M x K) . B (N x K)^T on the tensor cores as
// A_hi B_hi + A_hi B_lo + A_lo B_hi (hi/lo TF32 splits made in shared memory) with
// round-to-nearest FP32 sums of per-K-tile accumulations. *err (device int) receives a
// non-zero code if a bounded pipeline wait ran out. Returns cudaErrorInvalidValue for
// misaligned planes.
cudaError_t launch_gemm_tf32x3(const Plane& A, const Plane& B, int M, int N, int K, float* C, int64_t ldc, int* err,
                               cudaStream_t st);

}  // namespace tc
}  // namespace mpsvqe
