// Small complex-number helpers shared by the CUDA kernels (float and double).
#pragma once
#include <cuda_runtime.h>

namespace mpsvqe {

template <class R>
struct Cx {
  R x, y;
};

template <class R>
__host__ __device__ __forceinline__ Cx<R> cx(R a, R b) {
  Cx<R> o;
  o.x = a;
  o.y = b;
  return o;
}
template <class R>
__host__ __device__ __forceinline__ Cx<R> operator+(Cx<R> a, Cx<R> b) {
  return cx(a.x + b.x, a.y + b.y);
}
template <class R>
__host__ __device__ __forceinline__ Cx<R> operator-(Cx<R> a, Cx<R> b) {
  return cx(a.x - b.x, a.y - b.y);
}
template <class R>
__host__ __device__ __forceinline__ Cx<R> operator*(Cx<R> a, Cx<R> b) {
  return cx(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <class R>
__host__ __device__ __forceinline__ Cx<R> operator*(R s, Cx<R> a) {
  return cx(s * a.x, s * a.y);
}
template <class R>
__host__ __device__ __forceinline__ Cx<R> conj(Cx<R> a) {
  return cx(a.x, -a.y);
}
// acc += a * b
template <class R>
__device__ __forceinline__ void cmac(Cx<R>& acc, Cx<R> a, Cx<R> b) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(a.y, b.x, acc.y);
}
// acc += conj(a) * b
template <class R>
__device__ __forceinline__ void cmac_conj(Cx<R>& acc, Cx<R> a, Cx<R> b) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(-a.y, b.x, acc.y);
}
template <class R>
__device__ __forceinline__ R norm2(Cx<R> a) {
  return fma(a.x, a.x, a.y * a.y);
}

}  // namespace mpsvqe
