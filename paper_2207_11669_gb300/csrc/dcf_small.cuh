// r x r linear algebra on one CTA (shared memory), used by the reduction
// tails and by the adjoint of the unrolled network.
#pragma once
#include <cuda_runtime.h>

namespace dcf {

// ---------------------------------------------------------------------------
// FP64 Cholesky (lower, in place, row-major R x R in shared memory).
// Block-wide; every thread of the CTA must call it.
// ---------------------------------------------------------------------------
static __device__ __noinline__ void chol_inplace(double* A, int R) {
  for (int k = 0; k < R; ++k) {
    double d = sqrt(A[k * R + k]);
    __syncthreads();
    for (int i = k + threadIdx.x; i < R; i += blockDim.x) {
      if (i == k) A[k * R + k] = d;
      else A[i * R + k] = A[i * R + k] / d;
    }
    __syncthreads();
    const int nt = R - k - 1;
    for (int idx = threadIdx.x; idx < nt * nt; idx += blockDim.x) {
      int i = k + 1 + idx / nt, j = k + 1 + idx % nt;
      if (j <= i) A[i * R + j] -= A[i * R + k] * A[j * R + k];
    }
    __syncthreads();
  }
  for (int idx = threadIdx.x; idx < R * R; idx += blockDim.x) {
    int i = idx / R, j = idx % R;
    if (j > i) A[idx] = 0.0;
  }
  __syncthreads();
}

static __device__ __noinline__ int all_finite(const double* A, int n) {
  __shared__ int ok;
  if (threadIdx.x == 0) ok = 1;
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x)
    if (!isfinite(A[i])) ok = 0;
  __syncthreads();
  int r = ok;
  __syncthreads();
  return r;
}

// SPD inverse: FP64 Cholesky G = L L^T in place (the stability-critical step),
// then L^{-1} and G^{-1} = L^{-T} L^{-1} in FP32 from the rounded factor.
// A: R*R doubles (shared, destroyed); F: R*R floats (shared scratch).
// Block-wide.  The FP32 part keeps the work off GB300's slow FP64 pipe;
// its relative error is about cond(G) * 2^-24.
static __device__ __noinline__ void spd_inverse_f32(double* A, float* F, int R, float* out) {
  chol_inplace(A, R);
  for (int i = threadIdx.x; i < R * R; i += blockDim.x) F[i] = (float)A[i];
  __syncthreads();
  float* Li = reinterpret_cast<float*>(A);   // reuse: R*R floats fit in R*R doubles
  for (int c = threadIdx.x; c < R; c += blockDim.x) {
    for (int i = 0; i < R; ++i) {
      float y;
      if (i < c) {
        y = 0.f;
      } else if (i == c) {
        y = 1.0f / F[c * R + c];
      } else {
        float s = 0.f;
        for (int p = c; p < i; ++p) s = fmaf(F[i * R + p], Li[p * R + c], s);
        y = -s / F[i * R + i];
      }
      Li[i * R + c] = y;
    }
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < R * R; idx += blockDim.x) {
    int i = idx / R, j = idx % R;
    int k0 = i > j ? i : j;
    float s = 0.f;
    for (int k = k0; k < R; ++k) s = fmaf(Li[k * R + i], Li[k * R + j], s);
    out[idx] = s;
  }
  __syncthreads();
}


}  // namespace dcf
