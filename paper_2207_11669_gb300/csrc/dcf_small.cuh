// r x r linear algebra on one CTA (shared memory), used by the reduction
// tails and by the learned network.
//
// Cost model.  GB300 issues an FP64 warp instruction every 64 cycles per SM
// sub-partition (about 2 FP64 FMA/clk/SM), so the code below keeps FP64 to
// the factorisation itself, packs its trailing updates across all threads of
// the CTA, uses the root-free L D L^T form and replaces FP64 divisions by
// Newton steps from the FP32 estimate.  The triangular inverse and the final
// product are FP32 and run one warp per column.
#pragma once
#include <cuda_runtime.h>

#include "dcf_internal.cuh"

namespace dcf {

// ---------------------------------------------------------------------------
// FP64 root-free Cholesky G = L D L^T (L unit lower triangular), in place on a
// row-major R x R matrix in shared memory (R <= 64): on return the strict
// lower triangle holds L, the diagonal holds 1/D, the upper triangle is zero.
// Block-wide: every thread of the CTA must call it.  A non-positive pivot
// leaves NaN.
//
// Step k updates the trailing lower triangle with the unscaled column,
//   A_ij -= A_ik (A_jk / D_k),
// which needs one barrier per step: thread 0 updates A_{k+1,k+1} first and
// forms the next reciprocal 1/D_{k+1} (FP32 estimate, one FP64 Newton step)
// while warps 1.. finish the step.
// ---------------------------------------------------------------------------
static __device__ __forceinline__ double recip_f64(double a) {
  // FP32 estimate (relative error <= 2^-23), one Newton step: error ~ 2^-46
  const double r = a > 0.0 ? (double)__frcp_rn((float)a) : __longlong_as_double(0x7ff8000000000000LL);
  const double e = fma(-a, r, 1.0);
  return fma(r, e, r);
}

static __device__ __noinline__ void chol_inplace(double* A, int R) {
  __shared__ double s_r[kMaxR];          // 1 / D_k
  const int tid = threadIdx.x, nt = blockDim.x;
  if (tid == 0) s_r[0] = recip_f64(A[0]);
  __syncthreads();
  for (int k = 0; k + 1 < R; ++k) {
    const double rk = s_r[k];
    const int m = R - k - 1;
    const int count = m * (m + 1) / 2;     // entries (i, j), k < j <= i
    if (tid == 0) {
      // entry (k+1, k+1) first, then the next pivot's reciprocal
      const int i = k + 1;
      const double v = fma(-A[i * R + k], A[i * R + k] * rk, A[i * R + i]);
      A[i * R + i] = v;
      s_r[k + 1] = recip_f64(v);
    }
    // the other entries, flattened over warps 1 .. (so that warp 0 runs only
    // the pivot chain); entry t = 0 is (k+1, k+1)
    for (int t = tid - 31; t < count; t += nt - 32) {
      if (tid < 32) break;
      int ii = (int)((sqrtf(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);
      while ((ii + 1) * (ii + 2) / 2 <= t) ++ii;
      while (ii * (ii + 1) / 2 > t) --ii;
      const int jj = t - ii * (ii + 1) / 2;
      const int i = k + 1 + ii, j = k + 1 + jj;
      A[i * R + j] = fma(-A[i * R + k], A[j * R + k] * rk, A[i * R + j]);
    }
    __syncthreads();
  }
  // L_ik = A_ik / D_k below the diagonal; 1/D_k on it; zeros above
  for (int idx = tid; idx < R * R; idx += nt) {
    const int i = idx / R, j = idx % R;
    if (j < i) A[idx] *= s_r[j];
    else if (j == i) A[idx] = s_r[i];
    else A[idx] = 0.0;
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

// SPD inverse: FP64 factorisation G = L D L^T in place (the stability-critical
// step), then L^{-1} and G^{-1} = L^{-T} D^{-1} L^{-1} in FP32 from the
// rounded factors.  A: R*R doubles (shared, destroyed); F: R*R floats (shared
// scratch); out: R*R floats (any memory).  Block-wide, R <= 64, R even.
static __device__ __noinline__ void spd_inverse_f32(double* A, float* F, int R, float* out) {
  chol_inplace(A, R);
  const int tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
  // F = L^T in FP32 (row p of F is column p of L), so that a warp reads a
  // column of L with consecutive addresses
  for (int idx = tid; idx < R * R; idx += nt) {
    const int i = idx / R, p = idx % R;
    F[p * R + i] = (float)A[idx];
  }
  __syncthreads();
  float* Li = reinterpret_cast<float*>(A);   // R*R floats fit in the R*R doubles ...
  float* dinv = Li + R * R;                  // ... and so do R more
  for (int i = tid; i < R; i += nt) dinv[i] = F[i * R + i];
  __syncthreads();
  // L^{-1} (unit lower): one warp per column c (columns dealt in snake order
  // so that every warp gets the same number of steps), lanes hold rows
  // (lane, lane + 32)
  for (int round = 0; round * nw < R; ++round) {
    const int c = (round & 1) ? (round + 1) * nw - 1 - warp : round * nw + warp;
    if (c >= R) continue;
    float acc0 = 0.f, acc1 = 0.f, y0 = 0.f, y1 = 0.f;
    for (int i = c; i < R; ++i) {
      // row i finalises y_i = delta_ic - acc_i
      const float acc_i = __shfl_sync(0xffffffffu, i < 32 ? acc0 : acc1, i & 31);
      const float yi = (i == c ? 1.f : 0.f) - acc_i;
      if (lane == (i & 31)) { if (i < 32) y0 = yi; else y1 = yi; }
      // rows below i: acc_j += L_ji y_i  (L_ji = F[i][j])
      const int j0 = lane, j1 = lane + 32;
      if (j0 > i && j0 < R) acc0 = fmaf(F[i * R + j0], yi, acc0);
      if (j1 > i && j1 < R) acc1 = fmaf(F[i * R + j1], yi, acc1);
    }
    if (lane < R) Li[lane * R + c] = lane >= c ? y0 : 0.f;
    if (lane + 32 < R) Li[(lane + 32) * R + c] = lane + 32 >= c ? y1 : 0.f;
  }
  __syncthreads();
  // G^{-1}[i][j] = sum_{k >= max(i,j)} Li[k][i] D_k^{-1} Li[k][j]: 2 x 2 blocks
  // of the upper triangle, mirrored
  const int nb = R / 2;
  for (int b = tid; b < nb * nb; b += nt) {
    const int bi = b / nb, bj = b % nb;
    if (bi > bj) continue;
    const int i = 2 * bi, j = 2 * bj;
    float s00 = 0.f, s01 = 0.f, s10 = 0.f, s11 = 0.f;
    for (int k = j; k < R; ++k) {      // j >= i
      const float d = dinv[k];
      const float2 li = *reinterpret_cast<const float2*>(Li + k * R + i);
      float2 lj = *reinterpret_cast<const float2*>(Li + k * R + j);
      lj.x *= d;
      lj.y *= d;
      s00 = fmaf(li.x, lj.x, s00);
      s01 = fmaf(li.x, lj.y, s01);
      s10 = fmaf(li.y, lj.x, s10);
      s11 = fmaf(li.y, lj.y, s11);
    }
    // terms with k < max(row, column) vanish (Li is lower triangular), so
    // starting at k = j covers all four entries of the block
    out[i * R + j] = s00;
    out[i * R + j + 1] = s01;
    out[(i + 1) * R + j] = s10;
    out[(i + 1) * R + j + 1] = s11;
    out[j * R + i] = s00;
    out[(j + 1) * R + i] = s01;
    out[j * R + i + 1] = s10;
    out[(j + 1) * R + i + 1] = s11;
  }
  __syncthreads();
}

// Sum of v over the CTA (FP64, shuffle tree then one value per warp).
// Block-wide; `scratch` holds one double per warp.
static __device__ __forceinline__ double block_sum_f64(double v, double* scratch) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __syncthreads();
  if (lane == 0) scratch[warp] = v;
  __syncthreads();
  double t = 0.0;
  for (int w = 0; w < nw; ++w) t += scratch[w];
  __syncthreads();
  return t;
}

}  // namespace dcf
