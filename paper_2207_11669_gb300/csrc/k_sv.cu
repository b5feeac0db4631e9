// Singular values of a factored matrix L = X Y^T (X: N1 x p, Y: N2 x p,
// row-major), for the relative singular-value error of the upper-bound-rank
// experiments (§4.2 "Upper-bound rank recovery", Table 1).
//
// With G_x = X^T X and G_y = Y^T Y, the nonzero singular values of X Y^T are
// the square roots of the eigenvalues of the symmetric positive semidefinite
// p x p matrix G_x^{1/2} G_y G_x^{1/2}: it is similar to G_x G_y, whose
// eigenvalues are those of X^T X Y^T Y, i.e. the squared singular values of
// X Y^T.  Every product of two FP32 entries is exact in FP64, so the Gram
// matrices are summed in FP64 (k_gram64_part per row range, then a fixed-order
// sum over the ranges).  The square root of G_x and the eigenvalues come from
// the cyclic Jacobi method (Jacobi 1846; as in Golub and Van Loan,
// "Matrix Computations", §8.5): plane rotations J chosen to zero one
// off-diagonal pair each, A <- J^T A J, swept pair by pair until the
// off-diagonal mass is negligible.  Each problem runs in one warp.
#include "dcf_internal.cuh"

namespace dcf {

constexpr int kSvMax = 64;           // largest p
constexpr int kSvChunk = 32;         // rows staged in shared memory per step

// part[b][i * p + j] = sum over rows a in range b of X[a, i] * Y[a, j] (FP64)
__global__ void __launch_bounds__(256)
    k_gram64_part(const float* __restrict__ X, int ldx, const float* __restrict__ Y, int ldy,
                  int p, int64_t N, int64_t rows_per, double* __restrict__ part) {
  __shared__ float xs[kSvChunk * kSvMax], ys[kSvChunk * kSvMax];
  const int tid = threadIdx.x;
  const int ne = p * p;
  double acc[kSvMax * kSvMax / 256];
#pragma unroll
  for (int s = 0; s < kSvMax * kSvMax / 256; ++s) acc[s] = 0.0;
  const int64_t a0 = (int64_t)blockIdx.x * rows_per;
  const int64_t a1 = a0 + rows_per < N ? a0 + rows_per : N;
  for (int64_t c = a0; c < a1; c += kSvChunk) {
    const int rows = (int)(a1 - c < kSvChunk ? a1 - c : kSvChunk);
    __syncthreads();
    for (int i = tid; i < kSvChunk * p; i += 256) {
      const int rr = i / p, k = i % p;
      xs[i] = rr < rows ? X[(c + rr) * ldx + k] : 0.f;
      ys[i] = rr < rows ? Y[(c + rr) * ldy + k] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int s = 0; s < kSvMax * kSvMax / 256; ++s) {
      const int e = tid + 256 * s;
      if (e < ne) {
        const int i = e / p, j = e % p;
        double t = acc[s];
        for (int rr = 0; rr < rows; ++rr)
          t = fma((double)xs[rr * p + i], (double)ys[rr * p + j], t);
        acc[s] = t;
      }
    }
  }
#pragma unroll
  for (int s = 0; s < kSvMax * kSvMax / 256; ++s) {
    const int e = tid + 256 * s;
    if (e < ne) part[(size_t)blockIdx.x * ne + e] = acc[s];
  }
}

// out[e] = sum over b (in order) of part[b][e]
__global__ void k_gram64_reduce(const double* __restrict__ part, int nparts, int ne,
                                double* __restrict__ out) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= ne) return;
  double t = 0.0;
  for (int b = 0; b < nparts; ++b) t += part[(size_t)b * ne + e];
  out[e] = t;
}

// One cyclic Jacobi sweep set on the symmetric p x p matrix A (shared memory,
// row-major), by one warp; W (if non-NULL) accumulates the rotations, so that
// on return A_in = W diag(A) W^T.  Every lane computes the same rotation from
// the same shared values, so the decisions are uniform across the warp.
__device__ void jacobi_sym(double* A, double* W, int p) {
  const int lane = threadIdx.x & 31;
  for (int sweep = 0; sweep < 60; ++sweep) {
    double off = 0.0, dia = 0.0;
    for (int i = lane; i < p; i += 32) {
      dia += A[i * p + i] * A[i * p + i];
      for (int j = i + 1; j < p; ++j) off += A[i * p + j] * A[i * p + j];
    }
    for (int o = 16; o > 0; o >>= 1) {
      off += __shfl_xor_sync(0xffffffffu, off, o);
      dia += __shfl_xor_sync(0xffffffffu, dia, o);
    }
    if (!(off > 1e-32 * dia)) break;   // off-diagonal mass negligible (also when all zero)
    for (int pi = 0; pi < p - 1; ++pi) {
      for (int q = pi + 1; q < p; ++q) {
        const double apq = A[pi * p + q];
        const double app = A[pi * p + pi], aqq = A[q * p + q];
        // a negligible pair needs no rotation
        if (fabs(apq) <= 1e-18 * sqrt(fabs(app * aqq)) || apq == 0.0) continue;
        // J^T A J has (p,q) entry (c^2 - s^2) a_pq + c s (a_pp - a_qq); with
        // t = s / c that is zero for t^2 + 2 theta t - 1 = 0, theta =
        // (a_qq - a_pp) / (2 a_pq); the root of smaller magnitude keeps the
        // rotation angle at most pi/4
        const double theta = (aqq - app) / (2.0 * apq);
        const double t = fabs(theta) > 1e150
                             ? 0.5 / theta
                             : (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
        const double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
        __syncwarp();
        for (int k = lane; k < p; k += 32) {           // A <- A J (columns p, q)
          const double akp = A[k * p + pi], akq = A[k * p + q];
          A[k * p + pi] = c * akp - s * akq;
          A[k * p + q] = s * akp + c * akq;
          if (W) {
            const double wkp = W[k * p + pi], wkq = W[k * p + q];
            W[k * p + pi] = c * wkp - s * wkq;
            W[k * p + q] = s * wkp + c * wkq;
          }
        }
        __syncwarp();
        for (int k = lane; k < p; k += 32) {           // A <- J^T A (rows p, q)
          const double apk = A[pi * p + k], aqk = A[q * p + k];
          A[pi * p + k] = c * apk - s * aqk;
          A[q * p + k] = s * apk + c * aqk;
        }
        __syncwarp();
        if (lane == 0) {
          A[pi * p + q] = 0.0;
          A[q * p + pi] = 0.0;
        }
        __syncwarp();
      }
    }
  }
}

// Problem b: Gram matrices gram[b][0] = G_x, gram[b][1] = G_y (p_b x p_b,
// FP64).  Writes the p_b singular values of X Y^T, descending, to
// sig[b * kSvMax + i] (zero beyond p_b).  One warp per problem.
__global__ void __launch_bounds__(32) k_sv_factored(const double* __restrict__ gram,
                                                    const int* __restrict__ pdim,
                                                    double* __restrict__ sig) {
  extern __shared__ double svm[];
  const int b = blockIdx.x, lane = threadIdx.x;
  const int p = pdim[b];
  double* A = svm;                      // p x p working matrix
  double* W = svm + kSvMax * kSvMax;    // eigenvectors of G_x
  double* T = svm + 2 * kSvMax * kSvMax;
  const double* Gx = gram + (size_t)b * 2 * kSvMax * kSvMax;
  const double* Gy = Gx + kSvMax * kSvMax;
  for (int i = lane; i < kSvMax; i += 32) sig[b * kSvMax + i] = 0.0;
  if (p < 1) return;
  for (int e = lane; e < p * p; e += 32) {
    A[e] = Gx[e];
    W[e] = (e / p == e % p) ? 1.0 : 0.0;
  }
  __syncwarp();
  jacobi_sym(A, W, p);                  // G_x = W diag(lambda) W^T
  __syncwarp();
  // T = G_x^{1/2} = W diag(sqrt(max(lambda, 0))) W^T
  for (int e = lane; e < p * p; e += 32) {
    const int i = e / p, j = e % p;
    double t = 0.0;
    for (int k = 0; k < p; ++k) {
      const double lk = A[k * p + k];
      t = fma(W[i * p + k] * (lk > 0.0 ? sqrt(lk) : 0.0), W[j * p + k], t);
    }
    T[e] = t;
  }
  __syncwarp();
  // W <- T G_y, then A <- (T G_y) T = G_x^{1/2} G_y G_x^{1/2}
  for (int e = lane; e < p * p; e += 32) {
    const int i = e / p, j = e % p;
    double t = 0.0;
    for (int k = 0; k < p; ++k) t = fma(T[i * p + k], Gy[k * p + j], t);
    W[e] = t;
  }
  __syncwarp();
  for (int e = lane; e < p * p; e += 32) {
    const int i = e / p, j = e % p;
    double t = 0.0;
    for (int k = 0; k < p; ++k) t = fma(W[i * p + k], T[k * p + j], t);
    A[e] = t;
  }
  __syncwarp();
  for (int e = lane; e < p * p; e += 32) {   // exact symmetry before the rotations
    const int i = e / p, j = e % p;
    if (i < j) {
      const double v = 0.5 * (A[i * p + j] + A[j * p + i]);
      A[i * p + j] = v;
      A[j * p + i] = v;
    }
  }
  __syncwarp();
  jacobi_sym(A, nullptr, p);
  __syncwarp();
  if (lane == 0) {
    for (int i = 0; i < p; ++i) {
      const double v = A[i * p + i];
      T[i] = v > 0.0 ? sqrt(v) : 0.0;
    }
    for (int i = 1; i < p; ++i) {          // insertion sort, descending
      const double v = T[i];
      int j = i - 1;
      while (j >= 0 && T[j] < v) {
        T[j + 1] = T[j];
        --j;
      }
      T[j + 1] = v;
    }
    for (int i = 0; i < p; ++i) sig[b * kSvMax + i] = T[i];
  }
}

// err = max_i |sig[i] - sig0[i]| / sig0[k - 1] over i < kSvMax (missing values
// are zero): the relative singular-value error of Table 1, k = rank of L0.
__global__ void k_sv_error(const double* __restrict__ sig, const double* __restrict__ sig0,
                           int k, double* __restrict__ err) {
  if (threadIdx.x != 0) return;
  double mx = 0.0;
  for (int i = 0; i < kSvMax; ++i) mx = fmax(mx, fabs(sig[i] - sig0[i]));
  const double den = k >= 1 ? sig0[k - 1] : 0.0;
  *err = den > 0.0 ? mx / den : INFINITY;
}

size_t sv_part_doubles(int nparts) { return (size_t)nparts * kSvMax * kSvMax; }
size_t sv_smem_bytes() { return (size_t)3 * kSvMax * kSvMax * sizeof(double); }

cudaError_t sv_prepare() {
  return cudaFuncSetAttribute(k_sv_factored, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)sv_smem_bytes());
}

// gram_out (p x p, FP64) = X^T Y over N rows, through `part` (nparts partials)
cudaError_t launch_gram64(const float* X, int ldx, const float* Y, int ldy, int p, int64_t N,
                          double* part, int nparts, double* gram_out, cudaStream_t s) {
  if (p < 1 || p > kSvMax) return cudaErrorInvalidValue;
  if (nparts < 1) nparts = 1;
  const int64_t rows_per = (N + nparts - 1) / nparts;
  const int used = (int)((N + rows_per - 1) / rows_per);
  k_gram64_part<<<used, 256, 0, s>>>(X, ldx, Y, ldy, p, N, rows_per, part);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_gram64_reduce<<<(p * p + 255) / 256, 256, 0, s>>>(part, used, p * p, gram_out);
  return cudaGetLastError();
}

cudaError_t launch_sv_factored(const double* gram, const int* pdim, int nprob, double* sig,
                               cudaStream_t s) {
  k_sv_factored<<<nprob, 32, sv_smem_bytes(), s>>>(gram, pdim, sig);
  return cudaGetLastError();
}

cudaError_t launch_sv_error(const double* sig, const double* sig0, int k, double* err,
                            cudaStream_t s) {
  k_sv_error<<<1, 32, 0, s>>>(sig, sig0, k, err);
  return cudaGetLastError();
}

}  // namespace dcf
