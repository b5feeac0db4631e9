// r x r linear algebra on one CTA (shared memory), used by the reduction
// tails and by the learned network.
//
// Cost model.  GB300 issues an FP64 warp instruction every 64 cycles per SM
// sub-partition (about 2 FP64 FMA/clk/SM), and a factorisation is a chain of
// R dependent steps, so it runs in double-float arithmetic on the FP32 pipes
// (about 48 bits), packs its trailing updates across all threads of the CTA,
// uses the root-free L D L^T form and replaces divisions by Newton steps from
// the FP32 estimate.  A well-conditioned system (by a 1-norm estimate) is
// inverted in FP32: by Gauss-Jordan on one warp up to R = 32, from the
// rounded double-float factors at R = 64; otherwise the triangular inverse
// and the product run in double-float and the inverse is handed on as a pair
// of floats (hi, lo), so that its consumers can apply it to about twice FP32
// precision.  The tails run once per launch on one CTA, after larger kernels
// have evicted the instruction cache, so their loops are kept rolled.
#pragma once
#include <cuda_runtime.h>

#include "dcf_internal.cuh"

namespace dcf {

// ---------------------------------------------------------------------------
// Double-float arithmetic: a value is an unevaluated sum h + l of two floats
// with |l| <= ulp(h)/2 (about 48 significant bits).  The building blocks are
// Knuth's two-sum, Dekker's fast two-sum and the FMA form of the exact
// product (p = a b rounded, e = fma(a, b, -p), so that p + e = a b exactly).
// They run on the FP32 pipes, 64 times wider than the FP64 pipe of this GPU.
// ---------------------------------------------------------------------------
struct df2 {
  float h, l;
};

static __device__ __forceinline__ df2 df_fast_two_sum(float a, float b) {   // |a| >= |b|
  const float s = a + b;
  return {s, b - (s - a)};
}

static __device__ __forceinline__ df2 df_two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  return {s, (a - (s - bb)) + (b - bb)};
}

static __device__ __forceinline__ df2 df_mul(df2 x, df2 y) {
  const float p = x.h * y.h;
  float e = fmaf(x.h, y.h, -p);
  e = fmaf(x.h, y.l, e);
  e = fmaf(x.l, y.h, e);
  return df_fast_two_sum(p, e);
}

static __device__ __forceinline__ df2 df_sub(df2 x, df2 y) {
  const df2 s = df_two_sum(x.h, -y.h);
  return df_fast_two_sum(s.h, s.l + (x.l - y.l));
}

static __device__ __forceinline__ df2 df_add(df2 x, df2 y) {
  const df2 s = df_two_sum(x.h, y.h);
  return df_fast_two_sum(s.h, s.l + (x.l + y.l));
}

// 1/d: the hardware reciprocal estimate x0 (relative error about 2^-22),
// then one Newton step x0 + x0 (1 - d x0) with the residual formed exactly
// enough in double-float: relative error about 2^-44.  d <= 0 or non-finite
// gives NaN.
static __device__ __forceinline__ df2 df_recip(df2 d) {
  if (!(d.h > 0.f) || !isfinite(d.h)) return {__int_as_float(0x7fc00000), 0.f};
  const float x0 = __fdividef(1.f, d.h);
  const float p = d.h * x0;
  const float pe = fmaf(d.h, x0, -p);            // d.h x0 = p + pe exactly
  float e = (1.f - p) - pe;                      // 1 - p is exact (p is within 2^-21 of 1)
  e = fmaf(-d.l, x0, e);
  return df_fast_two_sum(x0, x0 * e);
}

// FP64 1/a: the FP32 estimate (relative error <= 2^-23) and one FP64 Newton
// step (error about 2^-46).
static __device__ __forceinline__ double recip_f64(double a) {
  const double r = a > 0.0 ? (double)__frcp_rn((float)a) : __longlong_as_double(0x7ff8000000000000LL);
  const double e = fma(-a, r, 1.0);
  return fma(r, e, r);
}

static __device__ __forceinline__ df2 df_from_double(double x) {
  const float h = (float)x;
  return {h, (float)(x - (double)h)};
}

// ---------------------------------------------------------------------------
// Root-free Cholesky G = L D L^T (L unit lower triangular) in double-float.
// Block-wide, 256 threads, R <= 64.  Thread t owns the lower-triangle entries
// e = t, t + 256, ... (e = i (i + 1) / 2 + j, j <= i) and keeps them in
// registers for the whole factorisation.  Step k updates every owned entry
// with j > k,
//   A_ij -= A_ik (A_jk / D_k),
// from column k, which the owners of that column publish to shared memory
// (double-buffered) together with 1/D_k; the owner of A_{k+1,k+1} forms
// 1/D_{k+1} right after its update.  One barrier per step.
//
// Input: A (R*R doubles, row-major, lower triangle read).  Output: F = L^T in
// double-float with 1/D_k on the diagonal (row p of F is column p of L) and
// zeros below its diagonal; s_r[k] = 1/D_k; Ff (optional, may alias the space
// of A, which is read only before the first barrier): the entries of F on and
// above its diagonal rounded to FP32.  A non-positive pivot leaves NaN.
// ---------------------------------------------------------------------------
constexpr int kCholThreads = 256;

// kCholSlots = ceil(R (R + 1) / 2 / 256) for the largest R of the instance
template <int kCholSlots>
static __device__ __noinline__ void chol_df(const double* A, int R, df2* F, float* Ff, df2* col,
                                            df2* s_r) {
  const int tid = threadIdx.x;
  const int ne = R * (R + 1) / 2;
  df2 a[kCholSlots];
  int ei[kCholSlots], ej[kCholSlots];
#pragma unroll
  for (int q = 0; q < kCholSlots; ++q) {
    const int e = tid + q * kCholThreads;
    int i = -1, j = 0;
    if (e < ne) {
      i = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);
      while ((i + 1) * (i + 2) / 2 <= e) ++i;
      while (i * (i + 1) / 2 > e) --i;
      j = e - i * (i + 1) / 2;
      a[q] = df_from_double(A[i * R + j]);
    } else {
      a[q] = {0.f, 0.f};
    }
    ei[q] = i;
    ej[q] = j;
  }
  for (int idx = tid; idx < R * R; idx += kCholThreads) F[idx] = {0.f, 0.f};
  // column 0 and 1/D_0
#pragma unroll
  for (int q = 0; q < kCholSlots; ++q) {
    if (ei[q] >= 0 && ej[q] == 0) col[ei[q]] = a[q];
    if (ei[q] == 0) s_r[0] = df_recip(a[q]);
  }
  __syncthreads();
  for (int k = 0; k + 1 < R; ++k) {
    const df2* ck = col + (k & 1) * kMaxR;          // column k
    df2* cn = col + ((k + 1) & 1) * kMaxR;          // column k + 1, published below
    const df2 rk = s_r[k];
    // every load of the step before any store, so that the owned entries'
    // updates overlap instead of queueing behind each other's stores
    df2 ci[kCholSlots], cj[kCholSlots];
#pragma unroll
    for (int q = 0; q < kCholSlots; ++q) {
      const bool act = ei[q] >= 0 && ej[q] > k;
      ci[q] = ck[act ? ei[q] : 0];
      cj[q] = ck[act ? ej[q] : 0];
    }
#pragma unroll
    for (int q = 0; q < kCholSlots; ++q)
      if (ei[q] >= 0 && ej[q] > k) a[q] = df_sub(a[q], df_mul(ci[q], df_mul(cj[q], rk)));
#pragma unroll
    for (int q = 0; q < kCholSlots; ++q) {
      if (ei[q] >= 0 && ej[q] == k + 1) {
        cn[ei[q]] = a[q];
        if (ei[q] == k + 1) s_r[k + 1] = df_recip(a[q]);
      }
    }
    __syncthreads();
  }
  // L_ij = A_ij / D_j below the diagonal, 1/D_i on it
#pragma unroll
  for (int q = 0; q < kCholSlots; ++q) {
    const int i = ei[q], j = ej[q];
    if (i < 0) continue;
    const df2 v = j < i ? df_mul(a[q], s_r[j]) : s_r[i];
    F[j * R + i] = v;
    if (Ff) Ff[j * R + i] = v.h + v.l;
  }
  __syncthreads();
}

// Row and column (i >= j) of entry e of a packed lower triangle.
static __device__ __forceinline__ void tri_decode(int e, int& i, int& j) {
  i = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);
  while ((i + 1) * (i + 2) / 2 <= e) ++i;
  while (i * (i + 1) / 2 > e) --i;
  j = e - i * (i + 1) / 2;
}

// The same L D L^T by blocks of 8 columns (R a multiple of 8), with the
// output contract of chol_df.  The unblocked form pays one block barrier per
// column on a chain of R dependent steps; here a block of 8 columns costs
// three: (a) warp 0 factors the 8 x 8 diagonal block (warp-synchronous
// steps), (b) the rows below it are brought through the block's 8 steps,
// 8 threads per row exchanging values by shuffles, (c) the trailing matrix
// takes the block's rank-8 update, every entry independently.  Working
// storage is F itself: row j of F holds column j of the lower triangle,
// unscaled (W = L D) until the end, where L = W D^{-1} and 1/D_k on the
// diagonal are written.
static __device__ __noinline__ void chol_df_blocked(const double* A, int R, df2* F, float* Ff,
                                                    df2* s_r) {
  __shared__ df2 Lt[8 * 8];        // Lt[m * 8 + c] = L_{k0+c, k0+m} of the diagonal block
  __shared__ df2 Lp[8 * kMaxR];    // Lp[m * R + i] = L_{i, k0+m} of the panel
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5;
  for (int idx = tid; idx < R * R; idx += nt) {
    const int r = idx / R, c = idx % R;
    F[idx] = c >= r ? df_from_double(A[idx]) : df2{0.f, 0.f};
  }
  __syncthreads();
  for (int k0 = 0; k0 < R; k0 += 8) {
    // (a) diagonal block
    if (warp == 0) {
      for (int mm = 0; mm < 8; ++mm) {
        const int m = k0 + mm;
        const df2 rm = df_recip(F[m * R + m]);
        if (lane == 0) s_r[m] = rm;
        const int nrem = 7 - mm;
        if (lane < nrem * (nrem + 1) / 2) {
          int ii, jj;
          tri_decode(lane, ii, jj);
          const int i = m + 1 + ii, j = m + 1 + jj;
          F[j * R + i] = df_sub(F[j * R + i], df_mul(F[m * R + i], df_mul(F[m * R + j], rm)));
        }
        __syncwarp();
      }
      for (int e = lane; e < 64; e += 32) {
        const int mm = e / 8, c = e % 8;
        Lt[e] = c > mm ? df_mul(F[(k0 + mm) * R + k0 + c], s_r[k0 + mm]) : df2{0.f, 0.f};
      }
    }
    __syncthreads();
    // (b) panel: rows i >= k0 + 8, thread (row, c) holds A_{i, k0+c}
    const int nrows = R - k0 - 8;
    const int tot = (nrows * 8 + 31) / 32 * 32;   // whole warps, for the shuffles
    for (int t = tid; t < tot; t += nt) {
      const int row = t / 8, c = t % 8, i = k0 + 8 + row;
      const bool act = row < nrows;
      df2 a = act ? F[(k0 + c) * R + i] : df2{0.f, 0.f};
      for (int mm = 0; mm < 7; ++mm) {
        const float ah = __shfl_sync(0xffffffffu, a.h, (lane & ~7) + mm);
        const float al = __shfl_sync(0xffffffffu, a.l, (lane & ~7) + mm);
        if (c > mm) a = df_sub(a, df_mul(df2{ah, al}, Lt[mm * 8 + c]));
      }
      if (act) {
        F[(k0 + c) * R + i] = a;
        Lp[c * R + i] = df_mul(a, s_r[k0 + c]);
      }
    }
    __syncthreads();
    // (c) trailing matrix: A_ij -= sum_m W_{i,m} L_{j,m} over the block's columns
    const int nt2 = nrows * (nrows + 1) / 2;
    for (int e = tid; e < nt2; e += nt) {
      int ii, jj;
      tri_decode(e, ii, jj);
      const int i = k0 + 8 + ii, j = k0 + 8 + jj;
      df2 acc = df_mul(F[k0 * R + i], Lp[j]);
#pragma unroll
      for (int mm = 1; mm < 8; ++mm) acc = df_add(acc, df_mul(F[(k0 + mm) * R + i], Lp[mm * R + j]));
      F[j * R + i] = df_sub(F[j * R + i], acc);
    }
    __syncthreads();
  }
  // L = W D^{-1} above the diagonal of F, 1/D_k on it
  for (int idx = tid; idx < R * R; idx += nt) {
    const int r = idx / R, c = idx % R;
    if (c < r) continue;
    const df2 v = c > r ? df_mul(F[idx], s_r[r]) : s_r[r];
    F[idx] = v;
    if (Ff) Ff[idx] = v.h + v.l;
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

// Column sums for a 1-norm: thread (column c, row phase p) sums rows
// p, p + nt/R, ... of column c of X (R x R floats, shared) into part[tid].
static __device__ __forceinline__ void colsum_part(const float* X, int R, int rn, float* part) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const int col = tid % R, phase = tid / R, nphase = nt / R;
  float cs = 0.f;
  if (col < rn && phase < nphase)
    for (int i = phase; i < rn; i += nphase) cs += fabsf(X[i * R + col]);
  part[tid] = cs;
}

// max over columns c < rn of the phase sums in part (filled by colsum_part
// or the same layout).  Block-wide; the same value on every thread.
static __device__ float part_colmax(const float* part, int R, int rn) {
  __shared__ float s_max;
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, nphase = nt / R;
  __syncthreads();
  if (tid < 32) {
    float mx = 0.f;
    for (int c = lane; c < rn; c += 32) {
      float sc = 0.f;
      for (int p = 0; p < nphase; ++p) sc += part[p * R + c];
      mx = fmaxf(mx, sc);
    }
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0) s_max = mx;
  }
  __syncthreads();
  const float r = s_max;
  __syncthreads();
  return r;
}

// |X|_1 restricted to the leading rn x rn block.  Block-wide.
static __device__ float colsum_max(const float* X, int R, int rn, float* part) {
  colsum_part(X, R, rn, part);
  return part_colmax(part, R, rn);
}

// In-place Gauss-Jordan inverse in FP32 on one warp, without pivoting (SPD
// systems need none): lane j holds column j of the matrix in registers.  Step
// k: lane k publishes its column to shared memory (pc), every lane reads the
// pivot and column k from there; row k, which the update also needs, is
// column k up to sign (the in-place sweep keeps a symmetric matrix
// symmetric in its unswept part and antisymmetric across the swept rows and
// columns: a[k][j] = -a[j][k] for j < k, a[j][k] for j > k), so lane j reads
// its own entry pc[j].  R dependent steps without barriers and without
// dynamically indexed registers.  Af: R*R floats (shared, row-major, SPD);
// pc: 2R floats (shared scratch).  Writes X = Af^{-1} to out_hi (out_lo
// zeroed when given) and returns max_{j < rn} sum_{i < rn} |X_ij| on every
// lane.  Warp-wide (one warp).
template <int R>
static __device__ __noinline__ float gj_inverse_f32(const float* Af, int rn, float* out_hi,
                                                    float* out_lo, float* pc) {
  static_assert(R <= 32, "one column per lane");
  const int lane = threadIdx.x & 31;
  float c[R];
#pragma unroll
  for (int i = 0; i < R; ++i) c[i] = lane < R ? Af[i * R + lane] : 0.f;
#pragma unroll 1
  for (int k = 0; k < R; ++k) {
    float* col = pc + (k & 1) * R;   // double-buffered: no write-after-read wait
    if (lane == k) {
#pragma unroll
      for (int i = 0; i < R; ++i) col[i] = c[i];
    }
    __syncwarp();
    // reciprocal: the fast estimate and one Newton step (an IEEE division is
    // a quarter of the step's time here)
    float pinv = __fdividef(1.f, col[k]);
    pinv = pinv * (2.f - col[k] * pinv);
    const float own = lane < R ? col[lane] : 0.f;
    const float rowk = lane == k ? pinv : (lane < k ? -own : own) * pinv;   // new a[k][j]
#pragma unroll
    for (int i = 0; i < R; ++i) {
      const float f = col[i];                              // a[i][k]
      const float v = fmaf(-f, rowk, lane == k ? 0.f : c[i]);
      c[i] = i == k ? rowk : v;
    }
  }
  float cs = 0.f;
#pragma unroll
  for (int i = 0; i < R; ++i) {
    if (lane < R) {
      out_hi[i * R + lane] = c[i];
      if (out_lo) out_lo[i * R + lane] = 0.f;
    }
    if (i < rn) cs += fabsf(c[i]);
  }
  cs = lane < rn ? cs : 0.f;
  for (int o = 16; o > 0; o >>= 1) cs = fmaxf(cs, __shfl_xor_sync(0xffffffffu, cs, o));
  return cs;
}

// SPD inverse G^{-1} of G = A (R x R, FP64 input):
//  - first in FP32: for R <= 32 by Gauss-Jordan on one warp
//    (gj_inverse_f32), for R = 64 from the double-float factorisation
//    G = L D L^T (blocked) with L^{-1} and G^{-1} = L^{-T} D^{-1} L^{-1} in
//    FP32 from the rounded factors; relative error about kappa 2^-24 times a
//    small multiple of R;
//  - when the 1-norm condition estimate kappa = |G|_1 |G^{-1}|_1 (over the
//    leading rn x rn block: the padded rank columns form the decoupled block
//    rho I) exceeds `df_above`, again from the double-float factorisation with
//    L^{-1} and the product in double-float (relative error about kappa
//    2^-44), handed on as the float pair out_hi + out_lo (out_lo is zero after
//    the FP32 route).
// A: R*R doubles (shared, both triangles, destroyed); F: R*R df2 (shared
// scratch); out_hi, out_lo: R*R floats each (any memory; out_lo may be NULL,
// then out_hi gets the rounded sum).  Returns kappa (the same value on every
// thread); *route (when given) records the route: 0 FP32, 1 double-float.
// Block-wide with 256 threads, R <= 64, R a multiple of 8.
static __device__ __noinline__ double spd_inverse(double* A, df2* F, int R, int rn,
                                                  float* out_hi, float* out_lo, double df_above,
                                                  int* route = nullptr) {
  __shared__ df2 s_r[kMaxR];             // 1 / D_k
  __shared__ df2 s_col[2 * kMaxR];       // the current column of the factorisation
  // partial column sums of |G| and |G^{-1}|: entry p R + c holds rows
  // p, p + nt/R, ... of column c (no atomics: they serialise on the columns)
  __shared__ float s_gpart[kCholThreads], s_xpart[kCholThreads];
  __shared__ float s_xnorm;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
  const int col = tid % R, phase = tid / R, nphase = nt / R;
  // |G|_1 in FP32 (an estimate needs no more)
  {
    float cs = 0.f;
    if (col < rn && phase < nphase)
      for (int i = phase; i < rn; i += nphase) cs += fabsf((float)A[i * R + col]);
    s_gpart[tid] = cs;
  }
  // the factorisation into F (and its FP32 rounding into the second half of
  // the space of A, for the FP32 route at R = 64)
  float* F32 = reinterpret_cast<float*>(A) + R * R;
  auto factor = [&](float* f32) {
    if (R == 64) chol_df_blocked(A, R, F, f32, s_r);
    else if (R <= 16) chol_df<1>(A, R, F, f32, s_col, s_r);
    else chol_df<3>(A, R, F, f32, s_col, s_r);
  };
  float xnorm;
  if (R <= 32) {
    // G in FP32 in the space of F (free until the factorisation)
    float* Af = reinterpret_cast<float*>(F);
    for (int i = tid; i < R * R; i += nt) Af[i] = (float)A[i];
    __syncthreads();
    if (warp == 0) {
      float xn;
      float* pc = reinterpret_cast<float*>(s_col);   // 2R floats, unused until the factorisation
      if (R == 8) xn = gj_inverse_f32<8>(Af, rn, out_hi, out_lo, pc);
      else if (R == 16) xn = gj_inverse_f32<16>(Af, rn, out_hi, out_lo, pc);
      else xn = gj_inverse_f32<32>(Af, rn, out_hi, out_lo, pc);
      if (lane == 0) s_xnorm = xn;
    }
    __syncthreads();
    xnorm = s_xnorm;
  } else {
    factor(F32);
    // FP32 route.  Li: R*R floats in the first half of the space of A;
    // |G^{-1}| for the estimate in the space of F32 once L^{-1} is formed
    const int nb = R / 2;
    {
      __shared__ float dinv[kMaxR];
      float* Li = reinterpret_cast<float*>(A);
      float* Xa = F32;
      for (int i = tid; i < R; i += nt) dinv[i] = s_r[i].h + s_r[i].l;
      for (int round = 0; round * nw < R; ++round) {
        const int c = (round & 1) ? (round + 1) * nw - 1 - warp : round * nw + warp;
        if (c >= R) continue;
        float acc0 = 0.f, acc1 = 0.f, y0 = 0.f, y1 = 0.f;
        for (int i = c; i < R; ++i) {
          const float acc_i = __shfl_sync(0xffffffffu, i < 32 ? acc0 : acc1, i & 31);
          const float yi = (i == c ? 1.f : 0.f) - acc_i;
          if (lane == (i & 31)) { if (i < 32) y0 = yi; else y1 = yi; }
          const int j0 = lane, j1 = lane + 32;
          if (j0 > i && j0 < R) acc0 = fmaf(F32[i * R + j0], yi, acc0);
          if (j1 > i && j1 < R) acc1 = fmaf(F32[i * R + j1], yi, acc1);
        }
        __syncwarp();
        if (lane < R) Li[lane * R + c] = lane >= c ? y0 : 0.f;
        if (lane + 32 < R) Li[(lane + 32) * R + c] = lane + 32 >= c ? y1 : 0.f;
      }
      __syncthreads();
      for (int b = tid; b < nb * nb; b += nt) {
        const int bi = b / nb, bj = b % nb;
        if (bi > bj) continue;
        const int i = 2 * bi, j = 2 * bj;
        float s00 = 0.f, s01 = 0.f, s10 = 0.f, s11 = 0.f;
#pragma unroll 4
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
        const float v[4] = {s00, s01, s10, s11};
        const int rr[4] = {i, i, i + 1, i + 1}, cc[4] = {j, j + 1, j, j + 1};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          out_hi[rr[q] * R + cc[q]] = v[q];
          out_hi[cc[q] * R + rr[q]] = v[q];
          Xa[rr[q] * R + cc[q]] = fabsf(v[q]);
          Xa[cc[q] * R + rr[q]] = fabsf(v[q]);
          if (out_lo) {
            out_lo[rr[q] * R + cc[q]] = 0.f;
            out_lo[cc[q] * R + rr[q]] = 0.f;
          }
        }
      }
    }
    __syncthreads();   // every |G^{-1}| entry of the product is written
    xnorm = colsum_max(F32, R, rn, s_xpart);
  }
  const float gnorm = part_colmax(s_gpart, R, rn);
  const double kappa = (double)gnorm * (double)xnorm;
  if (!(kappa > df_above)) {
    if (route && tid == 0) *route = 0;
    return kappa;
  }
  if (route && tid == 0) *route = 1;
  if (R <= 32) factor(nullptr);   // A is still intact there
  const int nb = R / 2;
  // ---- double-float route: Li as R*R df2 in the space of A
  df2* Li = reinterpret_cast<df2*>(A);
  for (int round = 0; round * nw < R; ++round) {
    const int c = (round & 1) ? (round + 1) * nw - 1 - warp : round * nw + warp;
    if (c >= R) continue;
    df2 acc0 = {0.f, 0.f}, acc1 = {0.f, 0.f}, y0 = {0.f, 0.f}, y1 = {0.f, 0.f};
    for (int i = c; i < R; ++i) {
      // row i finalises y_i = delta_ic - acc_i
      const df2 mine = i < 32 ? acc0 : acc1;
      const df2 acc_i = {__shfl_sync(0xffffffffu, mine.h, i & 31),
                         __shfl_sync(0xffffffffu, mine.l, i & 31)};
      const df2 yi = df_sub({i == c ? 1.f : 0.f, 0.f}, acc_i);
      if (lane == (i & 31)) { if (i < 32) y0 = yi; else y1 = yi; }
      // rows below i: acc_j += L_ji y_i  (L_ji = F[i][j])
      const int j0 = lane, j1 = lane + 32;
      if (j0 > i && j0 < R) acc0 = df_add(acc0, df_mul(F[i * R + j0], yi));
      if (j1 > i && j1 < R) acc1 = df_add(acc1, df_mul(F[i * R + j1], yi));
    }
    __syncwarp();
    if (lane < R) Li[lane * R + c] = lane >= c ? y0 : df2{0.f, 0.f};
    if (lane + 32 < R) Li[(lane + 32) * R + c] = lane + 32 >= c ? y1 : df2{0.f, 0.f};
  }
  __syncthreads();
  // G^{-1}[i][j] = sum_{k >= max(i,j)} Li[k][i] D_k^{-1} Li[k][j]: 2 x 2 blocks
  // of the upper triangle, mirrored
  for (int b = tid; b < nb * nb; b += nt) {
    const int bi = b / nb, bj = b % nb;
    if (bi > bj) continue;
    const int i = 2 * bi, j = 2 * bj;
    df2 s00 = {0.f, 0.f}, s01 = {0.f, 0.f}, s10 = {0.f, 0.f}, s11 = {0.f, 0.f};
    for (int k = j; k < R; ++k) {      // j >= i
      const df2 d = s_r[k];
      const df2 li0 = Li[k * R + i], li1 = Li[k * R + i + 1];
      const df2 lj0 = df_mul(Li[k * R + j], d), lj1 = df_mul(Li[k * R + j + 1], d);
      s00 = df_add(s00, df_mul(li0, lj0));
      s01 = df_add(s01, df_mul(li0, lj1));
      s10 = df_add(s10, df_mul(li1, lj0));
      s11 = df_add(s11, df_mul(li1, lj1));
    }
    // terms with k < max(row, column) vanish (Li is lower triangular), so
    // starting at k = j covers all four entries of the block
    const df2 v[4] = {s00, s01, s10, s11};
    const int rr[4] = {i, i, i + 1, i + 1}, cc[4] = {j, j + 1, j, j + 1};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      if (out_lo) {
        out_hi[rr[q] * R + cc[q]] = v[q].h;
        out_lo[rr[q] * R + cc[q]] = v[q].l;
        out_hi[cc[q] * R + rr[q]] = v[q].h;
        out_lo[cc[q] * R + rr[q]] = v[q].l;
      } else {
        out_hi[rr[q] * R + cc[q]] = v[q].h + v[q].l;
        out_hi[cc[q] * R + rr[q]] = v[q].h + v[q].l;
      }
    }
  }
  __syncthreads();
  return kappa;
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
