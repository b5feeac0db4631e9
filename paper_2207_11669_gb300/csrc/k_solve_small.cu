// Whole solve of a small problem in one CTA (exact consensus U-step).
//
// A problem whose M and factors fit in one SM's shared memory (the 200 x 200,
// E = 4 workload of §4.1 holds 160 KB of M) is latency-bound on the
// multi-kernel path: each iteration is seven or eight launches of a few
// microseconds of work.  Here one CTA keeps M, U, V and W in shared memory and
// runs every iteration of a dcf_step / dcf_solve call in one launch.
//
// One iteration, from (U, V) to (U', V'), the same arithmetic as the other
// paths (§2.2 S-step, App. B V-step, the consensus U-step, the factor-space
// metrics of the stop test):
//   G = U^T U (compensated FP32 sums, FP64 result), W = U (G + rho I)^{-1}
//   column j:  r_ij = M_ij - u_i.v_j,  x_ij = u_i.v_j + clamp(r_ij, -lambda, lambda)
//              (= M_ij - S_ij),  v'_j = sum_i x_ij w_i,  Huber sum of r_ij
//   Q' = V'^T V', X_v = V^T V',  H = (Q' + rho I)^{-1}
//   row i:     p_i = sum_j x_ij v'_j  (x recomputed),  u'_i = p_i H
//   G' = U'^T U', and with dU = U' - U, dV = V' - V the change Grams
//   A = U^T dU, D_u = dU^T dU, Y = V^T dV, D_v = dV^T dV:
//   dL^2 = <D_u, Q'> + 2 <A^T, Y + D_v> + <G, D_v>   (L' - L = dU V'^T + U dV^T;
//   every term of the size of the change), |L'|^2 = <G', Q'>,
//   objective = Huber + rho/2 (tr G + tr Q)
// The r x r inverses are FP64 (Gauss-Jordan in one warp), the long sums FP32.
#include <cuda_runtime.h>
#include <stdint.h>

#include "dcf.h"
#include "dcf_internal.cuh"
#include "dcf_small.cuh"

namespace dcf {

namespace {

constexpr int kSSThreads = 512;

// Shared-memory layout (bytes) for R and the problem size.
struct SSLayout {
  int RR;
  int64_t ldm;        // M is stored with leading dimension m + 1 (odd: no bank
                      // conflicts when threads walk different columns)
  size_t A, G, Q, Gn, Qn, XU, XV, DU, DV, WS;   // doubles
  size_t GI, HI, GP;                    // floats (GP: float2 Gram partials)
  size_t Ms, U0, U1, V0, V1, W;         // floats
  size_t total;
  __host__ __device__ SSLayout(int R, int64_t m, int64_t n) {
    RR = R * R;
    ldm = m + 1;
    size_t o = 0;
    A = o;  o += (size_t)RR * 2 * 8;    // [S + rho I | I] for the Gauss-Jordan inverse
    G = o;  o += (size_t)RR * 8;
    Q = o;  o += (size_t)RR * 8;
    Gn = o; o += (size_t)RR * 8;
    Qn = o; o += (size_t)RR * 8;
    XU = o; o += (size_t)RR * 8;
    XV = o; o += (size_t)RR * 8;
    DU = o; o += (size_t)RR * 8;
    DV = o; o += (size_t)RR * 8;
    WS = o; o += 8 * 32 * 8;
    GI = o; o += (size_t)RR * 4;
    HI = o; o += (size_t)RR * 4;
    GP = o; o += (size_t)kSSThreads * 8;
    Ms = o; o += ((size_t)ldm * n * 4 + 15) / 16 * 16;   // U, V, W rows are read as float4
    U0 = o; o += (size_t)m * R * 4;
    U1 = o; o += (size_t)m * R * 4;
    V0 = o; o += (size_t)n * R * 4;
    V1 = o; o += (size_t)n * R * 4;
    W = o;  o += (size_t)m * R * 4;
    total = o;
  }
};

__device__ __forceinline__ void ss_two_sum(float& hi, float& lo, float x) {
  const float t = hi + x;
  const float bp = t - hi;
  lo += (hi - (t - bp)) + (x - bp);
  hi = t;
}

// out[k*R + l] = sum_i x_k y_l over N rows, with (x, y) = (X_i, Y_i) in mode
// 0, (X_i, Y_i - X_i) in mode 1 and (Y_i - X_i, Y_i - X_i) in mode 2 (compensated FP32
// partials over row groups, FP64 result).  Block-wide.
template <int R, int kMode = 0>
__device__ void ss_gram(const float* X, const float* Y, int64_t N, double* out, float2* gp) {
  constexpr int RR = R * R;
  constexpr int NG = kSSThreads / RR >= 1 ? kSSThreads / RR : 1;   // row groups
  const int tid = threadIdx.x;
  for (int e0 = 0; e0 < RR; e0 += kSSThreads / NG) {
    const int e = e0 + tid % (kSSThreads / NG), g = tid / (kSSThreads / NG);
    float hi = 0.f, lo = 0.f;
    if (e < RR && g < NG) {
      const int k = e / R, l = e % R;
      for (int64_t i = g; i < N; i += NG) {
        const float xk = X[i * R + k], xl = X[i * R + l], yk = Y[i * R + k], yl = Y[i * R + l];
        const float a = kMode == 2 ? yk - xk : xk;
        const float b = kMode == 0 ? yl : yl - xl;
        ss_two_sum(hi, lo, a * b);
      }
    }
    __syncthreads();
    gp[tid] = make_float2(hi, lo);
    __syncthreads();
    if (tid < kSSThreads / NG && e0 + tid < RR) {
      float h = 0.f, l2 = 0.f;
      for (int q = 0; q < NG; ++q) {
        const float2 v = gp[q * (kSSThreads / NG) + tid];
        ss_two_sum(h, l2, v.x);
        l2 += v.y;
      }
      out[e0 + tid] = (double)h + (double)l2;
    }
  }
  __syncthreads();
}

// out (floats, R x R) = (S + rho I)^{-1} for a symmetric positive definite
// S + rho I, by FP64 Gauss-Jordan elimination on [S + rho I | I] in warp 0
// (no pivoting: the matrix is SPD; R <= 16, at most 16 entries per lane and
// step, one __syncwarp between the read and the write of a step).  Called by
// every thread; returns 0 when a pivot is not positive or a value not finite.
template <int R>
__device__ int ss_ridge_inverse(const double* S, float rho, double* A, float* out, int* okp) {
  constexpr int C = 2 * R, NE = R * C, PER = (NE + 31) / 32;
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    for (int e = lane; e < NE; e += 32) {
      const int i = e / C, j = e % C;
      A[e] = j < R ? S[i * R + j] + (i == j ? (double)rho : 0.0) : (j - R == i ? 1.0 : 0.0);
    }
    __syncwarp();
    int ok = 1;
    for (int k = 0; k < R; ++k) {
      const double piv = A[k * C + k];
      if (!(piv > 0.0) || !isfinite(piv)) ok = 0;
      const double ip = recip_f64(piv);
      double nv[PER];
#pragma unroll
      for (int q = 0; q < PER; ++q) {
        const int e = lane + 32 * q;
        if (e < NE) {
          const int i = e / C, j = e % C;
          const double akj = A[k * C + j] * ip;
          nv[q] = i == k ? akj : fma(-A[i * C + k], akj, A[e]);
        }
      }
      __syncwarp();
#pragma unroll
      for (int q = 0; q < PER; ++q) {
        const int e = lane + 32 * q;
        if (e < NE) A[e] = nv[q];
      }
      __syncwarp();
    }
    for (int e = lane; e < R * R; e += 32) {
      const double v = A[(e / R) * C + R + e % R];
      if (!isfinite(v)) ok = 0;
      out[e] = (float)v;
    }
    ok = __all_sync(0xffffffffu, ok);
    if (lane == 0) *okp = ok;
  }
  __syncthreads();
  return *okp;
}

}  // namespace

template <int R>
__global__ void __launch_bounds__(kSSThreads, 1) k_solve_small(SmallSolveArgs a) {
  extern __shared__ __align__(16) uint8_t smem[];
  const SSLayout L(R, a.m, a.n);
  double* A = reinterpret_cast<double*>(smem + L.A);
  double* G = reinterpret_cast<double*>(smem + L.G);
  double* Q = reinterpret_cast<double*>(smem + L.Q);
  double* Gn = reinterpret_cast<double*>(smem + L.Gn);
  double* Qn = reinterpret_cast<double*>(smem + L.Qn);
  double* XU = reinterpret_cast<double*>(smem + L.XU);
  double* XV = reinterpret_cast<double*>(smem + L.XV);
  double* DU = reinterpret_cast<double*>(smem + L.DU);
  double* DV = reinterpret_cast<double*>(smem + L.DV);
  double* ws = reinterpret_cast<double*>(smem + L.WS);
  float* GI = reinterpret_cast<float*>(smem + L.GI);
  float* HI = reinterpret_cast<float*>(smem + L.HI);
  float2* gp = reinterpret_cast<float2*>(smem + L.GP);
  float* Ms = reinterpret_cast<float*>(smem + L.Ms);
  // the two copies of U (and of V) are adjacent: copy c at base + c * rows * R
  float* Ub = reinterpret_cast<float*>(smem + L.U0);
  float* Vb = reinterpret_cast<float*>(smem + L.V0);
  float* Ws = reinterpret_cast<float*>(smem + L.W);
  __shared__ int s_flags[3];   // [0] stop the loop, [1] status, [2] inverse ok
  __shared__ double s_met[4];  // dL_rel, objective, Huber of the last iteration
  const int tid = threadIdx.x;
  const int64_t m = a.m, n = a.n, ldm = L.ldm;
  DevState* st = a.st;
  if (st->status != 0 || a.n_iter < 1) return;
  const int solve_mode = st->solve_mode;
  const double tol = st->tol;
  const float lam = a.lam, rho = a.rho;
  // adjacent threads per column (V-step) and per row (U-step): the largest power
  // of two up to 8 that keeps every column (row) within one pass of the CTA
  auto tpc_of = [](int64_t cnt) {
    int t = 1;
    while (t < 8 && (int64_t)(2 * t) * cnt <= kSSThreads) t *= 2;
    return t;
  };
  const int TPC = tpc_of(n), TPR = tpc_of(m);

  // ---- load M, U, V (copy cur) and the previous copies -------------------------
  for (int64_t e = tid; e < m * n; e += kSSThreads) {
    const int64_t j = e / m, i = e % m;
    Ms[j * ldm + i] = a.M[e];
  }
  int cur = a.cur;
  {
    const float* Ug = cur ? a.U[1] : a.U[0];
    const float* Vg = cur ? a.V[1] : a.V[0];
    for (int64_t e = tid; e < m * R; e += kSSThreads) Ub[cur * m * R + e] = Ug[e];
    for (int64_t e = tid; e < n * R; e += kSSThreads) Vb[cur * n * R + e] = Vg[e];
  }
  if (tid == 0) { s_flags[0] = 0; s_flags[1] = 0; }
  __syncthreads();
  ss_gram<R>(Ub + cur * m * R, Ub + cur * m * R, m, G, gp);
  ss_gram<R>(Vb + cur * n * R, Vb + cur * n * R, n, Q, gp);

  int done = 0;
  double last_dl = 0.0, last_obj = 0.0, last_hub = 0.0;
  for (int it = 0; it < a.n_iter; ++it) {
    const int nxt = cur ^ 1;
    const float* U = Ub + cur * m * R;
    const float* V = Vb + cur * n * R;
    float* Un = Ub + nxt * m * R;
    float* Vn = Vb + nxt * n * R;
    // ---- W = U (G + rho I)^{-1} -------------------------------------------------
    if (!ss_ridge_inverse<R>(G, rho, A, GI, &s_flags[2])) {
      if (tid == 0) s_flags[1] = DCF_ENONFINITE;
      __syncthreads();
      break;
    }
    for (int64_t e = tid; e < m * R; e += kSSThreads) {
      const int64_t i = e / R;
      const int l = (int)(e % R);
      float s = 0.f;
#pragma unroll
      for (int k = 0; k < R; ++k) s = fmaf(U[i * R + k], GI[k * R + l], s);
      Ws[e] = s;
    }
    __syncthreads();
    // ---- S-step and V-step: TPC adjacent threads per column, shuffle-combined ----
    {
      double hub_w = 0.0;
      for (int64_t jb = 0; jb < n; jb += kSSThreads / TPC) {
        const int64_t j = jb + tid / TPC;
        const int part = tid % TPC;
        const bool act = j < n;
        float v[R], acc[R];
#pragma unroll
        for (int k = 0; k < R; ++k) { v[k] = act ? V[j * R + k] : 0.f; acc[k] = 0.f; }
        float hub = 0.f;
        const float* Mc = Ms + (act ? j : 0) * ldm;
#pragma unroll 2
        for (int64_t i = part; act && i < m; i += TPC) {
          // rows of U and W as float4 (broadcast: the threads of a step read row i)
          const float4* u4 = reinterpret_cast<const float4*>(U + i * R);
          const float4* w4 = reinterpret_cast<const float4*>(Ws + i * R);
          float uv = 0.f;
#pragma unroll
          for (int k4 = 0; k4 < R / 4; ++k4) {
            const float4 u = u4[k4];
            uv = fmaf(u.x, v[4 * k4], uv);
            uv = fmaf(u.y, v[4 * k4 + 1], uv);
            uv = fmaf(u.z, v[4 * k4 + 2], uv);
            uv = fmaf(u.w, v[4 * k4 + 3], uv);
          }
          const float r = Mc[i] - uv;
          const float c = fminf(fmaxf(r, -lam), lam);
          hub = fmaf(c, r - 0.5f * c, hub);             // Huber H_lambda(r)
          const float x = uv + c;                       // M - S
#pragma unroll
          for (int k4 = 0; k4 < R / 4; ++k4) {
            const float4 w = w4[k4];
            acc[4 * k4] = fmaf(x, w.x, acc[4 * k4]);
            acc[4 * k4 + 1] = fmaf(x, w.y, acc[4 * k4 + 1]);
            acc[4 * k4 + 2] = fmaf(x, w.z, acc[4 * k4 + 2]);
            acc[4 * k4 + 3] = fmaf(x, w.w, acc[4 * k4 + 3]);
          }
        }
#pragma unroll
        for (int o = TPC / 2; o > 0; o >>= 1)
#pragma unroll
          for (int k = 0; k < R; ++k) acc[k] += __shfl_xor_sync(0xffffffffu, acc[k], o);
        if (act && part == 0)
#pragma unroll
          for (int k = 0; k < R; ++k) Vn[j * R + k] = acc[k];
        hub_w += (double)hub;
      }
      // per-warp Huber partial (summed by warp 0 with the metrics)
      for (int o = 16; o > 0; o >>= 1) hub_w += __shfl_xor_sync(0xffffffffu, hub_w, o);
      if ((tid & 31) == 0) ws[tid >> 5] = hub_w;
    }
    __syncthreads();
    ss_gram<R>(Vn, Vn, n, Qn, gp);
    ss_gram<R, 1>(V, Vn, n, XV, gp);      // V^T dV
    ss_gram<R, 2>(V, Vn, n, DV, gp);      // dV^T dV
    // ---- U-step: P = X V', U' = P (Q' + rho I)^{-1}, one thread per row ---------
    if (!ss_ridge_inverse<R>(Qn, rho, A, HI, &s_flags[2])) {
      if (tid == 0) s_flags[1] = DCF_ENONFINITE;
      __syncthreads();
      break;
    }
    for (int64_t ib = 0; ib < m; ib += kSSThreads / TPR) {
      const int64_t i = ib + tid / TPR;
      const int part = tid % TPR;
      const bool act = i < m;
      float u[R], p[R];
#pragma unroll
      for (int k = 0; k < R; ++k) { u[k] = act ? U[i * R + k] : 0.f; p[k] = 0.f; }
#pragma unroll 2
      for (int64_t j = part; act && j < n; j += TPR) {
        const float4* v4 = reinterpret_cast<const float4*>(V + j * R);
        const float4* vn4 = reinterpret_cast<const float4*>(Vn + j * R);
        float uv = 0.f;
#pragma unroll
        for (int k4 = 0; k4 < R / 4; ++k4) {
          const float4 v = v4[k4];
          uv = fmaf(u[4 * k4], v.x, uv);
          uv = fmaf(u[4 * k4 + 1], v.y, uv);
          uv = fmaf(u[4 * k4 + 2], v.z, uv);
          uv = fmaf(u[4 * k4 + 3], v.w, uv);
        }
        const float r = Ms[j * ldm + i] - uv;
        const float x = uv + fminf(fmaxf(r, -lam), lam);
#pragma unroll
        for (int k4 = 0; k4 < R / 4; ++k4) {
          const float4 w = vn4[k4];
          p[4 * k4] = fmaf(x, w.x, p[4 * k4]);
          p[4 * k4 + 1] = fmaf(x, w.y, p[4 * k4 + 1]);
          p[4 * k4 + 2] = fmaf(x, w.z, p[4 * k4 + 2]);
          p[4 * k4 + 3] = fmaf(x, w.w, p[4 * k4 + 3]);
        }
      }
#pragma unroll
      for (int o = TPR / 2; o > 0; o >>= 1)
#pragma unroll
        for (int k = 0; k < R; ++k) p[k] += __shfl_xor_sync(0xffffffffu, p[k], o);
      if (act && part == 0) {
#pragma unroll
        for (int l = 0; l < R; ++l) {
          float s2 = 0.f;
#pragma unroll
          for (int k = 0; k < R; ++k) s2 = fmaf(p[k], HI[k * R + l], s2);
          Un[i * R + l] = s2;
        }
      }
    }
    __syncthreads();
    ss_gram<R>(Un, Un, m, Gn, gp);
    ss_gram<R, 1>(U, Un, m, XU, gp);      // U^T dU
    ss_gram<R, 2>(U, Un, m, DU, gp);      // dU^T dU
    // ---- metrics and the stop test (warp 0) -----------------------------------------
    if (tid < 32) {
      double v[7] = {0, 0, 0, 0, 0, 0, 0};
      for (int e = tid; e < R * R; e += 32) {
        const int k = e / R, l = e % R;
        v[0] = fma(Gn[e], Qn[e], v[0]);
        v[1] = fma(DU[e], Qn[e], v[1]);
        v[2] = fma(XU[l * R + k], XV[e] + DV[e], v[2]);
        v[6] = fma(G[e], DV[e], v[6]);
        if (k == l) { v[3] += G[e]; v[4] += Q[e]; }
      }
      if (tid < kSSThreads / 32) v[5] = ws[tid];      // per-warp Huber partials
#pragma unroll
      for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int q = 0; q < 7; ++q) v[q] += __shfl_xor_sync(0xffffffffu, v[q], o);
      if (tid == 0) {
        double d2 = v[1] + 2.0 * v[2] + v[6];
        if (d2 < 0) d2 = 0;
        const double dl = v[0] > 0 ? sqrt(d2 / v[0]) : INFINITY;
        const double obj = v[5] + 0.5 * (double)rho * (v[3] + v[4]);
        s_met[0] = dl;
        s_met[1] = obj;
        s_met[2] = v[5];
        if (!isfinite(v[0]) || !isfinite(obj)) s_flags[1] = DCF_ENONFINITE;
        if (solve_mode && dl <= tol) s_flags[0] = 1;
      }
    }
    __syncthreads();
    last_dl = s_met[0];
    last_obj = s_met[1];
    last_hub = s_met[2];
    ++done;
    for (int e = tid; e < R * R; e += kSSThreads) { G[e] = Gn[e]; Q[e] = Qn[e]; }
    cur = nxt;
    __syncthreads();
    if (s_flags[0] || s_flags[1]) break;
  }

  // ---- write back: current and previous copies, state ---------------------------
  for (int64_t e = tid; e < m * R; e += kSSThreads) {
    a.U[0][e] = Ub[e];
    a.U[1][e] = Ub[m * R + e];
  }
  for (int64_t e = tid; e < n * R; e += kSSThreads) {
    a.V[0][e] = Vb[e];
    a.V[1][e] = Vb[n * R + e];
  }
  if (tid == 0) {
    st->iter += done;
    if (done > 0) {
      st->has_S = 1;
      st->dL_rel = last_dl;
      st->objective = last_obj;
      st->huber = last_hub;
    }
    if (s_flags[1]) st->status = s_flags[1];
    if (s_flags[0]) st->stop = 1;
  }
}

size_t solve_small_smem(int R, int64_t m, int64_t n) {
  return SSLayout(R, m, n).total;
}

cudaError_t solve_small_prepare(int R, size_t smem) {
  if (R == 8)
    return cudaFuncSetAttribute(k_solve_small<8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem);
  return cudaFuncSetAttribute(k_solve_small<16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)smem);
}

cudaError_t launch_solve_small(int R, const SmallSolveArgs& a, cudaStream_t s) {
  const size_t smem = solve_small_smem(R, a.m, a.n);
  if (R == 8) k_solve_small<8><<<1, kSSThreads, smem, s>>>(a);
  else k_solve_small<16><<<1, kSSThreads, smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace dcf
