// Small-matrix and per-row kernels of the DCF-PCA iteration.
//
//   k_gram_part      per-CTA partial Gram X^T Y over a row range (FP32 products,
//                    chunked FP32 sums folded into a compensated (TwoSum) pair)
//   k_reduce_parts   deterministic FP64 sum of those partials over many CTAs;
//                    the last CTA to finish runs the serial r x r tail:
//                      TAIL_Q : Q_t = V_t^T V_t, Cholesky of Q_t + rho I (U-step)
//                      TAIL_G : U_t^T U_t, metrics, stop test, Cholesky of
//                               U_t^T U_t + rho I (next V-step), t <- t + 1
//                      TAIL_INIT_G / TAIL_INIT_Q : the same for the start point
//   k_make_w         W = U (U^T U + rho I)^{-1} row by row (two triangular
//                    solves with the FP64 Cholesky factor rounded to float)
//   k_rows           consensus U-update row by row + Gram partials of U_t
//
// Why FP64 is confined to r x r work: GB300 executes FP64 at roughly two
// fused multiply-adds per clock per SM, so every O(m r) or O(n r) sum runs in
// FP32 with compensation and only the r x r Cholesky factorisations and the
// final cross-CTA sums (spread over many CTAs) use FP64.
#include "dcf_internal.cuh"
#include "dcf_small.cuh"

namespace dcf {

__host__ __device__ __forceinline__ int64_t dmin64(int64_t a, int64_t b) { return a < b ? a : b; }

// ---------------------------------------------------------------------------
// compensated accumulation (Knuth's TwoSum; exact error term of s + x)
// ---------------------------------------------------------------------------
__device__ __forceinline__ void two_sum_add(float& hi, float& lo, float x) {
  float t = hi + x;
  float bp = t - hi;
  float err = (hi - (t - bp)) + (x - bp);
  hi = t;
  lo += err;
}

// ---------------------------------------------------------------------------
// Gram partials:  part[b][k*cy + l] = sum_{rows a of CTA b} X[a,k] * Y[a,l]
// ---------------------------------------------------------------------------
constexpr int kGramChunk = 32;
constexpr int kGramMaxEntriesPerThread = 16;   // (64*64)/256

__global__ void __launch_bounds__(256)
k_gram_part(const float* __restrict__ X, int ldx, int cx,
            const float* __restrict__ Y, int ldy, int cy,
            int64_t N, int64_t rows_per_cta, double* __restrict__ part,
            const DevState* st, int respect_stop) {
  if (respect_stop && st->stop) return;
  extern __shared__ float sh[];
  float* Xs = sh;                           // [chunk][cx]
  float* Ys = sh + kGramChunk * cx;         // [chunk][cy]
  const int tid = threadIdx.x;
  const int ne = cx * cy;
  float hi[kGramMaxEntriesPerThread], lo[kGramMaxEntriesPerThread];
#pragma unroll
  for (int i = 0; i < kGramMaxEntriesPerThread; ++i) { hi[i] = 0.f; lo[i] = 0.f; }
  const int64_t a0 = (int64_t)blockIdx.x * rows_per_cta;
  const int64_t a1 = min(N, a0 + rows_per_cta);
  for (int64_t c = a0; c < a1; c += kGramChunk) {
    const int rows = (int)dmin64((int64_t)(kGramChunk), a1 - c);
    __syncthreads();
    for (int i = tid; i < kGramChunk * cx; i += blockDim.x) {
      int rr = i / cx, k = i % cx;
      Xs[i] = rr < rows ? X[(c + rr) * ldx + k] : 0.f;
    }
    for (int i = tid; i < kGramChunk * cy; i += blockDim.x) {
      int rr = i / cy, k = i % cy;
      Ys[i] = rr < rows ? Y[(c + rr) * ldy + k] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int s = 0; s < kGramMaxEntriesPerThread; ++s) {
      int e = tid + s * 256;
      if (e < ne) {
        int k = e / cy, l = e % cy;
        float acc = 0.f;
        for (int rr = 0; rr < rows; ++rr) acc = fmaf(Xs[rr * cx + k], Ys[rr * cy + l], acc);
        two_sum_add(hi[s], lo[s], acc);
      }
    }
  }
#pragma unroll
  for (int s = 0; s < kGramMaxEntriesPerThread; ++s) {
    int e = tid + s * 256;
    if (e < ne) part[(int64_t)blockIdx.x * ne + e] = (double)hi[s] + (double)lo[s];
  }
}

// ---------------------------------------------------------------------------
// Reduction of partials + serial tail
// ---------------------------------------------------------------------------
enum TailKind { TAIL_NONE = 0, TAIL_Q = 1, TAIL_G = 2, TAIL_INIT_G = 3, TAIL_INIT_Q = 4 };

struct ReduceArgs {
  const double* part[3];   // partial arrays ([nparts][count_s])
  int count[3];            // entries per matrix (0 = unused)
  double* out[3];          // destinations (FP64)
  int nparts[3];
  int total;               // count[0] + count[1] + count[2]
  int tail;
  int R;
  float rho;
  int u_mode;
  int copy;                // TAIL_INIT_*: copy written; TAIL_Q/G: copy holding U_{t-1}
  unsigned int* counter;   // last-block counter (starts at 0, reset by the tail)
  Smalls* sm;
  DevState* st;
};

constexpr int kRedEntriesPerCta = 16;

__device__ void tail_q(const ReduceArgs& a, double* A, float* F);
__device__ void tail_g(const ReduceArgs& a, double* A, float* F);

__global__ void __launch_bounds__(256) k_reduce_parts(ReduceArgs a) {
  if ((a.tail == TAIL_Q || a.tail == TAIL_G) && a.st->stop) return;
  __shared__ double red[256];
  __shared__ bool is_last;
  const int tid = threadIdx.x;
  const int e_local = tid % kRedEntriesPerCta;
  const int lane_p = tid / kRedEntriesPerCta;          // 0..15
  const int nsplit = 256 / kRedEntriesPerCta;
  const int e = blockIdx.x * kRedEntriesPerCta + e_local;
  double s = 0.0;
  int which = -1, idx = 0;
  if (e < a.total) {
    idx = e;
    which = 0;
    while (idx >= a.count[which]) { idx -= a.count[which]; ++which; }
    const double* p = a.part[which];
    const int cnt = a.count[which];
    for (int q = lane_p; q < a.nparts[which]; q += nsplit) s += p[(int64_t)q * cnt + idx];
  }
  red[tid] = s;
  __syncthreads();
  if (lane_p == 0 && which >= 0) {
    double t = 0.0;
    for (int q = 0; q < nsplit; ++q) t += red[q * kRedEntriesPerCta + e_local];
    a.out[which][idx] = t;
  }
  if (a.tail == TAIL_NONE) return;
  // last-block-done: the CTA that finishes last runs the serial tail
  __threadfence();
  __syncthreads();
  if (tid == 0) {
    unsigned int prev = atomicAdd(a.counter, 1u);
    is_last = (prev == gridDim.x - 1);
  }
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  extern __shared__ double dsh[];   // R*R doubles, then R*R floats
  float* F = reinterpret_cast<float*>(dsh + a.R * a.R);
  if (tid == 0) *a.counter = 0u;
  if (a.tail == TAIL_Q || a.tail == TAIL_INIT_Q) tail_q(a, dsh, F);
  else tail_g(a, dsh, F);
}

// Q_t is in out[0] (R*R), X_v = V_{t-1}^T V_t in out[1], Huber in out[2].
__device__ void tail_q(const ReduceArgs& a, double* A, float* F) {
  const int R = a.R;
  Smalls* sm = a.sm;
  DevState* st = a.st;
  if (a.tail == TAIL_INIT_Q) {
    // start point: only V0^T V0 is needed (for the first metrics)
    for (int i = threadIdx.x; i < R * R; i += blockDim.x) sm->q[a.copy][i] = __ldcg(a.out[0] + i);
    return;
  }
  const int nxt = a.copy ^ 1;
  for (int i = threadIdx.x; i < R * R; i += blockDim.x) {
    double q = __ldcg(a.out[0] + i);
    sm->q[nxt][i] = q;
    sm->xv[i] = __ldcg(a.out[1] + i);
    int r = i / R, c = i % R;
    double h = q + (r == c ? (double)a.rho : 0.0);
    A[i] = h;
    sm->qrho32[i] = (float)h;
  }
  if (threadIdx.x == 0) st->huber = __ldcg(a.out[2]);
  __syncthreads();
  if (!all_finite(A, R * R)) {
    if (threadIdx.x == 0) st->status = 4;  // DCF_ENONFINITE
    return;
  }
  if (a.u_mode == 0) spd_inverse_f32(A, F, R, sm->hinv32);
}

// Gram of U_t in out[0], X_u = U_{t-1}^T U_t in out[1].
__device__ void tail_g(const ReduceArgs& a, double* A, float* F) {
  const int R = a.R;
  Smalls* sm = a.sm;
  DevState* st = a.st;
  int tgt;
  if (a.tail == TAIL_INIT_G) {
    tgt = a.copy;
    for (int i = threadIdx.x; i < R * R; i += blockDim.x) sm->gram[tgt][i] = __ldcg(a.out[0] + i);
  } else {
    const int cur = a.copy;
    tgt = cur ^ 1;
    for (int i = threadIdx.x; i < R * R; i += blockDim.x) {
      sm->gram[tgt][i] = __ldcg(a.out[0] + i);
      sm->xu[i] = __ldcg(a.out[1] + i);
    }
    __syncthreads();
    // metrics: dL^2 = <G_t,Q_t> - 2 <X_u, X_v> + <G_{t-1}, Q_{t-1}>   (all r x r)
    __shared__ double red5[5][256];
    double s0 = 0, s1 = 0, s2 = 0, s3 = 0, s4 = 0;
    for (int i = threadIdx.x; i < R * R; i += blockDim.x) {
      s0 += sm->gram[tgt][i] * sm->q[tgt][i];
      s1 += sm->xu[i] * sm->xv[i];
      s2 += sm->gram[cur][i] * sm->q[cur][i];
      int r = i / R, c = i % R;
      if (r == c) { s3 += sm->gram[cur][i]; s4 += sm->q[cur][i]; }
    }
    red5[0][threadIdx.x] = s0;
    red5[1][threadIdx.x] = s1;
    red5[2][threadIdx.x] = s2;
    red5[3][threadIdx.x] = s3;
    red5[4][threadIdx.x] = s4;
    __syncthreads();
    if (threadIdx.x == 0) {
      double a0 = 0, a1 = 0, a2 = 0, t0 = 0, t1 = 0;
      for (int i = 0; i < blockDim.x; ++i) {
        a0 += red5[0][i]; a1 += red5[1][i]; a2 += red5[2][i];
        t0 += red5[3][i]; t1 += red5[4][i];
      }
      double d2 = a0 - 2.0 * a1 + a2;
      if (d2 < 0) d2 = 0;
      st->dL_rel = a0 > 0 ? sqrt(d2 / a0) : INFINITY;
      st->objective = st->huber + 0.5 * (double)a.rho * (t0 + t1);
      st->iter = st->iter + 1;
      st->has_S = 1;
      if (!isfinite(a0) || !isfinite(st->objective)) st->status = 4;
      if (st->solve_mode && st->dL_rel <= st->tol) st->stop = 1;
    }
    __syncthreads();
  }
  // (U^T U + rho I)^{-1} for the next V-step
  for (int i = threadIdx.x; i < R * R; i += blockDim.x) {
    int r = i / R, c = i % R;
    A[i] = sm->gram[tgt][i] + (r == c ? (double)a.rho : 0.0);
  }
  __syncthreads();
  if (!all_finite(A, R * R)) {
    if (threadIdx.x == 0) st->status = 4;
    return;
  }
  spd_inverse_f32(A, F, R, sm->ginv32);
}

// ---------------------------------------------------------------------------
// Row kernels: a CTA of 256 threads owns 32 rows; thread (row t/8, column
// group t%8) forms R/8 outputs of (row) x (R x R matrix).
// ---------------------------------------------------------------------------
constexpr int kRowsPerCta = 32;

// W = U (U^T U + rho I)^{-1}
template <int R>
__global__ void __launch_bounds__(256) k_make_w(const float* __restrict__ U,
                                                const DevState* st, const Smalls* sm,
                                                float* __restrict__ W, int64_t m,
                                                int respect_stop) {
  if (respect_stop && st->stop) return;
  constexpr int CG = R / 8;
  __shared__ __align__(16) float Gi[R * R];
  __shared__ __align__(16) float Us[kRowsPerCta * R];
  const int tid = threadIdx.x;
  const int64_t row0 = (int64_t)blockIdx.x * kRowsPerCta;
  for (int i = tid; i < R * R; i += 256) Gi[i] = sm->ginv32[i];
  for (int i = tid; i < kRowsPerCta * R; i += 256) {
    int64_t a = row0 + i / R;
    Us[i] = a < m ? U[row0 * R + i] : 0.f;
  }
  __syncthreads();
  const int ar = tid >> 3, g = tid & 7;
  const int64_t a = row0 + ar;
  if (a >= m) return;
  float acc[CG];
#pragma unroll
  for (int l = 0; l < CG; ++l) acc[l] = 0.f;
  for (int k = 0; k < R; ++k) {
    float u = Us[ar * R + k];
#pragma unroll
    for (int l = 0; l < CG; ++l) acc[l] = fmaf(u, Gi[k * R + g * CG + l], acc[l]);
  }
#pragma unroll
  for (int l = 0; l < CG; ++l) W[a * R + g * CG + l] = acc[l];
}

// Consensus U-update plus Gram partials of the new U:
//   exact:  U_t[a,:] = P[a,:] (Q_t + rho I)^{-1},  P[a,:] = sum_s part_p[s][a,:]
//   FedAvg: U_t[a,:] = U[a,:] - (eta_t/E) (U[a,:] (Q_t + rho I) - P[a,:])
template <int R>
__global__ void __launch_bounds__(256) k_rows(IterArgs a) {
  DevState* st = a.st;
  if (st->stop) return;
  constexpr int CG = R / 8;
  __shared__ __align__(16) float Mat[R * R];
  __shared__ __align__(16) float Ps[kRowsPerCta * R];
  __shared__ __align__(16) float Uo[kRowsPerCta * R];
  __shared__ __align__(16) float Un[kRowsPerCta * R];
  const int tid = threadIdx.x;
  const int cur = a.cur, nxt = cur ^ 1;
  const float* U = a.U[cur];
  float* Unew = a.U[nxt];
  const int64_t row0 = (int64_t)blockIdx.x * kRowsPerCta;
  const int rows = (int)dmin64((int64_t)kRowsPerCta, a.m - row0);
  if (a.add_uxv)
    for (int i = tid; i < R * R; i += 256) Mat[i] = (float)a.sm->xv[i];
  for (int i = tid; i < kRowsPerCta * R; i += 256) {
    const int rr = i / R;
    float hi = 0.f, lo = 0.f, uo = 0.f;
    if (rr < rows) {
      const int64_t off = row0 * R + i;
      for (int s = 0; s < a.n_splits; ++s) two_sum_add(hi, lo, a.part_p[(int64_t)s * a.m * R + off]);
      uo = U[off];
    }
    Ps[i] = hi + lo;
    Uo[i] = uo;
  }
  __syncthreads();
  const int ar = tid >> 3, g = tid & 7;
  if (a.add_uxv) {
    // P = U_{t-1} (V_{t-1}^T V_t) + C V'   (the fused pass returns only C V')
    float add[CG];
#pragma unroll
    for (int l = 0; l < CG; ++l) add[l] = 0.f;
    for (int k = 0; k < R; ++k) {
      const float u = Uo[ar * R + k];
#pragma unroll
      for (int l = 0; l < CG; ++l) add[l] = fmaf(u, Mat[k * R + g * CG + l], add[l]);
    }
    __syncthreads();
#pragma unroll
    for (int l = 0; l < CG; ++l) Ps[ar * R + g * CG + l] += add[l];
  }
  for (int i = tid; i < R * R; i += 256) Mat[i] = a.u_mode == 0 ? a.sm->hinv32[i] : a.sm->qrho32[i];
  __syncthreads();
  float acc[CG];
#pragma unroll
  for (int l = 0; l < CG; ++l) acc[l] = 0.f;
  const float* src = a.u_mode == 0 ? Ps : Uo;
  for (int k = 0; k < R; ++k) {
    float v = src[ar * R + k];
#pragma unroll
    for (int l = 0; l < CG; ++l) acc[l] = fmaf(v, Mat[k * R + g * CG + l], acc[l]);
  }
  if (a.u_mode != 0) {
    const double eta = st->eta0 / sqrt((double)st->iter + 1.0);
    const float step = (float)(eta / (double)a.E);
#pragma unroll
    for (int l = 0; l < CG; ++l) {
      const int c = g * CG + l;
      acc[l] = Uo[ar * R + c] - step * (acc[l] - Ps[ar * R + c]);
    }
  }
  if (a.u_mode == 0 && a.alpha != 1.0f) {
    // relaxed consensus step of the learned network: U_t = U + alpha (U* - U)
#pragma unroll
    for (int l = 0; l < CG; ++l) {
      const int c = g * CG + l;
      if (a.ustar_out && ar < rows) a.ustar_out[(row0 + ar) * R + c] = acc[l];
      acc[l] = fmaf(a.alpha, acc[l] - Uo[ar * R + c], Uo[ar * R + c]);
    }
  } else if (a.ustar_out && ar < rows) {
#pragma unroll
    for (int l = 0; l < CG; ++l) a.ustar_out[(row0 + ar) * R + g * CG + l] = acc[l];
  }
  bool finite = true;
#pragma unroll
  for (int l = 0; l < CG; ++l) {
    const int c = g * CG + l;
    const float v = ar < rows ? acc[l] : 0.f;
    finite = finite && isfinite(v);
    Un[ar * R + c] = v;
    if (ar < rows) Unew[(row0 + ar) * R + c] = v;
  }
  if (!finite) st->status = 4;
  __syncthreads();
  // Gram partials over this CTA's rows: G = Un^T Un, Xu = Uo^T Un
  for (int e = tid; e < R * R; e += 256) {
    int k = e / R, l = e % R;
    float gg = 0.f, xu = 0.f;
    for (int rr = 0; rr < rows; ++rr) {
      gg = fmaf(Un[rr * R + k], Un[rr * R + l], gg);
      xu = fmaf(Uo[rr * R + k], Un[rr * R + l], xu);
    }
    a.part_g[(int64_t)blockIdx.x * R * R + e] = (double)gg;
    a.part_xu[(int64_t)blockIdx.x * R * R + e] = (double)xu;
  }
}

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon et al., SC'11) for the default starting point U0.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void philox_round(uint32_t& x0, uint32_t& x1, uint32_t& x2,
                                             uint32_t& x3, uint32_t k0, uint32_t k1) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  uint32_t hi0 = __umulhi(M0, x0), lo0 = M0 * x0;
  uint32_t hi1 = __umulhi(M1, x2), lo1 = M1 * x2;
  uint32_t y0 = hi1 ^ x1 ^ k0, y1 = lo1, y2 = hi0 ^ x3 ^ k1, y3 = lo0;
  x0 = y0; x1 = y1; x2 = y2; x3 = y3;
}

__device__ void philox4x32_10(uint32_t ctr[4], uint32_t k0, uint32_t k1) {
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
  for (int i = 0; i < 10; ++i) {
    philox_round(ctr[0], ctr[1], ctr[2], ctr[3], k0, k1);
    k0 += W0;
    k1 += W1;
  }
}

// U0[a, k] ~ N(0, 1/m) for k < r, 0 in the padding.  Element e = a*r + k draws
// from counter (e/2, 0, 0, 0): two uniforms (words 0, 1) -> Box-Muller pair.
__global__ void k_philox_u0(float* U, int64_t m, int r, int R, uint64_t seed) {
  int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= m * R) return;
  int64_t a = idx / R;
  int k = (int)(idx % R);
  if (k >= r) { U[idx] = 0.f; return; }
  int64_t e = a * r + k;
  uint32_t c[4] = {(uint32_t)(e >> 1), (uint32_t)((uint64_t)e >> 33), 0u, 0u};
  philox4x32_10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
  float u1 = ((float)c[0] + 0.5f) * 2.3283064365386963e-10f;
  float u2 = ((float)c[1] + 0.5f) * 2.3283064365386963e-10f;
  float rad = sqrtf(-2.0f * logf(u1));
  float z = (e & 1) ? rad * sinf(6.283185307179586f * u2) : rad * cosf(6.283185307179586f * u2);
  U[idx] = z * rsqrtf((float)m);
}

__global__ void k_check_finite(const float* x, int64_t count, int* flag) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (; i < count; i += stride)
    if (!isfinite(x[i])) { atomicExch(flag, 1); return; }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
int pick_R(int r) { return r <= 8 ? 8 : r <= 16 ? 16 : r <= 32 ? 32 : 64; }

static size_t gram_smem(int cx, int cy) { return (size_t)kGramChunk * (cx + cy) * sizeof(float); }

cudaError_t launch_gram(const float* X, int ldx, int cx, const float* Y, int ldy, int cy,
                        int64_t N, double* part, int nparts, const DevState* st,
                        int respect_stop, cudaStream_t s) {
  int64_t rows_per = (N + nparts - 1) / nparts;
  k_gram_part<<<nparts, 256, gram_smem(cx, cy), s>>>(X, ldx, cx, Y, ldy, cy, N, rows_per, part,
                                                     st, respect_stop);
  return cudaGetLastError();
}

static cudaError_t launch_reduce(const ReduceArgs& ra, cudaStream_t s) {
  int grid = (ra.total + kRedEntriesPerCta - 1) / kRedEntriesPerCta;
  size_t smem = (size_t)ra.R * ra.R * (sizeof(double) + sizeof(float));
  k_reduce_parts<<<grid, 256, smem, s>>>(ra);
  return cudaGetLastError();
}

template <int R>
static cudaError_t make_w_T(const IterArgs& a, int copy, int respect_stop, cudaStream_t s) {
  int64_t blocks = (a.m + kRowsPerCta - 1) / kRowsPerCta;
  k_make_w<R><<<(unsigned)blocks, 256, 0, s>>>(a.U[copy], a.st, a.sm, a.W, a.m, respect_stop);
  return cudaGetLastError();
}

cudaError_t launch_make_w(const IterArgs& a, int copy, int respect_stop, cudaStream_t s) {
  switch (a.R) {
    case 8: return make_w_T<8>(a, copy, respect_stop, s);
    case 16: return make_w_T<16>(a, copy, respect_stop, s);
    case 32: return make_w_T<32>(a, copy, respect_stop, s);
    default: return make_w_T<64>(a, copy, respect_stop, s);
  }
}

// The reduction tail needs R*R*12 bytes of dynamic shared memory (48 KB at R = 64).
cudaError_t prepare_small_kernels() {
  return cudaFuncSetAttribute(k_reduce_parts, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              kMaxR * kMaxR * 12);
}

template <int R>
static cudaError_t rows_T(const IterArgs& a, cudaStream_t s) {
  k_rows<R><<<a.n_rblocks, 256, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_rows(const IterArgs& a, cudaStream_t s) {
  switch (a.R) {
    case 8: return rows_T<8>(a, s);
    case 16: return rows_T<16>(a, s);
    case 32: return rows_T<32>(a, s);
    default: return rows_T<64>(a, s);
  }
}

// reduction of V-side partials (Q_t, V_{t-1}^T V_t, Huber) + Cholesky(Q_t + rho I)
cudaError_t launch_reduce_q(const IterArgs& a, double* out_q, double* out_xv, double* out_h,
                            int nparts_gram, unsigned int* counter, cudaStream_t s) {
  ReduceArgs ra{};
  const int RR = a.R * a.R;
  ra.part[0] = a.part_q; ra.count[0] = RR; ra.out[0] = out_q; ra.nparts[0] = nparts_gram;
  ra.part[1] = a.part_xv; ra.count[1] = RR; ra.out[1] = out_xv; ra.nparts[1] = nparts_gram;
  ra.part[2] = a.part_h; ra.count[2] = 1; ra.out[2] = out_h; ra.nparts[2] = a.n_vblocks;
  ra.total = 2 * RR + 1;
  ra.tail = TAIL_Q;
  ra.copy = a.cur;
  ra.R = a.R; ra.rho = a.rho; ra.u_mode = a.u_mode;
  ra.counter = counter; ra.sm = a.sm; ra.st = a.st;
  return launch_reduce(ra, s);
}

cudaError_t launch_reduce_g(const IterArgs& a, double* out_g, double* out_xu,
                            unsigned int* counter, cudaStream_t s) {
  ReduceArgs ra{};
  const int RR = a.R * a.R;
  ra.part[0] = a.part_g; ra.count[0] = RR; ra.out[0] = out_g; ra.nparts[0] = a.n_rblocks;
  ra.part[1] = a.part_xu; ra.count[1] = RR; ra.out[1] = out_xu; ra.nparts[1] = a.n_rblocks;
  ra.total = 2 * RR;
  ra.tail = TAIL_G;
  ra.copy = a.cur;
  ra.R = a.R; ra.rho = a.rho; ra.u_mode = a.u_mode;
  ra.counter = counter; ra.sm = a.sm; ra.st = a.st;
  return launch_reduce(ra, s);
}

cudaError_t launch_reduce_init(const IterArgs& a, int which /*0: G, 1: Q*/, int copy,
                               const double* part, int nparts, double* out,
                               unsigned int* counter, cudaStream_t s) {
  ReduceArgs ra{};
  const int RR = a.R * a.R;
  ra.part[0] = part; ra.count[0] = RR; ra.out[0] = out; ra.nparts[0] = nparts;
  ra.total = RR;
  ra.tail = which == 0 ? TAIL_INIT_G : TAIL_INIT_Q;
  ra.R = a.R; ra.rho = a.rho; ra.u_mode = a.u_mode; ra.copy = copy;
  ra.counter = counter; ra.sm = a.sm; ra.st = a.st;
  return launch_reduce(ra, s);
}

cudaError_t launch_reduce_plain(const double* part, int nparts, int count, double* out,
                                cudaStream_t s) {
  ReduceArgs ra{};
  ra.part[0] = part; ra.count[0] = count; ra.out[0] = out; ra.nparts[0] = nparts;
  ra.total = count;
  ra.tail = TAIL_NONE;
  ra.R = 1;
  return launch_reduce(ra, s);
}

cudaError_t launch_philox_u0(float* U, int64_t m, int r, int R, uint64_t seed, cudaStream_t s) {
  int64_t tot = m * R;
  k_philox_u0<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(U, m, r, R, seed);
  return cudaGetLastError();
}

cudaError_t launch_check_finite(const float* x, int64_t count, int* flag, cudaStream_t s) {
  int64_t blocks = (count + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  if (blocks < 1) blocks = 1;
  k_check_finite<<<(unsigned)blocks, 256, 0, s>>>(x, count, flag);
  return cudaGetLastError();
}

}  // namespace dcf
