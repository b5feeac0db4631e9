// Streaming kernels over M (general path: any m, n_i, r <= 64).
//
// One DCF-PCA iteration touches every entry of M three times in arithmetic:
//   R = M - U V^T            (residual with the previous factors)
//   S = soft(R, lambda),  X = M - S = U V^T + clamp(R, -lambda, lambda)
//   V' = X^T W               (V-step, W = U (U^T U + rho I)^{-1})
//   P  = X V'                (numerator of the consensus U-step)
// V'[j,:] needs the whole column j of X before P can use it.  This general
// path resolves that dependency with two passes over M:
//   k_pass1  column strips: X and V' = X^T W, plus the Huber sum of R
//   k_pass2  row blocks x column splits: X again and P partials
// (8 bytes of M read per entry per iteration).  The single-pass cluster
// kernel is the fast path; this one covers every shape.
#include "dcf_internal.cuh"

namespace dcf {

__host__ __device__ __forceinline__ int64_t dmin64(int64_t a, int64_t b) { return a < b ? a : b; }

__device__ __forceinline__ void two_sum_add2(float& hi, float& lo, float x) {
  float t = hi + x;
  float bp = t - hi;
  float err = (hi - (t - bp)) + (x - bp);
  hi = t;
  lo += err;
}

__device__ __forceinline__ float huber1(float r, float lam) {
  float a = fabsf(r);
  return a <= lam ? 0.5f * r * r : lam * a - 0.5f * lam * lam;
}

// ---------------------------------------------------------------------------
// pass 1: V' = X^T W on column strips of 64 columns (persistent grid)
// mode_init = 1: X = M (the S = 0 sweep that forms V0), writes copy `out_copy`
// ---------------------------------------------------------------------------
constexpr int kP1Cols = 64;

template <int R>
struct P1Cfg {
  static constexpr int RC = R <= 32 ? 128 : 64;   // rows per chunk
  static constexpr int KQ = R / 4;                 // V' entries per thread
  static constexpr size_t smem_floats = (size_t)kP1Cols * (RC + 1) + 2 * (size_t)RC * R;
};

// One 64-column strip s of one problem: X and V'[strip] = X^T W, Huber sum
// added to (hub_hi, hub_lo).  Block-wide (256 threads); sh: P1Cfg smem.
template <int R>
__device__ __forceinline__ void pass1_strip(const IterArgs& a, int mode_init, int out_copy,
                                            int64_t s, float* sh, float& hub_hi, float& hub_lo) {
  using C = P1Cfg<R>;
  constexpr int RC = C::RC, KQ = C::KQ, LDM = RC + 1;
  float* Mt = sh;                              // [64][RC+1]   M, then X
  float* Us = Mt + kP1Cols * LDM;              // [RC][R]
  float* Ws = Us + RC * R;                     // [RC][R]
  const int tid = threadIdx.x;
  const int j = tid & 63, q = tid >> 6;
  const int cur = a.cur;
  const float* U = a.U[mode_init ? out_copy : cur];
  const float* Vold = a.V[cur];
  float* Vout = a.V[mode_init ? out_copy : (cur ^ 1)];
  const float lam = a.lam;
  const int64_t m = a.m, n = a.n;
  {
    const int64_t col = s * kP1Cols + j;
    const bool valid = col < n;
    float v[R];
#pragma unroll
    for (int k = 0; k < R; ++k) v[k] = (valid && !mode_init) ? Vold[col * R + k] : 0.f;
    float yhi[KQ], ylo[KQ];
#pragma unroll
    for (int kk = 0; kk < KQ; ++kk) { yhi[kk] = 0.f; ylo[kk] = 0.f; }
    for (int64_t a0 = 0; a0 < m; a0 += RC) {
      const int rows = (int)dmin64((int64_t)(RC), m - a0);
      __syncthreads();
      for (int idx = tid; idx < kP1Cols * RC; idx += 256) {
        int jj = idx / RC, aa = idx % RC;
        int64_t cc = s * kP1Cols + jj;
        Mt[jj * LDM + aa] = (aa < rows && cc < n) ? a.M[cc * m + a0 + aa] : 0.f;
      }
      for (int idx = tid; idx < RC * R; idx += 256) {
        int aa = idx / R;
        bool ok = aa < rows;
        Us[idx] = ok ? U[(a0 + aa) * R + (idx % R)] : 0.f;
        Ws[idx] = ok ? a.W[(a0 + aa) * R + (idx % R)] : 0.f;
      }
      __syncthreads();
      // X = U V^T + clamp(M - U V^T, -lambda, lambda)
      float hub = 0.f;
      for (int aa = q; aa < RC; aa += 4) {
        const float4* u4 = reinterpret_cast<const float4*>(Us + aa * R);
        float d = 0.f;
#pragma unroll
        for (int k4 = 0; k4 < R / 4; ++k4) {
          float4 u = u4[k4];
          d = fmaf(u.x, v[4 * k4], d);
          d = fmaf(u.y, v[4 * k4 + 1], d);
          d = fmaf(u.z, v[4 * k4 + 2], d);
          d = fmaf(u.w, v[4 * k4 + 3], d);
        }
        float mv = Mt[j * LDM + aa];
        float x;
        if (mode_init) {
          x = mv;
        } else {
          float r = mv - d;
          float c = fminf(fmaxf(r, -lam), lam);
          x = d + c;
          hub += huber1(r, lam);
        }
        Mt[j * LDM + aa] = x;
      }
      two_sum_add2(hub_hi, hub_lo, hub);
      __syncthreads();
      // V'[j, q*KQ .. q*KQ+KQ) += sum_a X[a,j] W[a,:]
      float yc[KQ];
#pragma unroll
      for (int kk = 0; kk < KQ; ++kk) yc[kk] = 0.f;
      for (int aa = 0; aa < rows; ++aa) {
        float x = Mt[j * LDM + aa];
        const float* w = Ws + aa * R + q * KQ;
#pragma unroll
        for (int kk = 0; kk < KQ; ++kk) yc[kk] = fmaf(x, w[kk], yc[kk]);
      }
#pragma unroll
      for (int kk = 0; kk < KQ; ++kk) two_sum_add2(yhi[kk], ylo[kk], yc[kk]);
    }
    if (valid) {
#pragma unroll
      for (int kk = 0; kk < KQ; ++kk) Vout[col * R + q * KQ + kk] = yhi[kk] + ylo[kk];
    }
  }
}

// Sum of (hi + lo) over the CTA into *out (thread 0); block-wide.
__device__ __forceinline__ void block_huber(float hub_hi, float hub_lo, double* out) {
  __shared__ double red[256];
  const int tid = threadIdx.x;
  __syncthreads();
  red[tid] = (double)hub_hi + (double)hub_lo;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (tid < w) red[tid] += red[tid + w];
    __syncthreads();
  }
  if (tid == 0) *out = red[0];
}

template <int R>
__global__ void __launch_bounds__(256) k_pass1(IterArgs a, int mode_init, int out_copy) {
  DevState* st = a.st;
  if (!mode_init && st->stop) return;
  extern __shared__ __align__(16) float sh[];
  const int64_t nstrips = (a.n + kP1Cols - 1) / kP1Cols;
  float hub_hi = 0.f, hub_lo = 0.f;
  for (int64_t s = blockIdx.x; s < nstrips; s += gridDim.x)
    pass1_strip<R>(a, mode_init, out_copy, s, sh, hub_hi, hub_lo);
  // Huber partial of this CTA
  if (!mode_init) block_huber(hub_hi, hub_lo, a.part_h + blockIdx.x);
}

// Batched pass 1: item (instance, strip); the Huber partial goes to the strip.
template <int R>
__global__ void __launch_bounds__(256) k_bpass1(const BInst* __restrict__ insts,
                                                const BItem* __restrict__ items, int nitems,
                                                int cur, int mode_init) {
  extern __shared__ __align__(16) float sh[];
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const BItem w = items[it];
    const BInst& I = insts[w.inst];
    if (!mode_init && I.st->stop) continue;   // uniform over the CTA
    const IterArgs a = batch_iter_args(I, cur);
    float hub_hi = 0.f, hub_lo = 0.f;
    __syncthreads();                           // shared memory of the previous item
    pass1_strip<R>(a, mode_init, cur, w.a, sh, hub_hi, hub_lo);
    if (!mode_init) block_huber(hub_hi, hub_lo, I.part_h + w.a);
  }
}

// ---------------------------------------------------------------------------
// pass 2: P partials = X V' over (128-row block) x (column split)
// ---------------------------------------------------------------------------
constexpr int kP2Rows = 128;
constexpr int kP2Cols = 32;

// One (128-row block rb) x (column split sp) item of one problem: P partial.
// Block-wide (256 threads).
template <int R>
__device__ __forceinline__ void pass2_block(const IterArgs& a, int64_t rb, int64_t sp) {
  constexpr int KH = R / 2;
  __shared__ __align__(16) float Mt[kP2Cols * kP2Rows];
  __shared__ __align__(16) float Vo[kP2Cols * R];
  __shared__ __align__(16) float Vn[kP2Cols * R];
  const int tid = threadIdx.x;
  const int ar = tid & (kP2Rows - 1), h = tid >> 7;
  const int cur = a.cur;
  const float* U = a.U[cur];
  const float* Vold = a.V[cur];
  const float* Vnew = a.V[cur ^ 1];
  const float lam = a.lam;
  const int64_t m = a.m, n = a.n;
  const int64_t a0 = rb * kP2Rows;
  const int64_t arow = a0 + ar;
  const bool rvalid = arow < m;
  const int64_t c_begin = sp * a.split_cols;
  const int64_t c_end = min(n, c_begin + a.split_cols);
  float u[R];
#pragma unroll
  for (int k = 0; k < R; ++k) u[k] = rvalid ? U[arow * R + k] : 0.f;
  float phi[KH], plo[KH];
#pragma unroll
  for (int kk = 0; kk < KH; ++kk) { phi[kk] = 0.f; plo[kk] = 0.f; }
  for (int64_t c0 = c_begin; c0 < c_end; c0 += kP2Cols) {
    const int cols = (int)dmin64((int64_t)(kP2Cols), c_end - c0);
    __syncthreads();
    for (int idx = tid; idx < kP2Cols * kP2Rows; idx += 256) {
      int jj = idx / kP2Rows, aa = idx % kP2Rows;
      Mt[idx] = (jj < cols && a0 + aa < m) ? a.M[(c0 + jj) * m + a0 + aa] : 0.f;
    }
    for (int idx = tid; idx < kP2Cols * R; idx += 256) {
      int jj = idx / R;
      bool ok = jj < cols;
      Vo[idx] = ok ? Vold[(c0 + jj) * R + (idx % R)] : 0.f;
      Vn[idx] = ok ? Vnew[(c0 + jj) * R + (idx % R)] : 0.f;
    }
    __syncthreads();
    for (int jj = h; jj < kP2Cols; jj += 2) {
      const float4* v4 = reinterpret_cast<const float4*>(Vo + jj * R);
      float d = 0.f;
#pragma unroll
      for (int k4 = 0; k4 < R / 4; ++k4) {
        float4 v = v4[k4];
        d = fmaf(u[4 * k4], v.x, d);
        d = fmaf(u[4 * k4 + 1], v.y, d);
        d = fmaf(u[4 * k4 + 2], v.z, d);
        d = fmaf(u[4 * k4 + 3], v.w, d);
      }
      float mv = Mt[jj * kP2Rows + ar];
      float r = mv - d;
      float c = fminf(fmaxf(r, -lam), lam);
      Mt[jj * kP2Rows + ar] = d + c;
    }
    __syncthreads();
    float pc[KH];
#pragma unroll
    for (int kk = 0; kk < KH; ++kk) pc[kk] = 0.f;
    for (int jj = 0; jj < cols; ++jj) {
      float x = Mt[jj * kP2Rows + ar];
      const float* vn = Vn + jj * R + h * KH;
#pragma unroll
      for (int kk = 0; kk < KH; ++kk) pc[kk] = fmaf(x, vn[kk], pc[kk]);
    }
#pragma unroll
    for (int kk = 0; kk < KH; ++kk) two_sum_add2(phi[kk], plo[kk], pc[kk]);
  }
  if (rvalid) {
    float* out = a.part_p + (sp * m + arow) * R + h * KH;
#pragma unroll
    for (int kk = 0; kk < KH; ++kk) out[kk] = phi[kk] + plo[kk];
  }
}

template <int R>
__global__ void __launch_bounds__(256) k_pass2(IterArgs a) {
  if (a.st->stop) return;
  pass2_block<R>(a, blockIdx.x, blockIdx.y);
}

// Batched pass 2: item (instance, row block, column split).
template <int R>
__global__ void __launch_bounds__(256) k_bpass2(const BInst* __restrict__ insts,
                                                const BItem* __restrict__ items, int nitems,
                                                int cur) {
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const BItem w = items[it];
    const BInst& I = insts[w.inst];
    if (I.st->stop) continue;
    const IterArgs a = batch_iter_args(I, cur);
    __syncthreads();                           // shared memory of the previous item
    pass2_block<R>(a, w.a, w.b);
  }
}

// ---------------------------------------------------------------------------
// L_i = U V_i^T (mode 0) or S_i = soft(M_i - U V_i^T, lambda) (mode 1),
// m x n_i column-major output with leading dimension m.
// ---------------------------------------------------------------------------
__global__ void k_materialize(const float* M, int64_t m, int64_t c0, int64_t ni,
                              const float* U, const float* V, int R, float lam, int mode,
                              float* out) {
  int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t tot = m * ni;
  if (idx >= tot) return;
  int64_t jj = idx / m, aa = idx % m;
  const float* u = U + aa * R;
  const float* v = V + (c0 + jj) * R;
  float d = 0.f;
  for (int k = 0; k < R; ++k) d = fmaf(u[k], v[k], d);
  if (mode == 0) {
    out[idx] = d;
  } else {
    float r = M[(c0 + jj) * m + aa] - d;
    float mag = fabsf(r) - lam;
    out[idx] = mag > 0.f ? copysignf(mag, r) : 0.f;
  }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
template <int R>
static cudaError_t pass1_T(const IterArgs& a, int grid, int mode_init, int out_copy,
                           cudaStream_t s) {
  size_t smem = P1Cfg<R>::smem_floats * sizeof(float);
  k_pass1<R><<<grid, 256, smem, s>>>(a, mode_init, out_copy);
  return cudaGetLastError();
}

template <int R>
static cudaError_t prep_pass1_T() {
  size_t smem = P1Cfg<R>::smem_floats * sizeof(float);
  return cudaFuncSetAttribute(k_pass1<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

// Raise the dynamic shared-memory limits once, outside any stream capture.
cudaError_t prepare_stream_kernels() {
  cudaError_t e;
  if ((e = prep_pass1_T<8>()) != cudaSuccess) return e;
  if ((e = prep_pass1_T<16>()) != cudaSuccess) return e;
  if ((e = prep_pass1_T<32>()) != cudaSuccess) return e;
  return prep_pass1_T<64>();
}

cudaError_t launch_pass1(const IterArgs& a, int grid, int mode_init, int out_copy,
                         cudaStream_t s) {
  switch (a.R) {
    case 8: return pass1_T<8>(a, grid, mode_init, out_copy, s);
    case 16: return pass1_T<16>(a, grid, mode_init, out_copy, s);
    case 32: return pass1_T<32>(a, grid, mode_init, out_copy, s);
    default: return pass1_T<64>(a, grid, mode_init, out_copy, s);
  }
}

template <int R>
static cudaError_t pass2_T(const IterArgs& a, cudaStream_t s) {
  dim3 grid((unsigned)((a.m + kP2Rows - 1) / kP2Rows), (unsigned)a.n_splits);
  k_pass2<R><<<grid, 256, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_pass2(const IterArgs& a, cudaStream_t s) {
  switch (a.R) {
    case 8: return pass2_T<8>(a, s);
    case 16: return pass2_T<16>(a, s);
    case 32: return pass2_T<32>(a, s);
    default: return pass2_T<64>(a, s);
  }
}

template <int R>
static cudaError_t bpass_T(const BInst* insts, const BItem* it1, int n1, int grid1,
                           const BItem* it2, int n2, int grid2, int cur, int which,
                           int mode_init, cudaStream_t s) {
  if (which == 1) {
    if (n1 == 0) return cudaSuccess;
    size_t smem = P1Cfg<R>::smem_floats * sizeof(float);
    k_bpass1<R><<<grid1, 256, smem, s>>>(insts, it1, n1, cur, mode_init);
  } else {
    if (n2 == 0) return cudaSuccess;
    k_bpass2<R><<<grid2, 256, 0, s>>>(insts, it2, n2, cur);
  }
  return cudaGetLastError();
}

// which = 1: batched pass 1 over items it1; which = 2: batched pass 2 over it2.
cudaError_t launch_bpass(int R, int which, const BInst* insts, const BItem* it1, int n1, int grid1,
                         const BItem* it2, int n2, int grid2, int cur, int mode_init,
                         cudaStream_t s) {
  switch (R) {
    case 8: return bpass_T<8>(insts, it1, n1, grid1, it2, n2, grid2, cur, which, mode_init, s);
    case 16: return bpass_T<16>(insts, it1, n1, grid1, it2, n2, grid2, cur, which, mode_init, s);
    default: return bpass_T<32>(insts, it1, n1, grid1, it2, n2, grid2, cur, which, mode_init, s);
  }
}

template <int R>
static cudaError_t prep_bpass1_T() {
  size_t smem = P1Cfg<R>::smem_floats * sizeof(float);
  return cudaFuncSetAttribute(k_bpass1<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

cudaError_t prepare_batch_stream_kernels() {
  cudaError_t e;
  if ((e = prep_bpass1_T<8>()) != cudaSuccess) return e;
  if ((e = prep_bpass1_T<16>()) != cudaSuccess) return e;
  return prep_bpass1_T<32>();
}

cudaError_t launch_materialize(const float* M, int64_t m, int64_t c0, int64_t ni,
                               const float* U, const float* V, int R, float lam, int mode,
                               float* out, cudaStream_t s) {
  int64_t tot = m * ni;
  k_materialize<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(M, m, c0, ni, U, V, R, lam, mode,
                                                               out);
  return cudaGetLastError();
}

}  // namespace dcf
