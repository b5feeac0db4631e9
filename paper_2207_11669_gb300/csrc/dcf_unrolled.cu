// Learned unrolled DCF network: K exact-consensus iterations with per-step
// parameters, evaluated on the GPU with checkpoints, and its adjoint.
//
// Step k (parameters a_k, b_k, c_k):
//   lambda_k = lambda e^{a_k},  rho_k = rho e^{b_k},  alpha_k = c_k
//   R = M - U V^T,  C = clamp(R, +-lambda_k),  X = U V^T + C        (S-step, Sec. 2.2)
//   G = U^T U + rho_k I,  W = U G^{-1},  V' = X^T W                  (V-step, App. B)
//   P = X V',  H = V'^T V' + rho_k I,  U* = P H^{-1}                 (exact consensus U-step)
//   U' = U + alpha_k (U* - U)                                        (relaxation)
// Loss: sum_k w_k ||U_k V_k^T - A B^T||_F^2 / ||A B^T||_F^2, evaluated through
// r x r and r x k Gram matrices, never through an m x n product.
//
// Forward: the plain iteration kernels run with the step's parameters; the
// U-step kernel applies the relaxation and stores U* as well.  Checkpoints are
// (U_k, V_k) for k = 0..K and U*_k: O(K (m + n) r) floats per problem.
//
// Backward, for k = K-1 .. 0 (reverse mode of the step; every m x n quantity is
// recomputed from M and the checkpoint, nothing of size m x n is stored):
//   Ubar' += w_k dLoss/dU_{k+1},  Vbar' += w_k dLoss/dV_{k+1}
//   alpha_bar = <Ubar', U* - U>,  Pbar = alpha Ubar' H^{-1}
//   Hbar = sym(-(U*^T alpha Ubar') H^{-1}),  rho_bar = tr Hbar
//   Vbar_tot = Vbar' + 2 V' Hbar + X^T Pbar          (pass A: column strips)
//   Xbar = Pbar V'^T + W Vbar_tot^T,  D = Xbar . 1[|R| > lambda_k]
//   Vbar = D^T U,  lambda_bar = sum D . sign(R)      (pass B: column strips)
//   Ubar_D = D V,  Wbar = X Vbar_tot                 (pass C: row blocks)
//   (for R <= 16 passes B and C are one kernel over row blocks x column
//   splits, k_adj_fused, with Vbar summed from per-row-block partials)
//   Gbar = sym(-(W^T Wbar) G^{-1}),  rho_bar += tr Gbar
//   Ubar = (1 - alpha) Ubar' + Ubar_D + Wbar G^{-1} + 2 U Gbar
//   grad a_k = lambda_bar lambda_k,  grad b_k = rho_bar rho_k,  grad c_k = alpha_bar
// r x r algebra is FP64 on one CTA; streams over M are FP32 with compensated
// accumulation.  Supported for the exact U-step and padded rank R <= 32.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <initializer_list>
#include <vector>

#include "dcf.h"
#include "dcf_handle.h"
#include "dcf_internal.cuh"
#include "dcf_small.cuh"

namespace dcf {
namespace {

constexpr int kUnrolledMaxR = 32;
constexpr int kSlot = kMaxR * kMaxR;

__host__ __device__ __forceinline__ int64_t imin64(int64_t a, int64_t b) { return a < b ? a : b; }

__device__ __forceinline__ void tsum(float& hi, float& lo, float x) {
  float t = hi + x;
  float bp = t - hi;
  float err = (hi - (t - bp)) + (x - bp);
  hi = t;
  lo += err;
}

// ---------------------------------------------------------------------------
// (U^T U + rho I)^{-1} of the current U, for a step whose rho differs from the
// one the previous U-step used.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_refactor_ginv(Smalls* sm, DevState* st, int cur, int R,
                                                       int r, float rho) {
  extern __shared__ double dsh[];   // R*R doubles, R*R double-floats
  df2* F = reinterpret_cast<df2*>(dsh + R * R);
  for (int i = threadIdx.x; i < R * R; i += blockDim.x) {
    int r = i / R, c = i % R;
    dsh[i] = sm->gram[cur][i] + (r == c ? (double)rho : 0.0);
  }
  __syncthreads();
  if (!all_finite(dsh, R * R)) {
    if (threadIdx.x == 0) st->status = DCF_ENONFINITE;
    return;
  }
  const double kappa = spd_inverse(dsh, F, R, r, sm->ginv32, sm->ginv32_lo, kDfKappa,
                                   &st->route_g);
  if (threadIdx.x == 0) st->kappa_g = kappa;
}

// ---------------------------------------------------------------------------
// r x r algebra of the network (one CTA of 256 threads)
// ---------------------------------------------------------------------------
enum SmallMode {
  SM_LOSS_C = 0,     // dsc[0] = <A^T A, B^T B> = ||A B^T||^2
  SM_LOSS_TERM = 1,  // loss[step] = ||U V^T - A B^T||^2 / ||A B^T||^2
  SM_LOSSGRAD = 2,   // matrices of w_k dLoss/dU, dLoss/dV
  SM_RECOMP = 3,     // G^{-1}, H^{-1}, alpha H^{-1}
  SM_HBAR = 4,       // alpha_bar, Hbar, rho_bar (H part)
  SM_GBAR = 5        // Gbar, rho_bar, lambda_bar; the three parameter gradients
};

// FP64 reduction slots (kSlot doubles each)
enum RedSlot { RD_UU = 0, RD_VV, RD_UA, RD_VB, RD_AA, RD_BB, RD_A1, RD_A2, RD_WWB, kNumRed };
// FP32 matrix slots (kSlot floats each)
enum MatSlot {
  MT_SVV = 0,  // s V^T V          (R x R)
  MT_SBV,      // -s (V^T B)^T     (k x R)
  MT_SUU,      // s U^T U          (R x R)
  MT_SAU,      // -s (U^T A)^T     (k x R)
  MT_GINV,     // G^{-1}
  MT_AHINV,    // alpha H^{-1}
  MT_HBAR2,    // 2 Hbar
  MT_GBAR2,    // 2 Gbar
  MT_HINV,     // H^{-1}
  kNumMat
};
// FP64 scalars
enum Scalar { SC_C = 0, SC_ABAR, SC_RBAR, kNumSc };

struct SmallArgs {
  int mode;
  int mode2;           // a second, independent mode run after the first (-1: none)
  int R, k;            // padded rank, truth rank
  int r;               // the solver's rank (leading block of the r x r systems)
  int K, step;
  double lam_k, rho_k, alpha_k, w_k;
  const double* red;   // [kNumRed][kSlot]
  const double* red_prev;   // SM_RECOMP: the slots whose RD_UU holds U_k^T U_k
  float* mats;         // [kNumMat][kSlot]
  double* sc;          // [kNumSc]
  double* loss;        // [K]
  double* grads;       // [3][K]
  const double* lam_part;
  int n_lam_part;
  DevState* st;
};

__device__ double block_sum(double v, double* red) {
  red[threadIdx.x] = v;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  double r = red[0];
  __syncthreads();
  return r;
}

__device__ void small_mode(const SmallArgs& a, int mode, double* dsh, double* red);

__global__ void __launch_bounds__(256) k_unrolled_small(SmallArgs a) {
  extern __shared__ double dsh[];   // 3 R*R doubles, R*R double-floats
  __shared__ double red[256];
  small_mode(a, a.mode, dsh, red);
  if (a.mode2 >= 0) {
    __syncthreads();
    small_mode(a, a.mode2, dsh, red);
  }
}

__device__ void small_mode(const SmallArgs& a, int mode, double* dsh, double* red) {
  const int R = a.R, k = a.k, RR = R * R;
  const int tid = threadIdx.x;
  const double* slot = a.red;
  auto S = [&](int s) { return slot + (size_t)s * kSlot; };
  float* mats = a.mats;
  auto Mt = [&](int s) { return mats + (size_t)s * kSlot; };
  switch (mode) {
    case SM_LOSS_C: {
      double v = 0;
      for (int i = tid; i < k * k; i += blockDim.x) v += S(RD_AA)[i] * S(RD_BB)[i];
      v = block_sum(v, red);
      if (tid == 0) a.sc[SC_C] = v;
      break;
    }
    case SM_LOSS_TERM: {
      double v1 = 0, v2 = 0;
      for (int i = tid; i < RR; i += blockDim.x) v1 += S(RD_UU)[i] * S(RD_VV)[i];
      for (int i = tid; i < R * k; i += blockDim.x) v2 += S(RD_UA)[i] * S(RD_VB)[i];
      v1 = block_sum(v1, red);
      v2 = block_sum(v2, red);
      if (tid == 0) {
        const double c = a.sc[SC_C];
        const double d2 = v1 - 2.0 * v2 + c;
        a.loss[a.step] = (d2 > 0 ? d2 : 0.0) / c;
      }
      break;
    }
    case SM_LOSSGRAD: {
      // dLoss/dU = (2/c)(U V^T V - A B^T V),  dLoss/dV = (2/c)(V U^T U - B A^T U)
      const double s = 2.0 * a.w_k / a.sc[SC_C];
      for (int i = tid; i < RR; i += blockDim.x) {
        Mt(MT_SVV)[i] = (float)(s * S(RD_VV)[i]);
        Mt(MT_SUU)[i] = (float)(s * S(RD_UU)[i]);
      }
      for (int i = tid; i < k * R; i += blockDim.x) {
        const int j = i / R, c = i % R;   // (k x R) row j, column c
        Mt(MT_SBV)[i] = (float)(-s * S(RD_VB)[c * k + j]);
        Mt(MT_SAU)[i] = (float)(-s * S(RD_UA)[c * k + j]);
      }
      break;
    }
    case SM_RECOMP: {
      double* A = dsh;
      df2* F = reinterpret_cast<df2*>(dsh + 3 * RR);
      for (int pass = 0; pass < 2; ++pass) {
        const double* g = pass == 0 ? a.red_prev + (size_t)RD_UU * kSlot : S(RD_VV);
        for (int i = tid; i < RR; i += blockDim.x)
          A[i] = g[i] + ((i / R) == (i % R) ? a.rho_k : 0.0);
        __syncthreads();
        if (!all_finite(A, RR)) {
          if (tid == 0) a.st->status = DCF_ENONFINITE;
          return;
        }
        spd_inverse(A, F, R, a.r, pass == 0 ? Mt(MT_GINV) : Mt(MT_HINV), nullptr, kDfKappa);
      }
      for (int i = tid; i < RR; i += blockDim.x)
        Mt(MT_AHINV)[i] = (float)(a.alpha_k * (double)Mt(MT_HINV)[i]);
      break;
    }
    case SM_HBAR: {
      // A1 = U*^T Ubar', A2 = U^T Ubar':  alpha_bar = tr A1 - tr A2
      // Hbar = sym(-alpha A1 H^{-1}),  rho_bar = tr Hbar
      double* T = dsh;
      double tr = 0;
      for (int i = tid; i < R; i += blockDim.x) tr += S(RD_A1)[i * R + i] - S(RD_A2)[i * R + i];
      tr = block_sum(tr, red);
      const float* Hi = Mt(MT_HINV);
      for (int i = tid; i < RR; i += blockDim.x) {
        const int r = i / R, c = i % R;
        double v = 0;
        for (int p = 0; p < R; ++p) v += S(RD_A1)[r * R + p] * (double)Hi[p * R + c];
        T[i] = -a.alpha_k * v;
      }
      __syncthreads();
      double trh = 0;
      for (int i = tid; i < RR; i += blockDim.x) {
        const int r = i / R, c = i % R;
        const double hb = 0.5 * (T[i] + T[c * R + r]);
        Mt(MT_HBAR2)[i] = (float)(2.0 * hb);
        if (r == c) trh += hb;
      }
      trh = block_sum(trh, red);
      if (tid == 0) {
        a.sc[SC_ABAR] = tr;
        a.sc[SC_RBAR] = trh;
      }
      break;
    }
    case SM_GBAR: {
      double* T = dsh;
      const float* Gi = Mt(MT_GINV);
      for (int i = tid; i < RR; i += blockDim.x) {
        const int r = i / R, c = i % R;
        double v = 0;
        for (int p = 0; p < R; ++p) v += S(RD_WWB)[r * R + p] * (double)Gi[p * R + c];
        T[i] = -v;
      }
      __syncthreads();
      double trg = 0;
      for (int i = tid; i < RR; i += blockDim.x) {
        const int r = i / R, c = i % R;
        const double gb = 0.5 * (T[i] + T[c * R + r]);
        Mt(MT_GBAR2)[i] = (float)(2.0 * gb);
        if (r == c) trg += gb;
      }
      trg = block_sum(trg, red);
      double lb = 0;
      for (int i = tid; i < a.n_lam_part; i += blockDim.x) lb += a.lam_part[i];
      lb = block_sum(lb, red);
      if (tid == 0) {
        const double rho_bar = a.sc[SC_RBAR] + trg;
        a.grads[a.step] = lb * a.lam_k;
        a.grads[a.K + a.step] = rho_bar * a.rho_k;
        a.grads[2 * a.K + a.step] = a.sc[SC_ABAR];
        if (!isfinite(lb) || !isfinite(rho_bar) || !isfinite(a.sc[SC_ABAR]))
          a.st->status = DCF_ENONFINITE;
      }
      break;
    }
    default:
      break;
  }
}

// ---------------------------------------------------------------------------
// Row kernel: out[a,:] = sum_t X_t[a, 0:cx_t] Mat_t + sum_s beta_s sum_p Y_s[p][a,:]
// (32 rows per CTA; thread (row t/8, column group t%8) forms R/8 outputs).
// `out` may alias a Y_s (each thread reads its own entries before writing).
// ---------------------------------------------------------------------------
struct RowLin {
  int64_t rows;
  float* out;
  int nmat;
  const float* X[3];
  int ldx[3];
  int cx[3];
  const float* Mat[3];    // cx x R row-major
  int nadd;
  const float* Y[3];
  float beta[3];
  int nparts[3];
  int64_t pstride[3];     // floats between the partial copies of Y_s
};

// Up to three independent row jobs in one launch (blockIdx.y = job).
struct RowLinSet {
  RowLin L[3];
  int n;
};

template <int R>
__global__ void __launch_bounds__(256) k_rowlin(RowLinSet S) {
  extern __shared__ float msh[];   // the Mat_t, concatenated
  constexpr int CG = R / 8;
  const RowLin& L = S.L[blockIdx.y];
  if ((int64_t)blockIdx.x * 32 >= L.rows) return;
  const int tid = threadIdx.x;
  int off[3] = {0, 0, 0};
  {
    int o = 0;
    for (int t = 0; t < L.nmat; ++t) {
      off[t] = o;
      for (int i = tid; i < L.cx[t] * R; i += 256) msh[o + i] = L.Mat[t][i];
      o += L.cx[t] * R;
    }
  }
  __syncthreads();
  const int64_t row = (int64_t)blockIdx.x * 32 + (tid >> 3);
  const int g = tid & 7;
  if (row >= L.rows) return;
  float acc[CG];
#pragma unroll
  for (int l = 0; l < CG; ++l) acc[l] = 0.f;
  for (int t = 0; t < L.nmat; ++t) {
    const float* x = L.X[t] + row * L.ldx[t];
    const float* mt = msh + off[t];
    for (int c = 0; c < L.cx[t]; ++c) {
      const float xv = __ldg(x + c);
#pragma unroll
      for (int l = 0; l < CG; ++l) acc[l] = fmaf(xv, mt[c * R + g * CG + l], acc[l]);
    }
  }
  for (int s = 0; s < L.nadd; ++s) {
#pragma unroll
    for (int l = 0; l < CG; ++l) {
      float sum = 0.f;
      for (int p = 0; p < L.nparts[s]; ++p) sum += L.Y[s][p * L.pstride[s] + row * R + g * CG + l];
      acc[l] = fmaf(L.beta[s], sum, acc[l]);
    }
  }
#pragma unroll
  for (int l = 0; l < CG; ++l) L.out[row * R + g * CG + l] = acc[l];
}

// ---------------------------------------------------------------------------
// Adjoint streams over M
// ---------------------------------------------------------------------------
struct AdjArgs {
  const float* M;
  int64_t m, n;
  float lam;
  const float* U;      // U_k      m x R
  const float* V;      // V_k      n x R
  const float* Pb;     // Pbar     m x R
  const float* W;      // W        m x R
  const float* Vn;     // V'       n x R
  const float* Vtot;   // Vbar_tot n x R
  float* Vbar;         // out: D^T U  (n x R)
  double* lam_part;    // out: per-CTA sum of D . sign(R)
  float* part_ud;      // out: [split][m][R]  D V partials
  float* part_wb;      // out: [split][m][R]  X Vbar_tot partials
  float* part_vb;      // out (fused kernel): [row block][n][R]  D^T U partials
  int64_t split_cols;
};

// pass B: column strips of 64 columns (persistent); all m rows per strip, so
// Vbar = D^T U is complete per strip.  Thread (column j, row quarter q).
constexpr int kAbCols = 64;
constexpr int kAbRows = 128;

template <int R>
struct AbCfg {
  static constexpr int KQ = R / 4;
  static constexpr size_t smem_floats = (size_t)kAbCols * (kAbRows + 1) + 3 * (size_t)kAbRows * R;
};

template <int R>
__global__ void __launch_bounds__(256) k_adj_cols(AdjArgs a) {
  constexpr int KQ = AbCfg<R>::KQ, LDM = kAbRows + 1;
  extern __shared__ __align__(16) float sh[];
  float* Dt = sh;                               // [64][129]  M, then D
  float* Us = Dt + kAbCols * LDM;               // [128][R]
  float* Ps = Us + kAbRows * R;                 // [128][R]
  float* Ws = Ps + kAbRows * R;                 // [128][R]
  const int tid = threadIdx.x;
  const int j = tid & 63, q = tid >> 6;
  const float lam = a.lam;
  const int64_t m = a.m, n = a.n;
  const int64_t nstrips = (n + kAbCols - 1) / kAbCols;
  float lb_hi = 0.f, lb_lo = 0.f;
  for (int64_t s = blockIdx.x; s < nstrips; s += gridDim.x) {
    const int64_t col = s * kAbCols + j;
    const bool valid = col < n;
    float v[R], vn[R], vb[R];
#pragma unroll
    for (int k = 0; k < R; ++k) {
      v[k] = valid ? a.V[col * R + k] : 0.f;
      vn[k] = valid ? a.Vn[col * R + k] : 0.f;
      vb[k] = valid ? a.Vtot[col * R + k] : 0.f;
    }
    float yhi[KQ], ylo[KQ];
#pragma unroll
    for (int kk = 0; kk < KQ; ++kk) { yhi[kk] = 0.f; ylo[kk] = 0.f; }
    for (int64_t a0 = 0; a0 < m; a0 += kAbRows) {
      const int rows = (int)imin64((int64_t)kAbRows, m - a0);
      __syncthreads();
      for (int idx = tid; idx < kAbCols * kAbRows; idx += 256) {
        const int jj = idx / kAbRows, aa = idx % kAbRows;
        const int64_t cc = s * kAbCols + jj;
        Dt[jj * LDM + aa] = (aa < rows && cc < n) ? a.M[cc * m + a0 + aa] : 0.f;
      }
      for (int idx = tid; idx < kAbRows * R; idx += 256) {
        const int aa = idx / R;
        const bool ok = aa < rows;
        const int64_t gi = (a0 + aa) * R + (idx % R);
        Us[idx] = ok ? a.U[gi] : 0.f;
        Ps[idx] = ok ? a.Pb[gi] : 0.f;
        Ws[idx] = ok ? a.W[gi] : 0.f;
      }
      __syncthreads();
      float lb = 0.f;
      for (int aa = q; aa < kAbRows; aa += 4) {
        const float* u = Us + aa * R;
        const float* p = Ps + aa * R;
        const float* w = Ws + aa * R;
        float d = 0.f, xb = 0.f;
#pragma unroll
        for (int k = 0; k < R; ++k) {
          d = fmaf(u[k], v[k], d);
          xb = fmaf(p[k], vn[k], xb);
          xb = fmaf(w[k], vb[k], xb);
        }
        const float r = Dt[j * LDM + aa] - d;
        const bool outside = fabsf(r) > lam;
        const float dv = outside ? xb : 0.f;
        lb += outside ? (r > 0.f ? xb : -xb) : 0.f;
        Dt[j * LDM + aa] = dv;
      }
      tsum(lb_hi, lb_lo, lb);
      __syncthreads();
      float yc[KQ];
#pragma unroll
      for (int kk = 0; kk < KQ; ++kk) yc[kk] = 0.f;
      for (int aa = 0; aa < rows; ++aa) {
        const float dv = Dt[j * LDM + aa];
        const float* u = Us + aa * R + q * KQ;
#pragma unroll
        for (int kk = 0; kk < KQ; ++kk) yc[kk] = fmaf(dv, u[kk], yc[kk]);
      }
#pragma unroll
      for (int kk = 0; kk < KQ; ++kk) tsum(yhi[kk], ylo[kk], yc[kk]);
    }
    if (valid) {
#pragma unroll
      for (int kk = 0; kk < KQ; ++kk) a.Vbar[col * R + q * KQ + kk] = yhi[kk] + ylo[kk];
    }
  }
  __shared__ double red[256];
  red[tid] = (double)lb_hi + (double)lb_lo;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (tid < w) red[tid] += red[tid + w];
    __syncthreads();
  }
  if (tid == 0) a.lam_part[blockIdx.x] = red[0];
}

// pass C: (128-row block) x (column split); thread (row ar, half h) forms
// R/2 entries of D V and of X Vbar_tot for its row.
constexpr int kAcRows = 128;
constexpr int kAcCols = 32;

template <int R>
struct AcCfg {
  static constexpr int LDR = R + 4;   // padded row stride of the row-block operands
  static constexpr size_t smem_floats =
      2 * (size_t)kAcCols * kAcRows + 3 * (size_t)kAcCols * R + 2 * (size_t)kAcRows * LDR;
};

template <int R>
__global__ void __launch_bounds__(256) k_adj_rows(AdjArgs a) {
  constexpr int KH = R / 2, LDR = AcCfg<R>::LDR;
  extern __shared__ __align__(16) float sh[];
  float* Xt = sh;                                 // [32][128]  X
  float* Dt = Xt + kAcCols * kAcRows;             // [32][128]  D
  float* Vs = Dt + kAcCols * kAcRows;             // [32][R]    V_k
  float* Vns = Vs + kAcCols * R;                  // [32][R]    V'
  float* Vbs = Vns + kAcCols * R;                 // [32][R]    Vbar_tot
  float* Ps = Vbs + kAcCols * R;                  // [128][LDR] Pbar rows
  float* Wsm = Ps + kAcRows * LDR;                // [128][LDR] W rows
  const int tid = threadIdx.x;
  const int ar = tid & (kAcRows - 1), h = tid >> 7;
  const float lam = a.lam;
  const int64_t m = a.m, n = a.n;
  const int64_t a0 = (int64_t)blockIdx.x * kAcRows;
  const int64_t arow = a0 + ar;
  const bool rvalid = arow < m;
  const int64_t c_begin = (int64_t)blockIdx.y * a.split_cols;
  const int64_t c_end = imin64(n, c_begin + a.split_cols);
  for (int idx = tid; idx < kAcRows * R; idx += 256) {
    const int aa = idx / R, k = idx % R;
    const bool ok = a0 + aa < m;
    Ps[aa * LDR + k] = ok ? a.Pb[(a0 + aa) * R + k] : 0.f;
    Wsm[aa * LDR + k] = ok ? a.W[(a0 + aa) * R + k] : 0.f;
  }
  float u[R];
#pragma unroll
  for (int k = 0; k < R; ++k) u[k] = rvalid ? a.U[arow * R + k] : 0.f;
  float dh[KH], dl[KH], wh[KH], wl[KH];
#pragma unroll
  for (int kk = 0; kk < KH; ++kk) { dh[kk] = 0.f; dl[kk] = 0.f; wh[kk] = 0.f; wl[kk] = 0.f; }
  for (int64_t c0 = c_begin; c0 < c_end; c0 += kAcCols) {
    const int cols = (int)imin64((int64_t)kAcCols, c_end - c0);
    __syncthreads();
    for (int idx = tid; idx < kAcCols * kAcRows; idx += 256) {
      const int jj = idx / kAcRows, aa = idx % kAcRows;
      Xt[idx] = (jj < cols && a0 + aa < m) ? a.M[(c0 + jj) * m + a0 + aa] : 0.f;
    }
    for (int idx = tid; idx < kAcCols * R; idx += 256) {
      const int jj = idx / R;
      const bool ok = jj < cols;
      const int64_t gi = (c0 + jj) * R + (idx % R);
      Vs[idx] = ok ? a.V[gi] : 0.f;
      Vns[idx] = ok ? a.Vn[gi] : 0.f;
      Vbs[idx] = ok ? a.Vtot[gi] : 0.f;
    }
    __syncthreads();
    const float* p = Ps + ar * LDR;
    const float* w = Wsm + ar * LDR;
    for (int jj = h; jj < kAcCols; jj += 2) {
      const float* v = Vs + jj * R;
      const float* vn = Vns + jj * R;
      const float* vb = Vbs + jj * R;
      float d = 0.f, xb = 0.f;
#pragma unroll
      for (int k = 0; k < R; ++k) {
        d = fmaf(u[k], v[k], d);
        xb = fmaf(p[k], vn[k], xb);
        xb = fmaf(w[k], vb[k], xb);
      }
      const float r = Xt[jj * kAcRows + ar] - d;
      const float c = fminf(fmaxf(r, -lam), lam);
      Xt[jj * kAcRows + ar] = d + c;
      Dt[jj * kAcRows + ar] = fabsf(r) > lam ? xb : 0.f;
    }
    __syncthreads();
    float dc[KH], wc[KH];
#pragma unroll
    for (int kk = 0; kk < KH; ++kk) { dc[kk] = 0.f; wc[kk] = 0.f; }
    for (int jj = 0; jj < cols; ++jj) {
      const float x = Xt[jj * kAcRows + ar];
      const float dv = Dt[jj * kAcRows + ar];
      const float* v = Vs + jj * R + h * KH;
      const float* vb = Vbs + jj * R + h * KH;
#pragma unroll
      for (int kk = 0; kk < KH; ++kk) {
        dc[kk] = fmaf(dv, v[kk], dc[kk]);
        wc[kk] = fmaf(x, vb[kk], wc[kk]);
      }
    }
#pragma unroll
    for (int kk = 0; kk < KH; ++kk) {
      tsum(dh[kk], dl[kk], dc[kk]);
      tsum(wh[kk], wl[kk], wc[kk]);
    }
  }
  if (rvalid) {
    const int64_t o = ((int64_t)blockIdx.y * m + arow) * R + h * KH;
#pragma unroll
    for (int kk = 0; kk < KH; ++kk) {
      a.part_ud[o + kk] = dh[kk] + dl[kk];
      a.part_wb[o + kk] = wh[kk] + wl[kk];
    }
  }
}

// Adjoint passes over M for R <= 16 (k_adj_a, k_adj_fused): a CTA takes a
// 128-row block and a column split and walks the split in chunks of 32
// columns, brought into shared memory by cp.async in two stages.
constexpr int kAfRows = 128;
constexpr int kAfCols = 32;
constexpr int kAfLdd = kAfCols + 1;   // D tile row stride: conflict-free by row and by column

// Shared-memory layout of the fused adjoint kernels: NV column-vector arrays
// per chunk (pass A: V; passes B and C: V, V', Vbar_tot).
template <int R, int NV>
struct AfCfg {
  static constexpr int MT = kAfCols * kAfRows;   // M tile, column-major [32][128]
  static constexpr int VT = NV * kAfCols * R;    // the column vectors of the chunk
  static constexpr int STAGE = MT + VT;
  static constexpr int DT = kAfRows * kAfLdd;    // D (or X) tile [128][33]
  static constexpr int US = kAfRows * R;         // rows of U (or Pbar) of the block
  static constexpr size_t smem_floats = 2 * (size_t)STAGE + DT + US;
};

// 4- and 16-byte asynchronous copies global -> shared; ok == false zero-fills
// the destination and reads nothing.
__device__ __forceinline__ void af_cp4(float* sdst, const float* gsrc, bool ok) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(sdst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(d), "l"(gsrc),
               "r"(ok ? 4 : 0)
               : "memory");
}
__device__ __forceinline__ void af_cp16(float* sdst, const float* gsrc, bool ok) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(sdst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(gsrc),
               "r"(ok ? 16 : 0)
               : "memory");
}
__device__ __forceinline__ void af_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void af_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// One chunk (columns [c0, c0 + 32) of the split, rows [a0, a0 + 128)) into a
// stage: the M tile and the rows of the NV column-vector arrays; columns at or
// past c_end and rows at or past m read as zero.  Block-wide; one commit group.
template <int R, int NV>
__device__ __forceinline__ void af_load_chunk(float* stage, const float* M, int64_t m,
                                              int64_t a0, int64_t c0, int64_t c_end,
                                              const float* v0, const float* v1,
                                              const float* v2) {
  using C = AfCfg<R, NV>;
  const int tid = threadIdx.x;
  float* Mt = stage;
  float* Vt = stage + C::MT;
  if ((m & 3) == 0) {   // columns of M start on 16-byte boundaries: groups of 4 rows
    for (int idx = tid; idx < C::MT / 4; idx += 256) {
      const int jj = idx / (kAfRows / 4), aq = idx % (kAfRows / 4);
      const int64_t col = c0 + jj, row = a0 + 4 * aq;
      const bool ok = col < c_end && row < m;
      af_cp16(Mt + jj * kAfRows + 4 * aq, ok ? M + col * m + row : M, ok);
    }
  } else {
    for (int idx = tid; idx < C::MT; idx += 256) {
      const int jj = idx / kAfRows, aa = idx % kAfRows;
      const int64_t col = c0 + jj, row = a0 + aa;
      const bool ok = col < c_end && row < m;
      af_cp4(Mt + idx, ok ? M + col * m + row : M, ok);
    }
  }
  for (int idx = tid; idx < NV * kAfCols * (R / 4); idx += 256) {
    const int q = idx / (kAfCols * (R / 4));
    const int rem = idx % (kAfCols * (R / 4));
    const int jj = rem / (R / 4), k4 = rem % (R / 4);
    const int64_t col = c0 + jj;
    const bool ok = col < c_end;
    const float* src = q == 0 ? v0 : q == 1 ? v1 : v2;
    af_cp16(Vt + (q * kAfCols + jj) * R + 4 * k4, ok ? src + col * R + 4 * k4 : src, ok);
  }
  af_commit();
}

// out[rb][col][k] = sum over the block's 128 rows of T[row][col] Y[row][k] for
// the chunk's columns (T: the [128][33] tile, Y: [128][R] rows in shared
// memory).  Warp w takes columns 4w .. 4w + 3; its lanes split the rows and
// the k values and a shuffle tree adds the row groups.  Block-wide (8 warps).
template <int R>
__device__ __forceinline__ void af_colsum(const float* T, const float* Y, float* out, int64_t n,
                                          int64_t rb, int64_t c0, int64_t c_end) {
  constexpr int NKG = R / 4;            // k groups of four
  constexpr int NRQ = 32 / NKG;         // row groups of a warp
  constexpr int RPL = kAfRows / NRQ;    // rows per lane
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int kg = lane % NKG, rq = lane / NKG;
  float acc[4][4];
#pragma unroll
  for (int cc = 0; cc < 4; ++cc)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[cc][q] = 0.f;
#pragma unroll 4
  for (int i = 0; i < RPL; ++i) {
    const int aa = i * NRQ + rq;
    const float4 yy = *reinterpret_cast<const float4*>(Y + aa * R + 4 * kg);
#pragma unroll
    for (int cc = 0; cc < 4; ++cc) {
      const float tv = T[aa * kAfLdd + 4 * warp + cc];
      acc[cc][0] = fmaf(tv, yy.x, acc[cc][0]);
      acc[cc][1] = fmaf(tv, yy.y, acc[cc][1]);
      acc[cc][2] = fmaf(tv, yy.z, acc[cc][2]);
      acc[cc][3] = fmaf(tv, yy.w, acc[cc][3]);
    }
  }
#pragma unroll
  for (int o = NKG; o < 32; o <<= 1)
#pragma unroll
    for (int cc = 0; cc < 4; ++cc)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[cc][q] += __shfl_xor_sync(0xffffffffu, acc[cc][q], o);
  if (rq == 0) {
#pragma unroll
    for (int cc = 0; cc < 4; ++cc) {
      const int64_t col = c0 + 4 * warp + cc;
      if (col < c_end)
        *reinterpret_cast<float4*>(out + (rb * n + col) * R + 4 * kg) =
            make_float4(acc[cc][0], acc[cc][1], acc[cc][2], acc[cc][3]);
    }
  }
}

// Pass A for R <= 16: y1 = X^T Pbar with X = U V^T + clamp(M - U V^T, +-lambda),
// per (128-row block) x (column split) as k_adj_fused; the row block's partial
// of y1 goes to part_vb.  2R flop per element.
template <int R>
__global__ void __launch_bounds__(256, 2) k_adj_a(AdjArgs a) {
  using C = AfCfg<R, 1>;
  static_assert(R % 4 == 0 && R <= 16, "register budget");
  constexpr int HC = kAfCols / 2;
  extern __shared__ __align__(16) float sh[];
  float* Xt = sh + 2 * C::STAGE;
  float* Ps = Xt + C::DT;
  const int tid = threadIdx.x;
  const int ar = tid & (kAfRows - 1), h = tid >> 7;
  const float lam = a.lam;
  const int64_t m = a.m, n = a.n;
  const int64_t a0 = (int64_t)blockIdx.x * kAfRows;
  const int64_t arow = a0 + ar;
  const bool rvalid = arow < m;
  const int64_t c_begin = (int64_t)blockIdx.y * a.split_cols;
  const int64_t c_end = imin64(n, c_begin + a.split_cols);
  const int nchunks = c_end > c_begin ? (int)((c_end - c_begin + kAfCols - 1) / kAfCols) : 0;
  if (nchunks > 0) af_load_chunk<R, 1>(sh, a.M, m, a0, c_begin, c_end, a.V, a.V, a.V);
  float u[R];
#pragma unroll
  for (int k = 0; k < R; ++k) u[k] = rvalid ? a.U[arow * R + k] : 0.f;
  for (int idx = tid; idx < kAfRows * R; idx += 256) {
    const int64_t row = a0 + idx / R;
    Ps[idx] = row < m ? a.Pb[row * R + idx % R] : 0.f;
  }
  for (int c = 0; c < nchunks; ++c) {
    const int64_t c0 = c_begin + (int64_t)c * kAfCols;
    if (c + 1 < nchunks) {
      af_load_chunk<R, 1>(sh + ((c + 1) & 1) * C::STAGE, a.M, m, a0, c0 + kAfCols, c_end, a.V,
                          a.V, a.V);
      af_wait<1>();
    } else {
      af_wait<0>();
    }
    __syncthreads();
    const float* Mt = sh + (c & 1) * C::STAGE;
    const float* Vs = Mt + C::MT;
#pragma unroll 2
    for (int i = 0; i < HC; ++i) {
      const int jj = h * HC + i;
      const float4* v4 = reinterpret_cast<const float4*>(Vs + jj * R);
      float d0 = 0.f, d1 = 0.f;
#pragma unroll
      for (int k4 = 0; k4 < R / 4; ++k4) {
        const float4 v = v4[k4];
        d0 = fmaf(u[4 * k4], v.x, d0);
        d1 = fmaf(u[4 * k4 + 1], v.y, d1);
        d0 = fmaf(u[4 * k4 + 2], v.z, d0);
        d1 = fmaf(u[4 * k4 + 3], v.w, d1);
      }
      const float d = d0 + d1;
      const float r = Mt[jj * kAfRows + ar] - d;
      Xt[ar * kAfLdd + jj] = d + fminf(fmaxf(r, -lam), lam);
    }
    __syncthreads();
    af_colsum<R>(Xt, Ps, a.part_vb, n, blockIdx.x, c0, c_end);
  }
}

// Passes B and C in one kernel (R <= 16): (128-row block) x (column split),
// chunks of 32 columns brought into shared memory by cp.async, two stages, so
// that the next chunk's loads overlap this chunk's arithmetic.  Thread (row
// ar, column half h) forms R, X, Xbar and D of its row for 16 columns of a
// chunk (U, Pbar and W of its row in registers) and accumulates D V and
// X Vbar_tot of its row over the split in registers (FP32).  Then Vbar = D^T U
// of the chunk's columns is summed over the block's rows (af_colsum) into the
// row block's partial in part_vb.  M is read once for both passes, and every
// value of an element is formed once (6R flop per element against 9R).
template <int R>
__global__ void __launch_bounds__(256, 2) k_adj_fused(AdjArgs a) {
  using C = AfCfg<R, 3>;
  static_assert(R % 4 == 0 && R <= 16, "register budget");
  static_assert(kAfRows * (2 * R + 1) <= C::STAGE, "final combine reuses the stages");
  constexpr int HC = kAfCols / 2;       // columns per thread and chunk
  extern __shared__ __align__(16) float sh[];
  float* Dt = sh + 2 * C::STAGE;
  float* Us = Dt + C::DT;
  const int tid = threadIdx.x;
  const int ar = tid & (kAfRows - 1), h = tid >> 7;
  const float lam = a.lam;
  const int64_t m = a.m, n = a.n;
  const int64_t a0 = (int64_t)blockIdx.x * kAfRows;
  const int64_t arow = a0 + ar;
  const bool rvalid = arow < m;
  const int64_t c_begin = (int64_t)blockIdx.y * a.split_cols;
  const int64_t c_end = imin64(n, c_begin + a.split_cols);
  const int nchunks = c_end > c_begin ? (int)((c_end - c_begin + kAfCols - 1) / kAfCols) : 0;
  if (nchunks > 0) af_load_chunk<R, 3>(sh, a.M, m, a0, c_begin, c_end, a.V, a.Vn, a.Vtot);
  float u[R], p[R], w[R];
#pragma unroll
  for (int k = 0; k < R; ++k) {
    u[k] = rvalid ? a.U[arow * R + k] : 0.f;
    p[k] = rvalid ? a.Pb[arow * R + k] : 0.f;
    w[k] = rvalid ? a.W[arow * R + k] : 0.f;
  }
  for (int idx = tid; idx < kAfRows * R; idx += 256) {
    const int64_t row = a0 + idx / R;
    Us[idx] = row < m ? a.U[row * R + idx % R] : 0.f;
  }
  float ud[R], wb[R];
#pragma unroll
  for (int k = 0; k < R; ++k) ud[k] = wb[k] = 0.f;
  float lb_hi = 0.f, lb_lo = 0.f;

  for (int c = 0; c < nchunks; ++c) {
    const int64_t c0 = c_begin + (int64_t)c * kAfCols;
    if (c + 1 < nchunks) {
      af_load_chunk<R, 3>(sh + ((c + 1) & 1) * C::STAGE, a.M, m, a0, c0 + kAfCols, c_end, a.V,
                          a.Vn, a.Vtot);
      af_wait<1>();
    } else {
      af_wait<0>();
    }
    __syncthreads();
    const float* Mt = sh + (c & 1) * C::STAGE;
    const float* Vs = Mt + C::MT;
    const float* Vns = Vs + kAfCols * R;
    const float* Vbs = Vns + kAfCols * R;
    float lb = 0.f;
#pragma unroll 1
    for (int i = 0; i < HC; ++i) {
      const int jj = h * HC + i;
      const float4* v4 = reinterpret_cast<const float4*>(Vs + jj * R);
      const float4* vn4 = reinterpret_cast<const float4*>(Vns + jj * R);
      const float4* vb4 = reinterpret_cast<const float4*>(Vbs + jj * R);
      // two chains each for U V^T and for Pbar V'^T + W Vbar_tot^T
      float d0 = 0.f, d1 = 0.f, x0 = 0.f, x1 = 0.f;
#pragma unroll
      for (int k4 = 0; k4 < R / 4; ++k4) {
        const float4 v = v4[k4], vn = vn4[k4], vb = vb4[k4];
        d0 = fmaf(u[4 * k4], v.x, d0);
        d1 = fmaf(u[4 * k4 + 1], v.y, d1);
        d0 = fmaf(u[4 * k4 + 2], v.z, d0);
        d1 = fmaf(u[4 * k4 + 3], v.w, d1);
        x0 = fmaf(p[4 * k4], vn.x, x0);
        x1 = fmaf(p[4 * k4 + 1], vn.y, x1);
        x0 = fmaf(p[4 * k4 + 2], vn.z, x0);
        x1 = fmaf(p[4 * k4 + 3], vn.w, x1);
        x0 = fmaf(w[4 * k4], vb.x, x0);
        x1 = fmaf(w[4 * k4 + 1], vb.y, x1);
        x0 = fmaf(w[4 * k4 + 2], vb.z, x0);
        x1 = fmaf(w[4 * k4 + 3], vb.w, x1);
      }
      const float d = d0 + d1, xb = x0 + x1;
      const float r = Mt[jj * kAfRows + ar] - d;
      const bool outside = fabsf(r) > lam;
      const float dv = outside ? xb : 0.f;
      const float x = d + fminf(fmaxf(r, -lam), lam);
      lb += outside ? (r > 0.f ? xb : -xb) : 0.f;
      Dt[ar * kAfLdd + jj] = dv;
#pragma unroll
      for (int k4 = 0; k4 < R / 4; ++k4) {
        const float4 v = v4[k4], vb = vb4[k4];
        ud[4 * k4] = fmaf(dv, v.x, ud[4 * k4]);
        ud[4 * k4 + 1] = fmaf(dv, v.y, ud[4 * k4 + 1]);
        ud[4 * k4 + 2] = fmaf(dv, v.z, ud[4 * k4 + 2]);
        ud[4 * k4 + 3] = fmaf(dv, v.w, ud[4 * k4 + 3]);
        wb[4 * k4] = fmaf(x, vb.x, wb[4 * k4]);
        wb[4 * k4 + 1] = fmaf(x, vb.y, wb[4 * k4 + 1]);
        wb[4 * k4 + 2] = fmaf(x, vb.z, wb[4 * k4 + 2]);
        wb[4 * k4 + 3] = fmaf(x, vb.w, wb[4 * k4 + 3]);
      }
    }
    tsum(lb_hi, lb_lo, lb);
    __syncthreads();
    af_colsum<R>(Dt, Us, a.part_vb, n, blockIdx.x, c0, c_end);
  }
  // the two column halves of each row: h = 1 hands its sums to h = 0
  __syncthreads();
  float* comb = sh;   // [128][2R + 1]
  if (h == 1) {
#pragma unroll
    for (int k = 0; k < R; ++k) {
      comb[ar * (2 * R + 1) + k] = ud[k];
      comb[ar * (2 * R + 1) + R + k] = wb[k];
    }
  }
  __syncthreads();
  if (h == 0 && rvalid) {
    const int64_t o = ((int64_t)blockIdx.y * m + arow) * R;
#pragma unroll
    for (int k = 0; k < R; ++k) {
      a.part_ud[o + k] = ud[k] + comb[ar * (2 * R + 1) + k];
      a.part_wb[o + k] = wb[k] + comb[ar * (2 * R + 1) + R + k];
    }
  }
  __shared__ double red[256];
  red[tid] = (double)lb_hi + (double)lb_lo;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (tid < s) red[tid] += red[tid + s];
    __syncthreads();
  }
  if (tid == 0) a.lam_part[(int64_t)blockIdx.y * gridDim.x + blockIdx.x] = red[0];
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
template <int R>
cudaError_t prep_T() {
  cudaError_t e = cudaFuncSetAttribute(k_adj_cols<R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)(AbCfg<R>::smem_floats * 4));
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_adj_rows<R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)(AcCfg<R>::smem_floats * 4));
}

cudaError_t prepare_unrolled_kernels() {
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(k_adj_fused<8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(AfCfg<8, 3>::smem_floats * 4))) != cudaSuccess ||
      (e = cudaFuncSetAttribute(k_adj_fused<16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(AfCfg<16, 3>::smem_floats * 4))) != cudaSuccess ||
      (e = cudaFuncSetAttribute(k_adj_a<8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(AfCfg<8, 1>::smem_floats * 4))) != cudaSuccess ||
      (e = cudaFuncSetAttribute(k_adj_a<16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(AfCfg<16, 1>::smem_floats * 4))) != cudaSuccess)
    return e;
  if ((e = prep_T<8>()) != cudaSuccess) return e;
  if ((e = prep_T<16>()) != cudaSuccess) return e;
  return prep_T<32>();
}

template <int R>
cudaError_t rowlin_T(const RowLinSet& S, cudaStream_t s) {
  size_t smem = 0;
  int64_t rows = 0;
  for (int j = 0; j < S.n; ++j) {
    size_t sj = 0;
    for (int t = 0; t < S.L[j].nmat; ++t) sj += (size_t)S.L[j].cx[t] * R * 4;
    smem = sj > smem ? sj : smem;
    rows = S.L[j].rows > rows ? S.L[j].rows : rows;
  }
  const dim3 grid((unsigned)((rows + 31) / 32), (unsigned)S.n);
  k_rowlin<R><<<grid, 256, smem, s>>>(S);
  return cudaGetLastError();
}

// Independent row jobs (no job reads what another writes) in one launch.
cudaError_t launch_rowlins(int R, std::initializer_list<RowLin> jobs, cudaStream_t s) {
  RowLinSet S{};
  for (const RowLin& L : jobs) {
    if (S.n == 3) return cudaErrorInvalidValue;
    S.L[S.n++] = L;
  }
  switch (R) {
    case 8: return rowlin_T<8>(S, s);
    case 16: return rowlin_T<16>(S, s);
    default: return rowlin_T<32>(S, s);
  }
}

cudaError_t launch_rowlin(int R, const RowLin& L, cudaStream_t s) {
  return launch_rowlins(R, {L}, s);
}

template <int R>
cudaError_t adj_T(const AdjArgs& a, int grid_cols, int n_splits, cudaStream_t s) {
  k_adj_cols<R><<<grid_cols, 256, AbCfg<R>::smem_floats * 4, s>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  dim3 g((unsigned)((a.m + kAcRows - 1) / kAcRows), (unsigned)n_splits);
  k_adj_rows<R><<<g, 256, AcCfg<R>::smem_floats * 4, s>>>(a);
  return cudaGetLastError();
}

// Passes B and C in one launch for R <= 16 (grid: row blocks x column splits).
cudaError_t launch_adjoint_fused(int R, const AdjArgs& a, int n_splits, cudaStream_t s) {
  const dim3 g((unsigned)((a.m + kAfRows - 1) / kAfRows), (unsigned)n_splits);
  if (R == 8)
    k_adj_fused<8><<<g, 256, AfCfg<8, 3>::smem_floats * 4, s>>>(a);
  else
    k_adj_fused<16><<<g, 256, AfCfg<16, 3>::smem_floats * 4, s>>>(a);
  return cudaGetLastError();
}

// Pass A (row-block partials of X^T Pbar into part_vb) for R <= 16.
cudaError_t launch_adjoint_a(int R, const AdjArgs& a, int n_splits, cudaStream_t s) {
  const dim3 g((unsigned)((a.m + kAfRows - 1) / kAfRows), (unsigned)n_splits);
  if (R == 8)
    k_adj_a<8><<<g, 256, AfCfg<8, 1>::smem_floats * 4, s>>>(a);
  else
    k_adj_a<16><<<g, 256, AfCfg<16, 1>::smem_floats * 4, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_adjoint_passes(int R, const AdjArgs& a, int grid_cols, int n_splits,
                                  cudaStream_t s) {
  switch (R) {
    case 8: return adj_T<8>(a, grid_cols, n_splits, s);
    case 16: return adj_T<16>(a, grid_cols, n_splits, s);
    default: return adj_T<32>(a, grid_cols, n_splits, s);
  }
}

cudaError_t launch_small(const SmallArgs& sa, cudaStream_t s) {
  const size_t smem = (size_t)sa.R * sa.R * (3 * sizeof(double) + sizeof(df2));
  k_unrolled_small<<<1, 256, smem, s>>>(sa);
  return cudaGetLastError();
}

}  // namespace
}  // namespace dcf

// ---------------------------------------------------------------------------
// per-handle state of the network
// ---------------------------------------------------------------------------
struct UnrolledState {
  int K = 0;
  // checkpoints
  float* ckU = nullptr;    // (K+1) x m x R
  float* ckV = nullptr;    // (K+1) x n x R
  float* ckUs = nullptr;   // K x m x R   (U* of each step)
  double* ckred = nullptr; // (K+1) x [kNumRed][kSlot]: block j holds the Grams of
                           // (U_j, V_j) the loss needs (RD_UU, RD_VV, RD_UA, RD_VB),
                           // formed by the forward and read again by the reverse
                           // pass; the reverse pass's own Grams of step j-1 go to
                           // the other slots of block j
  // adjoint buffers
  float* Ub[2] = {nullptr, nullptr};
  float* Vb[2] = {nullptr, nullptr};
  float* Pb = nullptr;
  float* Wk = nullptr;
  float* y1 = nullptr;     // X^T Pbar, then reused
  float* Vtot = nullptr;
  float* Wbar = nullptr;
  float* part_ud = nullptr;
  float* part_wb = nullptr;
  float* part_vb = nullptr;  // fused passes B, C: [row block][n][R]
  float* mats = nullptr;
  double* red = nullptr;
  float2* part = nullptr;
  double* sc = nullptr;
  double* loss = nullptr;  // [K]
  double* grads = nullptr; // [3K]
  double* lam_part = nullptr;
  double* hub_part = nullptr;
  dcf::DevState* st = nullptr;
  std::vector<double> lam_k, rho_k, alpha_k, w_k;
  bool have_forward = false;
  bool with_loss = false;
  int n_cols_grid = 0, n_splits = 0;
  bool fused_bc = false;     // passes B and C in one kernel (R <= 16)
  int n_rb = 0;              // its row blocks
  int n_lam = 0;             // lambda_bar partials
  int64_t split_cols = 0;
  int n_gram = 0;
};

namespace dcf {
namespace api {
void free_unrolled(dcf_handle h) {
  // buffers come from dev_alloc and are released with the handle's own list
  delete h->unrolled;
  h->unrolled = nullptr;
}
}  // namespace api
}  // namespace dcf

using namespace dcf;
using namespace dcf::api;

#define UCK(call, what)                                  \
  do {                                                   \
    cudaError_t e_ = (call);                             \
    if (e_ != cudaSuccess) return cuda_fail(h, e_, what); \
  } while (0)

namespace {

dcf_status ensure_unrolled(dcf_handle h, int K) {
  UnrolledState* u = h->unrolled;
  if (u && u->K >= K) return DCF_OK;
  if (!u) {
    UCK(prepare_unrolled_kernels(), "prepare kernels");
    u = new UnrolledState();
    h->unrolled = u;
  }
  const int64_t m = h->m, n = h->n;
  const int R = h->R;
  const size_t mR = (size_t)m * R * 4, nR = (size_t)n * R * 4;
  // launch geometry of the adjoint passes
  const int64_t nstrips = (n + kAbCols - 1) / kAbCols;
  int grid = (int)std::min<int64_t>(nstrips, 2LL * h->num_sms);
  {
    const int64_t waves = (nstrips + grid - 1) / grid;
    grid = (int)((nstrips + waves - 1) / waves);
  }
  const int64_t rb = (m + kAcRows - 1) / kAcRows;
  int64_t splits = std::max<int64_t>(1, (2LL * h->num_sms + rb - 1) / rb);
  splits = std::min<int64_t>(splits, (n + kAcCols - 1) / kAcCols);
  const int64_t split_cols = ((n + splits - 1) / splits + kAcCols - 1) / kAcCols * kAcCols;
  u->n_cols_grid = grid;
  u->split_cols = split_cols;
  u->n_splits = (int)((n + split_cols - 1) / split_cols);
  u->fused_bc = R <= 16;
  u->n_rb = (int)((m + kAfRows - 1) / kAfRows);
  u->n_lam = u->fused_bc ? u->n_rb * u->n_splits : grid;
  u->n_gram = (int)std::min<int64_t>(2LL * h->num_sms, std::max<int64_t>(1, std::max(m, n) / 32));
  // first-time buffers
  if (!u->Ub[0]) {
    for (int i = 0; i < 2; ++i) {
      u->Ub[i] = (float*)dev_alloc(h, mR);
      u->Vb[i] = (float*)dev_alloc(h, nR);
    }
    u->Pb = (float*)dev_alloc(h, mR);
    u->Wk = (float*)dev_alloc(h, mR);
    u->Wbar = (float*)dev_alloc(h, mR);
    u->y1 = (float*)dev_alloc(h, nR);
    u->Vtot = (float*)dev_alloc(h, nR);
    u->part_ud = (float*)dev_alloc(h, mR * u->n_splits);
    u->part_wb = (float*)dev_alloc(h, mR * u->n_splits);
    u->mats = (float*)dev_alloc(h, (size_t)kNumMat * kSlot * 4);
    u->red = (double*)dev_alloc(h, (size_t)kNumRed * kSlot * 8);
    u->part = (float2*)dev_alloc(h, (size_t)kMaxGramJobs * u->n_gram * kSlot * 8);
    u->sc = (double*)dev_alloc(h, (size_t)kNumSc * 8);
    u->lam_part = (double*)dev_alloc(h, (size_t)u->n_lam * 8);
    if (u->fused_bc) {
      u->part_vb = (float*)dev_alloc(h, (size_t)u->n_rb * nR);
      if (!u->part_vb) return fail(h, DCF_ENOMEM, "unrolled network buffers");
    }
    u->hub_part = (double*)dev_alloc(h, (size_t)std::max(grid, h->n_vblocks) * 8);
    u->st = (DevState*)dev_alloc(h, sizeof(DevState));
    if (!u->Ub[0] || !u->Ub[1] || !u->Vb[0] || !u->Vb[1] || !u->Pb || !u->Wk || !u->Wbar ||
        !u->y1 || !u->Vtot || !u->part_ud || !u->part_wb || !u->mats || !u->red || !u->part ||
        !u->sc || !u->lam_part || !u->hub_part || !u->st)
      return fail(h, DCF_ENOMEM, "unrolled network buffers");
    UCK(cudaMemsetAsync(u->mats, 0, (size_t)kNumMat * kSlot * 4, h->stream), "memset");
    UCK(cudaMemsetAsync(u->red, 0, (size_t)kNumRed * kSlot * 8, h->stream), "memset");
    UCK(cudaMemsetAsync(u->st, 0, sizeof(DevState), h->stream), "memset");
  }
  // checkpoints for K steps (grown on demand; the old arrays stay on the
  // handle's list until dcf_destroy)
  u->ckU = (float*)dev_alloc(h, mR * (K + 1));
  u->ckV = (float*)dev_alloc(h, nR * (K + 1));
  u->ckUs = (float*)dev_alloc(h, mR * K);
  u->ckred = (double*)dev_alloc(h, (size_t)(K + 1) * kNumRed * kSlot * 8);
  u->loss = (double*)dev_alloc(h, (size_t)K * 8);
  u->grads = (double*)dev_alloc(h, (size_t)3 * K * 8);
  if (!u->ckU || !u->ckV || !u->ckUs || !u->ckred || !u->loss || !u->grads)
    return fail(h, DCF_ENOMEM, "unrolled checkpoints");
  u->K = K;
  return DCF_OK;
}

// Grams X^T Y (N rows each) summed in FP64 into `out`: up to kMaxGramJobs in
// one launch of partials and one of sums.
struct GSpec {
  const float* X;
  int cx;
  const float* Y;
  int cy;
  int64_t N;
  double* out;
};

cudaError_t grams(dcf_handle h, std::initializer_list<GSpec> list) {
  UnrolledState* u = h->unrolled;
  GramJobs g{};
  for (const GSpec& q : list) {
    GramJob& j = g.j[g.n];
    j.X = q.X;
    j.Y = q.Y;
    j.ldx = j.cx = q.cx;
    j.ldy = j.cy = q.cy;
    j.N = q.N;
    j.nparts = (int)std::min<int64_t>(u->n_gram, std::max<int64_t>(1, q.N / 32));
    j.part = u->part + (size_t)g.n * u->n_gram * kSlot;
    j.out = q.out;
    ++g.n;
  }
  return launch_gram_jobs(g, h->stream);
}

// slot s of block j of the stored Grams
double* ckslot(UnrolledState* u, int j, int s) {
  return u->ckred + ((size_t)j * kNumRed + s) * kSlot;
}

SmallArgs small_args(dcf_handle h, int mode, int K, int step) {
  UnrolledState* u = h->unrolled;
  SmallArgs sa{};
  sa.mode = mode;
  sa.mode2 = -1;
  sa.R = h->R;
  sa.r = h->r;
  sa.k = h->k_truth;
  sa.K = K;
  sa.step = step;
  if (step >= 0 && step < (int)u->lam_k.size()) {
    sa.lam_k = u->lam_k[step];
    sa.rho_k = u->rho_k[step];
    sa.alpha_k = u->alpha_k[step];
    sa.w_k = u->w_k[step];
  }
  sa.red = u->red;
  sa.red_prev = u->red;
  sa.mats = u->mats;
  sa.sc = u->sc;
  sa.loss = u->loss;
  sa.grads = u->grads;
  sa.lam_part = u->lam_part;
  sa.n_lam_part = u->n_lam;
  sa.st = u->st;
  return sa;
}

float* mat(dcf_handle h, int slot) { return h->unrolled->mats + (size_t)slot * kSlot; }

RowLin rowlin(int64_t rows, float* out) {
  RowLin L{};
  L.rows = rows;
  L.out = out;
  return L;
}
void add_mat(RowLin& L, const float* X, int cx, const float* Mt) {
  L.X[L.nmat] = X;
  L.ldx[L.nmat] = cx;
  L.cx[L.nmat] = cx;
  L.Mat[L.nmat] = Mt;
  L.nmat++;
}
void add_term(RowLin& L, const float* Y, float beta, int nparts = 1, int64_t pstride = 0) {
  L.Y[L.nadd] = Y;
  L.beta[L.nadd] = beta;
  L.nparts[L.nadd] = nparts;
  L.pstride[L.nadd] = pstride;
  L.nadd++;
}

dcf_status check_device_status(dcf_handle h, DevState* dev_st) {
  int status = 0;
  UCK(cudaMemcpyAsync(&status, &dev_st->status, sizeof(int), cudaMemcpyDeviceToHost, h->stream),
      "read status");
  UCK(cudaStreamSynchronize(h->stream), "sync");
  if (status == DCF_ENONFINITE) return fail(h, DCF_ENONFINITE, "non-finite value in the network");
  return DCF_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// entry points
// ---------------------------------------------------------------------------
extern "C" dcf_status dcf_unrolled_forward(dcf_handle h, int K, const double* a, const double* b,
                                           const double* c, const double* weights,
                                           double* loss_terms, double* total_loss) {
  if (!h) return DCF_EINVAL;
  if (K < 1 || !a || !b || !c) return fail(h, DCF_EINVAL, "K < 1 or a parameter array is NULL");
  if (h->u_mode != 0) return fail(h, DCF_EINVAL, "the unrolled network uses the exact U-step");
  if (h->R > kUnrolledMaxR) return fail(h, DCF_EINVAL, "the unrolled network supports r <= 32");
  if (h->path == 3 || h->path == 4)
    return fail(h, DCF_EINVAL, "the unrolled network runs on the general and fused paths");
  // the loss (and with it the reverse pass) only when asked for
  const bool with_loss = loss_terms || total_loss;
  if (with_loss && !h->A_truth) return fail(h, DCF_ESTATE, "the loss needs dcf_set_truth first");
  std::vector<double> lam_k(K), rho_k(K), alpha_k(K), w_k(K);
  for (int k = 0; k < K; ++k) {
    lam_k[k] = h->lam * std::exp(a[k]);
    rho_k[k] = h->rho * std::exp(b[k]);
    alpha_k[k] = c[k];
    w_k[k] = weights ? weights[k] : 2.0 * (k + 1) / ((double)K * (K + 1));
    if (!(lam_k[k] > 0) || !(rho_k[k] > 0) || !std::isfinite(lam_k[k]) ||
        !std::isfinite(rho_k[k]) || !std::isfinite(alpha_k[k]) || !std::isfinite(w_k[k]))
      return fail(h, DCF_EINVAL, "non-finite network parameter");
  }
  dcf_status st = begin_work(h);
  if (st != DCF_OK) return st;
  if ((st = ensure_init(h)) != DCF_OK) return st;
  if ((st = ensure_unrolled(h, K)) != DCF_OK) return st;
  UnrolledState* u = h->unrolled;
  u->lam_k = lam_k;
  u->rho_k = rho_k;
  u->alpha_k = alpha_k;
  u->w_k = w_k;
  u->with_loss = with_loss;
  u->have_forward = false;
  if ((st = set_state_fields(h, 0, h->tol)) != DCF_OK) return st;
  cudaStream_t s = h->stream;
  const int64_t m = h->m, n = h->n;
  const int R = h->R, kt = h->k_truth;
  const size_t mR = (size_t)m * R, nR = (size_t)n * R;
  int cur = h->host_iter & 1;
  UCK(cudaMemcpyAsync(u->ckU, h->U[cur], mR * 4, cudaMemcpyDeviceToDevice, s), "checkpoint");
  UCK(cudaMemcpyAsync(u->ckV, h->V[cur], nR * 4, cudaMemcpyDeviceToDevice, s), "checkpoint");
  if (with_loss) {
    // ||A B^T||^2 from A^T A and B^T B; U_0^T U_0 for the reverse pass of step 0
    UCK(grams(h, {{h->A_truth, kt, h->A_truth, kt, m, u->red + (size_t)RD_AA * kSlot},
                  {h->B_truth, kt, h->B_truth, kt, n, u->red + (size_t)RD_BB * kSlot},
                  {h->U[cur], R, h->U[cur], R, m, ckslot(u, 0, RD_UU)}}),
        "grams");
    UCK(launch_small(small_args(h, SM_LOSS_C, K, -1), s), "loss scale");
  }
  const double lam0 = h->lam, rho0 = h->rho;
  const size_t ginv_smem = (size_t)R * R * 16;
  // rho of the (U^T U + rho I)^{-1} held now: the last U-step's tail formed
  // it with the plain rho; a step with another rho refactors first (with the
  // same rho nothing is recomputed, so that the untrained network repeats the
  // plain iteration bit for bit)
  float rho_inv = (float)rho0;
  cudaError_t e = cudaSuccess;
  for (int k = 0; k < K && e == cudaSuccess; ++k) {
    e = [&]() -> cudaError_t {
      cudaError_t e2;
      if ((float)rho_k[k] != rho_inv) {
        k_refactor_ginv<<<1, 256, ginv_smem, s>>>(h->sm, h->st, cur, R, h->r, (float)rho_k[k]);
        if ((e2 = cudaGetLastError()) != cudaSuccess) return e2;
      }
      rho_inv = (float)rho_k[k];   // also what the step's own tail uses
      h->lam = lam_k[k];
      h->rho = rho_k[k];
      h->alpha = (float)alpha_k[k];
      h->ustar_out = u->ckUs + (size_t)k * mR;
      if ((e2 = enqueue_iteration(h, cur, s, nullptr)) != cudaSuccess) return e2;
      h->host_iter++;
      cur ^= 1;
      if ((e2 = cudaMemcpyAsync(u->ckU + (size_t)(k + 1) * mR, h->U[cur], mR * 4,
                                cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
        return e2;
      if ((e2 = cudaMemcpyAsync(u->ckV + (size_t)(k + 1) * nR, h->V[cur], nR * 4,
                                cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
        return e2;
      if (with_loss) {
        SmallArgs sa = small_args(h, SM_LOSS_TERM, K, k);
        sa.red = ckslot(u, k + 1, 0);
        if ((e2 = grams(h, {{h->U[cur], R, h->U[cur], R, m, ckslot(u, k + 1, RD_UU)},
                            {h->V[cur], R, h->V[cur], R, n, ckslot(u, k + 1, RD_VV)},
                            {h->U[cur], R, h->A_truth, kt, m, ckslot(u, k + 1, RD_UA)},
                            {h->V[cur], R, h->B_truth, kt, n, ckslot(u, k + 1, RD_VB)}})) !=
                cudaSuccess ||
            (e2 = launch_small(sa, s)) != cudaSuccess)
          return e2;
      }
      return cudaSuccess;
    }();
  }
  // back to the plain parameters for later dcf_step / dcf_solve calls
  h->lam = lam0;
  h->rho = rho0;
  h->alpha = 1.0f;
  h->ustar_out = nullptr;
  if (e != cudaSuccess) return cuda_fail(h, e, "unrolled forward");
  if (rho_inv != (float)rho0) {
    k_refactor_ginv<<<1, 256, ginv_smem, s>>>(h->sm, h->st, cur, R, h->r, (float)rho0);
    UCK(cudaGetLastError(), "refactor");
  }
  std::vector<double> lk(K, 0.0);
  if (with_loss)
    UCK(cudaMemcpyAsync(lk.data(), u->loss, (size_t)K * 8, cudaMemcpyDeviceToHost, s), "loss");
  DevState ds{};
  if ((st = read_state(h, &ds)) != DCF_OK) return st;   // synchronises
  if (with_loss) {
    double tot = 0;
    for (int k = 0; k < K; ++k) tot += w_k[k] * lk[k];
    if (loss_terms) std::copy(lk.begin(), lk.end(), loss_terms);
    if (total_loss) *total_loss = tot;
  }
  u->have_forward = true;
  return end_work(h);
}

extern "C" dcf_status dcf_unrolled_backward(dcf_handle h, double* grad_a, double* grad_b,
                                            double* grad_c, float* grad_U0,
                                            float* const* grad_V0_i, int where) {
  if (!h) return DCF_EINVAL;
  if (where != 0 && where != 1) return fail(h, DCF_EINVAL, "where must be 0 or 1");
  UnrolledState* u = h->unrolled;
  if (!u || !u->have_forward) return fail(h, DCF_ESTATE, "dcf_unrolled_forward has not run");
  if (!u->with_loss || !h->A_truth)
    return fail(h, DCF_ESTATE, "the backward pass needs the loss (dcf_set_truth before forward)");
  dcf_status st = begin_work(h);
  if (st != DCF_OK) return st;
  cudaStream_t s = h->stream;
  const int K = (int)u->lam_k.size();
  const int64_t m = h->m, n = h->n;
  const int R = h->R, kt = h->k_truth;
  const size_t mR = (size_t)m * R, nR = (size_t)n * R;
  UCK(cudaMemsetAsync(u->st, 0, sizeof(DevState), s), "memset");
  UCK(cudaMemsetAsync(u->Ub[0], 0, mR * 4, s), "memset");
  UCK(cudaMemsetAsync(u->Vb[0], 0, nR * 4, s), "memset");
  UCK(cudaMemsetAsync(u->grads, 0, (size_t)3 * K * 8, s), "memset");
  int ib = 0;   // Ub[ib], Vb[ib] hold Ubar', Vbar' of the step being reversed
  for (int k = K - 1; k >= 0; --k) {
    const float* Uk = u->ckU + (size_t)k * mR;
    const float* Vk = u->ckV + (size_t)k * nR;
    const float* Uk1 = u->ckU + (size_t)(k + 1) * mR;
    const float* Vn = u->ckV + (size_t)(k + 1) * nR;
    const float* Us = u->ckUs + (size_t)k * mR;
    float* Ub = u->Ub[ib];
    float* Vb = u->Vb[ib];
    float* Ub2 = u->Ub[ib ^ 1];
    float* Vb2 = u->Vb[ib ^ 1];
    const float alpha = (float)u->alpha_k[k];
    // loss gradient at (U_{k+1}, V_{k+1}), from the Grams the forward formed
    double* blk = ckslot(u, k + 1, 0);
    auto small = [&](int mode, int mode2 = -1) {
      SmallArgs sa = small_args(h, mode, K, k);
      sa.mode2 = mode2;
      sa.red = blk;
      sa.red_prev = ckslot(u, k, 0);
      return launch_small(sa, s);
    };
    // with G^{-1}, H^{-1} of step k (independent of the loss gradient: one launch)
    UCK(small(SM_LOSSGRAD, SM_RECOMP), "loss grad, recompute");
    {
      RowLin L = rowlin(m, Ub);
      add_mat(L, Uk1, R, mat(h, MT_SVV));
      add_mat(L, h->A_truth, kt, mat(h, MT_SBV));
      add_term(L, Ub, 1.f);
      RowLin L2 = rowlin(n, Vb);
      add_mat(L2, Vn, R, mat(h, MT_SUU));
      add_mat(L2, h->B_truth, kt, mat(h, MT_SAU));
      add_term(L2, Vb, 1.f);
      // W = U_k G^{-1}
      RowLin L3 = rowlin(m, u->Wk);
      add_mat(L3, Uk, R, mat(h, MT_GINV));
      UCK(launch_rowlins(R, {L, L2, L3}, s), "rowlin");
    }
    // relaxation and U* = P H^{-1}
    UCK(grams(h, {{Us, R, Ub, R, m, blk + (size_t)RD_A1 * kSlot},
                  {Uk, R, Ub, R, m, blk + (size_t)RD_A2 * kSlot}}),
        "grams");
    UCK(small(SM_HBAR), "Hbar");
    {
      RowLin L = rowlin(m, u->Pb);
      add_mat(L, Ub, R, mat(h, MT_AHINV));
      UCK(launch_rowlin(R, L, s), "rowlin");
    }
    // pass A: y1 = X^T Pbar (R <= 16: k_adj_a's row-block partials; otherwise
    // the V-step kernel with Pbar in place of W)
    AdjArgs aa{};
    aa.M = h->M;
    aa.m = m;
    aa.n = n;
    aa.lam = (float)u->lam_k[k];
    aa.U = Uk;
    aa.V = Vk;
    aa.Pb = u->Pb;
    aa.W = u->Wk;
    aa.Vn = Vn;
    aa.Vtot = u->Vtot;
    aa.Vbar = Vb2;
    aa.lam_part = u->lam_part;
    aa.part_ud = u->part_ud;
    aa.part_wb = u->part_wb;
    aa.part_vb = u->part_vb;
    aa.split_cols = u->split_cols;
    if (u->fused_bc) {
      UCK(launch_adjoint_a(R, aa, u->n_splits, s), "adjoint pass A");
    } else {
      IterArgs ia{};
      ia.cur = 0;
      ia.M = h->M;
      ia.m = m;
      ia.n = n;
      ia.r = h->r;
      ia.R = R;
      ia.lam = (float)u->lam_k[k];
      ia.rho = (float)u->rho_k[k];
      ia.U[0] = const_cast<float*>(Uk);
      ia.U[1] = const_cast<float*>(Uk);
      ia.V[0] = const_cast<float*>(Vk);
      ia.V[1] = u->y1;
      ia.W = u->Pb;
      ia.part_h = u->hub_part;
      ia.st = u->st;
      ia.alpha = 1.f;
      UCK(launch_pass1(ia, h->n_vblocks, 0, 0, s), "adjoint pass A");
    }
    {
      RowLin L = rowlin(n, u->Vtot);
      add_mat(L, Vn, R, mat(h, MT_HBAR2));
      add_term(L, Vb, 1.f);
      if (u->fused_bc)
        add_term(L, u->part_vb, 1.f, u->n_rb, (int64_t)nR);
      else
        add_term(L, u->y1, 1.f);
      UCK(launch_rowlin(R, L, s), "rowlin");
    }
    // passes B and C
    {
      RowLin L = rowlin(m, u->Wbar);
      add_term(L, u->part_wb, 1.f, u->n_splits, (int64_t)mR);
      if (u->fused_bc) {
        UCK(launch_adjoint_fused(R, aa, u->n_splits, s), "adjoint passes B, C");
        RowLin L2 = rowlin(n, Vb2);
        add_term(L2, u->part_vb, 1.f, u->n_rb, (int64_t)nR);
        UCK(launch_rowlins(R, {L, L2}, s), "rowlin");
      } else {
        UCK(launch_adjoint_passes(R, aa, u->n_cols_grid, u->n_splits, s), "adjoint passes B, C");
        UCK(launch_rowlin(R, L, s), "rowlin");
      }
    }
    UCK(grams(h, {{u->Wk, R, u->Wbar, R, m, blk + (size_t)RD_WWB * kSlot}}), "gram");
    UCK(small(SM_GBAR), "Gbar");
    {
      RowLin L = rowlin(m, Ub2);
      add_mat(L, u->Wbar, R, mat(h, MT_GINV));
      add_mat(L, Uk, R, mat(h, MT_GBAR2));
      add_term(L, Ub, 1.f - alpha);
      add_term(L, u->part_ud, 1.f, u->n_splits, (int64_t)mR);
      UCK(launch_rowlin(R, L, s), "rowlin");
    }
    ib ^= 1;
  }
  std::vector<double> g(3 * (size_t)K);
  UCK(cudaMemcpyAsync(g.data(), u->grads, g.size() * 8, cudaMemcpyDeviceToHost, s), "grads");
  cudaMemcpyKind kind = where == 0 ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  if (grad_U0)
    UCK(cudaMemcpy2DAsync(grad_U0, h->r * 4, u->Ub[ib], R * 4, h->r * 4, m, kind, s), "copy");
  if (grad_V0_i) {
    for (int i = 0; i < h->E; ++i) {
      if (!grad_V0_i[i]) continue;
      UCK(cudaMemcpy2DAsync(grad_V0_i[i], h->r * 4, u->Vb[ib] + h->c_i[i] * R, R * 4, h->r * 4,
                            h->n_i[i], kind, s), "copy");
    }
  }
  if ((st = check_device_status(h, u->st)) != DCF_OK) return st;   // synchronises
  for (int k = 0; k < K; ++k) {
    if (grad_a) grad_a[k] = g[k];
    if (grad_b) grad_b[k] = g[K + k];
    if (grad_c) grad_c[k] = g[2 * K + k];
  }
  return end_work(h);
}
