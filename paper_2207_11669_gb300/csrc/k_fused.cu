// Fused single-pass DCF-PCA iteration on the Blackwell tensor cores.
//
// One iteration needs, for every column j of M (all client blocks at once),
//   R = M - U V^T,   C = clamp(R, -lambda, lambda),   S = R - C   (§2.2 eq. optS)
//   X = M - S = U V^T + C
//   V'[j,:] = X[:,j]^T W,  W = U (U^T U + rho I)^{-1}      (App. B eq. condition1)
//   P = X V'  and  Q = V'^T V'                             (consensus U-step)
// Splitting X = U V^T + C turns the two O(mnr) products that involve X into
//   V' = V Z + C^T W        with Z = U^T W = I - rho (U^T U + rho I)^{-1}
//   P  = U (V^T V') + C V'
// so the dense work is three tensor-core products per strip of 64 columns:
//   GEMM1  D1 = U V_s^T            (3-term fp16 split of U and V: ~FP32 accuracy;
//                                   R feeds the soft-threshold support)
//   GEMM2  Y  = C_s^T [W_hi|W_lo]  (C/lambda in [-1,1] stored once in fp16)
//   GEMM3  P_C += C_s [V'_hi|V'_lo]^T
// and V^T V' (= V_{t-1}^T V_t, also a metric) closes P in the r x r algebra.
//
// Parallel layout: a thread-block cluster of CS CTAs owns whole columns; CTA c
// of a cluster holds rows [256c, 256c+256) of U, W and of every M strip, so
// M is read from HBM once per iteration (TMA, 128x32 fp32 boxes).  The
// column sums of GEMM2 are reduced across the cluster through distributed
// shared memory (reduce-scatter on 8-column chunks, all-gather of the fp16
// V' image), which is the only cross-CTA exchange.  Each cluster walks the
// strips s = cluster_id, cluster_id + #clusters, ...
//
// Every wait on an mbarrier is bounded; on expiry the kernel records
// DCF_ETIMEOUT and runs to completion (all cluster barriers are still
// executed, tensor memory is always released).
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_fp16.h>

#include "dcf.h"
#include "dcf_internal.cuh"
#include "tc_ptx.cuh"

namespace dcf {

constexpr int kFW = 64;          // strip width (columns)
constexpr int kFH = 256;         // rows per CTA (2 row blocks of 128)
constexpr int kSubBytes = 128 * 32 * 4;
constexpr uint32_t kWaitLimit = 1u << 26;


template <int R, int NST>
struct FL {  // shared-memory layout (bytes)
  static constexpr int RING = 0;
  static constexpr int UIMG = RING + NST * kSubBytes;            // 2 terms x 256 x R fp16
  static constexpr int WIMG = UIMG + 2 * kFH * R * 2;            // 2R x 256 fp16
  static constexpr int CBUF = WIMG + 2 * R * kFH * 2;            // 256 x 64 fp16
  static constexpr int VIMG = CBUF + kFH * kFW * 2;              // 2 terms x 64 x R fp16
  static constexpr int PIMG = VIMG + 2 * kFW * R * 2;            // 2R x 64 fp16
  static constexpr int YPART = PIMG + 2 * R * kFW * 2;           // 64 x R fp32
  static constexpr int ZM = YPART + kFW * R * 4;                 // R x R fp32
  static constexpr int VSL = ZM + R * R * 4;                     // 8 x R fp32 (V_s rows)
  static constexpr int VNL = VSL + 8 * R * 4;                    // 8 x R fp32 (V' rows)
  static constexpr int STG = VNL + 8 * R * 4;                    // 2R x 8 fp16 image chunk
  static constexpr int BAR = STG + 2 * R * 8 * 2;                // mbarriers
  static constexpr int NBAR = NST + 4;                           // full[NST], g1, g2, g3, img
  static constexpr int TSLOT = BAR + NBAR * 8;
  static constexpr int RED = TSLOT + 16;                         // 8 doubles
  static constexpr int TOTAL = RED + 8 * 8;
};

__device__ __forceinline__ float pow2_scale_dev(float mx, float target) {
  if (!(mx > 0.f) || !isfinite(mx)) return 1.f;
  int e = (int)floorf(log2f(target / mx));
  e = max(-100, min(100, e));
  return ldexpf(1.f, e);
}

__device__ __forceinline__ void split_h(float x, float s, __half& hi, __half& lo) {
  float xs = x * s;
  hi = __float2half_rn(xs);
  lo = __float2half_rn(xs - __half2float(hi));
}

__device__ __forceinline__ void tsum(float& hi, float& lo, float x) {
  float t = hi + x;
  float bp = t - hi;
  lo += (hi - (t - bp)) + (x - bp);
  hi = t;
}

template <int R, int NST>
__global__ void __launch_bounds__(256, 1)
    k_fused(const __grid_constant__ CUtensorMap tmap, const FusedArgs a) {
  using L = FL<R, NST>;
  if (a.st->stop) return;  // uniform over the grid
  extern __shared__ __align__(1024) uint8_t smem[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t crank = tc::cluster_rank();
  const int cid = blockIdx.x / a.cs;
  const int slab = (int)(blockIdx.x % a.cs);   // == crank
  const int64_t row0 = (int64_t)slab * kFH;
  const uint32_t sbase = tc::smem_u32(smem);
  const uint32_t bar = sbase + L::BAR;
  auto full_bar = [&](int i) { return bar + 8u * i; };
  const uint32_t g1_bar = bar + 8u * NST, g2_bar = g1_bar + 8, g3_bar = g2_bar + 8,
                 img_bar = g3_bar + 8;
  float* ypart = reinterpret_cast<float*>(smem + L::YPART);
  float* zm = reinterpret_cast<float*>(smem + L::ZM);
  float* vsl = reinterpret_cast<float*>(smem + L::VSL);
  float* vnl = reinterpret_cast<float*>(smem + L::VNL);
  int err = 0;

  // ---- set-up -------------------------------------------------------------
  if (warp == 0) {
    tc::tmem_alloc(sbase + L::TSLOT, 512);
    tc::tmem_relinquish();
  }
  if (tid == 0) {
    for (int i = 0; i < L::NBAR; ++i) tc::mbar_init(bar + 8u * i, 1);
    tc::fence_mbar_init();
    tc::prefetch_tmap(&tmap);
  }
  for (int i = tid; i < R * R; i += 256) zm[i] = a.zmat[i];
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tbase = *reinterpret_cast<volatile uint32_t*>(smem + L::TSLOT);
  const uint32_t d1 = tbase, d2 = tbase + 128, d3 = tbase + 256;
  const float s_u = a.scales[2 * slab], s_w = a.scales[2 * slab + 1];
  const float s_v = a.scales[2 * a.nslabs];
  const float inv_uv = 1.f / (s_u * s_v);
  const float inv_lam = 1.f / a.lam;
  const float y_scale = a.lam / s_w;
  const int64_t nstrips = (a.n + kFW - 1) / kFW;
  const int my_strips = cid < nstrips ? (int)((nstrips - 1 - cid) / a.nclusters + 1) : 0;
  const int total_sub = my_strips * 4;

  auto issue_tma = [&](int g) {
    const int ls = g >> 2, sub = g & 3, b = sub >> 1, q = sub & 1;
    const int64_t s = cid + (int64_t)ls * a.nclusters;
    const int slot = g % NST;
    tc::mbar_arrive_expect_tx(full_bar(slot), kSubBytes);
    tc::tma_load_2d(sbase + L::RING + slot * kSubBytes, &tmap, (int)(row0 + 128 * b),
                    (int)(s * kFW + 32 * q), full_bar(slot));
  };
  if (tid == 0) {
    // U and W images of this row slab (prepared by k_fused_prep)
    const uint8_t* src = a.img + (size_t)slab * (4 * kFH * R * 2);
    tc::mbar_arrive_expect_tx(img_bar, 4 * kFH * R * 2);
    tc::bulk_load(sbase + L::UIMG, src, 2 * kFH * R * 2, img_bar);
    tc::bulk_load(sbase + L::WIMG, src + 2 * kFH * R * 2, 2 * kFH * R * 2, img_bar);
    for (int g = 0; g < NST && g < total_sub; ++g) issue_tma(g);
  }
  tc::cluster_sync();  // peers' barriers initialised before any remote access
  if (!tc::mbar_wait(img_bar, 0, kWaitLimit)) err = 1;

  constexpr int NE = (R * R + 255) / 256;   // Q/X_v entries per thread
  float q_hi[NE], q_lo[NE], x_hi[NE], x_lo[NE];
#pragma unroll
  for (int i = 0; i < NE; ++i) { q_hi[i] = q_lo[i] = x_hi[i] = x_lo[i] = 0.f; }
  float hub_hi = 0.f, hub_lo = 0.f, vmax = 0.f;
  const uint32_t idesc1 = tc::idesc_f16(128, kFW, 0, 0);
  const uint32_t idesc2 = tc::idesc_f16(64, 2 * R, 1, 0);
  const uint32_t idesc3 = tc::idesc_f16(128, 2 * R, 0, 0);
  constexpr uint32_t SB_R = (R / 8) * 128;    // M/N-direction core stride of K=R images

  for (int ls = 0; ls < my_strips; ++ls) {
    const int64_t col0 = (cid + (int64_t)ls * a.nclusters) * kFW;
    const uint32_t par = ls & 1;
    // (1) fp16 hi/lo image of V_s (B operand of GEMM1; GEMM1 of the previous
    //     strip completed before its epilogue, so the buffer is free)
    for (int idx = tid; idx < kFW * R; idx += 256) {
      const int j = idx / R, k = idx % R;
      const float v = col0 + j < a.n ? a.Vold[(col0 + j) * R + k] : 0.f;
      __half hi, lo;
      split_h(v, s_v, hi, lo);
      const int off = (j >> 3) * SB_R + (k >> 3) * 128 + (j & 7) * 16 + (k & 7) * 2;
      *reinterpret_cast<__half*>(smem + L::VIMG + off) = hi;
      *reinterpret_cast<__half*>(smem + L::VIMG + kFW * R * 2 + off) = lo;
    }
    tc::fence_proxy_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    // (2) GEMM1: D1_b = U_b V_s^T with terms (hi,hi), (hi,lo), (lo,hi)
    if (tid == 0) {
#pragma unroll
      for (int b = 0; b < 2; ++b) {
        int first = 1;
#pragma unroll
        for (int t = 0; t < 3; ++t) {
          const int tu = t == 2 ? 1 : 0, tv = t == 1 ? 1 : 0;
#pragma unroll
          for (int kk = 0; kk < R / 16; ++kk) {
            const uint64_t ad = tc::smem_desc(
                sbase + L::UIMG + tu * (kFH * R * 2) + b * 16 * SB_R + kk * 256, 128, SB_R);
            const uint64_t bd =
                tc::smem_desc(sbase + L::VIMG + tv * (kFW * R * 2) + kk * 256, 128, SB_R);
            tc::mma_ss(d1 + b * kFW, ad, bd, idesc1, first ? 0u : 1u);
            first = 0;
          }
        }
      }
      tc::mma_commit(g1_bar);
    }
    __syncwarp();
    if (!tc::mbar_wait(g1_bar, par, kWaitLimit)) err = 1;
    if (ls > 0 && !tc::mbar_wait(g3_bar, par ^ 1, kWaitLimit)) err = 1;  // C buffer free
    tc::fence_after_sync();
    // (3) epilogue: R, C/lambda (fp16), Huber; warp -> (row block, lane quarter)
    {
      const int b = warp >> 2, quarter = warp & 3;
      const int al = quarter * 32 + lane;      // row inside the block
      const int arow = b * 128 + al;           // row inside the slab
      float hub = 0.f;
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const int g = ls * 4 + b * 2 + q;
        const int slot = g % NST;
        if (!tc::mbar_wait(full_bar(slot), (uint32_t)((g / NST) & 1), kWaitLimit)) err = 1;
        float dv[32];
        const uint32_t ta = d1 + ((uint32_t)(quarter * 32) << 16) + b * kFW + q * 32;
        tc::tmem_ld16(ta, dv);
        tc::tmem_ld16(ta + 16, dv + 16);
        tc::tmem_ld_wait();
        const float* msub = reinterpret_cast<const float*>(smem + L::RING + slot * kSubBytes);
        uint32_t packed[16];
#pragma unroll
        for (int jj = 0; jj < 32; jj += 2) {
          float c2[2];
#pragma unroll
          for (int u = 0; u < 2; ++u) {
            const float mv = msub[(jj + u) * 128 + al];
            const float rn = (mv - dv[jj + u] * inv_uv) * inv_lam;   // R / lambda
            const float c = fminf(fmaxf(rn, -1.f), 1.f);             // C / lambda
            hub = fmaf(c, rn - 0.5f * c, hub);                       // H(R) / lambda^2
            c2[u] = c;
          }
          __half2 h2 = __floats2half2_rn(c2[0], c2[1]);
          packed[jj / 2] = *reinterpret_cast<uint32_t*>(&h2);
        }
#pragma unroll
        for (int ch = 0; ch < 4; ++ch) {
          const int j8 = (q * 32 + ch * 8) >> 3;
          const int off = j8 * (kFH * 16) + (arow >> 3) * 128 + (arow & 7) * 16;
          *reinterpret_cast<uint4*>(smem + L::CBUF + off) =
              make_uint4(packed[4 * ch], packed[4 * ch + 1], packed[4 * ch + 2], packed[4 * ch + 3]);
        }
      }
      tsum(hub_hi, hub_lo, hub);
    }
    tc::fence_proxy_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    // (4) refill the ring; GEMM2: Y = C_s^T [W_hi | W_lo] over the 256 rows
    if (tid == 0) {
      for (int g = ls * 4 + NST; g < ls * 4 + NST + 4 && g < total_sub; ++g) issue_tma(g);
#pragma unroll
      for (int kk = 0; kk < kFH / 16; ++kk) {
        const uint64_t ad = tc::smem_desc(sbase + L::CBUF + kk * 256, 128, kFH * 16);
        const uint64_t bd = tc::smem_desc(sbase + L::WIMG + kk * 256, 128, kFH * 16);
        tc::mma_ss(d2, ad, bd, idesc2, kk > 0 ? 1u : 0u);
      }
      tc::mma_commit(g2_bar);
    }
    __syncwarp();
    if (!tc::mbar_wait(g2_bar, par, kWaitLimit)) err = 1;
    tc::fence_after_sync();
    // (5) partial column sums: rows j = 16*quarter + lane (lane < 16) of the M=64 result
    if (warp < 4) {
      float yv[2 * R];
#pragma unroll
      for (int c = 0; c < 2 * R; c += 16)
        tc::tmem_ld16(d2 + ((uint32_t)(warp * 32) << 16) + c, yv + c);
      tc::tmem_ld_wait();
      if (lane < 16) {
        const int j = warp * 16 + lane;
#pragma unroll
        for (int k = 0; k < R; ++k) ypart[j * R + k] = (yv[k] + yv[R + k]) * y_scale;
      }
    }
    tc::fence_before_sync();
    tc::cluster_sync();  // #1: every CTA's partial column sums are visible
    tc::fence_after_sync();
    // (6) reduce-scatter over 8-column chunks, V' = V_s Z + Y, all-gather of the fp16 image
    for (int cc = (int)crank; cc < kFW / 8; cc += a.cs) {
      const int jl = tid / R, k = tid % R;  // active for tid < 8R
      if (tid < 8 * R) {
        const int64_t col = col0 + cc * 8 + jl;
        vsl[jl * R + k] = col < a.n ? a.Vold[col * R + k] : 0.f;
      }
      __syncthreads();
      if (tid < 8 * R) {
        const int j = cc * 8 + jl;
        const int64_t col = col0 + j;
        float y = 0.f;
        const uint32_t yaddr = sbase + L::YPART + (uint32_t)(j * R + k) * 4;
        for (int p = 0; p < a.cs; ++p) y += tc::ld_cluster_f32(tc::map_cluster(yaddr, p));
#pragma unroll 8
        for (int l = 0; l < R; ++l) y = fmaf(vsl[jl * R + l], zm[l * R + k], y);
        const float v = col < a.n ? y : 0.f;
        if (col < a.n) a.Vnew[col * R + k] = v;
        vnl[jl * R + k] = v;
        vmax = fmaxf(vmax, fabsf(v));
        __half hi, lo;
        split_h(v, s_v, hi, lo);
        // chunk image: entry (n, jl) at (n/8)*128 + (n%8)*16 + jl*2, n = k (hi) or R + k (lo)
        *reinterpret_cast<__half*>(smem + L::STG + (k >> 3) * 128 + (k & 7) * 16 + jl * 2) = hi;
        *reinterpret_cast<__half*>(smem + L::STG + ((R + k) >> 3) * 128 + (k & 7) * 16 + jl * 2) =
            lo;
      }
      __syncthreads();
      // Q_t and V_{t-1}^T V_t contributions of the 8 columns
#pragma unroll
      for (int i = 0; i < NE; ++i) {
        const int e = tid + 256 * i;
        if (e < R * R) {
          const int k1 = e / R, k2 = e % R;
          float qa = 0.f, xa = 0.f;
#pragma unroll
          for (int jj = 0; jj < 8; ++jj) {
            qa = fmaf(vnl[jj * R + k1], vnl[jj * R + k2], qa);
            xa = fmaf(vsl[jj * R + k1], vnl[jj * R + k2], xa);
          }
          tsum(q_hi[i], q_lo[i], qa);
          tsum(x_hi[i], x_lo[i], xa);
        }
      }
      // all-gather: 2R/8 groups of 128 contiguous bytes into every CTA's V' image
      constexpr int NPIECE = (2 * R / 8) * 8;   // 16-byte pieces per destination
      for (int idx = tid; idx < a.cs * NPIECE; idx += 256) {
        const int p = idx / NPIECE, pc = idx % NPIECE;
        const int g8 = pc >> 3, w16 = pc & 7;
        const uint4 v = *reinterpret_cast<const uint4*>(smem + L::STG + g8 * 128 + w16 * 16);
        const uint32_t dst = sbase + L::PIMG + g8 * (kFW / 8) * 128 + cc * 128 + w16 * 16;
        tc::st_cluster_u32x4(tc::map_cluster(dst, p), v);
      }
      __syncthreads();
    }
    asm volatile("fence.proxy.async;" ::: "memory");
    tc::fence_before_sync();
    tc::cluster_sync();  // #2: the V' image of the strip is complete in every CTA
    tc::fence_after_sync();
    // (7) GEMM3: P_C += C_s [V'_hi | V'_lo]^T for both row blocks
    if (tid == 0) {
      asm volatile("fence.proxy.async;" ::: "memory");
#pragma unroll
      for (int b = 0; b < 2; ++b) {
#pragma unroll
        for (int kk = 0; kk < kFW / 16; ++kk) {
          const uint64_t ad =
              tc::smem_desc(sbase + L::CBUF + b * 2048 + kk * 2 * (kFH * 16), kFH * 16, 128);
          const uint64_t bd =
              tc::smem_desc(sbase + L::PIMG + kk * 256, 128, (kFW / 8) * 128);
          tc::mma_ss(d3 + b * 2 * R, ad, bd, idesc3, (ls > 0 || kk > 0) ? 1u : 0u);
        }
      }
      tc::mma_commit(g3_bar);
    }
    __syncwarp();
  }

  // ---- P partial of this cluster's columns ---------------------------------
  if (my_strips > 0 && !tc::mbar_wait(g3_bar, (uint32_t)((my_strips - 1) & 1), kWaitLimit))
    err = 1;
  tc::fence_after_sync();
  {
    const int b = warp >> 2, quarter = warp & 3;
    const int al = quarter * 32 + lane;
    const int64_t arow = row0 + b * 128 + al;
    float pv[2 * R];
#pragma unroll
    for (int c = 0; c < 2 * R; c += 16)
      tc::tmem_ld16(d3 + ((uint32_t)(quarter * 32) << 16) + b * 2 * R + c, pv + c);
    tc::tmem_ld_wait();
    if (arow < a.m) {
      const float ps = a.lam / s_v;
      float* out = a.part_p + ((int64_t)cid * a.m + arow) * R;
#pragma unroll
      for (int k = 0; k < R; ++k) out[k] = my_strips > 0 ? (pv[k] + pv[R + k]) * ps : 0.f;
    }
  }
  // ---- per-CTA partials ----------------------------------------------------------
#pragma unroll
  for (int i = 0; i < NE; ++i) {
    const int e = tid + 256 * i;
    if (e < R * R) {
      a.part_q[(int64_t)blockIdx.x * R * R + e] = (double)q_hi[i] + (double)q_lo[i];
      a.part_xv[(int64_t)blockIdx.x * R * R + e] = (double)x_hi[i] + (double)x_lo[i];
    }
  }
  double* red = reinterpret_cast<double*>(smem + L::RED);
  {
    double hsum = ((double)hub_hi + (double)hub_lo) * (double)a.lam * (double)a.lam;
    for (int o = 16; o > 0; o >>= 1) hsum += __shfl_xor_sync(0xffffffffu, hsum, o);
    for (int o = 16; o > 0; o >>= 1) vmax = fmaxf(vmax, __shfl_xor_sync(0xffffffffu, vmax, o));
    if (lane == 0) red[warp] = hsum;
    if (lane == 0 && vmax > 0.f) atomicMax(a.vmax_out, __float_as_uint(vmax));
  }
  if (err) atomicExch(a.err, DCF_ETIMEOUT);
  tc::fence_before_sync();
  __syncthreads();
  if (tid == 0) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += red[w];
    a.part_h[blockIdx.x] = t;
  }
  if (warp == 0) tc::tmem_dealloc(tbase, 512);
  tc::cluster_sync();  // no CTA leaves while a peer may still address its shared memory
}

// ---------------------------------------------------------------------------
// Per-iteration preparation: W rows, fp16 hi/lo images of U and W per 256-row
// slab with power-of-two scales, Z = I - rho G^{-1}, and the V scale.
// ---------------------------------------------------------------------------
template <int R>
__global__ void __launch_bounds__(256) k_fused_prep(const float* __restrict__ U,
                                                    const Smalls* sm, const DevState* st,
                                                    int64_t m, int nslabs, float rho,
                                                    const unsigned int* vmax_in,
                                                    unsigned int* vmax_reset, uint8_t* img,
                                                    float* scales, float* zmat) {
  if (st->stop) return;
  __shared__ float gi[R * R];
  __shared__ __align__(16) uint8_t wst[2 * R * kFH * 2];
  __shared__ float red[2][8];
  const int tid = threadIdx.x, slab = blockIdx.x;
  for (int i = tid; i < R * R; i += 256) gi[i] = sm->ginv32[i];
  __syncthreads();
  const int64_t arow = (int64_t)slab * kFH + tid;
  float u[R], w[R];
  float umax = 0.f, wmax = 0.f;
#pragma unroll
  for (int k = 0; k < R; ++k) u[k] = arow < m ? U[arow * R + k] : 0.f;
#pragma unroll
  for (int l = 0; l < R; ++l) {
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < R; ++k) s = fmaf(u[k], gi[k * R + l], s);
    w[l] = s;
    wmax = fmaxf(wmax, fabsf(s));
    umax = fmaxf(umax, fabsf(u[l]));
  }
  for (int o = 16; o > 0; o >>= 1) {
    umax = fmaxf(umax, __shfl_xor_sync(0xffffffffu, umax, o));
    wmax = fmaxf(wmax, __shfl_xor_sync(0xffffffffu, wmax, o));
  }
  if ((tid & 31) == 0) { red[0][tid >> 5] = umax; red[1][tid >> 5] = wmax; }
  __syncthreads();
  umax = 0.f;
  wmax = 0.f;
  for (int i = 0; i < 8; ++i) { umax = fmaxf(umax, red[0][i]); wmax = fmaxf(wmax, red[1][i]); }
  const float s_u = pow2_scale_dev(umax, 16384.f), s_w = pow2_scale_dev(wmax, 16384.f);
  uint8_t* dst = img + (size_t)slab * (4 * kFH * R * 2);
  constexpr uint32_t SB_R = (R / 8) * 128;
  // U image: term t, row a, k -> t*(256*R*2) + (a/8)*SB_R + (k/8)*128 + (a%8)*16 + (k%8)*2
#pragma unroll
  for (int k8 = 0; k8 < R / 8; ++k8) {
    uint32_t ph[4], pl[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      __half h0, l0, h1, l1;
      split_h(u[k8 * 8 + 2 * i], s_u, h0, l0);
      split_h(u[k8 * 8 + 2 * i + 1], s_u, h1, l1);
      __half2 hh = __halves2half2(h0, h1), ll = __halves2half2(l0, l1);
      ph[i] = *reinterpret_cast<uint32_t*>(&hh);
      pl[i] = *reinterpret_cast<uint32_t*>(&ll);
    }
    const int off = (tid >> 3) * SB_R + k8 * 128 + (tid & 7) * 16;
    *reinterpret_cast<uint4*>(dst + off) = make_uint4(ph[0], ph[1], ph[2], ph[3]);
    *reinterpret_cast<uint4*>(dst + kFH * R * 2 + off) = make_uint4(pl[0], pl[1], pl[2], pl[3]);
  }
  // W image: entry (n, a), n < R -> W_hi[a, n], n >= R -> W_lo[a, n-R]:
  //   (n/8)*(256*16) + (a/8)*128 + (n%8)*16 + (a%8)*2
#pragma unroll
  for (int k = 0; k < R; ++k) {
    __half hi, lo;
    split_h(w[k], s_w, hi, lo);
    const int base = (tid >> 3) * 128 + (tid & 7) * 2;
    *reinterpret_cast<__half*>(wst + (k >> 3) * (kFH * 16) + (k & 7) * 16 + base) = hi;
    *reinterpret_cast<__half*>(wst + ((R + k) >> 3) * (kFH * 16) + (k & 7) * 16 + base) = lo;
  }
  __syncthreads();
  for (int i = tid; i < (2 * R * kFH * 2) / 16; i += 256)
    reinterpret_cast<uint4*>(dst + 2 * kFH * R * 2)[i] = reinterpret_cast<const uint4*>(wst)[i];
  if (tid == 0) {
    scales[2 * slab] = s_u;
    scales[2 * slab + 1] = s_w;
  }
  if (slab == 0) {
    for (int i = tid; i < R * R; i += 256)
      zmat[i] = ((i / R) == (i % R) ? 1.f : 0.f) - rho * gi[i];
    if (tid == 0) {
      const float vm = __uint_as_float(*vmax_in);
      scales[2 * nslabs] = pow2_scale_dev(vm, 1024.f);
      *vmax_reset = 0u;
    }
  }
}

__global__ void k_absmax(const float* x, int64_t count, unsigned int* out) {
  float mx = 0.f;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x)
    mx = fmaxf(mx, fabsf(x[i]));
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0 && mx > 0.f) atomicMax(out, __float_as_uint(mx));
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
constexpr int kNST32 = 6;
constexpr int kNST16 = 8;

template <int R, int NST>
static size_t fused_smem() {
  return FL<R, NST>::TOTAL;
}

template <int R, int NST>
static cudaError_t prep_attr() {
  cudaError_t e = cudaFuncSetAttribute(k_fused<R, NST>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)fused_smem<R, NST>());
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_fused<R, NST>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
}

cudaError_t fused_prepare(int R) {
  return R == 16 ? prep_attr<16, kNST16>() : prep_attr<32, kNST32>();
}

template <int R, int NST>
static int max_clusters_T(int cs) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(cs, 1, 1);
  cfg.blockDim = dim3(256, 1, 1);
  cfg.dynamicSmemBytes = fused_smem<R, NST>();
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = cs;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, (void*)k_fused<R, NST>, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

int fused_max_clusters(int R, int cs) {
  return R == 16 ? max_clusters_T<16, kNST16>(cs) : max_clusters_T<32, kNST32>(cs);
}

static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
  }
  return fn;
}

// 2-D tensor map over column-major M (dim 0 = rows, contiguous), 128 x 32 boxes.
int fused_make_tmap(void* tmap_out, const float* M, int64_t m, int64_t n) {
  auto fn = encode_fn();
  if (!fn) return -1;
  cuuint64_t dims[2] = {(cuuint64_t)m, (cuuint64_t)n};
  cuuint64_t strides[1] = {(cuuint64_t)m * sizeof(float)};
  cuuint32_t box[2] = {128, 32};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(reinterpret_cast<CUtensorMap*>(tmap_out), CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
                  const_cast<float*>(M), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? 0 : (int)r;
}

cudaError_t launch_fused_prep(int R, const float* U, const Smalls* sm, const DevState* st,
                              int64_t m, int nslabs, float rho, const unsigned int* vmax_in,
                              unsigned int* vmax_reset, uint8_t* img, float* scales, float* zmat,
                              cudaStream_t s) {
  if (R == 16)
    k_fused_prep<16><<<nslabs, 256, 0, s>>>(U, sm, st, m, nslabs, rho, vmax_in, vmax_reset, img,
                                            scales, zmat);
  else
    k_fused_prep<32><<<nslabs, 256, 0, s>>>(U, sm, st, m, nslabs, rho, vmax_in, vmax_reset, img,
                                            scales, zmat);
  return cudaGetLastError();
}

template <int R, int NST>
static cudaError_t launch_fused_T(const void* tmap, const FusedArgs& fa, cudaStream_t s) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(fa.cs * fa.nclusters, 1, 1);
  cfg.blockDim = dim3(256, 1, 1);
  cfg.dynamicSmemBytes = fused_smem<R, NST>();
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = fa.cs;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  const CUtensorMap* tm = reinterpret_cast<const CUtensorMap*>(tmap);
  return cudaLaunchKernelEx(&cfg, k_fused<R, NST>, *tm, fa);
}

cudaError_t launch_fused(int R, const void* tmap, const FusedArgs& fa, cudaStream_t s) {
  return R == 16 ? launch_fused_T<16, kNST16>(tmap, fa, s) : launch_fused_T<32, kNST32>(tmap, fa, s);
}

cudaError_t launch_absmax(const float* x, int64_t count, unsigned int* out, cudaStream_t s) {
  int64_t blocks = (count + 255) / 256;
  if (blocks > 1024) blocks = 1024;
  if (blocks < 1) blocks = 1;
  k_absmax<<<(unsigned)blocks, 256, 0, s>>>(x, count, out);
  return cudaGetLastError();
}

}  // namespace dcf
