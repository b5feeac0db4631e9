// Two-pass tensor-core DCF-PCA iteration, for problems the single-pass kernel
// does not take: more than 16 slabs of 256 rows (its cluster would not fit on
// the GPU), or r > 32 (its tensor memory would not hold R = 64).
//
// The arithmetic is the single-pass kernel's (§2.2 S-step, App. B V-step, the
// consensus U-step), split at the one point where a whole column must be
// reduced over all m rows before it can be used:
//   pass A   per 256-row slab and 64-column strip
//              GEMM1  D1 = U V_s^T  (3-term fp16 split), S-step epilogue:
//                     C/lambda = clamp(R/lambda, -1, 1) into a C tile, Huber
//              GEMM2  Y_slab = C^T W_hi + C^T W_lo  -> global partials
//   reduce   V' = V_old Z + sum over slabs of Y_slab, max |V'|
//   pass B   per slab and strip: GEMM1 and the epilogue again (C is not
//            stored: recomputing it costs one more read of M, storing it would
//            cost a write and a read of half that size plus the partial sums)
//              GEMM3  P_C += C V'_hi^T + C V'_lo^T   (tensor memory, per CTA)
// M is read twice per iteration (8 B per element) instead of once; there is
// no cross-CTA exchange, so no CTA waits on another.  Each CTA owns one slab
// (its U image in tensor memory, its W image in shared memory) and walks the
// strips g, g + G, g + 2G, ... of its strip group g; P partials are per strip
// group, column sums per slab.
//
// Every wait on an mbarrier is bounded.  The first wait that expires raises a
// CTA-wide abort flag; from then on no role issues another MMA, tcgen05.ld,
// TMA load or shared-memory write that the expired wait was guarding, and
// every role leaves its loop.  Before tensor memory is released the MMA
// issuer's final commit and the TMA loads still in flight are drained with
// bounded waits; if even that fails the tensor memory is left allocated.  The
// kernel records DCF_ETIMEOUT.
#include <cuda.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "dcf.h"
#include "dcf_internal.cuh"
#include "tc_ptx.cuh"

namespace dcf {

namespace {

constexpr int kTW = 64;            // strip width (columns)
constexpr int kTH = 256;           // rows per CTA (2 row blocks of 128)
constexpr int kTSubCols = 16;      // M sub-tile: 256 rows x 16 columns
constexpr int kTSubBytes = kTH * kTSubCols * 4;
constexpr int kTThreads = 512;     // 16 warps
constexpr int kTNC = 2;            // C tiles in shared memory
constexpr uint64_t kTDeadlineNs = 2000000000ull;

__device__ __forceinline__ float tpow2_scale(float mx, float target) {
  if (!(mx > 0.f) || !isfinite(mx)) return 1.f;
  int e = (int)floorf(log2f(target / mx));
  e = max(-100, min(100, e));
  return ldexpf(1.f, e);
}

__device__ __forceinline__ void tsplit(float x, float s, __half& hi, __half& lo) {
  const float xs = x * s;
  hi = __float2half_rn(xs);
  lo = __float2half_rn(xs - __half2float(hi));
}

__device__ __forceinline__ void ttwo_sum(float& hi, float& lo, float x) {
  const float t = hi + x;
  const float bp = t - hi;
  lo += (hi - (t - bp)) + (x - bp);
  hi = t;
}

// Shared-memory layout (bytes) of pass A (kB = false) or pass B (kB = true).
// kPair (pass A): the CTAs of a two-CTA cluster (two slabs) add their column
// sums before writing them: RECV holds the partner's half of a strip, two
// slots.
template <int R, int NST, bool kB, bool kPair = false>
struct TL {
  static constexpr int RING = 0;                                   // NST M sub-tiles
  static constexpr int WIMG = RING + NST * kTSubBytes;             // pass A: 2R x 256 fp16
  static constexpr int WBYTES = kB ? 0 : 2 * R * kTH * 2;
  static constexpr int CBYTES = kTH * kTW * 2;                     // one C tile (fp16)
  static constexpr int CBUF = WIMG + WBYTES;                       // kTNC C tiles
  static constexpr int VBYTES = 2 * kTW * R * 2;                   // V_old image (2 terms)
  static constexpr int VIMG = CBUF + kTNC * CBYTES;
  static constexpr int PBYTES = 2 * R * kTW * 2;                   // one V' image (2 terms)
  static constexpr int PIMG = VIMG + VBYTES;                       // pass B: 2 V' images
  static constexpr int RSLOT = kTW / 2 * R * 4;                    // half a strip's sums
  static constexpr int RECV = PIMG + (kB ? 2 * PBYTES : 0);        // kPair: 2 slots
  static constexpr int BAR = RECV + (kPair ? 2 * RSLOT : 0);
  // full/empty NST each; vfull, vempty; d1full, d1empty 2 each; cfull, cempty
  // kTNC each; d2full, d2empty (pass A) or pvfull, pvempty (pass B) 2 each;
  // img, last; kPair: yfull, yfree 2 each
  static constexpr int NBAR = 2 * NST + 2 + 4 + 2 * kTNC + 4 + 2 + (kPair ? 4 : 0);
  static constexpr int TSLOT = BAR + NBAR * 8;
  static constexpr int RED = TSLOT + 16;                           // 8 doubles
  static constexpr int ABRT = RED + 8 * 8;                         // abort flag (int)
  static constexpr int TOTAL = ABRT + 16;
  // tensor memory (512 columns): D1 2 x 128, U 2R, then D2 2 x R (A) or D3 2R (B)
  static constexpr int T_D1 = 0;
  static constexpr int T_U = 256;
  static constexpr int T_X = T_U + 2 * R;
  static_assert(T_X + 2 * R <= 512, "tensor memory");
  static_assert(TOTAL <= 232448, "shared memory");
};

}  // namespace


// Warp roles (16 warps):
//   warp 0       TMA producer: M sub-tiles into a ring of NST slots
//   warp 1       MMA issuer: GEMM1 (strip i), then GEMM2 (A) or GEMM3 (B) of strip i-1
//   warps 2-3    fp16 image of V_old (B operand of GEMM1), one strip ahead
//   warps 4-11   S-step epilogue: C/lambda into a C tile (and the Huber sum in A)
//   warps 12-15  pass A: column sums out of tensor memory into the slab's partials;
//                pass B: fp16 image of V' (B operand of GEMM3), double-buffered
template <int R, int NST, bool kB, bool kPair = false>
__global__ void __launch_bounds__(kTThreads, 1)
    k_tc2(const __grid_constant__ CUtensorMap tmap, const __grid_constant__ Tc2Args a) {
  static_assert(!(kPair && kB), "pairs reduce pass A's column sums");
  using L = TL<R, NST, kB, kPair>;
  if (a.st->stop) return;   // uniform over the grid
  extern __shared__ __align__(1024) uint8_t smem[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int slab = (int)(blockIdx.x % a.nslabs);
  const int grp = (int)(blockIdx.x / a.nslabs);
  const int64_t row0 = (int64_t)slab * kTH;
  const uint32_t sbase = tc::smem_u32(smem);
  const uint32_t bar0 = sbase + L::BAR;
  auto B = [&](int i) { return bar0 + 8u * (uint32_t)i; };
  const int b_full = 0, b_empty = NST, b_vfull = 2 * NST, b_vempty = b_vfull + 1,
            b_d1full = b_vempty + 1, b_d1empty = b_d1full + 2, b_cfull = b_d1empty + 2,
            b_cempty = b_cfull + kTNC, b_xfull = b_cempty + kTNC, b_xempty = b_xfull + 2,
            b_img = b_xempty + 2, b_last = b_img + 1, b_yfull = b_last + 1,
            b_yfree = b_yfull + 2;
  double* red = reinterpret_cast<double*>(smem + L::RED);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + L::ABRT);
  int err = 0;
  const uint64_t deadline = tc::globaltimer_ns() + kTDeadlineNs;
  // One thread's bounded wait; on expiry it raises the abort flag and returns
  // false.  The deadline is one instant for every role of the launch, so once
  // one wait has expired every later wait that is not already satisfied fails
  // at once; the flag stops the roles whose own waits still succeed.
  auto wait_ = [&](uint32_t bar, uint32_t parity) {
    if (tc::mbar_wait_deadline(bar, parity, deadline)) return true;
    *abort_flag = 1;
    err = 1;
    return false;
  };
  // The same wait by a whole warp, with one answer for all of its lanes.
  auto wait_w = [&](uint32_t bar, uint32_t parity) {
    const bool ok = wait_(bar, parity);
    return __all_sync(0xffffffffu, ok) != 0;
  };

  // ---- set-up ---------------------------------------------------------------
  if (warp == 1) {
    tc::tmem_alloc(sbase + L::TSLOT, 512);
    tc::tmem_relinquish();
  }
  if (tid == 0) {
    for (int i = 0; i < NST; ++i) {
      tc::mbar_init(B(b_full + i), 1);
      tc::mbar_init(B(b_empty + i), 8);     // the 8 epilogue warps
    }
    tc::mbar_init(B(b_vfull), 2);           // the 2 V image warps
    tc::mbar_init(B(b_vempty), 1);          // GEMM1 commit
    for (int p = 0; p < 2; ++p) {
      tc::mbar_init(B(b_d1full + p), 1);    // GEMM1 commit
      tc::mbar_init(B(b_d1empty + p), 8);   // the 8 epilogue warps
    }
    for (int p = 0; p < kTNC; ++p) {
      tc::mbar_init(B(b_cfull + p), 8);     // the 8 epilogue warps
      tc::mbar_init(B(b_cempty + p), 1);    // GEMM2 / GEMM3 commit
    }
    for (int p = 0; p < 2; ++p) {
      // pass A: D2 result (GEMM2 commit) / read by the 4 writer warps
      // pass B: V' image written (the 4 V' warps) / read by GEMM3 (commit)
      tc::mbar_init(B(b_xfull + p), kB ? 4 : 1);
      tc::mbar_init(B(b_xempty + p), kB ? 1 : 4);
    }
    tc::mbar_init(B(b_img), 1);
    tc::mbar_init(B(b_last), 1);
    if (kPair) {
      for (int p = 0; p < 2; ++p) {
        tc::mbar_init(B(b_yfull + p), 1);   // armed with the slot's bytes by one owner warp
        tc::mbar_init(B(b_yfree + p), 2);   // the partner's two owner warps, remotely
      }
    }
    *abort_flag = 0;
    tc::fence_mbar_init();
    tc::prefetch_tmap(&tmap);
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (kPair) tc::cluster_sync();   // the partner's barriers are initialised
  const uint32_t tbase = *reinterpret_cast<volatile uint32_t*>(smem + L::TSLOT);
  auto d1 = [&](int p) { return tbase + (uint32_t)(L::T_D1 + 128 * p); };
  const uint32_t tu = tbase + L::T_U, tx = tbase + L::T_X;
  const float s_u = a.scales[2 * slab];
  const float s_w = kB ? 1.f : a.scales[2 * slab + 1];
  const float s_v = a.scales[2 * a.nslabs];
  const float s_p = kB ? tpow2_scale(__uint_as_float(*a.vp_max), 1024.f) : 1.f;
  const int64_t nstrips = (a.n + kTW - 1) / kTW;
  const int S = grp < nstrips ? (int)((nstrips - 1 - grp) / a.G + 1) : 0;
  const uint8_t* slab_img = a.img + (size_t)slab * (4 * kTH * R * 2);
  auto strip_col0 = [&](int ls) { return (grp + (int64_t)ls * a.G) * kTW; };

  if (!kB && tid == 0) {
    tc::mbar_arrive_expect_tx(B(b_img), 2 * R * kTH * 2);
    tc::bulk_load(sbase + L::WIMG, slab_img + 2 * kTH * R * 2, 2 * R * kTH * 2, B(b_img));
  }
  // U rows (fp16 hi/lo pairs) into tensor memory, by the epilogue warps (thread = row)
  if (warp >= 4 && warp < 12) {
    const int quarter = warp & 3, rb = (warp - 4) >> 2;
    const int arow = rb * 128 + quarter * 32 + lane;
    const uint4* src = reinterpret_cast<const uint4*>(slab_img + (size_t)arow * R * 4);
    const uint32_t ta = tu + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(rb * R);
#pragma unroll
    for (int c = 0; c < R; c += 16) {
      uint32_t w[16];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const uint4 v = src[c / 4 + i];
        w[4 * i] = v.x; w[4 * i + 1] = v.y; w[4 * i + 2] = v.z; w[4 * i + 3] = v.w;
      }
      tc::tmem_st16(ta + (uint32_t)c, w);
    }
    tc::tmem_st_wait();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();

  constexpr uint32_t SB_R = (R / 8) * 128;    // N-direction core stride of the K=R V image
  int issued = 0;                             // TMA sub-tile loads issued (thread 0)
  int mma_drained = 1;                        // the MMA issuer's final commit landed
  if (warp == 0) {
    // ================= TMA producer ==========================================
    if (lane == 0) {
      const int total = S * 4;
      for (int g = 0; g < total; ++g) {
        const int slot = g % NST;
        if (g >= NST && !wait_(B(b_empty + slot), (uint32_t)((g / NST - 1) & 1))) break;
        if (*abort_flag != 0) break;
        const int ls = g >> 2, q = g & 3;
        tc::mbar_arrive_expect_tx(B(b_full + slot), kTSubBytes);
        tc::tma_load_2d(sbase + L::RING + slot * kTSubBytes, &tmap, (int)row0,
                        (int)(strip_col0(ls) + kTSubCols * q), B(b_full + slot));
        issued = g + 1;
      }
    }
  } else if (warp == 1) {
    // ================= MMA issuer ===============================================
    if (lane == 0) {
      const uint32_t idesc1 = tc::idesc_f16(128, kTW, 0, 0);
      const uint64_t vdesc0 = tc::smem_desc(sbase + L::VIMG, 128, SB_R);
      const bool img_ok = kB || wait_(B(b_img), 0);
      for (int i = 0; img_ok && i < S + 1; ++i) {
        if (i < S) {   // GEMM1(i): D1 = U_b V_s^T, terms (hi,hi), (hi,lo), (lo,hi)
          const int p = i & 1;
          if (!wait_(B(b_vfull), (uint32_t)(i & 1))) break;
          if (i >= 2 && !wait_(B(b_d1empty + p), (uint32_t)(((i >> 1) - 1) & 1))) break;
          tc::fence_after_sync();
#pragma unroll
          for (int b = 0; b < 2; ++b) {
#pragma unroll
            for (int t = 0; t < 3; ++t) {
              const int tuu = t == 2 ? 1 : 0, tvv = t == 1 ? 1 : 0;
#pragma unroll
              for (int kk = 0; kk < R / 16; ++kk)
                tc::mma_ts(d1(p) + b * kTW, tu + (uint32_t)((2 * b + tuu) * (R / 2) + kk * 8),
                           vdesc0 + (uint64_t)((tvv * (kTW * R * 2) + kk * 256) >> 4), idesc1,
                           (t > 0 || kk > 0) ? 1u : 0u);
            }
          }
          tc::mma_commit(B(b_d1full + p));
          tc::mma_commit(B(b_vempty));
        }
        if (i >= 1) {
          const int s2 = i - 1, q2 = s2 & 1, pc = s2 % kTNC;
          if (!wait_(B(b_cfull + pc), (uint32_t)((s2 / kTNC) & 1))) break;
          if (!kB) {
            // GEMM2(s2): Y = C^T W_hi + C^T W_lo; two D2 buffers, the writers
            // have read the result of strip s2 - 2
            if (s2 >= 2 && !wait_(B(b_xempty + q2), (uint32_t)(((s2 >> 1) - 1) & 1))) break;
            tc::fence_after_sync();
            const uint32_t idesc2 = tc::idesc_f16(64, R, 1, 0);
            const uint64_t cd = tc::smem_desc(sbase + L::CBUF + pc * L::CBYTES, 128, kTH * 16);
            const uint64_t wdesc0 = tc::smem_desc(sbase + L::WIMG, 128, kTH * 16);
#pragma unroll
            for (int t = 0; t < 2; ++t) {
#pragma unroll
              for (int kk = 0; kk < kTH / 16; ++kk)
                tc::mma_ss(tx + (uint32_t)(q2 * R), cd + (uint64_t)((kk * 256) >> 4),
                           wdesc0 + (uint64_t)((t * (R / 8) * (kTH * 16) + kk * 256) >> 4),
                           idesc2, (t > 0 || kk > 0) ? 1u : 0u);
            }
            tc::mma_commit(B(b_xfull + q2));
            tc::mma_commit(B(b_cempty + pc));
          } else {
            // GEMM3(s2): P_C += C V'_hi^T + C V'_lo^T (accumulated over the strips)
            if (!wait_(B(b_xfull + q2), (uint32_t)((s2 >> 1) & 1))) break;
            tc::fence_after_sync();
            const uint32_t idesc3 = tc::idesc_f16(128, R, 0, 0);
            const uint64_t cd = tc::smem_desc(sbase + L::CBUF + pc * L::CBYTES, kTH * 16, 128);
            const uint64_t pd = tc::smem_desc(sbase + L::PIMG + q2 * L::PBYTES, 128,
                                              (kTW / 8) * 128);
#pragma unroll
            for (int b = 0; b < 2; ++b) {
#pragma unroll
              for (int t = 0; t < 2; ++t) {
#pragma unroll
                for (int kk = 0; kk < kTW / 16; ++kk)
                  tc::mma_ss(tx + (uint32_t)(b * R),
                             cd + (uint64_t)((b * 2048 + kk * 2 * (kTH * 16)) >> 4),
                             pd + (uint64_t)((t * (R / 8) * (kTW / 8) * 128 + kk * 256) >> 4),
                             idesc3, (s2 > 0 || t > 0 || kk > 0) ? 1u : 0u);
              }
            }
            tc::mma_commit(B(b_cempty + pc));
            tc::mma_commit(B(b_xempty + q2));
          }
        }
      }
      // every MMA of this thread has completed (and its commits have landed)
      // before the CTA releases tensor memory and shared memory; pass B's
      // epilogue also reads the P partial after this.  This wait must not give
      // up because another role did: it drains the MMAs already issued.
      tc::mma_commit(B(b_last));
      if (!tc::mbar_wait_deadline(B(b_last), 0, deadline + 100000000ull)) {
        mma_drained = 0;
        *abort_flag = 1;
        err = 1;
      }
    }
    mma_drained = __shfl_sync(0xffffffffu, mma_drained, 0);
  } else if (warp == 2 || warp == 3) {
    // ================= V_old image (GEMM1 operand), one strip ahead ============
    // two warps, each a half of the strip's 64 x R floats (kTW * R / 256 float4
    // per lane), the next strip's half loaded while this one is written
    constexpr int V4 = kTW * R / 256;
    const int half = warp - 2;
    float4 vr[V4];
    auto load_v = [&](int ls) {
      const int64_t col0 = strip_col0(ls);
#pragma unroll
      for (int t = 0; t < V4; ++t) {
        const int e = 4 * (lane + 32 * (half * V4 + t)), j = e / R, k = e % R;
        vr[t] = col0 + j < a.n ? *reinterpret_cast<const float4*>(a.Vold + (col0 + j) * R + k)
                               : make_float4(0.f, 0.f, 0.f, 0.f);
      }
    };
    if (S > 0) load_v(0);
    for (int ls = 0; ls < S; ++ls) {
      if (ls >= 1 && !wait_w(B(b_vempty), (uint32_t)((ls - 1) & 1))) break;
      uint8_t* img = smem + L::VIMG;
#pragma unroll
      for (int t = 0; t < V4; ++t) {
        const int e = 4 * (lane + 32 * (half * V4 + t)), j = e / R, k = e % R;
        const float x[4] = {vr[t].x, vr[t].y, vr[t].z, vr[t].w};
        __half hi[4], lo[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) tsplit(x[u], s_v, hi[u], lo[u]);
        const int off = (j >> 3) * SB_R + (k >> 3) * 128 + (j & 7) * 16 + (k & 7) * 2;
        __half2 h01 = __halves2half2(hi[0], hi[1]), h23 = __halves2half2(hi[2], hi[3]);
        __half2 l01 = __halves2half2(lo[0], lo[1]), l23 = __halves2half2(lo[2], lo[3]);
        *reinterpret_cast<uint2*>(img + off) =
            make_uint2(*reinterpret_cast<uint32_t*>(&h01), *reinterpret_cast<uint32_t*>(&h23));
        *reinterpret_cast<uint2*>(img + kTW * R * 2 + off) =
            make_uint2(*reinterpret_cast<uint32_t*>(&l01), *reinterpret_cast<uint32_t*>(&l23));
      }
      tc::fence_proxy_async_smem();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(B(b_vfull));
      if (ls + 1 < S) load_v(ls + 1);
    }
  } else if (warp < 12) {
    // ================= S-step epilogue (256 threads, thread = row) ===============
    const int quarter = warp & 3, rb = (warp - 4) >> 2;
    const int arow = rb * 128 + quarter * 32 + lane;
    const float inv_uv = 1.f / (s_u * s_v);
    const float inv_lam = 1.f / a.lam;
    float hub_hi = 0.f, hub_lo = 0.f;
    bool ok = true;   // warp-uniform; false once a wait of this warp has failed
    for (int ls = 0; ls < S; ++ls) {
      const int p = ls & 1, pc = ls % kTNC;
      if (!wait_w(B(b_d1full + p), (uint32_t)((ls >> 1) & 1))) { ok = false; break; }
      // C slot: the GEMM that read it (strip ls - kTNC) has completed
      if (ls >= kTNC && !wait_w(B(b_cempty + pc), (uint32_t)(((ls / kTNC) - 1) & 1))) {
        ok = false;
        break;
      }
      tc::fence_after_sync();
      uint8_t* cbuf = smem + L::CBUF + pc * L::CBYTES;
      float hub = 0.f;
      // four sub-tiles of 16 columns; the loads of the next are in flight while
      // the current one is computed
      float dv[2][16], mv[2][16];
      // a failed wait for an M sub-tile leaves garbage in this strip, which is
      // never handed on
      auto load_sub = [&](int q, float* d, float* mm) {
        const int g = ls * 4 + q;
        const int rs = g % NST;
        if (!wait_w(B(b_full + rs), (uint32_t)((g / NST) & 1))) ok = false;
        const float* msub = reinterpret_cast<const float*>(smem + L::RING + rs * kTSubBytes);
        tc::tmem_ld16(d1(p) + ((uint32_t)(quarter * 32) << 16) + rb * kTW + q * kTSubCols, d);
#pragma unroll
        for (int jj = 0; jj < 16; ++jj) mm[jj] = msub[jj * kTH + arow];
      };
      load_sub(0, dv[0], mv[0]);
      tc::tmem_ld_wait();
      __syncwarp();
      if (ok && lane == 0) tc::mbar_arrive(B(b_empty + (ls * 4) % NST));
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int cb = q & 1;
        if (q < 3) load_sub(q + 1, dv[cb ^ 1], mv[cb ^ 1]);
        uint32_t packed[8];
#pragma unroll
        for (int jj = 0; jj < 16; jj += 2) {
          float c2[2];
#pragma unroll
          for (int u = 0; u < 2; ++u) {
            const float rn = (mv[cb][jj + u] - dv[cb][jj + u] * inv_uv) * inv_lam;   // R / lambda
            const float c = fminf(fmaxf(rn, -1.f), 1.f);                             // C / lambda
            if (!kB) hub = fmaf(c, rn - 0.5f * c, hub);                              // H(R) / lambda^2
            c2[u] = c;
          }
          __half2 h2 = __floats2half2_rn(c2[0], c2[1]);
          packed[jj / 2] = *reinterpret_cast<uint32_t*>(&h2);
        }
#pragma unroll
        for (int ch = 0; ch < 2; ++ch) {
          const int j8 = (q * kTSubCols + ch * 8) >> 3;
          const int off = j8 * (kTH * 16) + (arow >> 3) * 128 + (arow & 7) * 16;
          *reinterpret_cast<uint4*>(cbuf + off) =
              make_uint4(packed[4 * ch], packed[4 * ch + 1], packed[4 * ch + 2], packed[4 * ch + 3]);
        }
        if (q < 3) {
          tc::tmem_ld_wait();
          __syncwarp();
          if (ok && lane == 0) tc::mbar_arrive(B(b_empty + (ls * 4 + q + 1) % NST));
        }
      }
      if (!kB) ttwo_sum(hub_hi, hub_lo, hub);
      if (!ok) break;   // this strip's C tile is never handed to a GEMM
      tc::fence_before_sync();
      tc::fence_proxy_async_smem();
      __syncwarp();
      if (lane == 0) {
        tc::mbar_arrive(B(b_d1empty + p));
        tc::mbar_arrive(B(b_cfull + pc));
      }
    }
    if (kB && ok && wait_w(B(b_last), 0)) {
      // P partial of this strip group's columns for the CTA's rows
      tc::fence_after_sync();
      const int64_t grow = row0 + arow;
      const float ps = a.lam / s_p;
      float* out = a.part_p + ((int64_t)grp * a.m + grow) * R;
#pragma unroll
      for (int c = 0; c < R; c += 16) {
        float pv[16];
        tc::tmem_ld16(tx + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(rb * R + c), pv);
        tc::tmem_ld_wait();
        if (grow < a.m) {
#pragma unroll
          for (int k = 0; k < 16; k += 4)
            *reinterpret_cast<float4*>(out + c + k) =
                S > 0 ? make_float4(pv[k] * ps, pv[k + 1] * ps, pv[k + 2] * ps, pv[k + 3] * ps)
                      : make_float4(0.f, 0.f, 0.f, 0.f);
        }
      }
    } else if (!kB) {
      double hsum = ((double)hub_hi + (double)hub_lo) * (double)a.lam * (double)a.lam;
      for (int o = 16; o > 0; o >>= 1) hsum += __shfl_xor_sync(0xffffffffu, hsum, o);
      if (lane == 0) red[warp - 4] = hsum;
    }
  } else if (!kB) {
    // ================= pass A: column sums into the slab's partials =============
    // D2 (M = 64: strip column j in lane 16 (j / 16) + j % 16 of quarter j / 16)
    const int xw = warp & 3;
    const float y_scale = a.lam / s_w;
    // kPair: the cluster's two CTAs (slabs 2k, 2k + 1) share one partial per
    // column: cluster rank 0 owns strip columns 0..31 (writer warps 0, 1), rank
    // 1 columns 32..63 (warps 2, 3); a warp whose columns the partner owns
    // sends its sums into the partner's receive slot (st.async, counted on the
    // partner's yfull), an owner warp adds what it receives and writes.
    const uint32_t crank = kPair ? tc::cluster_rank() : 0u, partner = crank ^ 1u;
    const bool owner = !kPair || (xw >> 1) == (int)crank;
    const int jl = (xw & 1) * 16 + lane;          // column within the owner's half
    float* ybase = a.ypart + (int64_t)(kPair ? slab >> 1 : slab) * a.n * R;
    for (int ls = 0; ls < S; ++ls) {
      const int q2 = ls & 1;
      if (!wait_w(B(b_xfull + q2), (uint32_t)((ls >> 1) & 1))) break;
      tc::fence_after_sync();
      float yv[R];
#pragma unroll
      for (int c = 0; c < R; c += 16)
        tc::tmem_ld16(tx + (uint32_t)(q2 * R) + ((uint32_t)(xw * 32) << 16) + (uint32_t)c,
                      yv + c);
      tc::tmem_ld_wait();
      tc::fence_before_sync();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(B(b_xempty + q2));
      const int64_t col = strip_col0(ls) + xw * 16 + lane;
      if (kPair && !owner) {
        // the partner has consumed strip ls - 2 from this slot
        if (ls >= 2 && !wait_w(B(b_yfree + q2), (uint32_t)(((ls >> 1) - 1) & 1))) break;
        if (__any_sync(0xffffffffu, *abort_flag != 0)) break;   // one answer per warp
        if (lane < 16) {   // every column, zeros past n: the slot's byte count is fixed
          const uint32_t dst = tc::map_cluster(
              sbase + (uint32_t)(L::RECV + q2 * L::RSLOT + jl * R * 4), partner);
          const uint32_t bar = tc::map_cluster(B(b_yfull + q2), partner);
#pragma unroll
          for (int k = 0; k < R; k += 4) {
            uint4 v;
            v.x = __float_as_uint(yv[k] * y_scale);
            v.y = __float_as_uint(yv[k + 1] * y_scale);
            v.z = __float_as_uint(yv[k + 2] * y_scale);
            v.w = __float_as_uint(yv[k + 3] * y_scale);
            tc::st_async_u32x4(dst + (uint32_t)k * 4, v, bar);
          }
        }
        continue;
      }
      if (kPair) {
        if (lane == 0 && (xw & 1) == 0) tc::mbar_arrive_expect_tx(B(b_yfull + q2), L::RSLOT);
        if (!wait_w(B(b_yfull + q2), (uint32_t)((ls >> 1) & 1))) break;
      }
      if (lane < 16 && col < a.n) {
        float* dst = ybase + col * R;
        const float* rcv = reinterpret_cast<const float*>(smem + L::RECV + q2 * L::RSLOT) + jl * R;
#pragma unroll
        for (int k = 0; k < R; k += 4) {
          float4 y = make_float4(yv[k] * y_scale, yv[k + 1] * y_scale, yv[k + 2] * y_scale,
                                 yv[k + 3] * y_scale);
          if (kPair) {
            const float4 o = *reinterpret_cast<const float4*>(rcv + k);
            y.x += o.x; y.y += o.y; y.z += o.z; y.w += o.w;
          }
          *reinterpret_cast<float4*>(dst + k) = y;
        }
      }
      if (kPair) {
        __syncwarp();
        if (lane == 0) tc::mbar_arrive_cluster_relaxed(B(b_yfree + q2), partner);
      }
    }
  } else {
    // ================= pass B: V' image (GEMM3 operand), double-buffered ========
    // entry (n, j), n = k (hi) or R + k (lo), j the strip column:
    //   (n / 8) * 1024 + (j / 8) * 128 + (n % 8) * 16 + (j % 8) * 2
    // task (column group jb of 8, quad of k): 8 float4 loads, 4 x (16 bytes hi,
    // 16 bytes lo); 8 R / 4 tasks over the 128 threads, the next strip's values
    // loaded while this one is written
    constexpr int NT = 8 * R / 4;                 // tasks per strip
    constexpr int TPT = (NT + 127) / 128;         // tasks per thread
    const int xt = tid - 384;
    float4 pv[TPT][8];
    auto load_p = [&](int ls) {
      const int64_t col0 = strip_col0(ls);
#pragma unroll
      for (int u = 0; u < TPT; ++u) {
        const int task = xt + 128 * u;
        const int jb = task / (R / 4), k4 = (task % (R / 4)) * 4;
#pragma unroll
        for (int jj = 0; jj < 8; ++jj) {
          const int64_t c = col0 + jb * 8 + jj;
          pv[u][jj] = (task < NT && c < a.n) ? *reinterpret_cast<const float4*>(a.Vp + c * R + k4)
                                             : make_float4(0.f, 0.f, 0.f, 0.f);
        }
      }
    };
    if (S > 0) load_p(0);
    for (int ls = 0; ls < S; ++ls) {
      const int p = ls & 1;
      if (ls >= 2 && !wait_w(B(b_xempty + p), (uint32_t)(((ls >> 1) - 1) & 1))) break;
      uint8_t* img = smem + L::PIMG + p * L::PBYTES;
#pragma unroll
      for (int u = 0; u < TPT; ++u) {
        const int task = xt + 128 * u;
        if (task >= NT) continue;
        const int jb = task / (R / 4), k4 = (task % (R / 4)) * 4;
#pragma unroll
        for (int kq = 0; kq < 4; ++kq) {
          uint32_t hw[4], lw[4];
#pragma unroll
          for (int jj = 0; jj < 8; jj += 2) {
            const float x0 = kq == 0 ? pv[u][jj].x : kq == 1 ? pv[u][jj].y : kq == 2 ? pv[u][jj].z : pv[u][jj].w;
            const float x1 = kq == 0 ? pv[u][jj + 1].x : kq == 1 ? pv[u][jj + 1].y
                           : kq == 2 ? pv[u][jj + 1].z : pv[u][jj + 1].w;
            __half h0, l0, h1, l1;
            tsplit(x0, s_p, h0, l0);
            tsplit(x1, s_p, h1, l1);
            __half2 hh = __halves2half2(h0, h1), ll = __halves2half2(l0, l1);
            hw[jj / 2] = *reinterpret_cast<uint32_t*>(&hh);
            lw[jj / 2] = *reinterpret_cast<uint32_t*>(&ll);
          }
          const int k = k4 + kq;
          const int off = (k >> 3) * 1024 + jb * 128 + (k & 7) * 16;
          *reinterpret_cast<uint4*>(img + off) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
          *reinterpret_cast<uint4*>(img + (R / 8) * 1024 + off) =
              make_uint4(lw[0], lw[1], lw[2], lw[3]);
        }
      }
      tc::fence_proxy_async_smem();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(B(b_xfull + p));
      if (ls + 1 < S) load_p(ls + 1);
    }
  }

  // ---- end: Huber partial (pass A), tensor memory released ------------------------
  if (err) atomicExch(a.err, DCF_ETIMEOUT);
  tc::fence_before_sync();
  __syncthreads();
  // Every role has left its loop, so the flag is final and the same for all
  // threads.  After an expiry, drain the TMA loads thread 0 issued (the W
  // image and the last load of every ring slot) before the CTA leaves.
  if (*abort_flag != 0) {
    if (tid == 0) {
      const uint64_t dl = tc::globaltimer_ns() + 100000000ull;
      if (!kB) tc::mbar_wait_deadline(B(b_img), 0, dl);
      for (int slot = 0; slot < NST && slot < issued; ++slot) {
        const int g_last = slot + ((issued - 1 - slot) / NST) * NST;
        tc::mbar_wait_deadline(B(b_full + slot), (uint32_t)((g_last / NST) & 1), dl);
      }
    }
    __syncthreads();
  }
  if (!kB && tid == 0) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += red[w];
    a.part_h[blockIdx.x] = t;
  }
  // no CTA of a pair leaves while its partner may still address its shared memory
  if (kPair) tc::cluster_sync();
  // (if an MMA is still running after all that, the tensor memory stays allocated)
  if (warp == 1 && mma_drained) tc::tmem_dealloc(tbase, 512);
}

// V' = V_old Z + sum over the slabs of their column sums (FP32, slabs in
// order), written to Vnew; max |V'| into vmax (float bits; the scale of the
// V' image in pass B).
__global__ void __launch_bounds__(256) k_tc2_vreduce(const float* __restrict__ ypart,
                                                     int nslabs, const float* __restrict__ VZ,
                                                     int64_t count4, int64_t slab_stride4,
                                                     float* __restrict__ Vnew,
                                                     unsigned int* vmax, const DevState* st,
                                                     unsigned int* vmax_all) {
  if (st->stop) return;
  float mx = 0.f;
  const float4* y4 = reinterpret_cast<const float4*>(ypart);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count4;
       i += (int64_t)gridDim.x * blockDim.x) {
    float4 acc = reinterpret_cast<const float4*>(VZ)[i];
    for (int s = 0; s < nslabs; ++s) {
      const float4 y = y4[(int64_t)s * slab_stride4 + i];
      acc.x += y.x;
      acc.y += y.y;
      acc.z += y.z;
      acc.w += y.w;
    }
    reinterpret_cast<float4*>(Vnew)[i] = acc;
    mx = fmaxf(mx, fmaxf(fmaxf(fabsf(acc.x), fabsf(acc.y)), fmaxf(fabsf(acc.z), fabsf(acc.w))));
  }
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0 && mx > 0.f) {
    atomicMax(vmax, __float_as_uint(mx));
    if (vmax_all) atomicMax(vmax_all, __float_as_uint(mx));
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
namespace {

// ring depth per (R, pass): as deep as shared memory allows (one slot fewer
// for the receive slots of the paired pass A)
template <int R, bool kB, bool kPair = false>
constexpr int tc2_nst() {
  return R == 64 ? (kB ? 7 : (kPair ? 4 : 5)) : R == 32 ? (kB ? 8 : 7) : (kB ? 9 : 8);
}

template <int R, bool kB, bool kPair = false>
cudaError_t tc2_attr() {
  constexpr int NST = tc2_nst<R, kB, kPair>();
  return cudaFuncSetAttribute(k_tc2<R, NST, kB, kPair>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)TL<R, NST, kB, kPair>::TOTAL);
}

template <int R, bool kB>
cudaError_t tc2_launch(const void* tmap, const Tc2Args& a, cudaStream_t s) {
  constexpr int NST = tc2_nst<R, kB>();
  const CUtensorMap* tm = reinterpret_cast<const CUtensorMap*>(tmap);
  k_tc2<R, NST, kB><<<a.nslabs * a.G, kTThreads, TL<R, NST, kB>::TOTAL, s>>>(*tm, a);
  return cudaGetLastError();
}

// Pass A in two-CTA clusters (slabs 2k, 2k + 1 of a strip group).
template <int R>
cudaError_t tc2_launch_pair(const void* tmap, const Tc2Args& a, cudaStream_t s) {
  constexpr int NST = tc2_nst<R, false, true>();
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3((unsigned)(a.nslabs * a.G), 1, 1);
  cfg.blockDim = dim3(kTThreads, 1, 1);
  cfg.dynamicSmemBytes = TL<R, NST, false, true>::TOTAL;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 2;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  const CUtensorMap* tm = reinterpret_cast<const CUtensorMap*>(tmap);
  return cudaLaunchKernelEx(&cfg, k_tc2<R, NST, false, true>, *tm, a);
}

}  // namespace

// Whether pass A reduces its column sums in slab pairs (R = 64, an even
// number of slabs), and so how many partials per column it leaves.
bool tc2_paired(int R, int nslabs) { return R == 64 && nslabs % 2 == 0; }
int tc2_parts(int R, int nslabs) { return tc2_paired(R, nslabs) ? nslabs / 2 : nslabs; }

cudaError_t tc2_prepare(int R) {
  cudaError_t e;
  switch (R) {
    case 16:
      if ((e = tc2_attr<16, false>()) != cudaSuccess) return e;
      return tc2_attr<16, true>();
    case 32:
      if ((e = tc2_attr<32, false>()) != cudaSuccess) return e;
      return tc2_attr<32, true>();
    default:
      if ((e = tc2_attr<64, false>()) != cudaSuccess) return e;
      if ((e = tc2_attr<64, false, true>()) != cudaSuccess) return e;
      return tc2_attr<64, true>();
  }
}

cudaError_t launch_tc2(int R, int pass_b, const void* tmap, const Tc2Args& a, cudaStream_t s) {
  if (a.nslabs * a.G < 1) return cudaSuccess;
  switch (R) {
    case 16: return pass_b ? tc2_launch<16, true>(tmap, a, s) : tc2_launch<16, false>(tmap, a, s);
    case 32: return pass_b ? tc2_launch<32, true>(tmap, a, s) : tc2_launch<32, false>(tmap, a, s);
    default:
      if (pass_b) return tc2_launch<64, true>(tmap, a, s);
      return tc2_paired(64, a.nslabs) ? tc2_launch_pair<64>(tmap, a, s)
                                      : tc2_launch<64, false>(tmap, a, s);
  }
}

cudaError_t launch_tc2_vreduce(int R, const float* ypart, int nslabs, const float* VZ, int64_t n,
                               float* Vnew, unsigned int* vmax, const DevState* st,
                               int num_sms, cudaStream_t s, unsigned int* vmax_all) {
  const int64_t count4 = n * R / 4;
  int64_t blocks = (count4 + 255) / 256;
  if (blocks > 8LL * num_sms) blocks = 8LL * num_sms;
  if (blocks < 1) blocks = 1;
  k_tc2_vreduce<<<(unsigned)blocks, 256, 0, s>>>(ypart, nslabs, VZ, count4, count4, Vnew, vmax,
                                                 st, vmax_all);
  return cudaGetLastError();
}

}  // namespace dcf
