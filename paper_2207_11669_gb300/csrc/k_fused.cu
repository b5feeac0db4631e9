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
//   GEMM2  Y  = C_s^T W_hi + C_s^T W_lo   (C/lambda in [-1,1] stored once in fp16)
//   GEMM3  P_C += C_s V'_hi^T + C_s V'_lo^T
// V Z is precomputed (by the preparation kernel) and added by the reducers;
// V^T V' (= V_{t-1}^T V_t, also a metric) closes P in the r x r algebra and,
// with Q = V'^T V', comes from the Gram kernels after the pass.
//
// The epilogue writes each C tile twice: into shared memory for GEMM2 (freed
// as soon as GEMM2 completes) and into tensor memory as GEMM3's A operand
// (held across the cluster exchange, kNC tiles deep).  Keeping the long-lived
// copies out of shared memory leaves room for a deeper M ring.
//
// Parallel layout: a thread-block cluster of CS CTAs owns whole columns; CTA c
// of a cluster holds rows [256c, 256c+256) of U, W and of every M strip, so
// M is read from HBM once per iteration (TMA, 256x16 fp32 boxes).  The
// column sums of GEMM2 are reduced across the cluster through distributed
// shared memory (reduce-scatter on 8-column chunks, all-gather of the fp16
// V' image), which is the only cross-CTA exchange.  Each cluster walks the
// strips s = cluster_id, cluster_id + #clusters, ...
//
// Every wait on an mbarrier is bounded.  The first wait that expires raises a
// CTA-wide abort flag; from then on no role issues another MMA, tcgen05.st,
// TMA load or st.async that the expired wait was guarding, the single-thread
// roles and the epilogue leave their loops, and the exchange warps run their
// remaining strips without waiting or sending (their named barriers stay
// matched).  Before tensor memory is released the MMA issuers' final commits
// and the TMA loads still in flight are drained with bounded waits; if even
// that fails the tensor memory is left allocated.  The kernel records
// DCF_ETIMEOUT and every CTA still reaches the final cluster barrier.
#include <algorithm>

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_fp16.h>

#include "dcf.h"
#include "dcf_internal.cuh"
#include "tc_ptx.cuh"

namespace dcf {

constexpr int kFW = 64;          // strip width (columns)
constexpr int kFH = 256;         // rows per CTA (2 row blocks of 128)
// One M sub-tile: all 256 rows of the CTA x 16 columns, so that both row blocks
// of the epilogue consume the ring in the same order (a strip is 4 sub-tiles).
constexpr int kSubRows = kFH, kSubCols = 16;
constexpr int kSubBytes = kSubRows * kSubCols * 4;
// Every wait of a launch together gives up after this long (a launch takes
// milliseconds); on expiry the kernel records DCF_ETIMEOUT and runs out.
constexpr uint64_t kDeadlineNs = 2000000000ull;


constexpr int kFThreads = 640;   // 20 warps, see the role map below
constexpr int kChunk = 4;        // columns per reduce-scatter chunk (16 chunks per strip)
constexpr int kNC = 3;           // C tiles in flight in tensor memory (GEMM3's A operand): a
                                 // tile lives from the S-step epilogue of its strip until that
                                 // strip's GEMM3, i.e. across the cluster exchange, so this
                                 // sets the pipeline depth
constexpr int kNCS = 2;          // C tiles in shared memory (GEMM2's A operand), each freed as
                                 // soon as its GEMM2 has completed

template <int R, int NST>
struct FL {  // shared-memory layout (bytes)
  static constexpr int RING = 0;                                 // NST x (256 x 16 fp32)
  static constexpr int WIMG = RING + NST * kSubBytes;            // 2R x 256 fp16
  static constexpr int CBYTES = kFH * kFW * 2;                   // one C tile (256 x 64 fp16)
  static constexpr int CBUF = WIMG + 2 * R * kFH * 2;            // kNCS C tiles
  static constexpr int VBYTES = 2 * kFW * R * 2;                 // one V image (2 terms)
  static constexpr int VIMG = CBUF + kNCS * CBYTES;              // one V image
  static constexpr int PBYTES = 2 * R * kFW * 2;                 // one V' image (2R x 64 fp16)
  static constexpr int PIMG = VIMG + VBYTES;                     // 2 V' images
  static constexpr int YBYTES = kFW * R * 4;                     // one column-sum block
  static constexpr int YPART = PIMG + 2 * PBYTES;                // 2 x (64 x R fp32)
  static constexpr int STG = YPART + 2 * YBYTES;                 // 2R x 4 fp16 image chunk
  static constexpr int BAR = STG + 2 * (2 * R * kChunk * 2);     // mbarriers (2 staging chunks)
  // full/empty NST each; vfull, vempty, d1full, d1empty 2 each (only [0] of
  // each is used); cfull, cempty kNC each; c2free kNCS; d2full, d2empty,
  // g3done, yfull, yfree, pfull, pfree 2 each; img, last, fin1
  static constexpr int NBAR = 2 * NST + 8 + 2 * kNC + kNCS + 14 + 3;
  static constexpr int TSLOT = BAR + NBAR * 8;
  static constexpr int RED = TSLOT + 16;                         // 16 doubles
  static constexpr int ABRT = RED + 16 * 8;                      // abort flag (int)
  static constexpr int TOTAL = ABRT + 16;
  // tensor-memory columns (512 allocated)
  static constexpr int T_D1 = 0;                                 // 2 blocks x 64 (U V_s^T)
  static constexpr int T_D2 = 128;                               // 2 x (M=64 result, R columns)
  static constexpr int T_D3 = T_D2 + 2 * R;                      // 2 blocks x R (P_C)
  static constexpr int T_U = T_D3 + 2 * R;                       // U hi/lo, 2 blocks x 2 x R/2
  static constexpr int T_C = T_U + 2 * R;                        // kNC x (2 blocks x 32): C fp16 pairs
  static_assert(T_C + kNC * 64 <= 512, "tensor memory");
  static_assert(TOTAL <= 232448, "shared memory");
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

// Packed FP32 pairs (one instruction for two lanes of arithmetic).
__device__ __forceinline__ unsigned long long f2_bits(float2 v) {
  return (unsigned long long)__float_as_uint(v.x) |
         ((unsigned long long)__float_as_uint(v.y) << 32);
}
__device__ __forceinline__ float2 f2_from(unsigned long long b) {
  return make_float2(__uint_as_float((unsigned)b), __uint_as_float((unsigned)(b >> 32)));
}
__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c) {
  unsigned long long d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(f2_bits(a)), "l"(f2_bits(b)), "l"(f2_bits(c)));
  return f2_from(d);
}
__device__ __forceinline__ float2 fmul2(float2 a, float2 b) {
  unsigned long long d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(f2_bits(a)), "l"(f2_bits(b)));
  return f2_from(d);
}

__device__ __forceinline__ void tsum(float& hi, float& lo, float x) {
  float t = hi + x;
  float bp = t - hi;
  lo += (hi - (t - bp)) + (x - bp);
  hi = t;
}

// Warp-specialised pipeline over the strips of the cluster (20 warps):
//   warp 0       TMA producer: M sub-tiles into a ring of NST slots
//   warp 1       MMA issuer for GEMM1 (strip i) and GEMM2 (strip i-1); owns TMEM
//   warp 2       MMA issuer for GEMM3, which waits on the cluster exchange and
//                therefore must not hold up GEMM1/GEMM2 (tcgen05 ops complete in
//                the issuing thread's order)
//   warp 3       fp16 image of V_s (B operand of GEMM1), one strip ahead
//   warps 4-11   S-step epilogue: R, C/lambda into the C tile, Huber
//   warps 12-19  exchange, two groups of 4 warps for even and odd strips:
//                column sums out of tensor memory, pushed to the reducer of
//                their chunk (DSMEM), V' of this CTA's chunks, the V' image
//                pushed to every CTA
// Local mbarriers link the roles inside a CTA; four mbarriers per CTA link the
// CTAs of the cluster.  Data crosses the cluster only by st.async, whose bytes
// complete on the receiver's mbarrier (no fences, no release/acquire pairs):
//   yfull  (1 + bytes)  the column sums of this CTA's chunks from every CTA
//   yfree  (count CS)   every reducer has consumed this CTA's column sums
//   pfull  (1 + bytes)  every reducer's chunk of the V' image has landed here
//   pfree  (count CS)   every CTA's GEMM3 that read this V' image buffer is done
// Column sums and V' images are double-buffered, so each of these exists
// once per buffer and completes every other strip; an arrival for strip s+2
// can only happen after the phase of strip s has completed.  The exchange
// groups work on alternate strips with the buffers of their parity.
template <bool kTable>
__device__ __forceinline__ const FusedArgs& fused_args(const FusedArgs& ap,
                                                       const FusedArgs* table, int c) {
  if constexpr (kTable) return table[c];
  else return ap;
}

// kTable = false: one problem, its strips dealt to the clusters of the launch
// (cluster c takes strips c, c + #clusters, ...; P partial slot c).
// kTable = true: cluster c runs every strip of problem table[c] (P slot 0).
template <int R, int NST, bool kTable>
__global__ void __launch_bounds__(kFThreads, 1)
    k_fused(const __grid_constant__ CUtensorMap tmap, const __grid_constant__ FusedArgs ap,
            const FusedArgs* __restrict__ table) {
  using L = FL<R, NST>;
  const int cs = ap.cs;
  const FusedArgs& a = fused_args<kTable>(ap, table, (int)(blockIdx.x / cs));
  const void* tmp = kTable ? a.tmap_g : static_cast<const void*>(&tmap);
  if (a.st->stop) return;  // uniform over the cluster (over the grid for one problem)
  extern __shared__ __align__(1024) uint8_t smem[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t crank = tc::cluster_rank();
  const int cid = kTable ? 0 : (int)(blockIdx.x / cs);   // cluster index within the problem
  const int ncl = kTable ? 1 : ap.nclusters;             // clusters sharing the problem
  const int slab = (int)(blockIdx.x % cs);   // == crank
  const int64_t row0 = (int64_t)slab * kFH;
  const uint32_t sbase = tc::smem_u32(smem);
  const uint32_t bar0 = sbase + L::BAR;
  auto B = [&](int i) { return bar0 + 8u * (uint32_t)i; };
  // barrier indices
  const int b_full = 0, b_empty = NST, b_vfull = 2 * NST, b_vempty = b_vfull + 2,
            b_d1full = b_vempty + 2, b_d1empty = b_d1full + 2, b_cfull = b_d1empty + 2,
            b_cempty = b_cfull + kNC, b_c2free = b_cempty + kNC, b_d2full = b_c2free + kNCS,
            b_d2empty = b_d2full + 2,
            b_g3done = b_d2empty + 2, b_yfull = b_g3done + 2, b_yfree = b_yfull + 2,
            b_pfull = b_yfree + 2, b_pfree = b_pfull + 2, b_img = b_pfree + 2,
            b_last = b_img + 1, b_fin1 = b_last + 1;
  double* red = reinterpret_cast<double*>(smem + L::RED);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + L::ABRT);
  int err = 0;
  const uint64_t deadline = tc::globaltimer_ns() + kDeadlineNs;
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
  auto aborted = [&]() { return *abort_flag != 0; };

  // ---- set-up -------------------------------------------------------------
  if (warp == 1) {
    tc::tmem_alloc(sbase + L::TSLOT, 512);
    tc::tmem_relinquish();
  }
  if (tid == 0) {
    for (int i = 0; i < NST; ++i) {
      tc::mbar_init(B(b_full + i), 1);
      tc::mbar_init(B(b_empty + i), 8);     // the 8 epilogue warps
    }
    for (int p = 0; p < 2; ++p) {
      tc::mbar_init(B(b_vfull + p), 1);     // the V-image warp (only [0] is used)
      tc::mbar_init(B(b_vempty + p), 1);    // GEMM1 commit (only [0] is used)
      tc::mbar_init(B(b_d1full + p), 1);    // GEMM1 commit
      tc::mbar_init(B(b_d1empty + p), 8);   // the 8 epilogue warps
    }
    for (int p = 0; p < kNC; ++p) {
      tc::mbar_init(B(b_cfull + p), 8);     // the 8 epilogue warps: both C copies written
      tc::mbar_init(B(b_cempty + p), 1);    // GEMM3 commit: tensor-memory C slot free
    }
    for (int p = 0; p < kNCS; ++p) tc::mbar_init(B(b_c2free + p), 1);   // GEMM2 commit
    for (int p = 0; p < 2; ++p) {           // D2 buffers: GEMM2 of strip s uses s % 2
      tc::mbar_init(B(b_d2full + p), 1);
      tc::mbar_init(B(b_d2empty + p), 4);   // the 4 exchange warps
    }
    tc::mbar_init(B(b_g3done), 1);
    tc::mbar_init(B(b_g3done + 1), 1);
    for (int p = 0; p < 2; ++p) {           // cross-CTA, one per buffer of the pair
      tc::mbar_init(B(b_yfull + p), 1);     // armed by the local reducer; st.async bytes
      tc::mbar_init(B(b_yfree + p), cs);    // every reducer, remote arrivals
      tc::mbar_init(B(b_pfull + p), 1);     // armed by the GEMM3 issuer; st.async bytes
      tc::mbar_init(B(b_pfree + p), cs);    // every CTA's GEMM3, remote arrivals
    }
    tc::mbar_init(B(b_img), 1);
    tc::mbar_init(B(b_last), 1);            // every MMA of the GEMM3 issuer has completed
    tc::mbar_init(B(b_fin1), 1);            // every MMA of the GEMM1/GEMM2 issuer has completed
    *abort_flag = 0;
    tc::fence_mbar_init();
    tc::prefetch_tmap(tmp);
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tbase = *reinterpret_cast<volatile uint32_t*>(smem + L::TSLOT);
  const uint32_t d1 = tbase + L::T_D1;                   // one D1: GEMM1 waits for the epilogue
  auto tcs = [&](int pc) { return tbase + (uint32_t)(L::T_C + pc * 64); };   // C slot
  auto d2 = [&](int s) { return tbase + (uint32_t)(L::T_D2 + s * R); };
  const uint32_t d3 = tbase + L::T_D3, tu = tbase + L::T_U;
  const float s_u = a.scales[2 * slab], s_w = a.scales[2 * slab + 1];
  const float s_v = a.scales[2 * a.nslabs];
  const int64_t nstrips = (a.n + kFW - 1) / kFW;
  const int S = cid < nstrips ? (int)((nstrips - 1 - cid) / ncl + 1) : 0;
  const int nch = (int)((kFW / kChunk - 1 - (int)crank) / cs + 1);   // chunks this CTA reduces
  const uint8_t* slab_img = a.img + (size_t)slab * (4 * kFH * R * 2);
  auto strip_col0 = [&](int ls) { return (cid + (int64_t)ls * ncl) * kFW; };

  if (tid == 0) {
    tc::mbar_arrive_expect_tx(B(b_img), 2 * R * kFH * 2);
    tc::bulk_load(sbase + L::WIMG, slab_img + 2 * kFH * R * 2, 2 * R * kFH * 2, B(b_img));
  }
  // U rows (fp16 hi/lo pairs) into tensor memory, by the epilogue warps (thread = row)
  if (warp >= 4 && warp < 12) {
    const int quarter = warp & 3, rb = (warp - 4) >> 2;
    const int arow = rb * 128 + quarter * 32 + lane;
    const uint4* src = reinterpret_cast<const uint4*>(slab_img + (size_t)arow * R * 4);
    uint32_t w[R];
#pragma unroll
    for (int i = 0; i < R / 4; ++i) {
      const uint4 v = src[i];
      w[4 * i] = v.x; w[4 * i + 1] = v.y; w[4 * i + 2] = v.z; w[4 * i + 3] = v.w;
    }
    const uint32_t ta = tu + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(rb * R);
    if (R == 32) {
      tc::tmem_st16(ta, w);
      tc::tmem_st16(ta + 16, w + 16);
    } else {
      tc::tmem_st8(ta, w);
      tc::tmem_st8(ta + 8, w + 8);
    }
    tc::tmem_st_wait();
  }
  tc::fence_before_sync();
  tc::cluster_sync();  // peers' barriers initialised; U in tensor memory
  tc::fence_after_sync();

  constexpr uint32_t SB_R = (R / 8) * 128;    // N-direction core stride of the K=R V image
  int issued = 0;                             // TMA sub-tile loads issued (thread 0)
  if (warp == 0) {
    // ================= TMA producer ==========================================
    if (lane == 0) {
      const int total = S * 4;
      for (int g = 0; g < total; ++g) {
        const int slot = g % NST;
        if (g >= NST && !wait_(B(b_empty + slot), (uint32_t)((g / NST - 1) & 1))) break;
        if (aborted()) break;
        const int ls = g >> 2, q = g & 3;
        tc::mbar_arrive_expect_tx(B(b_full + slot), kSubBytes);
        tc::tma_load_2d(sbase + L::RING + slot * kSubBytes, tmp, (int)row0,
                        (int)(strip_col0(ls) + kSubCols * q), B(b_full + slot));
        issued = g + 1;
      }
    }
  } else if (warp == 1) {
    // ================= MMA issuer: GEMM1 and GEMM2 ============================
    if (lane == 0) {
      const bool img_ok = wait_(B(b_img), 0);
      const uint32_t idesc1 = tc::idesc_f16(128, kFW, 0, 0);
      const uint32_t idesc2 = tc::idesc_f16(64, R, 1, 0);
      // descriptors are built once; moving along K adds (bytes >> 4) to the address field
      const uint64_t vdesc0 = tc::smem_desc(sbase + L::VIMG, 128, SB_R);
      const uint64_t cdesc0 = tc::smem_desc(sbase + L::CBUF, 128, kFH * 16);
      const uint64_t wdesc0 = tc::smem_desc(sbase + L::WIMG, 128, kFH * 16);
      for (int i = 0; img_ok && i < S + 1; ++i) {
        if (i < S) {   // GEMM1(i): D1 = U_b V_s^T, terms (hi,hi), (hi,lo), (lo,hi)
          if (!wait_(B(b_vfull), (uint32_t)(i & 1))) break;
          // one D1: the epilogue of strip i-1 has read it
          if (i >= 1 && !wait_(B(b_d1empty), (uint32_t)((i - 1) & 1))) break;
          tc::fence_after_sync();
          const uint64_t vd = vdesc0;
#pragma unroll
          for (int b = 0; b < 2; ++b) {
#pragma unroll
            for (int t = 0; t < 3; ++t) {
              const int tuu = t == 2 ? 1 : 0, tvv = t == 1 ? 1 : 0;
#pragma unroll
              for (int kk = 0; kk < R / 16; ++kk)
                tc::mma_ts(d1 + b * kFW, tu + (uint32_t)((2 * b + tuu) * (R / 2) + kk * 8),
                           vd + (uint64_t)((tvv * (kFW * R * 2) + kk * 256) >> 4), idesc1,
                           (t > 0 || kk > 0) ? 1u : 0u);
            }
          }
          tc::mma_commit(B(b_d1full));
          tc::mma_commit(B(b_vempty));
        }
        if (i >= 1) {   // GEMM2(i-1): Y = C^T W_hi + C^T W_lo (same columns)
          const int s2 = i - 1, q2 = s2 & 1;
          const int pc = s2 % kNC;
          if (!wait_(B(b_cfull + pc), (uint32_t)((s2 / kNC) & 1))) break;
          // two D2 buffers: the exchange has read the result of strip s2-2
          if (s2 >= 2 && !wait_(B(b_d2empty + q2), (uint32_t)(((s2 >> 1) - 1) & 1))) break;
          tc::fence_after_sync();
          const int ps = s2 % kNCS;                       // shared-memory C slot
          const uint64_t cd = cdesc0 + (uint64_t)((ps * L::CBYTES) >> 4);
#pragma unroll
          for (int t = 0; t < 2; ++t) {
#pragma unroll
            for (int kk = 0; kk < kFH / 16; ++kk)
              tc::mma_ss(d2(q2), cd + (uint64_t)((kk * 256) >> 4),
                         wdesc0 + (uint64_t)((t * (R / 8) * (kFH * 16) + kk * 256) >> 4), idesc2,
                         (t > 0 || kk > 0) ? 1u : 0u);
          }
          tc::mma_commit(B(b_d2full + q2));
          tc::mma_commit(B(b_c2free + ps));
        }
      }
      // completes once every MMA this thread issued has completed (drained
      // before tensor memory is released when the kernel gave up)
      tc::mma_commit(B(b_fin1));
    }
  } else if (warp == 2) {
    // ================= MMA issuer: GEMM3 =======================================
    if (lane == 0) {
      const uint32_t idesc3 = tc::idesc_f16(128, R, 0, 0);
      const uint64_t pdesc0 = tc::smem_desc(sbase + L::PIMG, 128, (kFW / 8) * 128);
      for (int s3 = 0; s3 < S; ++s3) {   // P_C += C V'_hi^T + C V'_lo^T
        const int p = s3 & 1;
        tc::mbar_arrive_expect_tx(B(b_pfull + p), (uint32_t)L::PBYTES);
        if (!wait_(B(b_pfull + p), (uint32_t)((s3 >> 1) & 1))) break;
        const int pc = s3 % kNC;
        // the tensor-memory C tile of the strip was written before its cfull
        // phase (already complete: GEMM2 waited for it before the exchange)
        if (!wait_(B(b_cfull + pc), (uint32_t)((s3 / kNC) & 1))) break;
        tc::fence_proxy_async_smem();
        tc::fence_after_sync();
        const uint64_t pd = pdesc0 + (uint64_t)((p * L::PBYTES) >> 4);
#pragma unroll
        for (int b = 0; b < 2; ++b) {
#pragma unroll
          for (int t = 0; t < 2; ++t) {   // V'_hi then V'_lo into the same columns
#pragma unroll
            for (int kk = 0; kk < kFW / 16; ++kk)
              tc::mma_ts(d3 + b * R, tcs(pc) + (uint32_t)(b * 32 + kk * 8),
                         pd + (uint64_t)((t * (R / 8) * (kFW / 8) * 128 + kk * 256) >> 4), idesc3,
                         (s3 > 0 || t > 0 || kk > 0) ? 1u : 0u);
          }
        }
        tc::mma_commit(B(b_cempty + pc));
        tc::mma_commit(B(b_g3done + p));
      }
      // A parity wait only tells the current phase from the previous one, so the
      // final read-out waits on a barrier of its own rather than on g3done.
      tc::mma_commit(B(b_last));
    }
  } else if (warp == 3) {
    // ================= V image (one warp), one strip ahead =====================
    // The next strip's V rows (contiguous, 64 x R floats) are loaded into
    // registers while GEMM1 of the current strip runs.
    constexpr int V4 = kFW * R / 128;           // float4 per lane
    float4 vr[V4];
    auto load_v = [&](int ls) {
      const int64_t col0 = strip_col0(ls);
#pragma unroll
      for (int t = 0; t < V4; ++t) {
        const int e = 4 * (lane + 32 * t), j = e / R, k = e % R;
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
        const int e = 4 * (lane + 32 * t), j = e / R, k = e % R;
        const float x[4] = {vr[t].x, vr[t].y, vr[t].z, vr[t].w};
        __half hi[4], lo[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) split_h(x[u], s_v, hi[u], lo[u]);
        const int off = (j >> 3) * SB_R + (k >> 3) * 128 + (j & 7) * 16 + (k & 7) * 2;
        __half2 h01 = __halves2half2(hi[0], hi[1]), h23 = __halves2half2(hi[2], hi[3]);
        __half2 l01 = __halves2half2(lo[0], lo[1]), l23 = __halves2half2(lo[2], lo[3]);
        *reinterpret_cast<uint2*>(img + off) =
            make_uint2(*reinterpret_cast<uint32_t*>(&h01), *reinterpret_cast<uint32_t*>(&h23));
        *reinterpret_cast<uint2*>(img + kFW * R * 2 + off) =
            make_uint2(*reinterpret_cast<uint32_t*>(&l01), *reinterpret_cast<uint32_t*>(&l23));
      }
      tc::fence_proxy_async_smem();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(B(b_vfull));
      if (ls + 1 < S) load_v(ls + 1);
    }
  } else if (warp < 12) {
    // ================= S-step epilogue (256 threads) ==========================
    const int quarter = warp & 3, rb = (warp - 4) >> 2;
    const int al = quarter * 32 + lane;
    const int arow = rb * 128 + al;
    const float inv_uv = 1.f / (s_u * s_v);
    const float inv_lam = 1.f / a.lam;
    const float2 neg_inv_uv = make_float2(-inv_uv, -inv_uv);
    const float2 inv_lam2 = make_float2(inv_lam, inv_lam);
    const float2 minus_half = make_float2(-0.5f, -0.5f);
    float hub_hi = 0.f, hub_lo = 0.f;
    bool ok = true;   // warp-uniform; false once a wait of this warp has failed
    for (int ls = 0; ls < S; ++ls) {
      const int pc = ls % kNC, ps = ls % kNCS;
      // D1 of the strip, the tensor-memory C slot (GEMM3 of strip ls-kNC has
      // completed: without this the tcgen05.st below would race GEMM3's reads
      // of the slot) and the shared-memory C slot (GEMM2 of strip ls-kNCS);
      // one answer for the warp, which issues warp-wide tcgen05 loads and stores
      bool w_ok = wait_(B(b_d1full), (uint32_t)(ls & 1));
      if (w_ok && ls >= kNC) w_ok = wait_(B(b_cempty + pc), (uint32_t)(((ls / kNC) - 1) & 1));
      if (w_ok && ls >= kNCS) w_ok = wait_(B(b_c2free + ps), (uint32_t)(((ls / kNCS) - 1) & 1));
      if (!__all_sync(0xffffffffu, w_ok)) {
        ok = false;
        break;
      }
      tc::fence_after_sync();
      uint8_t* cbuf = smem + L::CBUF + ps * L::CBYTES;
      const uint32_t tcrow = tcs(pc) + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(rb * 32);
      float2 hub = make_float2(0.f, 0.f);   // even and odd columns
      // Software-pipelined over the 4 sub-tiles: the loads of sub-tile q+1 (D1
      // from tensor memory, M from the ring) are in flight while sub-tile q is
      // computed and stored.
      float dv[2][16], mv[2][16];
      // A failed wait for an M sub-tile leaves garbage in this strip (it is
      // never handed on) but nothing is issued that could race an MMA: D1 and
      // both C slots were waited for above.  m_ok is this lane's view; lane 0's
      // decides the arrivals, the warp's vote at the end of the strip the rest.
      bool m_ok = true;
      auto load_sub = [&](int q, float* d, float* mm) {
        const int g = ls * 4 + q;
        const int rs = g % NST;
        if (!wait_(B(b_full + rs), (uint32_t)((g / NST) & 1))) m_ok = false;
        const float* msub = reinterpret_cast<const float*>(smem + L::RING + rs * kSubBytes);
        tc::tmem_ld16(d1 + ((uint32_t)(quarter * 32) << 16) + rb * kFW + q * kSubCols, d);
#pragma unroll
        for (int jj = 0; jj < 16; ++jj) mm[jj] = msub[jj * kSubRows + arow];
      };
      auto release_sub = [&](int q) {   // after tcgen05.wait::ld: D1 and M of sub-tile q read
        if (q == 3) {   // this warp's last read of D1: GEMM1 of the next strip may start
          tc::fence_before_sync();
          __syncwarp();
          if (lane == 0 && m_ok) tc::mbar_arrive(B(b_d1empty));
        }
        __syncwarp();
        if (lane == 0 && m_ok) tc::mbar_arrive(B(b_empty + (ls * 4 + q) % NST));
      };
      load_sub(0, dv[0], mv[0]);
      tc::tmem_ld_wait();
      release_sub(0);
#pragma unroll
      for (int q = 0; q < 4; ++q) {   // sub-tile q: columns 16q .. 16q+15 of the strip
        const int cb = q & 1;
        if (q < 3) load_sub(q + 1, dv[cb ^ 1], mv[cb ^ 1]);
        uint32_t packed[8];
#pragma unroll
        for (int jj = 0; jj < 16; jj += 2) {   // two columns per packed instruction
          const float2 m2 = make_float2(mv[cb][jj], mv[cb][jj + 1]);
          const float2 d2 = make_float2(dv[cb][jj], dv[cb][jj + 1]);
          const float2 rn = fmul2(ffma2(d2, neg_inv_uv, m2), inv_lam2);    // R / lambda
          const float2 c = make_float2(fminf(fmaxf(rn.x, -1.f), 1.f),      // C / lambda
                                       fminf(fmaxf(rn.y, -1.f), 1.f));
          hub = ffma2(c, ffma2(c, minus_half, rn), hub);                   // H(R) / lambda^2
          __half2 h2 = __floats2half2_rn(c.x, c.y);
          packed[jj / 2] = *reinterpret_cast<uint32_t*>(&h2);
        }
#pragma unroll
        for (int ch = 0; ch < 2; ++ch) {
          const int j8 = (q * kSubCols + ch * 8) >> 3;
          const int off = j8 * (kFH * 16) + (arow >> 3) * 128 + (arow & 7) * 16;
          *reinterpret_cast<uint4*>(cbuf + off) =
              make_uint4(packed[4 * ch], packed[4 * ch + 1], packed[4 * ch + 2], packed[4 * ch + 3]);
        }
        // GEMM3's copy: row arow, K pairs (16q + 2w, 16q + 2w + 1) in column 8q + w
        tc::tmem_st8(tcrow + (uint32_t)(q * 8), packed);
        if (q < 3) {
          tc::tmem_ld_wait();
          release_sub(q + 1);
        }
      }
      tc::tmem_st_wait();
      tsum(hub_hi, hub_lo, hub.x + hub.y);
      if (!__all_sync(0xffffffffu, m_ok)) {   // this strip's C tiles are never handed on
        ok = false;
        break;
      }
      tc::fence_before_sync();
      tc::fence_proxy_async_smem();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(B(b_cfull + pc));
    }
    // P partial of this cluster's columns (after the last GEMM3; its issuer
    // commits b_last after its final MMA whether or not it gave up)
    if (ok && wait_w(B(b_last), 0)) {
      tc::fence_after_sync();
      const int64_t grow = row0 + arow;
      float pv[R];
#pragma unroll
      for (int c = 0; c < R; c += 16)
        tc::tmem_ld16(d3 + ((uint32_t)(quarter * 32) << 16) + rb * R + c, pv + c);
      tc::tmem_ld_wait();
      if (grow < a.m) {
        const float ps = a.lam / s_v;
        float* out = a.part_p + ((int64_t)cid * a.m + grow) * R;
#pragma unroll
        for (int k = 0; k < R; ++k) out[k] = S > 0 ? pv[k] * ps : 0.f;
      }
    }
    double hsum = ((double)hub_hi + (double)hub_lo) * (double)a.lam * (double)a.lam;
    for (int o = 16; o > 0; o >>= 1) hsum += __shfl_xor_sync(0xffffffffu, hsum, o);
    if (lane == 0) red[warp - 4] = hsum;
  } else {
    // ================= exchange: two groups of 128 threads =====================
    const int grp = (warp - 12) >> 2;    // 0: even strips, 1: odd strips
    const int xt = tid - 384 - 128 * grp;
    const int xw = warp & 3;             // == TMEM lane quarter
    const int nb = 1 + grp;              // named barrier of the group
    const int p = grp;                   // every strip of the group uses buffers [p]
    const float y_scale = a.lam / s_w;
    float vmax = 0.f;
    const bool act = xt < kChunk * R;
    const int jl = xt / R, kx = xt % R;
    auto vz_of = [&](int ls, int ci) {
      const int64_t col = strip_col0(ls) + ((int)crank + ci * cs) * kChunk + jl;
      return (act && col < a.n) ? a.VZ[col * R + kx] : 0.f;
    };
    // RECV[p]: the column sums this CTA reduces, [chunk ci][source][column jl][k]
    const uint32_t rbase = sbase + L::YPART + p * L::YBYTES;
    const float* recv = reinterpret_cast<const float*>(smem + L::YPART + p * L::YBYTES);
    const uint32_t pbase = sbase + L::PIMG + p * L::PBYTES;
    float vz_next = grp < S ? vz_of(grp, 0) : 0.f;
    for (int ls = grp; ls < S; ls += 2) {
      const uint32_t par = (uint32_t)((ls >> 1) & 1);
      const float vz_first = vz_next;
      if (ls + 2 < S) vz_next = vz_of(ls + 2, 0);   // in flight for a whole strip pair
      // Once the CTA has given up, the loop still runs to its end so that the
      // group's named barriers stay matched, but every wait returns at once
      // and nothing guarded by a failed wait is issued (tcgen05.ld, st.async,
      // remote arrivals).  The guard of the warp-wide tcgen05.ld is the warp's
      // vote; the others guard per-thread operations.
      // ---- column sums of this CTA's rows out of tensor memory ----
      const int q2 = ls & 1;                      // D2 buffer of the strip (== grp)
      const bool d2ok = wait_w(B(b_d2full + q2), (uint32_t)((ls >> 1) & 1));
      float yv[R];
      if (d2ok) {
        tc::fence_after_sync();
#pragma unroll
        for (int c = 0; c < R; c += 16)
          tc::tmem_ld16(d2(q2) + ((uint32_t)(xw * 32) << 16) + c, yv + c);
        tc::tmem_ld_wait();
        tc::fence_before_sync();
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(B(b_d2empty + q2));
      } else {
#pragma unroll
        for (int c = 0; c < R; ++c) yv[c] = 0.f;
      }
      // ---- send them to their reducers (every reducer has consumed strip ls-2) ----
      const bool yfree_ok = (ls < 2 || wait_(B(b_yfree + p), par ^ 1u)) && d2ok;
      if (yfree_ok && lane < 16) {
        const int j = xw * 16 + lane;               // strip column of this thread
        const int cc = j / kChunk, owner = cc % cs, ci = cc / cs, jj = j % kChunk;
        const uint32_t off = (uint32_t)(((ci * cs + (int)crank) * kChunk + jj) * R) * 4;
        const uint32_t dst = tc::map_cluster(rbase + off, (uint32_t)owner);
        const uint32_t bar = tc::map_cluster(B(b_yfull + p), (uint32_t)owner);
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
      // ---- GEMM3 of strip ls-2 done here: its V' image buffer may be refilled ----
      if (ls >= 2 && xw == 0) {
        if (wait_(B(b_g3done + p), par ^ 1u) && lane < cs)
          tc::mbar_arrive_cluster_relaxed(B(b_pfree + p), (uint32_t)lane);
      }
      // ---- reduce this CTA's chunks of strip ls ----
      if (xt == 0) tc::mbar_arrive_expect_tx(B(b_yfull + p), (uint32_t)L::YBYTES);
      const int64_t col0 = strip_col0(ls);
      const bool yfull_ok = wait_(B(b_yfull + p), par);
      bool pfree_ok = true;
      for (int ci = 0; ci < nch; ++ci) {
        const int cc = (int)crank + ci * cs;
        float y = ci == 0 ? vz_first : vz_of(ls, ci);
        if (act) {
          const float* src = recv + (size_t)ci * cs * kChunk * R + jl * R + kx;
          for (int s2 = 0; s2 < cs; ++s2) y += src[(size_t)s2 * kChunk * R];
        }
        if (ci == nch - 1) {
          // every read of this strip's sums is done (the values are in registers)
          tc::named_bar(nb, 128);
          if (yfull_ok && xt < cs) tc::mbar_arrive_cluster_relaxed(B(b_yfree + p), (uint32_t)xt);
        }
        if (act) {
          const int64_t col = col0 + cc * kChunk + jl;
          const float v = col < a.n ? y : 0.f;
          if (col < a.n) a.Vnew[col * R + kx] = v;
          vmax = fmaxf(vmax, fabsf(v));
          __half hi, lo;
          split_h(v, s_v, hi, lo);
          // chunk image: entry (n, jl) at n*8 + jl*2, n = k (hi) or R + k (lo)
          uint8_t* stg = smem + L::STG + grp * (2 * R * kChunk * 2);
          *reinterpret_cast<__half*>(stg + kx * 8 + jl * 2) = hi;
          *reinterpret_cast<__half*>(stg + (R + kx) * 8 + jl * 2) = lo;
        }
        // all-gather of the chunk's V' image into every CTA (after their GEMM3 of ls-2)
        if (ci == 0 && ls >= 2) pfree_ok = wait_(B(b_pfree + p), par ^ 1u);
        tc::named_bar(nb, 128);
        const uint8_t* stg = smem + L::STG + grp * (2 * R * kChunk * 2);
        const bool send = pfree_ok && !aborted();
        for (int idx = xt; send && idx < cs * 2 * R; idx += 128) {
          const int p2 = idx / (2 * R), nn = idx % (2 * R);
          const uint2 v = *reinterpret_cast<const uint2*>(stg + nn * 8);
          const uint32_t dst = pbase + (nn >> 3) * (kFW / 8) * 128 + (cc >> 1) * 128 +
                               (nn & 7) * 16 + (cc & 1) * 8;
          tc::st_async_u32x2(tc::map_cluster(dst, p2), v.x, v.y,
                             tc::map_cluster(B(b_pfull + p), (uint32_t)p2));
        }
        tc::named_bar(nb, 128);   // the staging chunk is reused by the next chunk
      }
    }
    for (int o = 16; o > 0; o >>= 1) vmax = fmaxf(vmax, __shfl_xor_sync(0xffffffffu, vmax, o));
    if (lane == 0 && vmax > 0.f) atomicMax(a.vmax_out, __float_as_uint(vmax));
  }

  if (err) atomicExch(a.err, DCF_ETIMEOUT);
  tc::fence_before_sync();
  __syncthreads();
  // Every role has left its loop, so the flag is final and the same for all
  // threads.  After an expiry, drain what may still be in flight before the
  // tensor memory is released and the CTA leaves: the W image copy and the
  // last TMA load of every ring slot (thread 0 issued them), and the final
  // commits of both MMA issuers (all of their MMAs have completed).
  bool tmem_free_ok = true;
  if (*abort_flag != 0) {
    const uint64_t dl = tc::globaltimer_ns() + 100000000ull;
    if (tid == 0) {
      tc::mbar_wait_deadline(B(b_img), 0, dl);
      for (int slot = 0; slot < NST && slot < issued; ++slot) {
        const int g_last = slot + ((issued - 1 - slot) / NST) * NST;
        tc::mbar_wait_deadline(B(b_full + slot), (uint32_t)((g_last / NST) & 1), dl);
      }
    }
    if (warp == 1) {
      int drained = 1;
      if (lane == 0)
        drained = tc::mbar_wait_deadline(B(b_fin1), 0, dl) &&
                  tc::mbar_wait_deadline(B(b_last), 0, dl);
      tmem_free_ok = __shfl_sync(0xffffffffu, drained, 0) != 0;
    }
    __syncthreads();
  }
  if (tid == 0) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += red[w];
    a.part_h[cid * cs + (int)crank] = t;
  }
  // (if an MMA is still running after all that, the tensor memory stays allocated)
  if (warp == 1 && tmem_free_ok) tc::tmem_dealloc(tbase, 512);
  tc::cluster_sync();  // no CTA leaves while a peer may still address its shared memory
}

// ---------------------------------------------------------------------------
// Per-iteration preparation: W rows, fp16 hi/lo images of U and W per 256-row
// slab with power-of-two scales, Z = I - rho G^{-1}, and the V scale.
// ---------------------------------------------------------------------------
// Dynamic shared memory of the preparation kernels: G^{-1} (R x R floats),
// the W image staging (2R x 256 fp16), 16 floats of reductions.
template <int R>
constexpr int prep_smem() {
  return 2 * R * R * 4 + 2 * R * kFH * 2 + 16 * 4;
}

// Row l of W for the thread's row u: sum_k u_k (gi + gl)[k][l] with
// compensated products (Dot2; the lo part of G^{-1} into the error term).
template <int R>
__device__ __forceinline__ float w_entry_df(const float (&u)[R], const float* gi, const float* gl,
                                            int l) {
  float s = 0.f, e = 0.f;
#pragma unroll
  for (int k = 0; k < R; ++k) {
    const float g = gi[k * R + l];
    const float p = u[k] * g;
    const float pe = fmaf(u[k], g, -p);
    const float t = s + p;
    const float bp = t - s;
    e += ((s - (t - bp)) + (p - bp)) + pe;
    e = fmaf(u[k], gl[k * R + l], e);
    s = t;
  }
  return s + e;
}

// One 256-row slab (block-wide, 256 threads).  df (ill-conditioned U^T U +
// rho I): W = U G^{-1} with compensated products against the double-float
// G^{-1}, formed twice (for the scale, then for the image) so that no row of
// W is held in registers; otherwise FP32 products with the hi part.
template <int R>
__device__ __forceinline__ void fused_prep_slab(const float* __restrict__ U, const Smalls* sm,
                                                int64_t m, int nslabs, float rho,
                                                const unsigned int* vmax_in,
                                                unsigned int* vmax_reset, uint8_t* img,
                                                float* scales, float* zmat, int slab, bool df) {
  extern __shared__ __align__(16) uint8_t psm[];
  float* gi = reinterpret_cast<float*>(psm);       // G^{-1} = gi + gl (double-float)
  float* gl = gi + R * R;
  uint8_t* wst = psm + 2 * R * R * 4;
  float(*red)[8] = reinterpret_cast<float(*)[8]>(wst + 2 * R * kFH * 2);
  const int tid = threadIdx.x;
  for (int i = tid; i < R * R; i += 256) {
    gi[i] = sm->ginv32[i];
    gl[i] = sm->ginv32_lo[i];
  }
  __syncthreads();
  const int64_t arow = (int64_t)slab * kFH + tid;
  float u[R], w[R];
  float umax = 0.f, wmax = 0.f;
#pragma unroll
  for (int k = 0; k < R; ++k) {
    u[k] = arow < m ? U[arow * R + k] : 0.f;
    umax = fmaxf(umax, fabsf(u[k]));
  }
  if (df) {
#pragma unroll 1
    for (int l = 0; l < R; ++l) wmax = fmaxf(wmax, fabsf(w_entry_df<R>(u, gi, gl, l)));
  } else {
#pragma unroll
    for (int l = 0; l < R; ++l) {
      float s = 0.f;
#pragma unroll
      for (int k = 0; k < R; ++k) s = fmaf(u[k], gi[k * R + l], s);
      w[l] = s;
      wmax = fmaxf(wmax, fabsf(s));
    }
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
  // U image for tensor memory: row a -> R/2 words of fp16 hi pairs, then R/2 of lo pairs
  {
    uint32_t wh[R / 2], wl[R / 2];
#pragma unroll
    for (int i = 0; i < R / 2; ++i) {
      __half h0, l0, h1, l1;
      split_h(u[2 * i], s_u, h0, l0);
      split_h(u[2 * i + 1], s_u, h1, l1);
      __half2 hh = __halves2half2(h0, h1), ll = __halves2half2(l0, l1);
      wh[i] = *reinterpret_cast<uint32_t*>(&hh);
      wl[i] = *reinterpret_cast<uint32_t*>(&ll);
    }
    uint4* row = reinterpret_cast<uint4*>(dst + (size_t)tid * R * 4);
#pragma unroll
    for (int i = 0; i < R / 8; ++i) {
      row[i] = make_uint4(wh[4 * i], wh[4 * i + 1], wh[4 * i + 2], wh[4 * i + 3]);
      row[R / 8 + i] = make_uint4(wl[4 * i], wl[4 * i + 1], wl[4 * i + 2], wl[4 * i + 3]);
    }
  }
  // W image: entry (n, a), n < R -> W_hi[a, n], n >= R -> W_lo[a, n-R]:
  //   (n/8)*(256*16) + (a/8)*128 + (n%8)*16 + (a%8)*2
  const int wbase = (tid >> 3) * 128 + (tid & 7) * 2;
  auto put_w = [&](int k, float v) {
    __half hi, lo;
    split_h(v, s_w, hi, lo);
    *reinterpret_cast<__half*>(wst + (k >> 3) * (kFH * 16) + (k & 7) * 16 + wbase) = hi;
    *reinterpret_cast<__half*>(wst + ((R + k) >> 3) * (kFH * 16) + (k & 7) * 16 + wbase) = lo;
  };
  if (df) {
#pragma unroll 1
    for (int k = 0; k < R; ++k) put_w(k, w_entry_df<R>(u, gi, gl, k));
  } else {
#pragma unroll
    for (int k = 0; k < R; ++k) put_w(k, w[k]);
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
      zmat[i] = fmaf(-rho, gl[i], fmaf(-rho, gi[i], (i / R) == (i % R) ? 1.f : 0.f));
    if (tid == 0) {
      const float vm = __uint_as_float(*vmax_in);
      scales[2 * nslabs] = pow2_scale_dev(vm, 1024.f);
      *vmax_reset = 0u;
    }
  }
}

// Batches: item (instance, slab), a persistent grid walks the list.
template <int R>
__global__ void __launch_bounds__(256) k_bfused_prep(const BInst* __restrict__ insts,
                                                     const BItem* __restrict__ items, int nitems,
                                                     int cur) {
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const BItem w = items[it];
    const BInst& I = insts[w.inst];
    if (I.st->stop) continue;            // uniform over the block
    __syncthreads();                     // the previous item's shared memory is free
    fused_prep_slab<R>(I.U[cur], I.sm, I.m, I.nslabs, I.rho, I.vmax + cur, I.vmax + (cur ^ 1),
                       I.img, I.scales, I.zmat, w.a, df_route(I.st));
  }
}

// out = in Z for n rows of R (V_old Z, added to the cluster's column sums),
// in entries (row, column group of 8), 256 per chunk.  The row's R inputs are
// fetched with vector loads before any arithmetic, so that they are in
// flight together.
// rowmat_fill_z: Z into shared memory; kFromGinv: zsrc, zlo are G^{-1} =
// zsrc + zlo (double-float) and Z = I - rho G^{-1} is formed here (as the
// preparation forms zmat); otherwise zsrc is Z itself.  Block-wide.
template <int R, bool kFromGinv>
__device__ __forceinline__ void rowmat_fill_z(float* Z, const float* __restrict__ zsrc,
                                              const float* __restrict__ zlo, float rho) {
  if constexpr (kFromGinv) {
    for (int i = threadIdx.x; i < R * R; i += 256)
      Z[i] = fmaf(-rho, zlo[i], fmaf(-rho, zsrc[i], (i / R) == (i % R) ? 1.f : 0.f));
  } else {
    for (int i = threadIdx.x; i < R * R / 4; i += 256)
      reinterpret_cast<float4*>(Z)[i] = reinterpret_cast<const float4*>(zsrc)[i];
  }
}

// Entry idx of out = in Z (nothing past row n).
template <int R>
__device__ __forceinline__ void rowmat_entry(const float* __restrict__ in, const float* Z,
                                             int64_t n, float* __restrict__ out, int64_t idx) {
  const int64_t row = idx / (R / 8);
  const int cg = (int)(idx % (R / 8));
  if (row >= n) return;
  float v[R];
  const float4* src = reinterpret_cast<const float4*>(in + row * R);
#pragma unroll
  for (int k = 0; k < R / 4; ++k) {
    const float4 t = src[k];
    v[4 * k] = t.x; v[4 * k + 1] = t.y; v[4 * k + 2] = t.z; v[4 * k + 3] = t.w;
  }
  float acc[8];
#pragma unroll
  for (int l = 0; l < 8; ++l) acc[l] = 0.f;
#pragma unroll
  for (int k = 0; k < R; ++k) {
    const float4 z0 = *reinterpret_cast<const float4*>(Z + k * R + cg * 8);
    const float4 z1 = *reinterpret_cast<const float4*>(Z + k * R + cg * 8 + 4);
    acc[0] = fmaf(v[k], z0.x, acc[0]);
    acc[1] = fmaf(v[k], z0.y, acc[1]);
    acc[2] = fmaf(v[k], z0.z, acc[2]);
    acc[3] = fmaf(v[k], z0.w, acc[3]);
    acc[4] = fmaf(v[k], z1.x, acc[4]);
    acc[5] = fmaf(v[k], z1.y, acc[5]);
    acc[6] = fmaf(v[k], z1.z, acc[6]);
    acc[7] = fmaf(v[k], z1.w, acc[7]);
  }
  float4* dst = reinterpret_cast<float4*>(out + row * R + cg * 8);
  dst[0] = make_float4(acc[0], acc[1], acc[2], acc[3]);
  dst[1] = make_float4(acc[4], acc[5], acc[6], acc[7]);
}

// Row `row` of out = in Z with all R outputs in one thread (R <= 32: the row
// and its sums fit in registers; Z by broadcast from shared memory).  The sums
// run over k in the order of rowmat_entry, so both give the same bits.
template <int R>
__device__ __forceinline__ void rowmat_row(const float* __restrict__ in, const float* Z, int64_t n,
                                           float* __restrict__ out, int64_t row) {
  static_assert(R <= 32, "registers");
  if (row >= n) return;
  float v[R];
  const float4* src = reinterpret_cast<const float4*>(in + row * R);
#pragma unroll
  for (int k = 0; k < R / 4; ++k) {
    const float4 t = src[k];
    v[4 * k] = t.x; v[4 * k + 1] = t.y; v[4 * k + 2] = t.z; v[4 * k + 3] = t.w;
  }
  float acc[R];
#pragma unroll
  for (int l = 0; l < R; ++l) acc[l] = 0.f;
#pragma unroll
  for (int k = 0; k < R; ++k) {
#pragma unroll
    for (int l4 = 0; l4 < R / 4; ++l4) {
      const float4 z = *reinterpret_cast<const float4*>(Z + k * R + 4 * l4);
      acc[4 * l4] = fmaf(v[k], z.x, acc[4 * l4]);
      acc[4 * l4 + 1] = fmaf(v[k], z.y, acc[4 * l4 + 1]);
      acc[4 * l4 + 2] = fmaf(v[k], z.z, acc[4 * l4 + 2]);
      acc[4 * l4 + 3] = fmaf(v[k], z.w, acc[4 * l4 + 3]);
    }
  }
  float4* dst = reinterpret_cast<float4*>(out + row * R);
#pragma unroll
  for (int l4 = 0; l4 < R / 4; ++l4)
    dst[l4] = make_float4(acc[4 * l4], acc[4 * l4 + 1], acc[4 * l4 + 2], acc[4 * l4 + 3]);
}

// One chunk blk of 256 entries (block-wide).
template <int R, bool kFromGinv = false>
__device__ __forceinline__ void rowmat_block(const float* __restrict__ in,
                                             const float* __restrict__ zsrc,
                                             const float* __restrict__ zlo, float rho, int64_t n,
                                             float* __restrict__ out, int64_t blk) {
  __shared__ __align__(16) float Z[R * R];
  rowmat_fill_z<R, kFromGinv>(Z, zsrc, zlo, rho);
  __syncthreads();
  rowmat_entry<R>(in, Z, n, out, blk * 256 + threadIdx.x);
}

// V_old Z at R = 64 in its own launch (the preparation's slab part takes every
// register there) as a register-tiled product: a CTA walks tiles of 64 rows,
// staged in shared memory by cp.async (two stages, the next tile in flight),
// and thread (row group rg, output group og) forms a 4 x 4 block of outputs
// with 16 FMAs per two 16-byte shared loads.  Z = I - rho G^{-1} is formed once
// per CTA.  Every output sums over k in order, as rowmat_entry does.
constexpr int kRm64Rows = 64;
constexpr int kRm64Ld = 68;                       // row stride (floats): 16-byte rows
constexpr size_t kRm64Smem = (64 * 64 + 2 * kRm64Rows * kRm64Ld) * sizeof(float);

__global__ void __launch_bounds__(256) k_rowmat64(const DevState* st, const Smalls* sm, float rho,
                                                  const float* __restrict__ Vold, int64_t n,
                                                  float* __restrict__ VZ) {
  if (st->stop) return;
  extern __shared__ __align__(16) float rsh[];
  float* Z = rsh;                                 // [64][64]
  float* Vs = rsh + 64 * 64;                      // [2][64 rows][68]
  const int tid = threadIdx.x;
  const int rg = tid >> 4, og = tid & 15;
  const int64_t ntiles = (n + kRm64Rows - 1) / kRm64Rows;
  auto stage = [&](int64_t tile, int b) {
    float* dst = Vs + b * kRm64Rows * kRm64Ld;
    const int64_t r0 = tile * kRm64Rows;
    for (int i = tid; i < kRm64Rows * 16; i += 256) {   // 16 float4 per row
      const int r = i >> 4, c4 = i & 15;
      const bool ok = r0 + r < n;
      const float* src = ok ? Vold + (r0 + r) * 64 + 4 * c4 : Vold;
      const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst + r * kRm64Ld + 4 * c4);
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(src),
                   "r"(ok ? 16 : 0)
                   : "memory");
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };
  int64_t tile = blockIdx.x;
  if (tile < ntiles) stage(tile, 0);
  rowmat_fill_z<64, true>(Z, sm->ginv32, sm->ginv32_lo, rho);
  for (int b = 0; tile < ntiles; tile += gridDim.x, b ^= 1) {
    const int64_t next = tile + gridDim.x;
    if (next < ntiles) {
      stage(next, b ^ 1);
      asm volatile("cp.async.wait_group 1;" ::: "memory");
    } else {
      asm volatile("cp.async.wait_group 0;" ::: "memory");
    }
    __syncthreads();
    const float* V = Vs + b * kRm64Rows * kRm64Ld + (4 * rg) * kRm64Ld;
    float acc[4][4];
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int o = 0; o < 4; ++o) acc[j][o] = 0.f;
#pragma unroll 4
    for (int k4 = 0; k4 < 16; ++k4) {
      float4 v[4], z[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) v[j] = *reinterpret_cast<const float4*>(V + j * kRm64Ld + 4 * k4);
#pragma unroll
      for (int i = 0; i < 4; ++i)
        z[i] = *reinterpret_cast<const float4*>(Z + (4 * k4 + i) * 64 + 4 * og);
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const float vk[4] = {v[j].x, v[j].y, v[j].z, v[j].w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          acc[j][0] = fmaf(vk[i], z[i].x, acc[j][0]);
          acc[j][1] = fmaf(vk[i], z[i].y, acc[j][1]);
          acc[j][2] = fmaf(vk[i], z[i].z, acc[j][2]);
          acc[j][3] = fmaf(vk[i], z[i].w, acc[j][3]);
        }
      }
    }
    const int64_t r0 = tile * kRm64Rows + 4 * rg;
#pragma unroll
    for (int j = 0; j < 4; ++j)
      if (r0 + j < n)
        *reinterpret_cast<float4*>(VZ + (r0 + j) * 64 + 4 * og) =
            make_float4(acc[j][0], acc[j][1], acc[j][2], acc[j][3]);
    __syncthreads();   // stage b is refilled two tiles on
  }
}

// The per-iteration preparation in one launch: blocks [0, nslabs) prepare the
// U/W slabs (fused_prep_slab), the other blocks form V_old Z for 256 (row,
// column group of 8) entries each, with Z = I - rho G^{-1} built in place.
template <int R>
__global__ void __launch_bounds__(256) k_fused_prep(const float* __restrict__ U,
                                                    const Smalls* sm, const DevState* st,
                                                    int64_t m, int nslabs, float rho,
                                                    const unsigned int* vmax_in,
                                                    unsigned int* vmax_reset, uint8_t* img,
                                                    float* scales, float* zmat,
                                                    const float* __restrict__ Vold, int64_t n,
                                                    float* __restrict__ VZ) {
  if (st->stop) return;
  if ((int)blockIdx.x < nslabs)
    fused_prep_slab<R>(U, sm, m, nslabs, rho, vmax_in, vmax_reset, img, scales, zmat,
                       (int)blockIdx.x, df_route(st));
  else
    rowmat_block<R, true>(Vold, sm->ginv32, sm->ginv32_lo, rho, n, VZ,
                          (int64_t)blockIdx.x - nslabs);
}

// Batches: item (instance, block of 256 rows of V_old Z), one row per thread.
template <int R>
__global__ void __launch_bounds__(256) k_browmat(const BInst* __restrict__ insts,
                                                 const BItem* __restrict__ items, int nitems,
                                                 int cur) {
  __shared__ __align__(16) float Z[R * R];
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const BItem w = items[it];
    const BInst& I = insts[w.inst];
    if (I.st->stop) continue;            // uniform over the block
    __syncthreads();                     // the previous item's shared Z is free
    rowmat_fill_z<R, false>(Z, I.zmat, nullptr, 0.f);
    __syncthreads();
    rowmat_row<R>(I.V[cur], Z, I.n, I.VZ, (int64_t)w.a * 256 + threadIdx.x);
  }
}

cudaError_t launch_bfused_small(int R, int kind, const BInst* insts, const BItem* items,
                                int nitems, int grid, int cur, cudaStream_t s) {
  if (nitems == 0) return cudaSuccess;
  if (kind == 0) {
    if (R == 16) k_bfused_prep<16><<<grid, 256, prep_smem<16>(), s>>>(insts, items, nitems, cur);
    else k_bfused_prep<32><<<grid, 256, prep_smem<32>(), s>>>(insts, items, nitems, cur);
  } else {
    if (R == 16) k_browmat<16><<<grid, 256, 0, s>>>(insts, items, nitems, cur);
    else k_browmat<32><<<grid, 256, 0, s>>>(insts, items, nitems, cur);
  }
  return cudaGetLastError();
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
constexpr int kNST32 = 5;
constexpr int kNST16 = 7;

template <int R, int NST>
static size_t fused_smem() {
  return FL<R, NST>::TOTAL;
}

template <int R, int NST, bool kTable>
static cudaError_t prep_attr1() {
  cudaError_t e = cudaFuncSetAttribute(k_fused<R, NST, kTable>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)fused_smem<R, NST>());
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_fused<R, NST, kTable>,
                              cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
}
template <int R, int NST>
static cudaError_t prep_attr() {
  cudaError_t e = prep_attr1<R, NST, false>();
  return e != cudaSuccess ? e : prep_attr1<R, NST, true>();
}

cudaError_t fused_prepare(int R) {
  return R == 16 ? prep_attr<16, kNST16>() : prep_attr<32, kNST32>();
}

template <int R, int NST>
static int max_clusters_T(int cs) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(cs, 1, 1);
  cfg.blockDim = dim3(kFThreads, 1, 1);
  cfg.dynamicSmemBytes = fused_smem<R, NST>();
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = cs;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, (void*)k_fused<R, NST, false>, &cfg) != cudaSuccess) {
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

// 2-D tensor map over column-major M (dim 0 = rows, contiguous), 256 x 16 boxes.
int fused_make_tmap(void* tmap_out, const float* M, int64_t m, int64_t n) {
  auto fn = encode_fn();
  if (!fn) return -1;
  cuuint64_t dims[2] = {(cuuint64_t)m, (cuuint64_t)n};
  cuuint64_t strides[1] = {(cuuint64_t)m * sizeof(float)};
  cuuint32_t box[2] = {(cuuint32_t)kSubRows, (cuuint32_t)kSubCols};
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
                              const float* Vold, int64_t n, float* VZ, cudaStream_t s) {
  const int64_t zblocks = (n * (R / 8) + 255) / 256;    // V_old Z blocks after the slabs
  if (R == 64) {
    // the slabs alone, then V_old Z in its own persistent launch
    k_fused_prep<64><<<(unsigned)nslabs, 256, prep_smem<64>(), s>>>(
        U, sm, st, m, nslabs, rho, vmax_in, vmax_reset, img, scales, zmat, Vold, n, VZ);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t tiles = (n + kRm64Rows - 1) / kRm64Rows;
    const int64_t g = std::max<int64_t>(1, std::min<int64_t>(tiles, 4LL * sms));
    k_rowmat64<<<(unsigned)g, 256, kRm64Smem, s>>>(st, sm, rho, Vold, n, VZ);
    return cudaGetLastError();
  }
  const unsigned grid = (unsigned)(nslabs + zblocks);
  if (R == 16)
    k_fused_prep<16><<<grid, 256, prep_smem<16>(), s>>>(U, sm, st, m, nslabs, rho, vmax_in,
                                                        vmax_reset, img, scales, zmat, Vold, n,
                                                        VZ);
  else if (R == 32)
    k_fused_prep<32><<<grid, 256, prep_smem<32>(), s>>>(U, sm, st, m, nslabs, rho, vmax_in,
                                                        vmax_reset, img, scales, zmat, Vold, n,
                                                        VZ);
  return cudaGetLastError();
}

cudaError_t fused_prep_prepare() {
  cudaError_t e = cudaFuncSetAttribute(k_fused_prep<64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       prep_smem<64>());
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_rowmat64, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)kRm64Smem);
}

template <int R, int NST>
static cudaError_t launch_fused_T(const void* tmap, const FusedArgs& fa, cudaStream_t s,
                                  const int* priority) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(fa.cs * fa.nclusters, 1, 1);
  cfg.blockDim = dim3(kFThreads, 1, 1);
  cfg.dynamicSmemBytes = fused_smem<R, NST>();
  cfg.stream = s;
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = fa.cs;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (priority) {
    attr[1].id = cudaLaunchAttributePriority;
    attr[1].val.priority = *priority;
    cfg.numAttrs = 2;
  }
  const CUtensorMap* tm = reinterpret_cast<const CUtensorMap*>(tmap);
  return cudaLaunchKernelEx(&cfg, k_fused<R, NST, false>, *tm, fa,
                            static_cast<const FusedArgs*>(nullptr));
}

cudaError_t launch_fused(int R, const void* tmap, const FusedArgs& fa, cudaStream_t s,
                         const int* priority) {
  return R == 16 ? launch_fused_T<16, kNST16>(tmap, fa, s, priority)
                 : launch_fused_T<32, kNST32>(tmap, fa, s, priority);
}

template <int R, int NST>
static cudaError_t launch_fused_table_T(int cs, int nclusters, const FusedArgs* table,
                                        cudaStream_t s) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(cs * nclusters, 1, 1);
  cfg.blockDim = dim3(kFThreads, 1, 1);
  cfg.dynamicSmemBytes = fused_smem<R, NST>();
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = cs;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  // the parameter-space tensor map is unused in table launches (each entry
  // carries its own); only cs is read from the parameter block
  CUtensorMap unused{};
  FusedArgs ap{};
  ap.cs = cs;
  ap.nclusters = nclusters;
  return cudaLaunchKernelEx(&cfg, k_fused<R, NST, true>, unused, ap, table);
}

cudaError_t launch_fused_table(int R, int cs, int nclusters, const FusedArgs* table,
                               cudaStream_t s) {
  if (nclusters < 1) return cudaSuccess;
  return R == 16 ? launch_fused_table_T<16, kNST16>(cs, nclusters, table, s)
                 : launch_fused_table_T<32, kNST32>(cs, nclusters, table, s);
}

cudaError_t launch_absmax(const float* x, int64_t count, unsigned int* out, cudaStream_t s) {
  int64_t blocks = (count + 255) / 256;
  if (blocks > 1024) blocks = 1024;
  if (blocks < 1) blocks = 1;
  k_absmax<<<(unsigned)blocks, 256, 0, s>>>(x, count, out);
  return cudaGetLastError();
}

}  // namespace dcf
