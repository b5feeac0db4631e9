// Self-test of the tensor-core conventions the fused kernel relies on: one
// tcgen05 MMA (fp16 x fp16 -> FP32 in TMEM) on integer-valued operands whose
// products and sums are exact in FP32, with the operand layout and the
// descriptor fields chosen by the caller.  The whole 128-lane x 256-column
// accumulator region is returned, so a test can check the data-path layout
// of the result (M = 128 and M = 64) as well as the values.
#include <cuda_fp16.h>

#include "dcf.h"
#include "tc_ptx.cuh"

namespace dcf {

struct SelfTestArgs {
  int M, N, K;
  int a_kind;               // 0: smem K-major, 1: smem MN-major, 2: TMEM
  int a_lbo, a_sbo;         // data layout of A (byte strides of core matrices along K / M)
  int da_lbo, da_sbo;       // values written into A's descriptor
  int b_lbo, b_sbo;         // data layout of B (K-major)
  int db_lbo, db_sbo;       // values written into B's descriptor
  float* out;               // [128][256]
  int* status;
};

// Hashed small integers (distinct rows, exact in fp16 and in FP32 sums).
__device__ __forceinline__ float st_a(int i, int k) {
  uint32_t h = (uint32_t)i * 2654435761u ^ (uint32_t)k * 40503u;
  return (float)((int)((h >> 13) % 9u) - 4);
}
__device__ __forceinline__ float st_b(int j, int k) {
  uint32_t h = (uint32_t)j * 2246822519u ^ (uint32_t)k * 3266489917u;
  return (float)((int)((h >> 15) % 7u) - 3);
}

__global__ void __launch_bounds__(128) k_tc_selftest(SelfTestArgs p) {
  extern __shared__ __align__(1024) uint8_t sm[];
  __half* As = reinterpret_cast<__half*>(sm);
  __half* Bs = reinterpret_cast<__half*>(sm + 32768);
  uint64_t* mbar = reinterpret_cast<uint64_t*>(sm + 65536);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + 65536 + 16);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  for (int i = tid; i < 65536 / 4; i += 128) reinterpret_cast<uint32_t*>(sm)[i] = 0u;
  __syncthreads();
  for (int idx = tid; idx < p.M * p.K; idx += 128) {
    int i = idx / p.K, k = idx % p.K;
    int off = p.a_kind == 1 ? (i / 8) * p.a_sbo + (k / 8) * p.a_lbo + (k % 8) * 16 + (i % 8) * 2
                            : (i / 8) * p.a_sbo + (k / 8) * p.a_lbo + (i % 8) * 16 + (k % 8) * 2;
    if (off >= 0 && off + 2 <= 32768) As[off / 2] = __float2half(st_a(i, k));
  }
  for (int idx = tid; idx < p.N * p.K; idx += 128) {
    int j = idx / p.K, k = idx % p.K;
    int off = (j / 8) * p.b_sbo + (k / 8) * p.b_lbo + (j % 8) * 16 + (k % 8) * 2;
    if (off >= 0 && off + 2 <= 32768) Bs[off / 2] = __float2half(st_b(j, k));
  }
  if (warp == 0) {
    tc::tmem_alloc(tc::smem_u32(tslot), 256);
    tc::tmem_relinquish();
  }
  if (tid == 0) {
    tc::mbar_init(tc::smem_u32(mbar), 1);
    tc::fence_mbar_init();
  }
  tc::fence_proxy_async_smem();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t taddr = *tslot;
  if (p.a_kind == 2) {
    // row i = lane (warp*32 + lane); K fp16 values packed two per 32-bit column
    const int i = warp * 32 + lane;
    uint32_t r[16];
#pragma unroll
    for (int c = 0; c < 16; ++c) {
      __half2 h2 = __floats2half2_rn(i < p.M && 2 * c < p.K ? st_a(i, 2 * c) : 0.f,
                                     i < p.M && 2 * c + 1 < p.K ? st_a(i, 2 * c + 1) : 0.f);
      r[c] = *reinterpret_cast<uint32_t*>(&h2);
    }
    tc::tmem_st16(taddr + ((uint32_t)(warp * 32) << 16) + 128u, r);
    tc::tmem_st_wait();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (tid == 0) {
    const uint32_t idesc = tc::idesc_f16(p.M, p.N, p.a_kind == 1 ? 1 : 0, 0);
    const uint32_t a0 = tc::smem_u32(As), b0 = tc::smem_u32(Bs);
    for (int kk = 0; kk < p.K / 16; ++kk) {
      uint64_t bd = tc::smem_desc(b0 + kk * 2 * p.b_lbo, p.db_lbo, p.db_sbo);
      if (p.a_kind == 2) {
        tc::mma_ts(taddr, taddr + 128u + 8u * kk, bd, idesc, kk > 0);
      } else {
        uint64_t ad = tc::smem_desc(a0 + kk * 2 * p.a_lbo, p.da_lbo, p.da_sbo);
        tc::mma_ss(taddr, ad, bd, idesc, kk > 0);
      }
    }
    tc::mma_commit(tc::smem_u32(mbar));
  }
  __syncwarp();
  bool ok = tc::mbar_wait(tc::smem_u32(mbar), 0, 1u << 22);
  if (!ok && lane == 0) atomicExch(p.status, DCF_ETIMEOUT);
  tc::fence_after_sync();
  if (ok) {
    for (int c = 0; c < 8; ++c) {
      float v[16];
      tc::tmem_ld16(taddr + ((uint32_t)(warp * 32) << 16) + (uint32_t)(c * 16), v);
      tc::tmem_ld_wait();
#pragma unroll
      for (int i = 0; i < 16; ++i) p.out[(warp * 32 + lane) * 256 + c * 16 + i] = v[i];
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(taddr, 256);
}

}  // namespace dcf

// Diagnostic entry point (declared in dcf.h).
extern "C" int dcf_tc_selftest(const int* cfg, float* out_host) {
  using namespace dcf;
  if (!cfg || !out_host) return DCF_EINVAL;
  SelfTestArgs a{};
  a.M = cfg[0]; a.N = cfg[1]; a.K = cfg[2]; a.a_kind = cfg[3];
  a.a_lbo = cfg[4]; a.a_sbo = cfg[5]; a.da_lbo = cfg[6]; a.da_sbo = cfg[7];
  a.b_lbo = cfg[8]; a.b_sbo = cfg[9]; a.db_lbo = cfg[10]; a.db_sbo = cfg[11];
  if (!(a.M == 64 || a.M == 128) || a.N < 16 || a.N > 128 || a.N % 16 || a.K < 16 || a.K > 32 ||
      a.K % 16 || a.a_kind < 0 || a.a_kind > 2)
    return DCF_EINVAL;
  for (int i = 4; i < 12; ++i)
    if (cfg[i] < 16 || cfg[i] > 8192 || cfg[i] % 16) return DCF_EINVAL;
  // every address the descriptors can reach must stay inside each 32 KB operand region
  const long reach_a = (long)(a.K / 16 - 1) * 2 * a.a_lbo + (long)(a.K / 8) * a.da_lbo +
                       (long)(a.M / 8) * a.da_sbo + 128;
  const long reach_b = (long)(a.K / 16 - 1) * 2 * a.b_lbo + (long)(a.K / 8) * a.db_lbo +
                       (long)(a.N / 8) * a.db_sbo + 128;
  if ((a.a_kind != 2 && reach_a > 32768) || reach_b > 32768) return DCF_EINVAL;
  float* d_out = nullptr;
  int* d_st = nullptr;
  if (cudaMalloc(&d_out, 128 * 256 * sizeof(float)) != cudaSuccess) return DCF_ENOMEM;
  if (cudaMalloc(&d_st, sizeof(int)) != cudaSuccess) { cudaFree(d_out); return DCF_ENOMEM; }
  cudaMemset(d_out, 0, 128 * 256 * sizeof(float));
  cudaMemset(d_st, 0, sizeof(int));
  a.out = d_out;
  a.status = d_st;
  const int smem = 65536 + 64;
  int rc = DCF_OK;
  if (cudaFuncSetAttribute(k_tc_selftest, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) !=
      cudaSuccess)
    rc = DCF_ECUDA;
  if (rc == DCF_OK) {
    k_tc_selftest<<<1, 128, smem>>>(a);
    if (cudaDeviceSynchronize() != cudaSuccess) rc = DCF_ECUDA;
  }
  int st = 0;
  if (rc == DCF_OK) {
    cudaMemcpy(out_host, d_out, 128 * 256 * sizeof(float), cudaMemcpyDeviceToHost);
    cudaMemcpy(&st, d_st, sizeof(int), cudaMemcpyDeviceToHost);
    if (st) rc = st;
  }
  cudaFree(d_out);
  cudaFree(d_st);
  return rc;
}
