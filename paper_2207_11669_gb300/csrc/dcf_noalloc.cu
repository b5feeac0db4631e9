// dcf_iterate_noalloc: one exact-consensus DCF-PCA iteration on buffers the
// caller owns, with every piece of scratch memory taken from one fixed,
// file-scope device array instead of being allocated.
//
// Who needs this: callers that may not allocate device memory behind their
// own back -- host frameworks that hand out all device memory from their own
// pools and forbid libraries to call cudaMalloc, and latency-critical loops
// where cudaMalloc and cudaFree can synchronise the device.  Such callers hand
// in M, U and V and receive the new U and V; the library allocates nothing on
// this path.
//
// The scratch array lives in the library's device image, so every GPU that
// loads libdcf.so holds kNoAllocScratchBytes of it until the process exits.
// All calls share it: two calls whose work overlaps on the GPU (different
// streams, or different host threads) race on it and must be serialised by
// the caller.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "dcf.h"
#include "dcf_internal.cuh"


using namespace dcf;

namespace {

constexpr size_t kNoAllocScratchBytes = DCF_NOALLOC_SCRATCH_BYTES;

// The scratch itself.  In host code `g_noalloc_scratch` is only a host-side
// stand-in for the symbol: its device address comes from
// cudaGetSymbolAddress, taken once per device with that device current.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
void* g_scratch_addr[kMaxDevices] = {};

// Once per device: resolve the scratch address and raise the kernels'
// shared-memory limits.  Neither step allocates memory.
dcf_status setup_device(int dev, unsigned char** out) {
  if (dev < 0 || dev >= kMaxDevices) return DCF_EINVAL;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return DCF_ECUDA;
    }
    if (prepare_stream_kernels() != cudaSuccess || prepare_small_kernels() != cudaSuccess) {
      cudaGetLastError();
      return DCF_ECUDA;
    }
    g_scratch_addr[dev] = p;
  }
  *out = static_cast<unsigned char*>(g_scratch_addr[dev]);
  return DCF_OK;
}

struct Carve {
  unsigned char* base;
  size_t used = 0;
  void* take(size_t bytes) {
    void* p = base ? base + used : nullptr;
    used += (bytes + 255) / 256 * 256;
    return p;
  }
};

}  // namespace

extern "C" dcf_status dcf_iterate_noalloc(const float* M, int64_t m, int64_t n, int r,
                                          double rho, double lambda, const float* U_in,
                                          const float* V_in, float* U_out, float* V_out,
                                          void* stream) {
  if (!M || !U_in || !V_in || !U_out || !V_out) return DCF_EINVAL;
  if (m < 1 || n < 1 || r < 1 || r > kMaxR || r > m) return DCF_EINVAL;
  if (!(rho > 0) || !(lambda > 0)) return DCF_EINVAL;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return DCF_ECUDA;
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return DCF_ECUDA;
  if (sms < 1) sms = 1;

  // launch geometry of the general two-pass kernels
  const int R = pick_R(r);
  const size_t RR = (size_t)R * R;
  const int64_t nstrips = (n + 63) / 64;
  int n_vblocks = (int)std::min<int64_t>(nstrips, 3LL * sms);
  {
    const int64_t waves = (nstrips + n_vblocks - 1) / n_vblocks;
    n_vblocks = (int)((nstrips + waves - 1) / waves);
  }
  const int64_t rb = (m + 127) / 128;
  int64_t splits = std::max<int64_t>(1, (4LL * sms + rb - 1) / rb);
  splits = std::min<int64_t>(splits, (n + 31) / 32);
  const int64_t split_cols = ((n + splits - 1) / splits + 31) / 32 * 32;
  const int n_splits = (int)((n + split_cols - 1) / split_cols);
  const int n_rblocks = (int)((m + 31) / 32);
  // the same V-Gram partition as the general path of dcf_step (one CTA per SM
  // at R >= 32, two below), so both sum the partials in the same order
  const int n_vgram = (int)std::min<int64_t>((R >= 32 ? 1LL : 2LL) * sms, (n + 31) / 32);
  const size_t ngp = (size_t)std::max(n_vgram, n_rblocks);

  // carve the scratch (a dry run first: reject sizes beyond the array)
  auto layout = [&](Carve& c, IterArgs& a, double** red, unsigned int** counters) {
    a.U[0] = (float*)c.take((size_t)m * R * 4);
    a.U[1] = (float*)c.take((size_t)m * R * 4);
    a.V[0] = (float*)c.take((size_t)n * R * 4);
    a.V[1] = (float*)c.take((size_t)n * R * 4);
    a.W = (float*)c.take((size_t)m * R * 4);
    a.part_p = (float*)c.take((size_t)n_splits * m * R * 4);
    a.part_h = (double*)c.take((size_t)n_vblocks * 8);
    a.part_q = (float2*)c.take(ngp * RR * 8);
    a.part_xv = (float2*)c.take((size_t)n_vgram * RR * 8);
    a.part_dv = (float2*)c.take((size_t)n_vgram * RR * 8);
    a.part_g = (float2*)c.take(ngp * RR * 8);
    a.part_xu = (float2*)c.take((size_t)n_rblocks * RR * 8);
    a.part_du = (float2*)c.take((size_t)n_rblocks * RR * 8);
    *red = (double*)c.take((6 * RR + 8) * 8);
    a.sm = (Smalls*)c.take(sizeof(Smalls));
    a.st = (DevState*)c.take(sizeof(DevState));
    *counters = (unsigned int*)c.take(4 * sizeof(unsigned int));
  };
  IterArgs a{};
  double* red = nullptr;
  unsigned int* counters = nullptr;
  {
    Carve dry{nullptr};
    layout(dry, a, &red, &counters);
    if (dry.used > kNoAllocScratchBytes) return DCF_EINVAL;   // problem too large for the array
  }
  unsigned char* base = nullptr;
  dcf_status st = setup_device(dev, &base);
  if (st != DCF_OK) return st;
  Carve c{base};
  a = IterArgs{};
  layout(c, a, &red, &counters);
  a.cur = 0;
  a.M = M;
  a.m = m;
  a.n = n;
  a.r = r;
  a.R = R;
  a.lam = (float)lambda;
  a.rho = (float)rho;
  a.u_mode = 0;
  a.E = 1;
  a.n_vblocks = n_vblocks;
  a.n_splits = n_splits;
  a.split_cols = split_cols;
  a.n_rblocks = n_rblocks;
  a.add_uxv = 0;
  a.alpha = 1.0f;
  a.ustar_out = nullptr;
  double* red_q = red;
  double* red_xv = red + RR;
  double* red_dv = red + 2 * RR;
  double* red_h = red + 3 * RR;
  double* red_g = red + 3 * RR + 8;
  double* red_xu = red + 4 * RR + 8;
  double* red_du = red + 5 * RR + 8;
  cudaStream_t s = (cudaStream_t)stream;

#define NA_CK(call)                                   \
  do {                                                \
    if ((call) != cudaSuccess) {                      \
      cudaGetLastError();                             \
      return DCF_ECUDA;                               \
    }                                                 \
  } while (0)
  // the array keeps the previous call's contents (possibly of another size or
  // rank): clear what must start at zero -- both copies of the factors and W,
  // whose columns r..R-1 are the exact zero padding of the rank, the
  // last-block counters, the state and the r x r workspace
  NA_CK(cudaMemsetAsync(a.U[0], 0, (size_t)m * R * 4, s));
  NA_CK(cudaMemsetAsync(a.U[1], 0, (size_t)m * R * 4, s));
  NA_CK(cudaMemsetAsync(a.V[0], 0, (size_t)n * R * 4, s));
  NA_CK(cudaMemsetAsync(a.V[1], 0, (size_t)n * R * 4, s));
  NA_CK(cudaMemsetAsync(a.W, 0, (size_t)m * R * 4, s));
  NA_CK(cudaMemsetAsync(counters, 0, 4 * sizeof(unsigned int), s));
  NA_CK(cudaMemsetAsync(a.st, 0, sizeof(DevState), s));
  NA_CK(cudaMemsetAsync(a.sm, 0, sizeof(Smalls), s));
  NA_CK(cudaMemcpy2DAsync(a.U[0], R * 4, U_in, r * 4, r * 4, m, cudaMemcpyDeviceToDevice, s));
  NA_CK(cudaMemcpy2DAsync(a.V[0], R * 4, V_in, r * 4, r * 4, n, cudaMemcpyDeviceToDevice, s));
  // start point: U^T U + rho I -> (.)^{-1}, and V^T V for the metrics
  NA_CK(launch_gram(a.U[0], R, R, a.U[0], R, R, m, a.part_g, n_rblocks, a.st, 0, s));
  NA_CK(launch_reduce_init(a, 0, 0, a.part_g, n_rblocks, red_g, counters + 2, s));
  NA_CK(launch_gram(a.V[0], R, R, a.V[0], R, R, n, a.part_q, n_vgram, a.st, 0, s));
  NA_CK(launch_reduce_init(a, 1, 0, a.part_q, n_vgram, red_q, counters + 3, s));
  // the iteration (the same kernels and order as the general path of dcf_step)
  NA_CK(launch_make_w(a, 0, 1, s));
  NA_CK(launch_pass1(a, n_vblocks, 0, 0, s));
  NA_CK(launch_pass2(a, s));
  NA_CK(launch_gram_vv(R, a.V[0], a.V[1], n, a.part_q, a.part_xv, a.part_dv, n_vgram, a.st, s));
  NA_CK(launch_reduce_q(a, red_q, red_xv, red_dv, red_h, n_vgram, counters + 0, s));
  NA_CK(launch_rows(a, s));
  NA_CK(launch_reduce_g(a, red_g, red_xu, red_du, counters + 1, s));
  NA_CK(cudaMemcpy2DAsync(U_out, r * 4, a.U[1], R * 4, r * 4, m, cudaMemcpyDeviceToDevice, s));
  NA_CK(cudaMemcpy2DAsync(V_out, r * 4, a.V[1], R * 4, r * 4, n, cudaMemcpyDeviceToDevice, s));
#undef NA_CK
  return DCF_OK;
}
