// Internal: the handle behind dcf_handle and the host helpers shared by the
// C-ABI translation units (dcf_api.cu, dcf_unrolled.cu).
#pragma once
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "dcf.h"
#include "dcf_internal.cuh"

struct UnrolledState;

struct dcf_handle_s {
  // problem
  int64_t m = 0, n = 0;
  int E = 0, r = 0, R = 0;
  double rho = 0, lam = 0, tol = 0, eta0 = 0;
  int max_iter = 0, u_mode = 0, local_steps = 1;
  double rho_u = 0;                   // rho of the U-step's ridge term when > 0 (a client
                                      // handle: rho n_i / n); 0: rho
  uint64_t seed = 0;
  std::vector<int64_t> n_i, c_i;
  std::vector<char> priv;
  // allocation
  dcf_alloc_fn alloc = nullptr;
  dcf_free_fn release = nullptr;
  void* alloc_ctx = nullptr;
  std::vector<void*> owned;
  // device
  int device = 0, num_sms = 0;
  cudaStream_t user_stream = nullptr;
  cudaStream_t stream = nullptr;     // internal capture/launch stream
  cudaStream_t side = nullptr;       // NaN/Inf checks of copied blocks, behind the copies;
                                     // the copies of asynchronous reloads
  cudaStream_t side2 = nullptr;      // the checks of asynchronous reloads
  cudaEvent_t ev_in = nullptr, ev_out = nullptr, ev_side = nullptr, ev_side2 = nullptr;
  float* M = nullptr;                 // the matrix the iterations read (Mbuf[mcur] unless borrowed)
  bool M_borrowed = false;
  // own copies of M, two for asynchronous reloads (the next step's M is copied
  // while the current one is iterated on)
  float* Mbuf[2] = {nullptr, nullptr};
  int mcur = 0;                       // buffer in use
  int pend = -1;                      // buffer of a pending asynchronous reload, -1: none
  int* mflag = nullptr;               // [2]: a NaN/Inf was found in Mbuf[b] by its last reload
  cudaEvent_t ev_copy = nullptr;      // the pending reload's copy and check are done (side)
  cudaEvent_t ev_used[2] = {nullptr, nullptr};   // last enqueued work that may read Mbuf[b]
  alignas(64) unsigned char tmaps[2][128];        // tensor maps over Mbuf[0], Mbuf[1]
  float* U[2] = {nullptr, nullptr};
  float* V[2] = {nullptr, nullptr};
  float* W = nullptr;
  float* part_p = nullptr;
  double* part_h = nullptr;
  float2* part_q = nullptr;
  float2* part_xv = nullptr;
  float2* part_dv = nullptr;
  float2* part_g = nullptr;
  float2* part_xu = nullptr;
  float2* part_du = nullptr;
  double* red = nullptr;             // reduction outputs: q, xv, dv, h (8), g, xu, du
  float2* truth_part = nullptr;
  double* truth_red = nullptr;
  double* sv_part = nullptr;         // singular values: FP64 Gram partials,
  double* sv_gram = nullptr;         //   [2 problems][G_x, G_y][64 x 64],
  int* sv_pdim = nullptr;            //   the two problems' ranks,
  double* sv_out = nullptr;          //   sigma [64], sigma0 [64], error
  dcf::Smalls* sm = nullptr;
  dcf::DevState* st = nullptr;
  unsigned int* counters = nullptr;  // 4 last-block counters
  int* flag = nullptr;
  float* A_truth = nullptr;
  float* B_truth = nullptr;
  int k_truth = 0;
  // launch geometry
  int n_vblocks = 0, n_splits = 0, n_rblocks = 0, n_vgram = 0;
  int64_t split_cols = 0;
  // fused single-pass path
  int path = 1;                       // 1 general, 2 fused, 3 two-pass tensor core,
                                      // 4 whole solve in one CTA
  int cs = 0, nclusters = 0, nslabs = 0;
  uint8_t* img = nullptr;
  float* scales = nullptr;
  float* zmat = nullptr;
  float* W_vz = nullptr;              // n x R, V_old Z (fused path)
  unsigned int* vmax = nullptr;       // [2]: max |V| of copy 0 / 1 (float bits)
  float* ypart = nullptr;             // two-pass tensor core: [nslabs][n][R] column sums
  int G = 0;                          // two-pass tensor core: strip groups (CTAs per slab)
  // fused path: the SMs that its clusters leave idle run the two-pass
  // tensor-core kernels on the last n_tail columns, concurrently with the fused
  // kernel on the first n - n_tail (0: not used)
  int64_t n_tail = 0;
  int G_tail = 0;                     // strip groups of the tail (CTAs per slab)
  float* ypart_tail = nullptr;        // [nslabs][n_tail][R] column sums of the tail
  unsigned int* vmax_tail = nullptr;  // [2]: max |V'| of the tail columns (float bits)
  alignas(64) unsigned char tmap_tail[128];         // tensor map over the tail columns of M
  alignas(64) unsigned char tmaps_tail[2][128];     // the same over Mbuf[0], Mbuf[1]
  cudaStream_t tail_stream = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  int prio_high = 0;                  // scheduling priority of the fused kernel
  int* kerr = nullptr;                // kernel-side error (DCF_ETIMEOUT)
  alignas(64) unsigned char tmap[128];
  // state
  bool loaded = false, initialized = false;
  int host_iter = 0;                  // iterations enqueued (mirrors DevState::iter)
  cudaGraphExec_t graph[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};   // [buffer][parity]
  float alpha = 1.0f;                 // relaxation of the U-step (learned network)
  float* ustar_out = nullptr;         // when set, the U-step also stores U* here
  UnrolledState* unrolled = nullptr;  // checkpoints and buffers of the learned network
  // K > 1 local steps of Algorithm 1 (FedAvg mode): one client handle per block,
  // each iterating on its own block (M borrowed from this handle) with its own U_i
  std::vector<dcf_handle_s*> clients;
  int client_path = 0;                // the path the clients' iterations run on
  const float** loc_uptr = nullptr;   // device array: every client's U after its K steps
  double* loc_h = nullptr;            // E Huber sums of the clients' first local steps
  std::string err;
};


namespace dcf {
namespace api {
dcf_status fail(dcf_handle h, dcf_status code, const std::string& msg);
dcf_status cuda_fail(dcf_handle h, cudaError_t e, const char* what);
void* dev_alloc(dcf_handle h, size_t bytes);
// The allocator hook set by dcf_set_allocator (NULL: cudaMalloc / cudaFree).
void current_allocator(dcf_alloc_fn* alloc, dcf_free_fn* release, void** ctx);
IterArgs iter_args(dcf_handle h, int cur);
cudaError_t enqueue_iteration(dcf_handle h, int cur, cudaStream_t s, cudaEvent_t* ev);
dcf_status begin_work(dcf_handle h);
dcf_status end_work(dcf_handle h);
dcf_status read_state(dcf_handle h, DevState* out);
dcf_status ensure_init(dcf_handle h);
dcf_status apply_pending(dcf_handle h);
dcf_status set_state_fields(dcf_handle h, int solve_mode, double tol);
void free_unrolled(dcf_handle h);
}  // namespace api
}  // namespace dcf
