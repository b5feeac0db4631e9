// C ABI of the DCF-PCA library: handle, buffers, launch sequence, CUDA graphs.
//
// One iteration (Algorithm 1 with the exact consensus U-step, or its FedAvg
// gradient step) is the launch sequence in enqueue_iteration().  It is
// captured once per parity of the iteration counter into a CUDA graph and
// replayed; the device-side stop flag turns every kernel of a replay into a
// no-op once dcf_solve's tolerance is met.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "dcf.h"
#include "dcf_handle.h"
#include "dcf_internal.cuh"


using namespace dcf;
using namespace dcf::api;

// ---------------------------------------------------------------------------
// allocator hook
// ---------------------------------------------------------------------------
static dcf_alloc_fn g_alloc = nullptr;
static dcf_free_fn g_free = nullptr;
static void* g_alloc_ctx = nullptr;

extern "C" void dcf_set_allocator(dcf_alloc_fn alloc, dcf_free_fn release, void* ctx) {
  g_alloc = alloc;
  g_free = release;
  g_alloc_ctx = ctx;
}


namespace dcf {
namespace api {

dcf_status fail(dcf_handle h, dcf_status code, const std::string& msg) {
  if (h) h->err = msg;
  return code;
}

dcf_status cuda_fail(dcf_handle h, cudaError_t e, const char* what) {
  return fail(h, DCF_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

// The fused path's concurrent tail (see dcf_create): the two-pass kernels'
// bytes of M per CTA and second (counting both of their reads of M) relative
// to a fused CTA's, at most this many strip groups, and only for problems of at
// least this many 64-column strips.
#ifndef DCF_TAIL_RATE
#define DCF_TAIL_RATE 0.7
#endif
constexpr double kTailRate = DCF_TAIL_RATE;
constexpr int kTailMaxGroups = 8;
constexpr int kTailMinStrips = 128;

#define CK(call, what)                                   \
  do {                                                   \
    cudaError_t e_ = (call);                             \
    if (e_ != cudaSuccess) return cuda_fail(h, e_, what); \
  } while (0)

void current_allocator(dcf_alloc_fn* alloc, dcf_free_fn* release, void** ctx) {
  *alloc = g_alloc;
  *release = g_free;
  *ctx = g_alloc_ctx;
}

void* dev_alloc(dcf_handle h, size_t bytes) {
  if (bytes == 0) bytes = 16;
  void* p = nullptr;
  if (h->alloc) {
    p = h->alloc(bytes, h->alloc_ctx);
    if (p && (reinterpret_cast<uintptr_t>(p) & 255u) != 0) {   // vector loads and TMA need it
      if (h->release) h->release(p, h->alloc_ctx);
      p = nullptr;
    }
  } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    p = nullptr;
  }
  if (p) h->owned.push_back(p);
  return p;
}

void dev_free_all(dcf_handle h) {
  for (void* p : h->owned) {
    if (h->release) h->release(p, h->alloc_ctx);
    else cudaFree(p);
  }
  h->owned.clear();
}

IterArgs iter_args(dcf_handle h, int cur) {
  IterArgs a{};
  a.cur = cur;
  a.M = h->M;
  a.m = h->m;
  a.n = h->n;
  a.r = h->r;
  a.R = h->R;
  a.lam = (float)h->lam;
  a.rho = (float)h->rho;
  a.rho_q = (float)h->rho_u;
  a.u_mode = h->u_mode;
  a.E = h->E;
  a.U[0] = h->U[0]; a.U[1] = h->U[1];
  a.V[0] = h->V[0]; a.V[1] = h->V[1];
  a.W = h->W;
  a.part_q = h->part_q;
  a.part_xv = h->part_xv;
  a.part_dv = h->part_dv;
  a.part_h = h->part_h;
  a.part_p = h->part_p;
  a.n_vblocks = h->n_vblocks;
  a.n_splits = h->n_splits;
  a.split_cols = h->split_cols;
  a.part_g = h->part_g;
  a.part_xu = h->part_xu;
  a.part_du = h->part_du;
  a.n_rblocks = h->n_rblocks;
  a.sm = h->sm;
  a.st = h->st;
  a.add_uxv = h->path == 2 ? 1 : 0;
  a.alpha = h->alpha;
  a.ustar_out = h->ustar_out;
  if (h->path == 2) {
    // per-CTA Huber partials of the fused kernel, then of the tail's pass A;
    // P partials: one per cluster, then one per strip group of the tail
    a.n_vblocks = h->cs * h->nclusters + (h->n_tail > 0 ? h->nslabs * h->G_tail : 0);
    a.n_splits = h->nclusters + (h->n_tail > 0 ? h->G_tail : 0);
  }
  if (h->path == 3) {
    a.add_uxv = 1;
    a.n_vblocks = h->nslabs * h->G;       // Huber partials: one per CTA of pass A
    a.n_splits = h->G;                    // P partials: one per strip group
  }
  return a;
}

// reduction outputs: Q, V-side cross, dV Gram, Huber (8), G, U-side cross, dU Gram
double* red_q(dcf_handle h) { return h->red; }
double* red_xv(dcf_handle h) { return h->red + (size_t)h->R * h->R; }
double* red_dv(dcf_handle h) { return h->red + 2 * (size_t)h->R * h->R; }
double* red_h(dcf_handle h) { return h->red + 3 * (size_t)h->R * h->R; }
double* red_g(dcf_handle h) { return h->red + 3 * (size_t)h->R * h->R + 8; }
double* red_xu(dcf_handle h) { return h->red + 4 * (size_t)h->R * h->R + 8; }
double* red_du(dcf_handle h) { return h->red + 5 * (size_t)h->R * h->R + 8; }

// Phases of one iteration, in launch order (names used by dcf_profile_*).
const char* const kPhaseNames[] = {"make_w", "pass1_vstep", "pass2_pstep", "gram_v",
                                   "reduce_q", "rows_ustep", "reduce_g"};
constexpr int kNumPhases = 7;
const char* const kFusedPhaseNames[] = {"fused_prep", "fused_step", "gram_v", "reduce_q",
                                        "rows_ustep", "reduce_g"};
constexpr int kNumFusedPhases = 6;
const char* const kTc2PhaseNames[] = {"tc_prep", "pass_a", "v_reduce", "gram_v",
                                      "reduce_q", "pass_b", "rows_ustep", "reduce_g"};
constexpr int kNumTc2Phases = 8;
const char* const kSmallPhaseNames[] = {"solve_small"};
int num_phases(dcf_handle h) {
  return h->path == 2 ? kNumFusedPhases
         : h->path == 3 ? kNumTc2Phases
         : h->path == 4 ? 1
                        : kNumPhases;
}
const char* phase_name(dcf_handle h, int p) {
  return h->path == 2 ? kFusedPhaseNames[p]
         : h->path == 3 ? kTc2PhaseNames[p]
         : h->path == 4 ? kSmallPhaseNames[p]
                        : kPhaseNames[p];
}

// Path 4: `n_iter` iterations of the whole-solve kernel from copy `cur`.
cudaError_t enqueue_small(dcf_handle h, int cur, int n_iter, cudaStream_t s) {
  SmallSolveArgs sa{};
  sa.M = h->M;
  sa.m = h->m;
  sa.n = h->n;
  sa.U[0] = h->U[0]; sa.U[1] = h->U[1];
  sa.V[0] = h->V[0]; sa.V[1] = h->V[1];
  sa.cur = cur;
  sa.n_iter = n_iter;
  sa.lam = (float)h->lam;
  sa.rho = (float)h->rho;
  sa.st = h->st;
  return launch_solve_small(h->R, sa, s);
}

// One iteration of the fused path: prep (W and fp16 images), the single pass
// over M, Q/X_v reduction with (Q + rho I)^{-1}, consensus rows, metrics.
cudaError_t enqueue_fused_iteration(dcf_handle h, int cur, cudaStream_t s, cudaEvent_t* ev) {
  IterArgs a = iter_args(h, cur);
  const int nxt = cur ^ 1;
  cudaError_t e;
  int ph = 0;
  auto mark = [&]() -> cudaError_t {
    if (ev) return cudaEventRecord(ev[ph++], s);
    return cudaSuccess;
  };
  if ((e = launch_fused_prep(h->R, h->U[cur], h->sm, h->st, h->m, h->nslabs, (float)h->rho,
                             h->vmax + cur, h->vmax + nxt, h->img, h->scales, h->zmat,
                             h->V[cur], h->n, h->W_vz, s)) != cudaSuccess ||
      (e = mark()) != cudaSuccess)
    return e;
  FusedArgs fa{};
  fa.cur = cur;
  fa.cs = h->cs;
  fa.nclusters = h->nclusters;
  fa.nslabs = h->nslabs;
  fa.m = h->m;
  fa.n = h->n;
  fa.lam = (float)h->lam;
  fa.Vold = h->V[cur];
  fa.Vnew = h->V[nxt];
  fa.img = h->img;
  fa.scales = h->scales;
  fa.zmat = h->zmat;
  fa.VZ = h->W_vz;
  fa.vmax_out = h->vmax + nxt;
  fa.part_h = h->part_h;
  fa.part_p = h->part_p;
  fa.st = h->st;
  fa.err = h->kerr;
  if (h->n_tail == 0) {
    if ((e = launch_fused(h->R, h->tmap, fa, s)) != cudaSuccess || (e = mark()) != cudaSuccess)
      return e;
  } else {
    // the fused kernel on the first n_head columns (its clusters first), and on
    // the SMs they leave idle the two-pass kernels on the last n_tail columns:
    // column sums (pass A), V' = V_old Z + their sum, P partials (pass B)
    const int64_t n_head = h->n - h->n_tail;
    fa.n = n_head;
    if ((e = cudaEventRecord(h->ev_fork, s)) != cudaSuccess ||
        (e = cudaStreamWaitEvent(h->tail_stream, h->ev_fork, 0)) != cudaSuccess ||
        (e = launch_fused(h->R, h->tmap, fa, s, &h->prio_high)) != cudaSuccess)
      return e;
    cudaStream_t t = h->tail_stream;
    Tc2Args ta{};
    ta.cur = cur;
    ta.nslabs = h->nslabs;
    ta.G = h->G_tail;
    ta.m = h->m;
    ta.n = h->n_tail;
    ta.lam = (float)h->lam;
    ta.Vold = h->V[cur] + n_head * h->R;
    ta.Vp = h->V[nxt] + n_head * h->R;
    ta.img = h->img;
    ta.scales = h->scales;
    ta.vp_max = h->vmax_tail + nxt;
    ta.ypart = h->ypart_tail;
    ta.part_h = h->part_h + (size_t)h->cs * h->nclusters;
    ta.part_p = h->part_p + (size_t)h->nclusters * h->m * h->R;
    ta.st = h->st;
    ta.err = h->kerr;
    if ((e = cudaMemsetAsync(h->vmax_tail + nxt, 0, sizeof(unsigned int), t)) != cudaSuccess ||
        (e = launch_tc2(h->R, 0, h->tmap_tail, ta, t)) != cudaSuccess ||
        (e = launch_tc2_vreduce(h->R, h->ypart_tail, tc2_parts(h->R, h->nslabs),
                                h->W_vz + n_head * h->R,
                                h->n_tail, h->V[nxt] + n_head * h->R, h->vmax_tail + nxt, h->st,
                                h->num_sms, t, h->vmax + nxt)) != cudaSuccess ||
        (e = launch_tc2(h->R, 1, h->tmap_tail, ta, t)) != cudaSuccess ||
        (e = cudaEventRecord(h->ev_join, t)) != cudaSuccess ||
        (e = cudaStreamWaitEvent(s, h->ev_join, 0)) != cudaSuccess || (e = mark()) != cudaSuccess)
      return e;
  }
  // Q_t = V_t^T V_t and V_{t-1}^T V_t from the new V (Gram partials)
  if ((e = launch_gram_vv(h->R, h->V[cur], h->V[nxt], h->n, h->part_q, h->part_xv, h->part_dv, h->n_vgram,
                          h->st, s)) != cudaSuccess ||
      (e = mark()) != cudaSuccess)
    return e;
  if ((e = launch_reduce_q(a, red_q(h), red_xv(h), red_dv(h), red_h(h), h->n_vgram, h->counters + 0, s)) !=
          cudaSuccess ||
      (e = mark()) != cudaSuccess)
    return e;
  if ((e = launch_rows(a, s)) != cudaSuccess || (e = mark()) != cudaSuccess) return e;
  if ((e = launch_reduce_g(a, red_g(h), red_xu(h), red_du(h), h->counters + 1, s)) != cudaSuccess) return e;
  return mark();
}

// One iteration of the two-pass tensor-core path: prep, pass A (column sums
// per slab), V' = V_old Z + their sum, Q/X_v and (Q + rho I)^{-1}, pass B (P
// partials per strip group), consensus rows, metrics.
cudaError_t enqueue_tc2_iteration(dcf_handle h, int cur, cudaStream_t s, cudaEvent_t* ev) {
  IterArgs a = iter_args(h, cur);
  const int nxt = cur ^ 1;
  cudaError_t e;
  int ph = 0;
  auto mark = [&]() -> cudaError_t {
    if (ev) return cudaEventRecord(ev[ph++], s);
    return cudaSuccess;
  };
  if ((e = launch_fused_prep(h->R, h->U[cur], h->sm, h->st, h->m, h->nslabs, (float)h->rho,
                             h->vmax + cur, h->vmax + nxt, h->img, h->scales, h->zmat,
                             h->V[cur], h->n, h->W_vz, s)) != cudaSuccess ||
      (e = mark()) != cudaSuccess)
    return e;
  Tc2Args ta{};
  ta.cur = cur;
  ta.nslabs = h->nslabs;
  ta.G = h->G;
  ta.m = h->m;
  ta.n = h->n;
  ta.lam = (float)h->lam;
  ta.Vold = h->V[cur];
  ta.Vp = h->V[nxt];
  ta.img = h->img;
  ta.scales = h->scales;
  ta.vp_max = h->vmax + nxt;
  ta.ypart = h->ypart;
  ta.part_h = h->part_h;
  ta.part_p = h->part_p;
  ta.st = h->st;
  ta.err = h->kerr;
  if ((e = launch_tc2(h->R, 0, h->tmap, ta, s)) != cudaSuccess || (e = mark()) != cudaSuccess)
    return e;
  if ((e = launch_tc2_vreduce(h->R, h->ypart, tc2_parts(h->R, h->nslabs), h->W_vz, h->n, h->V[nxt],
                              h->vmax + nxt, h->st, h->num_sms, s)) != cudaSuccess ||
      (e = mark()) != cudaSuccess)
    return e;
  if ((e = launch_gram_vv(h->R, h->V[cur], h->V[nxt], h->n, h->part_q, h->part_xv, h->part_dv, h->n_vgram,
                          h->st, s)) != cudaSuccess ||
      (e = mark()) != cudaSuccess)
    return e;
  if ((e = launch_reduce_q(a, red_q(h), red_xv(h), red_dv(h), red_h(h), h->n_vgram, h->counters + 0, s)) !=
          cudaSuccess ||
      (e = mark()) != cudaSuccess)
    return e;
  if ((e = launch_tc2(h->R, 1, h->tmap, ta, s)) != cudaSuccess || (e = mark()) != cudaSuccess)
    return e;
  if ((e = launch_rows(a, s)) != cudaSuccess || (e = mark()) != cudaSuccess) return e;
  if ((e = launch_reduce_g(a, red_g(h), red_xu(h), red_du(h), h->counters + 1, s)) != cudaSuccess) return e;
  return mark();
}

// Enqueue one iteration reading copy `cur` (capturable).  When `ev` is not
// NULL, event ev[p] is recorded after phase p (profiling path, not captured).
cudaError_t enqueue_iteration(dcf_handle h, int cur, cudaStream_t s, cudaEvent_t* ev) {
  if (h->path == 2) return enqueue_fused_iteration(h, cur, s, ev);
  if (h->path == 3) return enqueue_tc2_iteration(h, cur, s, ev);
  if (h->path == 4) {
    cudaError_t e = enqueue_small(h, cur, 1, s);
    if (e == cudaSuccess && ev) e = cudaEventRecord(ev[0], s);
    return e;
  }
  IterArgs a = iter_args(h, cur);
  const int nxt = cur ^ 1;
  cudaError_t e;
  int ph = 0;
  auto mark = [&]() -> cudaError_t {
    if (ev) return cudaEventRecord(ev[ph++], s);
    return cudaSuccess;
  };
  // V-step: W = U (U^T U + rho I)^{-1}; then S, X, V' = X^T W in one pass over M
  if ((e = launch_make_w(a, cur, 1, s)) != cudaSuccess || (e = mark()) != cudaSuccess) return e;
  if ((e = launch_pass1(a, h->n_vblocks, 0, 0, s)) != cudaSuccess || (e = mark()) != cudaSuccess)
    return e;
  // U-step numerator P = X V' (second pass over M)
  if ((e = launch_pass2(a, s)) != cudaSuccess || (e = mark()) != cudaSuccess) return e;
  // Q_t = V_t^T V_t and V_{t-1}^T V_t
  if ((e = launch_gram_vv(h->R, h->V[cur], h->V[nxt], h->n, h->part_q, h->part_xv, h->part_dv, h->n_vgram,
                          h->st, s)) != cudaSuccess ||
      (e = mark()) != cudaSuccess)
    return e;
  if ((e = launch_reduce_q(a, red_q(h), red_xv(h), red_dv(h), red_h(h), h->n_vgram, h->counters + 0, s)) !=
          cudaSuccess ||
      (e = mark()) != cudaSuccess)
    return e;
  // consensus U-update + Gram partials of U_t
  if ((e = launch_rows(a, s)) != cudaSuccess || (e = mark()) != cudaSuccess) return e;
  // U_t^T U_t, metrics, stop test, (U_t^T U_t + rho I)^{-1} for the next V-step
  if ((e = launch_reduce_g(a, red_g(h), red_xu(h), red_du(h), h->counters + 1, s)) != cudaSuccess) return e;
  return mark();
}

dcf_status build_graphs(dcf_handle h) {
  for (int p = 0; p < 2; ++p) {
    if (h->graph[h->mcur][p]) continue;
    cudaGraph_t g = nullptr;
    CK(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal), "begin capture");
    cudaError_t e = enqueue_iteration(h, p, h->stream, nullptr);
    cudaError_t e2 = cudaStreamEndCapture(h->stream, &g);
    if (e != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      return cuda_fail(h, e, "capture iteration");
    }
    CK(e2, "end capture");
    cudaError_t e3 = cudaGraphInstantiate(&h->graph[h->mcur][p], g, 0);
    cudaGraphDestroy(g);
    CK(e3, "instantiate graph");
  }
  return DCF_OK;
}

// A pending asynchronous reload becomes the M that work enqueued from now on
// reads: the internal stream waits for its copy and check, a failed check
// stops the solve (k_apply_mflag), and the buffers swap.  Called by the entry
// points that read M (through ensure_init, and the loads); calls that only
// read factors or statistics do not wait for a pending copy.
dcf_status apply_pending(dcf_handle h) {
  if (h->pend < 0) return DCF_OK;
  CK(cudaStreamWaitEvent(h->stream, h->ev_copy, 0), "wait");
  CK(launch_apply_mflag(h->mflag + h->pend, h->st, h->stream), "apply reload check");
  h->mcur = h->pend;
  h->M = h->Mbuf[h->mcur];
  std::memcpy(h->tmap, h->tmaps[h->mcur], sizeof(h->tmap));
  std::memcpy(h->tmap_tail, h->tmaps_tail[h->mcur], sizeof(h->tmap_tail));
  h->pend = -1;
  return DCF_OK;
}

// A load or a synchronous reload supersedes a pending asynchronous reload:
// its copy is waited for and its buffer stays out of use.
static dcf_status drop_pending(dcf_handle h) {
  if (h->pend < 0) return DCF_OK;
  CK(cudaStreamSynchronize(h->side), "sync");
  h->pend = -1;
  return DCF_OK;
}

// Order internal stream after the user's stream.
dcf_status begin_work(dcf_handle h) {
  CK(cudaSetDevice(h->device), "set device");
  CK(cudaEventRecord(h->ev_in, h->user_stream), "record");
  CK(cudaStreamWaitEvent(h->stream, h->ev_in, 0), "wait");
  return DCF_OK;
}

dcf_status end_work(dcf_handle h) {
  CK(cudaEventRecord(h->ev_used[h->mcur], h->stream), "record");
  CK(cudaEventRecord(h->ev_out, h->stream), "record");
  CK(cudaStreamWaitEvent(h->user_stream, h->ev_out, 0), "wait");
  return DCF_OK;
}

dcf_status read_state(dcf_handle h, DevState* out) {
  int kerr = 0;
  CK(cudaMemcpyAsync(out, h->st, sizeof(DevState), cudaMemcpyDeviceToHost, h->stream), "read state");
  CK(cudaMemcpyAsync(&kerr, h->kerr, sizeof(int), cudaMemcpyDeviceToHost, h->stream), "read err");
  CK(cudaStreamSynchronize(h->stream), "sync");
  if (kerr == DCF_ETIMEOUT)
    return fail(h, DCF_ETIMEOUT, "a bounded device-side wait expired in the fused kernel");
  if (out->status == DCF_ENONFINITE)
    return fail(h, DCF_ENONFINITE, "non-finite value in the iterates");
  return DCF_OK;
}

// Write the solve-control fields of the device state (stream-ordered; the
// host values are staged by cudaMemcpyAsync from pageable memory).
dcf_status set_state_fields(dcf_handle h, int solve_mode, double tol) {
  int zero = 0;
  CK(cudaMemcpyAsync(&h->st->solve_mode, &solve_mode, sizeof(int), cudaMemcpyHostToDevice,
                     h->stream), "write state");
  CK(cudaMemcpyAsync(&h->st->tol, &tol, sizeof(double), cudaMemcpyHostToDevice, h->stream),
     "write state");
  CK(cudaMemcpyAsync(&h->st->stop, &zero, sizeof(int), cudaMemcpyHostToDevice, h->stream),
     "write state");
  return DCF_OK;
}

// Start point: U0 in copy 0 -> Gram, Cholesky; V0 given or V-step with S = 0.
dcf_status finish_init(dcf_handle h, bool have_v0) {
  cudaStream_t s = h->stream;
  IterArgs a = iter_args(h, 0);
  DevState st0{};
  st0.eta0 = h->eta0;
  st0.tol = h->tol;
  CK(cudaMemcpyAsync(h->st, &st0, sizeof(DevState), cudaMemcpyHostToDevice, s), "init state");
  CK(cudaMemsetAsync(h->counters, 0, 4 * sizeof(unsigned int), s), "memset");
  CK(cudaMemsetAsync(h->sm, 0, sizeof(Smalls), s), "memset");
  // G0 = U0^T U0 and its Cholesky factor
  CK(launch_gram(h->U[0], h->R, h->R, h->U[0], h->R, h->R, h->m, h->part_g, h->n_rblocks, h->st,
                 0, s), "gram U0");
  CK(launch_reduce_init(a, 0, 0, h->part_g, h->n_rblocks, red_g(h), h->counters + 2, s),
     "reduce G0");
  if (!have_v0) {
    CK(launch_make_w(a, 0, 0, s), "W0");
    CK(launch_pass1(a, h->n_vblocks, 1, 0, s), "V0 sweep");
  }
  CK(launch_gram(h->V[0], h->R, h->R, h->V[0], h->R, h->R, h->n, h->part_q, h->n_vgram, h->st, 0,
                 s), "gram V0");
  if (h->path == 2 || h->path == 3) {
    CK(cudaMemsetAsync(h->vmax, 0, 2 * sizeof(unsigned int), s), "memset");
    CK(launch_absmax(h->V[0], h->n * h->R, h->vmax, s), "max |V0|");
  }
  CK(launch_reduce_init(a, 1, 0, h->part_q, h->n_vgram, red_q(h), h->counters + 3, s),
     "reduce Q0");
  h->host_iter = 0;
  h->initialized = true;
  return DCF_OK;
}

dcf_status ensure_init(dcf_handle h) {
  if (!h->loaded) return fail(h, DCF_ESTATE, "dcf_load_blocks has not been called");
  dcf_status pst = apply_pending(h);
  if (pst != DCF_OK) return pst;
  if (h->initialized) return DCF_OK;
  CK(launch_philox_u0(h->U[0], h->m, h->r, h->R, h->seed, h->stream), "philox U0");
  return finish_init(h, false);
}

}  // namespace api
}  // namespace dcf

// ---------------------------------------------------------------------------
// entry points
// ---------------------------------------------------------------------------
extern "C" const char* dcf_version(void) { return "dcf-gb300 0.1"; }

extern "C" const char* dcf_last_error(dcf_handle h) {
  if (!h) return "null handle";
  return h->err.c_str();
}

extern "C" dcf_status dcf_create(const dcf_params* p, dcf_handle* out) {
  if (!p || !out) return DCF_EINVAL;
  *out = nullptr;
  dcf_handle h = new (std::nothrow) dcf_handle_s();
  if (!h) return DCF_ENOMEM;
  auto bad = [&](const char* msg) {
    // keep the handle-less contract: report through a short-lived handle
    delete h;
    (void)msg;
    return DCF_EINVAL;
  };
  if (p->m < 1 || p->E < 1 || !p->n_i) return bad("m, E, n_i");
  if (p->r < 1 || p->r > kMaxR || p->r > p->m) return bad("r");
  if (!(p->rho > 0) || !(p->lambda > 0)) return bad("rho, lambda");
  if (p->u_mode != 0 && p->u_mode != 1) return bad("u_mode");
  if (p->local_steps < 1 || (p->local_steps > 1 && p->u_mode != 1)) return bad("local_steps");
  if (p->local_steps > 1 && p->path == 4) return bad("path");
  if (p->max_iter < 1) return bad("max_iter");
  if (p->path < 0 || p->path > 4) return bad("path");
  h->m = p->m;
  h->E = p->E;
  h->r = p->r;
  h->R = pick_R(p->r);
  h->rho = p->rho;
  h->lam = p->lambda;
  h->tol = p->tol;
  h->max_iter = p->max_iter;
  h->u_mode = p->u_mode;
  h->local_steps = p->local_steps;
  h->eta0 = p->eta0;
  h->seed = p->seed;
  h->n_i.assign(p->n_i, p->n_i + p->E);
  h->c_i.resize(p->E + 1);
  h->c_i[0] = 0;
  for (int i = 0; i < p->E; ++i) {
    if (h->n_i[i] < 1) return bad("n_i");
    h->c_i[i + 1] = h->c_i[i] + h->n_i[i];
  }
  h->n = h->c_i[p->E];
  h->priv.assign(p->E, 0);
  h->alloc = g_alloc;
  h->release = g_free;
  h->alloc_ctx = g_alloc_ctx;

  if (cudaGetDevice(&h->device) != cudaSuccess) { delete h; return DCF_ECUDA; }
  if (prepare_stream_kernels() != cudaSuccess || prepare_small_kernels() != cudaSuccess) {
    delete h;
    return DCF_ECUDA;
  }
  cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device);
  if (h->num_sms <= 0) h->num_sms = 1;
  if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&h->side2, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->ev_side2, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->ev_in, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->ev_out, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->ev_side, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->ev_copy, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->ev_used[0], cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->ev_used[1], cudaEventDisableTiming) != cudaSuccess) {
    dcf_destroy(h);
    return DCF_ECUDA;
  }

  // K > 1 local steps: this handle holds the round's U, V and metrics and runs
  // the server's kernels on the general path's buffers; the clients (created
  // below, one per block) run the local iterations on the requested path
  const bool local = p->local_steps > 1;
  // whole solve in one CTA: exact U-step, r <= 16, M and the factors in one
  // SM's shared memory; on request only (the learned network and the FedAvg
  // step run on the multi-kernel paths)
  if (!local) {
    const int Rs = pick_R(p->r);
    const bool small_ok = p->u_mode == 0 && p->r <= 16 &&
                          solve_small_smem(Rs, h->m, h->n) + 2048 <= 232448;
    if (p->path == 4 && !small_ok) {
      dcf_destroy(h);
      return DCF_EINVAL;
    }
    if (p->path == 4) {
      if (solve_small_prepare(Rs, solve_small_smem(Rs, h->m, h->n)) != cudaSuccess) {
        cudaGetLastError();
        dcf_destroy(h);
        return DCF_ECUDA;
      }
      h->path = 4;
      h->R = Rs;
    }
  }
  // fused single-pass path: r <= 32, m a multiple of 4 (TMA row stride), at most
  // 16 slabs of 256 rows per cluster, and the cluster shape must fit on the GPU
  if (!local) {
    const bool shape_ok = p->r <= 32 && h->m % 4 == 0 && (h->m + 255) / 256 <= 16;
    if (p->path == 2 && !shape_ok) {
      dcf_destroy(h);
      return DCF_EINVAL;
    }
    if ((p->path == 2 || (p->path == 0 && h->path == 1)) && shape_ok) {
      const int Rf = p->r <= 16 ? 16 : 32;
      // slabs of 256 rows, rounded up to a power of two: the cluster exchange
      // splits each 64-column strip into 16 chunks, so the cluster size divides 16
      // (slabs past the last row read zeros)
      int cs = 1;
      while (cs * 256 < h->m) cs *= 2;
      int ncl = 0;
      if (fused_prepare(Rf) == cudaSuccess) ncl = fused_max_clusters(Rf, cs);
      cudaGetLastError();
      if (ncl > 0) {
        h->path = 2;
        h->R = Rf;
        h->cs = cs;
        h->nslabs = cs;
        const int64_t nstrips64 = (h->n + 63) / 64;
        h->nclusters = (int)std::min<int64_t>(ncl, nstrips64);
        // the SMs the clusters leave idle (a cluster must fit in one GPC) take
        // a share of the columns on the two-pass kernels, one CTA per SM and
        // (slab, strip group); the share balances the two rates (kTailRate:
        // the two-pass kernels' bytes of M per CTA and second, two reads,
        // relative to a fused CTA's), in whole 64-column strips, every tail
        // CTA with a strip.  The strip groups follow the wave-cost rule of the
        // two-pass path over the idle SMs (16 slabs on 40 SMs: 5 groups, two
        // waves of 40 CTAs, against one wave of 32)
        const int idle = h->num_sms - h->cs * h->nclusters;
        int gt = 0;
        double tail_ctas = 0.0;   // tail CTAs running at a time
        if (idle >= h->nslabs) {
          auto waves = [&](int g) { return (h->nslabs * g + idle - 1) / idle; };
          auto cost = [&](int g) { return (double)waves(g) / (double)g; };
          double best = cost(1);
          for (int g = 2; g <= kTailMaxGroups; ++g) best = std::min(best, cost(g));
          gt = 1;
          while (cost(gt) > 1.06 * best) ++gt;
          tail_ctas = (double)h->nslabs * gt / waves(gt);
        }
        if (h->nclusters == ncl && gt >= 1 && nstrips64 >= kTailMinStrips) {
          const double tr = kTailRate * tail_ctas;
          int64_t st = (int64_t)((double)nstrips64 * tr / (tr + h->cs * h->nclusters));
          st = std::min<int64_t>(st, nstrips64 - h->nclusters);   // every cluster keeps a strip
          if (st >= 2 * gt && tc2_prepare(Rf) == cudaSuccess) {
            // whole strips for the head: a ragged last strip goes to the tail
            h->G_tail = gt;
            h->n_tail = st * 64 - (h->n % 64 ? 64 - h->n % 64 : 0);
          }
          cudaGetLastError();
        }
      } else if (p->path == 2) {
        dcf_destroy(h);
        return DCF_EINVAL;
      }
    }
  }
  // two-pass tensor-core path: any m that is a multiple of 4 (TMA row stride),
  // r <= 64; chosen automatically where the fused path does not apply because
  // of the size (m > 4096 or r > 32)
  if (!local) {
    const bool tc2_ok = h->m % 4 == 0;
    if (p->path == 3 && !tc2_ok) {
      dcf_destroy(h);
      return DCF_EINVAL;
    }
    const bool want = p->path == 3 || (p->path == 0 && h->path == 1 && tc2_ok &&
                                        (h->m > 4096 || p->r > 32));
    if (want) {
      const int Rt = p->r <= 16 ? 16 : p->r <= 32 ? 32 : 64;
      if (tc2_prepare(Rt) != cudaSuccess || (Rt == 64 && fused_prep_prepare() != cudaSuccess)) {
        cudaGetLastError();
        dcf_destroy(h);
        return DCF_ECUDA;
      }
      h->path = 3;
      h->R = Rt;
      h->nslabs = (int)((h->m + 255) / 256);
      const int64_t nstrips64 = (h->n + 63) / 64;
      // one CTA per SM (the kernels hold 200+ KB of shared memory).  G strip
      // groups per slab make nslabs x G equal CTAs in ceil(nslabs G / SMs) waves,
      // so a pass takes time in proportion to ceil(nslabs G / SMs) / G: the
      // smallest G within 6 % of the best (64 slabs on 152 SMs: G = 7, three
      // waves on every SM, against one wave of G = 2 on 128 SMs), every CTA
      // with at least one strip
      {
        const int64_t gmax = std::max<int64_t>(
            1, std::min<int64_t>(nstrips64, std::max<int64_t>(32, h->num_sms / h->nslabs)));
        auto cost = [&](int64_t g) {
          return (double)((h->nslabs * g + h->num_sms - 1) / h->num_sms) / (double)g;
        };
        double best = cost(1);
        for (int64_t g = 2; g <= gmax; ++g) best = std::min(best, cost(g));
        int64_t g = 1;
        while (cost(g) > 1.06 * best) ++g;
        h->G = (int)g;
      }
    }
  }
  // launch geometry
  const int64_t nstrips = (h->n + 63) / 64;
  h->n_vblocks = (int)std::min<int64_t>(nstrips, 3LL * h->num_sms);
  if (h->n_vblocks > 0) {
    int64_t waves = (nstrips + h->n_vblocks - 1) / h->n_vblocks;
    h->n_vblocks = (int)((nstrips + waves - 1) / waves);
  }
  const int64_t rb = (h->m + 127) / 128;
  int64_t splits = std::max<int64_t>(1, (4LL * h->num_sms + rb - 1) / rb);
  splits = std::min<int64_t>(splits, (h->n + 31) / 32);
  h->split_cols = ((h->n + splits - 1) / splits + 31) / 32 * 32;
  h->n_splits = (int)((h->n + h->split_cols - 1) / h->split_cols);
  h->n_rblocks = (int)((h->m + 31) / 32);
  // Gram partials of V: one CTA per SM at R >= 32 (4 x 4 register tiles), two below
  h->n_vgram = (int)std::min<int64_t>((h->R >= 32 ? 1LL : 2LL) * h->num_sms, (h->n + 31) / 32);

  const size_t R = h->R, RR = R * R;
  bool ok = true;
  auto A = [&](size_t bytes) {
    void* q = dev_alloc(h, bytes);
    if (!q) ok = false;
    return q;
  };
  h->U[0] = (float*)A(h->m * R * 4);
  h->U[1] = (float*)A(h->m * R * 4);
  h->V[0] = (float*)A(h->n * R * 4);
  h->V[1] = (float*)A(h->n * R * 4);
  h->W = (float*)A(h->m * R * 4);
  h->part_p = (float*)A((size_t)h->n_splits * h->m * R * 4);
  h->part_h = (double*)A((size_t)h->n_vblocks * 8);
  size_t ngp = std::max<size_t>(h->n_vgram, h->n_rblocks);
  h->part_q = (float2*)A(ngp * RR * 8);
  h->part_xv = (float2*)A((size_t)h->n_vgram * RR * 8);
  h->part_dv = (float2*)A((size_t)h->n_vgram * RR * 8);
  h->part_g = (float2*)A(ngp * RR * 8);
  h->part_xu = (float2*)A((size_t)h->n_rblocks * RR * 8);
  h->part_du = (float2*)A((size_t)h->n_rblocks * RR * 8);
  h->red = (double*)A((6 * RR + 8) * 8);
  h->sm = (Smalls*)A(sizeof(Smalls));
  h->st = (DevState*)A(sizeof(DevState));
  h->counters = (unsigned int*)A(4 * sizeof(unsigned int));
  h->flag = (int*)A(sizeof(int));
  h->mflag = (int*)A(2 * sizeof(int));
  h->kerr = (int*)A(sizeof(int));
  if (h->path == 2) {
    const size_t grid = (size_t)h->cs * h->nclusters;
    const size_t tail_ctas = h->n_tail > 0 ? (size_t)h->nslabs * h->G_tail : 0;
    const size_t tail_groups = h->n_tail > 0 ? (size_t)h->G_tail : 0;
    h->img = (uint8_t*)A((size_t)h->nslabs * 2048 * R);
    h->scales = (float*)A((2 * (size_t)h->nslabs + 1) * sizeof(float));
    h->zmat = (float*)A(RR * sizeof(float));
    h->W_vz = (float*)A((size_t)h->n * R * sizeof(float));
    h->vmax = (unsigned int*)A(2 * sizeof(unsigned int));
    h->part_p = (float*)A(((size_t)h->nclusters + tail_groups) * h->m * R * 4);
    h->part_h = (double*)A((grid + tail_ctas) * 8);
    if (h->n_tail > 0) {
      h->ypart_tail = (float*)A((size_t)h->nslabs * h->n_tail * R * sizeof(float));
      h->vmax_tail = (unsigned int*)A(2 * sizeof(unsigned int));
    }
  }
  if (h->path == 3) {
    h->img = (uint8_t*)A((size_t)h->nslabs * 2048 * R);
    h->scales = (float*)A((2 * (size_t)h->nslabs + 1) * sizeof(float));
    h->zmat = (float*)A(RR * sizeof(float));
    h->W_vz = (float*)A((size_t)h->n * R * sizeof(float));
    h->vmax = (unsigned int*)A(2 * sizeof(unsigned int));
    h->ypart = (float*)A((size_t)h->nslabs * h->n * R * sizeof(float));
    h->part_p = (float*)A((size_t)h->G * h->m * R * 4);
    h->part_h = (double*)A(std::max<size_t>((size_t)h->nslabs * h->G, h->n_vblocks) * 8);
  }
  if (!ok) {
    dcf_destroy(h);
    return DCF_ENOMEM;
  }
  if (h->n_tail > 0) {
    // the tail's stream at the lowest priority, the fused kernel at the highest,
    // so that its clusters are placed before the tail's CTAs fill the rest
    int least = 0, greatest = 0;
    if (cudaDeviceGetStreamPriorityRange(&least, &greatest) != cudaSuccess ||
        cudaStreamCreateWithPriority(&h->tail_stream, cudaStreamNonBlocking, least) !=
            cudaSuccess ||
        cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming) != cudaSuccess) {
      dcf_destroy(h);
      return DCF_ECUDA;
    }
    h->prio_high = greatest;
  }
  if (cudaMemsetAsync(h->U[0], 0, h->m * R * 4, h->stream) != cudaSuccess ||
      cudaMemsetAsync(h->U[1], 0, h->m * R * 4, h->stream) != cudaSuccess ||
      cudaMemsetAsync(h->V[0], 0, h->n * R * 4, h->stream) != cudaSuccess ||
      cudaMemsetAsync(h->V[1], 0, h->n * R * 4, h->stream) != cudaSuccess ||
      cudaMemsetAsync(h->counters, 0, 16, h->stream) != cudaSuccess ||
      cudaMemsetAsync(h->kerr, 0, sizeof(int), h->stream) != cudaSuccess ||
      cudaMemsetAsync(h->st, 0, sizeof(DevState), h->stream) != cudaSuccess ||
      cudaStreamSynchronize(h->stream) != cudaSuccess) {
    dcf_destroy(h);
    return DCF_ECUDA;
  }
  if (local) {
    // one client per block: its own U_i, the block's V_i, the block of M
    // borrowed from this handle at load, its share rho n_i / n of the ridge
    // term in the U-step, work ordered on this handle's internal stream
    dcf_params cp = *p;
    cp.E = 1;
    cp.local_steps = 1;
    cp.u_mode = 1;
    h->clients.assign(p->E, nullptr);
    for (int i = 0; i < p->E; ++i) {
      cp.n_i = &h->n_i[i];
      dcf_status cst = dcf_create(&cp, &h->clients[i]);
      if (cst != DCF_OK) {
        dcf_destroy(h);
        return cst;
      }
      h->clients[i]->rho_u = h->rho * (double)h->n_i[i] / (double)h->n;
      h->clients[i]->user_stream = h->stream;
    }
    h->client_path = h->clients[0]->path;
    h->loc_uptr = (const float**)dev_alloc(h, (size_t)p->E * sizeof(float*));
    h->loc_h = (double*)dev_alloc(h, (size_t)p->E * sizeof(double));
    if (!h->loc_uptr || !h->loc_h) {
      dcf_destroy(h);
      return DCF_ENOMEM;
    }
    // after its K local steps (started from copy 0) a client's U is in copy K & 1
    std::vector<const float*> up(p->E);
    for (int i = 0; i < p->E; ++i) up[i] = h->clients[i]->U[p->local_steps & 1];
    if (cudaMemcpy(h->loc_uptr, up.data(), up.size() * sizeof(float*),
                   cudaMemcpyHostToDevice) != cudaSuccess) {
      dcf_destroy(h);
      return DCF_ECUDA;
    }
  }
  const double mn = (double)h->m * (double)h->n;
  if (h->rho * h->rho > h->lam * h->lam * mn)
    h->err = "warning: rho^2 > lambda^2 m n; the necessary condition for exact recovery fails";
  *out = h;
  return DCF_OK;
}

extern "C" int dcf_kernels_per_iteration(dcf_handle h) {
  if (!h) return 0;
  if (!h->clients.empty()) return -1;   // rounds of local steps: not one fixed graph
  switch (h->path) {
    case 2: return h->n_tail > 0 ? 9 : 6;   // + the tail's pass A, V' reduction, pass B
    case 3: return h->R == 64 ? 9 : 8;     // V_old Z in its own launch at R = 64
    case 4: return 1;                      // every iteration of a call in one launch
    default: return 7;
  }
}

extern "C" int dcf_get_path(dcf_handle h) {
  if (!h) return 0;
  return h->clients.empty() ? h->path : h->client_path;
}

extern "C" dcf_status dcf_set_stream(dcf_handle h, void* stream) {
  if (!h) return DCF_EINVAL;
  h->user_stream = (cudaStream_t)stream;
  return DCF_OK;
}

namespace dcf {
namespace api {

// Enqueue the copy of the blocks into dst on stream cs and their NaN/Inf check
// into *flag on stream ks: block i is checked while block i + 1 is copied,
// and cs waits for the last check at the end.
static dcf_status enqueue_copy_check(dcf_handle h, float* dst, const float* const* M_i,
                                     const int64_t* ld_i, int where, int* flag, cudaStream_t cs,
                                     cudaStream_t ks, cudaEvent_t ev) {
  cudaMemcpyKind kind = where == 0 ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  CK(cudaMemsetAsync(flag, 0, sizeof(int), cs), "memset");
  for (int i = 0; i < h->E; ++i) {
    int64_t ld = ld_i ? ld_i[i] : h->m;
    float* d = dst + h->c_i[i] * h->m;
    CK(cudaMemcpy2DAsync(d, h->m * sizeof(float), M_i[i], ld * sizeof(float),
                         h->m * sizeof(float), h->n_i[i], kind, cs),
       "copy block");
    CK(cudaEventRecord(ev, cs), "record");
    CK(cudaStreamWaitEvent(ks, ev, 0), "wait");
    CK(launch_check_finite(d, h->m * h->n_i[i], flag, ks), "check block");
  }
  CK(cudaEventRecord(ev, ks), "record");
  CK(cudaStreamWaitEvent(cs, ev, 0), "wait");
  return DCF_OK;
}

// Copy the blocks into the buffer in use (h->M) and check them; returns after
// both have completed (*nonfinite set when a value failed).
static dcf_status copy_blocks_checked(dcf_handle h, const float* const* M_i, const int64_t* ld_i,
                                      int where, bool* nonfinite) {
  dcf_status st = enqueue_copy_check(h, h->M, M_i, ld_i, where, h->flag, h->stream, h->side,
                                     h->ev_side);
  if (st != DCF_OK) return st;
  int flag = 0;
  CK(cudaMemcpyAsync(&flag, h->flag, sizeof(int), cudaMemcpyDeviceToHost, h->stream), "flag");
  CK(cudaStreamSynchronize(h->stream), "sync");
  *nonfinite = flag != 0;
  return DCF_OK;
}

// Own buffer b of M (allocated on first use) and its tensor map.
static dcf_status ensure_mbuf(dcf_handle h, int b) {
  if (h->Mbuf[b]) return DCF_OK;
  h->Mbuf[b] = (float*)dev_alloc(h, (size_t)h->m * h->n * sizeof(float));
  if (!h->Mbuf[b]) return fail(h, DCF_ENOMEM, "cannot allocate M");
  if ((h->path == 2 || h->path == 3) && fused_make_tmap(h->tmaps[b], h->Mbuf[b], h->m, h->n) != 0)
    return fail(h, DCF_ECUDA, "cuTensorMapEncodeTiled failed for M");
  if (h->n_tail > 0 && fused_make_tmap(h->tmaps_tail[b], h->Mbuf[b] + (h->n - h->n_tail) * h->m,
                                       h->m, h->n_tail) != 0)
    return fail(h, DCF_ECUDA, "cuTensorMapEncodeTiled failed for the tail of M");
  return DCF_OK;
}

static dcf_status check_block_args(dcf_handle h, const float* const* M_i, const int64_t* ld_i,
                                   int where) {
  if (!M_i) return fail(h, DCF_EINVAL, "M_i is NULL");
  if (where != 0 && where != 1) return fail(h, DCF_EINVAL, "where must be 0 or 1");
  for (int i = 0; i < h->E; ++i) {
    if (!M_i[i]) return fail(h, DCF_EINVAL, "a block pointer is NULL");
    if (ld_i && ld_i[i] < h->m) return fail(h, DCF_EINVAL, "ld_i < m");
  }
  return DCF_OK;
}

}  // namespace api
}  // namespace dcf

extern "C" dcf_status dcf_load_blocks(dcf_handle h, const float* const* M_i, const int64_t* ld_i,
                                      int where, int borrow) {
  if (!h) return DCF_EINVAL;
  dcf_status st = check_block_args(h, M_i, ld_i, where);
  if (st != DCF_OK) return st;
  st = begin_work(h);
  if (st != DCF_OK) return st;
  if ((st = drop_pending(h)) != DCF_OK) return st;
  bool contiguous = where == 1;
  for (int i = 0; i < h->E && contiguous; ++i) {
    if (ld_i && ld_i[i] != h->m) contiguous = false;
    if (i > 0 && M_i[i] != M_i[i - 1] + h->m * h->n_i[i - 1]) contiguous = false;
  }
  bool nonfinite = false;
  if (borrow && where == 1) {
    if (!contiguous)
      return fail(h, DCF_EINVAL, "borrowed blocks must form one contiguous column-major matrix");
    h->M = const_cast<float*>(M_i[0]);
    h->M_borrowed = true;
    CK(cudaMemsetAsync(h->flag, 0, sizeof(int), h->stream), "memset");
    CK(launch_check_finite(h->M, h->m * h->n, h->flag, h->stream), "check M");
    int flag = 0;
    CK(cudaMemcpyAsync(&flag, h->flag, sizeof(int), cudaMemcpyDeviceToHost, h->stream), "flag");
    CK(cudaStreamSynchronize(h->stream), "sync");
    nonfinite = flag != 0;
  } else {
    if ((st = ensure_mbuf(h, h->mcur)) != DCF_OK) return st;
    h->M = h->Mbuf[h->mcur];
    h->M_borrowed = false;
    st = copy_blocks_checked(h, M_i, ld_i, where, &nonfinite);
    if (st != DCF_OK) return st;
  }
  if (nonfinite) return fail(h, DCF_ENONFINITE, "M contains NaN or Inf");
  if (h->path == 2 || h->path == 3) {
    if (h->M_borrowed) {
      if (fused_make_tmap(h->tmap, h->M, h->m, h->n) != 0)
        return fail(h, DCF_ECUDA, "cuTensorMapEncodeTiled failed for M");
      if (h->n_tail > 0 &&
          fused_make_tmap(h->tmap_tail, h->M + (h->n - h->n_tail) * h->m, h->m, h->n_tail) != 0)
        return fail(h, DCF_ECUDA, "cuTensorMapEncodeTiled failed for the tail of M");
    } else {
      std::memcpy(h->tmap, h->tmaps[h->mcur], sizeof(h->tmap));
      std::memcpy(h->tmap_tail, h->tmaps_tail[h->mcur], sizeof(h->tmap_tail));
    }
  }
  h->loaded = true;
  h->initialized = false;
  for (int b = 0; b < 2; ++b)
    for (int p = 0; p < 2; ++p)
      if (h->graph[b][p]) { cudaGraphExecDestroy(h->graph[b][p]); h->graph[b][p] = nullptr; }
  // clients of the local-step mode read their block of this handle's M in place
  for (int i = 0; i < (int)h->clients.size(); ++i) {
    const float* blk = h->M + h->c_i[i] * h->m;
    if ((st = dcf_load_blocks(h->clients[i], &blk, nullptr, 1, 1)) != DCF_OK)
      return fail(h, st, std::string("client block: ") + dcf_last_error(h->clients[i]));
  }
  return end_work(h);
}

extern "C" dcf_status dcf_reload_blocks(dcf_handle h, const float* const* M_i,
                                        const int64_t* ld_i, int where) {
  if (!h) return DCF_EINVAL;
  if (!h->loaded) return fail(h, DCF_ESTATE, "dcf_load_blocks has not been called");
  if (h->M_borrowed)
    return fail(h, DCF_ESTATE, "M is borrowed; write the new values into the borrowed matrix");
  dcf_status st = check_block_args(h, M_i, ld_i, where);
  if (st != DCF_OK) return st;
  st = begin_work(h);
  if (st != DCF_OK) return st;
  if ((st = drop_pending(h)) != DCF_OK) return st;
  bool nonfinite = false;
  st = copy_blocks_checked(h, M_i, ld_i, where, &nonfinite);
  if (st != DCF_OK) return st;
  if (nonfinite) {
    h->loaded = false;   // M now holds the rejected values: no step may run on them
    return fail(h, DCF_ENONFINITE, "M contains NaN or Inf");
  }
  return end_work(h);
}

extern "C" dcf_status dcf_reload_blocks_async(dcf_handle h, const float* const* M_i,
                                              const int64_t* ld_i, int where) {
  if (!h) return DCF_EINVAL;
  if (!h->clients.empty())
    return fail(h, DCF_EINVAL, "asynchronous reloads are not available with local_steps > 1");
  if (!h->loaded) return fail(h, DCF_ESTATE, "dcf_load_blocks has not been called");
  if (h->M_borrowed)
    return fail(h, DCF_ESTATE, "M is borrowed; write the new values into the borrowed matrix");
  dcf_status st = check_block_args(h, M_i, ld_i, where);
  if (st != DCF_OK) return st;
  st = begin_work(h);
  if (st != DCF_OK) return st;
  // a pending reload's buffer is overwritten (after its copy: same stream)
  const int tgt = h->pend >= 0 ? h->pend : 1 - h->mcur;
  if ((st = ensure_mbuf(h, tgt)) != DCF_OK) return st;
  // after every enqueued iteration that reads the target buffer, and for
  // device sources after the caller's stream (which may produce them; it is
  // itself behind the enqueued iterations, so host sources skip this wait)
  if (where == 1) CK(cudaStreamWaitEvent(h->side, h->ev_in, 0), "wait");
  CK(cudaStreamWaitEvent(h->side, h->ev_used[tgt], 0), "wait");
  st = enqueue_copy_check(h, h->Mbuf[tgt], M_i, ld_i, where, h->mflag + tgt, h->side, h->side2,
                          h->ev_side2);
  if (st != DCF_OK) return st;
  CK(cudaEventRecord(h->ev_copy, h->side), "record");
  h->pend = tgt;
  return end_work(h);
}

extern "C" dcf_status dcf_load_init(dcf_handle h, const float* U0, const float* const* V0_i,
                                    int where) {
  if (!h) return DCF_EINVAL;
  if (!h->loaded) return fail(h, DCF_ESTATE, "dcf_load_blocks has not been called");
  if (!U0) return fail(h, DCF_EINVAL, "U0 is NULL");
  if (where != 0 && where != 1) return fail(h, DCF_EINVAL, "where must be 0 or 1");
  dcf_status st = begin_work(h);
  if (st != DCF_OK) return st;
  if ((st = apply_pending(h)) != DCF_OK) return st;   // the start-point sweep reads M
  cudaMemcpyKind kind = where == 0 ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  CK(cudaMemsetAsync(h->U[0], 0, h->m * h->R * 4, h->stream), "memset");
  CK(cudaMemcpy2DAsync(h->U[0], h->R * 4, U0, h->r * 4, h->r * 4, h->m, kind, h->stream), "copy U0");
  bool have_v0 = V0_i != nullptr;
  if (have_v0) {
    CK(cudaMemsetAsync(h->V[0], 0, h->n * h->R * 4, h->stream), "memset");
    for (int i = 0; i < h->E; ++i) {
      if (!V0_i[i]) return fail(h, DCF_EINVAL, "a V0 block pointer is NULL");
      CK(cudaMemcpy2DAsync(h->V[0] + h->c_i[i] * h->R, h->R * 4, V0_i[i], h->r * 4, h->r * 4,
                           h->n_i[i], kind, h->stream), "copy V0");
    }
  }
  st = finish_init(h, have_v0);
  if (st != DCF_OK) return st;
  return end_work(h);
}

namespace dcf {
namespace api {

// One communication round t of Algorithm 1 with K = local_steps > 1 (FedAvg
// mode), enqueued on h->stream:
//   every client i starts from the round's U and its block V_i, then runs K
//   plain iterations of its own block in FedAvg mode with E = 1: S_i, V_i from
//   its current U_i (§2.2 eq. optS, App. B eq. condition1), then
//   U_i <- U_i - eta_t (U_i Q_i - P_i + rho (n_i / n) U_i)   (eq. U_local),
//   eta_t = eta0 / sqrt(t + 1) for all K steps of the round;
//   the server takes U_t = (1/E) sum_i U_i (eq. U_agg) and V_t = [V_1; ...; V_E].
// The clients' streams all wait on h->stream and h->stream waits on every
// client, so the clients of a round run concurrently.  The round's objective
// is that of the K = 1 case, at (U_{t-1}, V_{t-1}, S from the first local
// step): every client's first local step computes its Huber sum at
// (U_{t-1}, V_{i,t-1}).
dcf_status local_round(dcf_handle h) {
  const int cur = h->host_iter & 1, nxt = cur ^ 1;
  const int K = h->local_steps;
  const double eta = h->eta0 / std::sqrt((double)h->host_iter + 1.0);
  dcf_status st;
  for (int i = 0; i < h->E; ++i) {
    dcf_handle c = h->clients[i];
    if ((st = begin_work(c)) != DCF_OK) return fail(h, st, dcf_last_error(c));
    if ((st = apply_pending(c)) != DCF_OK) return fail(h, st, dcf_last_error(c));
    const int64_t ni = h->n_i[i];
    CK(cudaMemsetAsync(c->U[0], 0, (size_t)h->m * c->R * 4, c->stream), "client U");
    CK(cudaMemcpy2DAsync(c->U[0], c->R * 4, h->U[cur], h->R * 4, h->r * 4, h->m,
                         cudaMemcpyDeviceToDevice, c->stream), "client U");
    CK(cudaMemsetAsync(c->V[0], 0, (size_t)ni * c->R * 4, c->stream), "client V");
    CK(cudaMemcpy2DAsync(c->V[0], c->R * 4, h->V[cur] + h->c_i[i] * h->R, h->R * 4, h->r * 4, ni,
                         cudaMemcpyDeviceToDevice, c->stream), "client V");
    if ((st = finish_init(c, true)) != DCF_OK) return fail(h, st, dcf_last_error(c));
    CK(cudaMemcpyAsync(&c->st->eta_fixed, &eta, sizeof(double), cudaMemcpyHostToDevice,
                       c->stream), "client step size");
    if ((st = build_graphs(c)) != DCF_OK) return fail(h, st, dcf_last_error(c));
    for (int k = 0; k < K; ++k) {
      CK(cudaGraphLaunch(c->graph[c->mcur][c->host_iter & 1], c->stream), "client step");
      c->host_iter++;
      if (k == 0)
        CK(cudaMemcpyAsync(h->loc_h + i, &c->st->huber, sizeof(double),
                           cudaMemcpyDeviceToDevice, c->stream), "client Huber sum");
    }
    if ((st = end_work(c)) != DCF_OK) return fail(h, st, dcf_last_error(c));
  }
  for (int i = 0; i < h->E; ++i) {
    dcf_handle c = h->clients[i];
    CK(cudaMemcpy2DAsync(h->V[nxt] + h->c_i[i] * h->R, h->R * 4, c->V[K & 1], c->R * 4, h->r * 4,
                         h->n_i[i], cudaMemcpyDeviceToDevice, h->stream), "V_t");
  }
  IterArgs a = iter_args(h, cur);
  a.part_h = h->loc_h;
  a.n_vblocks = h->E;
  CK(launch_avg_rows(a, h->loc_uptr, h->E, h->clients[0]->R, h->stream), "average");
  CK(launch_gram_vv(h->R, h->V[cur], h->V[nxt], h->n, h->part_q, h->part_xv, h->part_dv, h->n_vgram, h->st,
                    h->stream), "gram V");
  CK(launch_reduce_q(a, red_q(h), red_xv(h), red_dv(h), red_h(h), h->n_vgram, h->counters + 0, h->stream),
     "reduce Q");
  CK(launch_reduce_g(a, red_g(h), red_xu(h), red_du(h), h->counters + 1, h->stream), "reduce G");
  h->host_iter++;
  return DCF_OK;
}

// A bounded wait that expired inside a client's kernels (DCF_ETIMEOUT).
dcf_status check_clients(dcf_handle h) {
  for (dcf_handle c : h->clients) {
    int kerr = 0;
    CK(cudaMemcpyAsync(&kerr, c->kerr, sizeof(int), cudaMemcpyDeviceToHost, c->stream), "err");
    CK(cudaStreamSynchronize(c->stream), "sync");
    if (kerr == DCF_ETIMEOUT)
      return fail(h, DCF_ETIMEOUT, "a bounded device-side wait expired in a client's kernels");
  }
  return DCF_OK;
}

}  // namespace api
}  // namespace dcf

extern "C" dcf_status dcf_step(dcf_handle h, int n_steps) {
  if (!h) return DCF_EINVAL;
  if (n_steps < 0) return fail(h, DCF_EINVAL, "n_steps < 0");
  dcf_status st = begin_work(h);
  if (st != DCF_OK) return st;
  if ((st = ensure_init(h)) != DCF_OK) return st;
  if (!h->clients.empty()) {   // K > 1 local steps per round
    for (int i = 0; i < n_steps; ++i)
      if ((st = local_round(h)) != DCF_OK) return st;
    return end_work(h);
  }
  if (h->path == 4) {   // every iteration in one launch of the whole-solve kernel
    if (n_steps > 0) {
      CK(enqueue_small(h, h->host_iter & 1, n_steps, h->stream), "whole solve");
      h->host_iter += n_steps;
    }
    return end_work(h);
  }
  if ((st = build_graphs(h)) != DCF_OK) return st;
  for (int i = 0; i < n_steps; ++i) {
    CK(cudaGraphLaunch(h->graph[h->mcur][h->host_iter & 1], h->stream), "graph launch");
    h->host_iter++;
  }
  return end_work(h);
}

extern "C" dcf_status dcf_solve(dcf_handle h, int* iters_out, double* final_dL_rel) {
  if (!h) return DCF_EINVAL;
  dcf_status st = begin_work(h);
  if (st != DCF_OK) return st;
  if ((st = ensure_init(h)) != DCF_OK) return st;
  const bool local = !h->clients.empty();
  if (h->path != 4 && !local && (st = build_graphs(h)) != DCF_OK) return st;
  if ((st = set_state_fields(h, 1, h->tol)) != DCF_OK) return st;
  DevState ds{};
  if ((st = read_state(h, &ds)) != DCF_OK) return st;
  const int start = ds.iter;
  int done = 0;
  const int batch = 8;
  // K > 1 local steps: one round at a time, the stop test read after each
  for (; local && done < h->max_iter; ++done) {
    if ((st = local_round(h)) != DCF_OK) return st;
    if ((st = read_state(h, &ds)) != DCF_OK) return st;
    if ((st = check_clients(h)) != DCF_OK) return st;
    if (ds.stop) {
      ++done;
      break;
    }
  }
  if (h->path == 4) {   // one launch runs until the stop test or max_iter
    CK(enqueue_small(h, h->host_iter & 1, h->max_iter, h->stream), "whole solve");
    if ((st = read_state(h, &ds)) != DCF_OK) return st;
    done = h->max_iter;
  }
  while (!local && done < h->max_iter) {
    int nb = std::min(batch, h->max_iter - done);
    for (int i = 0; i < nb; ++i) {
      CK(cudaGraphLaunch(h->graph[h->mcur][h->host_iter & 1], h->stream), "graph launch");
      h->host_iter++;
    }
    done += nb;
    if ((st = read_state(h, &ds)) != DCF_OK) return st;
    if (ds.stop) break;
  }
  h->host_iter = ds.iter;
  int ran = ds.iter - start;
  if (iters_out) *iters_out = ran;
  if (final_dL_rel) *final_dL_rel = ds.dL_rel;
  if ((st = set_state_fields(h, 0, h->tol)) != DCF_OK) return st;
  if ((st = end_work(h)) != DCF_OK) return st;
  if (!ds.stop) return fail(h, DCF_ENOTCONV, "max_iter reached above tol");
  return DCF_OK;
}

extern "C" dcf_status dcf_get_factors(dcf_handle h, float* U, float* const* V_i, int where) {
  if (!h) return DCF_EINVAL;
  if (where != 0 && where != 1) return fail(h, DCF_EINVAL, "where must be 0 or 1");
  dcf_status st = begin_work(h);
  if (st != DCF_OK) return st;
  if ((st = ensure_init(h)) != DCF_OK) return st;
  const int cur = h->host_iter & 1;
  cudaMemcpyKind kind = where == 0 ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  if (U)
    CK(cudaMemcpy2DAsync(U, h->r * 4, h->U[cur], h->R * 4, h->r * 4, h->m, kind, h->stream),
       "copy U");
  if (V_i) {
    for (int i = 0; i < h->E; ++i) {
      if (!V_i[i]) continue;
      CK(cudaMemcpy2DAsync(V_i[i], h->r * 4, h->V[cur] + h->c_i[i] * h->R, h->R * 4, h->r * 4,
                           h->n_i[i], kind, h->stream), "copy V");
    }
  }
  if (where == 0) CK(cudaStreamSynchronize(h->stream), "sync");
  return end_work(h);
}

extern "C" dcf_status dcf_set_private(dcf_handle h, int i, int is_private) {
  if (!h) return DCF_EINVAL;
  if (i < 0 || i >= h->E) return fail(h, DCF_EINVAL, "block index out of range");
  h->priv[i] = is_private ? 1 : 0;
  return DCF_OK;
}

extern "C" dcf_status dcf_get_LS(dcf_handle h, int i, float* L_i, float* S_i, int where) {
  if (!h) return DCF_EINVAL;
  if (i < 0 || i >= h->E) return fail(h, DCF_EINVAL, "block index out of range");
  if (where != 0 && where != 1) return fail(h, DCF_EINVAL, "where must be 0 or 1");
  if (h->priv[i]) return fail(h, DCF_EPRIVATE, "block is private");
  if (!h->initialized || h->host_iter < 1)
    return fail(h, DCF_ESTATE, "no iteration has run yet");
  dcf_status st = begin_work(h);
  if (st != DCF_OK) return st;
  const int cur = h->host_iter & 1, prev = cur ^ 1;
  const int64_t ni = h->n_i[i], c0 = h->c_i[i];
  const size_t bytes = (size_t)h->m * ni * sizeof(float);
  float* tmp = nullptr;
  if (where == 0) {
    CK(cudaMallocAsync((void**)&tmp, bytes, h->stream), "tmp");
  }
  for (int which = 0; which < 2; ++which) {
    float* dst = which == 0 ? L_i : S_i;
    if (!dst) continue;
    float* target = where == 0 ? tmp : dst;
    const float* Uu = which == 0 ? h->U[cur] : h->U[prev];
    const float* Vv = which == 0 ? h->V[cur] : h->V[prev];
    if (which == 1 && !h->clients.empty()) {
      // K > 1 local steps: the S of block i's last local step, from that
      // step's inputs (the client's copy before its last iteration)
      dcf_handle c = h->clients[i];
      const int cp = (c->host_iter & 1) ^ 1;
      CK(launch_materialize(c->M, h->m, 0, ni, c->U[cp], c->V[cp], c->R, (float)h->lam, 1,
                            target, h->stream), "materialize");
    } else {
      CK(launch_materialize(h->M, h->m, c0, ni, Uu, Vv, h->R, (float)h->lam, which, target,
                            h->stream), "materialize");
    }
    if (where == 0)
      CK(cudaMemcpyAsync(dst, tmp, bytes, cudaMemcpyDeviceToHost, h->stream), "copy out");
  }
  if (tmp) CK(cudaFreeAsync(tmp, h->stream), "free tmp");
  if (where == 0) CK(cudaStreamSynchronize(h->stream), "sync");
  return end_work(h);
}

extern "C" dcf_status dcf_get_stats(dcf_handle h, double* objective, double* dL_rel, int* iter) {
  if (!h) return DCF_EINVAL;
  dcf_status st = begin_work(h);
  if (st != DCF_OK) return st;
  DevState ds{};
  if ((st = read_state(h, &ds)) != DCF_OK) return st;
  if (objective) *objective = ds.objective;
  if (dL_rel) *dL_rel = ds.dL_rel;
  if (iter) *iter = ds.iter;
  return end_work(h);
}

extern "C" dcf_status dcf_get_conditioning(dcf_handle h, double* kappa_g, double* kappa_h,
                                           int* route_g, int* route_h) {
  if (!h) return DCF_EINVAL;
  dcf_status st = begin_work(h);
  if (st != DCF_OK) return st;
  DevState ds{};
  if ((st = read_state(h, &ds)) != DCF_OK) return st;
  if (kappa_g) *kappa_g = ds.kappa_g;
  if (kappa_h) *kappa_h = ds.kappa_h;
  if (route_g) *route_g = ds.route_g;
  if (route_h) *route_h = ds.route_h;
  return end_work(h);
}

extern "C" dcf_status dcf_set_truth(dcf_handle h, const float* A, const float* B, int k,
                                    int where) {
  if (!h) return DCF_EINVAL;
  if (!A || !B || k < 1 || k > kMaxR) return fail(h, DCF_EINVAL, "truth factors");
  if (where != 0 && where != 1) return fail(h, DCF_EINVAL, "where must be 0 or 1");
  dcf_status st = begin_work(h);
  if (st != DCF_OK) return st;
  if (!h->A_truth || h->k_truth != k) {
    h->A_truth = (float*)dev_alloc(h, (size_t)h->m * k * 4);
    h->B_truth = (float*)dev_alloc(h, (size_t)h->n * k * 4);
    h->truth_part = (float2*)dev_alloc(h, (size_t)2 * h->num_sms * kMaxR * kMaxR * 8);
    h->truth_red = (double*)dev_alloc(h, (size_t)6 * kMaxR * kMaxR * 8);
    if (!h->A_truth || !h->B_truth || !h->truth_part || !h->truth_red)
      return fail(h, DCF_ENOMEM, "truth buffers");
  }
  h->k_truth = k;
  cudaMemcpyKind kind = where == 0 ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  CK(cudaMemcpyAsync(h->A_truth, A, (size_t)h->m * k * 4, kind, h->stream), "copy A");
  CK(cudaMemcpyAsync(h->B_truth, B, (size_t)h->n * k * 4, kind, h->stream), "copy B");
  if (where == 0) CK(cudaStreamSynchronize(h->stream), "sync");
  return end_work(h);
}

extern "C" dcf_status dcf_singular_values(dcf_handle h, double* sigma, double* sigma0,
                                          double* err) {
  if (!h) return DCF_EINVAL;
  if (!sigma) return fail(h, DCF_EINVAL, "sigma is NULL");
  const bool want0 = sigma0 || err;
  if (want0 && !h->A_truth) return fail(h, DCF_ESTATE, "no truth registered");
  dcf_status st = begin_work(h);
  if (st != DCF_OK) return st;
  if ((st = ensure_init(h)) != DCF_OK) return st;
  const int nparts = std::max(1, 2 * h->num_sms);
  if (!h->sv_part) {
    CK(sv_prepare(), "singular-value kernel attributes");
    h->sv_part = (double*)dev_alloc(h, sv_part_doubles(nparts) * 8);
    h->sv_gram = (double*)dev_alloc(h, (size_t)4 * 64 * 64 * 8);
    h->sv_pdim = (int*)dev_alloc(h, 2 * sizeof(int));
    h->sv_out = (double*)dev_alloc(h, (size_t)(2 * 64 + 1) * 8);
    if (!h->sv_part || !h->sv_gram || !h->sv_pdim || !h->sv_out)
      return fail(h, DCF_ENOMEM, "singular-value buffers");
  }
  const int cur = h->host_iter & 1;
  const int r = h->r, R = h->R, k = h->k_truth;
  const int nprob = want0 ? 2 : 1;
  const int pd[2] = {r, want0 ? k : 0};
  const size_t G = (size_t)64 * 64;
  // problem 0: L = U V^T (first r columns of the padded factors);
  // problem 1: L0 = A B^T (the registered truth, rank <= k)
  CK(launch_gram64(h->U[cur], R, h->U[cur], R, r, h->m, h->sv_part, nparts, h->sv_gram,
                   h->stream), "gram U");
  CK(launch_gram64(h->V[cur], R, h->V[cur], R, r, h->n, h->sv_part, nparts, h->sv_gram + G,
                   h->stream), "gram V");
  if (want0) {
    CK(launch_gram64(h->A_truth, k, h->A_truth, k, k, h->m, h->sv_part, nparts,
                     h->sv_gram + 2 * G, h->stream), "gram A");
    CK(launch_gram64(h->B_truth, k, h->B_truth, k, k, h->n, h->sv_part, nparts,
                     h->sv_gram + 3 * G, h->stream), "gram B");
  }
  CK(cudaMemcpyAsync(h->sv_pdim, pd, sizeof(pd), cudaMemcpyHostToDevice, h->stream), "pdim");
  CK(launch_sv_factored(h->sv_gram, h->sv_pdim, nprob, h->sv_out, h->stream), "sv");
  if (want0) CK(launch_sv_error(h->sv_out, h->sv_out + 64, k, h->sv_out + 128, h->stream),
                "sv error");
  double host[2 * 64 + 1];
  CK(cudaMemcpyAsync(host, h->sv_out, sizeof(host), cudaMemcpyDeviceToHost, h->stream), "copy");
  CK(cudaStreamSynchronize(h->stream), "sync");
  for (int i = 0; i < r; ++i) sigma[i] = host[i];
  if (sigma0)
    for (int i = 0; i < k; ++i) sigma0[i] = host[64 + i];
  if (err) *err = host[128];
  return end_work(h);
}

extern "C" dcf_status dcf_rel_err(dcf_handle h, double* rel_err_L) {
  if (!h) return DCF_EINVAL;
  if (!h->A_truth) return fail(h, DCF_ESTATE, "no truth registered");
  if (!rel_err_L) return fail(h, DCF_EINVAL, "rel_err_L is NULL");
  dcf_status st = begin_work(h);
  if (st != DCF_OK) return st;
  if ((st = ensure_init(h)) != DCF_OK) return st;
  const int cur = h->host_iter & 1;
  const int R = h->R, k = h->k_truth;
  const int np = (int)std::min<int64_t>(2LL * h->num_sms, std::max<int64_t>(1, h->n / 32));
  // six Gram matrices: U^T U, V^T V, U^T A, V^T B, A^T A, B^T B
  struct G { const float* X; int cx; const float* Y; int cy; int64_t N; } gs[6] = {
      {h->U[cur], R, h->U[cur], R, h->m}, {h->V[cur], R, h->V[cur], R, h->n},
      {h->U[cur], R, h->A_truth, k, h->m}, {h->V[cur], R, h->B_truth, k, h->n},
      {h->A_truth, k, h->A_truth, k, h->m}, {h->B_truth, k, h->B_truth, k, h->n}};
  std::vector<double> host[6];
  for (int g = 0; g < 6; ++g) {
    int npg = (int)std::min<int64_t>(np, std::max<int64_t>(1, gs[g].N / 32));
    CK(launch_gram(gs[g].X, gs[g].cx, gs[g].cx, gs[g].Y, gs[g].cy, gs[g].cy, gs[g].N,
                   h->truth_part, npg, h->st, 0, h->stream), "truth gram");
    int cnt = gs[g].cx * gs[g].cy;
    CK(launch_reduce_plain(h->truth_part, npg, cnt, h->truth_red + (size_t)g * kMaxR * kMaxR,
                           h->stream), "truth reduce");
    host[g].resize(cnt);
  }
  for (int g = 0; g < 6; ++g)
    CK(cudaMemcpyAsync(host[g].data(), h->truth_red + (size_t)g * kMaxR * kMaxR,
                       host[g].size() * 8, cudaMemcpyDeviceToHost, h->stream), "copy");
  CK(cudaStreamSynchronize(h->stream), "sync");
  // ||UV^T - AB^T||^2 = <U^T U, V^T V> - 2 <U^T A, V^T B> + <A^T A, B^T B>  (r x r / r x k)
  double a = 0, b = 0, c = 0;
  for (int i = 0; i < R * R; ++i) a += host[0][i] * host[1][i];
  for (int i = 0; i < R * k; ++i) b += host[2][i] * host[3][i];
  for (int i = 0; i < k * k; ++i) c += host[4][i] * host[5][i];
  double d2 = std::max(0.0, a - 2 * b + c);
  *rel_err_L = c > 0 ? std::sqrt(d2 / c) : INFINITY;
  return end_work(h);
}

extern "C" int dcf_profile_phases(dcf_handle h, char* names_csv, int len) {
  if (!h) return -1;
  std::string all;
  for (int p = 0; p < num_phases(h); ++p) {
    if (p) all += ",";
    all += phase_name(h, p);
  }
  if (names_csv && len > 0) {
    std::strncpy(names_csv, all.c_str(), (size_t)len - 1);
    names_csv[len - 1] = 0;
  }
  return num_phases(h);
}

extern "C" dcf_status dcf_profile_step(dcf_handle h, int n_steps, double* phase_ms) {
  if (!h) return DCF_EINVAL;
  if (!h->clients.empty())
    return fail(h, DCF_EINVAL, "per-phase profiling is not available with local_steps > 1");
  if (n_steps < 1 || !phase_ms) return fail(h, DCF_EINVAL, "n_steps < 1 or phase_ms NULL");
  dcf_status st = begin_work(h);
  if (st != DCF_OK) return st;
  if ((st = ensure_init(h)) != DCF_OK) return st;
  const int np = num_phases(h);
  constexpr int kMaxPhases = kNumTc2Phases;   // the largest phase count of the three paths
  static_assert(kNumTc2Phases >= kNumPhases && kNumTc2Phases >= kNumFusedPhases, "phases");
  cudaEvent_t ev[kMaxPhases + 1];
  for (int p = 0; p <= np; ++p) CK(cudaEventCreate(&ev[p]), "event");
  for (int p = 0; p < np; ++p) phase_ms[p] = 0.0;
  for (int i = 0; i < n_steps; ++i) {
    CK(cudaEventRecord(ev[0], h->stream), "record");
    CK(enqueue_iteration(h, h->host_iter & 1, h->stream, ev + 1), "profiled iteration");
    h->host_iter++;
    CK(cudaEventSynchronize(ev[np]), "sync");
    for (int p = 0; p < np; ++p) {
      float ms = 0.f;
      CK(cudaEventElapsedTime(&ms, ev[p], ev[p + 1]), "elapsed");
      phase_ms[p] += ms;
    }
  }
  for (int p = 0; p <= np; ++p) cudaEventDestroy(ev[p]);
  return end_work(h);
}

extern "C" void dcf_destroy(dcf_handle h) {
  if (!h) return;
  if (h->stream) cudaStreamSynchronize(h->stream);
  for (dcf_handle c : h->clients) dcf_destroy(c);
  h->clients.clear();
  free_unrolled(h);
  if (h->side) cudaStreamSynchronize(h->side);
  for (int b = 0; b < 2; ++b)
    for (int p = 0; p < 2; ++p)
      if (h->graph[b][p]) cudaGraphExecDestroy(h->graph[b][p]);
  dev_free_all(h);
  if (h->ev_in) cudaEventDestroy(h->ev_in);
  if (h->ev_out) cudaEventDestroy(h->ev_out);
  if (h->ev_side) cudaEventDestroy(h->ev_side);
  if (h->ev_copy) cudaEventDestroy(h->ev_copy);
  if (h->ev_side2) cudaEventDestroy(h->ev_side2);
  for (int b = 0; b < 2; ++b)
    if (h->ev_used[b]) cudaEventDestroy(h->ev_used[b]);
  if (h->stream) cudaStreamDestroy(h->stream);
  if (h->tail_stream) cudaStreamDestroy(h->tail_stream);
  if (h->ev_fork) cudaEventDestroy(h->ev_fork);
  if (h->ev_join) cudaEventDestroy(h->ev_join);
  if (h->side) cudaStreamDestroy(h->side);
  if (h->side2) cudaStreamDestroy(h->side2);
  delete h;
}
