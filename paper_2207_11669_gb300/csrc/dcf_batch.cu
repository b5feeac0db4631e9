// Batches of independent DCF-PCA problems (dcf_batch_*): every instance has
// its own M (any m, column blocks n_i) and rank r <= 32, and one iteration of
// the whole batch is one CUDA graph whose kernels are persistent grids walking
// work-item lists (descriptor table BInst + items BItem).  Instances are
// grouped by padded rank R (8, 16, 32); each group has its own lists and
// launches.  An instance whose stop test has fired is skipped by every kernel
// (its items return at once), so the batch runs until every member converged.
//
// The per-item arithmetic is the general path's (pass1_strip, pass2_block,
// gram_vv_block, rows_block, make_w_block and the r x r tails), so a batched
// instance computes exactly what a single handle on the general path computes.
//
// Instances with at most 16 slabs of 256 rows run their pass over M on the
// tensor-core kernel instead (k_fused in table mode): one cluster of CS CTAs
// per instance, CS = slabs rounded up to a power of two, instances of one
// (R, CS) launched in waves of as many clusters as fit on the GPU, largest
// first.  The tensor map needs a row stride that is a multiple of 16 bytes, so
// such an instance is stored with m rounded up to a multiple of 4: the added
// rows of M and of U are zero and stay zero (their R, C and P rows vanish), so
// the iterates of the real rows are unchanged.
//
// Autotuner: the tile decisions with a real choice -- the column-split width
// of pass 2 and the persistent grid sizes of both passes -- are timed on the
// batch itself (the passes only write outputs that the next iteration
// rewrites) and the fastest is kept before the graphs are captured.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <string>
#include <vector>

#include "dcf.h"
#include "dcf_handle.h"
#include "dcf_internal.cuh"

using namespace dcf;

namespace dcf {
cudaError_t launch_philox_u0(float* U, int64_t m, int r, int R, uint64_t seed, cudaStream_t s);
}

namespace {

constexpr int kClasses = 3;               // padded rank 8, 16, 32
constexpr int kClassR[kClasses] = {8, 16, 32};
constexpr int kSplitCandidates[] = {256, 512, 1024, 2048};
constexpr int kMinSplit = 256;

int class_of(int r) { return r <= 8 ? 0 : r <= 16 ? 1 : 2; }

struct BatchClass {
  std::vector<int> insts;                 // instance indices of this class
  // device lists
  BItem* mw = nullptr;  int n_mw = 0;     // (inst, 32-row block): rows (every instance)
  BItem* mwg = nullptr; int n_mwg = 0;    // (inst, 32-row block): make_w (general path)
  BItem* fp = nullptr;  int n_fp = 0;     // (inst, slab): U / W images (fused path)
  BItem* fr = nullptr;  int n_fr = 0;     // (inst, block of 256 rows): V_old Z (fused path)
  BItem* p1 = nullptr;  int n_p1 = 0;     // (inst, strip)
  BItem* p2 = nullptr;  int n_p2 = 0;     // (inst, 128-row block, split)
  BItem* gv = nullptr;  int n_gv = 0;     // (inst, Gram chunk of V)
  BItem* gu = nullptr;  int n_gu = 0;     // (inst, Gram chunk of U)
  int* which = nullptr;                   // instance list for the reductions
  int grid_p1 = 0, grid_p2 = 0, split_cols = 1024;
};

// One launch of the fused kernel: a cluster per instance; an argument table
// per copy parity (the tables differ in cur, V_old, V_new and the V max slot).
struct FusedWave {
  int nclusters = 0;
  FusedArgs* table[2] = {nullptr, nullptr};
  int64_t cost = 0;                       // largest instance: strips x cluster size
  int lane = 0;                           // side stream it is launched on
};
struct FusedGroup {
  int R = 0, cs = 0;
  int ncl = 0;                            // clusters of this shape that fit on the GPU
  std::vector<int> insts;                 // largest first
  std::vector<FusedWave> waves;
};
constexpr int kFusedLanes = 16;           // side streams of the fused phase (at most)

constexpr int64_t kFusedMaxM = 4096;      // 16 slabs of 256 rows

}  // namespace

struct dcf_batch_s {
  int count = 0;
  int max_iter = 0;
  double tol = 0;
  uint64_t seed = 0;
  std::vector<BInst> host;                // descriptors (device pointers)
  std::vector<std::vector<int64_t>> n_i;  // column blocks per instance
  std::vector<std::vector<int64_t>> c_i;
  std::vector<char> loaded, have_init;
  BInst* dev = nullptr;                   // descriptor table on the device
  BatchClass cls[kClasses];
  std::vector<int64_t> m_user;            // rows as given (host[q].m may be padded)
  std::vector<FusedGroup> fgroups;
  std::vector<uint8_t*> tmaps;            // device tensor map of each fused instance
  int* kerr = nullptr;                    // fused kernel: a bounded wait expired
  // the waves of the fused phase run on side streams (forked from and joined
  // back to the batch stream): the block scheduler packs their clusters onto
  // the SMs as earlier ones finish, across waves and groups
  cudaEvent_t forked = nullptr;
  std::vector<cudaStream_t> lanes;
  std::vector<cudaEvent_t> joined;
  int nlanes = 0;                         // side streams in use (tuned)
  int wave_div = 1;                       // waves of ncl / wave_div clusters (tuned)
  // allocation
  dcf_alloc_fn alloc = nullptr;
  dcf_free_fn release = nullptr;
  void* alloc_ctx = nullptr;
  std::vector<void*> owned;
  int device = 0, num_sms = 0;
  cudaStream_t user_stream = nullptr, stream = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  bool initialized = false, tuned = false;
  int host_iter = 0;
  cudaGraphExec_t graph[2] = {nullptr, nullptr};
  std::string tune_report;
  std::string err;
};

namespace {

dcf_status bfail(dcf_batch b, dcf_status code, const std::string& msg) {
  if (b) b->err = msg;
  return code;
}

#define BCK(call, what)                                                                  \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess) return bfail(b, DCF_ECUDA, std::string(what) + ": " + cudaGetErrorString(e_)); \
  } while (0)

void* balloc(dcf_batch b, size_t bytes) {
  if (bytes == 0) bytes = 16;
  void* p = nullptr;
  if (b->alloc) {
    p = b->alloc(bytes, b->alloc_ctx);
  } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    p = nullptr;
  }
  if (p) b->owned.push_back(p);
  return p;
}

void bfree_all(dcf_batch b) {
  for (void* p : b->owned) {
    if (b->release) b->release(p, b->alloc_ctx);
    else cudaFree(p);
  }
  b->owned.clear();
}

// Carve a region into 256-byte aligned pieces (a dry run with base = 0 sizes it).
struct Arena {
  char* base = nullptr;
  size_t used = 0;
  template <class T>
  T* take(size_t count) {
    T* p = base ? reinterpret_cast<T*>(base + used) : nullptr;
    used += (count * sizeof(T) + 255) / 256 * 256;
    return p;
  }
};

// Per-instance buffers; the same call sizes (base = 0) and places them.
void layout_instance(Arena& ar, BInst& I) {
  const int64_t m = I.m, n = I.n;
  const int R = I.R;
  const int nsplit_max = (int)((n + kMinSplit - 1) / kMinSplit);
  const int ng = std::max(I.n_gitems, I.n_uitems);
  I.U[0] = ar.take<float>((size_t)m * R);
  I.U[1] = ar.take<float>((size_t)m * R);
  I.V[0] = ar.take<float>((size_t)n * R);
  I.V[1] = ar.take<float>((size_t)n * R);
  I.W = ar.take<float>((size_t)m * R);
  I.part_p = ar.take<float>((size_t)nsplit_max * m * R);
  I.part_h = ar.take<double>((size_t)std::max(I.n_strips, I.nslabs));
  I.part_q = ar.take<float2>((size_t)ng * R * R);
  I.part_xv = ar.take<float2>((size_t)ng * R * R);
  I.part_dv = ar.take<float2>((size_t)ng * R * R);
  I.part_g = ar.take<float2>((size_t)I.n_rblocks * R * R);
  I.part_xu = ar.take<float2>((size_t)I.n_rblocks * R * R);
  I.part_du = ar.take<float2>((size_t)I.n_rblocks * R * R);
  I.red = ar.take<double>((size_t)6 * R * R + 8);
  I.sm = ar.take<Smalls>(1);
  I.st = ar.take<DevState>(1);
  if (I.fused) {
    I.img = ar.take<uint8_t>((size_t)I.nslabs * 2048 * R);
    I.scales = ar.take<float>((size_t)2 * I.nslabs + 1);
    I.zmat = ar.take<float>((size_t)R * R);
    I.VZ = ar.take<float>((size_t)n * R);
    I.vmax = ar.take<unsigned int>(2);
  }
}

template <class T>
T* upload(dcf_batch b, const std::vector<T>& v) {
  T* d = (T*)balloc(b, v.size() * sizeof(T));
  if (d && !v.empty() &&
      cudaMemcpyAsync(d, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, b->stream) !=
          cudaSuccess)
    return nullptr;
  return d;
}

// Pass-2 items of a class for one split width (row blocks of 128, splits of split_cols).
std::vector<BItem> p2_items(dcf_batch b, const BatchClass& c, int split_cols) {
  std::vector<BItem> v;
  for (int q : c.insts) {
    const BInst& I = b->host[q];
    if (I.fused) continue;                 // the fused kernel forms its own P partial
    const int rb = (int)((I.m + 127) / 128);
    const int ns = (int)((I.n + split_cols - 1) / split_cols);
    for (int sp = 0; sp < ns; ++sp)
      for (int r = 0; r < rb; ++r) v.push_back(BItem{q, r, sp, 0});
  }
  return v;
}

void set_split(dcf_batch b, BatchClass& c, int split_cols) {
  c.split_cols = split_cols;
  for (int q : c.insts) {
    BInst& I = b->host[q];
    if (I.fused) continue;                 // one P partial, written by the fused kernel
    I.split_cols = split_cols;
    I.nsplit = (int)((I.n + split_cols - 1) / split_cols);
  }
}

}  // namespace

// ---------------------------------------------------------------------------
// launch sequences
// ---------------------------------------------------------------------------
namespace {

int grid_for(int items, int cap) { return std::max(1, std::min(items, cap)); }

// Phases of one batch iteration (names for dcf_batch_profile_step).
const char* const kBatchPhases[] = {"make_w", "pass1_vstep", "pass2_pstep", "gram_v",
                                    "reduce_q", "rows_ustep", "reduce_g"};
constexpr int kNumBatchPhases = 7;

// The single pass over M of every fused instance: the waves on the side
// streams in use, forked from and joined back to s.
cudaError_t enqueue_fused_phase(dcf_batch b, int cur, cudaStream_t s) {
  cudaError_t e = cudaEventRecord(b->forked, s);
  for (int l = 0; l < b->nlanes; ++l)
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->lanes[l], b->forked, 0);
  for (const FusedGroup& g : b->fgroups)
    for (const FusedWave& wv : g.waves)
      if (e == cudaSuccess)
        e = launch_fused_table(g.R, g.cs, wv.nclusters, wv.table[cur], b->lanes[wv.lane]);
  for (int l = 0; l < b->nlanes; ++l) {
    if (e == cudaSuccess) e = cudaEventRecord(b->joined[l], b->lanes[l]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, b->joined[l], 0);
  }
  return e;
}

// One iteration of every running instance, reading copy `cur`: each phase for
// every rank class, then the next phase.  With ev, ev[p] is recorded after
// phase p (profiling; not captured).
cudaError_t enqueue_batch_iteration(dcf_batch b, int cur, cudaStream_t s,
                                    cudaEvent_t* ev = nullptr) {
  cudaError_t e = cudaSuccess;
  const int S = b->num_sms;
  for (int ph = 0; ph < kNumBatchPhases; ++ph) {
    for (int k = 0; k < kClasses && e == cudaSuccess; ++k) {
      BatchClass& c = b->cls[k];
      if (c.insts.empty()) continue;
      const int R = kClassR[k];
      const int ni = (int)c.insts.size();
      switch (ph) {
        case 0:   // W = U G^{-1} (general); U / W images and V_old Z (fused)
          if (c.n_mwg > 0)
            e = launch_bsmall(R, 0, b->dev, c.mwg, c.n_mwg, nullptr, grid_for(c.n_mwg, 4 * S), cur,
                              1, s);
          if (e == cudaSuccess)
            e = launch_bfused_small(R, 0, b->dev, c.fp, c.n_fp, grid_for(c.n_fp, 4 * S), cur, s);
          if (e == cudaSuccess)
            e = launch_bfused_small(R, 1, b->dev, c.fr, c.n_fr, grid_for(c.n_fr, 8 * S), cur, s);
          break;
        case 1:   // X, V' = X^T W (general; the fused waves follow)
          if (c.n_p1 > 0)
            e = launch_bpass(R, 1, b->dev, c.p1, c.n_p1, c.grid_p1, nullptr, 0, 0, cur, 0, s);
          break;
        case 2:   // P = X V' partials (general)
          if (c.n_p2 > 0)
            e = launch_bpass(R, 2, b->dev, nullptr, 0, 0, c.p2, c.n_p2, c.grid_p2, cur, 0, s);
          break;
        case 3:   // Q = V'^T V', X_v partials
          // one Gram CTA per SM at R >= 32 (its 4 x 4 register tiles), two below
          e = launch_bsmall(R, 2, b->dev, c.gv, c.n_gv, nullptr,
                            grid_for(c.n_gv, (R >= 32 ? 1 : 2) * S), cur, 0, s);
          break;
        case 4:   // (Q + rho I)^{-1}
          e = launch_bsmall(R, 3, b->dev, nullptr, ni, c.which, 0, cur, 1, s);
          break;
        case 5:   // consensus U-step, Gram partials of U_t
          e = launch_bsmall(R, 1, b->dev, c.mw, c.n_mw, nullptr, grid_for(c.n_mw, 4 * S), cur, 0, s);
          break;
        default:  // metrics, stop test, (G + rho I)^{-1}
          e = launch_bsmall(R, 3, b->dev, nullptr, ni, c.which, 0, cur, 2, s);
          break;
      }
    }
    if (ph == 1 && !b->fgroups.empty()) {
      // the single pass over M of every fused instance: waves on the side
      // streams (forked here, joined before the next phase)
      if (e == cudaSuccess) e = enqueue_fused_phase(b, cur, s);
    }
    if (e != cudaSuccess) return e;
    if (ev && (e = cudaEventRecord(ev[ph], s)) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

dcf_status batch_begin(dcf_batch b) {
  BCK(cudaSetDevice(b->device), "set device");
  BCK(cudaEventRecord(b->ev_in, b->user_stream), "record");
  BCK(cudaStreamWaitEvent(b->stream, b->ev_in, 0), "wait");
  return DCF_OK;
}

dcf_status batch_end(dcf_batch b) {
  BCK(cudaEventRecord(b->ev_out, b->stream), "record");
  BCK(cudaStreamWaitEvent(b->user_stream, b->ev_out, 0), "wait");
  return DCF_OK;
}

// Start point of every instance: seeded U0 (unless loaded), G0, the S = 0
// sweep that forms V0 (unless loaded), Q0.
dcf_status batch_init(dcf_batch b) {
  if (b->initialized) return DCF_OK;
  for (int q = 0; q < b->count; ++q)
    if (!b->loaded[q]) return bfail(b, DCF_ESTATE, "instance " + std::to_string(q) + " has no M");
  cudaStream_t s = b->stream;
  for (int q = 0; q < b->count; ++q) {
    BInst& I = b->host[q];
    DevState st0{};
    st0.tol = b->tol;
    BCK(cudaMemcpyAsync(I.st, &st0, sizeof(DevState), cudaMemcpyHostToDevice, s), "init state");
    BCK(cudaMemsetAsync(I.sm, 0, sizeof(Smalls), s), "memset");
    if (!b->have_init[q]) {
      const uint64_t seed = b->seed + 0x9E3779B97F4A7C15ull * (uint64_t)(q + 1);
      // real rows only: padded rows of U stay zero
      BCK(launch_philox_u0(I.U[0], b->m_user[q], I.r, I.R, seed, s), "philox U0");
    }
  }
  const int S = b->num_sms;
  for (int k = 0; k < kClasses; ++k) {
    BatchClass& c = b->cls[k];
    if (c.insts.empty()) continue;
    const int R = kClassR[k];
    BCK(launch_bsmall(R, 2, b->dev, c.gu, c.n_gu, nullptr, grid_for(c.n_gu, 2 * S), 0, 1, s),
        "gram U0");
    BCK(launch_bsmall(R, 3, b->dev, nullptr, (int)c.insts.size(), c.which, 0, 0, 3, s), "G0");
  }
  // V0 = M^T W0 (S = 0) for the instances without a given V0; a loaded V0 is
  // kept: the sweep below writes copy 0 only for instances that need it, so
  // run it on a class list restricted to them.
  for (int k = 0; k < kClasses; ++k) {
    BatchClass& c = b->cls[k];
    if (c.insts.empty()) continue;
    const int R = kClassR[k];
    std::vector<BItem> mw0, p10;
    for (int q : c.insts) {
      if (b->have_init[q] == 2) continue;   // V0 given
      const BInst& I = b->host[q];
      for (int rb = 0; rb < I.n_rblocks; ++rb) mw0.push_back(BItem{q, rb, 0, 0});
      for (int st = 0; st < I.n_strips; ++st) p10.push_back(BItem{q, st, 0, 0});
    }
    if (!mw0.empty()) {
      BItem* dmw = upload(b, mw0);
      BItem* dp1 = upload(b, p10);
      if (!dmw || !dp1) return bfail(b, DCF_ENOMEM, "init lists");
      BCK(launch_bsmall(R, 0, b->dev, dmw, (int)mw0.size(), nullptr,
                        grid_for((int)mw0.size(), 4 * S), 0, 0, s), "W0");
      BCK(launch_bpass(R, 1, b->dev, dp1, (int)p10.size(), grid_for((int)p10.size(), 2 * S),
                       nullptr, 0, 0, 0, 1, s), "V0 sweep");
    }
    BCK(launch_bsmall(R, 2, b->dev, c.gv, c.n_gv, nullptr, grid_for(c.n_gv, 2 * S), 0, 2, s),
        "gram V0");
    BCK(launch_bsmall(R, 3, b->dev, nullptr, (int)c.insts.size(), c.which, 0, 0, 4, s), "Q0");
  }
  // fused instances: max |V0| sets the first V image scale
  for (int q = 0; q < b->count; ++q) {
    const BInst& I = b->host[q];
    if (!I.fused) continue;
    BCK(cudaMemsetAsync(I.vmax, 0, 2 * sizeof(unsigned int), s), "memset");
    BCK(launch_absmax(I.V[0], I.n * I.R, I.vmax, s), "max |V0|");
  }
  b->host_iter = 0;
  b->initialized = true;
  return DCF_OK;
}

// Waves of every fused group: its instances (largest first) in launches of at
// most ncl / div clusters, with an argument table per copy parity.
dcf_status build_waves(dcf_batch b, int div) {
  b->wave_div = div;
  for (FusedGroup& g : b->fgroups) {
    g.waves.clear();
    const int cap = std::max(1, g.ncl / div);
    for (size_t w0 = 0; w0 < g.insts.size(); w0 += (size_t)cap) {
      FusedWave wv;
      wv.nclusters = (int)std::min<size_t>((size_t)cap, g.insts.size() - w0);
      wv.cost = (int64_t)b->host[g.insts[w0]].n_strips * g.cs;
      for (int cur = 0; cur < 2; ++cur) {
        std::vector<FusedArgs> tab(wv.nclusters);
        for (int c = 0; c < wv.nclusters; ++c) {
          const int q = g.insts[w0 + c];
          const BInst& I = b->host[q];
          FusedArgs& f = tab[c];
          f = FusedArgs{};
          f.cur = cur;
          f.cs = g.cs;
          f.nclusters = 1;
          f.nslabs = I.nslabs;
          f.m = I.m;
          f.n = I.n;
          f.lam = I.lam;
          f.Vold = I.V[cur];
          f.Vnew = I.V[cur ^ 1];
          f.img = I.img;
          f.scales = I.scales;
          f.zmat = I.zmat;
          f.VZ = I.VZ;
          f.vmax_out = I.vmax + (cur ^ 1);
          f.part_h = I.part_h;
          f.part_p = I.part_p;
          f.st = I.st;
          f.err = b->kerr;
          f.tmap_g = b->tmaps[q];
        }
        wv.table[cur] = upload(b, tab);
        if (!wv.table[cur]) return bfail(b, DCF_ENOMEM, "wave tables");
      }
      g.waves.push_back(wv);
    }
  }
  return DCF_OK;
}

// The waves dealt, longest first, to the least loaded of `nl` side streams.
void deal_lanes(dcf_batch b, int nl) {
  std::vector<FusedWave*> all;
  for (FusedGroup& g : b->fgroups)
    for (FusedWave& wv : g.waves) all.push_back(&wv);
  std::stable_sort(all.begin(), all.end(),
                   [](const FusedWave* x, const FusedWave* y) { return x->cost > y->cost; });
  nl = std::max(1, std::min(nl, (int)b->lanes.size()));
  b->nlanes = std::min<int>(nl, (int)std::max<size_t>(1, all.size()));
  std::vector<int64_t> load(b->nlanes, 0);
  for (FusedWave* wv : all) {
    const int l = (int)(std::min_element(load.begin(), load.end()) - load.begin());
    wv->lane = l;
    load[l] += wv->cost;
  }
}

// Median device time (ms) of `reps` fused phases on the batch stream, with the
// current waves and lanes, reading copy 0 (the images of copy 0 are prepared).
float time_fused_phase(dcf_batch b, int reps) {
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  std::vector<float> t;
  for (int i = 0; i < reps; ++i) {
    cudaEventRecord(e0, b->stream);
    enqueue_fused_phase(b, 0, b->stream);
    cudaEventRecord(e1, b->stream);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    t.push_back(ms);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  std::sort(t.begin(), t.end());
  return t[t.size() / 2];
}

// Time `reps` launches of one pass of one class (median, ms).
float time_pass(dcf_batch b, int k, int which, int reps) {
  BatchClass& c = b->cls[k];
  const int R = kClassR[k];
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  std::vector<float> t;
  for (int i = 0; i < reps; ++i) {
    cudaEventRecord(e0, b->stream);
    launch_bpass(R, which, b->dev, c.p1, c.n_p1, c.grid_p1, c.p2, c.n_p2, c.grid_p2, 0, 0,
                 b->stream);
    cudaEventRecord(e1, b->stream);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    t.push_back(ms);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  std::sort(t.begin(), t.end());
  return t[t.size() / 2];
}

// Autotuner: per rank class, the pass-1 grid and the pass-2 (split width, grid)
// with the smallest median time; the state is at copy 0 with W valid.
dcf_status batch_tune(dcf_batch b, int reps) {
  const int S = b->num_sms;
  char line[256];
  b->tune_report.clear();
  BCK(cudaStreamSynchronize(b->stream), "sync");
  for (int k = 0; k < kClasses; ++k) {
    BatchClass& c = b->cls[k];
    if (c.insts.empty() || c.n_p1 == 0) continue;   // only general instances have passes
    // W for copy 0 (the passes read it)
    BCK(launch_bsmall(kClassR[k], 0, b->dev, c.mwg, c.n_mwg, nullptr, grid_for(c.n_mwg, 4 * S),
                      0, 0, b->stream), "tune W");
    float best1 = 1e30f;
    int g1best = c.grid_p1;
    for (int mult : {1, 2, 3, 4}) {
      c.grid_p1 = grid_for(c.n_p1, mult * S);
      time_pass(b, k, 1, 1);
      const float t = time_pass(b, k, 1, reps);
      snprintf(line, sizeof(line), "R=%d pass1 grid=%d: %.4f ms\n", kClassR[k], c.grid_p1, t);
      b->tune_report += line;
      if (t < best1) { best1 = t; g1best = c.grid_p1; }
    }
    c.grid_p1 = g1best;
    float best2 = 1e30f;
    int sbest = c.split_cols, g2best = c.grid_p2;
    for (int split : kSplitCandidates) {
      set_split(b, c, split);
      std::vector<BItem> v = p2_items(b, c, split);
      BItem* d = upload(b, v);
      if (!d) return bfail(b, DCF_ENOMEM, "tune lists");
      c.p2 = d;
      c.n_p2 = (int)v.size();
      BCK(cudaMemcpyAsync(b->dev, b->host.data(), b->host.size() * sizeof(BInst),
                          cudaMemcpyHostToDevice, b->stream), "descriptors");
      for (int mult : {2, 4, 8}) {
        c.grid_p2 = grid_for(c.n_p2, mult * S);
        time_pass(b, k, 2, 1);
        const float t = time_pass(b, k, 2, reps);
        snprintf(line, sizeof(line), "R=%d pass2 split=%d grid=%d: %.4f ms\n", kClassR[k], split,
                 c.grid_p2, t);
        b->tune_report += line;
        if (t < best2) { best2 = t; sbest = split; g2best = c.grid_p2; }
      }
    }
    set_split(b, c, sbest);
    std::vector<BItem> v = p2_items(b, c, sbest);
    c.p2 = upload(b, v);
    c.n_p2 = (int)v.size();
    c.grid_p2 = g2best;
    if (!c.p2) return bfail(b, DCF_ENOMEM, "tune lists");
    snprintf(line, sizeof(line), "R=%d chosen: pass1 grid=%d, pass2 split=%d grid=%d\n",
             kClassR[k], c.grid_p1, sbest, g2best);
    b->tune_report += line;
  }
  if (!b->fgroups.empty()) {
    // the tensor-core pass of the fused instances: wave size (ncl / div
    // clusters per launch) and side streams, timed as a whole phase on the
    // batch itself (the images and V_old Z of copy 0 prepared first)
    for (int k = 0; k < kClasses; ++k) {
      BatchClass& c = b->cls[k];
      if (c.insts.empty()) continue;
      BCK(launch_bfused_small(kClassR[k], 0, b->dev, c.fp, c.n_fp, grid_for(c.n_fp, 4 * S), 0,
                              b->stream), "tune images");
      BCK(launch_bfused_small(kClassR[k], 1, b->dev, c.fr, c.n_fr, grid_for(c.n_fr, 8 * S), 0,
                              b->stream), "tune V_old Z");
    }
    float best = 1e30f;
    int bdiv = 1, blanes = (int)b->lanes.size();
    for (int div : {1, 2}) {
      dcf_status st = build_waves(b, div);
      if (st != DCF_OK) return st;
      for (int nl : {1, 2, 4, 8, 16}) {
        if (nl > (int)b->lanes.size()) continue;
        deal_lanes(b, nl);
        time_fused_phase(b, 1);
        const float t = time_fused_phase(b, reps);
        BCK(cudaGetLastError(), "tune fused phase");
        int nw = 0;
        for (const FusedGroup& g : b->fgroups) nw += (int)g.waves.size();
        snprintf(line, sizeof(line),
                 "tensor-core pass: waves of ncl/%d clusters (%d waves), %d side streams: "
                 "%.4f ms\n", div, nw, b->nlanes, t);
        b->tune_report += line;
        if (t < best) { best = t; bdiv = div; blanes = nl; }
      }
    }
    dcf_status st = build_waves(b, bdiv);
    if (st != DCF_OK) return st;
    deal_lanes(b, blanes);
    for (const FusedGroup& g : b->fgroups) {
      snprintf(line, sizeof(line),
               "R=%d cs=%d chosen: tensor-core kernel, %d instances in %d waves of up to %d "
               "clusters on %d side streams (%.4f ms for the whole pass)\n",
               g.R, g.cs, (int)g.insts.size(), (int)g.waves.size(),
               g.waves.empty() ? 0 : g.waves[0].nclusters, b->nlanes, best);
      b->tune_report += line;
    }
    // the timed phases wrote copy 1 and its max |V|: the first step rewrites them
  }
  BCK(cudaMemcpyAsync(b->dev, b->host.data(), b->host.size() * sizeof(BInst),
                      cudaMemcpyHostToDevice, b->stream), "descriptors");
  BCK(cudaStreamSynchronize(b->stream), "sync");
  b->tuned = true;
  return DCF_OK;
}

dcf_status build_batch_graphs(dcf_batch b) {
  for (int p = 0; p < 2; ++p) {
    if (b->graph[p]) continue;
    cudaGraph_t g = nullptr;
    BCK(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal), "begin capture");
    cudaError_t e = enqueue_batch_iteration(b, p, b->stream);
    cudaError_t e2 = cudaStreamEndCapture(b->stream, &g);
    if (e != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      return bfail(b, DCF_ECUDA, std::string("capture: ") + cudaGetErrorString(e));
    }
    BCK(e2, "end capture");
    cudaError_t e3 = cudaGraphInstantiate(&b->graph[p], g, 0);
    cudaGraphDestroy(g);
    BCK(e3, "instantiate");
  }
  return DCF_OK;
}

dcf_status batch_ready(dcf_batch b) {
  dcf_status st = batch_init(b);
  if (st != DCF_OK) return st;
  if (!b->tuned) {
    if ((st = batch_tune(b, 3)) != DCF_OK) return st;
  }
  return build_batch_graphs(b);
}

dcf_status read_states(dcf_batch b, std::vector<DevState>& out) {
  out.resize(b->count);
  int kerr = 0;
  for (int q = 0; q < b->count; ++q)
    BCK(cudaMemcpyAsync(&out[q], b->host[q].st, sizeof(DevState), cudaMemcpyDeviceToHost,
                        b->stream), "read state");
  BCK(cudaMemcpyAsync(&kerr, b->kerr, sizeof(int), cudaMemcpyDeviceToHost, b->stream), "err");
  BCK(cudaStreamSynchronize(b->stream), "sync");
  if (kerr == DCF_ETIMEOUT)
    return bfail(b, DCF_ETIMEOUT, "a bounded device-side wait expired in the fused kernel");
  for (int q = 0; q < b->count; ++q)
    if (out[q].status == DCF_ENONFINITE)
      return bfail(b, DCF_ENONFINITE, "non-finite iterates in instance " + std::to_string(q));
  return DCF_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// entry points
// ---------------------------------------------------------------------------
extern "C" dcf_status dcf_batch_create(const dcf_problem* problems, int count, int max_iter,
                                       double tol, uint64_t seed, dcf_batch* out) {
  if (!out) return DCF_EINVAL;
  *out = nullptr;
  if (!problems || count < 1 || max_iter < 0 || !(tol >= 0)) return DCF_EINVAL;
  for (int q = 0; q < count; ++q) {
    const dcf_problem& p = problems[q];
    if (p.m < 1 || p.E < 1 || !p.n_i || p.r < 1 || p.r > 32 || p.r > p.m) return DCF_EINVAL;
    if (!(p.rho > 0) || !(p.lambda > 0)) return DCF_EINVAL;
    int64_t n = 0;
    for (int i = 0; i < p.E; ++i) {
      if (p.n_i[i] < 1) return DCF_EINVAL;
      n += p.n_i[i];
    }
    if (n < 1) return DCF_EINVAL;
  }
  dcf_batch b = new dcf_batch_s();
  b->count = count;
  b->max_iter = max_iter;
  b->tol = tol;
  b->seed = seed;
  dcf::api::current_allocator(&b->alloc, &b->release, &b->alloc_ctx);
  if (cudaGetDevice(&b->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, b->device) !=
          cudaSuccess ||
      cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming) != cudaSuccess ||
      prepare_stream_kernels() != cudaSuccess || prepare_small_kernels() != cudaSuccess ||
      prepare_batch_stream_kernels() != cudaSuccess || fused_prepare(16) != cudaSuccess ||
      fused_prepare(32) != cudaSuccess) {
    cudaGetLastError();
    dcf_batch_destroy(b);
    return DCF_ECUDA;
  }
  b->m_user.resize(count);
  b->host.resize(count);
  b->n_i.resize(count);
  b->c_i.resize(count);
  b->loaded.assign(count, 0);
  b->have_init.assign(count, 0);
  // descriptors (sizes first), then one arena for all per-instance buffers
  for (int q = 0; q < count; ++q) {
    const dcf_problem& p = problems[q];
    BInst& I = b->host[q];
    I = BInst{};
    b->m_user[q] = p.m;
    // the tensor-core path: at most 16 slabs of 256 rows, padded rank 16 or 32,
    // a cluster shape that fits on this GPU; M stored with m rounded up to 4
    const int64_t m_pad = (p.m + 3) / 4 * 4;
    const int Rf = p.r <= 16 ? 16 : 32;
    int cs = 1;
    while ((int64_t)cs * 256 < m_pad) cs *= 2;
    I.fused = (m_pad <= kFusedMaxM && fused_max_clusters(Rf, cs) > 0) ? 1 : 0;
    cudaGetLastError();
    I.m = I.fused ? m_pad : p.m;
    I.nslabs = I.fused ? cs : 1;
    I.E = p.E;
    I.r = p.r;
    I.R = I.fused ? Rf : pick_R(p.r);
    I.lam = (float)p.lambda;
    I.rho = (float)p.rho;
    I.u_mode = 0;
    b->n_i[q].assign(p.n_i, p.n_i + p.E);
    b->c_i[q].resize(p.E);
    int64_t n = 0;
    for (int i = 0; i < p.E; ++i) {
      b->c_i[q][i] = n;
      n += p.n_i[i];
    }
    I.n = n;
    I.n_strips = (int)((n + 63) / 64);
    I.n_rblocks = (int)((I.m + 31) / 32);
    I.n_gitems = (int)((n + kBGramRows - 1) / kBGramRows);
    I.n_uitems = (int)((I.m + kBGramRows - 1) / kBGramRows);
    I.split_cols = 1024;
    I.nsplit = I.fused ? 1 : (int)((n + 1023) / 1024);
    I.n_hparts = I.fused ? I.nslabs : I.n_strips;
  }
  size_t mbytes = 0, wbytes = 0;
  for (int q = 0; q < count; ++q) {
    mbytes += ((size_t)b->host[q].m * b->host[q].n * 4 + 255) / 256 * 256;   // padded m
    Arena dry;
    layout_instance(dry, b->host[q]);
    if (b->host[q].fused) dry.take<uint8_t>(128);   // its tensor map
    wbytes += dry.used;
  }
  char* mbase = (char*)balloc(b, mbytes);
  char* wbase = (char*)balloc(b, wbytes);
  if (!mbase || !wbase) {
    dcf_batch_destroy(b);
    return DCF_ENOMEM;
  }
  {
    Arena am{mbase, 0}, aw{wbase, 0};
    b->tmaps.assign(count, nullptr);
    for (int q = 0; q < count; ++q) {
      BInst& I = b->host[q];
      I.M = am.take<float>((size_t)I.m * I.n);
      layout_instance(aw, I);
      if (I.fused) b->tmaps[q] = aw.take<uint8_t>(128);   // 256-byte aligned
    }
  }
  // zero everything: padded rows of M and U stay zero
  if (cudaMemsetAsync(wbase, 0, wbytes, b->stream) != cudaSuccess ||
      cudaMemsetAsync(mbase, 0, mbytes, b->stream) != cudaSuccess) {
    cudaGetLastError();
    dcf_batch_destroy(b);
    return DCF_ECUDA;
  }
  // classes and their work lists
  // rank classes by the padded rank an instance runs with (R = 8 only on the
  // general path)
  for (int q = 0; q < count; ++q) b->cls[class_of(b->host[q].R)].insts.push_back(q);
  for (int k = 0; k < kClasses; ++k) {
    BatchClass& c = b->cls[k];
    if (c.insts.empty()) continue;
    std::vector<BItem> mw, mwg, p1, gv, gu, fp, fr;
    for (int q : c.insts) {
      const BInst& I = b->host[q];
      for (int rb = 0; rb < I.n_rblocks; ++rb) mw.push_back(BItem{q, rb, 0, 0});
      for (int g = 0; g < I.n_gitems; ++g) gv.push_back(BItem{q, g, 0, 0});
      for (int g = 0; g < I.n_uitems; ++g) gu.push_back(BItem{q, g, 0, 0});
      if (I.fused) {
        for (int sl = 0; sl < I.nslabs; ++sl) fp.push_back(BItem{q, sl, 0, 0});
        const int64_t blocks = (I.n + 255) / 256;   // V_old Z: 256 rows per item
        for (int64_t bk = 0; bk < blocks; ++bk) fr.push_back(BItem{q, (int)bk, 0, 0});
      } else {
        for (int rb = 0; rb < I.n_rblocks; ++rb) mwg.push_back(BItem{q, rb, 0, 0});
        for (int s = 0; s < I.n_strips; ++s) p1.push_back(BItem{q, s, 0, 0});
      }
    }
    set_split(b, c, 1024);
    std::vector<BItem> p2 = p2_items(b, c, 1024);
    c.mw = upload(b, mw);  c.n_mw = (int)mw.size();
    c.mwg = upload(b, mwg);  c.n_mwg = (int)mwg.size();
    c.fp = upload(b, fp);  c.n_fp = (int)fp.size();
    c.fr = upload(b, fr);  c.n_fr = (int)fr.size();
    c.p1 = upload(b, p1);  c.n_p1 = (int)p1.size();
    c.p2 = upload(b, p2);  c.n_p2 = (int)p2.size();
    c.gv = upload(b, gv);  c.n_gv = (int)gv.size();
    c.gu = upload(b, gu);  c.n_gu = (int)gu.size();
    c.which = upload(b, c.insts);
    c.grid_p1 = grid_for(c.n_p1, 2 * b->num_sms);
    c.grid_p2 = grid_for(c.n_p2, 4 * b->num_sms);
    if (!c.mw || !c.mwg || !c.fp || !c.fr || !c.p1 || !c.p2 || !c.gv || !c.gu || !c.which) {
      dcf_batch_destroy(b);
      return DCF_ENOMEM;
    }
  }
  b->kerr = (int*)balloc(b, sizeof(int));
  if (!b->kerr || cudaMemsetAsync(b->kerr, 0, sizeof(int), b->stream) != cudaSuccess) {
    cudaGetLastError();
    dcf_batch_destroy(b);
    return DCF_ENOMEM;
  }
  // fused groups by (R, cluster size): tensor maps, waves, argument tables
  for (int q = 0; q < count; ++q) {
    const BInst& I = b->host[q];
    if (!I.fused) continue;
    alignas(64) unsigned char tm[128];
    if (fused_make_tmap(tm, I.M, I.m, I.n) != 0 ||
        cudaMemcpyAsync(b->tmaps[q], tm, 128, cudaMemcpyHostToDevice, b->stream) != cudaSuccess ||
        cudaStreamSynchronize(b->stream) != cudaSuccess) {   // the host copy goes out of scope
      cudaGetLastError();
      dcf_batch_destroy(b);
      return DCF_ECUDA;
    }
    size_t gi = 0;
    while (gi < b->fgroups.size() && !(b->fgroups[gi].R == I.R && b->fgroups[gi].cs == I.nslabs))
      ++gi;
    if (gi == b->fgroups.size()) {
      FusedGroup g;
      g.R = I.R;
      g.cs = I.nslabs;
      b->fgroups.push_back(g);
    }
    b->fgroups[gi].insts.push_back(q);
  }
  for (FusedGroup& g : b->fgroups) {
    std::stable_sort(g.insts.begin(), g.insts.end(), [&](int x, int y) {
      return b->host[x].n_strips > b->host[y].n_strips;
    });
    g.ncl = fused_max_clusters(g.R, g.cs);
  }
  if (build_waves(b, 1) != DCF_OK) {
    dcf_batch_destroy(b);
    return DCF_ENOMEM;
  }
  // side streams (the tuner picks how many are used; 8 until then)
  {
    int nw = 0;
    for (const FusedGroup& g : b->fgroups) nw += (int)g.waves.size();
    bool ok = nw > 0 ? cudaEventCreateWithFlags(&b->forked, cudaEventDisableTiming) == cudaSuccess
                     : true;
    const int nl = nw > 0 ? kFusedLanes : 0;
    b->lanes.assign(nl, nullptr);
    b->joined.assign(nl, nullptr);
    for (int l = 0; l < nl && ok; ++l)
      ok = cudaStreamCreateWithFlags(&b->lanes[l], cudaStreamNonBlocking) == cudaSuccess &&
           cudaEventCreateWithFlags(&b->joined[l], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
      cudaGetLastError();
      dcf_batch_destroy(b);
      return DCF_ECUDA;
    }
    if (nl > 0) deal_lanes(b, 8);
  }
  b->dev = upload(b, b->host);
  if (!b->dev || cudaStreamSynchronize(b->stream) != cudaSuccess) {
    cudaGetLastError();
    dcf_batch_destroy(b);
    return DCF_ENOMEM;
  }
  *out = b;
  return DCF_OK;
}

extern "C" dcf_status dcf_batch_set_stream(dcf_batch b, void* stream) {
  if (!b) return DCF_EINVAL;
  b->user_stream = (cudaStream_t)stream;
  return DCF_OK;
}

extern "C" dcf_status dcf_batch_load(dcf_batch b, int i, const float* const* M_i,
                                     const int64_t* ld_i, int where) {
  if (!b) return DCF_EINVAL;
  if (i < 0 || i >= b->count) return bfail(b, DCF_EINVAL, "instance index out of range");
  if (!M_i || (where != 0 && where != 1)) return bfail(b, DCF_EINVAL, "blocks or where");
  const BInst& I = b->host[i];
  const int64_t mu = b->m_user[i];
  for (int k = 0; k < I.E; ++k) {
    if (!M_i[k]) return bfail(b, DCF_EINVAL, "NULL block");
    if (ld_i && ld_i[k] < mu) return bfail(b, DCF_EINVAL, "leading dimension < m");
  }
  dcf_status st = batch_begin(b);
  if (st != DCF_OK) return st;
  const cudaMemcpyKind kind = where == 0 ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  for (int k = 0; k < I.E; ++k) {
    const int64_t ld = ld_i ? ld_i[k] : mu;
    float* dst = const_cast<float*>(I.M) + b->c_i[i][k] * I.m;   // padded pitch I.m >= mu
    BCK(cudaMemcpy2DAsync(dst, (size_t)I.m * 4, M_i[k], (size_t)ld * 4, (size_t)mu * 4,
                          (size_t)b->n_i[i][k], kind, b->stream), "copy M");
  }
  if (where == 0) BCK(cudaStreamSynchronize(b->stream), "sync");
  b->loaded[i] = 1;
  return batch_end(b);
}

extern "C" dcf_status dcf_batch_load_init(dcf_batch b, int i, const float* U0,
                                          const float* const* V0_i, int where) {
  if (!b) return DCF_EINVAL;
  if (i < 0 || i >= b->count) return bfail(b, DCF_EINVAL, "instance index out of range");
  if (!U0 || (where != 0 && where != 1)) return bfail(b, DCF_EINVAL, "U0 or where");
  if (b->initialized) return bfail(b, DCF_ESTATE, "the batch has started");
  const BInst& I = b->host[i];
  dcf_status st = batch_begin(b);
  if (st != DCF_OK) return st;
  const cudaMemcpyKind kind = where == 0 ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  BCK(cudaMemcpy2DAsync(I.U[0], (size_t)I.R * 4, U0, (size_t)I.r * 4, (size_t)I.r * 4,
                        (size_t)b->m_user[i], kind, b->stream), "copy U0");
  b->have_init[i] = 1;
  if (V0_i) {
    for (int k = 0; k < I.E; ++k) {
      if (!V0_i[k]) return bfail(b, DCF_EINVAL, "NULL V0 block");
      BCK(cudaMemcpy2DAsync(I.V[0] + b->c_i[i][k] * I.R, (size_t)I.R * 4, V0_i[k],
                            (size_t)I.r * 4, (size_t)I.r * 4, (size_t)b->n_i[i][k], kind,
                            b->stream), "copy V0");
    }
    b->have_init[i] = 2;
  }
  if (where == 0) BCK(cudaStreamSynchronize(b->stream), "sync");
  return batch_end(b);
}

extern "C" dcf_status dcf_batch_tune(dcf_batch b, int reps, char* report, int report_len) {
  if (!b) return DCF_EINVAL;
  if (reps < 1) return bfail(b, DCF_EINVAL, "reps < 1");
  dcf_status st = batch_begin(b);
  if (st != DCF_OK) return st;
  if ((st = batch_init(b)) != DCF_OK) return st;
  if (b->host_iter != 0) return bfail(b, DCF_ESTATE, "tune before the first step");
  if ((st = batch_tune(b, reps)) != DCF_OK) return st;
  for (int p = 0; p < 2; ++p) {
    if (b->graph[p]) cudaGraphExecDestroy(b->graph[p]);
    b->graph[p] = nullptr;
  }
  if (report && report_len > 0) {
    snprintf(report, (size_t)report_len, "%s", b->tune_report.c_str());
  }
  return batch_end(b);
}

extern "C" dcf_status dcf_batch_step(dcf_batch b, int n_steps) {
  if (!b) return DCF_EINVAL;
  if (n_steps < 0) return bfail(b, DCF_EINVAL, "n_steps < 0");
  dcf_status st = batch_begin(b);
  if (st != DCF_OK) return st;
  if ((st = batch_ready(b)) != DCF_OK) return st;
  for (int i = 0; i < n_steps; ++i) {
    BCK(cudaGraphLaunch(b->graph[b->host_iter & 1], b->stream), "graph launch");
    b->host_iter++;
  }
  return batch_end(b);
}

extern "C" dcf_status dcf_batch_solve(dcf_batch b, int* iters_out, int* n_converged) {
  if (!b) return DCF_EINVAL;
  dcf_status st = batch_begin(b);
  if (st != DCF_OK) return st;
  if ((st = batch_ready(b)) != DCF_OK) return st;
  // solve mode on, stop flags cleared
  for (int q = 0; q < b->count; ++q) {
    const int one = 1, zero = 0;
    DevState* d = b->host[q].st;
    BCK(cudaMemcpyAsync(&d->solve_mode, &one, sizeof(int), cudaMemcpyHostToDevice, b->stream), "w");
    BCK(cudaMemcpyAsync(&d->tol, &b->tol, sizeof(double), cudaMemcpyHostToDevice, b->stream), "w");
    BCK(cudaMemcpyAsync(&d->stop, &zero, sizeof(int), cudaMemcpyHostToDevice, b->stream), "w");
  }
  std::vector<DevState> ds;
  if ((st = read_states(b, ds)) != DCF_OK) return st;
  std::vector<int> start(b->count);
  for (int q = 0; q < b->count; ++q) start[q] = ds[q].iter;
  int done = 0, conv = 0;
  while (done < b->max_iter) {
    const int nb = std::min(8, b->max_iter - done);
    for (int i = 0; i < nb; ++i) {
      BCK(cudaGraphLaunch(b->graph[b->host_iter & 1], b->stream), "graph launch");
      b->host_iter++;
    }
    done += nb;
    if ((st = read_states(b, ds)) != DCF_OK) return st;
    conv = 0;
    for (int q = 0; q < b->count; ++q) conv += ds[q].stop ? 1 : 0;
    if (conv == b->count) break;
  }
  if (iters_out)
    for (int q = 0; q < b->count; ++q) iters_out[q] = ds[q].iter - start[q];
  if (n_converged) *n_converged = conv;
  for (int q = 0; q < b->count; ++q) {
    const int zero = 0;
    BCK(cudaMemcpyAsync(&b->host[q].st->solve_mode, &zero, sizeof(int), cudaMemcpyHostToDevice,
                        b->stream), "w");
  }
  if ((st = batch_end(b)) != DCF_OK) return st;
  return conv == b->count ? DCF_OK : DCF_ENOTCONV;
}

extern "C" dcf_status dcf_batch_get_factors(dcf_batch b, int i, float* U, float* const* V_i,
                                            int where) {
  if (!b) return DCF_EINVAL;
  if (i < 0 || i >= b->count) return bfail(b, DCF_EINVAL, "instance index out of range");
  if (where != 0 && where != 1) return bfail(b, DCF_EINVAL, "where must be 0 or 1");
  dcf_status st = batch_begin(b);
  if (st != DCF_OK) return st;
  if ((st = batch_init(b)) != DCF_OK) return st;
  const BInst& I = b->host[i];
  DevState ds{};
  BCK(cudaMemcpyAsync(&ds, I.st, sizeof(DevState), cudaMemcpyDeviceToHost, b->stream), "state");
  BCK(cudaStreamSynchronize(b->stream), "sync");
  const int cur = ds.iter & 1;   // a stopped instance keeps the copy it stopped in
  const cudaMemcpyKind kind = where == 0 ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  if (U)
    BCK(cudaMemcpy2DAsync(U, (size_t)I.r * 4, I.U[cur], (size_t)I.R * 4, (size_t)I.r * 4,
                          (size_t)b->m_user[i], kind, b->stream), "copy U");
  if (V_i) {
    for (int k = 0; k < I.E; ++k) {
      if (!V_i[k]) continue;
      BCK(cudaMemcpy2DAsync(V_i[k], (size_t)I.r * 4, I.V[cur] + b->c_i[i][k] * I.R,
                            (size_t)I.R * 4, (size_t)I.r * 4, (size_t)b->n_i[i][k], kind,
                            b->stream), "copy V");
    }
  }
  if (where == 0) BCK(cudaStreamSynchronize(b->stream), "sync");
  return batch_end(b);
}

extern "C" dcf_status dcf_batch_get_stats(dcf_batch b, int i, double* objective, double* dL_rel,
                                          int* iter) {
  if (!b) return DCF_EINVAL;
  if (i < 0 || i >= b->count) return bfail(b, DCF_EINVAL, "instance index out of range");
  dcf_status st = batch_begin(b);
  if (st != DCF_OK) return st;
  if ((st = batch_init(b)) != DCF_OK) return st;
  DevState ds{};
  int kerr = 0;
  BCK(cudaMemcpyAsync(&ds, b->host[i].st, sizeof(DevState), cudaMemcpyDeviceToHost, b->stream),
      "state");
  BCK(cudaMemcpyAsync(&kerr, b->kerr, sizeof(int), cudaMemcpyDeviceToHost, b->stream), "err");
  BCK(cudaStreamSynchronize(b->stream), "sync");
  if (kerr == DCF_ETIMEOUT)
    return bfail(b, DCF_ETIMEOUT, "a bounded device-side wait expired in the fused kernel");
  if (ds.status == DCF_ENONFINITE) return bfail(b, DCF_ENONFINITE, "non-finite iterates");
  if (objective) *objective = ds.objective;
  if (dL_rel) *dL_rel = ds.dL_rel;
  if (iter) *iter = ds.iter;
  return batch_end(b);
}

extern "C" const char* dcf_batch_last_error(dcf_batch b) {
  return b ? b->err.c_str() : "NULL batch";
}

extern "C" void dcf_batch_destroy(dcf_batch b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  for (int p = 0; p < 2; ++p)
    if (b->graph[p]) cudaGraphExecDestroy(b->graph[p]);
  for (size_t l = 0; l < b->lanes.size(); ++l) {
    if (b->lanes[l]) {
      cudaStreamSynchronize(b->lanes[l]);
      cudaStreamDestroy(b->lanes[l]);
    }
    if (b->joined[l]) cudaEventDestroy(b->joined[l]);
  }
  if (b->forked) cudaEventDestroy(b->forked);
  bfree_all(b);
  if (b->ev_in) cudaEventDestroy(b->ev_in);
  if (b->ev_out) cudaEventDestroy(b->ev_out);
  if (b->stream) cudaStreamDestroy(b->stream);
  delete b;
}

extern "C" dcf_status dcf_batch_profile_step(dcf_batch b, int n_steps, double* phase_ms,
                                             int n_phases) {
  if (!b) return DCF_EINVAL;
  if (n_steps < 1 || !phase_ms || n_phases < kNumBatchPhases)
    return bfail(b, DCF_EINVAL, "n_steps < 1 or phase_ms too short");
  dcf_status st = batch_begin(b);
  if (st != DCF_OK) return st;
  if ((st = batch_ready(b)) != DCF_OK) return st;
  cudaEvent_t ev[kNumBatchPhases + 1];
  for (auto& x : ev) BCK(cudaEventCreate(&x), "event");
  for (int p = 0; p < kNumBatchPhases; ++p) phase_ms[p] = 0.0;
  for (int i = 0; i < n_steps; ++i) {
    BCK(cudaEventRecord(ev[kNumBatchPhases], b->stream), "record");
    BCK(enqueue_batch_iteration(b, b->host_iter & 1, b->stream, ev), "profiled iteration");
    b->host_iter++;
    BCK(cudaEventSynchronize(ev[kNumBatchPhases - 1]), "sync");
    float prev = 0.f;
    for (int p = 0; p < kNumBatchPhases; ++p) {
      float ms = 0.f;
      BCK(cudaEventElapsedTime(&ms, ev[kNumBatchPhases], ev[p]), "elapsed");
      phase_ms[p] += ms - prev;
      prev = ms;
    }
  }
  for (auto& x : ev) cudaEventDestroy(x);
  return batch_end(b);
}
