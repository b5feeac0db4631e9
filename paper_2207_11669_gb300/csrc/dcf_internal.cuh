// Internal declarations shared by the DCF-PCA CUDA translation units.
//
// Storage (device):
//   M      m x n float, column-major (ld = m); block i = columns [c_i, c_i + n_i)
//   U[2]   m x R float, row-major (ld = R); R = padded rank (8, 16, 32 or 64),
//          columns r..R-1 are zero and stay zero (the r x r solves are
//          block diagonal in the padding)
//   V[2]   n x R float, row-major
// Two copies of U and V alternate: iteration t reads copy (t-1) & 1 and writes
// copy t & 1, so two captured CUDA graphs (one per parity) serve every
// iteration and U_{t-1}, V_{t-1} stay available for the S output.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace dcf {

constexpr int kMaxR = 64;

// Device-side state of one problem (one instance).
struct DevState {
  int iter;          // completed iterations t
  int stop;          // set by the finish kernel when dL_rel <= tol (solve mode)
  int status;        // 0 ok; DCF_ENONFINITE when the iterates stop being finite
  int solve_mode;    // 1: the finish kernel may set `stop`
  int has_S;         // 1 once an iteration has run (S of the last round exists)
  int pad_;
  double tol;
  double eta0;       // FedAvg learning rate base
  double objective;  // objective at (U_{t-1}, V_{t-1}, S_t)
  double dL_rel;     // ||L_t - L_{t-1}||_F / ||L_t||_F
  double huber;      // sum H_lambda(R) of the last pass
  double eta_fixed;  // FedAvg step size when > 0 (a client's local steps all use the
                     // step size of their communication round); 0: eta0 / sqrt(t + 1)
  double kappa_g;    // 1-norm condition estimate of the latest U^T U + rho I
  double kappa_h;    //   and of the latest V^T V + rho I (exact U-step)
  int route_g;       // how their inverses were formed: 0 FP32 from the double-float
  int route_h;       //   factors, 1 double-float
};

// Condition estimate above which the r x r inverses are formed in double-float
// and the steps that apply them, or that feed them with cancelling sums (W,
// V_{t-1}^T V_t applied to U_{t-1}, the Grams of V), use compensated products.
// Below it the FP32 rounding errors, amplified by at most kappa, stay under
// about 1e-5 relative.
constexpr double kDfKappa = 100.0;

__device__ __forceinline__ bool df_route(const DevState* st) {
  return st->kappa_g > kDfKappa || st->kappa_h > kDfKappa;
}

// r x r FP64 workspace of one problem.
struct Smalls {
  double gram[2][kMaxR * kMaxR];   // U^T U for copy 0/1 of U
  double q[2][kMaxR * kMaxR];      // V^T V for copy 0/1 of V
  double xu[kMaxR * kMaxR];        // U_{t-1}^T (U_t - U_{t-1})
  double xv[kMaxR * kMaxR];        // V_{t-1}^T V_t
  float xv32[2][kMaxR * kMaxR];    // V_{t-1}^T V_t as the float pair hi, lo
  double dvy[kMaxR * kMaxR];       // V_{t-1}^T (V_t - V_{t-1})
  double dvv[kMaxR * kMaxR];       // (V_t - V_{t-1})^T (V_t - V_{t-1})
  float ginv32[kMaxR * kMaxR];     // (U^T U + rho I)^{-1} of the current U (hi part)
  float ginv32_lo[kMaxR * kMaxR];  //   and its lo part (the inverse is hi + lo)
  float hinv32[kMaxR * kMaxR];     // (V^T V + rho I)^{-1} of the new V (exact mode)
  float qrho32[kMaxR * kMaxR];     // (V^T V + rho I) in float (FedAvg mode)
};

struct IterArgs {
  int cur;           // copy holding U_{t-1}, V_{t-1}; the iteration writes cur ^ 1
  const float* M;
  int64_t m, n;
  int r, R;
  float lam;
  float rho;
  float rho_q;       // rho of the U-step's Q + rho I when > 0 (a client's local step:
                     // its share rho n_i / n of the ridge term); 0: rho
  int u_mode;        // 0 exact, 1 FedAvg
  int E;
  float* U[2];
  float* V[2];
  float* W;          // m x R
  // partial results of the streaming passes
  float2* part_q;    // [n_vblocks][R*R]   V'^T V'      (compensated pairs hi, lo)
  float2* part_xv;   // [n_vblocks][R*R]   V_old^T (V' - V_old)
  float2* part_dv;   // [n_vblocks][R*R]   (V' - V_old)^T (V' - V_old)
  double* part_h;    // [n_vblocks]        Huber partial
  float* part_p;     // [n_splits][m*R]    P partials (X V')
  int n_vblocks;
  int n_splits;
  int64_t split_cols;
  float2* part_g;    // [n_rblocks][R*R]   U_new^T U_new partials (hi, lo)
  float2* part_xu;   // [n_rblocks][R*R]   U_old^T (U_new - U_old) partials (hi, lo)
  float2* part_du;   // [n_rblocks][R*R]   (U_new - U_old)^T (U_new - U_old) partials
  int n_rblocks;
  Smalls* sm;
  DevState* st;
  int add_uxv;       // 1: P[a,:] += U_{t-1}[a,:] (V_{t-1}^T V_t)  (fused path)
  float alpha;       // U_t = U_{t-1} + alpha (U* - U_{t-1}) in exact mode (1: plain step)
  float* ustar_out;  // optional m x R copy of U* (learned network checkpoints)
};

// ---------------------------------------------------------------------------
// Batches of independent problems (dcf_batch_*): one descriptor per instance
// and, per kernel, a list of work items; a persistent grid walks the list.
// ---------------------------------------------------------------------------
struct BInst {
  const float* M;    // m x n, column-major
  int64_t m, n;
  int r, R, E, u_mode;
  float lam, rho;
  float* U[2];
  float* V[2];
  float* W;
  float* part_p;     // [nsplit][m][R]
  int nsplit;
  int64_t split_cols;
  double* part_h;    // [n_strips]       Huber partial per 64-column strip
  float2* part_q;    // [n_gitems][R*R]  Gram partials (V'^T V', or U^T U at the start)
  float2* part_xv;   // [n_gitems][R*R]  V_old^T (V' - V_old)
  float2* part_dv;   // [n_gitems][R*R]  (V' - V_old)^T (V' - V_old)
  int n_gitems;      // Gram items over the n rows of V
  int n_uitems;      // Gram items over the m rows of U (start point)
  float2* part_g;    // [n_rblocks][R*R]
  float2* part_xu;   // [n_rblocks][R*R]  U_old^T (U_new - U_old)
  float2* part_du;   // [n_rblocks][R*R]  (U_new - U_old)^T (U_new - U_old)
  int n_rblocks;     // 32-row blocks of U
  int n_strips;      // 64-column strips of M
  double* red;       // 6 R*R + 8 doubles: reduced Q, V-side cross, dV Gram, Huber (8),
                     // G, U-side cross, dU Gram
  Smalls* sm;
  DevState* st;
  // the tensor-core single-pass path (k_fused in table mode); 0 = general passes
  int fused;
  int nslabs;        // 256-row slabs = the cluster size
  int n_hparts;      // Huber partials written per iteration (n_strips, or nslabs)
  uint8_t* img;      // [nslabs][U image | W image]
  float* scales;     // 2 nslabs + 1
  float* zmat;       // R x R
  float* VZ;         // n x R, V_old Z
  unsigned int* vmax;  // [2] max |V| of copy 0 / 1 (float bits)
};
// Work item: instance and two indices whose meaning depends on the kernel
// (strip; row block and column split; Gram chunk; 32-row block).
struct BItem {
  int inst;
  int a;
  int b;
  int pad_;
};
constexpr int kBGramRows = 512;   // rows of V (or U) per Gram item

// The single-problem argument block of instance I (for the shared per-item code).
__device__ __forceinline__ IterArgs batch_iter_args(const BInst& I, int cur) {
  IterArgs a{};
  a.cur = cur;
  a.M = I.M;
  a.m = I.m;
  a.n = I.n;
  a.r = I.r;
  a.R = I.R;
  a.lam = I.lam;
  a.rho = I.rho;
  a.u_mode = I.u_mode;
  a.E = I.E;
  a.U[0] = I.U[0]; a.U[1] = I.U[1];
  a.V[0] = I.V[0]; a.V[1] = I.V[1];
  a.W = I.W;
  a.part_q = I.part_q;
  a.part_xv = I.part_xv;
  a.part_dv = I.part_dv;
  a.part_h = I.part_h;
  a.part_p = I.part_p;
  a.n_vblocks = I.n_strips;
  a.n_splits = I.nsplit;
  a.split_cols = I.split_cols;
  a.part_g = I.part_g;
  a.part_xu = I.part_xu;
  a.part_du = I.part_du;
  a.n_rblocks = I.n_rblocks;
  a.sm = I.sm;
  a.st = I.st;
  a.add_uxv = I.fused;   // the fused kernel leaves U_{t-1} (V_{t-1}^T V_t) to the rows
  a.alpha = 1.0f;
  a.ustar_out = nullptr;
  if (I.fused) a.n_vblocks = I.n_hparts;
  return a;
}

// Launchers (stream-ordered; return cudaGetLastError()).
// Gram partials part[b][k*cy + l] = sum over the rows of CTA b of X[a,k] Y[a,l],
// as compensated pairs (hi, lo).
cudaError_t launch_gram(const float* X, int ldx, int cx, const float* Y, int ldy, int cy,
                        int64_t N, float2* part, int nparts, const DevState* st,
                        int respect_stop, cudaStream_t s);
// Per-CTA Gram partials of the new V (Vn) against the old (Vo): Q = Vn^T Vn,
// Vo^T (Vn - Vo) into part_xv and (Vn - Vo)^T (Vn - Vo) into part_dv.
cudaError_t launch_gram_vv(int R, const float* Vo, const float* Vn, int64_t N, float2* part_q,
                           float2* part_xv, float2* part_dv, int nparts, const DevState* st,
                           cudaStream_t s);
cudaError_t launch_make_w(const IterArgs& a, int copy, int respect_stop, cudaStream_t s);
cudaError_t launch_rows(const IterArgs& a, cudaStream_t s);
// U_t = (1/E) sum_i Ui[i] (the server's average of the clients' U after their
// local steps; client rows of ldc >= R floats) with the Gram partials of U_t
// and of its change, as k_rows.
cudaError_t launch_avg_rows(const IterArgs& a, const float* const* Ui, int E, int ldc,
                            cudaStream_t s);
cudaError_t launch_reduce_q(const IterArgs& a, double* out_q, double* out_xv, double* out_dv,
                            double* out_h, int nparts_gram, unsigned int* counter,
                            cudaStream_t s);
cudaError_t launch_reduce_g(const IterArgs& a, double* out_g, double* out_xu, double* out_du,
                            unsigned int* counter, cudaStream_t s);
cudaError_t launch_reduce_init(const IterArgs& a, int which, int copy, const float2* part,
                               int nparts, double* out, unsigned int* counter, cudaStream_t s);
cudaError_t launch_reduce_plain(const float2* part, int nparts, int count, double* out,
                                cudaStream_t s);
// Up to kMaxGramJobs Grams X^T Y in two launches: the compensated partials of
// every job (blockIdx.y = job), then their FP64 sums (the same partials and
// order of summation as launch_gram followed by launch_reduce_plain).
struct GramJob {
  const float* X;
  const float* Y;
  int ldx, cx, ldy, cy;
  int64_t N;       // rows
  int nparts;      // CTAs, one partial each
  float2* part;    // [nparts][cx * cy] scratch
  double* out;     // cx * cy sums, row-major (k, l)
};
constexpr int kMaxGramJobs = 4;
struct GramJobs {
  GramJob j[kMaxGramJobs];
  int n;
};
cudaError_t launch_gram_jobs(const GramJobs& g, cudaStream_t s);
cudaError_t launch_pass1(const IterArgs& a, int grid, int mode_init, int out_copy,
                         cudaStream_t s);
cudaError_t launch_pass2(const IterArgs& a, cudaStream_t s);
cudaError_t prepare_stream_kernels();
// Batched kernels over work-item lists (R = 8, 16 or 32).
//   launch_bpass: which = 1 pass 1 over it1 (mode_init: the S = 0 sweep into copy 0),
//                 which = 2 pass 2 over it2
//   launch_bsmall: kind 0 make_w (arg: respect stop), 1 U-step rows, 2 Gram
//                  (arg: BG_* mode), 3 reduction + tail, one CTA per entry of
//                  `which` (nitems = its length, arg: tail kind)
cudaError_t launch_bpass(int R, int which, const BInst* insts, const BItem* it1, int n1, int grid1,
                         const BItem* it2, int n2, int grid2, int cur, int mode_init,
                         cudaStream_t s);
cudaError_t launch_bsmall(int R, int kind, const BInst* insts, const BItem* items, int nitems,
                          const int* which, int grid, int cur, int arg, cudaStream_t s);
cudaError_t prepare_batch_stream_kernels();
// Batched fused-path preparation: kind 0 U/W images per (instance, slab), kind 1
// V_old Z per (instance, block of 256 entries).
cudaError_t launch_bfused_small(int R, int kind, const BInst* insts, const BItem* items,
                                int nitems, int grid, int cur, cudaStream_t s);
cudaError_t prepare_small_kernels();
cudaError_t launch_materialize(const float* M, int64_t m, int64_t c0, int64_t ni,
                               const float* U, const float* V, int R, float lam,
                               int mode, float* out, cudaStream_t s);
cudaError_t launch_philox_u0(float* U, int64_t m, int r, int R, uint64_t seed,
                             cudaStream_t s);
cudaError_t launch_check_finite(const float* x, int64_t count, int* flag, cudaStream_t s);
cudaError_t launch_apply_mflag(const int* flag, DevState* st, cudaStream_t s);

int pick_R(int r);

// Fused single-pass path (k_fused.cu)
struct FusedArgs {
  int cur;                  // copy holding U_{t-1}, V_{t-1}
  int cs;                   // cluster size (CTAs per cluster)
  int nclusters;
  int nslabs;
  int64_t m, n;
  float lam;
  const float* Vold;        // n x R
  float* Vnew;              // n x R
  const uint8_t* img;       // [slab][U image | W image]
  const float* scales;      // [2*slab] = s_u, [2*slab+1] = s_w, [2*nslabs] = s_v
  const float* zmat;        // R x R, Z = I - rho (U^T U + rho I)^{-1}
  const float* VZ;          // n x R, V_old Z
  unsigned int* vmax_out;   // max |V'| (float bits)
  double* part_h;           // [grid]
  float* part_p;            // [nclusters][m][R]
  DevState* st;
  int* err;
  const void* tmap_g;       // tensor map of M in global memory (table launches)
};
// priority: NULL, or the scheduling priority of the launch (lower = sooner)
cudaError_t launch_fused(int R, const void* tmap, const FusedArgs& fa, cudaStream_t s,
                         const int* priority = nullptr);
// Many problems in one launch: cluster c runs every strip of problem table[c]
// (cs CTAs each; table in device memory, nclusters entries, each with its own
// tensor map in tmap_g, nclusters = 1 and cs equal to the launch's).
cudaError_t launch_fused_table(int R, int cs, int nclusters, const FusedArgs* table,
                               cudaStream_t s);
cudaError_t fused_prepare(int R);
int fused_max_clusters(int R, int cs);
int fused_make_tmap(void* tmap_out, const float* M, int64_t m, int64_t n);
cudaError_t launch_fused_prep(int R, const float* U, const Smalls* sm, const DevState* st,
                              int64_t m, int nslabs, float rho, const unsigned int* vmax_in,
                              unsigned int* vmax_reset, uint8_t* img, float* scales, float* zmat,
                              const float* Vold, int64_t n, float* VZ, cudaStream_t s);
cudaError_t launch_absmax(const float* x, int64_t count, unsigned int* out, cudaStream_t s);

// Whole solve of a small problem in one CTA (k_solve_small.cu), R = 8 or 16,
// exact U-step: n_iter iterations (solve mode: until the stop test) from copy
// `cur`; both copies of U and V are written back, and the state updated.
struct SmallSolveArgs {
  const float* M;     // m x n, column-major
  int64_t m, n;
  float* U[2];
  float* V[2];
  int cur;
  int n_iter;
  float lam, rho;
  DevState* st;
};
size_t solve_small_smem(int R, int64_t m, int64_t n);
cudaError_t solve_small_prepare(int R, size_t smem);
cudaError_t launch_solve_small(int R, const SmallSolveArgs& a, cudaStream_t s);

// Two-pass tensor-core path (k_tc2.cu), R = 16, 32 or 64.
struct Tc2Args {
  int cur;
  int nslabs;
  int G;                     // strip groups (CTAs per slab)
  int64_t m, n;
  float lam;
  const float* Vold;         // n x R
  const float* Vp;           // pass B: V' (n x R)
  const uint8_t* img;        // [slab][U image | W image]
  const float* scales;       // [2 slab] = s_u, [2 slab + 1] = s_w, [2 nslabs] = s_v
  const unsigned int* vp_max;  // pass B: max |V'| (float bits)
  float* ypart;              // pass A: [nslabs][n][R] column sums of C^T W
  double* part_h;            // pass A: [nslabs * G] Huber partials
  float* part_p;             // pass B: [G][m][R] P partials
  const DevState* st;
  int* err;
};
cudaError_t tc2_prepare(int R);
cudaError_t launch_tc2(int R, int pass_b, const void* tmap, const Tc2Args& a, cudaStream_t s);
// Pass A's column-sum partials per column: one per slab, or one per slab pair
// where pass A runs in two-CTA clusters (R = 64, even slab count).
int tc2_parts(int R, int nslabs);
// V' = V_old Z + sum over slabs; max |V'| into vmax and, when non-NULL, vmax_all.
cudaError_t launch_tc2_vreduce(int R, const float* ypart, int nslabs, const float* VZ, int64_t n,
                               float* Vnew, unsigned int* vmax, const DevState* st,
                               int num_sms, cudaStream_t s, unsigned int* vmax_all = nullptr);
// The image preparation of the tensor-core paths also takes R = 64 (dynamic
// shared memory above 48 KB): call once per process before the first launch.
cudaError_t fused_prep_prepare();

// Singular values of factored matrices X Y^T (k_sv.cu): FP64 Gram matrices,
// then one warp per problem (cyclic Jacobi).  sv_prepare once per process.
size_t sv_part_doubles(int nparts);
cudaError_t sv_prepare();
cudaError_t launch_gram64(const float* X, int ldx, const float* Y, int ldy, int p, int64_t N,
                          double* part, int nparts, double* gram_out, cudaStream_t s);
cudaError_t launch_sv_factored(const double* gram, const int* pdim, int nprob, double* sig,
                               cudaStream_t s);
cudaError_t launch_sv_error(const double* sig, const double* sig0, int k, double* err,
                            cudaStream_t s);

}  // namespace dcf
