/*
 * dcf.h -- C ABI of the GB300 DCF-PCA library (libdcf.so).
 *
 * DCF-PCA ("Distributed Robust Principal Component Analysis", arXiv
 * 2207.11669) minimises, over a matrix M = [M_1 ... M_E] split by columns
 * across E clients (§2.1),
 *
 *     1/2 ||U V^T + S - M||_F^2 + rho/2 (||U||_F^2 + ||V||_F^2) + lambda ||S||_1
 *
 * (§1, eq. noncovex_problem).  One iteration (one communication round of
 * Algorithm 1) does, for every client block i,
 *     S_i = soft(M_i - U V_i^T, lambda)                 (§2.2, eq. optS)
 *     V_i = (M_i - S_i)^T U (U^T U + rho I)^{-1}        (App. B, eq. condition1)
 * and then the consensus update of the shared U:
 *     exact mode    U = [sum_i (M_i - S_i) V_i] [sum_i V_i^T V_i + rho I]^{-1}
 *                   (the zero of the summed gradient of App. B, Lemma 2 proof)
 *     FedAvg mode   U_i = U - eta_t grad_U L_i, U = (1/E) sum_i U_i
 *                   (Algorithm 1, eqs. U_local and U_agg), eta_t = eta0/sqrt(t+1).
 * The E clients are column blocks of one device matrix; nothing is sharded.
 *
 * Conventions for every entry point:
 *   - Every call returns a dcf_status and never aborts.  DCF_OK is 0.  The
 *     message of the last failure is available from dcf_last_error().
 *   - Work is enqueued on the handle's stream (dcf_set_stream; default: the
 *     legacy default stream).  Calls that return host data synchronise that
 *     stream.  An error raised by a kernel surfaces at the next call that
 *     synchronises.
 *   - Matrices: M is m x n column-major (column j of block i starts at
 *     M_i + j*ld_i).  Factors are row-major: U is m x r with U[a*r + k],
 *     V_i is n_i x r with V_i[j*r + k].  L_i and S_i outputs are m x n_i
 *     column-major with leading dimension m.
 *   - `where` arguments: 0 = host memory, 1 = device memory of the current
 *     CUDA device.
 *   - The handle owns every buffer it allocates (through the allocator hook,
 *     or cudaMalloc).  The caller owns every buffer it passes in; with
 *     borrow = 1 the caller must keep M alive and unchanged until
 *     dcf_destroy.
 *   - A handle must not be used from two host threads at once.
 */
#ifndef DCF_H
#define DCF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dcf_handle_s* dcf_handle;

typedef enum {
  DCF_OK = 0,
  DCF_EINVAL = 1,      /* invalid argument or size                           */
  DCF_ENOMEM = 2,      /* device or host allocation failed                   */
  DCF_ECUDA = 3,       /* a CUDA runtime call failed                         */
  DCF_ENONFINITE = 4,  /* a NaN or Inf appeared in the data or the iterates  */
  DCF_ETIMEOUT = 5,    /* a bounded device-side wait expired                 */
  DCF_ENOTCONV = 6,    /* dcf_solve reached max_iter above tol               */
  DCF_EPRIVATE = 7,    /* output requested for a block marked private        */
  DCF_ESTATE = 8       /* call order violated (e.g. dcf_step before loading) */
} dcf_status;

/* Problem statement (§2.1) and the parameters of Algorithm 1. */
typedef struct {
  int64_t m;            /* rows of M (the shared dimension of U)              */
  int E;                /* number of client blocks                            */
  const int64_t* n_i;   /* E block widths (host array, copied); n = sum n_i  */
  int r;                /* factor rank, 1 <= r <= 64                          */
  double rho;           /* ridge weight rho > 0 (§1)                          */
  double lambda;        /* l1 weight lambda > 0 (§1)                          */
  int max_iter;         /* dcf_solve: iteration cap (>= 1)                    */
  double tol;           /* dcf_solve: stop when ||L_t-L_{t-1}||_F/||L_t||_F <= tol */
  int u_mode;           /* 0: exact consensus (default); 1: FedAvg gradient   */
  int local_steps;      /* K of Algorithm 1 (>= 1; > 1 needs u_mode = 1)      */
  double eta0;          /* FedAvg mode: eta_t = eta0 / sqrt(t + 1)             */
  uint64_t seed;        /* seed of the default initialisation                  */
  int path;             /* 0: automatic; 1: general two-pass kernels; 2: fused
                           single-pass tensor-core kernel (DCF_EINVAL if the
                           shape does not qualify: r <= 32, m % 4 == 0,
                           m <= 4096); 3: two-pass tensor-core kernels (M
                           read twice, no cross-CTA exchange; DCF_EINVAL
                           unless m % 4 == 0); 4: whole solve in one CTA,
                           every iteration of a dcf_step / dcf_solve call in
                           one launch (DCF_EINVAL unless u_mode = 0, r <= 16
                           and M with the factors fits in one SM's shared
                           memory, about 200 x 200; on request only).
                           Automatic: 2 where it qualifies, else 3 for
                           m % 4 == 0 with m > 4096 or r > 32, else 1         */
} dcf_params;

/* Device allocator hook (no counterpart in the paper: a deployment hook for
 * callers that manage device memory themselves).  alloc(bytes, ctx) returns device memory or NULL,
 * release(ptr, ctx) frees it.  Passing NULLs restores cudaMalloc/cudaFree.
 * Must be set before dcf_create to take effect for that handle.  Pointers
 * must be 256-byte aligned, as cudaMalloc's are; a misaligned one is released
 * again and the call that needed it fails with DCF_ENOMEM. */
typedef void* (*dcf_alloc_fn)(size_t bytes, void* ctx);
typedef void (*dcf_free_fn)(void* ptr, void* ctx);
void dcf_set_allocator(dcf_alloc_fn alloc, dcf_free_fn release, void* ctx);

/* The problem statement of §2.1 (M in R^{m x n} split by columns into E
 * client blocks M_i of n_i columns, rank r) with the weights rho, lambda of
 * §1 and Algorithm 1's round count and step size.
 * Validate `p` and create a handle.  Fails with DCF_EINVAL for m < 1, E < 1,
 * any n_i < 1, r outside [1, 64] or r > m, rho <= 0, lambda <= 0,
 * local_steps < 1, local_steps > 1 with u_mode != 1 (Algorithm 1's local
 * steps are FedAvg gradient steps) or with the whole-solve path 4, or u_mode
 * not in {0, 1}.  With local_steps = K > 1 every client iterates K times on
 * its own block and its own copy U_i before the server averages the U_i
 * (Algorithm 1 eqs. U_local, U_agg); dcf_reload_blocks_async and
 * dcf_profile_step are not available then.  When rho^2 > lambda^2 m n
 * (the necessary condition of §3.2 fails) the handle is still created and
 * dcf_last_error() carries a warning. */
dcf_status dcf_create(const dcf_params* p, dcf_handle* out);

/* (No counterpart in the paper.)  Kernels one iteration launches on the handle's
 * path (graph nodes that are kernels): 7 general, 6 fused (9 when the fused
 * kernel's idle SMs run a share of the columns on the two-pass kernels), 8
 * two-pass tensor core (9 at r > 32), 1 whole solve (per call); -1 with
 * local_steps > 1. */
int dcf_kernels_per_iteration(dcf_handle h);

/* (No counterpart in the paper.)  Which kernels run an iteration: 1 general two-pass path, 2 fused
 * single-pass tensor-core path, 3 two-pass tensor-core path, 4 whole solve in
 * one CTA. */
int dcf_get_path(dcf_handle h);

/* (No counterpart in the paper.)  Enqueue all further work of the handle on
 * `stream` (a cudaStream_t). */
dcf_status dcf_set_stream(dcf_handle h, void* stream);

/* The clients' local data of §2.1: M = [M_1 ... M_E], block M_i in
 * R^{m x n_i} held by client i (Algorithm 1, input).
 * Provide the blocks M_i (m x n_i column-major, leading dimension ld_i >= m).
 * where = 0: host pointers, copied to the device.  where = 1: device
 * pointers; with borrow = 1 the blocks must be one contiguous column-major
 * matrix (M_{i+1} == M_i + m*n_i, ld_i == m) that is used in place, otherwise
 * they are copied.  DCF_EINVAL on NULL pointers or ld_i < m. */
dcf_status dcf_load_blocks(dcf_handle h, const float* const* M_i, const int64_t* ld_i,
                           int where, int borrow);

/* Replace the values of M by new blocks of the same shape and keep the rest
 * of the state: U, V, the iteration count, the r x r workspace and the
 * captured iteration graphs.  The next dcf_step continues from the current
 * factors on the new data: a warm start, as when the clients' local data
 * change between the communication rounds of Algorithm 1.  M_i, ld_i and
 * where as for dcf_load_blocks; the values are copied into the buffer that
 * dcf_load_blocks allocated (its device address does not change).  Returns
 * once the copy and its NaN/Inf check have completed.  DCF_ESTATE before a
 * dcf_load_blocks or when M is borrowed (write the new values into the
 * borrowed matrix instead); DCF_EINVAL as for dcf_load_blocks;
 * DCF_ENONFINITE when a value is NaN or Inf, after which the handle needs a
 * dcf_load_blocks before the next step. */
dcf_status dcf_reload_blocks(dcf_handle h, const float* const* M_i, const int64_t* ld_i,
                             int where);

/* dcf_reload_blocks without waiting: the copy and its NaN/Inf check are
 * enqueued on an internal stream into a second M buffer and the call returns
 * at once.  The next call that iterates (dcf_step, dcf_solve, the learned
 * network's forward pass, dcf_load_init) waits for them on the device and
 * reads the new values, so the copy of the next step's M overlaps the
 * iterations already enqueued; calls that only read factors or statistics do
 * not wait for it, and dcf_get_LS keeps reading the M of the last iteration.
 * The blocks must stay valid and unchanged until the next iteration's results
 * have been read back (e.g. by dcf_get_factors).  A second call before the
 * next step replaces the first; dcf_load_blocks and dcf_reload_blocks discard
 * a pending one.  When the check finds a NaN or Inf, the next iteration stops
 * the solve: the iterations do nothing and dcf_get_stats reports
 * DCF_ENONFINITE until dcf_load_blocks.  DCF_ESTATE and DCF_EINVAL as for
 * dcf_reload_blocks.  The second buffer (m n floats) is allocated on the first
 * call. */
dcf_status dcf_reload_blocks_async(dcf_handle h, const float* const* M_i, const int64_t* ld_i,
                                   int where);

/* Algorithm 1's initialisation of U^(0) and the clients' V_i (the paper leaves
 * the law open; the default below is this library's reading).
 * Set the starting point U0 (m x r) and V0_i (n_i x r).  Without this call
 * dcf_step/dcf_solve start from U0 ~ N(0, 1/m) (counter-based Philox4x32-10,
 * keyed by params.seed) and V0 = M^T U0 (U0^T U0 + rho I)^{-1}, the V-step
 * with S = 0.  Passing V0_i = NULL keeps U0 and computes V0 that way.
 * Resets the iteration counter to 0. */
dcf_status dcf_load_init(dcf_handle h, const float* U0, const float* const* V0_i, int where);

/* Run exactly n_steps iterations, each one communication round t of
 * Algorithm 1: every client's S-step (§2.2 eq. optS) and V-step (App. B eq.
 * condition1), then the server's consensus U (exact, or eqs. U_local and
 * U_agg in FedAvg mode).  No stopping test, as in Algorithm 1's fixed T. */
dcf_status dcf_step(dcf_handle h, int n_steps);

/* Rounds of Algorithm 1 as in dcf_step, with a stopping rule.  The paper runs
 * a fixed number of rounds T and states no rule; the rule below is this
 * library's reading.
 * Iterate until ||U_t V_t^T - U_{t-1} V_{t-1}^T||_F / ||U_t V_t^T||_F <= tol
 * (evaluated exactly from r x r Gram matrices) or max_iter iterations in this
 * call.  Returns DCF_ENOTCONV when the cap is reached above tol.  The
 * iterations run and the last relative change are written when non-NULL. */
dcf_status dcf_solve(dcf_handle h, int* iters_out, double* final_dL_rel);

/* The factors of §2.1's L = U V^T (U shared, V_i per client; Algorithm 1's
 * outputs are L_i = U V_i^T, see dcf_get_LS).
 * Copy out U (m x r) and, when V_i is non-NULL, every V_i (n_i x r). */
dcf_status dcf_get_factors(dcf_handle h, float* U, float* const* V_i, int where);

/* Block i's outputs of Algorithm 1: L_i = U V_i^T and S_i, the S-step of the
 * last iteration, S_i = soft(M_i - U_{t-1} V_{i,t-1}^T, lambda).  Either
 * pointer may be NULL.  DCF_EPRIVATE if block i is marked private,
 * DCF_ESTATE before the first iteration. */
dcf_status dcf_get_LS(dcf_handle h, int i, float* L_i, float* S_i, int where);

/* Mark block i private (1) or public (0); private blocks are never returned
 * by dcf_get_LS (§2.2 "Privacy Preserving", Algorithm 1 output). */
dcf_status dcf_set_private(dcf_handle h, int i, int is_private);

/* (§1 eq. noncovex_problem in its Huber form of §2.2 eq. cancelV; the
 * relative change is the stopping quantity of dcf_solve.)
 * Statistics of the last iteration t: the objective of §1 at
 * (U_{t-1}, V_{t-1}, S_t), evaluated in its Huber form, the relative change
 * of L, and t.  Any pointer may be NULL. */
dcf_status dcf_get_stats(dcf_handle h, double* objective, double* dL_rel, int* iter);

/* (App. B eq. condition1: the ridge systems U^T U + rho I of the V-step and
 * V^T V + rho I of the exact U-step.)
 * 1-norm condition estimates |A|_1 |A^{-1}|_1 of the two r x r systems as the
 * last iteration formed them (0 before the first; kappa_h stays 0 in FedAvg
 * mode, which inverts no V-side system).  Above 100 the inverses are applied
 * in double-float with compensated products, and the Grams that feed them are
 * summed with compensated products (about 1e-5 relative accuracy of the
 * factors up to kappa ~ 1e8 instead of FP32 rounding times kappa).
 * route_g, route_h: how the last inverses were formed: 0 FP32 from the
 * double-float L D L^T factors, 1 double-float.  Any pointer may be NULL. */
dcf_status dcf_get_conditioning(dcf_handle h, double* kappa_g, double* kappa_h, int* route_g,
                                int* route_h);

/* The ground truth of the synthetic experiments of §4.1 (L0 = A B^T) and
 * the relative error of L against it (§4.1 "Evaluation Metric", here the
 * non-squared error of L alone).
 * Register a ground truth L* = A B^T (A: m x k, B: n x k, row-major) so that
 * dcf_rel_err can report ||U V^T - L*||_F / ||L*||_F (from Gram matrices). */
dcf_status dcf_set_truth(dcf_handle h, const float* A, const float* B, int k, int where);
dcf_status dcf_rel_err(dcf_handle h, double* rel_err_L);

/* The relative singular-value error of the upper-bound-rank experiments
 * (§4.2 "Upper-bound rank recovery", Table 1): with a factor rank r above the
 * rank k of the truth (r = p = 2k there), max_i |sigma_i(L) - sigma_i(L0)| /
 * sigma_k(L0), L = U V^T the current iterate and L0 = A B^T the registered
 * truth (dcf_set_truth), sigma_i = 0 beyond a matrix's rank.
 * sigma (required): r host doubles, the singular values of L in descending
 * order.  sigma0 (k host doubles, those of L0) and err may be NULL; asking for
 * either without a registered truth is DCF_ESTATE.  Computed on the device in
 * FP64: Gram matrices G_u = U^T U, G_v = V^T V (exact FP32 products, FP64
 * sums), sigma_i^2 = the eigenvalues of G_u^{1/2} G_v G_u^{1/2} by cyclic
 * Jacobi rotations; likewise for A, B.  Synchronous.  The factors of the
 * current iterate are read in place; the handle allocates its work buffers
 * (partial sums of 64 x 64 doubles for two row ranges per SM, about 10 MB on
 * a 152-SM GPU) on the first call. */
dcf_status dcf_singular_values(dcf_handle h, double* sigma, double* sigma0, double* err);

/* (No counterpart in the paper.)  Message of the last failure (or warning) on
 * this handle; never NULL. */
const char* dcf_last_error(dcf_handle h);

/* (No counterpart in the paper.)  Release everything the handle owns.  Safe on NULL. */
void dcf_destroy(dcf_handle h);

/* (No counterpart in the paper.)  Profiling: number of kernel phases of one iteration (the names, comma
 * separated, are copied into names_csv when it is non-NULL), and
 * dcf_profile_step(), which runs n_steps iterations launching each phase
 * separately (no CUDA graph) and adds each phase's CUDA-event time in
 * milliseconds, measured on the handle's launch stream, to phase_ms[p]. */
int dcf_profile_phases(dcf_handle h, char* names_csv, int len);
dcf_status dcf_profile_step(dcf_handle h, int n_steps, double* phase_ms);

/* Diagnostic: one tcgen05 MMA (fp16 operands, FP32 accumulators in tensor
 * memory) on integer test data with caller-chosen operand layouts and
 * descriptor strides; copies the 128 x 256 accumulator region to out_host.
 * cfg = {M, N, K, a_kind (0 smem K-major, 1 smem MN-major, 2 TMEM),
 *        a_lbo, a_sbo, desc_a_lbo, desc_a_sbo, b_lbo, b_sbo, desc_b_lbo,
 *        desc_b_sbo}.  Used by the tests that pin the tensor-core layouts the
 * fused kernel uses; no counterpart in the paper. */
int dcf_tc_selftest(const int* cfg, float* out_host);

/* ---- Allocation-free iteration ----------------------------------------------
 * One exact-consensus DCF-PCA iteration on buffers the caller owns, for
 * callers that cannot let a library allocate device memory: frameworks that
 * hand out all device memory from their own pools and forbid libraries to
 * call cudaMalloc, and latency-critical loops where cudaMalloc/cudaFree would
 * synchronise the device.  The paper has no counterpart; it is a deployment
 * variant of the general two-pass path of dcf_step (same kernels, same
 * partition of the partial sums).
 *
 * Inputs (device memory of the current device): M, m x n column-major
 * (one block; exact consensus does not depend on the client split); U_in,
 * m x r row-major; V_in, n x r row-major.  Outputs: U_out (m x r) and V_out
 * (n x r), row-major, device memory, not aliasing the inputs.  The work is
 * enqueued on `stream` (a cudaStream_t, NULL = legacy default stream) and is
 * asynchronous; results are valid once the stream has completed it.
 *
 * Scratch: a fixed device array of DCF_NOALLOC_SCRATCH_BYTES inside the
 * library, held by every GPU that loads the library until the process
 * exits.  Returns DCF_EINVAL, touching nothing, when the problem needs more
 * scratch than that (about 4(3m + 2n)R + 4mR*splits bytes plus r x r
 * workspace, R = r rounded up to 8, 16, 32 or 64; m = 300, n = 317, r = 16
 * fits easily, m = 4096, n = 65536, r = 32 does not), and for invalid sizes,
 * rho <= 0, lambda <= 0 or NULL pointers.  Never calls cudaMalloc, cudaFree
 * or any allocating routine.
 *
 * The first call on a device resolves the scratch array's address on that
 * device and raises kernel attributes; make that first call before any stream
 * capture.  Every call shares the array and leaves its contents behind (each
 * call clears what must start at zero), so calls whose work overlaps on the
 * GPU -- on different streams or from different host threads -- race and
 * must be serialised by the caller. */
#define DCF_NOALLOC_SCRATCH_BYTES ((size_t)16 << 20)
dcf_status dcf_iterate_noalloc(const float* M, int64_t m, int64_t n, int r, double rho,
                               double lambda, const float* U_in, const float* V_in,
                               float* U_out, float* V_out, void* stream);

/* ------------------------------------------------------------------------
 * Learned unrolled network (K iterations with per-step parameters) and its
 * adjoint.
 *
 * Step k runs one exact-consensus iteration (S-step of Sec. 2.2, V-step and
 * U-step of App. B) with lambda_k = lambda * exp(a[k]), rho_k = rho * exp(b[k])
 * and the relaxed update U <- U + c[k] (U* - U), where U* is the consensus
 * U-step.  a = b = 0, c = 1 gives K plain iterations.  The loss is
 *   sum_k w_k ||U_k V_k^T - A B^T||_F^2 / ||A B^T||_F^2   (k = 1..K),
 * A, B from dcf_set_truth, w_k = weights[k-1] or 2k / (K (K + 1)) when
 * weights is NULL; it is evaluated through rank-sized Gram matrices.
 * ------------------------------------------------------------------------ */

/* Forward pass from the handle's current factors (the seeded start point if
 * nothing ran yet).  a, b, c: K host doubles each; weights: K host doubles or
 * NULL.  loss_terms (K host doubles, the unweighted per-step losses) and
 * total_loss may be NULL; when either is given, dcf_set_truth must have been
 * called (DCF_ESTATE otherwise).  Afterwards the handle holds U_K, V_K, so
 * dcf_step / dcf_solve continue with plain iterations (lambda, rho of the
 * params).  Checkpoints (U_k, V_k, U*_k): (K+1)(m+n)r + K m r floats on the
 * device, owned by the handle.  Requires u_mode = 0 and r <= 32
 * (DCF_EINVAL).  With loss_terms and total_loss both NULL the loss is not
 * evaluated (inference) and dcf_unrolled_backward is not available for this
 * pass.  Synchronous. */
dcf_status dcf_unrolled_forward(dcf_handle h, int K, const double* a, const double* b,
                                const double* c, const double* weights, double* loss_terms,
                                double* total_loss);

/* Reverse mode of the last dcf_unrolled_forward (which must have had a truth
 * registered; DCF_ESTATE otherwise): d loss / d a[k], d b[k], d c[k] into
 * grad_a, grad_b, grad_c (K host doubles each, any may be NULL), and the
 * gradient with respect to the start point: grad_U0 (m x r row-major) and
 * grad_V0_i[i] (n_i x r row-major), each NULL to skip, on the host
 * (where = 0) or the device (where = 1).  Every m x n quantity is recomputed
 * from M and the checkpoints.  M must be the one the forward pass used.
 * Synchronous. */
dcf_status dcf_unrolled_backward(dcf_handle h, double* grad_a, double* grad_b, double* grad_c,
                                 float* grad_U0, float* const* grad_V0_i, int where);

/* ------------------------------------------------------------------------
 * Batches of independent problems.
 *
 * Many independent DCF-PCA problems (each its own M = [M_1 ... M_E], m, n_i,
 * r <= 32, rho, lambda: the problem of Sec. 2.1 / Algorithm 1 per instance)
 * advance together: one iteration of the whole batch is one CUDA graph of
 * persistent kernels over work-item lists, with the exact consensus U-step of
 * each instance.  An instance whose stop test fired (solve mode) is skipped
 * from then on.  Per-instance results equal those of a single handle on the
 * general path.  All device memory is owned by the batch; M is copied in.
 * ------------------------------------------------------------------------ */
typedef struct dcf_batch_s* dcf_batch;

typedef struct {
  int64_t m;              /* rows */
  int E;                  /* column blocks */
  const int64_t* n_i;     /* E block widths (read during dcf_batch_create only) */
  int r;                  /* rank, 1 <= r <= min(32, m) */
  double rho, lambda;     /* > 0 */
} dcf_problem;

/* count problems; max_iter and tol drive dcf_batch_solve (stop when
 * ||L_t - L_{t-1}||_F / ||L_t||_F <= tol); seed gives each instance's
 * default U0.  DCF_EINVAL on a bad problem, DCF_ENOMEM, DCF_ECUDA. */
dcf_status dcf_batch_create(const dcf_problem* problems, int count, int max_iter, double tol,
                            uint64_t seed, dcf_batch* out);
dcf_status dcf_batch_set_stream(dcf_batch b, void* stream);
/* Copy instance i's blocks (column-major, leading dimension ld_i[k] >= m, or m
 * when ld_i is NULL) from the host (where = 0, synchronous) or the device (1). */
dcf_status dcf_batch_load(dcf_batch b, int i, const float* const* M_i, const int64_t* ld_i,
                          int where);
/* Optional start point of instance i (U0 m x r row-major; V0_i[k] n_k x r or
 * V0_i = NULL for the S = 0 sweep); before the first step only. */
dcf_status dcf_batch_load_init(dcf_batch b, int i, const float* U0, const float* const* V0_i,
                               int where);
/* Autotuner: times the candidate tile shapes of the two streaming passes on
 * this batch (reps launches each) and keeps the fastest; runs by itself
 * before the first step when not called.  The report (one line per
 * candidate and the choice) is copied to report[0 .. report_len). */
dcf_status dcf_batch_tune(dcf_batch b, int reps, char* report, int report_len);
/* n_steps iterations of every running instance (asynchronous). */
dcf_status dcf_batch_step(dcf_batch b, int n_steps);
/* Iterate until every instance met tol or max_iter iterations passed
 * (DCF_ENOTCONV then).  iters_out: count ints (iterations each instance ran),
 * n_converged: instances that met tol; either may be NULL. */
dcf_status dcf_batch_solve(dcf_batch b, int* iters_out, int* n_converged);
/* Instance i's current U (m x r) and V_i (n_k x r), row-major. */
dcf_status dcf_batch_get_factors(dcf_batch b, int i, float* U, float* const* V_i, int where);
dcf_status dcf_batch_get_stats(dcf_batch b, int i, double* objective, double* dL_rel, int* iter);
/* Diagnostics: n_steps iterations launched phase by phase with CUDA events;
 * phase_ms[p] (n_phases >= 7) receives the summed milliseconds of phase p:
 * make_w, pass1_vstep, pass2_pstep, gram_v, reduce_q, rows_ustep, reduce_g. */
dcf_status dcf_batch_profile_step(dcf_batch b, int n_steps, double* phase_ms, int n_phases);
const char* dcf_batch_last_error(dcf_batch b);
void dcf_batch_destroy(dcf_batch b);

/* Library version string. */
const char* dcf_version(void);

#ifdef __cplusplus
}
#endif
#endif /* DCF_H */
