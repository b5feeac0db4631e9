// Small-matrix and per-row kernels of the DCF-PCA iteration.
//
//   k_gram_part      per-CTA partial Gram X^T Y over a row range (compensated
//                    Dot2 products: a float pair per entry)
//   k_reduce_parts   deterministic FP64 sum of those partials over many CTAs;
//                    the last CTA to finish runs the serial r x r tail:
//                      TAIL_Q : Q_t = V_t^T V_t, Cholesky of Q_t + rho I (U-step)
//                      TAIL_G : U_t^T U_t, metrics, stop test, Cholesky of
//                               U_t^T U_t + rho I (next V-step), t <- t + 1
//                      TAIL_INIT_G / TAIL_INIT_Q : the same for the start point
//   k_make_w         W = U (U^T U + rho I)^{-1} row by row (two triangular
//                    solves with the FP64 Cholesky factor rounded to float)
//   k_rows           consensus U-update row by row + Gram partials of U_t
//
// Why FP64 is confined to r x r work: GB300 executes FP64 at roughly two
// fused multiply-adds per clock per SM, so every O(m r) or O(n r) sum runs in
// FP32 with compensation and only the r x r Cholesky factorisations and the
// final cross-CTA sums (spread over many CTAs) use FP64.
#include "dcf_internal.cuh"
#include "dcf_small.cuh"

namespace dcf {

__host__ __device__ __forceinline__ int64_t dmin64(int64_t a, int64_t b) { return a < b ? a : b; }

// ---------------------------------------------------------------------------
// compensated accumulation (Knuth's TwoSum; exact error term of s + x)
// ---------------------------------------------------------------------------
// 16-byte asynchronous global -> shared copy; src_bytes < 16 zero-fills the
// rest (0: nothing is read).
__device__ __forceinline__ void cp_async16(float* sdst, const float* gsrc, int src_bytes) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(sdst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(gsrc),
               "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

__device__ __forceinline__ void two_sum_add(float& hi, float& lo, float x) {
  float t = hi + x;
  float bp = t - hi;
  float err = (hi - (t - bp)) + (x - bp);
  hi = t;
  lo += err;
}

// hi + lo += x * y with the product's rounding error kept (the FMA gives the
// exact error of the FP32 product): the compensated dot product "Dot2" of
// Ogita, Rump and Oishi, "Accurate sum and dot product" (SIAM J. Sci. Comput.,
// 2005), about twice FP32 precision.  Used for the Gram matrices whose
// inverse the next step applies (U^T U, and the start point's Grams), so that
// a nearly singular U^T U + rho I is not perturbed by the FP32 rounding of
// its products.
__device__ __forceinline__ void dot2_add(float& hi, float& lo, float x, float y) {
  const float p = x * y;
  const float e = fmaf(x, y, -p);
  two_sum_add(hi, lo, p);
  lo += e;
}

// ---------------------------------------------------------------------------
// Gram partials:  part[b][k*cy + l] = sum_{rows a of CTA b} X[a,k] * Y[a,l]
// as compensated pairs (hi, lo) (Dot2 per row).  Generic shapes (cx, cy <= 64);
// the per-iteration V Grams use the register-blocked k_gram_vv below.  NS is
// the number of entries per thread (ceil(cx cy / 256)); the loops stay short
// because a launch runs only a few chunks per CTA with a cold instruction
// cache, so unrolled code costs more than it saves.
// ---------------------------------------------------------------------------
constexpr int kGramChunk = 32;

// Partial of CTA b over rows [b rows_per, (b + 1) rows_per) into part[b][*].
template <int NS>
__device__ __forceinline__ void gram_part_body(const float* __restrict__ X, int ldx, int cx,
                                               const float* __restrict__ Y, int ldy, int cy,
                                               int64_t N, int64_t rows_per_cta, int64_t b,
                                               float2* __restrict__ part, float* sh) {
  float* Xs = sh;                           // [chunk][cx]
  float* Ys = sh + kGramChunk * cx;         // [chunk][cy]
  const int tid = threadIdx.x;
  const int ne = cx * cy;
  float hi[NS], lo[NS];
  int xo[NS], yo[NS];
  bool on[NS];
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    hi[s] = 0.f;
    lo[s] = 0.f;
    const int e = tid + s * 256;
    on[s] = e < ne;
    xo[s] = on[s] ? e / cy : 0;
    yo[s] = on[s] ? e % cy : 0;
  }
  const int64_t a0 = b * rows_per_cta;
  const int64_t a1 = min(N, a0 + rows_per_cta);
#pragma unroll 1
  for (int64_t c = a0; c < a1; c += kGramChunk) {
    const int rows = (int)dmin64((int64_t)(kGramChunk), a1 - c);
    __syncthreads();
#pragma unroll 1
    for (int i = tid; i < kGramChunk * cx; i += blockDim.x) {
      const int rr = i / cx, k = i - rr * cx;
      Xs[i] = rr < rows ? X[(c + rr) * ldx + k] : 0.f;
    }
#pragma unroll 1
    for (int i = tid; i < kGramChunk * cy; i += blockDim.x) {
      const int rr = i / cy, k = i - rr * cy;
      Ys[i] = rr < rows ? Y[(c + rr) * ldy + k] : 0.f;
    }
    __syncthreads();
#pragma unroll 4
    for (int rr = 0; rr < rows; ++rr) {
#pragma unroll
      for (int s = 0; s < NS; ++s)
        if (on[s]) dot2_add(hi[s], lo[s], Xs[rr * cx + xo[s]], Ys[rr * cy + yo[s]]);
    }
  }
#pragma unroll
  for (int s = 0; s < NS; ++s)
    if (on[s]) part[b * ne + tid + s * 256] = make_float2(hi[s], lo[s]);
}

template <int NS>
__global__ void __launch_bounds__(256)
k_gram_part(const float* __restrict__ X, int ldx, int cx,
            const float* __restrict__ Y, int ldy, int cy,
            int64_t N, int64_t rows_per_cta, float2* __restrict__ part,
            const DevState* st, int respect_stop) {
  if (respect_stop && st->stop) return;
  extern __shared__ float sh[];
  gram_part_body<NS>(X, ldx, cx, Y, ldy, cy, N, rows_per_cta, blockIdx.x, part, sh);
}

template <int NS>
__global__ void __launch_bounds__(256) k_gram_jobs(GramJobs g) {
  const GramJob& j = g.j[blockIdx.y];
  if ((int)blockIdx.x >= j.nparts) return;
  extern __shared__ float sh[];
  const int64_t rows_per = (j.N + j.nparts - 1) / j.nparts;
  gram_part_body<NS>(j.X, j.ldx, j.cx, j.Y, j.ldy, j.cy, j.N, rows_per, blockIdx.x, j.part, sh);
}

// The Grams of the new V in one pass:  Q = V'^T V',  Y = V_old^T dV  and
// D = dV^T dV with dV = V' - V_old.  (The change metric of the stop test is
// formed from Y and D, which are of the size of the change itself, so that it
// does not cancel against |L|^2; V_old^T V' = Q_old + Y for the fused path.)
// df (ill-conditioned systems): Q and Y are sums of compensated products
// (Dot2), and dV enters Y exactly (TwoSum pair): Q + rho I is inverted for the
// U-step and Q_old + Y is applied to U_{t-1}, where nearly collinear columns
// cancel and FP32 sums of the products would be amplified by the condition
// number.  Otherwise, and always for D (metric only), FP32 sums per chunk.
// Thread tile TB x TB of each output (R >= 32: 4 x 4, R = 16: 2 x 2, R = 8:
// 1 x 1) with 256 / (R/TB)^2 row groups; chunks of rows staged in shared
// memory by a three-stage cp.async ring.  With 4 x 4 tiles a warp reads a
// row's operands in 4 shared-memory wavefronts.
// kDelta = false: Q alone (Vo unused), for start-point Grams.
template <int R>
struct GvvCfg {
  static constexpr int TB = R >= 32 ? 4 : R >= 16 ? 2 : 1;
  static constexpr int NT = R / TB;                 // tiles per dimension
  static constexpr int GROUPS = 256 / (NT * NT);    // row groups
  static constexpr int CH = R >= 64 ? 32 : 64;      // rows per chunk
  static constexpr int NV = (CH * R / 4 + 255) / 256;   // float4 per thread per chunk and array
  static constexpr int STAGES = 3;                  // chunks in flight (cp.async ring)
  static constexpr size_t data_bytes = (size_t)STAGES * 2 * CH * R * 4;
  // the row groups' partial tiles (3 outputs x hi, lo) are combined one tile
  // row at a time
  static constexpr size_t cmb_bytes = GROUPS > 1 ? (size_t)GROUPS * NT * NT * TB * 6 * 4 : 0;
  static constexpr size_t smem_bytes = data_bytes > cmb_bytes ? data_bytes : cmb_bytes;
};

// Rows [a0, a1) of one problem; writes the R*R partials at out_q, out_y, out_d.
// Block-wide (256 threads); gsh: GvvCfg smem.
template <int R, bool kDelta>
__device__ __forceinline__ void gram_vv_block(const float* __restrict__ Vo,
                                              const float* __restrict__ Vn, int64_t a0,
                                              int64_t a1, float2* __restrict__ out_q,
                                              float2* __restrict__ out_y,
                                              float2* __restrict__ out_d, float* gsh, bool df) {
  using C = GvvCfg<R>;
  constexpr int TB = C::TB, NT = C::NT, G = C::GROUPS, CH = C::CH, NV = C::NV, ST = C::STAGES;
  float* So = gsh;              // [CH][R]  V_old rows of the current chunk's stage
  float* Sn = gsh + CH * R;     // [CH][R]  V' rows
  const int tid = threadIdx.x;
  const int tile = tid % (NT * NT), grp = tid / (NT * NT);
  const int k0 = (tile / NT) * TB, l0 = (tile % NT) * TB;
  float qh[TB][TB], ql[TB][TB], yh[TB][TB], yl[TB][TB], dh[TB][TB], dl[TB][TB];
#pragma unroll
  for (int i = 0; i < TB; ++i)
#pragma unroll
    for (int j = 0; j < TB; ++j) {
      qh[i][j] = ql[i][j] = yh[i][j] = yl[i][j] = dh[i][j] = dl[i][j] = 0.f;
    }
  // chunk c into ring stage st: asynchronous copies (no registers held), rows
  // past a1 zero-filled; every thread commits one group per chunk (empty past
  // the end) so that the group counts stay uniform
  auto issue = [&](int64_t c, int st) {
    if (c < a1) {
      const int rows = (int)dmin64((int64_t)CH, a1 - c);
      float* so = gsh + (size_t)st * 2 * CH * R;
      float* sn = so + CH * R;
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        const int i = tid + v * 256;
        if (i < CH * R / 4) {
          const bool in = (4 * i) / R < rows;
          const int64_t off = in ? c * R + 4 * i : c * R;   // a valid address either way
          if (kDelta) cp_async16(so + 4 * i, Vo + off, in ? 16 : 0);
          cp_async16(sn + 4 * i, Vn + off, in ? 16 : 0);
        }
      }
    }
    cp_async_commit();
  };
  const int64_t nch = a0 < a1 ? (a1 - a0 + CH - 1) / CH : 0;
  for (int t = 0; t < ST - 1; ++t) issue(a0 + (int64_t)t * CH, t);
  for (int64_t t = 0; t < nch; ++t) {
    const int64_t c = a0 + t * CH;
    issue(c + (int64_t)(ST - 1) * CH, (int)((t + ST - 1) % ST));
    cp_async_wait<ST - 1>();   // this thread's copies of chunk t have landed
    __syncthreads();           // and every thread's
    So = gsh + (size_t)(t % ST) * 2 * CH * R;
    Sn = So + CH * R;
    float da[TB][TB];
#pragma unroll
    for (int i = 0; i < TB; ++i)
#pragma unroll
      for (int j = 0; j < TB; ++j) da[i][j] = 0.f;
    auto load_row = [&](int rr, float* nk, float* nl, float* ok, float* ol) {
      if constexpr (TB == 4) {
        const float4 a = *reinterpret_cast<const float4*>(Sn + rr * R + k0);
        const float4 d = *reinterpret_cast<const float4*>(Sn + rr * R + l0);
        nk[0] = a.x; nk[1] = a.y; nk[2] = a.z; nk[3] = a.w;
        nl[0] = d.x; nl[1] = d.y; nl[2] = d.z; nl[3] = d.w;
        if (kDelta) {
          const float4 b = *reinterpret_cast<const float4*>(So + rr * R + k0);
          const float4 e = *reinterpret_cast<const float4*>(So + rr * R + l0);
          ok[0] = b.x; ok[1] = b.y; ok[2] = b.z; ok[3] = b.w;
          ol[0] = e.x; ol[1] = e.y; ol[2] = e.z; ol[3] = e.w;
        }
      } else {
#pragma unroll
        for (int i = 0; i < TB; ++i) {
          nk[i] = Sn[rr * R + k0 + i];
          nl[i] = Sn[rr * R + l0 + i];
          if (kDelta) {
            ok[i] = So[rr * R + k0 + i];
            ol[i] = So[rr * R + l0 + i];
          }
        }
      }
    };
    if (df) {
      for (int rr = grp; rr < CH; rr += G) {
        float nk[TB], nl[TB], ok[TB], ol[TB];
        load_row(rr, nk, nl, ok, ol);
        // dV = V' - V_old exactly, as the pair dvh + dvl (TwoSum)
        float dvh[TB], dvl[TB];
        if (kDelta) {
#pragma unroll
          for (int j = 0; j < TB; ++j) {
            dvh[j] = nl[j] - ol[j];
            const float bp = dvh[j] - nl[j];
            dvl[j] = (nl[j] - (dvh[j] - bp)) + (-ol[j] - bp);
          }
        }
#pragma unroll
        for (int i = 0; i < TB; ++i)
#pragma unroll
          for (int j = 0; j < TB; ++j) {
            dot2_add(qh[i][j], ql[i][j], nk[i], nl[j]);
            if (kDelta) {
              dot2_add(yh[i][j], yl[i][j], ok[i], dvh[j]);
              yl[i][j] = fmaf(ok[i], dvl[j], yl[i][j]);
              da[i][j] = fmaf(nk[i] - ok[i], dvh[j], da[i][j]);
            }
          }
      }
    } else {
      // FP32 sums per chunk, compensated across chunks
      float qa[TB][TB], ya[TB][TB];
#pragma unroll
      for (int i = 0; i < TB; ++i)
#pragma unroll
        for (int j = 0; j < TB; ++j) qa[i][j] = ya[i][j] = 0.f;
      // two rows per trip: the next row's shared loads overlap this row's FMAs
#pragma unroll 2
      for (int rr = grp; rr < CH; rr += G) {
        float nk[TB], nl[TB], ok[TB], ol[TB], dk[TB], dl[TB];
        load_row(rr, nk, nl, ok, ol);
#pragma unroll
        for (int i = 0; i < TB; ++i) {
          dk[i] = nk[i] - ok[i];
          dl[i] = nl[i] - ol[i];
        }
#pragma unroll
        for (int i = 0; i < TB; ++i)
#pragma unroll
          for (int j = 0; j < TB; ++j) {
            qa[i][j] = fmaf(nk[i], nl[j], qa[i][j]);
            if (kDelta) {
              ya[i][j] = fmaf(ok[i], dl[j], ya[i][j]);
              da[i][j] = fmaf(dk[i], dl[j], da[i][j]);
            }
          }
      }
#pragma unroll
      for (int i = 0; i < TB; ++i)
#pragma unroll
        for (int j = 0; j < TB; ++j) {
          two_sum_add(qh[i][j], ql[i][j], qa[i][j]);
          if (kDelta) two_sum_add(yh[i][j], yl[i][j], ya[i][j]);
        }
    }
    if (kDelta) {
#pragma unroll
      for (int i = 0; i < TB; ++i)
#pragma unroll
        for (int j = 0; j < TB; ++j) two_sum_add(dh[i][j], dl[i][j], da[i][j]);
    }
    __syncthreads();   // this stage is refilled by the next iteration's issue
  }
  cp_async_wait<0>();   // only empty groups remain; the ring memory is reused below
  // combine the row groups through shared memory, one tile row at a time:
  // cmb[g][tile][j][6] = (hi, lo of Q, Y, D)
  if (G > 1) {
    float* cmb = gsh;
#pragma unroll
    for (int i = 0; i < TB; ++i) {
      __syncthreads();
      if (grp > 0) {
#pragma unroll
        for (int j = 0; j < TB; ++j) {
          float* d = cmb + (((size_t)grp * NT * NT + tile) * TB + j) * 6;
          d[0] = qh[i][j]; d[1] = ql[i][j]; d[2] = yh[i][j]; d[3] = yl[i][j];
          d[4] = dh[i][j]; d[5] = dl[i][j];
        }
      }
      __syncthreads();
      if (grp == 0) {
        for (int g2 = 1; g2 < G; ++g2) {
#pragma unroll
          for (int j = 0; j < TB; ++j) {
            const float* d = cmb + (((size_t)g2 * NT * NT + tile) * TB + j) * 6;
            two_sum_add(qh[i][j], ql[i][j], d[0]);
            ql[i][j] += d[1];
            two_sum_add(yh[i][j], yl[i][j], d[2]);
            yl[i][j] += d[3];
            two_sum_add(dh[i][j], dl[i][j], d[4]);
            dl[i][j] += d[5];
          }
        }
      }
    }
  }
  if (grp == 0) {
#pragma unroll
    for (int i = 0; i < TB; ++i)
#pragma unroll
      for (int j = 0; j < TB; ++j) {
        const int e = (k0 + i) * R + l0 + j;
        out_q[e] = make_float2(qh[i][j], ql[i][j]);
        if (kDelta) {
          out_y[e] = make_float2(yh[i][j], yl[i][j]);
          out_d[e] = make_float2(dh[i][j], dl[i][j]);
        }
      }
  }
}

template <int R>
__global__ void __launch_bounds__(256)
k_gram_vv(const float* __restrict__ Vo, const float* __restrict__ Vn, int64_t N,
          int64_t rows_per_cta, float2* __restrict__ part_q, float2* __restrict__ part_xv,
          float2* __restrict__ part_dv, const DevState* st) {
  if (st->stop) return;
  extern __shared__ __align__(16) float gsh[];
  const int64_t a0 = (int64_t)blockIdx.x * rows_per_cta;
  const int64_t a1 = min(N, a0 + rows_per_cta);
  const int64_t base = (int64_t)blockIdx.x * R * R;
  gram_vv_block<R, true>(Vo, Vn, a0, a1, part_q + base, part_xv + base, part_dv + base, gsh,
                         df_route(st));
}

// ---------------------------------------------------------------------------
// Reduction of partials + serial tail
// ---------------------------------------------------------------------------
enum TailKind { TAIL_NONE = 0, TAIL_Q = 1, TAIL_G = 2, TAIL_INIT_G = 3, TAIL_INIT_Q = 4 };

struct ReduceArgs {
  const float2* part[3];   // compensated partial arrays ([nparts][count_s]) of inputs 0..2
  const double* hpart;     // input 3: FP64 partials (the Huber sum), count[3] <= 1
  int count[4];            // entries per input (0 = unused)
  double* out[4];          // destinations (FP64)
  int nparts[4];
  int total;               // count[0] + ... + count[3]
  int tail;
  int R;
  int r;                   // rank: the leading r x r block of the r x r systems (the
                           // rest is the padding's decoupled rho I); 0: R
  float rho;
  float rho_q;             // rho of Q + rho I in the Q tail when > 0, else rho
  int u_mode;
  int copy;                // TAIL_INIT_*: copy written; TAIL_Q/G: copy holding U_{t-1}
  unsigned int* counter;   // last-block counter (starts at 0, reset by the tail)
  Smalls* sm;
  DevState* st;
};

constexpr int kRedEntriesPerCta = 16;

// The tails leave the r x r system to invert in A and return whether there
// is one; invert_tail then inverts it (one call site for both systems).
__device__ bool tail_q(const ReduceArgs& a, double* A);
__device__ bool tail_g(const ReduceArgs& a, double* A);
__device__ void invert_tail(const ReduceArgs& a, double* A, df2* F);

// Dynamic shared memory of a reduction tail: R*R doubles (A), R*R
// double-floats (F).
constexpr size_t tail_smem(int R) { return (size_t)R * R * (sizeof(double) + sizeof(df2)); }

__global__ void __launch_bounds__(256) k_reduce_parts(ReduceArgs a) {
  if ((a.tail == TAIL_Q || a.tail == TAIL_G) && a.st->stop) return;
  __shared__ double red[256];
  __shared__ bool is_last;
  const int tid = threadIdx.x;
  const int e_local = tid % kRedEntriesPerCta;
  const int lane_p = tid / kRedEntriesPerCta;          // 0..15
  const int nsplit = 256 / kRedEntriesPerCta;
  const int e = blockIdx.x * kRedEntriesPerCta + e_local;
  __shared__ float2 red2[256];
  float hi = 0.f, lo = 0.f;
  double hs = 0.0;
  int which = -1, idx = 0;
  if (e < a.total) {
    idx = e;
    which = 0;
    while (idx >= a.count[which]) { idx -= a.count[which]; ++which; }
    if (which < 3) {
      const float2* p = a.part[which];
      const int cnt = a.count[which];
      const int np = a.nparts[which];
      // groups of 8 loads issued together, summed in order
      for (int q0 = lane_p; q0 < np; q0 += 8 * nsplit) {
        float2 v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int q = q0 + u * nsplit;
          v[u] = q < np ? p[(int64_t)q * cnt + idx] : make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          two_sum_add(hi, lo, v[u].x);
          lo += v[u].y;
        }
      }
    } else {
      for (int q = lane_p; q < a.nparts[3]; q += nsplit) hs += a.hpart[q];
    }
  }
  red2[tid] = make_float2(hi, lo);
  red[tid] = hs;
  __syncthreads();
  if (lane_p == 0 && which >= 0) {
    if (which < 3) {
      float th = 0.f, tl = 0.f;
      for (int q = 0; q < nsplit; ++q) {
        const float2 v = red2[q * kRedEntriesPerCta + e_local];
        two_sum_add(th, tl, v.x);
        tl += v.y;
      }
      a.out[which][idx] = (double)th + (double)tl;
    } else {
      double t = 0.0;
      for (int q = 0; q < nsplit; ++q) t += red[q * kRedEntriesPerCta + e_local];
      a.out[which][idx] = t;
    }
  }
  if (a.tail == TAIL_NONE) return;
  // last-block-done: the CTA that finishes last runs the serial tail
  __threadfence();
  __syncthreads();
  if (tid == 0) {
    unsigned int prev = atomicAdd(a.counter, 1u);
    is_last = (prev == gridDim.x - 1);
  }
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  extern __shared__ double dsh[];   // tail_smem(R): A, F
  df2* F = reinterpret_cast<df2*>(dsh + a.R * a.R);
  if (tid == 0) *a.counter = 0u;
  const bool inv = (a.tail == TAIL_Q || a.tail == TAIL_INIT_Q) ? tail_q(a, dsh) : tail_g(a, dsh);
  if (inv) invert_tail(a, dsh, F);
}

// Q_t is in out[0] (R*R), Y = V_{t-1}^T (V_t - V_{t-1}) in out[1], the Gram of
// V_t - V_{t-1} in out[2], Huber in out[3].  V_{t-1}^T V_t = Q_{t-1} + Y.
__device__ bool tail_q(const ReduceArgs& a, double* A) {
  const int R = a.R;
  Smalls* sm = a.sm;
  DevState* st = a.st;
  if (a.tail == TAIL_INIT_Q) {
    // start point: only V0^T V0 is needed (for the first metrics)
    for (int i = threadIdx.x; i < R * R; i += blockDim.x) sm->q[a.copy][i] = __ldcg(a.out[0] + i);
    return false;
  }
  const int cur = a.copy, nxt = cur ^ 1;
  // a rolled loop: this tail runs once on one CTA with the instruction cache
  // cold, so code size costs more than load latency
  const double rq = (double)(a.rho_q > 0.f ? a.rho_q : a.rho);
#pragma unroll 1
  for (int i = threadIdx.x; i < R * R; i += blockDim.x) {
    const double qv = __ldcg(a.out[0] + i), yv = __ldcg(a.out[1] + i);
    const double dv = __ldcg(a.out[2] + i), qo = sm->q[cur][i];
    sm->q[nxt][i] = qv;
    sm->dvy[i] = yv;
    sm->dvv[i] = dv;
    const double xv = qo + yv;
    sm->xv[i] = xv;
    const float xh = (float)xv;
    sm->xv32[0][i] = xh;
    sm->xv32[1][i] = (float)(xv - (double)xh);
    const double h = qv + ((i / R) == (i % R) ? rq : 0.0);
    A[i] = h;
    sm->qrho32[i] = (float)h;
  }
  if (threadIdx.x == 0) st->huber = __ldcg(a.out[3]);
  __syncthreads();
  if (!all_finite(A, R * R)) {
    if (threadIdx.x == 0) st->status = 4;  // DCF_ENONFINITE
    return false;
  }
  return a.u_mode == 0;   // FedAvg steps with Q_t + rho I itself
}

// (Q_t + rho I)^{-1} (hi + lo rounded) or (U_t^T U_t + rho I)^{-1} (hi, lo).
__device__ void invert_tail(const ReduceArgs& a, double* A, df2* F) {
  const bool q = a.tail == TAIL_Q || a.tail == TAIL_INIT_Q;
  Smalls* sm = a.sm;
  DevState* st = a.st;
  float* hi = q ? sm->hinv32 : sm->ginv32;
  float* lo = q ? nullptr : sm->ginv32_lo;
  const double kappa = spd_inverse(A, F, a.R, a.r > 0 ? a.r : a.R, hi, lo, kDfKappa,
                                   q ? &st->route_h : &st->route_g);
  if (threadIdx.x == 0) {
    if (q) st->kappa_h = kappa;
    else st->kappa_g = kappa;
  }
}

// Gram of U_t in out[0], U_{t-1}^T (U_t - U_{t-1}) in out[1], the Gram of
// U_t - U_{t-1} in out[2].
__device__ bool tail_g(const ReduceArgs& a, double* A) {
  const int R = a.R;
  Smalls* sm = a.sm;
  DevState* st = a.st;
  int tgt;
  if (a.tail == TAIL_INIT_G) {
    tgt = a.copy;
    for (int i = threadIdx.x; i < R * R; i += blockDim.x) sm->gram[tgt][i] = __ldcg(a.out[0] + i);
  } else {
    const int cur = a.copy;
    tgt = cur ^ 1;
    // metrics.  With dU = U_t - U_{t-1}, dV = V_t - V_{t-1}:
    //   L_t - L_{t-1} = dU V_t^T + U_{t-1} dV^T, so
    //   |L_t - L_{t-1}|^2 = <dU^T dU, Q_t> + 2 <(U_{t-1}^T dU)^T, V_t^T dV>
    //                       + <G_{t-1}, dV^T dV>,   V_t^T dV = Y + dV^T dV,
    // every term of the size of the change (no cancellation against |L|^2);
    // |L_t|^2 = <G_t, Q_t>.  Six FP64 sums in one reduction: per-thread partials,
    // a shuffle tree per warp, then the per-warp values across lanes of warp 0.
    // Every load of the thread's entries is issued before any store or product;
    // the new Gram also goes straight into A (G_t + rho I) for the inverse below.
    // The loops are rolled: this tail runs once on one CTA with the
    // instruction cache cold, so code size costs more than load latency.
    __shared__ double s6[6][256];   // per-thread partial sums, then the six totals in [q][0]
    double v0 = 0, v1 = 0, v2 = 0, v3 = 0, v4 = 0, v5 = 0;
#pragma unroll 1
    for (int i = threadIdx.x; i < R * R; i += blockDim.x) {
      const int r = i / R, c = i % R;
      const double gn = __ldcg(a.out[0] + i), a2 = __ldcg(a.out[1] + i);
      const double a2t = __ldcg(a.out[1] + c * R + r), a1 = __ldcg(a.out[2] + i);
      const double qn = sm->q[tgt][i], b3 = sm->dvv[i], b2 = sm->dvy[i] + b3;
      const double go = sm->gram[cur][i], qo = sm->q[cur][i];
      sm->gram[tgt][i] = gn;
      sm->xu[i] = a2;
      A[i] = gn + (r == c ? (double)a.rho : 0.0);
      v0 = fma(gn, qn, v0);
      v1 = fma(a1, qn, v1);
      v2 = fma(a2t, b2, v2);
      v3 = fma(go, b3, v3);
      if (r == c) {
        v4 += go;
        v5 += qo;
      }
    }
    s6[0][threadIdx.x] = v0; s6[1][threadIdx.x] = v1; s6[2][threadIdx.x] = v2;
    s6[3][threadIdx.x] = v3; s6[4][threadIdx.x] = v4; s6[5][threadIdx.x] = v5;
    __syncthreads();
    // warp q < 6 adds row q of s6
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (wid < 6) {
      double t = 0.0;
#pragma unroll 1
      for (int k = lane; k < 256; k += 32) t += s6[wid][k];
#pragma unroll 1
      for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
      __syncwarp();
      if (lane == 0) s6[wid][0] = t;
    }
    __syncthreads();
    double v[6];
    if (threadIdx.x == 0)
      for (int q = 0; q < 6; ++q) v[q] = s6[q][0];
    if (threadIdx.x == 0) {
      const double a0 = v[0];
      double d2 = v[1] + 2.0 * v[2] + v[3];
      if (d2 < 0) d2 = 0;
      st->dL_rel = a0 > 0 ? sqrt(d2 / a0) : INFINITY;
      st->objective = st->huber + 0.5 * (double)a.rho * (v[4] + v[5]);
      st->iter = st->iter + 1;
      st->has_S = 1;
      if (!isfinite(a0) || !isfinite(st->objective)) st->status = 4;
      if (st->solve_mode && st->dL_rel <= st->tol) st->stop = 1;
    }
    __syncthreads();
  }
  // (U^T U + rho I)^{-1} for the next V-step (A already holds it after the metrics)
  if (a.tail == TAIL_INIT_G)
    for (int i = threadIdx.x; i < R * R; i += blockDim.x) {
      const int r = i / R, c = i % R;
      A[i] = sm->gram[tgt][i] + (r == c ? (double)a.rho : 0.0);
    }
  __syncthreads();
  if (!all_finite(A, R * R)) {
    if (threadIdx.x == 0) st->status = 4;
    return false;
  }
  return true;
}

// ---------------------------------------------------------------------------
// Row kernels: a CTA of 256 threads owns 32 rows; thread (row t/8, column
// group t%8) forms R/8 outputs of (row) x (R x R matrix).
// ---------------------------------------------------------------------------
constexpr int kRowsPerCta = 32;

// W = U (U^T U + rho I)^{-1}
// Rows [32 rb, 32 rb + 32) of W = U G^{-1}; block-wide (256 threads).  df: G
// is ill-conditioned, G^{-1} is the double-float pair hi + lo and the products
// with hi are compensated (Dot2), so that W carries the inverse's ~44 bits up
// to its own FP32 rounding (the rows of U G^{-1} cancel then).
template <int R>
__device__ __forceinline__ void make_w_block(const float* __restrict__ U, const Smalls* sm,
                                             float* __restrict__ W, int64_t m, int64_t rb,
                                             bool df) {
  constexpr int CG = R / 8;
  __shared__ __align__(16) float Gi[R * R];
  __shared__ __align__(16) float Gl[R * R];
  __shared__ __align__(16) float Us[kRowsPerCta * R];
  const int tid = threadIdx.x;
  const int64_t row0 = rb * kRowsPerCta;
  for (int i = tid; i < R * R; i += 256) {
    Gi[i] = sm->ginv32[i];
    Gl[i] = sm->ginv32_lo[i];
  }
  for (int i = tid; i < kRowsPerCta * R; i += 256) {
    int64_t a = row0 + i / R;
    Us[i] = a < m ? U[row0 * R + i] : 0.f;
  }
  __syncthreads();
  const int ar = tid >> 3, g = tid & 7;
  const int64_t a = row0 + ar;
  if (a >= m) return;
  float acc[CG], lo[CG];
#pragma unroll
  for (int l = 0; l < CG; ++l) acc[l] = lo[l] = 0.f;
  if (df) {
    for (int k = 0; k < R; ++k) {
      const float u = Us[ar * R + k];
#pragma unroll
      for (int l = 0; l < CG; ++l) {
        dot2_add(acc[l], lo[l], u, Gi[k * R + g * CG + l]);
        lo[l] = fmaf(u, Gl[k * R + g * CG + l], lo[l]);
      }
    }
  } else {
    for (int k = 0; k < R; ++k) {
      const float u = Us[ar * R + k];
#pragma unroll
      for (int l = 0; l < CG; ++l) acc[l] = fmaf(u, Gi[k * R + g * CG + l], acc[l]);
    }
  }
#pragma unroll
  for (int l = 0; l < CG; ++l) W[a * R + g * CG + l] = acc[l] + lo[l];
}

template <int R>
__global__ void __launch_bounds__(256) k_make_w(const float* __restrict__ U,
                                                const DevState* st, const Smalls* sm,
                                                float* __restrict__ W, int64_t m,
                                                int respect_stop) {
  if (respect_stop && st->stop) return;
  make_w_block<R>(U, sm, W, m, blockIdx.x, df_route(st));
}

// Gram partials over a CTA's rows of U: G = Un^T Un (compensated products:
// its inverse is applied in the next V-step), Uo^T dU and dU^T dU with
// dU = Un - Uo (the change metric is formed from the last two, which are of
// the size of the change).  Block-wide; Uo, Un: rows x R in shared memory.
template <int R>
__device__ __forceinline__ void rows_gram_partials(const IterArgs& a, const float* Uo,
                                                   const float* Un, int rows, int64_t rb) {
  for (int e = threadIdx.x; e < R * R; e += blockDim.x) {
    const int k = e / R, l = e % R;
    float gh = 0.f, gl = 0.f, xu = 0.f, du = 0.f;
    for (int rr = 0; rr < rows; ++rr) {
      const float dk = Un[rr * R + k] - Uo[rr * R + k];
      const float dl = Un[rr * R + l] - Uo[rr * R + l];
      dot2_add(gh, gl, Un[rr * R + k], Un[rr * R + l]);
      xu = fmaf(Uo[rr * R + k], dl, xu);
      du = fmaf(dk, dl, du);
    }
    a.part_g[rb * R * R + e] = make_float2(gh, gl);
    a.part_xu[rb * R * R + e] = make_float2(xu, 0.f);
    a.part_du[rb * R * R + e] = make_float2(du, 0.f);
  }
}

// Consensus U-update plus Gram partials of the new U:
//   exact:  U_t[a,:] = P[a,:] (Q_t + rho I)^{-1},  P[a,:] = sum_s part_p[s][a,:]
//   FedAvg: U_t[a,:] = U[a,:] - (eta_t/E) (U[a,:] (Q_t + rho I) - P[a,:])
// 32-row block rb of the U-step and its Gram partials; block-wide (256 threads).
template <int R>
__device__ __forceinline__ void rows_block(const IterArgs& a, int64_t rb) {
  DevState* st = a.st;
  constexpr int CG = R / 8;
  __shared__ __align__(16) float Mat[R * R];
  __shared__ __align__(16) float Ps[kRowsPerCta * R];
  __shared__ __align__(16) float Uo[kRowsPerCta * R];
  __shared__ __align__(16) float Un[kRowsPerCta * R];
  const int tid = threadIdx.x;
  const int cur = a.cur, nxt = cur ^ 1;
  const float* U = a.U[cur];
  float* Unew = a.U[nxt];
  const int64_t row0 = rb * kRowsPerCta;
  const int rows = (int)dmin64((int64_t)kRowsPerCta, a.m - row0);
  if (a.add_uxv)
    for (int i = tid; i < R * R; i += 256) Mat[i] = a.sm->xv32[0][i];
  // The thread's PER entries: U and the partials of P, every load of a group
  // of 8 splits in flight together (one latency round per group instead of
  // one per entry and group).
  constexpr int PER = kRowsPerCta * R / 256;
  {
    float hi[PER], lo[PER], uo[PER];
    int64_t off[PER];
    bool in[PER];
#pragma unroll
    for (int u = 0; u < PER; ++u) {
      const int i = tid + u * 256;
      in[u] = i / R < rows;
      off[u] = row0 * R + i;
      uo[u] = in[u] ? U[off[u]] : 0.f;
      hi[u] = lo[u] = 0.f;
    }
    for (int s0 = 0; s0 < a.n_splits; s0 += 8) {
      float v[8][PER];
#pragma unroll
      for (int q = 0; q < 8; ++q)
#pragma unroll
        for (int u = 0; u < PER; ++u)
          v[q][u] = s0 + q < a.n_splits && in[u]
                        ? a.part_p[(int64_t)(s0 + q) * a.m * R + off[u]] : 0.f;
#pragma unroll
      for (int q = 0; q < 8; ++q)
#pragma unroll
        for (int u = 0; u < PER; ++u)
          if (s0 + q < a.n_splits) two_sum_add(hi[u], lo[u], v[q][u]);
    }
#pragma unroll
    for (int u = 0; u < PER; ++u) {
      Ps[tid + u * 256] = hi[u] + lo[u];
      Uo[tid + u * 256] = uo[u];
    }
  }
  __syncthreads();
  const int ar = tid >> 3, g = tid & 7;
  if (a.add_uxv) {
    // P = U_{t-1} (V_{t-1}^T V_t) + C V'   (the fused pass returns only C V').
    // V_{t-1}^T V_t = hi + lo, compensated products: with nearly collinear
    // columns the terms of U_{t-1} (V_{t-1}^T V_t) cancel.
    // (Ill-conditioned systems only; otherwise FP32 products with hi.)
    const float* __restrict__ Xl = a.sm->xv32[1];
    float add[CG], addl[CG];
#pragma unroll
    for (int l = 0; l < CG; ++l) add[l] = addl[l] = 0.f;
    if (df_route(st)) {
      for (int k = 0; k < R; ++k) {
        const float u = Uo[ar * R + k];
#pragma unroll
        for (int l = 0; l < CG; ++l) {
          dot2_add(add[l], addl[l], u, Mat[k * R + g * CG + l]);
          addl[l] = fmaf(u, __ldg(Xl + k * R + g * CG + l), addl[l]);
        }
      }
    } else {
      for (int k = 0; k < R; ++k) {
        const float u = Uo[ar * R + k];
#pragma unroll
        for (int l = 0; l < CG; ++l) add[l] = fmaf(u, Mat[k * R + g * CG + l], add[l]);
      }
    }
    __syncthreads();
#pragma unroll
    for (int l = 0; l < CG; ++l) {
      float h = add[l], lo = addl[l];
      two_sum_add(h, lo, Ps[ar * R + g * CG + l]);
      Ps[ar * R + g * CG + l] = h + lo;
    }
  }
  for (int i = tid; i < R * R; i += 256) Mat[i] = a.u_mode == 0 ? a.sm->hinv32[i] : a.sm->qrho32[i];
  __syncthreads();
  float acc[CG];
#pragma unroll
  for (int l = 0; l < CG; ++l) acc[l] = 0.f;
  const float* src = a.u_mode == 0 ? Ps : Uo;
  for (int k = 0; k < R; ++k) {
    const float v = src[ar * R + k];
#pragma unroll
    for (int l = 0; l < CG; ++l) acc[l] = fmaf(v, Mat[k * R + g * CG + l], acc[l]);
  }
  if (a.u_mode != 0) {
    const double eta =
        st->eta_fixed > 0.0 ? st->eta_fixed : st->eta0 / sqrt((double)st->iter + 1.0);
    const float step = (float)(eta / (double)a.E);
#pragma unroll
    for (int l = 0; l < CG; ++l) {
      const int c = g * CG + l;
      acc[l] = Uo[ar * R + c] - step * (acc[l] - Ps[ar * R + c]);
    }
  }
  if (a.u_mode == 0 && a.alpha != 1.0f) {
    // relaxed consensus step of the learned network: U_t = U + alpha (U* - U)
#pragma unroll
    for (int l = 0; l < CG; ++l) {
      const int c = g * CG + l;
      if (a.ustar_out && ar < rows) a.ustar_out[(row0 + ar) * R + c] = acc[l];
      acc[l] = fmaf(a.alpha, acc[l] - Uo[ar * R + c], Uo[ar * R + c]);
    }
  } else if (a.ustar_out && ar < rows) {
#pragma unroll
    for (int l = 0; l < CG; ++l) a.ustar_out[(row0 + ar) * R + g * CG + l] = acc[l];
  }
  bool finite = true;
#pragma unroll
  for (int l = 0; l < CG; ++l) {
    const int c = g * CG + l;
    const float v = ar < rows ? acc[l] : 0.f;
    finite = finite && isfinite(v);
    Un[ar * R + c] = v;
    if (ar < rows) Unew[(row0 + ar) * R + c] = v;
  }
  if (!finite) st->status = 4;
  __syncthreads();
  rows_gram_partials<R>(a, Uo, Un, rows, rb);
}

template <int R>
__global__ void __launch_bounds__(256) k_rows(IterArgs a) {
  if (a.st->stop) return;
  rows_block<R>(a, blockIdx.x);
}

// The server's step of Algorithm 1 (eq. U_agg) after the clients' local steps:
// U_t[a,:] = (1/E) sum_i Ui[i][a,:], the clients summed in order, plus the
// Gram partials of the 32-row block (rows_gram_partials), as the consensus
// rows kernel leaves them for the metrics.  The clients' rows
// have ldc >= R entries (their own padded rank); columns past R are zero.
template <int R>
__global__ void __launch_bounds__(256) k_avg_rows(IterArgs a, const float* const* __restrict__ Ui,
                                                  int E, int ldc) {
  if (a.st->stop) return;
  __shared__ __align__(16) float Uo[kRowsPerCta * R];
  __shared__ __align__(16) float Un[kRowsPerCta * R];
  const int tid = threadIdx.x;
  const int64_t rb = blockIdx.x;
  const float* U = a.U[a.cur];
  float* Unew = a.U[a.cur ^ 1];
  const int64_t row0 = rb * kRowsPerCta;
  const int rows = (int)dmin64((int64_t)kRowsPerCta, a.m - row0);
  const float invE = 1.f / (float)E;
  bool finite = true;
  for (int i = tid; i < kRowsPerCta * R; i += 256) {
    const int rr = i / R;
    float uo = 0.f, un = 0.f;
    if (rr < rows) {
      const int64_t off = row0 * R + i;
      const int64_t offc = (row0 + rr) * ldc + (i % R);
      uo = U[off];
      float hi = 0.f, lo = 0.f;
      for (int c = 0; c < E; ++c) two_sum_add(hi, lo, Ui[c][offc]);
      un = (hi + lo) * invE;
      finite = finite && isfinite(un);
      Unew[off] = un;
    }
    Uo[i] = uo;
    Un[i] = un;
  }
  if (!finite) a.st->status = 4;
  __syncthreads();
  rows_gram_partials<R>(a, Uo, Un, rows, rb);
}

// ---------------------------------------------------------------------------
// Batches of independent problems: the per-item functions above, driven by
// work-item lists, and one reduction CTA per instance.
// ---------------------------------------------------------------------------
enum BGramMode { BG_ITER = 0, BG_INIT_U = 1, BG_INIT_V = 2 };

template <int R>
__global__ void __launch_bounds__(256) k_bmake_w(const BInst* __restrict__ insts,
                                                 const BItem* __restrict__ items, int nitems,
                                                 int cur, int respect_stop) {
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const BItem w = items[it];
    const BInst& I = insts[w.inst];
    if (respect_stop && I.st->stop) continue;
    __syncthreads();
    make_w_block<R>(I.U[cur], I.sm, I.W, I.m, w.a, df_route(I.st));
  }
}

template <int R>
__global__ void __launch_bounds__(256) k_brows(const BInst* __restrict__ insts,
                                               const BItem* __restrict__ items, int nitems,
                                               int cur) {
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const BItem w = items[it];
    const BInst& I = insts[w.inst];
    if (I.st->stop) continue;
    const IterArgs a = batch_iter_args(I, cur);
    __syncthreads();
    rows_block<R>(a, w.a);
  }
}

// Gram items: BG_ITER  Q = V'^T V', X_v = V^T V'   (item a: chunk of kBGramRows rows of V)
//             BG_INIT_U  U0^T U0 into part_q          (chunks of the m rows of U)
//             BG_INIT_V  V0^T V0 into part_q
template <int R>
__global__ void __launch_bounds__(256) k_bgram(const BInst* __restrict__ insts,
                                               const BItem* __restrict__ items, int nitems,
                                               int cur, int mode) {
  extern __shared__ __align__(16) float gsh[];
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const BItem w = items[it];
    const BInst& I = insts[w.inst];
    if (mode == BG_ITER && I.st->stop) continue;
    const float* X = mode == BG_ITER ? I.V[cur] : mode == BG_INIT_U ? I.U[0] : I.V[0];
    const float* Y = mode == BG_ITER ? I.V[cur ^ 1] : X;
    const int64_t N = mode == BG_INIT_U ? I.m : I.n;
    const int64_t a0 = (int64_t)w.a * kBGramRows;
    const int64_t a1 = min(N, a0 + (int64_t)kBGramRows);
    __syncthreads();
    const int64_t base = (int64_t)w.a * R * R;
    if (mode == BG_ITER)
      gram_vv_block<R, true>(X, Y, a0, a1, I.part_q + base, I.part_xv + base, I.part_dv + base,
                             gsh, df_route(I.st));
    else   // start point (once): compensated
      gram_vv_block<R, false>(X, Y, a0, a1, I.part_q + base, nullptr, nullptr, gsh, true);
  }
}

// One CTA per instance (list `which`): reduce the instance's partials in
// compensated FP32 pairs, store them in FP64, then run the r x r tail.
//   tail TAIL_Q      Q, V-side cross, dV Gram (Gram items), Huber (strips) -> (Q + rho I)^{-1}
//   tail TAIL_G      G, U-side cross, dU Gram (32-row blocks) -> metrics, stop, (G + rho I)^{-1}
//   tail TAIL_INIT_G U0^T U0 (Gram items over m rows);  TAIL_INIT_Q  V0^T V0
// red layout: Q, V-side cross, dV Gram (R*R each), Huber (8), G, U-side cross, dU Gram.
template <int R>
__global__ void __launch_bounds__(256) k_breduce(const BInst* __restrict__ insts,
                                                 const int* __restrict__ which, int cur,
                                                 int tail) {
  const BInst& I = insts[which[blockIdx.x]];
  if ((tail == TAIL_Q || tail == TAIL_G) && I.st->stop) return;
  constexpr int RR = R * R;
  double* red = I.red;
  const bool gside = tail == TAIL_G || tail == TAIL_INIT_G;
  double* out0 = gside ? red + 3 * RR + 8 : red;
  double* out1 = out0 + RR;
  double* out2 = out1 + RR;
  const float2* p0 = gside && tail == TAIL_G ? I.part_g : I.part_q;
  const float2* p1 = tail == TAIL_G ? I.part_xu : I.part_xv;
  const float2* p2 = tail == TAIL_G ? I.part_du : I.part_dv;
  const int np = tail == TAIL_G ? I.n_rblocks : tail == TAIL_INIT_G ? I.n_uitems : I.n_gitems;
  const bool three = tail == TAIL_Q || tail == TAIL_G;
  for (int e = threadIdx.x; e < RR; e += blockDim.x) {
    float h0 = 0.f, l0 = 0.f, h1 = 0.f, l1 = 0.f, h2 = 0.f, l2 = 0.f;
    for (int q = 0; q < np; ++q) {
      const float2 v0 = p0[(int64_t)q * RR + e];
      two_sum_add(h0, l0, v0.x);
      l0 += v0.y;
      if (three) {
        const float2 v1 = p1[(int64_t)q * RR + e];
        two_sum_add(h1, l1, v1.x);
        l1 += v1.y;
        const float2 v2 = p2[(int64_t)q * RR + e];
        two_sum_add(h2, l2, v2.x);
        l2 += v2.y;
      }
    }
    out0[e] = (double)h0 + (double)l0;
    if (three) {
      out1[e] = (double)h1 + (double)l1;
      out2[e] = (double)h2 + (double)l2;
    }
  }
  if (tail == TAIL_Q && threadIdx.x < 32) {
    double hs = 0.0;
    for (int q = threadIdx.x; q < I.n_hparts; q += 32) hs += I.part_h[q];
    for (int o = 16; o > 0; o >>= 1) hs += __shfl_xor_sync(0xffffffffu, hs, o);
    if (threadIdx.x == 0) red[3 * RR] = hs;
  }
  __threadfence();
  __syncthreads();
  ReduceArgs ra{};
  ra.out[0] = out0;
  ra.out[1] = out1;
  ra.out[2] = out2;
  ra.out[3] = red + 3 * RR;
  ra.tail = tail;
  ra.R = R;
  ra.r = I.r;
  ra.rho = I.rho;
  ra.u_mode = I.u_mode;
  ra.copy = (tail == TAIL_INIT_G || tail == TAIL_INIT_Q) ? 0 : cur;
  ra.sm = I.sm;
  ra.st = I.st;
  extern __shared__ double dsh[];   // tail_smem(R): A, F
  df2* F = reinterpret_cast<df2*>(dsh + RR);
  const bool inv = (tail == TAIL_Q || tail == TAIL_INIT_Q) ? tail_q(ra, dsh) : tail_g(ra, dsh);
  if (inv) invert_tail(ra, dsh, F);
}

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon et al., SC'11) for the default starting point U0.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void philox_round(uint32_t& x0, uint32_t& x1, uint32_t& x2,
                                             uint32_t& x3, uint32_t k0, uint32_t k1) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  uint32_t hi0 = __umulhi(M0, x0), lo0 = M0 * x0;
  uint32_t hi1 = __umulhi(M1, x2), lo1 = M1 * x2;
  uint32_t y0 = hi1 ^ x1 ^ k0, y1 = lo1, y2 = hi0 ^ x3 ^ k1, y3 = lo0;
  x0 = y0; x1 = y1; x2 = y2; x3 = y3;
}

__device__ void philox4x32_10(uint32_t ctr[4], uint32_t k0, uint32_t k1) {
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
  for (int i = 0; i < 10; ++i) {
    philox_round(ctr[0], ctr[1], ctr[2], ctr[3], k0, k1);
    k0 += W0;
    k1 += W1;
  }
}

// U0[a, k] ~ N(0, 1/m) for k < r, 0 in the padding.  Element e = a*r + k draws
// from counter (e/2, 0, 0, 0): two uniforms (words 0, 1) -> Box-Muller pair.
__global__ void k_philox_u0(float* U, int64_t m, int r, int R, uint64_t seed) {
  int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= m * R) return;
  int64_t a = idx / R;
  int k = (int)(idx % R);
  if (k >= r) { U[idx] = 0.f; return; }
  int64_t e = a * r + k;
  uint32_t c[4] = {(uint32_t)(e >> 1), (uint32_t)((uint64_t)e >> 33), 0u, 0u};
  philox4x32_10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
  float u1 = ((float)c[0] + 0.5f) * 2.3283064365386963e-10f;
  float u2 = ((float)c[1] + 0.5f) * 2.3283064365386963e-10f;
  float rad = sqrtf(-2.0f * logf(u1));
  float z = (e & 1) ? rad * sinf(6.283185307179586f * u2) : rad * cosf(6.283185307179586f * u2);
  U[idx] = z * rsqrtf((float)m);
}

// A reloaded M that failed its NaN/Inf check ends the solve before any step
// reads it: status DCF_ENONFINITE, and the stop flag every kernel tests.
__global__ void k_apply_mflag(const int* flag, DevState* st) {
  if (*flag) {
    st->status = 4;   // DCF_ENONFINITE
    st->stop = 1;
  }
}

__global__ void k_check_finite(const float* x, int64_t count, int* flag) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (; i < count; i += stride)
    if (!isfinite(x[i])) { atomicExch(flag, 1); return; }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
int pick_R(int r) { return r <= 8 ? 8 : r <= 16 ? 16 : r <= 32 ? 32 : 64; }

static size_t gram_smem(int cx, int cy) { return (size_t)kGramChunk * (cx + cy) * sizeof(float); }

cudaError_t launch_gram(const float* X, int ldx, int cx, const float* Y, int ldy, int cy,
                        int64_t N, float2* part, int nparts, const DevState* st,
                        int respect_stop, cudaStream_t s) {
  const int64_t rows_per = (N + nparts - 1) / nparts;
  const size_t smem = gram_smem(cx, cy);
  const int ns = (cx * cy + 255) / 256;
  if (ns <= 1)
    k_gram_part<1><<<nparts, 256, smem, s>>>(X, ldx, cx, Y, ldy, cy, N, rows_per, part, st,
                                             respect_stop);
  else if (ns <= 4)
    k_gram_part<4><<<nparts, 256, smem, s>>>(X, ldx, cx, Y, ldy, cy, N, rows_per, part, st,
                                             respect_stop);
  else
    k_gram_part<16><<<nparts, 256, smem, s>>>(X, ldx, cx, Y, ldy, cy, N, rows_per, part, st,
                                              respect_stop);
  return cudaGetLastError();
}

template <int R>
static cudaError_t gram_vv_T(const float* Vo, const float* Vn, int64_t N, float2* pq,
                             float2* pxv, float2* pdv, int nparts, const DevState* st,
                             cudaStream_t s) {
  const int64_t rows_per = (N + nparts - 1) / nparts;
  k_gram_vv<R><<<nparts, 256, GvvCfg<R>::smem_bytes, s>>>(Vo, Vn, N, rows_per, pq, pxv, pdv, st);
  return cudaGetLastError();
}

cudaError_t launch_gram_vv(int R, const float* Vo, const float* Vn, int64_t N, float2* part_q,
                           float2* part_xv, float2* part_dv, int nparts, const DevState* st,
                           cudaStream_t s) {
  switch (R) {
    case 8: return gram_vv_T<8>(Vo, Vn, N, part_q, part_xv, part_dv, nparts, st, s);
    case 16: return gram_vv_T<16>(Vo, Vn, N, part_q, part_xv, part_dv, nparts, st, s);
    case 32: return gram_vv_T<32>(Vo, Vn, N, part_q, part_xv, part_dv, nparts, st, s);
    default: return gram_vv_T<64>(Vo, Vn, N, part_q, part_xv, part_dv, nparts, st, s);
  }
}

// Batched launchers.  kind: 0 make_w, 1 rows, 2 gram (mode), 3 reduce (tail)
template <int R>
static cudaError_t bsmall_T(int kind, const BInst* insts, const BItem* items, int nitems,
                            const int* which, int grid, int cur, int arg, cudaStream_t s) {
  if (nitems == 0) return cudaSuccess;
  switch (kind) {
    case 0: k_bmake_w<R><<<grid, 256, 0, s>>>(insts, items, nitems, cur, arg); break;
    case 1: k_brows<R><<<grid, 256, 0, s>>>(insts, items, nitems, cur); break;
    case 2: k_bgram<R><<<grid, 256, GvvCfg<R>::smem_bytes, s>>>(insts, items, nitems, cur, arg); break;
    default:
      k_breduce<R><<<nitems, 256, tail_smem(R), s>>>(insts, which, cur, arg);
      break;
  }
  return cudaGetLastError();
}

cudaError_t launch_bsmall(int R, int kind, const BInst* insts, const BItem* items, int nitems,
                          const int* which, int grid, int cur, int arg, cudaStream_t s) {
  switch (R) {
    case 8: return bsmall_T<8>(kind, insts, items, nitems, which, grid, cur, arg, s);
    case 16: return bsmall_T<16>(kind, insts, items, nitems, which, grid, cur, arg, s);
    default: return bsmall_T<32>(kind, insts, items, nitems, which, grid, cur, arg, s);
  }
}

static cudaError_t launch_reduce(const ReduceArgs& ra, cudaStream_t s) {
  int grid = (ra.total + kRedEntriesPerCta - 1) / kRedEntriesPerCta;
  size_t smem = tail_smem(ra.R);
  k_reduce_parts<<<grid, 256, smem, s>>>(ra);
  return cudaGetLastError();
}

template <int R>
static cudaError_t make_w_T(const IterArgs& a, int copy, int respect_stop, cudaStream_t s) {
  int64_t blocks = (a.m + kRowsPerCta - 1) / kRowsPerCta;
  k_make_w<R><<<(unsigned)blocks, 256, 0, s>>>(a.U[copy], a.st, a.sm, a.W, a.m, respect_stop);
  return cudaGetLastError();
}

cudaError_t launch_make_w(const IterArgs& a, int copy, int respect_stop, cudaStream_t s) {
  switch (a.R) {
    case 8: return make_w_T<8>(a, copy, respect_stop, s);
    case 16: return make_w_T<16>(a, copy, respect_stop, s);
    case 32: return make_w_T<32>(a, copy, respect_stop, s);
    default: return make_w_T<64>(a, copy, respect_stop, s);
  }
}

// The reduction tail needs tail_smem(R) bytes of dynamic shared memory (64 KB at R = 64).
cudaError_t prepare_small_kernels() {
  return cudaFuncSetAttribute(k_reduce_parts, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)tail_smem(kMaxR));
}

template <int R>
static cudaError_t rows_T(const IterArgs& a, cudaStream_t s) {
  k_rows<R><<<a.n_rblocks, 256, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_rows(const IterArgs& a, cudaStream_t s) {
  switch (a.R) {
    case 8: return rows_T<8>(a, s);
    case 16: return rows_T<16>(a, s);
    case 32: return rows_T<32>(a, s);
    default: return rows_T<64>(a, s);
  }
}

cudaError_t launch_avg_rows(const IterArgs& a, const float* const* Ui, int E, int ldc,
                            cudaStream_t s) {
  if (ldc < a.R) return cudaErrorInvalidValue;
  switch (a.R) {
    case 8: k_avg_rows<8><<<a.n_rblocks, 256, 0, s>>>(a, Ui, E, ldc); break;
    case 16: k_avg_rows<16><<<a.n_rblocks, 256, 0, s>>>(a, Ui, E, ldc); break;
    case 32: k_avg_rows<32><<<a.n_rblocks, 256, 0, s>>>(a, Ui, E, ldc); break;
    default: k_avg_rows<64><<<a.n_rblocks, 256, 0, s>>>(a, Ui, E, ldc); break;
  }
  return cudaGetLastError();
}

// reduction of V-side partials (Q_t, V_{t-1}^T V_t, Huber) + Cholesky(Q_t + rho I)
cudaError_t launch_reduce_q(const IterArgs& a, double* out_q, double* out_xv, double* out_dv,
                            double* out_h, int nparts_gram, unsigned int* counter,
                            cudaStream_t s) {
  ReduceArgs ra{};
  const int RR = a.R * a.R;
  ra.part[0] = a.part_q; ra.count[0] = RR; ra.out[0] = out_q; ra.nparts[0] = nparts_gram;
  ra.part[1] = a.part_xv; ra.count[1] = RR; ra.out[1] = out_xv; ra.nparts[1] = nparts_gram;
  ra.part[2] = a.part_dv; ra.count[2] = RR; ra.out[2] = out_dv; ra.nparts[2] = nparts_gram;
  ra.hpart = a.part_h; ra.count[3] = 1; ra.out[3] = out_h; ra.nparts[3] = a.n_vblocks;
  ra.total = 3 * RR + 1;
  ra.tail = TAIL_Q;
  ra.copy = a.cur;
  ra.R = a.R; ra.r = a.r; ra.rho = a.rho; ra.rho_q = a.rho_q; ra.u_mode = a.u_mode;
  ra.counter = counter; ra.sm = a.sm; ra.st = a.st;
  return launch_reduce(ra, s);
}

cudaError_t launch_reduce_g(const IterArgs& a, double* out_g, double* out_xu, double* out_du,
                            unsigned int* counter, cudaStream_t s) {
  ReduceArgs ra{};
  const int RR = a.R * a.R;
  ra.part[0] = a.part_g; ra.count[0] = RR; ra.out[0] = out_g; ra.nparts[0] = a.n_rblocks;
  ra.part[1] = a.part_xu; ra.count[1] = RR; ra.out[1] = out_xu; ra.nparts[1] = a.n_rblocks;
  ra.part[2] = a.part_du; ra.count[2] = RR; ra.out[2] = out_du; ra.nparts[2] = a.n_rblocks;
  ra.total = 3 * RR;
  ra.tail = TAIL_G;
  ra.copy = a.cur;
  ra.R = a.R; ra.r = a.r; ra.rho = a.rho; ra.u_mode = a.u_mode;
  ra.counter = counter; ra.sm = a.sm; ra.st = a.st;
  return launch_reduce(ra, s);
}

cudaError_t launch_reduce_init(const IterArgs& a, int which /*0: G, 1: Q*/, int copy,
                               const float2* part, int nparts, double* out,
                               unsigned int* counter, cudaStream_t s) {
  ReduceArgs ra{};
  const int RR = a.R * a.R;
  ra.part[0] = part; ra.count[0] = RR; ra.out[0] = out; ra.nparts[0] = nparts;
  ra.total = RR;
  ra.tail = which == 0 ? TAIL_INIT_G : TAIL_INIT_Q;
  ra.R = a.R; ra.r = a.r; ra.rho = a.rho; ra.u_mode = a.u_mode; ra.copy = copy;
  ra.counter = counter; ra.sm = a.sm; ra.st = a.st;
  return launch_reduce(ra, s);
}

// FP64 sums of the partials of several Gram jobs: the summation of
// k_reduce_parts (16 entries per CTA, 16 lanes per entry, each lane's
// partials in order, then the lanes in order), without a tail.
__global__ void __launch_bounds__(256) k_reduce_jobs(GramJobs g) {
  __shared__ float2 red2[256];
  const int tid = threadIdx.x;
  const int e_local = tid % kRedEntriesPerCta;
  const int lane_p = tid / kRedEntriesPerCta;
  constexpr int nsplit = 256 / kRedEntriesPerCta;
  int idx = blockIdx.x * kRedEntriesPerCta + e_local;
  int which = -1;
  for (int q = 0; q < g.n; ++q) {
    const int c = g.j[q].cx * g.j[q].cy;
    if (idx < c) {
      which = q;
      break;
    }
    idx -= c;
  }
  float hi = 0.f, lo = 0.f;
  if (which >= 0) {
    const float2* p = g.j[which].part;
    const int cnt = g.j[which].cx * g.j[which].cy;
    const int np = g.j[which].nparts;
    for (int q0 = lane_p; q0 < np; q0 += 8 * nsplit) {
      float2 v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int q = q0 + u * nsplit;
        v[u] = q < np ? p[(int64_t)q * cnt + idx] : make_float2(0.f, 0.f);
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        two_sum_add(hi, lo, v[u].x);
        lo += v[u].y;
      }
    }
  }
  red2[tid] = make_float2(hi, lo);
  __syncthreads();
  if (lane_p == 0 && which >= 0) {
    float th = 0.f, tl = 0.f;
    for (int q = 0; q < nsplit; ++q) {
      const float2 v = red2[q * kRedEntriesPerCta + e_local];
      two_sum_add(th, tl, v.x);
      tl += v.y;
    }
    g.j[which].out[idx] = (double)th + (double)tl;
  }
}

cudaError_t launch_gram_jobs(const GramJobs& g, cudaStream_t s) {
  if (g.n <= 0 || g.n > kMaxGramJobs) return g.n == 0 ? cudaSuccess : cudaErrorInvalidValue;
  int maxp = 0, maxe = 0, total = 0;
  size_t smem = 0;
  for (int q = 0; q < g.n; ++q) {
    const GramJob& j = g.j[q];
    if (j.cx < 1 || j.cy < 1 || j.cx > kMaxR || j.cy > kMaxR || j.nparts < 1)
      return cudaErrorInvalidValue;
    maxp = j.nparts > maxp ? j.nparts : maxp;
    maxe = j.cx * j.cy > maxe ? j.cx * j.cy : maxe;
    total += j.cx * j.cy;
    smem = gram_smem(j.cx, j.cy) > smem ? gram_smem(j.cx, j.cy) : smem;
  }
  const dim3 grid((unsigned)maxp, (unsigned)g.n);
  const int ns = (maxe + 255) / 256;
  if (ns <= 1) k_gram_jobs<1><<<grid, 256, smem, s>>>(g);
  else if (ns <= 4) k_gram_jobs<4><<<grid, 256, smem, s>>>(g);
  else k_gram_jobs<16><<<grid, 256, smem, s>>>(g);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_reduce_jobs<<<(total + kRedEntriesPerCta - 1) / kRedEntriesPerCta, 256, 0, s>>>(g);
  return cudaGetLastError();
}

cudaError_t launch_reduce_plain(const float2* part, int nparts, int count, double* out,
                                cudaStream_t s) {
  ReduceArgs ra{};
  ra.part[0] = part; ra.count[0] = count; ra.out[0] = out; ra.nparts[0] = nparts;
  ra.total = count;
  ra.tail = TAIL_NONE;
  ra.R = 1;
  return launch_reduce(ra, s);
}

cudaError_t launch_philox_u0(float* U, int64_t m, int r, int R, uint64_t seed, cudaStream_t s) {
  int64_t tot = m * R;
  k_philox_u0<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(U, m, r, R, seed);
  return cudaGetLastError();
}

cudaError_t launch_apply_mflag(const int* flag, DevState* st, cudaStream_t s) {
  k_apply_mflag<<<1, 1, 0, s>>>(flag, st);
  return cudaGetLastError();
}

cudaError_t launch_check_finite(const float* x, int64_t count, int* flag, cudaStream_t s) {
  int64_t blocks = (count + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  if (blocks < 1) blocks = 1;
  k_check_finite<<<(unsigned)blocks, 256, 0, s>>>(x, count, flag);
  return cudaGetLastError();
}

}  // namespace dcf
