// Internal declarations shared by the library's translation units.
//
// Device layout: rows of A (constraints) and of A^T (variables) are stored in
// "bin order" -- grouped by row length so that each group is processed by a
// matching number of lanes -- and every vector lives in that permuted order.
// The host maps to and from the caller's order only when copying in and out.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>

#include <nvtx3/nvToolsExt.h>

#include "layout_types.h"

namespace lpop {

// A named NVTX range for the lifetime of the object (the library's phases
// show up in profilers; costs nothing measurable when no tool listens).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

template <class V>
struct CsrT {
  const int* rp;  // [rows+1]
  const int* ci;  // [nnz]
  const V* v;     // [nnz]
};
using Csr = CsrT<double>;

// The per-iteration vectors and matrix values of one precision.  The FP64 set
// always exists; the FP32 set only in mixed precision.  All in bin order.
template <class V>
struct Vecs {
  V *Av, *Atv;  // values of A and A^T (same structure as the int arrays of Dev)
  V *b, *c, *l, *u;
  V *x[2], *y[2], *ax[2], *xbar[2], *ybar[2];
  V *T, *invT, *S, *invS, *GT, *GS, *q, *p;
  V *x_last, *y_last, *ax_avg;
};

// Options fixed for the life of a problem; passed by value to kernels.
struct Params {
  int m, n;
  int mode;
  int sched;
  int phi;
  int normalize;
  int restart;
  int check_every;
  double alpha;
  double floor;
  double b_norm;  // ||b||_2, user units
  double c_norm;  // ||c||_2, user units
  double refine_tol;  // mixed precision: FP32 -> FP64 hand-over threshold
  int refine_stall;   // ... or after this many checks without a 10% KKT gain
};

// Device-resident solver state.  Written only by single-thread control code
// (the last block of a reduction kernel) and by the host between launches.
struct DevState {
  int cur;        // which half of the double buffers holds the current iterate
  int status;     // 0 running, 1 optimal, 4 numerical error
  long long k;    // accepted steps
  int k_mod;      // k mod phi (kept with k: no 64-bit division in the step control)
  long long attempts;
  double eta;
  double omega;
  double inv_omega;  // 1 / omega, set wherever omega is
  double wsum;    // sum of eta over accepted steps since the last restart
  double tol;
  // pending online update, applied by the next primal / dual kernel
  int pend_p;
  int pend_d;
  double up_scale_p;  // q_j -> grad_j factor: -(eta/omega) [/ ||g||^2]
  double up_scale_d;  // p_i -> grad_i factor: -(eta omega) [/ ||b - A x||^2]
  double gp_norm;     // scalar AdaGrad accumulators
  double gd_norm;
  // restart bookkeeping
  double klast_p2, klast_d2, klast_g2;
  double k_prev;
  long long last_restart_attempt;
  long long restarts;
  int checked0;
  int restart_action;  // set by the check: 0 none, 1 restart at current, 2 restart at average
  int adopt_avg;       // the check found the average optimal: copy it into the current
  double apply_w;      // average weight used by the apply step (restart / adoption at the average)
  // statistics of the last check
  double pobj, dobj, rel_pres, rel_dres, rel_gap;
  int stats_from_avg;
  // last attempt (debug)
  int last_accept;
  double last_eta_max;
  // grid handshake counter for last-block reductions
  unsigned int counter;
  // derived scalars, refreshed whenever eta, omega, k or the AdaGrad-norm sums change
  int collect;        // the next attempt records q / p (k mod phi == 0)
  double step_p;      // eta / omega
  double step_d;      // eta * omega
  double sqrt_gp;     // sqrt of gp_norm (0 when it is 0)
  double sqrt_gd;
  // device-side solve loop (batched kernel)
  int initial_checked;  // the check before the first attempt has run
  int phase32;          // mixed precision: still in the FP32 phase
  int stall;            // checks since the relative KKT error last dropped by 10%
  double best_kkt;
};

// +1 or -1 for index j from the top bit of SplitMix64 (Steele, Lea and Flood,
// OOPSLA 2014) seeded so that output j is the generator's (j+1)-th: the
// second start direction of the power iteration when the all-ones direction
// lies in the null space of A.
__host__ __device__ inline double splitmix_sign(unsigned long long j) {
  unsigned long long z = (j + 1ULL) * 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  z ^= z >> 31;
  return (z >> 63) ? -1.0 : 1.0;
}

// Entries of the step-size schedule table (attempt counts below this use the table).
constexpr int kStepTab = 1 << 20;

// Refresh the derived scalars of a state (host and device).  Runs once per
// attempt in a single thread, where every FP64 division and square root is
// a long dependent chain on GB300: 1/omega is kept with omega, and the
// square roots are taken only for the scheduler that uses them.
__host__ __device__ inline void refresh_derived(DevState& s, int phi, int sched) {
  s.collect = phi > 0 && s.k_mod == 0;
  s.step_p = s.eta * s.inv_omega;
  s.step_d = s.eta * s.omega;
  const bool norm = sched == kAdagradNorm;
  s.sqrt_gp = norm && s.gp_norm > 0.0 ? sqrt(s.gp_norm) : 0.0;
  s.sqrt_gd = norm && s.gd_norm > 0.0 ? sqrt(s.gd_norm) : 0.0;
}

// Factors of the next-step-size rule for attempt t: 1 - (t+1)^-0.3 and
// 1 + (t+1)^-0.6 (tabulated below kStepTab).
__device__ inline void step_factors(const double* step_tab, long long t, double* f1, double* f2) {
  if (t < kStepTab) {
    *f1 = __ldg(step_tab + t);
    *f2 = __ldg(step_tab + kStepTab + t);
  } else {
    *f1 = 1.0 - pow((double)t + 1.0, -0.3);
    *f2 = 1.0 + pow((double)t + 1.0, -0.6);
  }
}

// All device buffers of one problem.
struct Dev {
  int m, n;
  long long nnz;
  Csr A;    // m rows, FP64 values
  Csr At;   // n rows, FP64 values
  int *A_rp, *A_ci, *At_rp, *At_ci;
  double *A_v, *At_v;  // == f64.Av, f64.Atv
  double *dr, *dc;     // A~ = diag(dr) A diag(dc)
  double *inv_dr, *inv_dc;  // 1 / dr, 1 / dc (the KKT checks' user-unit residuals)
  uint8_t* sense;
  Vecs<double> f64;
  Vecs<float> f32;    // null pointers unless mixed precision
  // partial sums of the A^T-row kernels, records of kMaxPartials doubles:
  // [gridAt] one per block, then [binsAt.seg_rows] one per segmented row;
  // partials2 the same for the A-row kernels
  double* partials;
  double* partials2;
  double* work;       // small scratch for setup reductions
  double* work2;      // [max(m, n)] FP64 staging of FP32 vectors read by the host
  const double* step_tab;  // [2 * kStepTab]: 1 - (t+1)^-0.3 and 1 + (t+1)^-0.6 for t < kStepTab
  DevState* st;
  unsigned int* bad_gathers;  // checked builds: gathers whose index fell outside the vector
  BinTable binsA, binsAt;
  int gridA, gridAt;      // blocks launched for the A / A^T row kernels (FP64)
  int gridA32, gridAt32;  // the same for the FP32 kernels (fewer registers, more resident blocks)
  int max_grid;
};

// Grids of the row kernels of precision V.
template <class V>
__host__ __device__ inline int grid_at(const Dev& d) { return sizeof(V) == 4 ? d.gridAt32 : d.gridAt; }
template <class V>
__host__ __device__ inline int grid_a(const Dev& d) { return sizeof(V) == 4 ? d.gridA32 : d.gridA; }

// Slots of the segmented rows within a partials array (after the block
// records of the precision-V kernels); records to sum.
template <class V>
__host__ __device__ inline double* row_slots_at(const Dev& d, double* part) {
  return part + (size_t)grid_at<V>(d) * kMaxPartials;
}
template <class V>
__host__ __device__ inline double* row_slots_a(const Dev& d, double* part) {
  return part + (size_t)grid_a<V>(d) * kMaxPartials;
}
template <class V>
__host__ __device__ inline int partial_rows_at(const Dev& d) { return grid_at<V>(d) + d.binsAt.seg_rows; }
template <class V>
__host__ __device__ inline int partial_rows_a(const Dev& d) { return grid_a<V>(d) + d.binsA.seg_rows; }

template <class V>
__host__ __device__ inline const Vecs<V>& vecs(const Dev& d);
template <>
__host__ __device__ inline const Vecs<double>& vecs<double>(const Dev& d) { return d.f64; }
template <>
__host__ __device__ inline const Vecs<float>& vecs<float>(const Dev& d) { return d.f32; }

template <class V>
__host__ __device__ inline CsrT<V> csr_a(const Dev& d) { return CsrT<V>{d.A_rp, d.A_ci, vecs<V>(d).Av}; }
template <class V>
__host__ __device__ inline CsrT<V> csr_at(const Dev& d) { return CsrT<V>{d.At_rp, d.At_ci, vecs<V>(d).Atv}; }

// ---------------------------------------------------------------------------
// Block reductions (fixed shuffle tree then fixed smem order: deterministic)
// ---------------------------------------------------------------------------
template <int N, class T>
__device__ inline void block_sum(T (&v)[N], T* smem /* [32 * N] */) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < N; ++q) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v[q] += __shfl_xor_sync(0xffffffffu, v[q], off);
  }
  __syncthreads();
  if (lane == 0) {
#pragma unroll
    for (int q = 0; q < N; ++q) smem[warp * N + q] = v[q];
  }
  __syncthreads();
  const int nw = blockDim.x >> 5;
  if (warp == 0) {
#pragma unroll
    for (int q = 0; q < N; ++q) {
      T t = lane < nw ? smem[lane * N + q] : T(0);
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
      v[q] = t;  // valid in warp 0
    }
  }
  __syncthreads();
}

// Block sum through shared memory: every thread stores its N values, then one
// warp adds them (8 per lane as a pairwise tree, then a shuffle tree).  Far fewer FP64
// instructions than a shuffle tree in every warp.  Result valid in thread 0.
// smem must hold N * blockDim.x doubles; blockDim.x must be 256.
template <int N>
__device__ inline void block_sum_smem(double (&v)[N], double* smem) {
  const int tid = threadIdx.x;
#pragma unroll
  for (int q = 0; q < N; ++q) smem[q * 256 + tid] = v[q];
  __syncthreads();
  if (tid < 32) {
#pragma unroll
    for (int q = 0; q < N; ++q) {
      double a[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) a[k] = smem[q * 256 + tid + 32 * k];
      // pairwise (depth 3, the same 7 adds as a chain)
      double t = ((a[0] + a[1]) + (a[2] + a[3])) + ((a[4] + a[5]) + (a[6] + a[7]));
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
      v[q] = t;
    }
  }
  __syncthreads();
}

// Order-preserving integer key of a double (not NaN): comparisons of keys
// agree with floating-point comparisons, and -0.0 and +0.0 get the same key.
// Lets clamps and sign tests run on the integer pipes instead of the FP64 pipe.
__device__ __forceinline__ long long ord_key(double v) {
  const long long b = __double_as_longlong(v);
  const long long mag = b & 0x7fffffffffffffffLL;
  return b < 0 ? -mag : mag;
}

__device__ __forceinline__ int ord_key(float v) {
  const int b = __float_as_int(v);
  const int mag = b & 0x7fffffff;
  return b < 0 ? -mag : mag;
}

// min(max(v, lo), hi) for lo <= hi, on the integer pipes.
template <class V, class K>
__device__ __forceinline__ V clamp_keys(V v, K kv, V lo, K kl, V hi, K kh) {
  V r = kv < kl ? lo : v;
  return kv > kh ? hi : r;
}

// Reductions across blocks.  Every block of a row kernel stores one record
// of its partial sums.  The records of an A^T-row kernel are folded into the
// records of the A-row kernel that follows it: block b of that kernel copies
// records b, b + grid, ... (at most kFold) into shared memory while it works
// (cp.async, no registers held) and adds them, in that order, to its own
// record.  The last block of the A-row kernel then sums all records with the
// whole block.  Every sum has a fixed order, so results do not depend on
// which block finishes when.
constexpr int kFold = 8;

__device__ __forceinline__ void cp_async8(double* dst, const double* src) {
  const unsigned int sa = (unsigned int)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(sa), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Start copying this block's share of `count` records (N fields each) into
// fold[kFold * N]; returns how many records it is.  Before reading fold:
// cp_async_wait_all() in every thread, then a barrier.
template <int N>
__device__ inline int fold_begin(const double* rec, int count, double* fold) {
  const int b = (int)blockIdx.x, g = (int)gridDim.x;
  const int k = b < count ? min(kFold, (count - 1 - b) / g + 1) : 0;
  for (int t = (int)threadIdx.x; t < k * N; t += (int)blockDim.x) {
    const int r = t / N, q = t - r * N;
    cp_async8(fold + t, rec + (size_t)(b + r * g) * kMaxPartials + q);
  }
  return k;
}

// Records not folded by a grid of `grid` blocks: [kFold * grid, count).
__host__ __device__ inline int unfolded_first(int grid) { return kFold * grid; }

// Store this block's record (thread 0 holds v); returns true, in every
// thread, in the last block to finish.  The ticket is a release-acquire
// atomic at GPU scope: it orders each block's record store before its
// ticket, and the last block's acquire -- extended to its other threads by
// the barrier -- makes every record visible, with no separate fences.
template <int N>
__device__ inline bool publish_last(const double (&v)[N], double* part, unsigned int* counter, int* s_flag) {
  if (threadIdx.x == 0) {
#pragma unroll
    for (int q = 0; q < N; ++q) part[(size_t)blockIdx.x * kMaxPartials + q] = v[q];
    unsigned int t;
    asm volatile("atom.add.acq_rel.gpu.u32 %0, [%1], 1;" : "=r"(t) : "l"(counter) : "memory");
    *s_flag = t == gridDim.x - 1;
  }
  __syncthreads();
  return *s_flag != 0;
}

// v[0] <- v[0] + ... + v[n-1] (1 <= n <= M) as a pairwise tree in a fixed
// order.  On GB300 a dependent FP64 add takes ~64 cycles, so a sum that one
// thread forms on the critical path is kept log2(n) deep instead of n.
template <int M>
__device__ __forceinline__ double tree_sum(double (&v)[M], int n) {
#pragma unroll
  for (int w = 1; w < M; w <<= 1) {
#pragma unroll
    for (int i = 0; i + w < M; i += 2 * w)
      if (i + w < n) v[i] += v[i + w];
  }
  return v[0];
}

// Field-wise totals of records [0, count) of rec (fields 0..N-1) plus records
// [0, count2) of rec2 (their fields 0..N2-1 added to fields q2..q2+N2-1),
// with the whole block and in a fixed order; the totals end up in thread 0.
// GB300 runs FP64 at 2 lanes per SM per cycle with ~64 cycles per dependent
// add, so the sum is laid out for full lanes and shallow trees: thread t
// loads field t % N of up to 8 records (one L2 round trip) and adds them as
// a tree; warp 0 then adds each field's slices (32 / N lanes per field, a
// tree each) and the lanes' results (a tree).  blockDim.x must be kBlock;
// smem must hold kBlock + 32 doubles.
template <int N, int N2>
__device__ inline void block_sum_records(const double* rec, int count, const double* rec2, int count2, int q2,
                                         double (&out)[N], double* smem) {
  static_assert(N <= 32 && N2 <= N, "record layout");
  constexpr int S = kBlock / N;              // slices
  constexpr int P = 32 / N;                  // lanes of warp 0 per field
  constexpr int MX = (S + P - 1) / P;        // slices per lane
  const int t = (int)threadIdx.x;
  const int q = t % N, sl = t / N;
  double acc = 0.0;
  if (sl < S) {
    for (int r0 = sl; r0 < count; r0 += 8 * S) {
      double v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int r = r0 + u * S;
        v[u] = r < count ? __ldcg(rec + (size_t)r * kMaxPartials + q) : 0.0;
      }
      // records in this batch: the warp's largest count (the extra terms are zeros)
      const int nv = min(8, (count - 1 - r0) / S + 1);
      acc += tree_sum(v, __reduce_max_sync(__activemask(), nv));
    }
    if (q >= q2 && q < q2 + N2) {
      for (int r = sl; r < count2; r += S) acc += __ldcg(rec2 + (size_t)r * kMaxPartials + (q - q2));
    }
  }
  smem[t] = acc;
  __syncthreads();
  if (t < 32) {
    double part = 0.0;
    if (t < N * P) {
      const int fq = t % N, fp = t / N;
      double v[MX];
#pragma unroll
      for (int u = 0; u < MX; ++u) {
        const int x = fp + u * P;
        v[u] = x < S ? smem[x * N + fq] : 0.0;
      }
      part = tree_sum(v, MX);
    }
    smem[kBlock + t] = part;
    __syncwarp();
    if (t < N) {
      double v[P];
#pragma unroll
      for (int x = 0; x < P; ++x) v[x] = smem[kBlock + x * N + t];
      smem[t] = tree_sum(v, P);  // slice values are no longer needed
    }
    __syncwarp();
    if (t == 0) {
#pragma unroll
      for (int f = 0; f < N; ++f) out[f] = smem[f];
    }
  }
}

// Programmatic dependent launch of the kernels of a check period.  Each
// starts with pdl_wait() (its predecessor has completed and its writes are
// visible) and calls pdl_trigger() only once the rest of its grid is done:
// at the end of a block for the primal kernels, in the last block only --
// before its reduction and control -- for the dual kernels.  The successor's
// blocks then become resident while that single block finishes, not while
// the whole grid still runs (letting them in earlier, at kernel start, made
// graph replay slower).
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <class... KArgs, class... Args>
inline void launch_pdl(void (*kernel)(KArgs...), int grid, cudaStream_t s, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid, 1, 1);
  cfg.blockDim = dim3(kBlock, 1, 1);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, kernel, args...);  // errors surface through cudaGetLastError
}

// ---------------------------------------------------------------------------
// Launchers (defined in the .cu files)
// ---------------------------------------------------------------------------
// one step attempt = primal kernel + dual kernel (the dual kernel's last block runs the step control)
// fp32 selects the FP32 vector set (mixed precision); reductions and scalars stay FP64
void launch_primal(const Dev& d, const Params& prm, bool fp32, cudaStream_t s);
void launch_dual(const Dev& d, const Params& prm, bool fp32, cudaStream_t s);
// KKT check: primal-side reductions, dual-side reductions + decision, apply
void launch_check(const Dev& d, const Params& prm, int eval_only, bool fp32, cudaStream_t s);
// apply a pending preconditioner update now (debug reads)
void launch_flush_update(const Dev& d, const Params& prm, bool fp32, cudaStream_t s);
// recompute 1/T and 1/Sigma after T / Sigma were written from outside
void launch_inverse_preconditioners(const Dev& d, bool fp32, cudaStream_t s);
// mixed precision: FP32 copies of the problem data and the initial FP32 state
void launch_make_fp32(const Dev& d, cudaStream_t s);
// the sliced copy (column indices and values, `total` entries) of the kSell
// bins of bt from the permuted CSR arrays rp, ci, v
void launch_fill_sliced(const BinTable& bt, const int* rp, const int* ci, const double* v, int* sell_ci,
                        double* sell_v, long long total, cudaStream_t s);
// out[i] = (float)in[i]
void launch_narrow(const double* in, float* out, long long n, cudaStream_t s);
// FP32 iterate -> FP64 iterate (refinement phase); FP64 -> FP32 (state import)
void launch_promote_state(const Dev& d, cudaStream_t s);
void launch_demote_state(const Dev& d, cudaStream_t s);
// out[i] = (double) in[i] (reading FP32 vectors for the host)
void launch_widen(double* out, const float* in, int n, cudaStream_t s);
int check_kernel_count();

// setup
void launch_fill(double* v, double val, long long n, cudaStream_t s);
// Ruiz-style rounds on both CSR copies (rows of A and of A^T in bin order,
// longest first; rows from split on have at most 32 entries):
//   norms: fr = row infinity norms of A, fc = those of A^T (columns of A);
//   apply: f <- f > 0 ? 1/sqrt(f) : 1 for fr and fc, dr *= fr, dc *= fc, and
//          every entry a_ij <- (a_ij fr_i) fc_j in both copies.
// How the Ruiz kernels cut the rows of one matrix: rows [0, nlong) (the
// whole-block rows) in chunks of kRuizChunk entries, one warp each
// (chunk_pre: device prefix of their chunk counts, nlong + 1 entries, nchunks
// in all), rows [nlong, split) a warp each, rows [split, rows) (at most 32
// entries) a thread each.
constexpr int kRuizChunk = 1024;
struct RuizSplit {
  int split;
  int nlong;
  int nchunks;
  const int* chunk_pre;
};
void launch_ruiz_norms(const Dev& d, const RuizSplit& a, const RuizSplit& at, double* fr, double* fc, cudaStream_t s);
void launch_ruiz_apply(const Dev& d, const RuizSplit& a, const RuizSplit& at, double* fr, double* fc, cudaStream_t s);
// out[r] = sum over row r of |a|^beta (optionally its square root); rows [0, nlong) are the whole-block
// rows, rows [split, rows) those of at most 32 entries
void launch_row_powsum(const Csr& M, int rows, int nlong, int split, double beta, int square_root, double* out,
                       cudaStream_t s);
void launch_scale_problem_vectors(const Dev& d, cudaStream_t s);
void launch_init_vectors(const Dev& d, cudaStream_t s);
void launch_spmv_binned(const Csr& M, const BinTable& bt, int grid, const double* x, double* y, cudaStream_t s);
void launch_norm2(const double* v, int n, double* out, cudaStream_t s);  // out[0] = ||v||_2; out[1..1025) scratch
void launch_absmax(const double* v, long long n, double* out, cudaStream_t s);
void launch_scale_by_inv(double* v, int n, const double* denom, cudaStream_t s);  // v /= denom[0]

}  // namespace lpop
