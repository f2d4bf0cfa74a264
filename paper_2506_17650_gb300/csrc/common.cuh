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

#include "layout_types.h"

namespace lpop {

struct Csr {
  const int* rp;     // [rows+1]
  const int* ci;     // [nnz]
  const double* v;   // [nnz]
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
};

// Device-resident solver state.  Written only by single-thread control code
// (the last block of a reduction kernel) and by the host between launches.
struct DevState {
  int cur;        // which half of the double buffers holds the current iterate
  int status;     // 0 running, 1 optimal, 4 numerical error
  long long k;    // accepted steps
  long long attempts;
  double eta;
  double omega;
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
};

// All device buffers of one problem.
struct Dev {
  int m, n;
  Csr A;    // m rows
  Csr At;   // n rows
  int *A_rp, *A_ci, *At_rp, *At_ci;
  double *A_v, *At_v;
  double *b, *c, *l, *u, *dr, *dc;  // preprocessed data, bin order
  uint8_t* sense;
  double *x[2], *y[2], *ax[2], *xbar[2], *ybar[2];
  double *T, *S, *GT, *GS, *q, *p;
  double *x_last, *y_last, *ax_avg;
  double* partials;   // [max_grid * kMaxPartials] written by primal/check-primal kernels
  double* partials2;  // same, written by dual/check-dual kernels
  double* work;       // small scratch for setup reductions
  DevState* st;
  BinTable binsA, binsAt;
  int gridA, gridAt;  // blocks launched for the A / A^T row kernels
  int max_grid;
};

// ---------------------------------------------------------------------------
// Block reductions (fixed shuffle tree then fixed smem order: deterministic)
// ---------------------------------------------------------------------------
template <int N>
__device__ inline void block_sum(double (&v)[N], double* smem /* [32 * N] */) {
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
      double t = lane < nw ? smem[lane * N + q] : 0.0;
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
      v[q] = t;  // valid in warp 0
    }
  }
  __syncthreads();
}

// Sum `rows` partial records of width N (stride kMaxPartials) in a fixed order; result in thread 0.
template <int N>
__device__ inline void sum_partials(const double* part, int rows, double (&out)[N], double* smem) {
#pragma unroll
  for (int q = 0; q < N; ++q) out[q] = 0.0;
  for (int r = threadIdx.x; r < rows; r += blockDim.x) {
#pragma unroll
    for (int q = 0; q < N; ++q) out[q] += __ldcg(part + (size_t)r * kMaxPartials + q);
  }
  block_sum<N>(out, smem);
}

// Write this block's partial sums; returns true (in every thread) for the last block to finish.
template <int N>
__device__ inline bool publish_partials(double (&v)[N], double* part, unsigned int* counter, double* smem) {
  block_sum<N>(v, smem);
  __shared__ int s_last;
  if (threadIdx.x == 0) {
#pragma unroll
    for (int q = 0; q < N; ++q) part[(size_t)blockIdx.x * kMaxPartials + q] = v[q];
    __threadfence();
    unsigned int t = atomicAdd(counter, 1u);
    s_last = (t == gridDim.x - 1);
  }
  __syncthreads();
  const bool last = s_last != 0;
  if (last) __threadfence();
  return last;
}

// ---------------------------------------------------------------------------
// Launchers (defined in the .cu files)
// ---------------------------------------------------------------------------
// one step attempt = primal kernel + dual kernel (the dual kernel's last block runs the step control)
void launch_primal(const Dev& d, const Params& prm, cudaStream_t s);
void launch_dual(const Dev& d, const Params& prm, cudaStream_t s);
// KKT check: primal-side reductions, dual-side reductions + decision, apply
void launch_check(const Dev& d, const Params& prm, int eval_only, cudaStream_t s);
// apply a pending preconditioner update now (debug reads)
void launch_flush_update(const Dev& d, const Params& prm, cudaStream_t s);
int check_kernel_count();

// setup
void launch_fill(double* v, double val, long long n, cudaStream_t s);
void launch_row_absmax(const Csr& M, int rows, double* out, cudaStream_t s);
void launch_row_powsum(const Csr& M, int rows, double beta, int square_root, double* out, cudaStream_t s);
void launch_factor_from_norm(double* f, int n, cudaStream_t s);  // f <- f > 0 ? 1/sqrt(f) : 1
void launch_scale_values(int* rp, int* ci, double* v, int rows, const double* frow, const double* fcol,
                         int row_is_a_row, cudaStream_t s);
void launch_mul_inplace(double* a, const double* f, int n, cudaStream_t s);
void launch_scale_problem_vectors(const Dev& d, cudaStream_t s);
void launch_init_vectors(const Dev& d, cudaStream_t s);
void launch_spmv_binned(const Csr& M, const BinTable& bt, int grid, const double* x, double* y, cudaStream_t s);
void launch_norm2(const double* v, int n, double* out, cudaStream_t s);  // out[0] = ||v||_2; out[1..1025) scratch
void launch_absmax(const double* v, long long n, double* out, cudaStream_t s);
void launch_scale_by_inv(double* v, int n, const double* denom, cudaStream_t s);  // v /= denom[0]

}  // namespace lpop
