// One step attempt of PDHG with online preconditioning (Algorithm 1 with the
// step of Eq. (6)) as two fused kernels:
//
//   primal_step: rows j of A^T.  g_j = c_j - (A^T y)_j,
//                x+_j = proj_[l_j,u_j](x_j - (eta/omega) T_j g_j)            (Eq. (6), line 1)
//                plus the partial sums of the step-size test and, on update
//                attempts, q_j = g_j^2 I(l_j <= x_half_j <= u_j) for Eq. (7).
//   dual_step:   rows i of A.  (A x+)_i, r_i = b_i - (2 A x+ - A x)_i,
//                y+_i = proj_sense(y_i + eta omega Sigma_i r_i)              (Eq. (6), line 2)
//                plus partial sums and p_i = (b - A x)_i r_i I(y_half_i in cone).
//                Its blocks fold the primal kernel's per-block sums into their
//                own, and its last block to finish sums all of them in a
//                fixed order and runs the step control: accept/reject (adaptive step),
//                next eta, swap of the double buffers, and the scalars of a
//                pending online update of T and Sigma (Eq. (7), Algorithm 1).
//
// The pending update is applied by the next primal / dual kernel to its own
// rows before they use T_j / Sigma_i, so the update costs no extra launch.
//
// GB300 runs FP64 at a small fraction of its FP32 rate, so these kernels are
// written to the FP64 instruction count: no divisions per row (1/T and
// 1/Sigma are kept as vectors and rewritten only when T / Sigma change),
// clamps and sign projections on the integer pipes (ordered keys), step
// scalars precomputed by the control thread, and block sums done by one warp.
#include "common.cuh"
#include "ops.cuh"
#include "spmv.cuh"

namespace lpop {

namespace {

// Resident blocks per SM the step kernels are compiled for: the FP64
// instances need 80 registers a thread (3 blocks), the FP32 ones fit in 64
// without spilling (4 blocks, a third more warps to hide latency).
template <class V>
constexpr int kStepBlocksPerSm = sizeof(V) == 4 ? 4 : 3;

template <class V>
__global__ void __launch_bounds__(kBlock, kStepBlocksPerSm<V>) primal_step_kernel(Dev d, Params prm) {
  __shared__ double smem[kBlock * 3];
  pdl_wait();
  const Vecs<V>& v = vecs<V>(d);
  PrimalOp<V> op;
  op.sc = read_scalars<V>(d.st, true);
  const int cur = op.sc.cur, nxt = cur ^ 1;
  op.prm = prm;
  op.c = v.c; op.l = v.l; op.u = v.u;
  op.xc = v.x[cur]; op.xbarc = v.xbar[cur];
  op.T = v.T; op.invT = v.invT; op.GT = v.GT; op.q = v.q;
  op.xn = v.x[nxt]; op.xbarn = v.xbar[nxt];
  op.acc[0] = op.acc[1] = op.acc[2] = V(0);
  Gather<1, V> g;
  g.x[0] = v.y[cur];
  g.n = d.m;
  g.bad = d.bad_gathers;
  for_each_row<1, V, V>(d.binsAt, csr_at<V>(d), g, op, smem, row_slots_at<V>(d, d.partials));
  double a[3] = {(double)op.acc[0], (double)op.acc[1], (double)op.acc[2]};
  block_sum_smem<3>(a, smem);
  if (threadIdx.x == 0) {
    double* rec = d.partials + (size_t)blockIdx.x * kMaxPartials;
    rec[0] = a[0]; rec[1] = a[1]; rec[2] = a[2];
  }
  pdl_trigger();
}

template <class V>
__global__ void __launch_bounds__(kBlock, kStepBlocksPerSm<V>) dual_step_kernel(Dev d, Params prm) {
  __shared__ double smem[kBlock * 7];
  __shared__ double fold[kFold * 3];
  __shared__ DevState s_st;  // the state does not change until the step control, at the very end
  __shared__ double s_f[2];
  pdl_wait();
  // copied while the rows run: this block's share of the primal kernel's
  // records, and the state for the step control
  const int nfold = fold_begin<3>(d.partials, partial_rows_at<V>(d), fold);
  {
    static_assert(sizeof(DevState) % 8 == 0, "state copied in 8-byte words");
    const double* src = reinterpret_cast<const double*>(d.st);
    double* dst = reinterpret_cast<double*>(&s_st);
    for (int t = threadIdx.x; t < (int)(sizeof(DevState) / 8); t += blockDim.x) cp_async8(dst + t, src + t);
  }
  const Vecs<V>& v = vecs<V>(d);
  DualOp<V> op;
  op.sc = read_scalars<V>(d.st, false);
  const int cur = op.sc.cur, nxt = cur ^ 1;
  op.prm = prm;
  op.b = v.b; op.sense = d.sense;
  op.axc = v.ax[cur]; op.yc = v.y[cur]; op.ybarc = v.ybar[cur];
  op.S = v.S; op.invS = v.invS; op.GS = v.GS; op.p = v.p;
  op.yn = v.y[nxt]; op.axn = v.ax[nxt]; op.ybarn = v.ybar[nxt];
  op.acc[0] = op.acc[1] = op.acc[2] = op.acc[3] = V(0);
  Gather<1, V> g;
  g.x[0] = v.x[nxt];  // x+ written by the primal kernel
  g.n = d.n;
  g.bad = d.bad_gathers;
  for_each_row<1, V, V>(d.binsA, csr_a<V>(d), g, op, smem, row_slots_a<V>(d, d.partials2));
  double a[4] = {(double)op.acc[0], (double)op.acc[1], (double)op.acc[2], (double)op.acc[3]};
  block_sum_smem<4>(a, smem);
  cp_async_wait_all();
  __syncthreads();
  double rec[7] = {a[0], a[1], a[2], a[3], 0.0, 0.0, 0.0};
  const long long tnext = s_st.attempts + 1;
  if (threadIdx.x == 0) {
    // step-size factors of the next attempt, in case this block runs the control
    if (tnext < kStepTab) {
      cp_async8(s_f, d.step_tab + tnext);
      cp_async8(s_f + 1, d.step_tab + kStepTab + tnext);
    }
    for (int k = 0; k < nfold; ++k) {
#pragma unroll
      for (int q = 0; q < 3; ++q) rec[4 + q] += fold[3 * k + q];
    }
  }
  __shared__ int s_last;
  if (!publish_last<7>(rec, d.partials2, &d.st->counter, &s_last)) return;
  pdl_trigger();  // the other blocks have exited: let the next kernel launch during the control
  // totals: this kernel's records (own sums, folded primal sums) and its
  // segmented rows' slots, then any primal records beyond the folded ones
  double tot[7];
  const int f0 = unfolded_first(grid_a<V>(d)), np = partial_rows_at<V>(d);
  block_sum_records<7, 3>(d.partials2, partial_rows_a<V>(d), d.partials + (size_t)f0 * kMaxPartials,
                          np > f0 ? np - f0 : 0, 4, tot, smem);
  if (threadIdx.x == 0) {
    const double t1[3] = {tot[4], tot[5], tot[6]};
    const double t2[4] = {tot[0], tot[1], tot[2], tot[3]};
    double f1, f2;
    if (tnext < kStepTab) {
      cp_async_wait_all();
      f1 = s_f[0];
      f2 = s_f[1];
    } else {
      step_factors(d.step_tab, tnext, &f1, &f2);
    }
    step_control_state(s_st, prm, f1, f2, t1, t2);  // on the shared copy: no register-held state
  }
  __syncthreads();
  {  // written back by the block, word by word
    const double* src = reinterpret_cast<const double*>(&s_st);
    double* dst = reinterpret_cast<double*>(d.st);
    for (int t = threadIdx.x; t < (int)(sizeof(DevState) / 8); t += blockDim.x) dst[t] = src[t];
  }
}

// Apply a pending update of T and Sigma immediately (used before debug reads).
template <class V>
__global__ void flush_update_kernel(Dev d, Params prm) {
  const Vecs<V>& v = vecs<V>(d);
  const DevState* st = d.st;
  const int pp = st->pend_p, pd = st->pend_d;
  const V sp = (V)st->up_scale_p, sd = (V)st->up_scale_d;
  const V gp = (V)st->sqrt_gp, gd = (V)st->sqrt_gd;
  const int stride = gridDim.x * blockDim.x;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < d.n && pp; j += stride) {
    v.T[j] = ogd_entry<V>(v.T[j], v.GT + j, sp * v.q[j], prm, gp);
    v.invT[j] = V(1) / v.T[j];
  }
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < d.m && pd; i += stride) {
    v.S[i] = ogd_entry<V>(v.S[i], v.GS + i, sd * v.p[i], prm, gd);
    v.invS[i] = V(1) / v.S[i];
  }
}

__global__ void clear_pending_kernel(DevState* st) {
  st->pend_p = 0;
  st->pend_d = 0;
}

// 1 / T and 1 / Sigma after T / Sigma were written from outside (reset, resume).
template <class V>
__global__ void inverse_kernel(Dev d) {
  const Vecs<V>& v = vecs<V>(d);
  const int stride = gridDim.x * blockDim.x;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < d.n; j += stride) v.invT[j] = V(1) / v.T[j];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < d.m; i += stride) v.invS[i] = V(1) / v.S[i];
}

int elementwise_grid(const Dev& d) {
  const int rows = d.n > d.m ? d.n : d.m;
  int grid = (rows + kBlock - 1) / kBlock;
  if (grid > 4096) grid = 4096;
  return grid < 1 ? 1 : grid;
}

}  // namespace

void launch_primal(const Dev& d, const Params& prm, bool fp32, cudaStream_t s) {
  if (fp32) launch_pdl(primal_step_kernel<float>, d.gridAt32, s, d, prm);
  else launch_pdl(primal_step_kernel<double>, d.gridAt, s, d, prm);
}

void launch_dual(const Dev& d, const Params& prm, bool fp32, cudaStream_t s) {
  if (fp32) launch_pdl(dual_step_kernel<float>, d.gridA32, s, d, prm);
  else launch_pdl(dual_step_kernel<double>, d.gridA, s, d, prm);
}

void launch_flush_update(const Dev& d, const Params& prm, bool fp32, cudaStream_t s) {
  if (fp32) flush_update_kernel<float><<<elementwise_grid(d), kBlock, 0, s>>>(d, prm);
  else flush_update_kernel<double><<<elementwise_grid(d), kBlock, 0, s>>>(d, prm);
  clear_pending_kernel<<<1, 1, 0, s>>>(d.st);
}

void launch_inverse_preconditioners(const Dev& d, bool fp32, cudaStream_t s) {
  if (fp32) inverse_kernel<float><<<elementwise_grid(d), kBlock, 0, s>>>(d);
  else inverse_kernel<double><<<elementwise_grid(d), kBlock, 0, s>>>(d);
}

// Resident blocks per SM of the two step kernels, FP64 (primal, dual) and
// FP32 (primal32, dual32); they size the grids.
void row_kernel_blocks_per_sm(int* primal, int* dual, int* primal32, int* dual32) {
  auto occ = [](auto kernel) {
    int a = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, kernel, kBlock, 0) != cudaSuccess || a < 1) a = 1;
    return a;
  };
  *primal = occ(primal_step_kernel<double>);
  *dual = occ(dual_step_kernel<double>);
  *primal32 = occ(primal_step_kernel<float>);
  *dual32 = occ(dual_step_kernel<float>);
}

}  // namespace lpop
