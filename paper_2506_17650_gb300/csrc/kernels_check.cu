// KKT check, termination and adaptive restart (Section 3.2: restarts follow
// PDLP and keep T, Sigma; Section 4.1: relative tolerance).
//
//   check_primal: rows j of A^T, gathers y (and the average's y-sum).  Reduced
//                 cost rc = c - A^T y split by bound kind into a multiplier and a
//                 dual residual; partial sums of ||dres||^2 (user and scaled
//                 units), the bound terms of the dual objective, c^T x, and
//                 ||x - x_last_restart||^2; the same for the average.
//   check_dual:   rows i of A, gathers the average's x-sum.  Primal residual by
//                 row sense (user and scaled units), b^T y, ||y - y_last||^2;
//                 the same for the average.  The last block forms the relative
//                 KKT errors, decides termination and restart, and updates the
//                 primal weight.
//   check_apply:  carries out the decision on the vectors (restart point,
//                 move to the average, zero the averages).
#include "common.cuh"
#include "ops.cuh"
#include "spmv.cuh"

namespace lpop {

namespace {

// The FP64 check kernels are compiled for 3 resident blocks per SM, so that
// their grid (the FP64 step kernels' grid) runs in one wave; the FP32 ones
// keep their registers (their grid is sized for 4 blocks per SM anyway).
template <class V>
constexpr int kCheckBlocksPerSm = sizeof(V) == 8 ? 3 : 1;

template <bool AVG, class V>
__global__ void __launch_bounds__(kBlock, kCheckBlocksPerSm<V>) check_primal_kernel(Dev d) {
  __shared__ double smem[kBlock * 10];
  pdl_wait();
  constexpr int NV = AVG ? 2 : 1;
  const Vecs<V>& v = vecs<V>(d);
  const DevState* st = d.st;
  const int cur = st->cur;
  CheckPrimalOp<NV, V> op;
  op.c = v.c; op.l = v.l; op.u = v.u; op.inv_dc = d.inv_dc;
  op.xc = v.x[cur]; op.xbarc = v.xbar[cur]; op.xlast = v.x_last;
  const double w = st->wsum;
  op.avg = AVG && w > 0.0;
  op.inv_w = op.avg ? 1.0 / w : 0.0;
#pragma unroll
  for (int q = 0; q < 10; ++q) op.acc[q] = 0.0;
  Gather<NV, V> g;
  g.x[0] = v.y[cur];
  if (NV > 1) g.x[NV - 1] = v.ybar[cur];
  g.n = d.m;
  g.bad = d.bad_gathers;
  for_each_row<NV, V, double>(d.binsAt, csr_at<V>(d), g, op, smem, row_slots_at<V>(d, d.partials));
  block_sum_smem<10>(op.acc, smem);
  if (threadIdx.x == 0) {
    double* rec = d.partials + (size_t)blockIdx.x * kMaxPartials;
#pragma unroll
    for (int q = 0; q < 10; ++q) rec[q] = op.acc[q];
  }
  pdl_trigger();
}

template <bool AVG, class V>
__global__ void __launch_bounds__(kBlock, kCheckBlocksPerSm<V>) check_dual_kernel(Dev d, Params prm, int eval_only) {
  __shared__ double smem[kBlock * 8];
  pdl_wait();
  __shared__ double fold[kFold * 10];
  const int nfold = fold_begin<10>(d.partials, partial_rows_at<V>(d), fold);
  const Vecs<V>& v = vecs<V>(d);
  DevState* st = d.st;
  const int cur = st->cur;
  const double w = st->wsum;
  const int avg_ok = AVG && w > 0.0;
  CheckDualOp<V> op;
  op.b = v.b; op.inv_dr = d.inv_dr; op.sense = d.sense;
  op.axc = v.ax[cur]; op.yc = v.y[cur]; op.ybarc = v.ybar[cur]; op.ylast = v.y_last;
  op.ax_avg = v.ax_avg;
  op.inv_w = avg_ok ? 1.0 / w : 0.0;
  op.avg = avg_ok;
#pragma unroll
  for (int q = 0; q < 8; ++q) op.acc[q] = 0.0;
  if (AVG) {
    Gather<1, V> g;
    g.x[0] = v.xbar[cur];
    g.n = d.n;
    g.bad = d.bad_gathers;
    for_each_row<1, V, double>(d.binsA, csr_a<V>(d), g, op, smem, row_slots_a<V>(d, d.partials2));
  } else {
    // without an average candidate only the cached A x is needed: no sparse product
    const double s0[1] = {0.0};
    const int stride = gridDim.x * blockDim.x;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < d.m; i += stride) op.row(i, s0);
  }
  block_sum_smem<8>(op.acc, smem);
  cp_async_wait_all();
  __syncthreads();
  double rec[18];
#pragma unroll
  for (int q = 0; q < 8; ++q) rec[q] = op.acc[q];
#pragma unroll
  for (int q = 8; q < 18; ++q) rec[q] = 0.0;
  if (threadIdx.x == 0) {
    for (int k = 0; k < nfold; ++k) {
#pragma unroll
      for (int q = 0; q < 10; ++q) rec[8 + q] += fold[10 * k + q];
    }
  }
  __shared__ int s_last;
  if (!publish_last<18>(rec, d.partials2, &st->counter, &s_last)) return;
  pdl_trigger();
  double tot[18];
  // the segmented rows of A write their slots only when the average's product runs
  const int f0 = unfolded_first(grid_a<V>(d)), np = partial_rows_at<V>(d);
  block_sum_records<18, 10>(d.partials2, AVG ? partial_rows_a<V>(d) : grid_a<V>(d), d.partials + (size_t)f0 * kMaxPartials,
                            np > f0 ? np - f0 : 0, 8, tot, smem);
  double p1[10], p2[8];
#pragma unroll
  for (int q = 0; q < 10; ++q) p1[q] = tot[8 + q];
#pragma unroll
  for (int q = 0; q < 8; ++q) p2[q] = tot[q];
  if (threadIdx.x == 0) {
    DevState s = *st;  // register copy, written back once
    check_control(&s, prm, p1, p2, eval_only, avg_ok);
    refresh_derived(s, prm.phi, prm.sched);  // omega may have changed at a restart
    s.counter = 0;
    *st = s;
  }
}

template <class V>
__global__ void check_apply_kernel(Dev d) {
  pdl_wait();
  pdl_trigger();
  const DevState s = *d.st;
  apply_decision<V>(d, s, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x);
}

}  // namespace

int check_kernel_count() { return 3; }

template <class V>
void launch_check_t(const Dev& d, const Params& prm, int eval_only, cudaStream_t s) {
  const bool avg = prm.mode == kPdlp && eval_only != 1;
  if (avg) {
    launch_pdl(check_primal_kernel<true, V>, grid_at<V>(d), s, d);
    launch_pdl(check_dual_kernel<true, V>, grid_a<V>(d), s, d, prm, eval_only);
  } else {
    launch_pdl(check_primal_kernel<false, V>, grid_at<V>(d), s, d);
    launch_pdl(check_dual_kernel<false, V>, grid_a<V>(d), s, d, prm, eval_only);
  }
  const int rows = d.n > d.m ? d.n : d.m;
  int grid = (rows + kBlock - 1) / kBlock;
  if (grid > 4 * 152) grid = 4 * 152;
  if (grid < 1) grid = 1;
  launch_pdl(check_apply_kernel<V>, grid, s, d);
}

void launch_check(const Dev& d, const Params& prm, int eval_only, bool fp32, cudaStream_t s) {
  if (fp32) launch_check_t<float>(d, prm, eval_only, s);
  else launch_check_t<double>(d, prm, eval_only, s);
}

}  // namespace lpop
