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
#include "spmv.cuh"

namespace lpop {

namespace {

// Vectors of type V (FP64, or FP32 in the mixed-precision phase); every
// quantity of the check is formed and summed in FP64.
template <int NV, class V>
struct CheckPrimalOp {
  const V *c, *l, *u, *xc, *xbarc, *xlast;
  const double* dc;
  double w;
  int avg;
  double acc[10];
  __device__ __forceinline__ void prefetch(int) {}

  __device__ __forceinline__ void side(int j, double rc, double x, double* a) {
    const double lo = (double)__ldg(l + j), hi = (double)__ldg(u + j);
    const bool lf = isfinite(lo), uf = isfinite(hi);
    double lam;
    if (lf && uf) lam = rc;
    else if (lf) lam = fmax(rc, 0.0);
    else if (uf) lam = fmin(rc, 0.0);
    else lam = 0.0;
    const double ds = rc - lam;
    const double du = ds / __ldg(dc + j);
    a[0] += du * du;
    a[1] += ds * ds;
    a[2] += (lf ? lo * fmax(lam, 0.0) : 0.0) - (uf ? hi * fmax(-lam, 0.0) : 0.0);
    a[3] += (double)__ldg(c + j) * x;
    const double dx = x - (double)xlast[j];
    a[4] += dx * dx;
  }

  __device__ __forceinline__ void row(int j, const double (&s)[NV]) {
    const double cj = (double)__ldg(c + j);
    side(j, cj - s[0], (double)xc[j], acc);
    if (NV > 1 && avg) side(j, cj - s[NV - 1] / w, (double)xbarc[j] / w, acc + 5);
  }
};

template <class V>
struct CheckDualOp {
  const V *b, *axc, *yc, *ybarc, *ylast;
  const double* dr;
  const uint8_t* sense;
  V* ax_avg;
  double w;
  int avg;
  double acc[8];
  __device__ __forceinline__ void prefetch(int) {}

  __device__ __forceinline__ void side(int i, double ax, double y, double* a) {
    const double bi = (double)__ldg(b + i);
    const double rs = ax - bi;
    const uint8_t sn = __ldg(sense + i);
    const double ps = sn == kEq ? rs : (sn == kGe ? fmax(-rs, 0.0) : fmax(rs, 0.0));
    const double pu = ps / __ldg(dr + i);
    a[0] += pu * pu;
    a[1] += ps * ps;
    a[2] += bi * y;
    const double dy = y - (double)ylast[i];
    a[3] += dy * dy;
  }

  // s[0] = (A xbar)_i, used only when the average is a candidate
  __device__ __forceinline__ void row(int i, const double (&s)[1]) {
    side(i, (double)axc[i], (double)yc[i], acc);
    if (avg) {
      const double axa = s[0] / w;
      ax_avg[i] = (V)axa;
      side(i, axa, (double)ybarc[i] / w, acc + 4);
    }
  }
};

template <bool AVG, class V>
__global__ void __launch_bounds__(kBlock) check_primal_kernel(Dev d) {
  __shared__ double smem[32 * kMaxPartials];
  constexpr int NV = AVG ? 2 : 1;
  const Vecs<V>& v = vecs<V>(d);
  const DevState* st = d.st;
  const int cur = st->cur;
  CheckPrimalOp<NV, V> op;
  op.c = v.c; op.l = v.l; op.u = v.u; op.dc = d.dc;
  op.xc = v.x[cur]; op.xbarc = v.xbar[cur]; op.xlast = v.x_last;
  op.w = st->wsum;
  op.avg = AVG && op.w > 0.0;
#pragma unroll
  for (int q = 0; q < 10; ++q) op.acc[q] = 0.0;
  Gather<NV, V> g;
  g.x[0] = v.y[cur];
  if (NV > 1) g.x[NV - 1] = v.ybar[cur];
  for_each_row<NV, V, double>(d.binsAt, csr_at<V>(d), g, op, smem);
  block_sum<10>(op.acc, smem);
  if (threadIdx.x == 0) {
    double* part = d.partials + (size_t)blockIdx.x * kMaxPartials;
#pragma unroll
    for (int q = 0; q < 10; ++q) part[q] = op.acc[q];
  }
}

struct Cand {
  double pobj, dobj, rel_p, rel_d, rel_g, p2, d2, g2, dist_x2, dist_y2;
};

__device__ __forceinline__ double kw(double p2, double d2, double g2, double omega) {
  return sqrt(omega * omega * p2 + d2 / (omega * omega) + g2);
}

__device__ __forceinline__ bool converged(const Cand& c, double tol) {
  return c.rel_p <= tol && c.rel_d <= tol && c.rel_g <= tol;
}

__device__ void check_control(DevState* st, const Params& prm, const double (&p1)[10], const double (&p2)[8],
                              int eval_only, int avg_ok) {
  Cand cd[2];
  for (int k = 0; k < 2; ++k) {
    Cand& c = cd[k];
    c.pobj = p1[3 + 5 * k];
    c.dobj = p2[2 + 4 * k] + p1[2 + 5 * k];
    const double pn = sqrt(p2[0 + 4 * k]);
    const double dn = sqrt(p1[0 + 5 * k]);
    c.rel_p = pn / (1.0 + prm.b_norm);
    c.rel_d = dn / (1.0 + prm.c_norm);
    const double gap = c.pobj - c.dobj;
    c.rel_g = fabs(gap) / (1.0 + fabs(c.pobj) + fabs(c.dobj));
    c.p2 = p2[1 + 4 * k];
    c.d2 = p1[1 + 5 * k];
    c.g2 = gap * gap;
    c.dist_x2 = p1[4 + 5 * k];
    c.dist_y2 = p2[3 + 4 * k];
  }
  st->restart_action = 0;
  st->adopt_avg = 0;
  st->pobj = cd[0].pobj; st->dobj = cd[0].dobj;
  st->rel_pres = cd[0].rel_p; st->rel_dres = cd[0].rel_d; st->rel_gap = cd[0].rel_g;
  st->stats_from_avg = 0;
  if (eval_only) return;
  const int ncand = avg_ok ? 2 : 1;
  for (int k = 0; k < ncand; ++k) {
    if (!(isfinite(cd[k].rel_p) && isfinite(cd[k].rel_d) && isfinite(cd[k].rel_g))) {
      st->status = 4;
      return;
    }
  }
  for (int k = 0; k < ncand; ++k) {
    if (converged(cd[k], st->tol)) {
      st->status = 1;
      st->pobj = cd[k].pobj; st->dobj = cd[k].dobj;
      st->rel_pres = cd[k].rel_p; st->rel_dres = cd[k].rel_d; st->rel_gap = cd[k].rel_g;
      st->stats_from_avg = k;
      if (k == 1) {
        st->adopt_avg = 1;
        st->apply_w = st->wsum;
      }
      return;
    }
  }
  if (prm.mode != kPdlp) return;  // plain mode: no restarts, no restart reference
  const double omega = st->omega;
  if (!st->checked0) {
    st->klast_p2 = cd[0].p2; st->klast_d2 = cd[0].d2; st->klast_g2 = cd[0].g2;
    st->k_prev = kw(cd[0].p2, cd[0].d2, cd[0].g2, omega);
    st->last_restart_attempt = st->attempts;
    st->checked0 = 1;
    st->restart_action = 3;
    return;
  }
  if (!prm.restart) return;
  const double K0 = kw(cd[0].p2, cd[0].d2, cd[0].g2, omega);
  const double K1 = ncand > 1 ? kw(cd[1].p2, cd[1].d2, cd[1].g2, omega) : INFINITY;
  const int pick = (ncand > 1 && K1 < K0) ? 1 : 0;
  const double K = pick ? K1 : K0;
  const double Klast = kw(st->klast_p2, st->klast_d2, st->klast_g2, omega);
  const double since = (double)(st->attempts - st->last_restart_attempt);
  const bool do_restart = (K <= 0.2 * Klast) || (K <= 0.8 * Klast && K > st->k_prev) ||
                          (since >= 0.36 * (double)st->attempts);
  st->k_prev = K;
  if (!do_restart) return;
  const double dx = sqrt(cd[pick].dist_x2), dy = sqrt(cd[pick].dist_y2);
  if (dx > 1e-10 && dy > 1e-10) st->omega = exp(0.5 * log(dy / dx) + 0.5 * log(omega));
  st->restart_action = pick ? 2 : 1;
  st->apply_w = st->wsum;
  st->wsum = 0.0;
  st->klast_p2 = cd[pick].p2; st->klast_d2 = cd[pick].d2; st->klast_g2 = cd[pick].g2;
  st->last_restart_attempt = st->attempts;
  st->restarts += 1;
}

template <bool AVG, class V>
__global__ void __launch_bounds__(kBlock) check_dual_kernel(Dev d, Params prm, int eval_only) {
  __shared__ double smem[32 * kMaxPartials];
  const Vecs<V>& v = vecs<V>(d);
  DevState* st = d.st;
  const int cur = st->cur;
  const double w = st->wsum;
  const int avg_ok = AVG && w > 0.0;
  CheckDualOp<V> op;
  op.b = v.b; op.dr = d.dr; op.sense = d.sense;
  op.axc = v.ax[cur]; op.yc = v.y[cur]; op.ybarc = v.ybar[cur]; op.ylast = v.y_last;
  op.ax_avg = v.ax_avg;
  op.w = w;
  op.avg = avg_ok;
#pragma unroll
  for (int q = 0; q < 8; ++q) op.acc[q] = 0.0;
  if (AVG) {
    Gather<1, V> g;
    g.x[0] = v.xbar[cur];
    for_each_row<1, V, double>(d.binsA, csr_a<V>(d), g, op, smem);
  } else {
    // without an average candidate only the cached A x is needed: no sparse product
    const double s0[1] = {0.0};
    const int stride = gridDim.x * blockDim.x;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < d.m; i += stride) op.row(i, s0);
  }
  const bool last = publish_partials<8>(op.acc, d.partials2, &st->counter, smem);
  if (!last) return;
  double p1[10], p2[8];
  sum_partials<10>(d.partials, d.gridAt, p1, smem);
  sum_partials<8>(d.partials2, d.gridA, p2, smem);
  if (threadIdx.x == 0) {
    DevState s = *st;  // register copy, written back once
    check_control(&s, prm, p1, p2, eval_only, avg_ok);
    refresh_derived(s, prm.phi);  // omega may have changed at a restart
    s.counter = 0;
    *st = s;
  }
}

template <class V>
__global__ void check_apply_kernel(Dev d) {
  const Vecs<V>& v = vecs<V>(d);
  const DevState* st = d.st;
  const int action = st->restart_action;
  const int adopt = st->adopt_avg;
  if (action == 0 && !adopt) return;
  const int cur = st->cur;
  const double w = st->apply_w;
  const bool to_avg = adopt || action == 2;
  const bool mark = action >= 1;
  const bool reset = action == 1 || action == 2;
  const int stride = gridDim.x * blockDim.x;
  V *x = v.x[cur], *xb = v.xbar[cur], *y = v.y[cur], *yb = v.ybar[cur], *ax = v.ax[cur];
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < d.n; j += stride) {
    V val = x[j];
    if (to_avg) {
      val = (V)((double)xb[j] / w);
      x[j] = val;
    }
    if (mark) v.x_last[j] = val;
    if (reset) xb[j] = V(0);
  }
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < d.m; i += stride) {
    V val = y[i];
    if (to_avg) {
      val = (V)((double)yb[i] / w);
      y[i] = val;
      ax[i] = v.ax_avg[i];
    }
    if (mark) v.y_last[i] = val;
    if (reset) yb[i] = V(0);
  }
}

}  // namespace

int check_kernel_count() { return 3; }

template <class V>
void launch_check_t(const Dev& d, const Params& prm, int eval_only, cudaStream_t s) {
  const bool avg = prm.mode == kPdlp && !eval_only;
  if (avg) {
    check_primal_kernel<true, V><<<d.gridAt, kBlock, 0, s>>>(d);
    check_dual_kernel<true, V><<<d.gridA, kBlock, 0, s>>>(d, prm, eval_only);
  } else {
    check_primal_kernel<false, V><<<d.gridAt, kBlock, 0, s>>>(d);
    check_dual_kernel<false, V><<<d.gridA, kBlock, 0, s>>>(d, prm, eval_only);
  }
  const int rows = d.n > d.m ? d.n : d.m;
  int grid = (rows + kBlock - 1) / kBlock;
  if (grid > 4 * 152) grid = 4 * 152;
  if (grid < 1) grid = 1;
  check_apply_kernel<V><<<grid, kBlock, 0, s>>>(d);
}

void launch_check(const Dev& d, const Params& prm, int eval_only, bool fp32, cudaStream_t s) {
  if (fp32) launch_check_t<float>(d, prm, eval_only, s);
  else launch_check_t<double>(d, prm, eval_only, s);
}

}  // namespace lpop
