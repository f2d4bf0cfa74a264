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
//                Its last block to finish sums all partials in a fixed order
//                and runs the step control: accept/reject (adaptive step),
//                next eta, swap of the double buffers, and the scalars of a
//                pending online update of T and Sigma (Eq. (7), Algorithm 1).
//
// The pending update is applied by the next primal / dual kernel to its own
// rows before they use T_j / Sigma_i, so the update costs no extra launch.
#include "common.cuh"
#include "spmv.cuh"

namespace lpop {

namespace {

struct StepScalars {
  int cur;
  int collect;  // k mod phi == 0: record q / p for the online gradient
  int pend;     // apply the pending update of this side
  double eta, omega;
  double up_scale;
  double sqrt_gnorm;
};

__device__ __forceinline__ StepScalars read_scalars(const DevState* st, const Params& prm, bool primal) {
  StepScalars s;
  s.cur = st->cur;
  s.eta = st->eta;
  s.omega = st->omega;
  const long long k = st->k;
  s.collect = prm.phi > 0 && (k % prm.phi) == 0;
  s.pend = primal ? st->pend_p : st->pend_d;
  s.up_scale = primal ? st->up_scale_p : st->up_scale_d;
  const double gn = primal ? st->gp_norm : st->gd_norm;
  s.sqrt_gnorm = gn > 0.0 ? sqrt(gn) : 0.0;
  return s;
}

// One projected online-gradient step of a diagonal preconditioner entry with
// the chosen learning-rate rule (Section 3.1 OGD, Section 4.1 AdaGrad).
__device__ __forceinline__ double ogd_entry(double P, double* G, double grad, const Params& prm, double sqrt_gnorm) {
  if (prm.sched == kAdagrad) {
    const double Gn = *G + grad * grad;
    *G = Gn;
    if (Gn > 0.0) P = P - prm.alpha * (grad / sqrt(Gn));
  } else if (prm.sched == kAdagradNorm) {
    if (sqrt_gnorm > 0.0) P = P - prm.alpha * (grad / sqrt_gnorm);
  } else {
    P = P - prm.alpha * grad;
  }
  return fmax(P, prm.floor);
}

struct PrimalOp {
  const double *c, *l, *u, *xc, *xbarc;
  double *T, *GT, *q, *xn, *xbarn;
  Params prm;
  StepScalars sc;
  double step;  // eta / omega
  double acc[3];  // sum dx^2 / T, ||g||^2, sum q^2

  __device__ __forceinline__ void row(int j, const double (&s)[1]) {
    double Tj = T[j];
    if (sc.pend) {
      Tj = ogd_entry(Tj, GT + j, sc.up_scale * q[j], prm, sc.sqrt_gnorm);
      T[j] = Tj;
    }
    const double g = __ldg(c + j) - s[0];
    const double x0 = xc[j];
    const double xh = x0 - step * Tj * g;
    const double lo = __ldg(l + j), hi = __ldg(u + j);
    const double x1 = fmin(fmax(xh, lo), hi);
    xn[j] = x1;
    if (prm.mode == kPdlp) xbarn[j] = xbarc[j] + sc.eta * x1;
    const double dx = x1 - x0;
    acc[0] += dx * dx / Tj;
    if (sc.collect) {
      const double gi = (xh >= lo && xh <= hi) ? g : 0.0;
      const double qj = gi * g;
      q[j] = qj;
      acc[1] += g * g;
      acc[2] += qj * qj;
    }
  }
};

struct DualOp {
  const double *b, *axc, *yc, *ybarc;
  const uint8_t* sense;
  double *S, *GS, *p, *yn, *axn, *ybarn;
  Params prm;
  StepScalars sc;
  double step;  // eta * omega
  double acc[4];  // sum dy^2 / Sigma, dy . A dx, ||b - A x||^2, sum p^2

  __device__ __forceinline__ void row(int i, const double (&s)[1]) {
    double Si = S[i];
    if (sc.pend) {
      Si = ogd_entry(Si, GS + i, sc.up_scale * p[i], prm, sc.sqrt_gnorm);
      S[i] = Si;
    }
    const double a1 = s[0];
    const double a0 = axc[i];
    const double bi = __ldg(b + i);
    const double r = bi - (2.0 * a1 - a0);
    const double y0 = yc[i];
    const double yh = y0 + step * Si * r;
    const uint8_t sn = __ldg(sense + i);
    const double y1 = sn == kEq ? yh : (sn == kLe ? fmin(yh, 0.0) : fmax(yh, 0.0));
    yn[i] = y1;
    axn[i] = a1;
    if (prm.mode == kPdlp) ybarn[i] = ybarc[i] + sc.eta * y1;
    const double dy = y1 - y0;
    acc[0] += dy * dy / Si;
    acc[1] += dy * (a1 - a0);
    if (sc.collect) {
      const double res = bi - a0;
      const bool inside = sn == kEq || (sn == kLe ? yh <= 0.0 : yh >= 0.0);
      const double pi = inside ? res * r : 0.0;
      p[i] = pi;
      acc[2] += res * res;
      acc[3] += pi * pi;
    }
  }
};

__global__ void __launch_bounds__(kBlock) primal_step_kernel(Dev d, Params prm) {
  __shared__ double smem[32 * kMaxPartials];
  PrimalOp op;
  op.sc = read_scalars(d.st, prm, true);
  const int cur = op.sc.cur, nxt = cur ^ 1;
  op.prm = prm;
  op.c = d.c; op.l = d.l; op.u = d.u;
  op.xc = d.x[cur]; op.xbarc = d.xbar[cur];
  op.T = d.T; op.GT = d.GT; op.q = d.q;
  op.xn = d.x[nxt]; op.xbarn = d.xbar[nxt];
  op.step = op.sc.eta / op.sc.omega;
  op.acc[0] = op.acc[1] = op.acc[2] = 0.0;
  Gather<1> g;
  g.x[0] = d.y[cur];
  for_each_row<1>(d.binsAt, d.At, g, op, smem);
  block_sum<3>(op.acc, smem);
  if (threadIdx.x == 0) {
    double* part = d.partials + (size_t)blockIdx.x * kMaxPartials;
    part[0] = op.acc[0]; part[1] = op.acc[1]; part[2] = op.acc[2];
  }
}

// Step control (single thread): adaptive step test of Eq. (6) in the T^-1 /
// Sigma^-1 weighted norms, next step size, buffer swap, online-update scalars.
__device__ void step_control(const Dev& d, const Params& prm, const double (&t1)[3], const double (&t2)[4]) {
  DevState* st = d.st;
  const double eta = st->eta, omega = st->omega;
  const long long k = st->k;
  const bool collect = prm.phi > 0 && (k % prm.phi) == 0;
  st->pend_p = 0;  // applied by this attempt's kernels
  st->pend_d = 0;
  st->attempts += 1;
  bool accept = true;
  double eta_next = eta;
  if (prm.mode == kPdlp) {
    const double movement = omega * t1[0] + t2[0] / omega;
    const double interaction = fabs(t2[1]);
    const double eta_max = interaction > 0.0 ? movement / (2.0 * interaction) : INFINITY;
    accept = eta <= eta_max;
    const double t = (double)st->attempts;
    eta_next = fmin((1.0 - pow(t + 1.0, -0.3)) * eta_max, (1.0 + pow(t + 1.0, -0.6)) * eta);
    st->last_eta_max = eta_max;
  }
  if (accept) {
    if (collect) {
      if (!prm.normalize || t1[1] > 0.0) {
        const double sc = -(eta / omega) * (prm.normalize ? 1.0 / t1[1] : 1.0);
        st->up_scale_p = sc;
        st->pend_p = 1;
        if (prm.sched == kAdagradNorm) st->gp_norm += sc * sc * t1[2];
      }
      if (!prm.normalize || t2[2] > 0.0) {
        const double sc = -(eta * omega) * (prm.normalize ? 1.0 / t2[2] : 1.0);
        st->up_scale_d = sc;
        st->pend_d = 1;
        if (prm.sched == kAdagradNorm) st->gd_norm += sc * sc * t2[3];
      }
    }
    if (prm.mode == kPdlp) st->wsum += eta;
    st->cur ^= 1;
    st->k = k + 1;
  }
  st->eta = eta_next;
  st->last_accept = accept ? 1 : 0;
}

__global__ void __launch_bounds__(kBlock) dual_step_kernel(Dev d, Params prm) {
  __shared__ double smem[32 * kMaxPartials];
  DualOp op;
  op.sc = read_scalars(d.st, prm, false);
  const int cur = op.sc.cur, nxt = cur ^ 1;
  op.prm = prm;
  op.b = d.b; op.sense = d.sense;
  op.axc = d.ax[cur]; op.yc = d.y[cur]; op.ybarc = d.ybar[cur];
  op.S = d.S; op.GS = d.GS; op.p = d.p;
  op.yn = d.y[nxt]; op.axn = d.ax[nxt]; op.ybarn = d.ybar[nxt];
  op.step = op.sc.eta * op.sc.omega;
  op.acc[0] = op.acc[1] = op.acc[2] = op.acc[3] = 0.0;
  Gather<1> g;
  g.x[0] = d.x[nxt];  // x+ written by the primal kernel
  for_each_row<1>(d.binsA, d.A, g, op, smem);
  const bool last = publish_partials<4>(op.acc, d.partials2, &d.st->counter, smem);
  if (!last) return;
  double t1[3], t2[4];
  sum_partials<3>(d.partials, d.gridAt, t1, smem);
  sum_partials<4>(d.partials2, d.gridA, t2, smem);
  if (threadIdx.x == 0) {
    step_control(d, prm, t1, t2);
    d.st->counter = 0;
  }
}

// Apply a pending update of T and Sigma immediately (used before debug reads).
__global__ void flush_update_kernel(Dev d, Params prm) {
  const DevState* st = d.st;
  const int pp = st->pend_p, pd = st->pend_d;
  const double sp = st->up_scale_p, sd = st->up_scale_d;
  const double gp = st->gp_norm > 0.0 ? sqrt(st->gp_norm) : 0.0;
  const double gd = st->gd_norm > 0.0 ? sqrt(st->gd_norm) : 0.0;
  const int stride = gridDim.x * blockDim.x;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < d.n && pp; j += stride)
    d.T[j] = ogd_entry(d.T[j], d.GT + j, sp * d.q[j], prm, gp);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < d.m && pd; i += stride)
    d.S[i] = ogd_entry(d.S[i], d.GS + i, sd * d.p[i], prm, gd);
}

__global__ void clear_pending_kernel(DevState* st) {
  st->pend_p = 0;
  st->pend_d = 0;
}

}  // namespace

void launch_primal(const Dev& d, const Params& prm, cudaStream_t s) {
  primal_step_kernel<<<d.gridAt, kBlock, 0, s>>>(d, prm);
}

void launch_dual(const Dev& d, const Params& prm, cudaStream_t s) {
  dual_step_kernel<<<d.gridA, kBlock, 0, s>>>(d, prm);
}

void launch_flush_update(const Dev& d, const Params& prm, cudaStream_t s) {
  const int rows = d.n > d.m ? d.n : d.m;
  int grid = (rows + kBlock - 1) / kBlock;
  if (grid < 1) grid = 1;
  flush_update_kernel<<<grid, kBlock, 0, s>>>(d, prm);
  clear_pending_kernel<<<1, 1, 0, s>>>(d.st);
}

}  // namespace lpop

namespace lpop {
// Resident blocks per SM of the heavier of the two step kernels (sizes the grids).
int row_kernel_blocks_per_sm() {
  int a = 0, b = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, primal_step_kernel, kBlock, 0) != cudaSuccess) a = 1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, dual_step_kernel, kBlock, 0) != cudaSuccess) b = 1;
  return a < b ? a : b;
}
}  // namespace lpop
