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
//
// GB300 runs FP64 at a small fraction of its FP32 rate, so these kernels are
// written to the FP64 instruction count: no divisions per row (1/T and
// 1/Sigma are kept as vectors and rewritten only when T / Sigma change),
// clamps and sign projections on the integer pipes (ordered keys), step
// scalars precomputed by the control thread, and block sums done by one warp.
#include "common.cuh"
#include "spmv.cuh"

namespace lpop {

namespace {

template <class V>
struct StepScalars {
  int cur;
  int collect;  // k mod phi == 0: record q / p for the online gradient
  int pend;     // apply the pending update of this side
  V eta;
  V step;  // eta / omega (primal) or eta * omega (dual)
  V up_scale;
  V sqrt_gnorm;
};

template <class V>
__device__ __forceinline__ StepScalars<V> read_scalars(const DevState* st, bool primal) {
  StepScalars<V> s;
  s.cur = st->cur;
  s.eta = (V)st->eta;
  s.collect = st->collect;
  s.step = (V)(primal ? st->step_p : st->step_d);
  s.pend = primal ? st->pend_p : st->pend_d;
  s.up_scale = (V)(primal ? st->up_scale_p : st->up_scale_d);
  s.sqrt_gnorm = (V)(primal ? st->sqrt_gp : st->sqrt_gd);
  return s;
}

// One projected online-gradient step of a diagonal preconditioner entry with
// the chosen learning-rate rule (Section 3.1 OGD, Section 4.1 AdaGrad).
template <class V>
__device__ __forceinline__ V ogd_entry(V P, V* G, V grad, const Params& prm, V sqrt_gnorm) {
  const V alpha = (V)prm.alpha;
  if (prm.sched == kAdagrad) {
    const V Gn = *G + grad * grad;
    *G = Gn;
    if (Gn > V(0)) P = P - alpha * (grad / sqrt(Gn));
  } else if (prm.sched == kAdagradNorm) {
    if (sqrt_gnorm > V(0)) P = P - alpha * (grad / sqrt_gnorm);
  } else {
    P = P - alpha * grad;
  }
  return fmax(P, (V)prm.floor);
}

template <class V>
struct PrimalOp {
  const V *c, *l, *u, *xc, *xbarc;
  V *T, *invT, *GT, *q, *xn, *xbarn;
  Params prm;
  StepScalars<V> sc;
  V acc[3];  // sum dx^2 / T, ||g||^2, sum q^2 (per thread; combined across threads in FP64)
  V pT, piT, pc, px, pl, pu, pxb;  // operands of the row being processed, loaded early

  __device__ __forceinline__ void prefetch(int j) {
    pT = T[j];
    piT = invT[j];
    pc = __ldg(c + j);
    px = xc[j];
    pl = __ldg(l + j);
    pu = __ldg(u + j);
    if (prm.mode == kPdlp) pxb = xbarc[j];
  }

  __device__ __forceinline__ void row(int j, const V (&s)[1]) {
    V Tj = pT, iT = piT;
    if (sc.pend) {  // pending online update of T_j (rare: once every phi accepted steps)
      Tj = ogd_entry<V>(Tj, GT + j, sc.up_scale * q[j], prm, sc.sqrt_gnorm);
      iT = V(1) / Tj;
      T[j] = Tj;
      invT[j] = iT;
    }
    const V g = pc - s[0];
    const V x0 = px;
    const V xh = x0 - sc.step * Tj * g;
    const V lo = pl, hi = pu;
    const auto kx = ord_key(xh), kl = ord_key(lo), kh = ord_key(hi);
    const V x1 = clamp_keys(xh, kx, lo, kl, hi, kh);
    xn[j] = x1;
    if (prm.mode == kPdlp) xbarn[j] = pxb + sc.eta * x1;
    const V dx = x1 - x0;
    acc[0] += dx * dx * iT;
    if (sc.collect) {
      const V gi = (kx >= kl && kx <= kh) ? g : V(0);
      const V qj = gi * g;
      q[j] = qj;
      acc[1] += g * g;
      acc[2] += qj * qj;
    }
  }
};

template <class V>
struct DualOp {
  const V *b, *axc, *yc, *ybarc;
  const uint8_t* sense;
  V *S, *invS, *GS, *p, *yn, *axn, *ybarn;
  Params prm;
  StepScalars<V> sc;
  V acc[4];  // sum dy^2 / Sigma, dy . A dx, ||b - A x||^2, sum p^2
  V pS, piS, pa0, pb, py, pyb;  // operands of the row being processed, loaded early
  uint8_t psn;

  __device__ __forceinline__ void prefetch(int i) {
    pS = S[i];
    piS = invS[i];
    pa0 = axc[i];
    pb = __ldg(b + i);
    py = yc[i];
    psn = __ldg(sense + i);
    if (prm.mode == kPdlp) pyb = ybarc[i];
  }

  __device__ __forceinline__ void row(int i, const V (&s)[1]) {
    V Si = pS, iS = piS;
    if (sc.pend) {
      Si = ogd_entry<V>(Si, GS + i, sc.up_scale * p[i], prm, sc.sqrt_gnorm);
      iS = V(1) / Si;
      S[i] = Si;
      invS[i] = iS;
    }
    const V a1 = s[0];
    const V a0 = pa0;
    const V bi = pb;
    const V r = bi - (V(2) * a1 - a0);
    const V y0 = py;
    const V yh = y0 + sc.step * Si * r;
    const uint8_t sn = psn;
    const auto ky = ord_key(yh);
    // <= rows keep y <= 0, >= rows keep y >= 0, equality rows are free
    const bool outside = (sn == kLe && ky > 0) || (sn == kGe && ky < 0);
    const V y1 = outside ? V(0) : yh;
    yn[i] = y1;
    axn[i] = a1;
    if (prm.mode == kPdlp) ybarn[i] = pyb + sc.eta * y1;
    const V dy = y1 - y0;
    acc[0] += dy * dy * iS;
    acc[1] += dy * (a1 - a0);
    if (sc.collect) {
      const V res = bi - a0;
      const V pi = outside ? V(0) : res * r;
      p[i] = pi;
      acc[2] += res * res;
      acc[3] += pi * pi;
    }
  }
};

template <class V>
__global__ void __launch_bounds__(kBlock) primal_step_kernel(Dev d, Params prm) {
  __shared__ double smem[kBlock * 3];
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
  for_each_row<1, V, V>(d.binsAt, csr_at<V>(d), g, op, smem);
  double a[3] = {(double)op.acc[0], (double)op.acc[1], (double)op.acc[2]};
  block_sum_smem<3>(a, smem);
  if (threadIdx.x == 0) {
    double* part = d.partials + (size_t)blockIdx.x * kMaxPartials;
    part[0] = a[0]; part[1] = a[1]; part[2] = a[2];
  }
}

// Step control (single thread): adaptive step test of Eq. (6) in the T^-1 /
// Sigma^-1 weighted norms, next step size, buffer swap, online-update scalars.
// Works on a register copy of the state and writes it back once.
__device__ void step_control(const Dev& d, const Params& prm, const double (&t1)[3], const double (&t2)[4]) {
  DevState s = *d.st;
  const double eta = s.eta, omega = s.omega;
  const bool collect = s.collect;
  s.pend_p = 0;  // applied by this attempt's kernels
  s.pend_d = 0;
  s.attempts += 1;
  bool accept = true;
  double eta_next = eta;
  if (prm.mode == kPdlp) {
    const double movement = omega * t1[0] + t2[0] / omega;
    const double interaction = fabs(t2[1]);
    const double eta_max = interaction > 0.0 ? movement / (2.0 * interaction) : INFINITY;
    accept = eta <= eta_max;
    const long long t = s.attempts;
    double f1, f2;
    if (t < kStepTab) {
      f1 = __ldg(d.step_tab + t);
      f2 = __ldg(d.step_tab + kStepTab + t);
    } else {
      f1 = 1.0 - pow((double)t + 1.0, -0.3);
      f2 = 1.0 + pow((double)t + 1.0, -0.6);
    }
    eta_next = fmin(f1 * eta_max, f2 * eta);
    s.last_eta_max = eta_max;
  }
  if (accept) {
    if (collect) {
      if (!prm.normalize || t1[1] > 0.0) {
        const double sc = -(eta / omega) * (prm.normalize ? 1.0 / t1[1] : 1.0);
        s.up_scale_p = sc;
        s.pend_p = 1;
        if (prm.sched == kAdagradNorm) s.gp_norm += sc * sc * t1[2];
      }
      if (!prm.normalize || t2[2] > 0.0) {
        const double sc = -(eta * omega) * (prm.normalize ? 1.0 / t2[2] : 1.0);
        s.up_scale_d = sc;
        s.pend_d = 1;
        if (prm.sched == kAdagradNorm) s.gd_norm += sc * sc * t2[3];
      }
    }
    if (prm.mode == kPdlp) s.wsum += eta;
    s.cur ^= 1;
    s.k += 1;
  }
  s.eta = eta_next;
  s.last_accept = accept ? 1 : 0;
  s.counter = 0;
  refresh_derived(s, prm.phi);
  *d.st = s;
}

template <class V>
__global__ void __launch_bounds__(kBlock) dual_step_kernel(Dev d, Params prm) {
  __shared__ double smem[kBlock * 4];
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
  for_each_row<1, V, V>(d.binsA, csr_a<V>(d), g, op, smem);
  double a[4] = {(double)op.acc[0], (double)op.acc[1], (double)op.acc[2], (double)op.acc[3]};
  block_sum_smem<4>(a, smem);
  __shared__ int s_last;
  if (threadIdx.x == 0) {
    double* part = d.partials2 + (size_t)blockIdx.x * kMaxPartials;
    part[0] = a[0]; part[1] = a[1]; part[2] = a[2]; part[3] = a[3];
    __threadfence();
    const unsigned int t = atomicAdd(&d.st->counter, 1u);
    s_last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  double t1[3], t2[4];
  sum_partials<3>(d.partials, d.gridAt, t1, smem);
  sum_partials<4>(d.partials2, d.gridA, t2, smem);
  if (threadIdx.x == 0) step_control(d, prm, t1, t2);
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
  if (fp32) primal_step_kernel<float><<<d.gridAt, kBlock, 0, s>>>(d, prm);
  else primal_step_kernel<double><<<d.gridAt, kBlock, 0, s>>>(d, prm);
}

void launch_dual(const Dev& d, const Params& prm, bool fp32, cudaStream_t s) {
  if (fp32) dual_step_kernel<float><<<d.gridA, kBlock, 0, s>>>(d, prm);
  else dual_step_kernel<double><<<d.gridA, kBlock, 0, s>>>(d, prm);
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

// Resident blocks per SM of the two step kernels (they size the grids; the
// FP64 instances use more registers, so their occupancy bounds both).
void row_kernel_blocks_per_sm(int* primal, int* dual) {
  int a = 0, b = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, primal_step_kernel<double>, kBlock, 0) != cudaSuccess || a < 1)
    a = 1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, dual_step_kernel<double>, kBlock, 0) != cudaSuccess || b < 1)
    b = 1;
  *primal = a;
  *dual = b;
}

}  // namespace lpop
