// Per-row operations and single-thread control logic of the method, shared
// by the single-problem kernels (kernels_iter.cu, kernels_check.cu) and the
// batched kernel (batch.cu).
//
//   PrimalOp / DualOp: epilogues of the two fused products of one step
//     attempt (Eq. (6)), with the pending online preconditioner update
//     (Eq. (7), Algorithm 1) applied to the row first.
//   step_control_state: adaptive step test and step size, buffer swap and
//     online-update scalars.
//   CheckPrimalOp / CheckDualOp / check_control: KKT quantities of the current
//     and averaged iterates, termination and restart decisions.
#pragma once

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

// Step control (single thread): adaptive step test of Eq. (6) in the T^-1 /
// Sigma^-1 weighted norms, next step size, buffer swap, online-update scalars.
// Works on a copy of the state held by the caller.
// f1, f2: step_factors() of attempt s.attempts + 1.
//
// It runs once per attempt in one thread of one block, so it is written for
// latency on GB300, where a dependent FP64 operation takes ~64 cycles, an
// FP64 min ~160 and a division ~550, and where the code runs with cold
// instruction caches: comparisons and the min are done on the integer bits
// of the (non-negative) operands, the mode is a template parameter, and the
// online-update scalars (once every phi accepted attempts) are set out of line.

// Bits of a double that is NaN (any sign).
__device__ __forceinline__ bool nan_bits(long long b) { return (b & 0x7fffffffffffffffLL) > 0x7ff0000000000000LL; }

// Accepted attempt that records q / p: scalars of the pending update of T and
// Sigma (Eq. (7), Algorithm 1; normalised by ||g||^2 and ||b - A x||^2).
__device__ __noinline__ void control_collect(DevState& s, int normalize, int sched, double eta, double omega,
                                             double inv_omega, double gp2, double q2, double rd2, double p2) {
  s.pend_p = 0;
  s.pend_d = 0;
  if (!normalize || gp2 > 0.0) {
    const double sc = -(eta * inv_omega) * (normalize ? 1.0 / gp2 : 1.0);
    s.up_scale_p = sc;
    s.pend_p = 1;
    if (sched == kAdagradNorm) s.gp_norm += sc * sc * q2;
  }
  if (!normalize || rd2 > 0.0) {
    const double sc = -(eta * omega) * (normalize ? 1.0 / rd2 : 1.0);
    s.up_scale_d = sc;
    s.pend_d = 1;
    if (sched == kAdagradNorm) s.gd_norm += sc * sc * p2;
  }
  if (sched == kAdagradNorm) {
    s.sqrt_gp = s.gp_norm > 0.0 ? sqrt(s.gp_norm) : 0.0;
    s.sqrt_gd = s.gd_norm > 0.0 ? sqrt(s.gd_norm) : 0.0;
  }
}

template <bool Pdlp>
__device__ inline void step_control_t(DevState& s, const Params& prm, double f1, double f2, const double (&t1)[3],
                                      const double (&t2)[4]) {
  const double eta = s.eta, omega = s.omega, inv_omega = s.inv_omega;
  const int collect = s.collect;
  bool accept = true;
  double eta_next = eta;
  if (Pdlp) {
    const double movement = omega * t1[0] + t2[0] * inv_omega;
    const double interaction = fabs(t2[1]);
    // no interaction (exactly 0): every step passes; a NaN interaction gives a
    // NaN limit, which rejects the attempt
    const long long ib = __double_as_longlong(interaction);
    const double eta_max = ib == 0 ? INFINITY : movement / (2.0 * interaction);
    // eta <= eta_max (both >= 0; false for NaN)
    const long long mb = __double_as_longlong(eta_max);
    accept = !nan_bits(mb) && __double_as_longlong(eta) <= mb;
    // fmin(f1 eta_max, f2 eta) (both >= 0)
    const double a = f1 * eta_max, b = f2 * eta;
    const long long ab = __double_as_longlong(a), bb = __double_as_longlong(b);
    eta_next = nan_bits(ab) ? b : (nan_bits(bb) ? a : (ab < bb ? a : b));
    s.last_eta_max = eta_max;
  }
  const int k_mod_next = s.k_mod + 1 == prm.phi ? 0 : s.k_mod + 1;
  s.pend_p = 0;  // applied by this attempt's kernels
  s.pend_d = 0;
  s.attempts += 1;
  if (accept) {
    if (Pdlp) s.wsum += eta;
    s.cur ^= 1;
    s.k += 1;
    if (prm.phi > 0) s.k_mod = k_mod_next;
  }
  s.eta = eta_next;
  s.last_accept = accept ? 1 : 0;
  s.counter = 0;
  // derived scalars (refresh_derived); the square roots of the AdaGrad-norm
  // sums change only where the sums do (control_collect)
  s.collect = prm.phi > 0 && s.k_mod == 0;
  s.step_p = eta_next * inv_omega;
  s.step_d = eta_next * omega;
  if (prm.sched != kAdagradNorm) {
    s.sqrt_gp = 0.0;
    s.sqrt_gd = 0.0;
  }
  if (accept && collect) control_collect(s, prm.normalize, prm.sched, eta, omega, inv_omega, t1[1], t1[2], t2[2], t2[3]);
}

__device__ inline void step_control_state(DevState& s, const Params& prm, double f1, double f2,
                                          const double (&t1)[3], const double (&t2)[4]) {
  if (prm.mode == kPdlp) step_control_t<true>(s, prm, f1, f2, t1, t2);
  else step_control_t<false>(s, prm, f1, f2, t1, t2);
}

// Vectors of type V (FP64, or FP32 in the mixed-precision phase); every
// quantity of the check is formed and summed in FP64.
template <int NV, class V>
struct CheckPrimalOp {
  const V *c, *l, *u, *xc, *xbarc, *xlast;
  const double* inv_dc;  // 1 / dc: user-unit dual residuals without a division per row
  double inv_w;          // 1 / (average weight)
  int avg;
  double acc[10];
  static constexpr bool kNoPair = true;  // one row per thread: no second set of 10 accumulators
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
    const double du = ds * __ldg(inv_dc + j);
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
    if (NV > 1 && avg) side(j, cj - s[NV - 1] * inv_w, (double)xbarc[j] * inv_w, acc + 5);
  }
};

template <class V>
struct CheckDualOp {
  const V *b, *axc, *yc, *ybarc, *ylast;
  const double* inv_dr;  // 1 / dr: user-unit primal residuals without a division per row
  const uint8_t* sense;
  V* ax_avg;
  double inv_w;  // 1 / (average weight)
  int avg;
  double acc[8];
  static constexpr bool kNoPair = true;
  __device__ __forceinline__ void prefetch(int) {}

  __device__ __forceinline__ void side(int i, double ax, double y, double* a) {
    const double bi = (double)__ldg(b + i);
    const double rs = ax - bi;
    const uint8_t sn = __ldg(sense + i);
    const double ps = sn == kEq ? rs : (sn == kGe ? fmax(-rs, 0.0) : fmax(rs, 0.0));
    const double pu = ps * __ldg(inv_dr + i);
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
      const double axa = s[0] * inv_w;
      ax_avg[i] = (V)axa;
      side(i, axa, (double)ybarc[i] * inv_w, acc + 4);
    }
  }
};

struct Cand {
  double pobj, dobj, rel_p, rel_d, rel_g, p2, d2, g2, dist_x2, dist_y2;
};

__device__ __forceinline__ double kw(double p2, double d2, double g2, double omega) {
  return sqrt(omega * omega * p2 + d2 / (omega * omega) + g2);
}

__device__ __forceinline__ bool converged(const Cand& c, double tol) {
  return c.rel_p <= tol && c.rel_d <= tol && c.rel_g <= tol;
}

// Check decision (single thread) from the KKT partial sums.  eval_only: 0 =
// full check (termination, then restart and primal weight), 1 = record the
// current iterate's KKT only, 2 = termination test only (no restart logic;
// confirms in FP64 a tolerance that the FP32 phase reported).
__device__ inline void check_control(DevState* st, const Params& prm, const double (&p1)[10], const double (&p2)[8],
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
  if (!eval_only) st->initial_checked = 1;
  st->pobj = cd[0].pobj; st->dobj = cd[0].dobj;
  st->rel_pres = cd[0].rel_p; st->rel_dres = cd[0].rel_d; st->rel_gap = cd[0].rel_g;
  st->stats_from_avg = 0;
  if (eval_only == 1) return;
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
  if (eval_only == 2) return;  // termination test only
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
  if (dx > 1e-10 && dy > 1e-10) {
    st->omega = exp(0.5 * log(dy / dx) + 0.5 * log(omega));
    st->inv_omega = 1.0 / st->omega;
  }
  st->restart_action = pick ? 2 : 1;
  st->apply_w = st->wsum;
  st->wsum = 0.0;
  st->klast_p2 = cd[pick].p2; st->klast_d2 = cd[pick].d2; st->klast_g2 = cd[pick].g2;
  st->last_restart_attempt = st->attempts;
  st->restarts += 1;
}

// Carry out a check's decision on the vectors (restart point, move to the
// average, zeroing of the averages) for indices start, start + stride, ...
template <class V>
__device__ inline void apply_decision(const Dev& d, const DevState& s, int start, int stride) {
  const int action = s.restart_action;
  const int adopt = s.adopt_avg;
  if (action == 0 && !adopt) return;
  const Vecs<V>& v = vecs<V>(d);
  const int cur = s.cur;
  const double w = s.apply_w;
  const bool to_avg = adopt || action == 2;
  const bool mark = action >= 1;
  const bool reset = action == 1 || action == 2;
  V *x = v.x[cur], *xb = v.xbar[cur], *y = v.y[cur], *yb = v.ybar[cur], *ax = v.ax[cur];
  for (int j = start; j < d.n; j += stride) {
    V val = x[j];
    if (to_avg) {
      val = (V)((double)xb[j] / w);
      x[j] = val;
    }
    if (mark) v.x_last[j] = val;
    if (reset) xb[j] = V(0);
  }
  for (int i = start; i < d.m; i += stride) {
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
}  // namespace lpop
