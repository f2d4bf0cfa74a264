// Batched solves: many LPs advance together in one persistent launch.
//
// Each member is an ordinary problem (lp_create: its own preprocessed data
// and device-resident state).  One launch of batch_round_kernel runs every
// listed member for up to `attempts` step attempts of Algorithm 1 (checks and
// restarts included), entirely on the device.  The work is split by nonzero
// count: members with at least `wide_nnz` nonzeros are solved by a whole
// thread-block cluster of C CTAs (a "wide" team: rows split over the CTAs,
// reductions combined over distributed shared memory in rank order, hardware
// cluster barriers between the phases), the others by single CTAs.  Members
// are assigned to teams longest-first by nonzero count.  The team's CTAs hold
// the member's solver state in shared memory and run the same single-thread
// control code, so their decisions agree exactly.
#include <cooperative_groups.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <cstring>
#include <numeric>
#include <string>
#include <thread>
#include <vector>

#include "../../include/lpop.h"
#include "common.cuh"
#include "host_layout.hpp"
#include "ops.cuh"
#include "spmv.cuh"

namespace cg = cooperative_groups;

namespace lpop {

struct MemberView {
  Dev d;
  Params prm;
  cudaStream_t stream;
  int device;
  bool mixed;
};
int member_view(lp_problem* p, MemberView* out);                 // api.cu
int member_after_batch(lp_problem* p, const DevState& s);         // api.cu
void set_thread_error(const std::string& msg);                    // api.cu

namespace {

struct Member {
  Dev d;
  Params prm;
};

constexpr int kSlots = 32;  // team partial slots: primal 3 | dual 4 | check 10 + 8

template <int N>
__device__ void team_reduce(double (&v)[N], double* blk, double* slot, int T, bool wide) {
  if (N <= 4) block_sum_smem<N>(v, blk);
  else block_sum<N>(v, blk);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int q = 0; q < N; ++q) slot[q] = v[q];
  }
  if (wide) cg::this_cluster().sync();
  else __syncthreads();
  double tot[N];
#pragma unroll
  for (int q = 0; q < N; ++q) tot[q] = 0.0;
  if (wide) {
    cg::cluster_group cl = cg::this_cluster();
    for (int r = 0; r < T; ++r) {
      const double* rs = cl.map_shared_rank(slot, r);
#pragma unroll
      for (int q = 0; q < N; ++q) tot[q] += rs[q];
    }
  } else {
#pragma unroll
    for (int q = 0; q < N; ++q) tot[q] = slot[q];
  }
#pragma unroll
  for (int q = 0; q < N; ++q) v[q] = tot[q];
}

__device__ __forceinline__ void team_sync(bool wide) {
  if (wide) cg::this_cluster().sync();
  else __syncthreads();
}

struct StoreRowOp {
  double* y;
  __device__ __forceinline__ void prefetch(int) {}
  __device__ __forceinline__ void row(int r, const double (&s)[1]) { y[r] = s[0]; }
};

// KKT check, termination / restart decision and its application (a team-wide
// version of the check kernels).
template <class V>
__device__ void team_check(const Dev& d, const Params& prm, DevState& s, int rank, int T, bool wide, double* blk,
                           double* slots, int eval_only = 0) {
  const Vecs<V>& v = vecs<V>(d);
  const int cur = s.cur;
  const bool avg = prm.mode == kPdlp && s.wsum > 0.0;
  double p1[10], p2[8];
  if (prm.mode == kPdlp) {
    CheckPrimalOp<2, V> op;
    op.c = v.c; op.l = v.l; op.u = v.u; op.inv_dc = d.inv_dc;
    op.xc = v.x[cur]; op.xbarc = v.xbar[cur]; op.xlast = v.x_last;
    op.inv_w = s.wsum > 0.0 ? 1.0 / s.wsum : 0.0;
    op.avg = avg;
#pragma unroll
    for (int q = 0; q < 10; ++q) op.acc[q] = 0.0;
    Gather<2, V> g;
    g.x[0] = v.y[cur];
    g.x[1] = v.ybar[cur];
    g.n = d.m;
    g.bad = d.bad_gathers;
    for_each_row_range<2, V, double>(d.binsAt, csr_at<V>(d), g, op, blk, rank, T);
#pragma unroll
    for (int q = 0; q < 10; ++q) p1[q] = op.acc[q];
  } else {
    CheckPrimalOp<1, V> op;
    op.c = v.c; op.l = v.l; op.u = v.u; op.inv_dc = d.inv_dc;
    op.xc = v.x[cur]; op.xbarc = v.xbar[cur]; op.xlast = v.x_last;
    op.inv_w = s.wsum > 0.0 ? 1.0 / s.wsum : 0.0;
    op.avg = 0;
#pragma unroll
    for (int q = 0; q < 10; ++q) op.acc[q] = 0.0;
    Gather<1, V> g;
    g.x[0] = v.y[cur];
    g.n = d.m;
    g.bad = d.bad_gathers;
    for_each_row_range<1, V, double>(d.binsAt, csr_at<V>(d), g, op, blk, rank, T);
#pragma unroll
    for (int q = 0; q < 10; ++q) p1[q] = op.acc[q];
  }
  team_reduce<10>(p1, blk, slots + 7, T, wide);
  {
    CheckDualOp<V> op;
    op.b = v.b; op.inv_dr = d.inv_dr; op.sense = d.sense;
    op.axc = v.ax[cur]; op.yc = v.y[cur]; op.ybarc = v.ybar[cur]; op.ylast = v.y_last;
    op.ax_avg = v.ax_avg;
    op.inv_w = s.wsum > 0.0 ? 1.0 / s.wsum : 0.0;
    op.avg = avg;
#pragma unroll
    for (int q = 0; q < 8; ++q) op.acc[q] = 0.0;
    if (prm.mode == kPdlp) {
      Gather<1, V> g;
      g.x[0] = v.xbar[cur];
      g.n = d.n;
      g.bad = d.bad_gathers;
      for_each_row_range<1, V, double>(d.binsA, csr_a<V>(d), g, op, blk, rank, T);
    } else {
      const double s0[1] = {0.0};
      for (int i = rank * blockDim.x + threadIdx.x; i < d.m; i += T * blockDim.x) op.row(i, s0);
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) p2[q] = op.acc[q];
  }
  team_reduce<8>(p2, blk, slots + 17, T, wide);
  if (threadIdx.x == 0) {
    check_control(&s, prm, p1, p2, eval_only, avg ? 1 : 0);
    refresh_derived(s, prm.phi, prm.sched);
  }
  __syncthreads();
  apply_decision<V>(d, s, rank * blockDim.x + threadIdx.x, T * blockDim.x);
  team_sync(wide);
}

// FP32 iterate -> FP64 iterate, then A x recomputed in FP64.
__device__ void team_promote(const Dev& d, const DevState& s, int rank, int T, bool wide, double* blk) {
  const Vecs<float>& a = d.f32;
  const Vecs<double>& b = d.f64;
  const int cur = s.cur;
  const int start = rank * blockDim.x + threadIdx.x, stride = T * blockDim.x;
  for (int j = start; j < d.n; j += stride) {
    b.x[cur][j] = a.x[cur][j];
    b.xbar[cur][j] = a.xbar[cur][j];
    b.T[j] = a.T[j];
    b.invT[j] = 1.0 / b.T[j];
    b.GT[j] = a.GT[j];
    b.q[j] = a.q[j];
    b.x_last[j] = a.x_last[j];
  }
  for (int i = start; i < d.m; i += stride) {
    b.y[cur][i] = a.y[cur][i];
    b.ybar[cur][i] = a.ybar[cur][i];
    b.S[i] = a.S[i];
    b.invS[i] = 1.0 / b.S[i];
    b.GS[i] = a.GS[i];
    b.p[i] = a.p[i];
    b.y_last[i] = a.y_last[i];
    b.ax_avg[i] = a.ax_avg[i];
  }
  team_sync(wide);
  StoreRowOp op{b.ax[cur]};
  Gather<1, double> g;
  g.x[0] = b.x[cur];
  g.n = d.n;
  g.bad = d.bad_gathers;
  for_each_row_range<1, double, double>(d.binsA, d.A, g, op, blk, rank, T);
  team_sync(wide);
}

// The FP32 phase reached the tolerance against the FP32 copy of A~: end the
// phase and let an FP64 termination test of the promoted point decide.
__device__ void team_certify(const Dev& d, const Params& prm, DevState& s, int rank, int T, bool wide, double* blk,
                             double* slots) {
  if (threadIdx.x == 0) {
    s.status = 0;
    s.phase32 = 0;
  }
  __syncthreads();
  team_promote(d, s, rank, T, wide, blk);
  team_check<double>(d, prm, s, rank, T, wide, blk, slots, 2);
}

// Up to `budget` step attempts of one member in precision V.  Returns true when
// the member handed over from FP32 to FP64 with attempts left.
template <class V>
__device__ bool team_round(const Member& mb, DevState& s, int& budget, int rank, int T, bool wide, double* blk,
                           double* slots) {
  const Dev& d = mb.d;
  const Params& prm = mb.prm;
  const Vecs<V>& v = vecs<V>(d);
  if (!s.initial_checked) {
    team_check<V>(d, prm, s, rank, T, wide, blk, slots);
    if (sizeof(V) == sizeof(float) && s.status == 1) {
      team_certify(d, prm, s, rank, T, wide, blk, slots);
      return s.status == 0 && budget > 0;
    }
    if (s.status != 0) return false;
  }
  while (budget > 0 && s.status == 0) {
    double t1[3], t2[4];
    {
      PrimalOp<V> op;
      op.sc = read_scalars<V>(&s, true);
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
      for_each_row_range<1, V, V>(d.binsAt, csr_at<V>(d), g, op, blk, rank, T);
      t1[0] = op.acc[0]; t1[1] = op.acc[1]; t1[2] = op.acc[2];
    }
    team_reduce<3>(t1, blk, slots + 0, T, wide);
    {
      DualOp<V> op;
      op.sc = read_scalars<V>(&s, false);
      const int cur = op.sc.cur, nxt = cur ^ 1;
      op.prm = prm;
      op.b = v.b; op.sense = d.sense;
      op.axc = v.ax[cur]; op.yc = v.y[cur]; op.ybarc = v.ybar[cur];
      op.S = v.S; op.invS = v.invS; op.GS = v.GS; op.p = v.p;
      op.yn = v.y[nxt]; op.axn = v.ax[nxt]; op.ybarn = v.ybar[nxt];
      op.acc[0] = op.acc[1] = op.acc[2] = op.acc[3] = V(0);
      Gather<1, V> g;
      g.x[0] = v.x[nxt];
      g.n = d.n;
      g.bad = d.bad_gathers;
      for_each_row_range<1, V, V>(d.binsA, csr_a<V>(d), g, op, blk, rank, T);
      t2[0] = op.acc[0]; t2[1] = op.acc[1]; t2[2] = op.acc[2]; t2[3] = op.acc[3];
    }
    team_reduce<4>(t2, blk, slots + 3, T, wide);
    if (threadIdx.x == 0) {
      double f1, f2;
      step_factors(d.step_tab, s.attempts + 1, &f1, &f2);
      step_control_state(s, prm, f1, f2, t1, t2);
    }
    __syncthreads();
    --budget;
    if (s.attempts % prm.check_every == 0) {
      team_check<V>(d, prm, s, rank, T, wide, blk, slots);
      if (sizeof(V) == sizeof(float) && s.status == 1) {
        team_certify(d, prm, s, rank, T, wide, blk, slots);
        return s.status == 0 && budget > 0;
      }
      if (s.status != 0) break;
      if (sizeof(V) == sizeof(float) && s.phase32) {
        // mixed precision hand-over: at refine_tol, or after refine_stall checks without a 10% gain
        if (threadIdx.x == 0) {
          const double kkt = fmax(s.rel_pres, fmax(s.rel_dres, s.rel_gap));
          if (kkt < 0.9 * s.best_kkt) {
            s.best_kkt = kkt;
            s.stall = 0;
          } else {
            s.stall += 1;
          }
          if (kkt <= prm.refine_tol || s.stall >= prm.refine_stall || !isfinite(kkt)) s.phase32 = 0;
        }
        __syncthreads();
        if (!s.phase32) {
          team_promote(d, s, rank, T, wide, blk);
          return budget > 0;
        }
      }
    }
  }
  return false;
}

__global__ void __launch_bounds__(kBlock) batch_round_kernel(const Member* members, const int* queue,
                                                             const int* cta_q0, const int* cta_q1,
                                                             const int* cluster_wide, int C, int attempts) {
  __shared__ Member mb;
  __shared__ DevState s;
  __shared__ double slots[kSlots];
  __shared__ double blk[kBlock * 4];
  const int cid = blockIdx.x / C;
  const int crank = blockIdx.x % C;
  const bool wide = C > 1 && cluster_wide[cid] != 0;
  const int T = wide ? C : 1;
  const int rank = wide ? crank : 0;
  const int q0 = cta_q0[blockIdx.x], q1 = cta_q1[blockIdx.x];
  for (int qi = q0; qi < q1; ++qi) {
    const int id = queue[qi];
    {
      const int* src = reinterpret_cast<const int*>(members + id);
      int* dst = reinterpret_cast<int*>(&mb);
      for (int w = threadIdx.x; w < (int)(sizeof(Member) / sizeof(int)); w += blockDim.x) dst[w] = src[w];
    }
    __syncthreads();
    if (threadIdx.x == 0) s = *mb.d.st;
    __syncthreads();
    int budget = attempts;
    if (s.status == 0) {
      if (s.phase32) {
        if (team_round<float>(mb, s, budget, rank, T, wide, blk, slots))
          team_round<double>(mb, s, budget, rank, T, wide, blk, slots);
      } else {
        team_round<double>(mb, s, budget, rank, T, wide, blk, slots);
      }
    }
    if (rank == 0 && threadIdx.x == 0) *mb.d.st = s;
    team_sync(wide);
  }
}

// Copies every member's solver state into one array (one read-back per round).
__global__ void gather_states_kernel(const Member* members, int count, DevState* out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) out[i] = *members[i].d.st;
}

// Sets the tolerance of the listed members and re-opens them (status 0).
__global__ void set_tolerance_kernel(const Member* members, const int* ids, int count, double tol) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
    DevState* st = members[ids[i]].d.st;
    st->tol = tol;
    st->status = 0;
  }
}

}  // namespace
}  // namespace lpop

using namespace lpop;

struct lp_batch {
  int device = 0;
  cudaStream_t stream = nullptr;  // owned by the batch, created on `device`
  int stream_device = -1;
  std::vector<lp_problem*> probs;
  std::vector<Member> host_members;
  std::vector<long long> nnz;
  Member* d_members = nullptr;
  int member_cap = 0;
  int* d_sched = nullptr;  // queue | cta_q0 | cta_q1 | cluster_wide
  size_t sched_cap = 0;
  DevState* d_states = nullptr;
  std::vector<DevState> states;
  int cluster = 1;
  long long wide_nnz = (1LL << 62);
  // lp_batch_solve: a member still open after `handoff` attempts (0: never)
  // finishes on the single-problem kernels, on its own stream and host
  // thread, while the batch goes on with the others
  long long handoff = 0;
  std::vector<char> handed;
  int sms = 0;
  long long launches = 0;
  std::string err;
};

namespace {

int berr(lp_batch* b, int code, const std::string& msg) {
  if (b) b->err = msg;
  set_thread_error(msg);
  return code;
}

#define BCK(call)                                                                                   \
  do {                                                                                              \
    cudaError_t e_ = (call);                                                                        \
    if (e_ != cudaSuccess) return berr(b, LP_ERR_CUDA, std::string(#call) + " failed: " + cudaGetErrorString(e_)); \
  } while (0)

int load_members(lp_batch* b, int count, lp_problem* const* members) {
  b->probs.assign(members, members + count);
  b->host_members.resize(count);
  b->nnz.resize(count);
  for (int i = 0; i < count; ++i) {
    MemberView v;
    if (!members[i]) return berr(b, LP_ERR_INVALID_ARG, "member " + std::to_string(i) + " is NULL");
    int rc = member_view(members[i], &v);
    if (rc != LP_OK) return berr(b, rc, "member " + std::to_string(i) + ": cannot read its device layout");
    if (i == 0) {
      b->device = v.device;
    } else if (v.device != b->device) {
      return berr(b, LP_ERR_INVALID_ARG, "all members must live on one device");
    }
    // the batch's kernels run on its own stream: a member's earlier work on its stream comes first
    BCK(cudaSetDevice(v.device));
    BCK(cudaStreamSynchronize(v.stream));
    b->host_members[i].d = v.d;
    // a team walks all of a member's units with its own threads: full units of kBlock rows
    set_sliced_unit_rows(b->host_members[i].d.binsA, kBlock);
    set_sliced_unit_rows(b->host_members[i].d.binsAt, kBlock);
    b->host_members[i].prm = v.prm;
    b->nnz[i] = v.d.nnz;
  }
  BCK(cudaSetDevice(b->device));
  if (b->stream && b->stream_device != b->device) {
    cudaSetDevice(b->stream_device);
    cudaStreamSynchronize(b->stream);
    cudaStreamDestroy(b->stream);
    b->stream = nullptr;
    BCK(cudaSetDevice(b->device));
  }
  if (!b->stream) {
    BCK(cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking));
    b->stream_device = b->device;
  }
  if (count > b->member_cap || !b->d_members) {  // grow only: a serving loop reloads members every round
    if (b->d_members) cudaFree(b->d_members);
    if (b->d_states) cudaFree(b->d_states);
    b->d_members = nullptr;
    b->d_states = nullptr;
    b->member_cap = count > 0 ? count : 1;
    BCK(cudaMalloc(&b->d_members, sizeof(Member) * b->member_cap));
    BCK(cudaMalloc(&b->d_states, sizeof(DevState) * b->member_cap));
  }
  if (count > 0)
    BCK(cudaMemcpyAsync(b->d_members, b->host_members.data(), sizeof(Member) * count, cudaMemcpyHostToDevice,
                        b->stream));
  BCK(cudaStreamSynchronize(b->stream));
  b->states.resize(count);
  return LP_OK;
}

int read_states(lp_batch* b) {
  const int count = (int)b->probs.size();
  if (count == 0) return LP_OK;
  gather_states_kernel<<<(count + 255) / 256, 256, 0, b->stream>>>(b->d_members, count, b->d_states);
  BCK(cudaGetLastError());
  BCK(cudaMemcpyAsync(b->states.data(), b->d_states, sizeof(DevState) * count, cudaMemcpyDeviceToHost, b->stream));
  BCK(cudaStreamSynchronize(b->stream));
  b->launches += 1;
  return LP_OK;
}

// Longest-first assignment of the active members: those with >= wide_nnz
// nonzeros to wide clusters, the rest to single CTAs; each team's load is its
// members' nonzero counts divided by the team size.
int build_schedule(lp_batch* b, const std::vector<int>& active, int total_ctas, std::vector<int>& h) {
  const int C = b->cluster;
  const int nclusters = total_ctas / C;
  std::vector<int> wide, narrow;
  for (int id : active) (C > 1 && b->nnz[id] >= b->wide_nnz ? wide : narrow).push_back(id);
  auto by_nnz = [&](int a, int c) { return b->nnz[a] > b->nnz[c]; };
  std::sort(wide.begin(), wide.end(), by_nnz);
  std::sort(narrow.begin(), narrow.end(), by_nnz);
  double wide_work = 0, narrow_work = 0;
  for (int id : wide) wide_work += (double)b->nnz[id] + 1.0;
  for (int id : narrow) narrow_work += (double)b->nnz[id] + 1.0;
  int nwide = 0;
  if (!wide.empty()) {
    nwide = (int)std::lround(nclusters * wide_work / (wide_work + narrow_work));
    nwide = std::max(1, std::min(nwide, std::min((int)wide.size(), nclusters - (narrow.empty() ? 0 : 1))));
    if (nwide < 1) nwide = 1;
  }
  // teams: wide clusters first (one team each), then every CTA of the remaining clusters
  const int nteams_narrow = (nclusters - nwide) * C;
  std::vector<std::vector<int>> wlist(nwide), nlist(std::max(nteams_narrow, 0));
  std::vector<double> wload(nwide, 0.0), nload(nlist.size(), 0.0);
  for (int id : wide) {
    const int t = (int)(std::min_element(wload.begin(), wload.end()) - wload.begin());
    wlist[t].push_back(id);
    wload[t] += (double)b->nnz[id] / C + 1.0;
  }
  for (int id : narrow) {
    if (nlist.empty()) {
      return berr(b, LP_ERR_INVALID_ARG, "no single-CTA teams left for the small members");
    }
    const int t = (int)(std::min_element(nload.begin(), nload.end()) - nload.begin());
    nlist[t].push_back(id);
    nload[t] += (double)b->nnz[id] + 1.0;
  }
  // flatten: queue | cta_q0[total_ctas] | cta_q1[total_ctas] | cluster_wide[nclusters]
  std::vector<int> queue, q0(total_ctas, 0), q1(total_ctas, 0), cw(nclusters, 0);
  for (int c = 0; c < nwide; ++c) {
    const int a = (int)queue.size();
    queue.insert(queue.end(), wlist[c].begin(), wlist[c].end());
    for (int r = 0; r < C; ++r) {
      q0[c * C + r] = a;
      q1[c * C + r] = (int)queue.size();
    }
    cw[c] = 1;
  }
  for (int t = 0; t < nteams_narrow; ++t) {
    const int cta = nwide * C + t;
    q0[cta] = (int)queue.size();
    queue.insert(queue.end(), nlist[t].begin(), nlist[t].end());
    q1[cta] = (int)queue.size();
  }
  h.clear();
  h.push_back((int)queue.size());
  h.insert(h.end(), queue.begin(), queue.end());
  h.insert(h.end(), q0.begin(), q0.end());
  h.insert(h.end(), q1.begin(), q1.end());
  h.insert(h.end(), cw.begin(), cw.end());
  return LP_OK;
}

int launch_round(lp_batch* b, const std::vector<int>& active, int attempts) {
  if (active.empty()) return LP_OK;
  const int C = b->cluster;
  // CTAs: as many clusters as fit at once (persistent)
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.blockDim = dim3(kBlock, 1, 1);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = b->stream;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int max_clusters = 0;
  cfg.gridDim = dim3(C, 1, 1);
  cudaError_t e = cudaOccupancyMaxActiveClusters(&max_clusters, batch_round_kernel, &cfg);
  if (e != cudaSuccess || max_clusters < 1)
    return berr(b, LP_ERR_CUDA, std::string("cluster size ") + std::to_string(C) + " cannot be launched: " +
                                    cudaGetErrorString(e));
  const int total = max_clusters * C;
  std::vector<int> h;
  int rc = build_schedule(b, active, total, h);
  if (rc != LP_OK) return rc;
  if (h.size() > b->sched_cap) {
    if (b->d_sched) cudaFree(b->d_sched);
    b->d_sched = nullptr;
    b->sched_cap = h.size() * 2;
    BCK(cudaMalloc(&b->d_sched, sizeof(int) * b->sched_cap));
  }
  BCK(cudaMemcpyAsync(b->d_sched, h.data(), sizeof(int) * h.size(), cudaMemcpyHostToDevice, b->stream));
  const int qn = h[0];
  const int* queue = b->d_sched + 1;
  const int* q0 = queue + qn;
  const int* q1 = q0 + total;
  const int* cw = q1 + total;
  cfg.gridDim = dim3(total, 1, 1);
  BCK(cudaLaunchKernelEx(&cfg, batch_round_kernel, (const Member*)b->d_members, queue, q0, q1, cw, C, attempts));
  b->launches += 1;
  return LP_OK;
}

std::vector<int> active_members(lp_batch* b, long long iter_limit) {
  std::vector<int> act;
  for (int i = 0; i < (int)b->probs.size(); ++i) {
    if (!b->handed.empty() && b->handed[i]) continue;
    if (b->states[i].status == 0 && b->states[i].attempts < iter_limit) act.push_back(i);
  }
  return act;
}

int sync_members(lp_batch* b) {
  for (int i = 0; i < (int)b->probs.size(); ++i) {
    if (!b->handed.empty() && b->handed[i]) continue;  // its own solve keeps it current
    int rc = member_after_batch(b->probs[i], b->states[i]);
    if (rc != LP_OK) return berr(b, rc, "member " + std::to_string(i) + ": state refresh failed");
  }
  return LP_OK;
}

}  // namespace

extern "C" {

int lp_batch_create(int32_t count, lp_problem* const* members, lp_batch** out) {
  if (!out) return berr(nullptr, LP_ERR_INVALID_ARG, "out must not be NULL");
  *out = nullptr;
  if (count < 0 || (count > 0 && !members)) return berr(nullptr, LP_ERR_INVALID_ARG, "bad member list");
  lp_batch* b = new lp_batch();
  int sms = 0;
  cudaError_t e = cudaGetDevice(&b->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device);
  if (e != cudaSuccess) {
    delete b;
    return berr(nullptr, LP_ERR_CUDA, std::string("no usable CUDA device: ") + cudaGetErrorString(e));
  }
  b->sms = sms;
  int rc = load_members(b, count, members);
  if (rc != LP_OK) {
    lp_batch_destroy(b);
    return rc;
  }
  rc = read_states(b);
  if (rc != LP_OK) {
    lp_batch_destroy(b);
    return rc;
  }
  *out = b;
  return LP_OK;
}

int lp_batch_set_members(lp_batch* b, int32_t count, lp_problem* const* members) {
  if (!b) return berr(nullptr, LP_ERR_INVALID_ARG, "batch handle is NULL");
  if (count < 0 || (count > 0 && !members)) return berr(b, LP_ERR_INVALID_ARG, "bad member list");
  int rc = load_members(b, count, members);
  if (rc != LP_OK) return rc;
  return read_states(b);
}

int lp_batch_set_schedule(lp_batch* b, int32_t cluster_size, int64_t wide_nnz) {
  if (!b) return berr(nullptr, LP_ERR_INVALID_ARG, "batch handle is NULL");
  if (cluster_size != 1 && cluster_size != 2 && cluster_size != 4 && cluster_size != 8)
    return berr(b, LP_ERR_INVALID_ARG, "cluster_size must be 1, 2, 4 or 8");
  if (wide_nnz < 0) return berr(b, LP_ERR_INVALID_ARG, "wide_nnz must be >= 0");
  b->cluster = cluster_size;
  b->wide_nnz = wide_nnz;
  return LP_OK;
}

int lp_batch_round(lp_batch* b, double rel_kkt_tol, int32_t attempts, int64_t iter_limit, int32_t* active_out) {
  if (!b) return berr(nullptr, LP_ERR_INVALID_ARG, "batch handle is NULL");
  if (attempts < 1 || !(rel_kkt_tol >= 0.0)) return berr(b, LP_ERR_INVALID_ARG, "need attempts >= 1 and tol >= 0");
  NvtxRange range("lpop batch round");
  BCK(cudaSetDevice(b->device));
  const int count = (int)b->probs.size();
  if (count == 0) {
    if (active_out) *active_out = 0;
    return LP_OK;
  }
  int rc = read_states(b);
  if (rc != LP_OK) return rc;
  // members still running, and members that stopped under another tolerance
  std::vector<int> act;
  for (int i = 0; i < count; ++i) {
    if (!b->handed.empty() && b->handed[i]) continue;  // running on the single-problem path
    if (b->states[i].attempts < iter_limit && (b->states[i].status == 0 || b->states[i].tol != rel_kkt_tol))
      act.push_back(i);
  }
  if (act.empty()) {
    if (active_out) *active_out = 0;
    return sync_members(b);
  }
  int budget = attempts;
  for (int id : act) {
    const long long left = iter_limit - b->states[id].attempts;
    if (left < budget) budget = (int)left;
  }
  if (b->sched_cap < act.size() + 1) {
    if (b->d_sched) cudaFree(b->d_sched);
    b->d_sched = nullptr;
    b->sched_cap = 2 * (act.size() + 1);
    BCK(cudaMalloc(&b->d_sched, sizeof(int) * b->sched_cap));
  }
  BCK(cudaMemcpyAsync(b->d_sched, act.data(), sizeof(int) * act.size(), cudaMemcpyHostToDevice, b->stream));
  set_tolerance_kernel<<<((int)act.size() + 255) / 256, 256, 0, b->stream>>>(b->d_members, b->d_sched,
                                                                            (int)act.size(), rel_kkt_tol);
  BCK(cudaGetLastError());
  b->launches += 1;
  BCK(cudaStreamSynchronize(b->stream));  // the id list buffer is reused for the schedule
  rc = launch_round(b, act, budget);
  if (rc != LP_OK) return rc;
  rc = read_states(b);
  if (rc != LP_OK) return rc;
  rc = sync_members(b);
  if (rc != LP_OK) return rc;
  if (active_out) *active_out = (int)active_members(b, iter_limit).size();
  return LP_OK;
}

int lp_batch_solve(lp_batch* b, double rel_kkt_tol, int64_t iter_limit, int32_t round_attempts, int32_t* n_optimal) {
  if (!b) return berr(nullptr, LP_ERR_INVALID_ARG, "batch handle is NULL");
  if (round_attempts < 1) return berr(b, LP_ERR_INVALID_ARG, "round_attempts must be >= 1");
  const int count = (int)b->probs.size();
  b->handed.assign(count, 0);
  std::vector<int> worker_rc(count, LP_OK);
  // handed-off members wait in a queue for a bounded pool of host threads
  std::mutex mu;
  std::condition_variable cv;
  std::deque<int> queue;
  bool closed = false;
  std::vector<std::thread> workers;
  const unsigned hw = std::thread::hardware_concurrency();
  const size_t max_workers = std::min<size_t>(16, hw == 0 ? 4 : hw);
  const int dev = b->device;
  auto worker = [&]() {
    cudaSetDevice(dev);
    for (;;) {
      int i;
      {
        std::unique_lock<std::mutex> lk(mu);
        cv.wait(lk, [&] { return closed || !queue.empty(); });
        if (queue.empty()) return;
        i = queue.front();
        queue.pop_front();
      }
      worker_rc[i] = lp_solve(b->probs[i], rel_kkt_tol, iter_limit, nullptr);
    }
  };
  int rc = LP_OK;
  int active = 1;
  long long guard = 0;
  while (active > 0) {
    rc = lp_batch_round(b, rel_kkt_tol, round_attempts, iter_limit, &active);
    if (rc != LP_OK) break;
    if (b->handoff > 0) {
      // the rule depends only on the member's own attempts (round boundaries are
      // multiples of round_attempts), so its result does not depend on the mix
      for (int i = 0; i < count; ++i) {
        const DevState& st = b->states[i];
        if (b->handed[i] || st.status != 0 || st.attempts >= iter_limit || st.attempts < b->handoff) continue;
        b->handed[i] = 1;
        --active;
        {
          std::lock_guard<std::mutex> lk(mu);
          queue.push_back(i);
        }
        cv.notify_one();
        if (workers.size() < max_workers) workers.emplace_back(worker);
      }
    }
    if (++guard > 100000000) break;
  }
  {
    std::lock_guard<std::mutex> lk(mu);
    closed = true;
  }
  cv.notify_all();
  for (std::thread& t : workers) t.join();
  b->handed.clear();
  if (rc != LP_OK) return rc;
  for (int i = 0; i < count; ++i)
    if (worker_rc[i] != LP_OK) return berr(b, worker_rc[i], "member " + std::to_string(i) + ": single-problem solve failed");
  rc = read_states(b);
  if (rc != LP_OK) return rc;
  rc = sync_members(b);
  if (rc != LP_OK) return rc;
  if (n_optimal) {
    int k = 0;
    for (const DevState& s : b->states) k += s.status == 1;
    *n_optimal = k;
  }
  return LP_OK;
}

int lp_batch_set_handoff(lp_batch* b, int64_t attempts) {
  if (!b) return berr(nullptr, LP_ERR_INVALID_ARG, "batch handle is NULL");
  if (attempts < 0) return berr(b, LP_ERR_INVALID_ARG, "handoff attempts must be >= 0");
  b->handoff = attempts;
  return LP_OK;
}

// rounds of the autotuner's trial solves (the binding's default for lp_batch_solve)
constexpr int32_t kTuneRound = 256;

int lp_batch_autotune(lp_batch* b, double rel_kkt_tol, int32_t trial_attempts, int32_t* cluster_size,
                      int64_t* wide_nnz, double* trial_ms) {
  if (!b) return berr(nullptr, LP_ERR_INVALID_ARG, "batch handle is NULL");
  if (trial_attempts < 1) return berr(b, LP_ERR_INVALID_ARG, "trial_attempts must be >= 1");
  BCK(cudaSetDevice(b->device));
  const int count = (int)b->probs.size();
  if (count == 0) return LP_OK;
  // candidate wide thresholds: nonzero counts at the 50/80/95/99th percentiles (and "no wide teams")
  std::vector<long long> sorted(b->nnz);
  std::sort(sorted.begin(), sorted.end());
  std::vector<long long> thresholds = {1LL << 62};
  for (double q : {0.5, 0.8, 0.95, 0.99}) thresholds.push_back(sorted[(size_t)(q * (count - 1))]);
  double best = 1e300;
  int best_c = 1;
  long long best_w = 1LL << 62;
  for (int C : {1, 2, 4, 8}) {
    for (long long w : thresholds) {
      if (C == 1 && w != (1LL << 62)) continue;
      if (C > 1 && w == (1LL << 62)) continue;
      for (lp_problem* p : b->probs) {
        const int rc = lp_reset(p);
        if (rc != LP_OK) return berr(b, rc, "reset of a member failed");
      }
      int rc = read_states(b);
      if (rc != LP_OK) return rc;
      b->cluster = C;
      b->wide_nnz = w;
      BCK(cudaStreamSynchronize(b->stream));
      const auto t0 = std::chrono::steady_clock::now();
      rc = lp_batch_solve(b, rel_kkt_tol, trial_attempts, kTuneRound, nullptr);
      if (rc != LP_OK) {
        if (C > 1) continue;  // a cluster size the device cannot launch is skipped
        return rc;
      }
      const double ms = 1e3 * std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
      if (ms < best) {
        best = ms;
        best_c = C;
        best_w = w;
      }
    }
  }
  for (lp_problem* p : b->probs) {
    const int rc = lp_reset(p);
    if (rc != LP_OK) return berr(b, rc, "reset of a member failed");
  }
  int rc = read_states(b);
  if (rc != LP_OK) return rc;
  rc = sync_members(b);
  if (rc != LP_OK) return rc;
  b->cluster = best_c;
  b->wide_nnz = best_w;
  if (cluster_size) *cluster_size = best_c;
  if (wide_nnz) *wide_nnz = best_w;
  if (trial_ms) *trial_ms = best;
  return LP_OK;
}

int lp_batch_status(lp_batch* b, int32_t* status, int64_t* iterations) {
  if (!b) return berr(nullptr, LP_ERR_INVALID_ARG, "batch handle is NULL");
  int rc = read_states(b);
  if (rc != LP_OK) return rc;
  for (int i = 0; i < (int)b->states.size(); ++i) {
    if (status) status[i] = b->states[i].status == 1 ? LP_OPTIMAL : (b->states[i].status == 4 ? LP_NUMERICAL_ERROR : 0);
    if (iterations) iterations[i] = b->states[i].attempts;
  }
  return LP_OK;
}

int lp_batch_launches(const lp_batch* b, int64_t* launches) {
  if (!b || !launches) return berr(nullptr, LP_ERR_INVALID_ARG, "NULL argument");
  *launches = b->launches;
  return LP_OK;
}

void lp_batch_destroy(lp_batch* b) {
  if (!b) return;
  if (b->stream) {
    cudaSetDevice(b->stream_device);
    cudaStreamSynchronize(b->stream);
  }
  if (b->d_members) cudaFree(b->d_members);
  if (b->d_states) cudaFree(b->d_states);
  if (b->d_sched) cudaFree(b->d_sched);
  if (b->stream) cudaStreamDestroy(b->stream);
  delete b;
}

}  // extern "C"
