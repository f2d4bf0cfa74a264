// C ABI of the library (declared in include/lpop.h).
//
// lp_create validates on the host, copies the caller's arrays to the device
// once, builds the bin-ordered CSR copies of A and A^T there and runs the
// preprocessing kernels.  lp_solve drives the
// device-resident iteration: one check period (check_every step attempts and
// the KKT check) is captured once as a CUDA graph and replayed; the host only
// reads one status word per period.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <thread>
#include <string>
#include <vector>

#include "../../include/lpop.h"
#include "common.cuh"
#include "device_layout.hpp"
#include "host_layout.hpp"

using namespace lpop;

namespace lpop {
void launch_scatter_perm(double* out, const double* a, const double* f, const int* perm, int n, cudaStream_t s);
void launch_gather_perm(double* out, const double* a, const int* perm, int n, cudaStream_t s);
void row_kernel_blocks_per_sm(int* primal, int* dual, int* primal32, int* dual32);
}  // namespace lpop

static thread_local std::string g_last_error;

namespace lpop {
// Lets other translation units report an error through lp_last_error(NULL).
void set_thread_error(const std::string& msg) { g_last_error = msg; }
}  // namespace lpop

struct lp_problem {
  lp_options opt{};
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  Dev d{};
  Params prm{};
  std::vector<int> prow, pcol;
  int* d_prow = nullptr;  // the same permutations on the device
  int* d_pcol = nullptr;
  double eta0 = 1.0, omega0 = 1.0, norm_est = 0.0, amax = 0.0;
  long long nnz = 0;
  bool initial_check_done = false;
  bool solved_once = false;
  int last_status = LP_STATUS_NONE;
  double last_solve_ms = 0.0;
  long long host_attempts = 0;
  long long launches = 0;
  std::string err;
  cudaGraphExec_t gexec = nullptr;    // FP64 check period
  cudaGraphExec_t gexec32 = nullptr;  // FP32 check period (mixed precision)
  bool mixed = false;
  bool fp32_phase = false;  // mixed precision before the hand-over to FP64
  double best_kkt = INFINITY;
  int stall = 0;
  std::vector<cudaEvent_t> events;  // 3 per timed sample: before primal, between, after dual
  int samples = 0;
  double kt_ms[2] = {0.0, 0.0};
  long long kt_n[2] = {0, 0};
  int* h_status = nullptr;  // pinned
  double* h_scratch = nullptr;  // pinned, 8 doubles
  // device memory: one allocation of the lp_memory_bytes bound, handed out
  // by dalloc in 256-byte steps; anything beyond it gets its own allocation
  // (cudaMalloc, or the caller's device_alloc with its size kept for device_free)
  char* arena = nullptr;
  size_t arena_size = 0, arena_used = 0;
  std::vector<void*> allocs;
  std::vector<std::pair<void*, size_t>> ext_allocs;
  // sliced copies of the kSell bins of A (0) and A^T (1): entries, column
  // indices and values, filled on the device once the preprocessed values
  // are final
  long long sell_n[2] = {0, 0};
  RuizSplit ruiz[2] = {};  // how the Ruiz kernels cut the rows of A / A^T
  long long checks_seen = 0;  // KKT checks run by lp_solve since create (for log_every)
  int* sell_ci[2] = {nullptr, nullptr};
  double* sell_v[2] = {nullptr, nullptr};
  float* sell_v32[2] = {nullptr, nullptr};
};

namespace {

// Step-size schedule factors 1 - (t+1)^-0.3 and 1 + (t+1)^-0.6 of the adaptive
// step (PDLP rule) for t < kStepTab, computed once per device with the host
// libm pow and shared by every problem on that device.
std::mutex g_tab_mutex;
double* g_step_tab[64] = {nullptr};

const double* step_table(int dev, cudaStream_t s, cudaError_t* err) {
  std::lock_guard<std::mutex> lock(g_tab_mutex);
  *err = cudaSuccess;
  if (dev < 0 || dev >= 64) {
    *err = cudaErrorInvalidDevice;
    return nullptr;
  }
  if (!g_step_tab[dev]) {
    std::vector<double> h(2 * (size_t)kStepTab);
    // every entry on its own, so the host threads' split does not change the table
    auto fill = [&h](int t0, int t1) {
      for (int t = t0; t < t1; ++t) {
        const double tp1 = (double)t + 1.0;
        h[t] = 1.0 - std::pow(tp1, -0.3);
        h[kStepTab + t] = 1.0 + std::pow(tp1, -0.6);
      }
    };
    const unsigned hw = std::thread::hardware_concurrency();
    const int T = (int)std::min<unsigned>(hw == 0 ? 1u : hw, 8u);
    std::vector<std::thread> pool;
    for (int i = 1; i < T; ++i) pool.emplace_back(fill, (int)((long long)kStepTab * i / T), (int)((long long)kStepTab * (i + 1) / T));
    fill(0, (int)((long long)kStepTab / T));
    for (auto& th : pool) th.join();
    void* dptr = nullptr;
    *err = cudaMalloc(&dptr, h.size() * sizeof(double));
    if (*err != cudaSuccess) return nullptr;
    *err = cudaMemcpyAsync(dptr, h.data(), h.size() * sizeof(double), cudaMemcpyHostToDevice, s);
    if (*err == cudaSuccess) *err = cudaStreamSynchronize(s);
    if (*err != cudaSuccess) {
      cudaFree(dptr);
      return nullptr;
    }
    g_step_tab[dev] = static_cast<double*>(dptr);
  }
  return g_step_tab[dev];
}

int set_err(lp_problem* p, int code, const std::string& msg) {
  if (p) p->err = msg;
  g_last_error = msg;
  return code;
}

#define CK(call)                                                                              \
  do {                                                                                        \
    cudaError_t e_ = (call);                                                                  \
    if (e_ != cudaSuccess)                                                                    \
      return set_err(p, e_ == cudaErrorMemoryAllocation ? LP_ERR_OOM : LP_ERR_CUDA,           \
                     std::string(#call) + " failed: " + cudaGetErrorString(e_));              \
  } while (0)

template <class T>
int dalloc(lp_problem* p, T** ptr, size_t count) {
  *ptr = nullptr;
  if (count == 0) count = 1;
  const size_t bytes = (count * sizeof(T) + 255) / 256 * 256;
  if (p->arena && bytes <= p->arena_size - p->arena_used) {
    *ptr = reinterpret_cast<T*>(p->arena + p->arena_used);
    p->arena_used += bytes;
    return LP_OK;
  }
  void* v = nullptr;
  if (p->opt.device_alloc) {
    v = p->opt.device_alloc(bytes, p->opt.alloc_ctx);
    if (!v) return set_err(p, LP_ERR_OOM, "device_alloc of " + std::to_string(bytes) + " bytes returned NULL");
    if (reinterpret_cast<uintptr_t>(v) & 255u) {  // the kernels' vector loads need the 256-byte alignment
      p->opt.device_free(v, bytes, p->opt.alloc_ctx);
      return set_err(p, LP_ERR_INVALID_ARG, "device_alloc returned an address that is not 256-byte aligned");
    }
    p->ext_allocs.emplace_back(v, bytes);
    *ptr = static_cast<T*>(v);
    return LP_OK;
  }
  cudaError_t e = cudaMalloc(&v, count * sizeof(T));
  if (e != cudaSuccess) {
    return set_err(p, e == cudaErrorMemoryAllocation ? LP_ERR_OOM : LP_ERR_CUDA,
                   std::string("cudaMalloc of ") + std::to_string(count * sizeof(T)) + " bytes failed: " +
                       cudaGetErrorString(e));
  }
  p->allocs.push_back(v);
  *ptr = static_cast<T*>(v);
  return LP_OK;
}

#define TRY(expr)            \
  do {                       \
    int rc_ = (expr);        \
    if (rc_ != LP_OK) return rc_; \
  } while (0)

int check_options(const lp_options& o, std::string& msg) {
  if (o.mode != LP_MODE_PLAIN && o.mode != LP_MODE_PDLP) return msg = "mode must be LP_MODE_PLAIN or LP_MODE_PDLP", 1;
  if (o.scheduler < 0 || o.scheduler > 2) return msg = "unknown scheduler", 1;
  if (!(o.alpha >= 0.0) || !std::isfinite(o.alpha)) return msg = "alpha must be finite and >= 0", 1;
  if (!(o.precond_floor > 0.0) || !std::isfinite(o.precond_floor)) return msg = "precond_floor must be > 0", 1;
  if (o.ruiz_iters < 0 || o.ruiz_iters > 1000) return msg = "ruiz_iters must be in [0, 1000]", 1;
  if (!(o.pc_beta >= 0.0 && o.pc_beta <= 2.0)) return msg = "pc_beta must be in [0, 2]", 1;
  if (o.check_every < 1 || o.check_every > (1 << 16)) return msg = "check_every must be in [1, 65536]", 1;
  if (o.power_iters < 1) return msg = "power_iters must be >= 1", 1;
  if (!(o.plain_step_factor > 0.0)) return msg = "plain_step_factor must be > 0", 1;
  if (o.precision != LP_PREC_FP64 && o.precision != LP_PREC_MIXED) return msg = "unknown precision", 1;
  if (o.kernel_timing < 0) return msg = "kernel_timing must be >= 0", 1;
  if (!(o.refine_tol >= 0.0)) return msg = "refine_tol must be >= 0", 1;
  if (o.refine_stall < 1) return msg = "refine_stall must be >= 1", 1;
  if ((o.device_alloc == nullptr) != (o.device_free == nullptr))
    return msg = "device_alloc and device_free must be given together", 1;
  if (o.log_every < 0) return msg = "log_every must be >= 0", 1;
  return 0;
}

int select_device(lp_problem* p) {
  CK(cudaSetDevice(p->device));
  return LP_OK;
}

int read_status(lp_problem* p, int* status) {
  CK(cudaMemcpyAsync(p->h_status, &p->d.st->status, sizeof(int), cudaMemcpyDeviceToHost, p->stream));
  CK(cudaStreamSynchronize(p->stream));
  *status = *p->h_status;
  return LP_OK;
}

int init_state(lp_problem* p) {
  DevState s0;
  std::memset(&s0, 0, sizeof(s0));
  s0.cur = 0;
  s0.eta = p->eta0;
  s0.omega = p->omega0;
  s0.inv_omega = 1.0 / p->omega0;
  s0.tol = 1e-4;
  s0.k_prev = INFINITY;
  s0.phase32 = p->mixed ? 1 : 0;
  s0.best_kkt = INFINITY;
  refresh_derived(s0, p->prm.phi, p->prm.sched);
  CK(cudaMemcpyAsync(p->d.st, &s0, sizeof(s0), cudaMemcpyHostToDevice, p->stream));
  launch_init_vectors(p->d, p->stream);
  launch_spmv_binned(p->d.A, p->d.binsA, p->d.gridA, p->d.f64.x[0], p->d.f64.ax[0], p->stream);
  if (p->mixed) launch_demote_state(p->d, p->stream);
  CK(cudaGetLastError());
  p->fp32_phase = p->mixed;
  p->best_kkt = INFINITY;
  p->stall = 0;
  CK(cudaStreamSynchronize(p->stream));
  p->initial_check_done = false;
  p->solved_once = false;
  p->host_attempts = 0;
  p->launches = 0;
  p->kt_ms[0] = p->kt_ms[1] = 0.0;
  p->kt_n[0] = p->kt_n[1] = 0;
  p->last_status = LP_STATUS_NONE;
  return LP_OK;
}

double read_scalar(lp_problem* p, const double* dptr, int* rc) {
  cudaError_t e = cudaMemcpyAsync(p->h_scratch, dptr, sizeof(double), cudaMemcpyDeviceToHost, p->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
  if (e != cudaSuccess) {
    *rc = set_err(p, LP_ERR_CUDA, std::string("reading a device scalar failed: ") + cudaGetErrorString(e));
    return 0.0;
  }
  return p->h_scratch[0];
}

int preprocess(lp_problem* p) {
  NvtxRange range("lpop preprocess");
  Dev& d = p->d;
  cudaStream_t s = p->stream;
  const int m = d.m, n = d.n;
  double* fr = d.work;           // [m]
  double* fc = d.work + m;       // [n]
  double* red = d.work + m + n;  // reduction scratch [1 + 1024]
  launch_fill(d.dr, 1.0, m, s);
  launch_fill(d.dc, 1.0, n, s);
  auto apply = [&]() { launch_ruiz_apply(d, p->ruiz[0], p->ruiz[1], fr, fc, s); };
  for (int r = 0; r < p->opt.ruiz_iters; ++r) {
    launch_ruiz_norms(d, p->ruiz[0], p->ruiz[1], fr, fc, s);
    apply();
  }
  if (p->opt.mode == LP_MODE_PDLP) {
    launch_row_powsum(d.A, m, p->ruiz[0].nlong, p->ruiz[0].split, p->opt.pc_beta, 0, fr, s);
    launch_row_powsum(d.At, n, p->ruiz[1].nlong, p->ruiz[1].split, 2.0 - p->opt.pc_beta, 0, fc, s);
  } else {
    launch_row_powsum(d.A, m, p->ruiz[0].nlong, p->ruiz[0].split, 2.0, 1, fr, s);
    launch_row_powsum(d.At, n, p->ruiz[1].nlong, p->ruiz[1].split, 2.0, 1, fc, s);
  }
  apply();
  CK(cudaGetLastError());
  int rc = LP_OK;
  // norms of the caller's b and c (still unscaled), then rescale the vectors
  launch_norm2(d.f64.b, m, red, s);
  p->prm.b_norm = m > 0 ? read_scalar(p, red, &rc) : 0.0;
  TRY(rc);
  launch_norm2(d.f64.c, n, red, s);
  p->prm.c_norm = read_scalar(p, red, &rc);
  TRY(rc);
  launch_scale_problem_vectors(d, s);
  launch_norm2(d.f64.b, m, red, s);
  const double bn = m > 0 ? read_scalar(p, red, &rc) : 0.0;
  TRY(rc);
  launch_norm2(d.f64.c, n, red, s);
  const double cn = read_scalar(p, red, &rc);
  TRY(rc);
  p->omega0 = (bn > 0.0 && cn > 0.0) ? cn / bn : 1.0;
  if (p->nnz > 0) {
    launch_absmax(d.A_v, p->nnz, red, s);
    p->amax = read_scalar(p, red, &rc);
    TRY(rc);
  } else {
    p->amax = 0.0;
  }
  if (p->opt.mode == LP_MODE_PDLP) {
    p->eta0 = p->amax > 0.0 ? 1.0 / p->amax : 1.0;
  } else {
    // ||A~||_2 by power iteration on A~^T A~ from the all-ones direction; if
    // the first product is exactly zero (A~ 1 = 0), again from the +-1
    // direction of SplitMix64 signs of the caller's column index
    double* v = d.f64.q;       // [n]
    double* t = d.f64.ax_avg;  // [m]
    double* w = fc;        // [n]
    p->norm_est = 0.0;
    if (p->nnz > 0) {
      launch_fill(v, 1.0 / std::sqrt((double)n), n, s);
      bool restarted = false;
      for (int it = 0; it < p->opt.power_iters; ++it) {
        launch_spmv_binned(d.A, d.binsA, d.gridA, v, t, s);
        launch_spmv_binned(d.At, d.binsAt, d.gridAt, t, w, s);
        launch_norm2(w, n, red, s);
        if (it == 0 && !restarted) {
          const double nw0 = read_scalar(p, red, &rc);
          TRY(rc);
          if (nw0 == 0.0) {
            std::vector<double> h(n);
            const double sc = 1.0 / std::sqrt((double)n);
            for (int j = 0; j < n; ++j) h[j] = splitmix_sign((unsigned long long)p->pcol[j]) * sc;
            CK(cudaMemcpyAsync(v, h.data(), sizeof(double) * n, cudaMemcpyHostToDevice, s));
            CK(cudaStreamSynchronize(s));
            restarted = true;
            it = -1;
            continue;
          }
        }
        launch_scale_by_inv(w, n, red, s);
        CK(cudaMemcpyAsync(v, w, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
      }
      const double nw = read_scalar(p, red, &rc);
      TRY(rc);
      p->norm_est = nw > 0.0 && std::isfinite(nw) ? std::sqrt(nw) : 0.0;
    }
    p->eta0 = p->norm_est > 0.0 ? p->opt.plain_step_factor / p->norm_est : 1.0;
  }
  if (p->mixed) launch_make_fp32(d, s);
  // the values are final: fill the sliced copies, then let the kernels use them
  for (int which = 0; which < 2; ++which) {
    if (p->sell_n[which] == 0) continue;
    BinTable& bt = which ? d.binsAt : d.binsA;
    launch_fill_sliced(bt, which ? d.At_rp : d.A_rp, which ? d.At_ci : d.A_ci, which ? d.At_v : d.A_v,
                       p->sell_ci[which], p->sell_v[which], p->sell_n[which], s);
    if (p->mixed) launch_narrow(p->sell_v[which], p->sell_v32[which], p->sell_n[which], s);
    bt.sell_ci = p->sell_ci[which];
    bt.sell_v = p->sell_v[which];
    bt.sell_v32 = p->sell_v32[which];
  }
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(s));
  return LP_OK;
}

template <class V>
int alloc_vecs(lp_problem* p, Vecs<V>& v, int m, int n, bool values) {
  if (values) {
    TRY(dalloc(p, &v.Av, (size_t)p->d.nnz));
    TRY(dalloc(p, &v.Atv, (size_t)p->d.nnz));
  }
  // (vectors already allocated, like the FP64 b, c, l and u the layout build fills, are kept)
  V** vm[] = {&v.b, &v.y[0], &v.y[1], &v.ax[0], &v.ax[1], &v.ybar[0], &v.ybar[1],
              &v.S, &v.invS, &v.GS, &v.p, &v.y_last, &v.ax_avg};
  for (V** q : vm)
    if (!*q) TRY(dalloc(p, q, m));
  V** vn[] = {&v.c, &v.l, &v.u, &v.x[0], &v.x[1], &v.xbar[0], &v.xbar[1], &v.T, &v.invT, &v.GT, &v.q, &v.x_last};
  for (V** q : vn)
    if (!*q) TRY(dalloc(p, q, n));
  return LP_OK;
}

// Rows per sliced unit for a matrix whose units do not fill the grid: of
// 256, 224, ..., 128 rows per thread column (units of twice that for the
// two-rows-per-thread bins) the one (the largest on ties) that gives the
// busiest SM the fewest rows -- its blocks times the rows of a unit -- with
// every unit still resident at once.  The transport LP's 50,000 rows of A in
// 206 units of 256 rows put two units on 54 SMs (512 rows); 192-row units put
// at most 384 rows on an SM, and its 200,000 columns in units of 448 instead
// of 512 at most 1,344 instead of 1,536 (a check-free attempt: 24.4 instead
// of 26.0 us).  A matrix with
// at least a grid's worth of units keeps 256 (fewer rows per unit would only
// idle threads: 458 instead of 434 us per attempt on the power-law LP at 192).
int sliced_unit_rows(const BinTable& bt, int cap, int sms) {
  if (bt.nunits >= cap || sms < 1) return kBlock;
  int best = kBlock;
  long long best_load = -1;
  for (int rows = kBlock; rows >= 128; rows -= 32) {
    BinTable t = bt;
    set_sliced_unit_rows(t, rows);
    if (t.nunits > cap) continue;
    const long long load = (long long)((t.nunits + sms - 1) / sms) * rows;
    if (best_load < 0 || load < best_load) {
      best_load = load;
      best = rows;
    }
  }
  return best;
}

// Device buffers and the layout: the CSR copies of A and A^T and the vectors
// in bin order are built on the device from the caller's (valid, canonical)
// arrays, with scratch taken from the arena and given back afterwards.
int upload(lp_problem* p, int m, int n, long long nz, const int64_t* row_ptr, const int32_t* col_idx,
           const double* val, const double* b, const double* c, const double* lb, const double* ub,
           const char* sense) {
  Dev& d = p->d;
  d.m = m;
  d.n = n;
  TRY(dalloc(p, &d.A_rp, m + 1));
  TRY(dalloc(p, &d.A_ci, nz));
  TRY(dalloc(p, &d.A_v, nz));
  TRY(dalloc(p, &d.At_rp, n + 1));
  TRY(dalloc(p, &d.At_ci, nz));
  TRY(dalloc(p, &d.At_v, nz));
  d.nnz = nz;
  d.f64.Av = d.A_v;
  d.f64.Atv = d.At_v;
  TRY(dalloc(p, &d.f64.b, m));
  TRY(dalloc(p, &d.sense, m));
  TRY(dalloc(p, &d.f64.c, n));
  TRY(dalloc(p, &d.f64.l, n));
  TRY(dalloc(p, &d.f64.u, n));
  TRY(dalloc(p, &p->d_prow, m));
  TRY(dalloc(p, &p->d_pcol, n));
  LayoutInfo lay;
  {
    const size_t mark_used = p->arena_used, mark_allocs = p->allocs.size(), mark_ext = p->ext_allocs.size();
    const ScratchAlloc scratch = [p](void** ptr, size_t bytes) {
      char* q = nullptr;
      const int rc = dalloc(p, &q, bytes);
      *ptr = q;
      return rc;
    };
    const LayoutArrays arr{d.A_rp, d.A_ci, d.A_v, d.At_rp, d.At_ci, d.At_v, p->d_prow, p->d_pcol};
    const LayoutVectors vecs{b, c, lb, ub, sense, d.f64.b, d.f64.c, d.f64.l, d.f64.u, d.sense};
    std::string msg;
    NvtxRange range("lpop layout");
    // FP64 rows take one lane up to kSellMaxLen entries whatever the matrix size (widen 1):
    // extra lanes cost FP64 shuffle adds, which outweigh the added parallelism on GB300
    const int rc = build_layout_device(m, n, nz, row_ptr, col_idx, val, 1, 1, arr, &vecs, lay, scratch, p->stream, msg);
    // the scratch is dead once the build has returned: give it back
    cudaStreamSynchronize(p->stream);
    for (size_t k = mark_allocs; k < p->allocs.size(); ++k) cudaFree(p->allocs[k]);
    p->allocs.resize(mark_allocs);
    for (size_t k = mark_ext; k < p->ext_allocs.size(); ++k)
      p->opt.device_free(p->ext_allocs[k].first, p->ext_allocs[k].second, p->opt.alloc_ctx);
    p->ext_allocs.resize(mark_ext);
    p->arena_used = mark_used;
    if (rc != LP_OK) return set_err(p, rc, "layout build: " + msg);
  }
  p->prow = std::move(lay.prow);
  p->pcol = std::move(lay.pcol);
  TRY(dalloc(p, &d.dr, m));
  TRY(dalloc(p, &d.dc, n));
  TRY(dalloc(p, &d.inv_dr, m));
  TRY(dalloc(p, &d.inv_dc, n));
  TRY(alloc_vecs(p, d.f64, m, n, false));
  if (p->mixed) TRY(alloc_vecs(p, d.f32, m, n, true));
  TRY(dalloc(p, &d.work2, (size_t)(m > n ? m : n) + 1));
  TRY(dalloc(p, &d.work, (size_t)m + n + 2048));
  TRY(dalloc(p, &d.st, 1));
  TRY(dalloc(p, &d.bad_gathers, 1));
  CK(cudaMemsetAsync(d.bad_gathers, 0, sizeof(unsigned int), p->stream));
  {
    cudaError_t te = cudaSuccess;
    d.step_tab = step_table(p->device, p->stream, &te);
    if (!d.step_tab) return set_err(p, LP_ERR_CUDA, std::string("step-size table: ") + cudaGetErrorString(te));
  }

  int sms = 0;
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p->device));
  int per_sm_p = 1, per_sm_d = 1, per_sm_p32 = 1, per_sm_d32 = 1;
  row_kernel_blocks_per_sm(&per_sm_p, &per_sm_d, &per_sm_p32, &per_sm_d32);
  d.max_grid = sms * std::max(std::max(per_sm_p, per_sm_d), std::max(per_sm_p32, per_sm_d32));
  d.binsA = lay.binsA;
  d.binsAt = lay.binsAt;
  // grids from the unit counts; rows longer than half a block's share of the
  // work are then cut into segments, which adds units
  const int cap_d = sms * per_sm_d, cap_p = sms * per_sm_p;
  set_sliced_unit_rows(d.binsA, sliced_unit_rows(d.binsA, cap_d, sms));
  set_sliced_unit_rows(d.binsAt, sliced_unit_rows(d.binsAt, cap_p, sms));
  auto grid_of = [](int units, int cap) { return units < 1 ? 1 : (units < cap ? units : cap); };
  std::vector<int> segA = segment_long_rows(d.binsA, lay.A_head, segment_length(nz, grid_of(d.binsA.nunits, cap_d)));
  std::vector<int> segAt =
      segment_long_rows(d.binsAt, lay.At_head, segment_length(nz, grid_of(d.binsAt.nunits, cap_p)));
  d.gridA = grid_of(d.binsA.nunits, cap_d);
  d.gridAt = grid_of(d.binsAt.nunits, cap_p);
  d.gridA32 = grid_of(d.binsA.nunits, sms * per_sm_d32);
  d.gridAt32 = grid_of(d.binsAt.nunits, sms * per_sm_p32);
  for (int which = 0; which < 2; ++which) {
    BinTable& bt = which ? d.binsAt : d.binsA;
    const std::vector<int>& units = which ? segAt : segA;
    if (units.empty()) continue;
    int* su = nullptr;
    TRY(dalloc(p, &su, units.size()));
    TRY(dalloc(p, &bt.seg_sum, units.size()));
    TRY(dalloc(p, &bt.ticket, (size_t)bt.seg_rows));
    CK(cudaMemcpyAsync(su, units.data(), sizeof(int) * units.size(), cudaMemcpyHostToDevice, p->stream));
    CK(cudaMemsetAsync(bt.ticket, 0, sizeof(unsigned int) * bt.seg_rows, p->stream));
    bt.seg_unit = su;
  }
  for (int which = 0; which < 2; ++which) {  // Ruiz units: whole-block rows in chunks, then warp and thread rows
    const std::vector<int>& head = which ? lay.At_head : lay.A_head;
    RuizSplit& rs = p->ruiz[which];
    rs.split = lay.split[which];
    rs.nlong = head.empty() ? 0 : (int)head.size() - 1;
    rs.nchunks = 0;
    rs.chunk_pre = nullptr;
    if (rs.nlong == 0) continue;
    std::vector<int> pre((size_t)rs.nlong + 1, 0);
    for (int r = 0; r < rs.nlong; ++r) pre[r + 1] = pre[r] + (head[r + 1] - head[r] + kRuizChunk - 1) / kRuizChunk;
    rs.nchunks = pre[rs.nlong];
    int* dp = nullptr;
    TRY(dalloc(p, &dp, pre.size()));
    CK(cudaMemcpyAsync(dp, pre.data(), sizeof(int) * pre.size(), cudaMemcpyHostToDevice, p->stream));
    CK(cudaStreamSynchronize(p->stream));
    rs.chunk_pre = dp;
  }
  for (int which = 0; which < 2; ++which) {  // sliced copies: filled on the device once the values are final
    const long long ns = sliced_entries(which ? d.binsAt : d.binsA);
    p->sell_n[which] = ns;
    if (ns == 0) continue;
    TRY(dalloc(p, &p->sell_ci[which], (size_t)ns));
    TRY(dalloc(p, &p->sell_v[which], (size_t)ns));
    if (p->mixed) TRY(dalloc(p, &p->sell_v32[which], (size_t)ns));
  }
  CK(cudaStreamSynchronize(p->stream));
  const int rows_a = std::max(partial_rows_a<double>(d), partial_rows_a<float>(d));
  const int rows_at = std::max(partial_rows_at<double>(d), partial_rows_at<float>(d));
  const int maxg = rows_a > rows_at ? rows_a : rows_at;
  TRY(dalloc(p, &d.partials, (size_t)maxg * kMaxPartials));
  TRY(dalloc(p, &d.partials2, (size_t)maxg * kMaxPartials));
  d.A = Csr{d.A_rp, d.A_ci, d.A_v};
  d.At = Csr{d.At_rp, d.At_ci, d.At_v};
  return LP_OK;
}

// Attempts per timed sample: kernel_timing 1 times one attempt in 8, k >= 2 one in k.
int timing_stride(const lp_problem* p) { return p->opt.kernel_timing == 1 ? 8 : p->opt.kernel_timing; }

int create_events(lp_problem* p) {
  if (!p->opt.kernel_timing) return LP_OK;
  p->samples = (p->opt.check_every - 1) / timing_stride(p) + 1;  // attempts 0, stride, ... of a period
  p->events.resize(3 * p->samples, nullptr);
  for (auto& e : p->events) CK(cudaEventCreate(&e));
  return LP_OK;
}

bool sampled(const lp_problem* p, int a) { return p->opt.kernel_timing && (a % timing_stride(p)) == 0; }

int capture_graph(lp_problem* p, bool fp32) {
  cudaGraphExec_t* slot = fp32 ? &p->gexec32 : &p->gexec;
  if (*slot) return LP_OK;
  cudaGraph_t g = nullptr;
  CK(cudaStreamBeginCapture(p->stream, cudaStreamCaptureModeThreadLocal));
  const int ce = p->opt.check_every;
  for (int a = 0; a < ce; ++a) {
    const bool tm = sampled(p, a);
    const int sidx = a / (p->opt.kernel_timing ? timing_stride(p) : 1);
    if (tm) cudaEventRecordWithFlags(p->events[3 * sidx], p->stream, cudaEventRecordExternal);
    launch_primal(p->d, p->prm, fp32, p->stream);
    if (tm) cudaEventRecordWithFlags(p->events[3 * sidx + 1], p->stream, cudaEventRecordExternal);
    launch_dual(p->d, p->prm, fp32, p->stream);
    if (tm) cudaEventRecordWithFlags(p->events[3 * sidx + 2], p->stream, cudaEventRecordExternal);
  }
  launch_check(p->d, p->prm, 0, fp32, p->stream);
  cudaError_t e = cudaStreamEndCapture(p->stream, &g);
  if (e != cudaSuccess) return set_err(p, LP_ERR_CUDA, std::string("graph capture failed: ") + cudaGetErrorString(e));
  e = cudaGraphInstantiate(slot, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    *slot = nullptr;
    return set_err(p, LP_ERR_CUDA, std::string("graph instantiation failed: ") + cudaGetErrorString(e));
  }
  return LP_OK;
}

int collect_times(lp_problem* p) {
  if (!p->opt.kernel_timing) return LP_OK;
  for (int sidx = 0; sidx < p->samples; ++sidx) {
    float a = 0.f, b = 0.f;
    CK(cudaEventElapsedTime(&a, p->events[3 * sidx], p->events[3 * sidx + 1]));
    CK(cudaEventElapsedTime(&b, p->events[3 * sidx + 1], p->events[3 * sidx + 2]));
    p->kt_ms[0] += a;
    p->kt_ms[1] += b;
    p->kt_n[0] += 1;
    p->kt_n[1] += 1;
  }
  return LP_OK;
}

int download_vec(lp_problem* p, const double* dsrc, const double* dscale, int len, const int* dperm, double* out);

// The current phase's copy of a vector as FP64 on the device (FP32 vectors are widened into work2).
const double* phase_vec(lp_problem* p, const double* v64, const float* v32, int len) {
  if (!p->fp32_phase) return v64;
  launch_widen(p->d.work2, v32, len, p->stream);
  return p->d.work2;
}

// A device vector in the caller's order (out[perm[i]] = src[i], times
// scale[i] when given), put together on the device and copied into out.
int download_vec(lp_problem* p, const double* dsrc, const double* dscale, int len, const int* dperm, double* out) {
  if (!out || len == 0) return LP_OK;
  double* tmp = p->d.work;  // [m + n + 2048] >= len
  launch_scatter_perm(tmp, dsrc, dscale, dperm, len, p->stream);
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(out, tmp, sizeof(double) * len, cudaMemcpyDeviceToHost, p->stream));
  CK(cudaStreamSynchronize(p->stream));
  return LP_OK;
}

// The caller's vector into a device vector in bin order (dst[i] = host[perm[i]]).
int upload_vec(lp_problem* p, double* ddst, const double* host, int len, const int* dperm) {
  if (len == 0) return LP_OK;
  double* tmp = p->d.work;  // [m + n + 2048] >= len
  CK(cudaMemcpyAsync(tmp, host, sizeof(double) * len, cudaMemcpyHostToDevice, p->stream));
  launch_gather_perm(ddst, tmp, dperm, len, p->stream);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(p->stream));
  return LP_OK;
}

int get_state_impl(lp_problem* p, double* vn, double* vm, double* scal) {
  TRY(select_device(p));
  launch_flush_update(p->d, p->prm, p->fp32_phase, p->stream);
  CK(cudaGetLastError());
  DevState hs;
  CK(cudaMemcpyAsync(&hs, p->d.st, sizeof(hs), cudaMemcpyDeviceToHost, p->stream));
  CK(cudaStreamSynchronize(p->stream));
  const int n = p->d.n, m = p->d.m, c = hs.cur;
  const Dev& d = p->d;
  if (vn) {
    const double* s64[5] = {d.f64.x[c], d.f64.xbar[c], d.f64.T, d.f64.GT, d.f64.x_last};
    const float* s32[5] = {d.f32.x[c], d.f32.xbar[c], d.f32.T, d.f32.GT, d.f32.x_last};
    for (int k = 0; k < 5; ++k)
      TRY(download_vec(p, phase_vec(p, s64[k], s32[k], n), nullptr, n, p->d_pcol, vn + (size_t)k * n));
  }
  if (vm) {
    const double* s64[6] = {d.f64.y[c], d.f64.ybar[c], d.f64.ax[c], d.f64.S, d.f64.GS, d.f64.y_last};
    const float* s32[6] = {d.f32.y[c], d.f32.ybar[c], d.f32.ax[c], d.f32.S, d.f32.GS, d.f32.y_last};
    for (int k = 0; k < 6; ++k)
      TRY(download_vec(p, phase_vec(p, s64[k], s32[k], m), nullptr, m, p->d_prow, vm + (size_t)k * m));
  }
  if (scal) {
    const double v[16] = {hs.eta, hs.omega, hs.wsum, hs.gp_norm, hs.gd_norm, hs.klast_p2, hs.klast_d2,
                          hs.klast_g2, hs.k_prev, (double)hs.k, (double)hs.attempts,
                          (double)hs.last_restart_attempt, (double)hs.restarts, (double)hs.checked0,
                          p->initial_check_done ? 1.0 : 0.0, 0.0};
    std::memcpy(scal, v, sizeof(v));
  }
  return LP_OK;
}

int set_state_impl(lp_problem* p, const double* vn, const double* vm, const double* scal) {
  if (!(std::isfinite(scal[0]) && scal[0] > 0.0 && std::isfinite(scal[1]) && scal[1] > 0.0))
    return set_err(p, LP_ERR_INVALID_INPUT, "state: eta and omega must be finite and positive");
  TRY(select_device(p));
  CK(cudaStreamSynchronize(p->stream));
  DevState hs;
  CK(cudaMemcpyAsync(&hs, p->d.st, sizeof(hs), cudaMemcpyDeviceToHost, p->stream));
  CK(cudaStreamSynchronize(p->stream));
  const int n = p->d.n, m = p->d.m, c = hs.cur;
  const Dev& d = p->d;
  double* dn[5] = {d.f64.x[c], d.f64.xbar[c], d.f64.T, d.f64.GT, d.f64.x_last};
  for (int k = 0; k < 5; ++k) TRY(upload_vec(p, dn[k], vn + (size_t)k * n, n, p->d_pcol));
  double* dm[6] = {d.f64.y[c], d.f64.ybar[c], d.f64.ax[c], d.f64.S, d.f64.GS, d.f64.y_last};
  for (int k = 0; k < 6; ++k) TRY(upload_vec(p, dm[k], vm + (size_t)k * m, m, p->d_prow));
  hs.eta = scal[0];
  hs.omega = scal[1];
  hs.inv_omega = 1.0 / hs.omega;
  hs.wsum = scal[2];
  hs.gp_norm = scal[3];
  hs.gd_norm = scal[4];
  hs.klast_p2 = scal[5];
  hs.klast_d2 = scal[6];
  hs.klast_g2 = scal[7];
  hs.k_prev = scal[8];
  hs.k = (long long)scal[9];
  hs.k_mod = p->prm.phi > 0 ? (int)(hs.k % p->prm.phi) : 0;
  hs.attempts = (long long)scal[10];
  hs.last_restart_attempt = (long long)scal[11];
  hs.restarts = (long long)scal[12];
  hs.checked0 = scal[13] != 0.0;
  hs.pend_p = hs.pend_d = 0;
  hs.status = 0;
  hs.counter = 0;
  hs.restart_action = 0;
  hs.adopt_avg = 0;
  hs.initial_checked = scal[14] != 0.0;
  hs.phase32 = p->fp32_phase ? 1 : 0;
  refresh_derived(hs, p->prm.phi, p->prm.sched);
  CK(cudaMemcpyAsync(p->d.st, &hs, sizeof(hs), cudaMemcpyHostToDevice, p->stream));
  launch_inverse_preconditioners(p->d, false, p->stream);
  if (p->fp32_phase) launch_demote_state(p->d, p->stream);  // the FP32 phase continues from the imported state
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(p->stream));
  p->host_attempts = hs.attempts;
  p->initial_check_done = scal[14] != 0.0;
  p->solved_once = false;
  return LP_OK;
}

void release(lp_problem* p) {
  if (!p) return;
  cudaSetDevice(p->device);
  if (p->stream) cudaStreamSynchronize(p->stream);
  if (p->gexec) cudaGraphExecDestroy(p->gexec);
  if (p->gexec32) cudaGraphExecDestroy(p->gexec32);
  for (auto e : p->events)
    if (e) cudaEventDestroy(e);
  for (void* v : p->allocs) cudaFree(v);
  for (const auto& a : p->ext_allocs) p->opt.device_free(a.first, a.second, p->opt.alloc_ctx);
  if (p->arena) {
    if (p->opt.device_alloc) p->opt.device_free(p->arena, p->arena_size, p->opt.alloc_ctx);
    else cudaFree(p->arena);
  }
  if (p->h_status) cudaFreeHost(p->h_status);
  if (p->h_scratch) cudaFreeHost(p->h_scratch);
  if (p->own_stream && p->stream) cudaStreamDestroy(p->stream);
  delete p;
}

int create_impl(int32_t m, int32_t n, int64_t nnz, const int64_t* row_ptr, const int32_t* col_idx,
                const double* val, const double* b, const double* c, const double* lb, const double* ub,
                const char* sense, const lp_options* opt, lp_problem** out) {
  lp_problem* p = nullptr;
  if (!out) return set_err(nullptr, LP_ERR_INVALID_ARG, "out must not be NULL");
  *out = nullptr;
  lp_options o;
  if (opt) o = *opt;
  else lp_options_default(&o);
  std::string msg;
  if (check_options(o, msg)) return set_err(nullptr, LP_ERR_INVALID_ARG, msg);
  if (m < 0 || n < 1) return set_err(nullptr, LP_ERR_INVALID_ARG, "need m >= 0 and n >= 1");
  if ((m > 0 && (!b || !sense)) || !c || !lb || !ub)
    return set_err(nullptr, LP_ERR_INVALID_ARG, "b, c, lb, ub and sense must not be NULL");
  // the first offending row, then the first offending column (on host
  // threads; the tests are combined with | so that a scan has no branches)
  auto bad_row = [&](long long i) -> bool {
    const char sn = sense[i];
    return !std::isfinite(b[i]) | ((sn != 'E') & (sn != 'L') & (sn != 'G'));
  };
  auto bad_bounds = [&](long long j) -> bool {
    const double l = lb[j], u = ub[j];
    return std::isnan(l) | std::isnan(u) | (l == INFINITY) | (u == -INFINITY) | (l > u);
  };
  const long long i0 = first_bad_index(m, bad_row);
  if (i0 < m) {
    if (!std::isfinite(b[i0])) return set_err(nullptr, LP_ERR_INVALID_INPUT, "b[" + std::to_string(i0) + "] is not finite");
    return set_err(nullptr, LP_ERR_INVALID_INPUT, "sense[" + std::to_string(i0) + "] must be 'E', 'L' or 'G'");
  }
  const long long j0 = first_bad_index(n, [&](long long j) -> bool { return !std::isfinite(c[j]) | bad_bounds(j); });
  if (j0 < n) {
    if (!std::isfinite(c[j0])) return set_err(nullptr, LP_ERR_INVALID_INPUT, "c[" + std::to_string(j0) + "] is not finite");
    return set_err(nullptr, LP_ERR_INVALID_INPUT,
                   "bounds of variable " + std::to_string(j0) + " are invalid (need lb <= ub, lb < inf, ub > -inf)");
  }
  bool canonical = true;
  int rc = validate_csr(m, n, nnz, row_ptr, col_idx, val, canonical, msg);
  if (rc != LP_OK) return set_err(nullptr, rc, msg);
  // rows out of column order or with repeated entries: sorted and merged (summed) here first
  std::vector<int64_t> rp_m;
  std::vector<int> ci_m;
  std::vector<double> cv_m;
  if (!canonical) merge_rows(m, row_ptr, col_idx, val, rp_m, ci_m, cv_m);
  const int64_t* rp = canonical ? row_ptr : rp_m.data();
  const int32_t* ci = canonical ? col_idx : ci_m.data();
  const double* cv = canonical ? val : cv_m.data();
  const long long nz = canonical ? (long long)nnz : (long long)ci_m.size();

  p = new lp_problem();
  p->opt = o;
  p->mixed = o.precision == LP_PREC_MIXED;
  p->nnz = nz;
  auto fail = [&](int code) {
    g_last_error = p->err;
    release(p);
    return code;
  };
  cudaError_t e = cudaSuccess;
  if (o.device >= 0) e = cudaSetDevice(o.device);
  if (e == cudaSuccess) e = cudaGetDevice(&p->device);
  if (e != cudaSuccess) {
    set_err(p, LP_ERR_CUDA, std::string("no usable CUDA device: ") + cudaGetErrorString(e));
    return fail(LP_ERR_CUDA);
  }
  if (o.stream) {
    p->stream = static_cast<cudaStream_t>(o.stream);
  } else {
    e = cudaStreamCreateWithFlags(&p->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      set_err(p, LP_ERR_CUDA, std::string("stream creation failed: ") + cudaGetErrorString(e));
      return fail(LP_ERR_CUDA);
    }
    p->own_stream = true;
  }
  if (cudaMallocHost(&p->h_status, sizeof(int)) != cudaSuccess ||
      cudaMallocHost(&p->h_scratch, 8 * sizeof(double)) != cudaSuccess) {
    set_err(p, LP_ERR_OOM, "pinned host allocation failed");
    return fail(LP_ERR_OOM);
  }
  p->prm.m = m;
  p->prm.n = n;
  p->prm.mode = o.mode;
  p->prm.sched = o.scheduler;
  p->prm.phi = o.phi;
  p->prm.normalize = o.normalize ? 1 : 0;
  p->prm.restart = o.restart ? 1 : 0;
  p->prm.check_every = o.check_every;
  p->prm.alpha = o.alpha;
  p->prm.floor = o.precond_floor;
  p->prm.refine_tol = o.refine_tol;
  p->prm.refine_stall = o.refine_stall;
  {
    int64_t bytes = 0;
    if (lp_memory_bytes(m, n, nz, &o, &bytes) == LP_OK && bytes > 0) {
      void* a = nullptr;
      if (o.device_alloc) {
        a = o.device_alloc((size_t)bytes, o.alloc_ctx);
        if (!a) {
          set_err(p, LP_ERR_OOM, "device_alloc of " + std::to_string(bytes) + " bytes returned NULL");
          return fail(LP_ERR_OOM);
        }
        if (reinterpret_cast<uintptr_t>(a) & 255u) {  // buffers are carved from it in 256-byte steps
          o.device_free(a, (size_t)bytes, o.alloc_ctx);
          set_err(p, LP_ERR_INVALID_ARG, "device_alloc returned an address that is not 256-byte aligned");
          return fail(LP_ERR_INVALID_ARG);
        }
        p->arena = static_cast<char*>(a);
        p->arena_size = (size_t)bytes;
      } else if (cudaMalloc(&a, (size_t)bytes) == cudaSuccess) {
        p->arena = static_cast<char*>(a);
        p->arena_size = (size_t)bytes;
      } else {
        cudaGetLastError();  // no room for one block: every buffer gets its own cudaMalloc
      }
    }
  }
  if ((rc = upload(p, m, n, nz, rp, ci, cv, b, c, lb, ub, sense)) != LP_OK) return fail(rc);
  if ((rc = preprocess(p)) != LP_OK) return fail(rc);
  if ((rc = create_events(p)) != LP_OK) return fail(rc);
  if ((rc = init_state(p)) != LP_OK) return fail(rc);
  *out = p;
  return LP_OK;
}

// Relative KKT error (max of the three ratios) of the last check's point.
int read_kkt(lp_problem* p, double* kkt) {
  CK(cudaMemcpyAsync(p->h_scratch, &p->d.st->pobj, 5 * sizeof(double), cudaMemcpyDeviceToHost, p->stream));
  CK(cudaStreamSynchronize(p->stream));
  const double* v = p->h_scratch;  // pobj, dobj, rel_pres, rel_dres, rel_gap
  *kkt = std::fmax(v[2], std::fmax(v[3], v[4]));
  return LP_OK;
}

// Mixed precision: after a check in the FP32 phase, hand over to FP64 once the
// relative KKT error is at most refine_tol or after refine_stall checks without a 10% gain.
int maybe_refine(lp_problem* p) {
  if (!p->fp32_phase) return LP_OK;
  double kkt = 0.0;
  TRY(read_kkt(p, &kkt));
  if (kkt < 0.9 * p->best_kkt) {
    p->best_kkt = kkt;
    p->stall = 0;
  } else {
    p->stall += 1;
  }
  if (kkt <= p->opt.refine_tol || p->stall >= p->opt.refine_stall || !std::isfinite(kkt)) {
    launch_promote_state(p->d, p->stream);
    CK(cudaGetLastError());
    *p->h_status = 0;
    CK(cudaMemcpyAsync(&p->d.st->phase32, p->h_status, sizeof(int), cudaMemcpyHostToDevice, p->stream));
    CK(cudaStreamSynchronize(p->stream));
    p->launches += 2;
    p->fp32_phase = false;
  }
  return LP_OK;
}

// A tolerance reached in the FP32 phase is measured against the FP32 copy of
// A~; it ends the FP32 phase instead, and an FP64 termination test of the
// promoted point decides.
int certify_fp32(lp_problem* p, int* status) {
  if (!p->fp32_phase || *status != 1) return LP_OK;
  launch_promote_state(p->d, p->stream);
  CK(cudaGetLastError());
  p->h_status[0] = 0;
  CK(cudaMemcpyAsync(&p->d.st->phase32, p->h_status, sizeof(int), cudaMemcpyHostToDevice, p->stream));
  CK(cudaMemcpyAsync(&p->d.st->status, p->h_status, sizeof(int), cudaMemcpyHostToDevice, p->stream));
  p->fp32_phase = false;
  launch_check(p->d, p->prm, 2, false, p->stream);
  CK(cudaGetLastError());
  p->launches += 2 + check_kernel_count();
  return read_status(p, status);
}

// One line on stderr per log_every checks: the state the last check left.
int maybe_log(lp_problem* p) {
  if (p->opt.log_every <= 0 || ++p->checks_seen % p->opt.log_every != 0) return LP_OK;
  DevState hs;
  CK(cudaMemcpyAsync(&hs, p->d.st, sizeof(hs), cudaMemcpyDeviceToHost, p->stream));
  CK(cudaStreamSynchronize(p->stream));
  std::fprintf(stderr,
               "lpop: attempts %lld accepted %lld restarts %lld rel_pres %.3e rel_dres %.3e rel_gap %.3e "
               "pobj %.10g dobj %.10g eta %.4e omega %.4e %s\n",
               hs.attempts, hs.k, hs.restarts, hs.rel_pres, hs.rel_dres, hs.rel_gap, hs.pobj, hs.dobj, hs.eta,
               hs.omega, p->fp32_phase ? "fp32" : "fp64");
  return LP_OK;
}

int solve_impl(lp_problem* p, double tol, int64_t iter_limit, int32_t* status_out) {
  TRY(select_device(p));
  const auto t0 = std::chrono::steady_clock::now();
  const int ce = p->opt.check_every;
  // tolerance and a cleared status for this call
  p->h_scratch[0] = tol;
  CK(cudaMemcpyAsync(&p->d.st->tol, p->h_scratch, sizeof(double), cudaMemcpyHostToDevice, p->stream));
  *p->h_status = 0;
  CK(cudaMemcpyAsync(&p->d.st->status, p->h_status, sizeof(int), cudaMemcpyHostToDevice, p->stream));
  int status = 0;
  if (!p->initial_check_done) {
    launch_check(p->d, p->prm, 0, p->fp32_phase, p->stream);
    CK(cudaGetLastError());
    p->launches += check_kernel_count();
    p->initial_check_done = true;
    TRY(read_status(p, &status));
    TRY(certify_fp32(p, &status));
    TRY(maybe_log(p));
  }
  int out_status = LP_STATUS_NONE;
  while (status == 0 && p->host_attempts < iter_limit) {
    NvtxRange period("lpop check period");
    const bool fp32 = p->fp32_phase;
    const long long to_boundary = ce - p->host_attempts % ce;
    const long long remaining = iter_limit - p->host_attempts;
    bool checked = false;
    if (p->opt.use_graph && to_boundary == ce && remaining >= ce) {
      TRY(capture_graph(p, fp32));
      CK(cudaGraphLaunch(fp32 ? p->gexec32 : p->gexec, p->stream));
      p->launches += 2LL * ce + check_kernel_count();
      p->host_attempts += ce;
      checked = true;
      TRY(read_status(p, &status));
      TRY(collect_times(p));
    } else {
      const long long nrun = to_boundary < remaining ? to_boundary : remaining;
      for (long long a = 0; a < nrun; ++a) {
        launch_primal(p->d, p->prm, fp32, p->stream);
        launch_dual(p->d, p->prm, fp32, p->stream);
      }
      CK(cudaGetLastError());
      p->launches += 2 * nrun;
      p->host_attempts += nrun;
      if (p->host_attempts % ce == 0) {
        launch_check(p->d, p->prm, 0, fp32, p->stream);
        CK(cudaGetLastError());
        p->launches += check_kernel_count();
        checked = true;
      }
      TRY(read_status(p, &status));
    }
    TRY(certify_fp32(p, &status));
    if (checked) TRY(maybe_log(p));
    if (status == 0 && checked) TRY(maybe_refine(p));
    if (p->opt.time_limit > 0.0) {
      const double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
      if (status == 0 && el > p->opt.time_limit) {
        out_status = LP_TIME_LIMIT;
        break;
      }
    }
  }
  if (status == 1) out_status = LP_OPTIMAL;
  else if (status == 4) out_status = LP_NUMERICAL_ERROR;
  else if (out_status == LP_STATUS_NONE) out_status = LP_ITERATION_LIMIT;
  if ((out_status == LP_ITERATION_LIMIT || out_status == LP_TIME_LIMIT) && p->host_attempts % ce != 0) {
    launch_check(p->d, p->prm, 1, p->fp32_phase, p->stream);
    CK(cudaGetLastError());
    p->launches += check_kernel_count();
  }
  CK(cudaStreamSynchronize(p->stream));
  p->last_status = out_status;
  p->solved_once = true;
  p->last_solve_ms = 1e3 * std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (status_out) *status_out = out_status;
  return LP_OK;
}

}  // namespace

namespace lpop {

struct MemberView {
  Dev d;
  Params prm;
  cudaStream_t stream;
  int device;
  bool mixed;
};

// Device layout of a problem, for the batched kernel.
int member_view(lp_problem* p, MemberView* out) {
  if (!p || !out) return LP_ERR_INVALID_ARG;
  out->d = p->d;
  out->prm = p->prm;
  out->stream = p->stream;
  out->device = p->device;
  out->mixed = p->mixed;
  return LP_OK;
}

// Host-side view of a problem after a batched kernel advanced its device state.
int member_after_batch(lp_problem* p, const DevState& s) {
  if (!p) return LP_ERR_INVALID_ARG;
  p->host_attempts = s.attempts;
  p->initial_check_done = s.initial_checked != 0;
  p->fp32_phase = s.phase32 != 0;
  p->solved_once = true;
  p->last_status = s.status == 1 ? LP_OPTIMAL : (s.status == 4 ? LP_NUMERICAL_ERROR : LP_ITERATION_LIMIT);
  return LP_OK;
}

}  // namespace lpop

extern "C" {

void lp_options_default(lp_options* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->mode = LP_MODE_PDLP;
  o->scheduler = LP_SCHED_ADAGRAD;
  o->alpha = 0.0;
  o->phi = 20;
  o->normalize = 1;
  o->precond_floor = 1e-6;
  o->ruiz_iters = 10;
  o->pc_beta = 1.0;
  o->check_every = 64;
  o->restart = 1;
  o->power_iters = 200;
  o->plain_step_factor = 0.9;
  o->time_limit = 0.0;
  o->use_graph = 1;
  o->kernel_timing = 0;
  o->device = -1;
  o->stream = nullptr;
  o->precision = LP_PREC_FP64;
  o->refine_tol = 1e-6;
  o->refine_stall = 16;
  o->log_every = 0;
}

const char* lp_last_error(const lp_problem* p) {
  if (p) return p->err.c_str();
  return g_last_error.c_str();
}

int lp_create(int32_t m, int32_t n, int64_t nnz, const int64_t* row_ptr, const int32_t* col_idx, const double* val,
              const double* b, const double* c, const double* lb, const double* ub, const char* sense,
              const lp_options* opt, lp_problem** out) {
  try {
    NvtxRange range("lpop create");
    return create_impl(m, n, nnz, row_ptr, col_idx, val, b, c, lb, ub, sense, opt, out);
  } catch (const std::exception& ex) {
    return set_err(nullptr, LP_ERR_OOM, std::string("host exception: ") + ex.what());
  }
}

int lp_solve(lp_problem* p, double rel_kkt_tol, int64_t iter_limit, int32_t* status_out) {
  if (!p) return set_err(nullptr, LP_ERR_INVALID_ARG, "problem handle is NULL");
  if (!(rel_kkt_tol >= 0.0)) return set_err(p, LP_ERR_INVALID_ARG, "rel_kkt_tol must be >= 0");
  if (iter_limit < 0) return set_err(p, LP_ERR_INVALID_ARG, "iter_limit must be >= 0");
  try {
    NvtxRange range("lpop solve");
    return solve_impl(p, rel_kkt_tol, iter_limit, status_out);
  } catch (const std::exception& ex) {
    return set_err(p, LP_ERR_OOM, std::string("host exception: ") + ex.what());
  }
}

int lp_result(lp_problem* p, double* x, double* y, lp_stats* st) {
  if (!p) return set_err(nullptr, LP_ERR_INVALID_ARG, "problem handle is NULL");
  if (!p->solved_once) return set_err(p, LP_ERR_NOT_SOLVED, "lp_result called before lp_solve");
  TRY(select_device(p));
  DevState hs;
  CK(cudaMemcpyAsync(&hs, p->d.st, sizeof(hs), cudaMemcpyDeviceToHost, p->stream));
  CK(cudaStreamSynchronize(p->stream));
  if (x) TRY(download_vec(p, phase_vec(p, p->d.f64.x[hs.cur], p->d.f32.x[hs.cur], p->d.n), p->d.dc, p->d.n, p->d_pcol, x));
  if (y) TRY(download_vec(p, phase_vec(p, p->d.f64.y[hs.cur], p->d.f32.y[hs.cur], p->d.m), p->d.dr, p->d.m, p->d_prow, y));
  if (st) {
    std::memset(st, 0, sizeof(*st));
    st->pobj = hs.pobj;
    st->dobj = hs.dobj;
    st->rel_pres = hs.rel_pres;
    st->rel_dres = hs.rel_dres;
    st->rel_gap = hs.rel_gap;
    st->iterations = hs.attempts;
    st->accepted = hs.k;
    st->restarts = hs.restarts;
    st->eta = hs.eta;
    st->omega = hs.omega;
    st->solve_ms = p->last_solve_ms;
    st->status = p->last_status;
  }
  return LP_OK;
}

int lp_get_iterate(lp_problem* p, double* x, double* y, double* T, double* Sigma, double* scal) {
  if (!p) return set_err(nullptr, LP_ERR_INVALID_ARG, "problem handle is NULL");
  TRY(select_device(p));
  launch_flush_update(p->d, p->prm, p->fp32_phase, p->stream);
  CK(cudaGetLastError());
  DevState hs;
  CK(cudaMemcpyAsync(&hs, p->d.st, sizeof(hs), cudaMemcpyDeviceToHost, p->stream));
  CK(cudaStreamSynchronize(p->stream));
  const Dev& d = p->d;
  const int c = hs.cur;
  if (x) TRY(download_vec(p, phase_vec(p, d.f64.x[c], d.f32.x[c], d.n), nullptr, d.n, p->d_pcol, x));
  if (y) TRY(download_vec(p, phase_vec(p, d.f64.y[c], d.f32.y[c], d.m), nullptr, d.m, p->d_prow, y));
  if (T) TRY(download_vec(p, phase_vec(p, d.f64.T, d.f32.T, d.n), nullptr, d.n, p->d_pcol, T));
  if (Sigma) TRY(download_vec(p, phase_vec(p, d.f64.S, d.f32.S, d.m), nullptr, d.m, p->d_prow, Sigma));
  if (scal) {
    scal[0] = hs.eta;
    scal[1] = hs.omega;
    scal[2] = (double)hs.k;
    scal[3] = (double)hs.attempts;
    scal[4] = hs.wsum;
    scal[5] = (double)hs.restarts;
    scal[6] = hs.last_eta_max;
    scal[7] = (double)hs.last_accept;
  }
  return LP_OK;
}

int lp_get_scaling(lp_problem* p, double* dr, double* dc, double* scal) {
  if (!p) return set_err(nullptr, LP_ERR_INVALID_ARG, "problem handle is NULL");
  TRY(select_device(p));
  TRY(download_vec(p, p->d.dr, nullptr, p->d.m, p->d_prow, dr));
  TRY(download_vec(p, p->d.dc, nullptr, p->d.n, p->d_pcol, dc));
  if (scal) {
    scal[0] = p->eta0;
    scal[1] = p->omega0;
    scal[2] = p->norm_est;
    scal[3] = p->amax;
    scal[4] = p->d.gridA;
    scal[5] = p->d.gridAt;
    scal[6] = p->d.binsA.nunits;
    scal[7] = p->d.binsAt.nunits;
  }
  return LP_OK;
}

int lp_get_state(lp_problem* p, double* vec_n, double* vec_m, double* scal) {
  if (!p) return set_err(nullptr, LP_ERR_INVALID_ARG, "problem handle is NULL");
  try {
    return get_state_impl(p, vec_n, vec_m, scal);
  } catch (const std::exception& ex) {
    return set_err(p, LP_ERR_OOM, std::string("host exception: ") + ex.what());
  }
}

int lp_set_state(lp_problem* p, const double* vec_n, const double* vec_m, const double* scal) {
  if (!p) return set_err(nullptr, LP_ERR_INVALID_ARG, "problem handle is NULL");
  if (!vec_n || !scal || (!vec_m && p->d.m > 0)) return set_err(p, LP_ERR_INVALID_ARG, "state arrays must not be NULL");
  try {
    return set_state_impl(p, vec_n, vec_m, scal);
  } catch (const std::exception& ex) {
    return set_err(p, LP_ERR_OOM, std::string("host exception: ") + ex.what());
  }
}

int lp_reset(lp_problem* p) {
  if (!p) return set_err(nullptr, LP_ERR_INVALID_ARG, "problem handle is NULL");
  TRY(select_device(p));
  return init_state(p);
}

int lp_memory_bytes(int32_t m, int32_t n, int64_t nnz, const lp_options* opt, int64_t* bytes) {
  if (!bytes || m < 0 || n < 1 || nnz < 0) return set_err(nullptr, LP_ERR_INVALID_ARG, "bad sizes or NULL bytes");
  lp_options o;
  if (opt) o = *opt;
  else lp_options_default(&o);
  // mirrors upload(): every buffer is a 256-byte multiple of the block lp_create allocates
  auto r = [](long long b) { return ((b < 8 ? 8 : b) + 255) / 256 * 256; };
  long long t = 0;
  t += r(4LL * (m + 1)) + 2 * r(4LL * nnz) + 2 * r(8LL * nnz) + r(4LL * (n + 1));  // CSR of A and A^T
  t += 2 * (r(8LL * m) + r(8LL * n));                                              // dr, dc and reciprocals
  t += 13 * r(8LL * m) + 12 * r(8LL * n);                                          // FP64 vector set
  if (o.precision == LP_PREC_MIXED) t += 2 * r(4LL * nnz) + 13 * r(4LL * m) + 12 * r(4LL * n);  // FP32 set
  t += r(8LL * (m > n ? m : n) + 8) + r(m) + r(8LL * ((long long)m + n + 2048)) + r(sizeof(DevState));
  t += r(4);  // count of out-of-range gathers (checked builds)
  // segmented rows (segments are at least 4096 entries): at most S rows and 2 S units per matrix
  const long long S = nnz / 4096 + 1;
  t += 2 * (r(8LL * 2 * S) + r(16LL * 2 * S) + r(4LL * S));
  t += 2 * r(8LL * kMaxPartials * (4096 + S));  // per-block records (upper bound of the grid) and row slots
  t += 2 * r(4LL * (nnz / 2048 + 2));             // chunk tables of the whole-block rows (Ruiz)
  t += r(4LL * m) + r(4LL * n);                    // the row and column permutations
  // sliced copies of the rows of up to kSellMaxLen entries (at most nnz entries plus the
  // padding of the last slices of kSellMaxLen + 1 bins)
  const long long SE = nnz + (kSellMaxLen + 1LL) * 31 * kSellMaxLen;
  t += 2 * (r(4LL * SE) + r(8LL * SE) + (o.precision == LP_PREC_MIXED ? r(4LL * SE) : 0));
  *bytes = t;
  return LP_OK;
}

int lp_kernel_times(lp_problem* p, double* ms, int64_t* samples, int32_t n_kernels, int64_t* launches) {
  if (!p) return set_err(nullptr, LP_ERR_INVALID_ARG, "problem handle is NULL");
  if (n_kernels < 0) return set_err(p, LP_ERR_INVALID_ARG, "n_kernels must be >= 0");
  for (int k = 0; k < n_kernels; ++k) {
    if (ms) ms[k] = k < 2 ? p->kt_ms[k] : 0.0;
    if (samples) samples[k] = k < 2 ? p->kt_n[k] : 0;
  }
  if (launches) *launches = p->launches;
  return LP_OK;
}

void lp_destroy(lp_problem* p) { release(p); }

#ifdef LPOP_CHECK_BOUNDS
// Checked builds only (not declared in lpop.h): gathers of the problem's
// kernels whose column index fell outside the gathered vector, counted and
// skipped instead of read.
int lpop_bad_gathers(lp_problem* p, unsigned long long* count) {
  if (!p || !count) return LP_ERR_INVALID_ARG;
  unsigned int h = 0;
  if (cudaMemcpy(&h, p->d.bad_gathers, sizeof(h), cudaMemcpyDeviceToHost) != cudaSuccess) return LP_ERR_CUDA;
  *count = h;
  return LP_OK;
}
#endif

}  // extern "C"

namespace lpop {

namespace {
// out[perm[i]] = a[i] (times f[i] when f is given)
__global__ void scatter_perm_kernel(double* out, const double* a, const double* f, const int* perm, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    out[perm[i]] = f ? a[i] * f[i] : a[i];
}

// out[i] = a[perm[i]]
__global__ void gather_perm_kernel(double* out, const double* a, const int* perm, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) out[i] = a[perm[i]];
}

int perm_grid(int n) {
  int g = (n + kBlock - 1) / kBlock;
  if (g > 4096) g = 4096;
  return g < 1 ? 1 : g;
}
}  // namespace

void launch_scatter_perm(double* out, const double* a, const double* f, const int* perm, int n, cudaStream_t s) {
  scatter_perm_kernel<<<perm_grid(n), kBlock, 0, s>>>(out, a, f, perm, n);
}

void launch_gather_perm(double* out, const double* a, const int* perm, int n, cudaStream_t s) {
  gather_perm_kernel<<<perm_grid(n), kBlock, 0, s>>>(out, a, perm, n);
}

}  // namespace lpop
