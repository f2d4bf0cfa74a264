// lp_power_norm_noalloc: the power-iteration estimate of ||A||_2 (the one
// lp_create runs in plain mode to pick the vanilla step size 0.9 / ||A||_2)
// for callers that cannot allocate device memory.
//
// Who needs it: code that runs where cudaMalloc is not available or not
// allowed -- a plugin inside a host framework that has reserved all of device
// memory for its own pool, a real-time loop that must not allocate, or a
// caller whose device buffers come from another allocator.  Such a caller
// already holds its matrix on the device and only wants the estimate.
//
// The scratch (three work vectors and the norm reduction's partial sums) lives
// in one file-scope device array of fixed size, so the call allocates nothing.
// Every GPU that loads the library keeps that array until the process exits.
#include <cstring>
#include <mutex>
#include <string>

#include "../../include/lpop.h"
#include "common.cuh"

namespace lpop {
void set_thread_error(const std::string& msg);  // api.cu

namespace {

// 2^20 doubles = 8 MiB of scratch per device
constexpr long long kScratchDoubles = 1LL << 20;
constexpr long long kReduceDoubles = 1 + 1024;  // norm result + per-block partials of launch_norm2

__device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

constexpr int kMaxDevices = 64;
double* g_scratch_addr[kMaxDevices] = {nullptr};
std::mutex g_scratch_mutex;

int fail(int code, const std::string& msg) {
  set_thread_error(msg);  // reported by lp_last_error(NULL)
  return code;
}

// Device address of the scratch array on the current device, looked up once per device.
int scratch_address(int dev, double** out) {
  if (dev < 0 || dev >= kMaxDevices) return fail(LP_ERR_INVALID_ARG, "device ordinal out of range");
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (!g_scratch_addr[dev]) {
    void* ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess) return fail(LP_ERR_CUDA, std::string("cudaGetSymbolAddress failed: ") + cudaGetErrorString(e));
    g_scratch_addr[dev] = static_cast<double*>(ptr);
  }
  *out = g_scratch_addr[dev];
  return LP_OK;
}

// v[j] = scale * (+-1 from SplitMix64 of j): the power iteration's second start direction.
__global__ void splitmix_fill_kernel(double* v, int n, double scale) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x)
    v[j] = scale * splitmix_sign((unsigned long long)j);
}

}  // namespace
}  // namespace lpop

using namespace lpop;

extern "C" int lp_power_norm_noalloc(int32_t m, int32_t n, const int32_t* a_row_ptr, const int32_t* a_col_idx,
                                     const double* a_val, const int32_t* at_row_ptr, const int32_t* at_col_idx,
                                     const double* at_val, int32_t iters, void* stream, double* norm_out) {
  if (!norm_out) return fail(LP_ERR_INVALID_ARG, "norm_out must not be NULL");
  *norm_out = 0.0;
  if (m < 1 || n < 1 || iters < 1) return fail(LP_ERR_INVALID_ARG, "need m >= 1, n >= 1 and iters >= 1");
  if (!a_row_ptr || !a_col_idx || !a_val || !at_row_ptr || !at_col_idx || !at_val)
    return fail(LP_ERR_INVALID_ARG, "matrix pointers must not be NULL");
  const long long need = 2LL * n + m + kReduceDoubles;
  if (need > kScratchDoubles)
    return fail(LP_ERR_INVALID_ARG, "problem too large for the fixed scratch: need 2 n + m + 1025 = " +
                                        std::to_string(need) + " doubles, the maximum is " +
                                        std::to_string(kScratchDoubles));
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(LP_ERR_CUDA, std::string("cudaGetDevice failed: ") + cudaGetErrorString(e));
  double* scratch = nullptr;
  int rc = scratch_address(dev, &scratch);
  if (rc != LP_OK) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  double* v = scratch;
  double* t = v + n;
  double* w = t + m;
  double* red = w + n;

  // every row with 8 lanes: one work-unit class covering all rows (no host-side look at row lengths)
  BinTable ba{}, bat{};
  ba.nbins = bat.nbins = 1;
  ba.bin[0] = Bin{0, m, 8, 0};
  bat.bin[0] = Bin{0, n, 8, 0};
  ba.nunits = (m + kBlock / 8 - 1) / (kBlock / 8);
  bat.nunits = (n + kBlock / 8 - 1) / (kBlock / 8);
  const int grid_a = ba.nunits < 1024 ? ba.nunits : 1024;
  const int grid_at = bat.nunits < 1024 ? bat.nunits : 1024;
  const Csr A{a_row_ptr, a_col_idx, a_val};
  const Csr At{at_row_ptr, at_col_idx, at_val};

  launch_fill(v, 1.0 / std::sqrt((double)n), n, s);
  bool restarted = false;
  for (int it = 0; it < iters; ++it) {
    launch_spmv_binned(A, ba, grid_a, v, t, s);
    launch_spmv_binned(At, bat, grid_at, t, w, s);
    launch_norm2(w, n, red, s);
    if (it == 0 && !restarted) {
      // a zero first product (every row of A sums to zero): start again from
      // the SplitMix64 sign direction, as lp_create does
      double nw0 = 0.0;
      e = cudaMemcpyAsync(&nw0, red, sizeof(double), cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) return fail(LP_ERR_CUDA, std::string("reading the norm failed: ") + cudaGetErrorString(e));
      if (nw0 == 0.0) {
        splitmix_fill_kernel<<<(n + kBlock - 1) / kBlock < 1024 ? (n + kBlock - 1) / kBlock : 1024, kBlock, 0, s>>>(
            v, n, 1.0 / std::sqrt((double)n));
        restarted = true;
        it = -1;
        continue;
      }
    }
    launch_scale_by_inv(w, n, red, s);
    double* tmp = v;  // the normalised w becomes the next v
    v = w;
    w = tmp;
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return fail(LP_ERR_CUDA, std::string("kernel launch failed: ") + cudaGetErrorString(e));
  double nw = 0.0;
  e = cudaMemcpyAsync(&nw, red, sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fail(LP_ERR_CUDA, std::string("reading the result failed: ") + cudaGetErrorString(e));
  *norm_out = nw > 0.0 && std::isfinite(nw) ? std::sqrt(nw) : 0.0;
  return LP_OK;
}
