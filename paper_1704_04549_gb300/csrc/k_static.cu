// dg_apply_sumfact_static: the operator with its face-trace scratch in a
// file-scope device array instead of the context workspace.
//
// For callers that cannot allocate device memory themselves (their device
// memory is handed out by an allocator they do not control, or their budget
// is fixed once at start-up) and that therefore cannot provide scratch space
// beyond the vectors they pass in.  The traces are written in full by the
// trace kernel before the element kernel reads them, so nothing in the array
// needs clearing between calls.  The paper has no counterpart to this.
#include <mutex>
#include <string>

#include "tpp_internal.cuh"

// 4 MiB of doubles: 2D problems with num_elem * nrhs * 4 * n <= 524288 face-trace
// values (e.g. 64 x 64 elements up to n = 32 with one right-hand side).  Every GPU that loads libtpp
// holds this array until the process exits.  All calls share it and it keeps
// the last call's contents; calls that overlap on the GPU race on it.
constexpr size_t kStaticTraceDoubles = size_t(1) << 19;

static __device__ __align__(256) double g_trace_scratch[kStaticTraceDoubles];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_scratch_addr[kMaxDevices] = {nullptr};

// Device address of g_trace_scratch on the current device (looked up once per
// device; in host code the symbol is only a host-side stand-in).
tpp_status scratch_address(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return tpp::cuda_check(e, "cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) {
    tpp::set_error("device ordinal out of range for the static scratch table");
    return TPP_ERR_UNSUPPORTED;
  }
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_trace_scratch);
    if (e != cudaSuccess) return tpp::cuda_check(e, "cudaGetSymbolAddress(g_trace_scratch)");
    g_scratch_addr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_addr[dev];
  return TPP_OK;
}

}  // namespace

extern "C" tpp_status dg_apply_sumfact_static(const tpp_ctx* c, const double* x, double* y,
                                              int32_t nrhs, void* stream) {
  if (!c) {
    tpp::set_error("context is NULL");
    return TPP_ERR_INVALID_ARG;
  }
  if (!x || !y || x == y) {
    tpp::set_error("x and y must be non-NULL and distinct");
    return TPP_ERR_INVALID_ARG;
  }
  if (c->dim != 2) {
    tpp::set_error("dg_apply_sumfact_static supports 2D problems only");
    return TPP_ERR_UNSUPPORTED;
  }
  if (nrhs < 1 || nrhs > c->R) {
    tpp::set_error("nrhs must be in [1, the problem's nrhs]");
    return TPP_ERR_INVALID_ARG;
  }
  const size_t need = (size_t)c->E * nrhs * 4 * (size_t)c->nfq;
  if (need > kStaticTraceDoubles) {
    tpp::set_error("dg_apply_sumfact_static: num_elem * nrhs * 4 * mu = " + std::to_string(need) +
                   " face-trace values exceed the static scratch of " +
                   std::to_string(kStaticTraceDoubles) + " doubles");
    return TPP_ERR_INVALID_ARG;
  }
  int dev = -1;
  cudaError_t ed = cudaGetDevice(&dev);
  if (ed != cudaSuccess) return tpp::cuda_check(ed, "cudaGetDevice");
  if (dev != c->device) {
    // the scratch address below belongs to the current device, the workspace and the
    // vectors to the context's: refuse rather than mix two GPUs' memory
    tpp::set_error("dg_apply_sumfact_static: current device " + std::to_string(dev) +
                   " is not the context's device " + std::to_string(c->device));
    return TPP_ERR_INVALID_ARG;
  }
  double* tr = nullptr;
  if (tpp_status st = scratch_address(&tr)) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const tpp_ctx v = tpp::call_view(c, nrhs);
  cudaError_t e = tpp::launch_traces(&v, x, tr, s);
  if (e != cudaSuccess) return tpp::cuda_check(e, "k_traces");
  e = tpp::launch_dg_apply(&v, x, tr, y, nullptr, s);
  if (e != cudaSuccess) return tpp::cuda_check(e, "k_dg_apply_2d");
  return TPP_OK;
}
