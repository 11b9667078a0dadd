// cbx_solve_noalloc: the batch solver for callers that must not allocate GPU
// memory during a solve.
//
// cbx_solve takes its per-launch scratch (per-CTA Jacobian/rate workspace and
// the next-cell counter) from the stream-ordered allocator. Some callers
// cannot do that: a host that pre-reserves all device memory for its own pool
// at start-up and forbids any later allocation by third-party code, a
// latency-critical loop that must not enter the driver's allocator (which may
// synchronise or grow its pool at unpredictable cost), or a process that runs
// right at its memory budget. This entry point gives them the same kernel with
// its scratch in a fixed array that is part of the library image on each GPU.
//
// The array below is a file-scope __device__ array: every GPU that loads this
// library holds kScratchBytes of it until the process exits, whether or not
// this entry point is ever called. In host code its name is only a host-side
// stand-in; the device address is obtained with cudaGetSymbolAddress on the
// first call made in a given CUDA context (with its device current) and
// cached with that context's unique id, so that a context that is destroyed
// and created again (cudaDeviceReset, a released primary context) gets the
// address looked up again instead of a stale one.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <mutex>
#include <string>

#include "internal.h"

namespace {

constexpr size_t kScratchBytes = 16u << 20;  // 16 MiB per GPU
constexpr size_t kCounterBytes = 256;        // next-cell counter, cleared every call

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
struct ScratchAddr {
  unsigned long long ctx_id = 0;  // 0: not cached
  void* ptr = nullptr;
};
ScratchAddr g_scratch[kMaxDevices];

int fail(int code, const std::string& msg) { return cbx::record_error(code, msg); }

// Unique id of the calling thread's current CUDA context, 0 when there is none
// or the driver cannot tell (then the address is looked up on every call).
// The driver functions are fetched through the runtime, so the library does not
// link the driver library itself.
unsigned long long current_context_id() {
  using GetCurrent = CUresult (*)(CUcontext*);
  using GetId = CUresult (*)(CUcontext, unsigned long long*);
  static GetCurrent get_current = nullptr;
  static GetId get_id = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_current = (GetCurrent)f;
    f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_id = (GetId)f;
    cudaGetLastError();
  });
  if (!get_current || !get_id) return 0;
  CUcontext ctx = nullptr;
  unsigned long long id = 0;
  if (get_current(&ctx) != CUDA_SUCCESS || !ctx || get_id(ctx, &id) != CUDA_SUCCESS) return 0;
  return id;
}

}  // namespace

extern "C" int cbx_solve_noalloc(cbx_network* net, const cbx_cell_params* phi, const double* x0, int C, double t0,
                                 double t_end, const cbx_options* opt, void* stream, double* x_out,
                                 int* cell_status, cbx_cell_stats* stats) {
  using namespace cbx;
  if (!net) return fail(CBX_E_ARG, "net is NULL");
  if (C < 0) return fail(CBX_E_ARG, "C must be >= 0");
  if (C > 0 && (!phi || !x0 || !x_out || !cell_status)) return fail(CBX_E_ARG, "NULL array with C > 0");
  if (!std::isfinite(t0) || !std::isfinite(t_end) || t_end < t0) return fail(CBX_E_ARG, "need finite t0 <= t_end");
  cbx_options o;
  cbx_default_options(&o);
  if (opt) o = *opt;
  if (!(o.rtol > 0.0) || !std::isfinite(o.rtol) || !(o.atol >= 0.0) || !std::isfinite(o.atol) || o.max_steps < 1 ||
      (o.precision != CBX_FP64 && o.precision != CBX_MIXED) || (o.precision == CBX_MIXED && o.max_refine < 1) ||
      !(o.refine_tol >= 0.0))
    return fail(CBX_E_ARG, "invalid options (see cbx_options in carbox.h)");
  if (o.method != CBX_METHOD_BDF) return fail(CBX_E_ARG, "cbx_solve_noalloc runs CBX_METHOD_BDF only");
  if (C == 0) return CBX_OK;
  if (!net->dbuf) return fail(CBX_E_ARG, "network tables are not on a device: create the network with a GPU present");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(CBX_E_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev != net->device) return fail(CBX_E_ARG, "the current device is not the device holding the network tables");
  if (dev < 0 || dev >= kMaxDevices) return fail(CBX_E_ARG, "device index out of range");
  void* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    const unsigned long long id = current_context_id();
    if (id != 0 && g_scratch[dev].ctx_id == id) {
      scratch = g_scratch[dev].ptr;
    } else {
      e = cudaGetSymbolAddress(&scratch, g_noalloc_scratch);
      if (e != cudaSuccess) {
        g_scratch[dev] = ScratchAddr{};
        return fail(CBX_E_CUDA, std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
      }
      g_scratch[dev] = ScratchAddr{current_context_id(), scratch};
    }
  }
  const HostNet& h = net->host;
  const bool mixed = o.precision == CBX_MIXED;
  const SolverPlan plan = plan_solver(h.S, h.R, h.nseg, h.nnzJ, mixed, h.head_ints);
  const int occ = plan.occupancy;
  if (occ < 1) return fail(CBX_E_TOO_LARGE, "network too large for the solver");
  const long long stride = plan.ws_stride;
  const long long fit = (long long)((kScratchBytes - kCounterBytes) / (stride * sizeof(double)));
  if (fit < 1) {
    char m[200];
    snprintf(m, sizeof m, "network needs %lld bytes of scratch per CTA; the fixed scratch of cbx_solve_noalloc holds %zu",
             (long long)(stride * sizeof(double)), kScratchBytes - kCounterBytes);
    return fail(CBX_E_TOO_LARGE, m);
  }
  const int grid = (int)std::min<long long>(std::min<long long>(C, (long long)occ * device_sm_count()), fit);
  SolveArgs a{};
  a.net = net->dev;
  a.alpha = net->dev.alpha;
  a.phi = phi;
  a.x0 = x0;
  a.C = C;
  a.t0 = t0;
  a.t_end = t_end;
  a.rtol = o.rtol;
  a.atol = o.atol;
  a.newton_tol = std::max(10.0 * 2.220446049250313e-16 / o.rtol, std::min(0.03, std::sqrt(o.rtol)));
  a.refine_tol = o.refine_tol;
  a.max_steps = o.max_steps;
  a.max_refine = o.max_refine;
  for (int q = 0; q < kMaxOrder + 2; ++q) {
    double g = 0.0;
    for (int j = 1; j <= q; ++j) g += 1.0 / j;
    a.gam[q] = g;
  }
  a.x_out = x_out;
  a.status = cell_status;
  a.stats = stats;
  a.ws_stride = stride;
  a.counter = (int*)scratch;
  a.ws = (double*)((unsigned char*)scratch + kCounterBytes);
  e = cudaMemsetAsync(a.counter, 0, sizeof(int), (cudaStream_t)stream);
  if (e != cudaSuccess) return fail(CBX_E_CUDA, std::string("cudaMemsetAsync(counter): ") + cudaGetErrorString(e));
  e = (cudaError_t)launch_solver(a, plan, grid, stream);
  if (e != cudaSuccess) return fail(CBX_E_CUDA, std::string("solver launch: ") + cudaGetErrorString(e));
  return CBX_OK;
}
