// Continuous-batching request server.
//
// Requests (a network, C cells, a time span, options) are submitted from any
// host thread and admitted by a scheduler thread as soon as a CUDA stream of
// the pool and enough of the device-memory budget are free; requests that
// arrive while others run are admitted into the freed stream/memory and their
// kernels run concurrently with the running ones. Each admitted request gets
// its own device buffers (inputs, outputs, solver workspace), an H2D copy, a
// solver launch with at most `max_ctas` persistent CTAs (so several requests,
// of any network size, share the SMs; each CTA keeps a cell's solver state on
// chip, retires it and back-fills from the request's cell counter), a D2H
// copy and a stream-ordered free. A host callback marks it done. A cell's
// result does not depend on the other requests in flight (fixed per-cell
// arithmetic order), so results are the same alone and in the mix.
#include <cuda_runtime.h>

#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "internal.h"

using namespace cbx;

namespace {

double now_s() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

enum ReqState { kQueued = 0, kRunning = 1, kDone = 2, kFailed = 3 };

}  // namespace

struct cbx_server;

struct ServerRequest {
  cbx_server* srv = nullptr;
  uint64_t id = 0;
  cbx_network* net = nullptr;
  int C = 0, S = 0;
  double t0 = 0, t_end = 0;
  cbx_options opt{};
  cbx_cell_params* h_phi = nullptr;  // pinned staging
  double* h_x = nullptr;             // pinned: x0 in, x_out back
  int* h_status = nullptr;           // pinned
  size_t bytes = 0;                  // device-memory reservation
  int stream = -1;
  int state = kQueued;
  int rc = CBX_OK;
  double t_submit = 0, t_start = 0, t_done = 0;
};

struct cbx_server {
  size_t budget = 0, in_use = 0;
  int max_ctas = 0;
  int device = 0;
  std::vector<cudaStream_t> streams;
  std::vector<char> busy;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<ServerRequest*> queue;
  std::map<uint64_t, ServerRequest*> reqs;
  uint64_t next_id = 1;
  bool stop = false;
  std::thread sched;
  size_t peak_in_use = 0;
  int peak_running = 0;
};

namespace {

// Device bytes a request needs: inputs, outputs, status, workspace.
size_t request_bytes(cbx_network* net, int C, bool mixed) {
  const HostNet& h = net->host;
  const SolverPlan p = plan_solver(h.S, h.R, h.nseg, h.nnzJ, mixed, h.head_ints);
  const int grid = std::max(1, std::min(C, std::max(1, p.occupancy) * device_sm_count()));
  return (size_t)C * (sizeof(cbx_cell_params) + 2 * h.S * sizeof(double) + sizeof(int)) +
         (size_t)grid * p.ws_stride * sizeof(double) + 4096;
}

void CUDART_CB on_done(void* arg) {
  ServerRequest* r = (ServerRequest*)arg;
  cbx_server* s = r->srv;
  std::lock_guard<std::mutex> lock(s->mu);
  r->t_done = now_s();
  if (r->state == kRunning) r->state = r->rc == CBX_OK ? kDone : kFailed;
  s->busy[r->stream] = 0;
  s->in_use -= r->bytes;
  s->cv.notify_all();
}

void launch(cbx_server* s, ServerRequest* r) {
  cudaStream_t st = s->streams[r->stream];
  const size_t b_phi = (size_t)r->C * sizeof(cbx_cell_params), b_x = (size_t)r->S * r->C * sizeof(double),
               b_st = (size_t)r->C * sizeof(int);
  auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
  char* d = nullptr;
  cudaError_t e = cudaMallocAsync((void**)&d, al(b_phi) + 2 * al(b_x) + al(b_st), st);
  int rc = CBX_OK;
  if (e == cudaSuccess) {
    cbx_cell_params* d_phi = (cbx_cell_params*)d;
    double* d_x0 = (double*)(d + al(b_phi));
    double* d_xo = (double*)(d + al(b_phi) + al(b_x));
    int* d_st = (int*)(d + al(b_phi) + 2 * al(b_x));
    e = cudaMemcpyAsync(d_phi, r->h_phi, b_phi, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_x0, r->h_x, b_x, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) {
      rc = solve_device(r->net, d_phi, d_x0, r->C, r->t0, r->t_end, &r->opt, st, d_xo, d_st, s->max_ctas);
      if (rc == CBX_OK) {
        e = cudaMemcpyAsync(r->h_x, d_xo, b_x, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(r->h_status, d_st, b_st, cudaMemcpyDeviceToHost, st);
      }
    }
    cudaFreeAsync(d, st);
  }
  if (e != cudaSuccess && rc == CBX_OK) rc = CBX_E_CUDA;
  r->rc = rc;
  e = cudaLaunchHostFunc(st, on_done, r);
  if (e != cudaSuccess) {
    // no callback will come: finish the bookkeeping here
    cudaStreamSynchronize(st);
    r->rc = CBX_E_CUDA;
    on_done(r);
  }
}

void scheduler(cbx_server* s) {
  cudaSetDevice(s->device);
  std::unique_lock<std::mutex> lock(s->mu);
  for (;;) {
    if (s->stop) break;
    bool launched = false;
    for (auto it = s->queue.begin(); it != s->queue.end(); ++it) {
      ServerRequest* r = *it;
      int free_stream = -1;
      for (size_t k = 0; k < s->busy.size(); ++k)
        if (!s->busy[k]) {
          free_stream = (int)k;
          break;
        }
      if (free_stream < 0) break;
      if (s->in_use + r->bytes > s->budget && s->in_use > 0) continue;  // later, smaller requests may fit
      s->queue.erase(it);
      s->busy[free_stream] = 1;
      s->in_use += r->bytes;
      s->peak_in_use = std::max(s->peak_in_use, s->in_use);
      int running = 0;
      for (char b : s->busy) running += b;
      s->peak_running = std::max(s->peak_running, running);
      r->stream = free_stream;
      r->state = kRunning;
      r->t_start = now_s();
      lock.unlock();
      launch(s, r);
      lock.lock();
      launched = true;
      break;  // the queue may have changed
    }
    if (!launched) s->cv.wait(lock);
  }
}

}  // namespace

extern "C" {

int cbx_server_create(size_t mem_budget, int n_streams, int max_ctas, cbx_server** out) {
  if (!out) return record_error(CBX_E_ARG, "out is NULL");
  *out = nullptr;
  if (n_streams < 1 || n_streams > 64) return record_error(CBX_E_ARG, "n_streams must be in 1..64");
  if (max_ctas < 0) return record_error(CBX_E_ARG, "max_ctas must be >= 0");
  cbx_server* s = new (std::nothrow) cbx_server();
  if (!s) return record_error(CBX_E_NOMEM, "host allocation failed");
  cudaGetDevice(&s->device);
  s->budget = mem_budget;
  s->max_ctas = max_ctas;
  for (int k = 0; k < n_streams; ++k) {
    cudaStream_t st;
    cudaError_t e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      for (cudaStream_t x : s->streams) cudaStreamDestroy(x);
      delete s;
      return record_error(CBX_E_CUDA, std::string("cudaStreamCreate: ") + cudaGetErrorString(e));
    }
    s->streams.push_back(st);
  }
  s->busy.assign(n_streams, 0);
  s->sched = std::thread(scheduler, s);
  *out = s;
  return CBX_OK;
}

int cbx_server_submit(cbx_server* s, cbx_network* net, const cbx_cell_params* phi, const double* x0, int C,
                      double t0, double t_end, const cbx_options* opt, uint64_t* request_id) {
  if (!s || !net || !request_id) return record_error(CBX_E_ARG, "NULL argument");
  if (C < 1 || !phi || !x0) return record_error(CBX_E_ARG, "need C >= 1 and host arrays");
  if (!(t_end >= t0)) return record_error(CBX_E_ARG, "need t0 <= t_end");
  ServerRequest* r = new (std::nothrow) ServerRequest();
  if (!r) return record_error(CBX_E_NOMEM, "host allocation failed");
  r->srv = s;
  r->net = net;
  r->C = C;
  r->S = net->host.S;
  r->t0 = t0;
  r->t_end = t_end;
  cbx_default_options(&r->opt);
  if (opt) r->opt = *opt;
  r->bytes = request_bytes(net, C, r->opt.precision == CBX_MIXED);
  if (r->bytes > s->budget) {
    delete r;
    return record_error(CBX_E_TOO_LARGE, "request larger than the server's memory budget");
  }
  cudaError_t e = cudaMallocHost((void**)&r->h_phi, (size_t)C * sizeof(cbx_cell_params));
  if (e == cudaSuccess) e = cudaMallocHost((void**)&r->h_x, (size_t)r->S * C * sizeof(double));
  if (e == cudaSuccess) e = cudaMallocHost((void**)&r->h_status, (size_t)C * sizeof(int));
  if (e != cudaSuccess) {
    cudaFreeHost(r->h_phi);
    cudaFreeHost(r->h_x);
    cudaFreeHost(r->h_status);
    delete r;
    return record_error(CBX_E_NOMEM, "pinned staging allocation failed");
  }
  memcpy(r->h_phi, phi, (size_t)C * sizeof(cbx_cell_params));
  memcpy(r->h_x, x0, (size_t)r->S * C * sizeof(double));
  std::lock_guard<std::mutex> lock(s->mu);
  r->id = s->next_id++;
  r->t_submit = now_s();
  s->reqs[r->id] = r;
  s->queue.push_back(r);
  *request_id = r->id;
  s->cv.notify_all();
  return CBX_OK;
}

int cbx_server_poll(cbx_server* s, uint64_t request_id, int* state, double* latency_s) {
  if (!s) return record_error(CBX_E_ARG, "server is NULL");
  std::lock_guard<std::mutex> lock(s->mu);
  auto it = s->reqs.find(request_id);
  if (it == s->reqs.end()) return record_error(CBX_E_ARG, "unknown request id");
  ServerRequest* r = it->second;
  if (state) *state = r->state;
  if (latency_s) *latency_s = r->state >= kDone ? r->t_done - r->t_submit : -1.0;
  return CBX_OK;
}

int cbx_server_wait(cbx_server* s, uint64_t request_id, double* x_out, int* cell_status, double* times) {
  if (!s) return record_error(CBX_E_ARG, "server is NULL");
  std::unique_lock<std::mutex> lock(s->mu);
  auto it = s->reqs.find(request_id);
  if (it == s->reqs.end()) return record_error(CBX_E_ARG, "unknown request id");
  ServerRequest* r = it->second;
  s->cv.wait(lock, [&] { return r->state >= kDone; });
  const int rc = r->rc;
  if (rc == CBX_OK) {
    if (x_out) memcpy(x_out, r->h_x, (size_t)r->S * r->C * sizeof(double));
    if (cell_status) memcpy(cell_status, r->h_status, (size_t)r->C * sizeof(int));
  }
  if (times) {
    times[0] = r->t_submit;
    times[1] = r->t_start;
    times[2] = r->t_done;
  }
  s->reqs.erase(it);
  lock.unlock();
  cudaFreeHost(r->h_phi);
  cudaFreeHost(r->h_x);
  cudaFreeHost(r->h_status);
  delete r;
  return rc == CBX_OK ? CBX_OK : record_error(rc, "request failed");
}

int cbx_server_stats(cbx_server* s, size_t* peak_bytes, int* peak_running, int* queued) {
  if (!s) return record_error(CBX_E_ARG, "server is NULL");
  std::lock_guard<std::mutex> lock(s->mu);
  if (peak_bytes) *peak_bytes = s->peak_in_use;
  if (peak_running) *peak_running = s->peak_running;
  if (queued) *queued = (int)s->queue.size();
  return CBX_OK;
}

int cbx_server_destroy(cbx_server* s) {
  if (!s) return CBX_OK;
  {
    std::unique_lock<std::mutex> lock(s->mu);
    s->cv.wait(lock, [&] {
      for (char b : s->busy)
        if (b) return false;
      return true;
    });
    s->stop = true;
    s->cv.notify_all();
  }
  s->sched.join();
  for (cudaStream_t st : s->streams) cudaStreamDestroy(st);
  for (auto& kv : s->reqs) {
    cudaFreeHost(kv.second->h_phi);
    cudaFreeHost(kv.second->h_x);
    cudaFreeHost(kv.second->h_status);
    delete kv.second;
  }
  delete s;
  return CBX_OK;
}

}  // extern "C"
