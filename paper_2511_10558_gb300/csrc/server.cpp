// Continuous-batching request server.
//
// Requests (a network, C cells, a time span, options) are submitted from any
// host thread and admitted by a scheduler thread as soon as a CUDA stream of
// the pool and enough of the device-memory budget are free. Queued requests
// for the same network with the same options and start time are merged into
// one launch: their cells are concatenated (each keeps its own end time), so
// the launch's persistent CTAs back-fill across requests; a cell's solver
// state stays on chip for its whole solve. Requests that arrive while others
// run are admitted into the freed streams and memory, and their kernels run
// concurrently with the running ones; each launch uses at most `max_ctas`
// CTAs so that several launches, of any network size, share the SMs.
//
// Per launch: device buffers (inputs, outputs, per-cell end times, solver
// workspace), the H2D copies of every merged request (strided copies into the
// [S][C] layout), the solver, the D2H copies back into each request's pinned
// buffers, a stream-ordered free, and a host callback that completes the
// requests. A cell's result does not depend on what else is in flight or in
// the same launch (fixed per-cell arithmetic order), so results are the same
// alone, merged and in the mix.
//
// Admission order: arrival order; a request that does not fit the free memory
// may be passed by later, smaller ones at most kMaxPasses times, after which
// nothing else is admitted before it.
//
// Locking: no CUDA call is made while the server's mutex is held, because the
// completion callback runs on a CUDA driver thread and takes that mutex; a
// request's launch sizing is therefore computed at submit, outside the lock.
#include <cuda_runtime.h>

#include <algorithm>
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

constexpr int kMaxPasses = 8;            // times a waiting request may be passed by later ones
constexpr int kMaxMergedCells = 1 << 16;  // cells of one merged launch

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
  double* h_tend = nullptr;          // pinned: t_end per cell
  int* h_status = nullptr;           // pinned
  int state = kQueued;
  int rc = CBX_OK;
  int passed = 0;                    // times a later request was admitted before it
  // launch sizing, computed at submit (no CUDA call may run under the server's
  // lock: the completion callback, on a driver thread, takes that lock)
  size_t cell_bytes = 0, cta_bytes = 0;
  int grid_cap = 1;
  double t_submit = 0, t_start = 0, t_done = 0;
};

// One launch: one or more merged requests on one stream.
struct ServerLaunch {
  cbx_server* srv = nullptr;
  std::vector<ServerRequest*> reqs;
  int C = 0;
  size_t bytes = 0;
  int stream = -1;
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
  int waiting = 0;  // threads inside cbx_server_wait
  std::thread sched;
  size_t peak_in_use = 0;
  int peak_running = 0;
  long long launches = 0, merged_requests = 0;
};

namespace {

// Launch sizing of a request's kind (network, precision, CTA cap): CUDA calls,
// so only outside the server's lock.
void size_request(ServerRequest* r, int max_ctas) {
  const HostNet& h = r->net->host;
  const SolverPlan p = plan_solver(h.S, h.R, h.nseg, h.nnzJ, r->opt.precision == CBX_MIXED, h.head_ints);
  r->cell_bytes = sizeof(cbx_cell_params) + 2 * h.S * sizeof(double) + sizeof(double) + sizeof(int);
  r->cta_bytes = (size_t)p.ws_stride * sizeof(double);
  r->grid_cap = std::max(1, std::max(1, p.occupancy) * device_sm_count());
  if (max_ctas > 0) r->grid_cap = std::min(r->grid_cap, max_ctas);
}

// Device bytes of a launch of C cells of r's kind: inputs, outputs, end times,
// status, workspace (pure arithmetic: safe under the lock).
size_t launch_bytes(const ServerRequest* r, int C) {
  return (size_t)C * r->cell_bytes + (size_t)std::min(C, r->grid_cap) * r->cta_bytes + 8192;
}

bool same_kind(const ServerRequest* a, const ServerRequest* b) {
  return a->net == b->net && a->t0 == b->t0 && memcmp(&a->opt, &b->opt, sizeof(cbx_options)) == 0;
}

void free_request(ServerRequest* r) {
  cudaFreeHost(r->h_phi);
  cudaFreeHost(r->h_x);
  cudaFreeHost(r->h_tend);
  cudaFreeHost(r->h_status);
  delete r;
}

void CUDART_CB on_done(void* arg) {
  ServerLaunch* L = (ServerLaunch*)arg;
  cbx_server* s = L->srv;
  {
    std::lock_guard<std::mutex> lock(s->mu);
    const double t = now_s();
    for (ServerRequest* r : L->reqs) {
      r->t_done = t;
      if (r->state == kRunning) r->state = r->rc == CBX_OK ? kDone : kFailed;
    }
    s->busy[L->stream] = 0;
    s->in_use -= L->bytes;
  }
  s->cv.notify_all();
  delete L;
}

void launch(cbx_server* s, ServerLaunch* L) {
  cudaStream_t st = s->streams[L->stream];
  ServerRequest* r0 = L->reqs[0];
  const int C = L->C, S = r0->S;
  auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
  const size_t b_phi = (size_t)C * sizeof(cbx_cell_params), b_x = (size_t)S * C * sizeof(double),
               b_t = (size_t)C * sizeof(double), b_st = (size_t)C * sizeof(int);
  char* d = nullptr;
  cudaError_t e = cudaMallocAsync((void**)&d, al(b_phi) + 2 * al(b_x) + al(b_t) + al(b_st), st);
  int rc = CBX_OK;
  if (e == cudaSuccess) {
    cbx_cell_params* d_phi = (cbx_cell_params*)d;
    double* d_x0 = (double*)(d + al(b_phi));
    double* d_xo = (double*)(d + al(b_phi) + al(b_x));
    double* d_t = (double*)(d + al(b_phi) + 2 * al(b_x));
    int* d_st = (int*)(d + al(b_phi) + 2 * al(b_x) + al(b_t));
    double t_max = r0->t0;
    int o = 0;
    for (ServerRequest* r : L->reqs) {
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_phi + o, r->h_phi, r->C * sizeof(cbx_cell_params), cudaMemcpyHostToDevice, st);
      if (e == cudaSuccess)  // x0 rows of this request into columns o..o+C_r-1 of [S][C]
        e = cudaMemcpy2DAsync(d_x0 + o, C * sizeof(double), r->h_x, r->C * sizeof(double), r->C * sizeof(double), S,
                              cudaMemcpyHostToDevice, st);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_t + o, r->h_tend, r->C * sizeof(double), cudaMemcpyHostToDevice, st);
      t_max = std::max(t_max, r->t_end);
      o += r->C;
    }
    if (e == cudaSuccess) {
      rc = solve_device(r0->net, d_phi, d_x0, C, r0->t0, t_max, &r0->opt, st, d_xo, d_st, s->max_ctas, d_t);
      o = 0;
      for (ServerRequest* r : L->reqs) {
        if (rc == CBX_OK && e == cudaSuccess)
          e = cudaMemcpy2DAsync(r->h_x, r->C * sizeof(double), d_xo + o, C * sizeof(double), r->C * sizeof(double), S,
                                cudaMemcpyDeviceToHost, st);
        if (rc == CBX_OK && e == cudaSuccess)
          e = cudaMemcpyAsync(r->h_status, d_st + o, r->C * sizeof(int), cudaMemcpyDeviceToHost, st);
        o += r->C;
      }
    }
    cudaFreeAsync(d, st);
  }
  if (e != cudaSuccess && rc == CBX_OK) rc = CBX_E_CUDA;
  for (ServerRequest* r : L->reqs) r->rc = rc;
  e = cudaLaunchHostFunc(st, on_done, L);
  if (e != cudaSuccess) {
    // no callback will come: finish the bookkeeping here
    cudaStreamSynchronize(st);
    for (ServerRequest* r : L->reqs) r->rc = CBX_E_CUDA;
    on_done(L);
  }
}

// Pick the next launch from the queue (lock held): the first request that
// fits, unless an earlier one has been passed too often, plus the queued
// requests of the same kind that fit with it. Returns null when nothing fits.
ServerLaunch* next_launch(cbx_server* s) {
  auto fits = [&](size_t bytes) { return s->in_use + bytes <= s->budget || s->in_use == 0; };
  ServerRequest* head = nullptr;
  for (ServerRequest* r : s->queue) {
    if (fits(launch_bytes(r, r->C))) {
      head = r;
      break;
    }
    if (r->passed >= kMaxPasses) return nullptr;  // it goes next, when memory frees up
  }
  if (!head) return nullptr;
  ServerLaunch* L = new ServerLaunch();
  L->srv = s;
  for (ServerRequest* r : s->queue) {
    if (r != head && !(same_kind(r, head) && L->C > 0)) continue;
    // a merged launch must fit the budget itself (the head alone always may run on an idle server)
    if (r == head || (L->C + r->C <= kMaxMergedCells && s->in_use + launch_bytes(head, L->C + r->C) <= s->budget)) {
      L->reqs.push_back(r);
      L->C += r->C;
    }
  }
  // head first in the launch: requests merged before it in arrival order were skipped above
  L->bytes = launch_bytes(head, L->C);
  for (ServerRequest* r : s->queue) {
    if (r == head) break;
    if (std::find(L->reqs.begin(), L->reqs.end(), r) == L->reqs.end()) r->passed++;
  }
  std::deque<ServerRequest*> rest;
  for (ServerRequest* r : s->queue)
    if (std::find(L->reqs.begin(), L->reqs.end(), r) == L->reqs.end()) rest.push_back(r);
  s->queue.swap(rest);
  return L;
}

void scheduler(cbx_server* s) {
  cudaSetDevice(s->device);
  std::unique_lock<std::mutex> lock(s->mu);
  for (;;) {
    if (s->stop) break;
    int free_stream = -1;
    for (size_t k = 0; k < s->busy.size(); ++k)
      if (!s->busy[k]) {
        free_stream = (int)k;
        break;
      }
    ServerLaunch* L = free_stream >= 0 && !s->queue.empty() ? next_launch(s) : nullptr;
    if (!L) {
      s->cv.wait(lock);
      continue;
    }
    L->stream = free_stream;
    s->busy[free_stream] = 1;
    s->in_use += L->bytes;
    s->peak_in_use = std::max(s->peak_in_use, s->in_use);
    int running = 0;
    for (char b : s->busy) running += b;
    s->peak_running = std::max(s->peak_running, running);
    s->launches++;
    s->merged_requests += (long long)L->reqs.size() - 1;
    const double t = now_s();
    for (ServerRequest* r : L->reqs) {
      r->state = kRunning;
      r->t_start = t;
    }
    lock.unlock();
    launch(s, L);
    lock.lock();
  }
}

}  // namespace

extern "C" {

int cbx_server_create(size_t mem_budget, int n_streams, int max_ctas, cbx_server** out) {
  if (!out) return record_error(CBX_E_ARG, "out is NULL");
  *out = nullptr;
  if (n_streams < 1 || n_streams > 64) return record_error(CBX_E_ARG, "n_streams must be in 1..64");
  if (max_ctas < 0) return record_error(CBX_E_ARG, "max_ctas must be >= 0");
  size_t free_b = 0, total_b = 0;
  cudaError_t e = cudaMemGetInfo(&free_b, &total_b);
  if (e != cudaSuccess) return record_error(CBX_E_CUDA, std::string("cudaMemGetInfo: ") + cudaGetErrorString(e));
  const size_t derived = free_b / 10 * 8;  // 80 % of the memory free now
  cbx_server* s = new (std::nothrow) cbx_server();
  if (!s) return record_error(CBX_E_NOMEM, "host allocation failed");
  cudaGetDevice(&s->device);
  s->budget = mem_budget == 0 ? derived : std::min(mem_budget, derived);
  s->max_ctas = max_ctas;
  for (int k = 0; k < n_streams; ++k) {
    cudaStream_t st;
    e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
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
  if (C > kMaxMergedCells) return record_error(CBX_E_TOO_LARGE, "request has more cells than one launch takes (65536)");
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
  size_request(r, s->max_ctas);
  if (launch_bytes(r, C) > s->budget) {
    delete r;
    return record_error(CBX_E_TOO_LARGE, "request larger than the server's memory budget");
  }
  cudaError_t e = cudaMallocHost((void**)&r->h_phi, (size_t)C * sizeof(cbx_cell_params));
  if (e == cudaSuccess) e = cudaMallocHost((void**)&r->h_x, (size_t)r->S * C * sizeof(double));
  if (e == cudaSuccess) e = cudaMallocHost((void**)&r->h_tend, (size_t)C * sizeof(double));
  if (e == cudaSuccess) e = cudaMallocHost((void**)&r->h_status, (size_t)C * sizeof(int));
  if (e != cudaSuccess) {
    free_request(r);
    return record_error(CBX_E_NOMEM, "pinned staging allocation failed");
  }
  memcpy(r->h_phi, phi, (size_t)C * sizeof(cbx_cell_params));
  memcpy(r->h_x, x0, (size_t)r->S * C * sizeof(double));
  for (int c = 0; c < C; ++c) r->h_tend[c] = t_end;
  {
    std::unique_lock<std::mutex> lock(s->mu);
    if (s->stop) {
      lock.unlock();
      free_request(r);
      return record_error(CBX_E_ARG, "the server is being destroyed");
    }
    r->id = s->next_id++;
    r->t_submit = now_s();
    s->reqs[r->id] = r;
    s->queue.push_back(r);
    *request_id = r->id;
  }
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
  s->waiting++;
  s->cv.wait(lock, [&] { return r->state >= kDone; });
  s->waiting--;
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
  s->reqs.erase(request_id);
  lock.unlock();
  s->cv.notify_all();  // cbx_server_destroy may wait for the last waiter
  free_request(r);
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

int cbx_server_info(cbx_server* s, size_t* budget, long long* launches, long long* merged_requests) {
  if (!s) return record_error(CBX_E_ARG, "server is NULL");
  std::lock_guard<std::mutex> lock(s->mu);
  if (budget) *budget = s->budget;
  if (launches) *launches = s->launches;
  if (merged_requests) *merged_requests = s->merged_requests;
  return CBX_OK;
}

int cbx_server_destroy(cbx_server* s) {
  if (!s) return CBX_OK;
  {
    std::unique_lock<std::mutex> lock(s->mu);
    s->stop = true;
    // queued requests will not run: fail them so that their waiters return
    for (ServerRequest* r : s->queue) {
      r->state = kFailed;
      r->rc = CBX_E_ARG;
      r->t_done = now_s();
    }
    s->queue.clear();
    s->cv.notify_all();
    s->cv.wait(lock, [&] {
      for (char b : s->busy)
        if (b) return false;
      return s->waiting == 0;
    });
  }
  s->sched.join();
  for (cudaStream_t st : s->streams) cudaStreamDestroy(st);
  for (auto& kv : s->reqs) free_request(kv.second);
  delete s;
  return CBX_OK;
}

}  // extern "C"
