// C ABI glue: argument checks, device upload of compiled networks, workspace
// and launches. Every entry point returns a CBX_* code and records a message.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <algorithm>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "internal.h"

using namespace cbx;


namespace {

thread_local std::string g_err;

int fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}

int cuda_fail(cudaError_t e, const char* what) {
  return fail(CBX_E_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

// Pack int and double tables into one device buffer.
struct Packer {
  std::vector<unsigned char> bytes;
  template <typename T>
  size_t add(const std::vector<T>& v) {
    size_t off = (bytes.size() + 255) & ~size_t(255);
    bytes.resize(off + v.size() * sizeof(T) + 1);
    if (!v.empty()) memcpy(bytes.data() + off, v.data(), v.size() * sizeof(T));
    return off;
  }
};

int check_options(const cbx_options& o) {
  if (!(o.rtol > 0.0) || !std::isfinite(o.rtol)) return fail(CBX_E_ARG, "rtol must be finite and > 0");
  if (!(o.atol >= 0.0) || !std::isfinite(o.atol)) return fail(CBX_E_ARG, "atol must be finite and >= 0");
  if (o.max_steps < 1) return fail(CBX_E_ARG, "max_steps must be >= 1");
  if (o.precision != CBX_FP64 && o.precision != CBX_MIXED) return fail(CBX_E_ARG, "precision must be CBX_FP64 or CBX_MIXED");
  if (o.precision == CBX_MIXED && o.max_refine < 1) return fail(CBX_E_ARG, "max_refine must be >= 1");
  if (!(o.refine_tol >= 0.0)) return fail(CBX_E_ARG, "refine_tol must be >= 0");
  if (o.method != CBX_METHOD_BDF && o.method != CBX_METHOD_ESDIRK)
    return fail(CBX_E_ARG, "method must be CBX_METHOD_BDF or CBX_METHOD_ESDIRK");
  return CBX_OK;
}

// Upload the compiled tables to the current device (once per network).
int upload(cbx_network* n) {
  std::lock_guard<std::mutex> lock(n->mu);
  if (n->dbuf) return CBX_OK;
  const HostNet& h = n->host;
  Packer pk;
  size_t o_rtype = pk.add(h.rtype), o_alpha = pk.add(h.alpha), o_beta = pk.add(h.beta),
         o_gamma = pk.add(h.gamma), o_ra = pk.add(h.ra), o_rb = pk.add(h.rb), o_seg = pk.add(h.seg_ptr),
         o_sps = pk.add(h.spec_seg), o_ent = pk.add(h.rhs_ent), o_jrow = pk.add(h.jrow),
         o_jcol = pk.add(h.jcol), o_jrp = pk.add(h.jrow_ptr), o_jgp = pk.add(h.jg_ptr),
         o_jgs = pk.add(h.jg_slot), o_jgl = pk.add(h.jg_len), o_jgt = pk.add(h.jg_term), o_plp = pk.add(h.piv_lptr), o_pl = pk.add(h.piv_l),
         o_pup = pk.add(h.piv_uptr), o_pu = pk.add(h.piv_u), o_perm = pk.add(h.perm),
         o_rprod = pk.add(h.rprod), o_rj = pk.add(h.rj), o_gb = pk.add(h.gbeta), o_gg = pk.add(h.ggamma);
  cudaGetDevice(&n->device);
  cudaError_t e = cudaMalloc(&n->dbuf, pk.bytes.size());
  if (e != cudaSuccess) {
    n->dbuf = nullptr;
    return cuda_fail(e, "cudaMalloc(network tables)");
  }
  e = cudaMemcpy(n->dbuf, pk.bytes.data(), pk.bytes.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaFree(n->dbuf);
    n->dbuf = nullptr;
    return cuda_fail(e, "cudaMemcpy(network tables)");
  }
  unsigned char* b = (unsigned char*)n->dbuf;
  DevNet& d = n->dev;
  d.S = h.S;
  d.R = h.R;
  d.nnzJ = h.nnzJ;
  d.nseg = h.nseg;
  d.kdense = h.kdense;
  d.sparse_panels = h.sparse_panels;
  d.rtype = (const int*)(b + o_rtype);
  d.alpha = (const double*)(b + o_alpha);
  d.beta = (const double*)(b + o_beta);
  d.gamma = (const double*)(b + o_gamma);
  d.ra = (const int*)(b + o_ra);
  d.rb = (const int*)(b + o_rb);
  d.seg_ptr = (const int*)(b + o_seg);
  d.spec_seg = (const int*)(b + o_sps);
  d.rhs_ent = (const int*)(b + o_ent);
  d.jrow = (const int*)(b + o_jrow);
  d.jcol = (const int*)(b + o_jcol);
  d.jrow_ptr = (const int*)(b + o_jrp);
  d.njg = h.njg;
  d.jg_ptr = (const int*)(b + o_jgp);
  d.jg_slot = (const int*)(b + o_jgs);
  d.jg_len = (const int*)(b + o_jgl);
  d.jg_term = (const int*)(b + o_jgt);
  d.piv_lptr = (const int*)(b + o_plp);
  d.piv_l = (const int*)(b + o_pl);
  d.piv_uptr = (const int*)(b + o_pup);
  d.piv_u = (const int*)(b + o_pu);
  d.perm = (const int*)(b + o_perm);
  d.rprod = (const int*)(b + o_rprod);
  for (int t = 0; t <= kNumTypes; ++t) d.tptr[t] = h.tptr[t];
  d.rj = (const int*)(b + o_rj);
  d.gbeta = (const double*)(b + o_gb);
  d.ggamma = (const double*)(b + o_gg);
  d.albedo_factor = 1.0 / (1.0 - h.albedo);
  return CBX_OK;
}

}  // namespace

struct cbx_tape {
  cbx_network* net = nullptr;
  int C = 0, S = 0;
  TapeDev dev;
  void* dbuf = nullptr;
  cbx_cell_params* phi = nullptr;  // [C] copy of the recorded solve's parameters
  double* x0 = nullptr;            // [S][C] copy of its initial abundances
  int* status = nullptr;           // [C] its cell status
  double* alpha = nullptr;         // [R] the alpha values the recorded solve used
  double* track = nullptr;         // [C][K][6] copy of the recorded solve's tracks (own allocation)
  size_t track_cap = 0;            // doubles allocated at track
  int K = 0;                       // 0: the recorded solve had a constant environment
  double t0 = 0.0;
  int recorded_C = 0;
};

namespace cbx {
// Record an error message for cbx_last_error() from another translation unit.
int record_error(int code, const std::string& msg) { return fail(code, msg); }
}  // namespace cbx

extern "C" {

int cbx_version(void) { return CBX_VERSION; }

const char* cbx_last_error(void) { return g_err.c_str(); }

int cbx_default_options(cbx_options* out) {
  if (!out) return fail(CBX_E_ARG, "out is NULL");
  memset(out, 0, sizeof *out);
  out->rtol = 1e-4;
  out->atol = 1e-20;
  out->max_steps = 100000;
  out->precision = CBX_FP64;
  out->max_refine = 5;
  out->refine_tol = 1e-10;
  out->method = CBX_METHOD_BDF;
  return CBX_OK;
}

int cbx_network_create(const cbx_species* species, int S, const cbx_reaction* reactions, int R,
                       cbx_network** out) {
  if (!out) return fail(CBX_E_ARG, "out is NULL");
  *out = nullptr;
  cbx_network* n = new (std::nothrow) cbx_network();
  if (!n) return fail(CBX_E_NOMEM, "host allocation failed");
  std::string msg = compile_network(species, S, reactions, R, &n->host);
  if (!msg.empty()) {
    delete n;
    return fail(CBX_E_ARG, msg);
  }
  int dc = 0;
  if (cudaGetDeviceCount(&dc) == cudaSuccess && dc > 0) {
    const int rc = upload(n);
    if (rc != CBX_OK) {
      delete n;
      return rc;
    }
  } else {
    cudaGetLastError();
  }
  *out = n;
  return CBX_OK;
}

int cbx_network_destroy(cbx_network* net) {
  if (!net) return CBX_OK;
  if (net->dbuf) cudaFree(net->dbuf);
  delete net;
  return CBX_OK;
}

int cbx_network_info(const cbx_network* net, cbx_netinfo* out) {
  if (!net || !out) return fail(CBX_E_ARG, "NULL argument");
  const HostNet& h = net->host;
  out->S = h.S;
  out->R = h.R;
  out->nnz_jac = h.nnzJ;
  out->nnz_lu = h.nnzLU;
  out->lu_flops = h.lu_flops;
  out->lu_flops_dense = 2.0 * h.S * (double)h.S * h.S / 3.0;
  out->smem_bytes_fp64 = (int)smem_bytes(h.S, h.R, h.nseg, false, false, h.head_ints);
  out->smem_bytes_mixed = (int)smem_bytes(h.S, h.R, h.nseg, true, false);
  return CBX_OK;
}

int cbx_network_symbolic(const cbx_network* net, int* perm, unsigned char* fill, int* kdense) {
  if (!net) return fail(CBX_E_ARG, "net is NULL");
  const HostNet& h = net->host;
  const int S = h.S;
  if (perm)
    for (int i = 0; i < S; ++i) perm[i] = h.perm[i];
  if (kdense) *kdense = h.kdense;
  if (fill) {
    memset(fill, 0, (size_t)S * S);
    for (int k = 0; k < S; ++k) {
      fill[(size_t)k * S + k] = 1;
      for (int e = h.piv_lptr[k]; e < h.piv_lptr[k + 1]; ++e) fill[(size_t)h.piv_l[e] * S + k] = 1;
      for (int e = h.piv_uptr[k]; e < h.piv_uptr[k + 1]; ++e) fill[(size_t)k * S + h.piv_u[e]] = 1;
    }
  }
  return CBX_OK;
}

}  // extern "C"

static int solve_impl(cbx_network* net, const cbx_cell_params* phi, const double* x0, int C, double t0,
                      double t_end, const cbx_options* opt, void* stream, double* x_out, int* cell_status,
                      cbx_cell_stats* stats, cbx_tape* tape, int max_grid = 0, const double* track = nullptr,
                      int K = 0, const double* alpha = nullptr, const double* t_end_cell = nullptr) {
  if (!net) return fail(CBX_E_ARG, "net is NULL");
  if (C < 0) return fail(CBX_E_ARG, "C must be >= 0");
  if (C > 0 && ((!phi && !track) || !x0 || !x_out || !cell_status)) return fail(CBX_E_ARG, "NULL array with C > 0");
  if (!std::isfinite(t0) || !std::isfinite(t_end) || t_end < t0) return fail(CBX_E_ARG, "need finite t0 <= t_end");
  cbx_options o;
  cbx_default_options(&o);
  if (opt) o = *opt;
  int rc = check_options(o);
  if (rc) return rc;
  const bool rk = o.method == CBX_METHOD_ESDIRK;
  if (rk && tape) return fail(CBX_E_ARG, "recording (the adjoint) is implemented for CBX_METHOD_BDF only");
  if (C == 0) return CBX_OK;
  rc = upload(net);
  if (rc) return rc;
  const HostNet& h = net->host;
  const bool mixed = o.precision == CBX_MIXED;
  const SolverPlan plan = plan_solver(h.S, h.R, h.nseg, h.nnzJ, mixed, h.head_ints);
  const int occ = plan.occupancy;
  if (occ < 1) {
    char m[200];
    snprintf(m, sizeof m, "network (S=%d, R=%d) needs %zu B of shared memory per CTA (S <= %d); the device allows %zu",
             h.S, h.R, plan.smem, 512, device_smem_optin());
    return fail(CBX_E_TOO_LARGE, m);
  }
  int grid = std::min(C, occ * device_sm_count());
  if (max_grid > 0) grid = std::min(grid, max_grid);
  cudaStream_t st = (cudaStream_t)stream;
  SolveArgs a{};
  a.net = net->dev;
  a.alpha = alpha ? alpha : net->dev.alpha;
  a.phi = phi;
  a.track = track;
  a.K = K;
  a.t_end_cell = t_end_cell;
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
  if (tape) a.tape = tape->dev;
  a.ws_stride = plan.ws_stride;
  const size_t ws_bytes = (size_t)grid * a.ws_stride * sizeof(double) + 256;
  void* ws = nullptr;
  cudaError_t e = cudaMallocAsync(&ws, ws_bytes, st);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMallocAsync(workspace)");
  a.ws = (double*)ws;
  a.counter = (int*)((char*)ws + (size_t)grid * a.ws_stride * sizeof(double));
  if (rk) {
    const EsdirkTableau& tb = esdirk_tableau();
    for (int i = 0; i < 5; ++i) {
      a.rk_c[i] = tb.c[i];
      for (int j = 0; j < 5; ++j) a.rk_a[i][j] = tb.a[i][j];
    }
  }
  e = cudaMemsetAsync(a.counter, 0, sizeof(int), st);
  if (e == cudaSuccess)
    e = (cudaError_t)(rk ? launch_solver_rk(a, plan, grid, stream) : launch_solver(a, plan, grid, stream));
  cudaError_t e2 = cudaFreeAsync(ws, st);
  if (e != cudaSuccess) return cuda_fail(e, "solver launch");
  if (e2 != cudaSuccess) return cuda_fail(e2, "cudaFreeAsync(workspace)");
  if (tape) {
    e = cudaSuccess;
    if (track) {
      const size_t nd = (size_t)C * K * 6;
      if (tape->track_cap < nd) {
        if (tape->track) {
          cudaStreamSynchronize(st);
          cudaFree(tape->track);
          tape->track = nullptr;
          tape->track_cap = 0;
        }
        e = cudaMalloc(&tape->track, nd * sizeof(double));
        if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(tape track)");
        tape->track_cap = nd;
      }
      e = cudaMemcpyAsync(tape->track, track, nd * sizeof(double), cudaMemcpyDeviceToDevice, st);
      tape->K = K;
    } else {
      e = cudaMemcpyAsync(tape->phi, phi, C * sizeof(cbx_cell_params), cudaMemcpyDeviceToDevice, st);
      tape->K = 0;
    }
    tape->t0 = t0;
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(tape->x0, x0, (size_t)h.S * C * sizeof(double), cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(tape->status, cell_status, C * sizeof(int), cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess && h.R > 0)
      e = cudaMemcpyAsync(tape->alpha, a.alpha, (size_t)h.R * sizeof(double), cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync(tape copies)");
    tape->recorded_C = C;
  }
  return CBX_OK;
}


extern "C" {

int cbx_solve(cbx_network* net, const cbx_cell_params* phi, const double* x0, int C, double t0,
              double t_end, const cbx_options* opt, void* stream, double* x_out, int* cell_status,
              cbx_cell_stats* stats) {
  return solve_impl(net, phi, x0, C, t0, t_end, opt, stream, x_out, cell_status, stats, nullptr);
}

int cbx_solve_track(cbx_network* net, const double* track, int K, const double* x0, int C, double t0, double t_end,
                    const cbx_options* opt, void* stream, double* x_out, int* cell_status, cbx_cell_stats* stats) {
  if (K < 1) return fail(CBX_E_ARG, "K must be >= 1");
  if (C > 0 && !track) return fail(CBX_E_ARG, "track is NULL");
  return solve_impl(net, nullptr, x0, C, t0, t_end, opt, stream, x_out, cell_status, stats, nullptr, 0, track, K);
}

int cbx_solve_host(cbx_network* net, const cbx_cell_params* phi, const double* x0, int C, double t0,
                   double t_end, const cbx_options* opt, void* stream, double* x_out,
                   int* cell_status, cbx_cell_stats* stats) {
  if (!net) return fail(CBX_E_ARG, "net is NULL");
  if (C < 0) return fail(CBX_E_ARG, "C must be >= 0");
  if (C > 0 && (!phi || !x0 || !x_out || !cell_status)) return fail(CBX_E_ARG, "NULL array with C > 0");
  if (C == 0) return cbx_solve(net, phi, x0, 0, t0, t_end, opt, stream, x_out, cell_status, stats);
  cudaStream_t st = (cudaStream_t)stream;
  const size_t S = net->host.S;
  const size_t b_phi = C * sizeof(cbx_cell_params), b_x = S * C * sizeof(double), b_st = C * sizeof(int),
               b_stats = stats ? C * sizeof(cbx_cell_stats) : 0;
  char* d = nullptr;
  const size_t o_x0 = (b_phi + 255) & ~size_t(255), o_xo = o_x0 + ((b_x + 255) & ~size_t(255)),
               o_st = o_xo + ((b_x + 255) & ~size_t(255)), o_stats = o_st + ((b_st + 255) & ~size_t(255)),
               total = o_stats + b_stats + 256;
  cudaError_t e = cudaMallocAsync((void**)&d, total, st);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMallocAsync(host-call buffers)");
  int rc = CBX_OK;
  e = cudaMemcpyAsync(d, phi, b_phi, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d + o_x0, x0, b_x, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) {
    rc = cuda_fail(e, "cudaMemcpyAsync(H2D)");
  } else {
    rc = cbx_solve(net, (const cbx_cell_params*)d, (const double*)(d + o_x0), C, t0, t_end, opt, stream,
                   (double*)(d + o_xo), (int*)(d + o_st), stats ? (cbx_cell_stats*)(d + o_stats) : nullptr);
    if (rc == CBX_OK) {
      e = cudaMemcpyAsync(x_out, d + o_xo, b_x, cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess) e = cudaMemcpyAsync(cell_status, d + o_st, b_st, cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess && stats) e = cudaMemcpyAsync(stats, d + o_stats, b_stats, cudaMemcpyDeviceToHost, st);
      if (e != cudaSuccess) rc = cuda_fail(e, "cudaMemcpyAsync(D2H)");
    }
  }
  cudaFreeAsync(d, st);
  e = cudaStreamSynchronize(st);
  if (rc == CBX_OK && e != cudaSuccess) rc = cuda_fail(e, "cudaStreamSynchronize");
  return rc;
}

int cbx_network_set_alpha(cbx_network* net, const double* alpha) {
  if (!net || (!alpha && net->host.R > 0)) return fail(CBX_E_ARG, "NULL argument");
  for (int j = 0; j < net->host.R; ++j)
    if (!(alpha[j] == alpha[j])) return fail(CBX_E_ARG, "alpha has a NaN");
  std::lock_guard<std::mutex> lock(net->mu);
  for (int j = 0; j < net->host.R; ++j) net->host.alpha[j] = alpha[j];
  if (net->dbuf && net->host.R > 0) {
    cudaError_t e = cudaMemcpy((void*)net->dev.alpha, alpha, net->host.R * sizeof(double), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy(alpha)");
  }
  return CBX_OK;
}

int cbx_network_set_albedo(cbx_network* net, double omega) {
  if (!net) return fail(CBX_E_ARG, "net is NULL");
  if (!(omega >= 0.0 && omega < 1.0)) return fail(CBX_E_ARG, "omega must be in [0, 1)");
  std::lock_guard<std::mutex> lock(net->mu);
  net->host.albedo = omega;
  net->dev.albedo_factor = 1.0 / (1.0 - omega);
  return CBX_OK;
}

int cbx_tape_create(cbx_network* net, int C, int max_steps, cbx_tape** out) {
  if (!net || !out) return fail(CBX_E_ARG, "NULL argument");
  *out = nullptr;
  if (C < 1 || max_steps < 1) return fail(CBX_E_ARG, "need C >= 1 and max_steps >= 1");
  int rc = upload(net);
  if (rc) return rc;
  cbx_tape* t = new (std::nothrow) cbx_tape();
  if (!t) return fail(CBX_E_NOMEM, "host allocation failed");
  t->net = net;
  t->C = C;
  t->S = net->host.S;
  t->dev.cap_steps = max_steps;
  t->dev.cap_ops = 4 * max_steps + 16;
  const size_t n_ops = (size_t)C * t->dev.cap_ops;
  auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
  const size_t o_nops = 0, o_kq = o_nops + al(C * 4), o_v = o_kq + al(n_ops * 4), o_y = o_v + al(n_ops * 8),
               o_ts = o_y + al((size_t)C * max_steps * t->S * 8), o_phi = o_ts + al((size_t)C * max_steps * 8),
               o_x0 = o_phi + al(C * sizeof(cbx_cell_params)),
               o_st = o_x0 + al((size_t)t->S * C * 8), o_al = o_st + al(C * 4),
               total = o_al + al((size_t)net->host.R * 8 + 8);
  cudaError_t e = cudaMalloc(&t->dbuf, total);
  if (e != cudaSuccess) {
    delete t;
    return cuda_fail(e, "cudaMalloc(tape)");
  }
  char* b = (char*)t->dbuf;
  t->dev.nops = (int*)(b + o_nops);
  t->dev.ops_kq = (int*)(b + o_kq);
  t->dev.ops_v = (double*)(b + o_v);
  t->dev.ys = (double*)(b + o_y);
  t->dev.ts = (double*)(b + o_ts);
  t->phi = (cbx_cell_params*)(b + o_phi);
  t->x0 = (double*)(b + o_x0);
  t->status = (int*)(b + o_st);
  t->alpha = (double*)(b + o_al);
  e = cudaMemset(t->dev.nops, 0, C * sizeof(int));
  if (e != cudaSuccess) {
    cudaFree(t->dbuf);
    delete t;
    return cuda_fail(e, "cudaMemset(tape)");
  }
  *out = t;
  return CBX_OK;
}

int cbx_tape_destroy(cbx_tape* tape) {
  if (!tape) return CBX_OK;
  if (tape->dbuf) cudaFree(tape->dbuf);
  if (tape->track) cudaFree(tape->track);
  delete tape;
  return CBX_OK;
}

int cbx_solve_record(cbx_network* net, const cbx_cell_params* phi, const double* x0, int C, double t0,
                     double t_end, const cbx_options* opt, void* stream, double* x_out, int* cell_status,
                     cbx_cell_stats* stats, cbx_tape* tape) {
  if (!tape) return fail(CBX_E_ARG, "tape is NULL");
  if (tape->net != net) return fail(CBX_E_ARG, "the tape belongs to another network");
  if (C > tape->C) return fail(CBX_E_ARG, "C exceeds the tape's capacity");
  return solve_impl(net, phi, x0, C, t0, t_end, opt, stream, x_out, cell_status, stats, tape);
}

int cbx_solve_with_alpha(cbx_network* net, const double* alpha, const cbx_cell_params* phi, const double* x0, int C,
                         double t0, double t_end, const cbx_options* opt, void* stream, double* x_out,
                         int* cell_status, cbx_cell_stats* stats, cbx_tape* tape) {
  if (!alpha && net && net->host.R > 0) return fail(CBX_E_ARG, "alpha is NULL");
  if (tape) {
    if (tape->net != net) return fail(CBX_E_ARG, "the tape belongs to another network");
    if (C > tape->C) return fail(CBX_E_ARG, "C exceeds the tape's capacity");
  }
  return solve_impl(net, phi, x0, C, t0, t_end, opt, stream, x_out, cell_status, stats, tape, 0, nullptr, 0, alpha);
}

int cbx_solve_track_record(cbx_network* net, const double* track, int K, const double* x0, int C, double t0,
                           double t_end, const cbx_options* opt, void* stream, double* x_out, int* cell_status,
                           cbx_cell_stats* stats, cbx_tape* tape) {
  if (!tape) return fail(CBX_E_ARG, "tape is NULL");
  if (tape->net != net) return fail(CBX_E_ARG, "the tape belongs to another network");
  if (C > tape->C) return fail(CBX_E_ARG, "C exceeds the tape's capacity");
  if (K < 1) return fail(CBX_E_ARG, "K must be >= 1");
  if (C > 0 && !track) return fail(CBX_E_ARG, "track is NULL");
  return solve_impl(net, nullptr, x0, C, t0, t_end, opt, stream, x_out, cell_status, stats, tape, 0, track, K);
}

int cbx_tape_step_times(const cbx_tape* tape, int cell, double* t_new, int cap) {
  if (!tape || cell < 0 || cell >= tape->C || cap < 0) return fail(CBX_E_ARG, "bad argument");
  int nops = 0;
  cudaError_t e = cudaMemcpy(&nops, tape->dev.nops + cell, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy(tape)");
  std::vector<int> kq(nops);
  if (nops > 0) {
    e = cudaMemcpy(kq.data(), tape->dev.ops_kq + (size_t)cell * tape->dev.cap_ops, nops * sizeof(int),
                   cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy(tape)");
  }
  int n = 0;
  for (int v : kq) n += (v >> 8) == kOpStep;
  const int m = std::min(n, cap);
  if (m > 0 && t_new) {
    e = cudaMemcpy(t_new, tape->dev.ts + (size_t)cell * tape->dev.cap_steps, m * sizeof(double),
                   cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy(tape)");
  }
  return n;
}

int cbx_grad(cbx_tape* tape, const double* cot_x, void* stream, double* g_logalpha, double* g_lognH,
             double* g_T) {
  return cbx_grad_env(tape, cot_x, stream, g_logalpha, g_lognH, g_T, nullptr, nullptr, nullptr);
}

int cbx_grad_env(cbx_tape* tape, const double* cot_x, void* stream, double* g_logalpha, double* g_lognH,
                 double* g_T, double* g_lnzeta, double* g_lnG0, double* g_AV) {
  if (!tape) return fail(CBX_E_ARG, "tape is NULL");
  const int C = tape->recorded_C;
  if (C < 1) return fail(CBX_E_ARG, "nothing recorded on this tape");
  if (!cot_x) return fail(CBX_E_ARG, "cot_x is NULL");
  cbx_network* net = tape->net;
  const HostNet& h = net->host;
  const int occ = grad_occupancy(h.S, h.R, h.nseg);
  if (occ < 1) return fail(CBX_E_TOO_LARGE, "the adjoint supports networks whose FP64 matrix fits in shared memory");
  const int grid = std::min(C, occ * device_sm_count());
  cudaStream_t st = (cudaStream_t)stream;
  GradArgs a{};
  a.net = net->dev;
  a.alpha = tape->alpha;
  a.tape = tape->dev;
  a.phi = tape->K > 0 ? nullptr : tape->phi;
  a.track = tape->K > 0 ? tape->track : nullptr;
  a.K = tape->K;
  a.t0 = tape->t0;
  a.status = tape->status;
  a.x0 = tape->x0;
  a.cot = cot_x;
  a.C = C;
  for (int q = 0; q < kMaxOrder + 2; ++q) {
    double g = 0.0;
    for (int j = 1; j <= q; ++j) g += 1.0 / j;
    a.gam[q] = g;
  }
  a.g_lognH = g_lognH;
  a.g_T = g_T;
  a.ws_stride = grad_workspace_doubles(h.S, h.R, h.nnzJ);
  const size_t b_gcell = ((size_t)C * h.R * 8 + 255) & ~size_t(255);
  const size_t b_ws = (size_t)grid * a.ws_stride * 8;
  char* buf = nullptr;
  cudaError_t e = cudaMallocAsync((void**)&buf, b_gcell + b_ws + 256, st);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMallocAsync(adjoint workspace)");
  a.gcell = (double*)buf;
  a.ws = (double*)(buf + b_gcell);
  a.counter = (int*)(buf + b_gcell + b_ws);
  e = cudaMemsetAsync(a.counter, 0, sizeof(int), st);
  if (e == cudaSuccess) e = (cudaError_t)launch_grad(a, grid, stream);
  if (e == cudaSuccess && g_logalpha) e = (cudaError_t)launch_reduce_cells(a.gcell, C, h.R, g_logalpha, stream);
  if (e == cudaSuccess && (g_lnzeta || g_lnG0 || g_AV))
    e = (cudaError_t)launch_env_grad(a.gcell, C, net->dev, g_lnzeta, g_lnG0, g_AV, stream);
  cudaError_t e2 = cudaFreeAsync(buf, st);
  if (e != cudaSuccess) return cuda_fail(e, "adjoint launch");
  if (e2 != cudaSuccess) return cuda_fail(e2, "cudaFreeAsync(adjoint workspace)");
  return CBX_OK;
}

int cbx_tape_program(const cbx_tape* tape, int cell, int* kinds, int* qs, double* values, int cap) {
  if (!tape || cell < 0 || cell >= tape->C || cap < 0) return fail(CBX_E_ARG, "bad argument");
  int n = 0;
  cudaError_t e = cudaMemcpy(&n, tape->dev.nops + cell, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy(tape)");
  const int m = std::min(n, cap);
  if (m > 0) {
    std::vector<int> kq(m);
    e = cudaMemcpy(kq.data(), tape->dev.ops_kq + (size_t)cell * tape->dev.cap_ops, m * sizeof(int), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && values)
      e = cudaMemcpy(values, tape->dev.ops_v + (size_t)cell * tape->dev.cap_ops, m * sizeof(double), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy(tape)");
    for (int i = 0; i < m; ++i) {
      if (kinds) kinds[i] = kq[i] >> 8;
      if (qs) qs[i] = kq[i] & 255;
    }
  }
  return n;
}

}  // extern "C"

namespace cbx {
int solve_device(cbx_network* net, const cbx_cell_params* phi, const double* x0, int C, double t0, double t_end,
                 const cbx_options* opt, void* stream, double* x_out, int* cell_status, int max_grid,
                 const double* t_end_cell) {
  return solve_impl(net, phi, x0, C, t0, t_end, opt, stream, x_out, cell_status, nullptr, nullptr, max_grid, nullptr,
                    0, nullptr, t_end_cell);
}
}  // namespace cbx
