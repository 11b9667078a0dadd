// Device code of the persistent per-cell solver, shared by the translation
// units that instantiate its kernels (one per precision and matrix placement,
// compiled in parallel) and by the adjoint. Everything here has internal
// linkage (anonymous namespace): each translation unit gets its own copy.
//
// Persistent per-cell BDF solver for sm_103a.
//
// One CTA integrates one cell at a time from t0 to t_end entirely on chip and
// then takes the next cell from an atomic counter (cells finish at different
// step counts; the counter keeps every SM busy until the batch is done). The
// cell's Newton matrix M = I - cJ lives densely in shared memory (the symbolic
// LU fill of these networks is ~80 % dense), the network tables are read-only
// and shared by all CTAs through L1/L2, and the per-cell FP64 Jacobian values
// sit in a per-CTA global workspace (L2-resident).
//
// The integrator is the variable-order (1..5), quasi-constant-step BDF in
// backward-difference form (Shampine & Reichelt 1997, kappa = 0) - the BDF
// family that Sec. 1 of the paper names as the field's stiff integrator - with
// a simplified Newton iteration on (I - cJ) dy = c f(y) - psi - d, c = h/gamma_q.
// Constants and policies:
//   Newton        <= 4 iterations; rate = |dy_k| / |dy_{k-1}|; fail when
//                 rate >= 1 or rate^(4-k)/(1-rate) |dy_k| > tol_N; converged
//                 when |dy| = 0 or rate/(1-rate) |dy| < tol_N
//   norms         weighted RMS, weights 1/(atol + rtol |y|): predictor for
//                 Newton, result for the error test
//   error test    |d/(q+1)| <= 1; on failure h *= max(0.2, 0.9 err^(-1/(q+1)))
//   Newton fail   re-evaluate J if it is stale, else h *= 0.5
//   step/order    after q+1 equal steps: estimates at q-1, q, q+1, the largest
//                 factor err_k^(-1/(k+1)) wins; h *= min(10, 0.9 factor)
//   LU            refactored whenever h or J changed
//   initial step  Hairer, Norsett & Wanner I, Sec. II.4 (order 1)
//   limits        max_steps attempts; h < 10 ulp(t) -> H_UNDERFLOW
//
// FP64 on GB300 retires about 2 FMA per clock per SM, so one warp-wide FP64
// instruction holds the SM's FP64 pipe for ~16 clocks whatever its active
// lanes: the vector loops below keep lanes full, and scalar FP64 work (pow,
// the rescale matrix) runs on one thread or one warp and is broadcast.
#pragma once
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>

#include "internal.h"

#ifndef CBX_THREADS
#define CBX_THREADS 256
#endif

namespace cbx {
namespace {

constexpr int NT = CBX_THREADS;  // threads per CTA
constexpr int NW = NT / 32;
constexpr int kNewtonMaxIter = 4;
constexpr int kMaxColRegs = 8;  // columns per lane in the LU update: S <= 256
constexpr unsigned FULL = 0xffffffffu;

// ---------------------------------------------------------------- helpers

__device__ __forceinline__ unsigned long long globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

// Deterministic block sum: warp trees, then the NW partials in a fixed order.
// Every thread returns the same value. Contains two barriers.
__device__ __forceinline__ double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    double s = 0.0;
    for (int i = 0; i < NW; ++i) s += red[i];
    if (threadIdx.x == 0) red[NW] = s;
  }
  __syncthreads();
  const double s = red[NW];
  __syncthreads();
  return s;
}

// sqrt(mean((a * v_i * w_i)^2)), w = reciprocal weights
__device__ double wrms(const double* v, const double* w, double a, int S, double* red) {
  double acc = 0.0;
  for (int i = threadIdx.x; i < S; i += NT) {
    const double t = a * v[i] * w[i];
    acc = fma(t, t, acc);
  }
  return sqrt(block_sum(acc, red) / S);
}

// One thread computes pow(x, y); everybody gets it.
__device__ double uniform_pow(double x, double y, double* slot) {
  if (threadIdx.x == 0) *slot = pow(x, y);
  __syncthreads();
  const double v = *slot;
  __syncthreads();
  return v;
}

__device__ __forceinline__ double growth(double err, int p, double* slot) {
  return err == 0.0 ? INFINITY : uniform_pow(err, -1.0 / p, slot);
}

// ---------------------------------------------------------------- chemistry

// kappa_j of one cell (Sec. 2 two-body and cosmic-ray forms, App. B.1 photo
// and cosmic-ray-induced photo forms); two-body values carry the n_H factor
// of x = n / n_H. The reactions of each type form one contiguous group of the
// network's grouped tables (Sec. 4: rates of identical mechanisms are
// evaluated together), so every loop below is free of divergent branches.
// alpha: [R], the alpha values of this solve.
__device__ void rate_coefficients(const DevNet& n, const double* __restrict__ alpha, const cbx_cell_params& p,
                                  double* kap) {
  const double lnT = log(p.T / 300.0);
  const double invT = 1.0 / p.T;
  for (int e = n.tptr[CBX_TWO_BODY] + threadIdx.x; e < n.tptr[CBX_TWO_BODY + 1]; e += NT) {
    const int j = __ldg(n.rj + e);
    kap[j] = alpha[j] * exp(__ldg(n.gbeta + e) * lnT - __ldg(n.ggamma + e) * invT) * p.n_H;
  }
  for (int e = n.tptr[CBX_COSMIC_RAY] + threadIdx.x; e < n.tptr[CBX_COSMIC_RAY + 1]; e += NT) {
    const int j = __ldg(n.rj + e);
    kap[j] = alpha[j] * p.zeta;
  }
  for (int e = n.tptr[CBX_PHOTO] + threadIdx.x; e < n.tptr[CBX_PHOTO + 1]; e += NT) {
    const int j = __ldg(n.rj + e);
    kap[j] = alpha[j] * p.G0 * exp(-__ldg(n.ggamma + e) * p.A_V);
  }
  // k = alpha (T/300)^beta E / (1 - omega) zeta, E in the gamma field
  const double crp = p.zeta * n.albedo_factor;
  for (int e = n.tptr[CBX_CR_PHOTO] + threadIdx.x; e < n.tptr[CBX_CR_PHOTO + 1]; e += NT) {
    const int j = __ldg(n.rj + e);
    kap[j] = alpha[j] * exp(__ldg(n.gbeta + e) * lnT) * __ldg(n.ggamma + e) * crp;
  }
}

// f = nu r(y): reaction rates into r, signed segment sums into part, then
// per-species sums of the segments (fixed order: bitwise reproducible). The
// network tables stream from L2, so each thread issues all its table loads
// of a pass before it uses any of them (one round trip instead of one per
// entry).
constexpr int kRatesPerPass = 8;
__device__ void rhs(const DevNet& n, const double* __restrict__ kap, const double* y, double* f,
                    double* r, double* part) {
  for (int j0 = threadIdx.x; j0 < n.R; j0 += kRatesPerPass * NT) {
    int ia[kRatesPerPass], ib[kRatesPerPass];
    double kv[kRatesPerPass];
#pragma unroll
    for (int u = 0; u < kRatesPerPass; ++u) {
      const int j = j0 + u * NT;
      const bool ok = j < n.R;
      ia[u] = ok ? __ldg(n.ra + j) : 0;
      ib[u] = ok ? __ldg(n.rb + j) : -1;
      kv[u] = ok ? kap[j] : 0.0;
    }
#pragma unroll
    for (int u = 0; u < kRatesPerPass; ++u) {
      const int j = j0 + u * NT;
      if (j < n.R) {
        double v = kv[u] * y[ia[u]];
        if (ib[u] >= 0) v *= y[ib[u]];
        r[j] = v;
      }
    }
  }
  __syncthreads();
  for (int sg = threadIdx.x; sg < n.nseg; sg += NT) {
    const int e0 = __ldg(n.seg_ptr + sg), len = __ldg(n.seg_ptr + sg + 1) - e0;
    int t[kSegLen];
#pragma unroll
    for (int u = 0; u < kSegLen; ++u) t[u] = u < len ? __ldg(n.rhs_ent + e0 + u) : 0;
    double v[kSegLen];
#pragma unroll
    for (int u = 0; u < kSegLen; ++u) v[u] = r[t[u] >> 1];
    double acc0 = 0.0, acc1 = 0.0;
#pragma unroll
    for (int u = 0; u < kSegLen; u += 2) {
      if (u < len) acc0 += (t[u] & 1) ? -v[u] : v[u];
      if (u + 1 < len) acc1 += (t[u + 1] & 1) ? -v[u + 1] : v[u + 1];
    }
    part[sg] = acc0 + acc1;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < n.S; i += NT) {
    double acc = 0.0;
    const int s1 = __ldg(n.spec_seg + i + 1);
    for (int sg = __ldg(n.spec_seg + i); sg < s1; ++sg) acc += part[sg];
    f[i] = acc;
  }
  __syncthreads();
}

// Analytic Jacobian values per slot: J(i,l) = sum nu_ij dr_j/dx_l, with the
// reaction partials g[2j+s] = d r_j / d x(reactant s).
__device__ void jacobian(const DevNet& n, const double* __restrict__ kap, const double* y, double* g,
                         double* Jv) {
  for (int j = threadIdx.x; j < n.R; j += NT) {
    const int b = n.rb[j];
    const double k = kap[j];
    if (b >= 0) {
      g[2 * j] = k * y[b];
      g[2 * j + 1] = k * y[n.ra[j]];
    } else {
      g[2 * j] = k;
      g[2 * j + 1] = 0.0;
    }
  }
  __syncthreads();
  // one warp per group of 32 slots; each lane sums its slot's terms in list
  // order (four loads ahead, one accumulator)
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int gi = warp; gi < n.njg; gi += NW) {
    const int s = __ldg(n.jg_slot + gi * 32 + lane);
    const int len = __ldg(n.jg_len + gi * 32 + lane);
    const int p0 = __ldg(n.jg_ptr + gi), cnt = (__ldg(n.jg_ptr + gi + 1) - p0) >> 5;
    const int* tp = n.jg_term + p0 + lane;
    double acc = 0.0;
    int e = 0;
    for (; e + 4 <= cnt; e += 4) {
      int t[4];
      double v[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) t[u] = __ldg(tp + 32 * (e + u));
#pragma unroll
      for (int u = 0; u < 4; ++u) v[u] = g[t[u] >> 1];
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (e + u < len) acc += (t[u] & 1) ? -v[u] : v[u];
    }
    for (; e < cnt; ++e) {
      const int t = __ldg(tp + 32 * e);
      const double v = g[t >> 1];
      if (e < len) acc += (t & 1) ? -v : v;
    }
    if (s >= 0) Jv[s] = acc;
  }
  __syncthreads();
}

// ---------------------------------------------------------------- linear algebra

__host__ __device__ inline int lead_dim(int S) { return S | 1; }  // odd: conflict-free column access

template <typename LT>
__device__ void build_matrix(const DevNet& n, const double* Jv, double c, LT* M) {
  const int S = n.S, ld = lead_dim(S);
  for (int idx = threadIdx.x; idx < S * ld; idx += NT) M[idx] = LT(0);
  __syncthreads();
  for (int s = threadIdx.x; s < n.nnzJ; s += NT) {
    const int i = n.jrow[s], l = n.jcol[s];
    const double cj = c * Jv[s];
    M[i * ld + l] = (LT)(i == l ? 1.0 - cj : -cj);
  }
  __syncthreads();
}

// ---------------------------------------------------------------- FP64 LU (Crout form)
//
// M = L U with L lower triangular (its diagonal holds the pivots) and U unit
// upper triangular, in place, without pivoting, on the static fill pattern.
// Row k of U is stored pre-scaled by 1/pivot_k, so every warp applies the
// rank-1 update a_ij -= a_ik u_kj (rows i of L(:,k), columns j of U(k,:)) with
// no separate scaling phase: one barrier per pivot in the sparse range. Warp 0
// updates row k+1 first and then prepares pivot k+1 (reciprocal pivot, row
// scaling) while the other warps work on their rows. Pivots k >= kd are
// factored over the full ranges k+1..S-1 (entries outside the pattern are
// exact zeros), without the per-pivot index lists, and there two pivots share
// one barrier (dense_rank_rows).

// Index lists of the sparse pivots k < kd (from the network tables, or a
// copy of their head in shared memory).
struct PivLists {
  int S, kd;
  const int* lptr;  // [kd+1]
  const int* l;
  const int* uptr;  // [kd+1]
  const int* u;
};

__device__ __forceinline__ PivLists global_pivots(const DevNet& n) {
  return PivLists{n.S, n.kdense, n.piv_lptr, n.piv_l, n.piv_uptr, n.piv_u};
}

__device__ __forceinline__ int lrow(const PivLists& P, bool dense, int k, int e) {
  return dense ? k + 1 + e : P.l[e];
}

// Reciprocal pivot and scaling of row k of U (warp-wide call).
__device__ void prep_pivot(const PivLists& P, double* M, double* invd, int k, int lane) {
  const int S = P.S, ld = lead_dim(S), kd = P.kd;
  const double inv = __drcp_rn(M[k * ld + k]);  // correctly rounded: equals 1.0 / pivot
  if (lane == 0) invd[k] = inv;
  if (k >= kd) {
    for (int j = k + 1 + lane; j < S; j += 32) M[k * ld + j] *= inv;
  } else {
    const int u1 = P.uptr[k + 1];
    for (int e = P.uptr[k] + lane; e < u1; e += 32) M[k * ld + P.u[e]] *= inv;
  }
}

// Rows r0 and (if two) r1 of L(:,k) minus their multiple of U(k,:), MC
// column groups per lane.
template <int MC>
__device__ __forceinline__ void update_rows(double* r0, double* r1, bool two, int k, const int (&jc)[MC],
                                            const double (&uv)[MC], int nu, int lane) {
  const double a = r0[k], b = r1[k];
  double x0[MC], x1[MC];
#pragma unroll
  for (int m = 0; m < MC; ++m) {
    x0[m] = r0[jc[m]];
    x1[m] = r1[jc[m]];
  }
#pragma unroll
  for (int m = 0; m < MC; ++m) x0[m] = fma(-a, uv[m], x0[m]);
  if (two) {
#pragma unroll
    for (int m = 0; m < MC; ++m) x1[m] = fma(-b, uv[m], x1[m]);
  }
#pragma unroll
  for (int m = 0; m < MC; ++m) {
    if (lane + 32 * m < nu) {
      r0[jc[m]] = x0[m];
      if (two) r1[jc[m]] = x1[m];
    }
  }
}

// All rows of L(:,k) assigned to this warp, with exactly MC column groups of
// U(k,:) per lane (a predicated FP64 instruction still takes the FP64 pipe).
// When row k+1 is in L(:,k), warp 0 updates it alone and prepares pivot k+1
// (in the dense trailing block the scaling by 1/pivot is applied in registers
// before the single store); the other warps take the other rows in pairs.
template <int MC>
__device__ __forceinline__ void crout_rows(const PivLists& P, double* M, double* invd, int k, bool dense,
                                           int l0, int l1, int u0, int nu, bool next_in_l) {
  const int ld = lead_dim(P.S);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int jc[MC];
  double uv[MC];
#pragma unroll
  for (int m = 0; m < MC; ++m) {
    const int b = lane + 32 * m;
    jc[m] = 0;
    uv[m] = 0.0;
    if (b < nu) {
      jc[m] = dense ? k + 1 + b : P.u[u0 + b];
      uv[m] = M[k * ld + jc[m]];
    }
  }
  if (next_in_l && w == 0) {
    double* r0 = M + (k + 1) * ld;
    const double a = r0[k];
    double x0[MC];
#pragma unroll
    for (int m = 0; m < MC; ++m) x0[m] = fma(-a, uv[m], r0[jc[m]]);
    if (dense) {
      // lane 0, group 0 holds the new diagonal (column k+1)
      const double inv = __drcp_rn(__shfl_sync(FULL, x0[0], 0));
      if (lane == 0) invd[k + 1] = inv;
#pragma unroll
      for (int m = 0; m < MC; ++m)
        if (lane + 32 * m < nu) r0[jc[m]] = jc[m] > k + 1 ? x0[m] * inv : x0[m];
    } else {
#pragma unroll
      for (int m = 0; m < MC; ++m)
        if (lane + 32 * m < nu) r0[jc[m]] = x0[m];
      __syncwarp();
      prep_pivot(P, M, invd, k + 1, lane);
    }
    return;
  }
  const int first = next_in_l ? l0 + 1 : l0;
  const int nw = next_in_l ? NW - 1 : NW;
  const int wi = next_in_l ? w - 1 : w;
  for (int e = first + wi; e < l1; e += 2 * nw) {
    const bool two = e + nw < l1;
    double* r0 = M + lrow(P, dense, k, e) * ld;
    double* r1 = two ? M + lrow(P, dense, k, e + nw) * ld : r0;
    update_rows<MC>(r0, r1, two, k, jc, uv, nu, lane);
  }
}

// Dense range, R pivots per barrier (R = 1 or 2): U rows k .. k+R-1 are final
// on entry; every later row i takes their updates, all columns j >= k+R. For
// R = 2 the L entry of column k+1 is formed first, b = M[i][k+1] - M[i][k]
// U[k][k+1], then each element takes -M[i][k] U[k][j] and -b U[k+1][j] in
// that order: the operations, and so the roundings, of two single-pivot
// steps. Warp 0 takes rows p = k+R and p+1 and finishes both as U rows
// (reciprocal pivot, pivot p applied to row p+1 from registers, scaling), so
// that the next step finds them final; the other warps take the rows from
// p+2 on, two at a time.
#ifndef CBX_DENSE_PAIRS
#define CBX_DENSE_PAIRS 1
#endif

template <int MC, int R>
__device__ __forceinline__ void dense_rank_rows(double* M, double* invd, int S, int k) {
  const int ld = lead_dim(S);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int c0 = k + R, nu = S - c0;  // columns c0 .. S-1, lane + 32 m
  double u0[MC], u1[MC];
#pragma unroll
  for (int m = 0; m < MC; ++m) {
    const bool in = lane + 32 * m < nu;
    u0[m] = in ? M[k * ld + c0 + lane + 32 * m] : 0.0;
    u1[m] = R == 2 && in ? M[(k + 1) * ld + c0 + lane + 32 * m] : 0.0;
  }
  const double u01 = R == 2 ? M[k * ld + k + 1] : 0.0;  // U(k, k+1)
  // one row's update into x; returns its L entry of column k+1 (R = 2)
  auto row_update = [&](const double* r, double (&x)[MC]) {
    const double a = r[k];
    const double b = R == 2 ? fma(-a, u01, r[k + 1]) : 0.0;
#pragma unroll
    for (int m = 0; m < MC; ++m) x[m] = lane + 32 * m < nu ? r[c0 + lane + 32 * m] : 0.0;
#pragma unroll
    for (int m = 0; m < MC; ++m) x[m] = fma(-a, u0[m], x[m]);
    if (R == 2) {
#pragma unroll
      for (int m = 0; m < MC; ++m) x[m] = fma(-b, u1[m], x[m]);
    }
    return b;
  };
  if (w == 0) {
    const int p = c0;
    double* rp = M + p * ld;
    double up[MC];  // row p: the diagonal at e = 0, U(p, :) after it
    const double bp = row_update(rp, up);
    const double inv_p = __drcp_rn(__shfl_sync(FULL, up[0], 0));  // column p: lane 0, group 0
#pragma unroll
    for (int m = 0; m < MC; ++m)
      if (lane + 32 * m >= 1) up[m] *= inv_p;
    if (lane == 0) {
      invd[p] = inv_p;
      if (R == 2) rp[k + 1] = bp;
    }
#pragma unroll
    for (int m = 0; m < MC; ++m)
      if (lane + 32 * m < nu) rp[c0 + lane + 32 * m] = up[m];
    if (p + 1 < S) {
      double* rq = rp + ld;
      double xq[MC];
      const double bq = row_update(rq, xq);
      const double ap = __shfl_sync(FULL, xq[0], 0);  // L(p+1, p), stays
#pragma unroll
      for (int m = 0; m < MC; ++m)
        if (lane + 32 * m >= 1) xq[m] = fma(-ap, up[m], xq[m]);
      const double inv_q = __drcp_rn(__shfl_sync(FULL, xq[0], 1));  // column p+1: lane 1, group 0
      if (lane == 0) {
        invd[p + 1] = inv_q;
        if (R == 2) rq[k + 1] = bq;
      }
#pragma unroll
      for (int m = 0; m < MC; ++m) {
        const int e = lane + 32 * m;
        if (e < nu) rq[c0 + e] = e <= 1 ? xq[m] : xq[m] * inv_q;
      }
    }
    return;
  }
  const int first = c0 + 2, nrow = S - first, nw = NW - 1;
  for (int e = w - 1; e < nrow; e += 2 * nw) {
    const bool two = e + nw < nrow;
    double* r0 = M + (first + e) * ld;
    double* r1 = two ? r0 + nw * ld : r0;
    double x0[MC], x1[MC];
    const double b0 = row_update(r0, x0);
    double b1 = 0.0;
    if (two) b1 = row_update(r1, x1);
    if (R == 2 && lane == 0) {
      r0[k + 1] = b0;
      if (two) r1[k + 1] = b1;
    }
#pragma unroll
    for (int m = 0; m < MC; ++m) {
      if (lane + 32 * m < nu) {
        r0[c0 + lane + 32 * m] = x0[m];
        if (two) r1[c0 + lane + 32 * m] = x1[m];
      }
    }
  }
}

// at most DENSE_PAIR_COLS columns (4 groups per lane): the step's register
// footprint stays within the kernel's budget
constexpr int DENSE_PAIR_COLS = 128;

template <int R>
__device__ __forceinline__ void dense_rank_step(double* M, double* invd, int S, int k) {
  switch ((S - k - R + 31) >> 5) {
    case 1: dense_rank_rows<1, R>(M, invd, S, k); break;
    case 2: dense_rank_rows<2, R>(M, invd, S, k); break;
    case 3: dense_rank_rows<3, R>(M, invd, S, k); break;
    default: dense_rank_rows<4, R>(M, invd, S, k); break;
  }
}

__device__ void lu_crout64(const PivLists& P, double* M, double* invd) {
  const int S = P.S, ld = lead_dim(S), kd = P.kd;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (w == 0) prep_pivot(P, M, invd, 0, lane);
  __syncthreads();
  // with pairs, the single-pivot loop stops at kp: the first dense pivot
  // with at most DENSE_PAIR_COLS columns after it
  const int kp = max(kd, S - 1 - DENSE_PAIR_COLS);
  const bool pairs = CBX_DENSE_PAIRS && S - kp >= 3;
  const int k_single = pairs ? kp : S - 1;
  for (int k = 0; k < k_single; ++k) {
    const bool dense = k >= kd;
    int l0, l1, u0, nu;
    if (dense) {
      l0 = 0;
      l1 = S - k - 1;
      u0 = 0;
      nu = S - k - 1;
    } else {
      l0 = P.lptr[k];
      l1 = P.lptr[k + 1];
      u0 = P.uptr[k];
      nu = P.uptr[k + 1] - u0;
    }
    const bool next_in_l = l1 > l0 && lrow(P, dense, k, l0) == k + 1;
    if (w == 0 && !next_in_l) prep_pivot(P, M, invd, k + 1, lane);
    if (nu > 0) {
      switch ((nu + 31) >> 5) {
        case 1: crout_rows<1>(P, M, invd, k, dense, l0, l1, u0, nu, next_in_l); break;
        case 2: crout_rows<2>(P, M, invd, k, dense, l0, l1, u0, nu, next_in_l); break;
        case 3: crout_rows<3>(P, M, invd, k, dense, l0, l1, u0, nu, next_in_l); break;
        case 4: crout_rows<4>(P, M, invd, k, dense, l0, l1, u0, nu, next_in_l); break;
        case 5: crout_rows<5>(P, M, invd, k, dense, l0, l1, u0, nu, next_in_l); break;
        case 6: crout_rows<6>(P, M, invd, k, dense, l0, l1, u0, nu, next_in_l); break;
        case 7: crout_rows<7>(P, M, invd, k, dense, l0, l1, u0, nu, next_in_l); break;
        default: crout_rows<8>(P, M, invd, k, dense, l0, l1, u0, nu, next_in_l); break;
      }
    } else if (w == 0 && next_in_l) {
      prep_pivot(P, M, invd, k + 1, lane);
    }
    __syncthreads();
  }
  if (pairs) {
    // U row kp is final; pivot kp alone brings rows kp+1 and kp+2 to final,
    // then pivots go in pairs while rows remain below them
    dense_rank_step<1>(M, invd, S, kp);
    __syncthreads();
    for (int k = kp + 1; k + 2 < S; k += 2) {
      dense_rank_step<2>(M, invd, S, k);
      __syncthreads();
    }
  }
  // L(:,k) /= pivot_k: M now holds L (unit lower), the pivots in invd (as
  // reciprocals) and U (unit upper), so both triangular solves are unit.
  for (int i = 1 + (threadIdx.x >> 5); i < S; i += NW)
    for (int k = lane; k < i; k += 32) M[i * ld + k] *= invd[k];
  __syncthreads();
}

// Triangular solves with the Crout factors, blocks of 32 with look-ahead.
// Warp w runs on the SM sub-partition w % 4, and one warp issues at most one
// FP64 instruction per ~67 cycles, so the 32-step chain of a diagonal block
// (warp 0, shuffles) alone leaves most of the SM's FP64 pipe idle. While warp
// 0 solves block b, the warps on the other three sub-partitions apply the
// previous block to the rows beyond the next block (one thread per row, four
// partial sums); after the barrier, warps 0..3 (one per sub-partition,
// LA_COLS columns each) apply block b to the next block's rows alone, into
// partial sums `part` [4][32] that warp 0 takes when it starts that block's
// chain. Two barriers per block, as without look-ahead; the critical path per
// block is the chain plus an eighth of the next block's update.
constexpr int LA_COLS = 8;

// bulk-update worker index of warp w (0..5 for the warps not on warp 0's
// sub-partition), or -1
__device__ __forceinline__ int la_worker(int w) { return (w & 3) == 0 ? -1 : (w >> 2) * 3 + (w & 3) - 1; }
constexpr int LA_WORKERS = (NW / 4) * 3;

// v[i] -= sum_{c < nc} row_i[c] y[c] for rows i in [i0, i1), one thread per
// row of this worker
__device__ __forceinline__ void la_bulk(const double* M, int ld, const double* y, int c0, int nc, double* v, int i0,
                                        int i1, int wk, int lane) {
  for (int i = i0 + 32 * wk + lane; i < i1; i += 32 * LA_WORKERS) {
    const double* row = M + i * ld + c0;
    double p0 = v[i], p1 = 0.0, p2 = 0.0, p3 = 0.0;
    int c = 0;
    for (; c + 4 <= nc; c += 4) {
      p0 = fma(-row[c], y[c], p0);
      p1 = fma(-row[c + 1], y[c + 1], p1);
      p2 = fma(-row[c + 2], y[c + 2], p2);
      p3 = fma(-row[c + 3], y[c + 3], p3);
    }
    for (; c < nc; ++c) p0 = fma(-row[c], y[c], p0);
    v[i] = (p0 + p1) + (p2 + p3);
  }
}

// part[32 w + lane] = sum of row (r0 + lane)'s entries in columns
// c0 + LA_COLS w .. (below c0 + nc) times y; warps 0..3
__device__ __forceinline__ void la_next(const double* M, int ld, const double* v, int c0, int nc, int r0, int r1,
                                        double* part, int w, int lane) {
  const int i = r0 + lane, cw = LA_COLS * w;
  double p = 0.0, q = 0.0;
  if (i < r1) {
    const double* row = M + i * ld + c0 + cw;
    const double* y = v + c0 + cw;
#pragma unroll
    for (int c = 0; c < LA_COLS; c += 2) {
      if (cw + c < nc) p = fma(row[c], y[c], p);
      if (cw + c + 1 < nc) q = fma(row[c + 1], y[c + 1], q);
    }
  }
  part[32 * w + lane] = p + q;
}

// v <- D^{-1} L^{-1} v (L unit lower, D the pivots with reciprocals in invd);
// D^{-1} last, element-wise. part: 128 doubles of shared scratch.
__device__ void forward_crout64(const double* M, const double* invd, int S, double* v, double* part) {
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, ld = lead_dim(S);
  const int nblk = (S + 31) / 32, wk = la_worker(w);
  for (int b = 0; b < nblk; ++b) {
    const int kb = 32 * b, nb = min(32, S - kb);
    if (w == 0) {
      double val = 0.0;
      if (lane < nb) {
        val = v[kb + lane];
        if (b > 0) val -= (part[lane] + part[32 + lane]) + (part[64 + lane] + part[96 + lane]);
      }
      const double* row = M + (kb + min(lane, nb - 1)) * ld + kb;
#pragma unroll
      for (int c = 0; c < 32; ++c) {
        if (c < nb) {
          const double yc = __shfl_sync(FULL, val, c);
          if (lane > c && lane < nb) val = fma(-row[c], yc, val);
        }
      }
      if (lane < nb) v[kb + lane] = val;
    } else if (wk >= 0 && b > 0) {
      // block b-1 (full) on the rows below block b (block b took it through
      // the partial sums)
      la_bulk(M, ld, v + kb - 32, kb - 32, 32, v, kb + 32, S, wk, lane);
    }
    __syncthreads();
    if (b + 1 < nblk && w < 4) la_next(M, ld, v, kb, 32, kb + 32, S, part, w, lane);
    __syncthreads();
  }
  for (int i = threadIdx.x; i < S; i += NT) v[i] *= invd[i];
  __syncthreads();
}

// v <- U^{-1} v for the unit upper Crout factor, blocks of 32 from the bottom
// (the bottom block may be partial; the others are full).
__device__ void backward_crout64(const double* M, int S, double* v, double* part) {
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, ld = lead_dim(S);
  const int nblk = (S + 31) / 32, wk = la_worker(w);
  for (int b = nblk - 1; b >= 0; --b) {
    const int kb = 32 * b, nb = min(32, S - kb);
    if (w == 0) {
      double val = 0.0;
      if (lane < nb) {
        val = v[kb + lane];
        if (b + 1 < nblk) val -= (part[lane] + part[32 + lane]) + (part[64 + lane] + part[96 + lane]);
      }
      const double* row = M + (kb + min(lane, nb - 1)) * ld + kb;
#pragma unroll
      for (int c = 31; c >= 0; --c) {
        if (c < nb) {
          const double xc = __shfl_sync(FULL, val, c);
          if (lane < c) val = fma(-row[c], xc, val);
        }
      }
      if (lane < nb) v[kb + lane] = val;
    } else if (wk >= 0 && b + 1 < nblk && b > 0) {
      // block b+1 (possibly the partial bottom block) on the rows above block b
      // (block b took it through the partial sums)
      const int kn = kb + 32;
      la_bulk(M, ld, v + kn, kn, min(32, S - kn), v, 0, kb, wk, lane);
    }
    __syncthreads();
    if (b > 0 && w < 4) la_next(M, ld, v, kb, nb, kb - 32, kb, part, w, lane);
    __syncthreads();
  }
}

// ---------------------------------------------------------------- blocked LU (FP32 path)

constexpr int NB = 32;  // panel width

#ifndef CBX_TC_LU
#define CBX_TC_LU 1  // FP32 trailing updates of large networks on the tensor cores (mma.sync TF32, split form)
#endif

// Right-looking blocked LU without pivoting, panel width NB, on a dense
// row-major matrix (leading dimension ld). Per panel: (1) the panel columns are
// factored with one barrier per column, each thread keeping one row of the
// panel in registers (the column loop is unrolled at compile time, so register
// indices and bounds are static); (2) thread-per-column forward substitution
// forms U12 = L11^{-1} A12 in registers and, on NB appended identity columns,
// L11^{-1}, which then replaces L11 in place for the block forward solves;
// (3) register-tiled update A22 -= L21 U12. After the last panel the upper
// diagonal blocks are replaced by U_bb^{-1} (strict upper part; the diagonal
// reciprocals stay in invd).

__device__ __forceinline__ float recip(float x) { return __frcp_rn(x); }
__device__ __forceinline__ double recip(double x) { return 1.0 / x; }

template <typename LT, bool FULL, int RPT>
__device__ __forceinline__ void panel_factor(LT* M, LT* invd, int S, int ld, int kb, int nb) {
  const int tid = threadIdx.x;
  LT r[RPT][NB];
#pragma unroll
  for (int p = 0; p < RPT; ++p) {
    const int i = kb + tid + NT * p;
#pragma unroll
    for (int jj = 0; jj < NB; ++jj) r[p][jj] = i < S && (FULL || jj < nb) ? M[i * ld + kb + jj] : LT(0);
  }
#pragma unroll
  for (int c = 0; c < NB; ++c) {
    if (FULL || c < nb) {
      const int k = kb + c;
      if (tid == k - kb) {  // the pivot row is row kb + c, owned by thread c (p = 0)
#pragma unroll
        for (int jj = c; jj < NB; ++jj)
          if (FULL || jj < nb) M[k * ld + kb + jj] = r[0][jj];
      }
      __syncthreads();
      const LT* prow = M + k * ld + kb;
      const LT inv = recip(prow[c]);
#pragma unroll
      for (int p = 0; p < RPT; ++p) {
        const int i = kb + tid + NT * p;
        if (i < S && i > k) {
          const LT l = r[p][c] * inv;
          r[p][c] = l;
#pragma unroll
          for (int jj = c + 1; jj < NB; ++jj)
            if (FULL || jj < nb) r[p][jj] -= l * prow[jj];
        }
      }
      if (tid == 0) invd[k] = inv;
    }
  }
  __syncthreads();
#pragma unroll
  for (int p = 0; p < RPT; ++p) {
    const int i = kb + tid + NT * p;
    if (i >= S) continue;
    if (i >= kb + nb) {
#pragma unroll
      for (int jj = 0; jj < NB; ++jj)
        if (FULL || jj < nb) M[i * ld + kb + jj] = r[p][jj];
    } else {
      // rows of the diagonal block: only their L part (columns < own row) is new
#pragma unroll
      for (int jj = 0; jj < NB; ++jj)
        if (kb + jj < i) M[i * ld + kb + jj] = r[p][jj];
    }
  }
  __syncthreads();
}

// Forward substitution of one column (NB values in registers) with the unit
// lower L11 of the panel.
template <typename LT, bool FULL>
__device__ __forceinline__ void l11_solve(const LT* L, int ld, int nb, LT (&v)[NB]) {
#pragma unroll
  for (int c = 0; c < NB - 1; ++c) {
#pragma unroll
    for (int r = c + 1; r < NB; ++r)
      if (FULL || r < nb) v[r] -= L[r * ld + c] * v[c];
  }
}

template <typename LT, bool FULL>
__device__ __forceinline__ void panel_u12(LT* M, int S, int ld, int kb, int nb) {
  const int ke = kb + nb, ncol = S - ke;
  const LT* L = M + kb * ld + kb;
  if (ncol + nb <= NT) {
    // one pass: threads < ncol take A12 columns, the next nb the identity
    // columns; L11^{-1} is written over L11 after everyone has read it
    const int t = threadIdx.x;
    const bool a12 = t < ncol, ident = !a12 && t < ncol + nb;
    const int col = ke + t, jj = t - ncol;
    LT v[NB];
#pragma unroll
    for (int r = 0; r < NB; ++r)
      v[r] = a12 && (FULL || r < nb) ? M[(kb + r) * ld + col] : (ident && r == jj ? LT(1) : LT(0));
    if (a12 || ident) l11_solve<LT, FULL>(L, ld, nb, v);
    __syncthreads();
    if (a12) {
#pragma unroll
      for (int r = 0; r < NB; ++r)
        if (FULL || r < nb) M[(kb + r) * ld + col] = v[r];
    } else if (ident) {
#pragma unroll
      for (int r = 0; r < NB; ++r)
        if (r > jj && (FULL || r < nb)) M[(kb + r) * ld + kb + jj] = v[r];
    }
    __syncthreads();
    return;
  }
  // U12 = L11^{-1} A12, one column per thread (A12 does not overlap L11)
  for (int t = threadIdx.x; t < ncol; t += NT) {
    const int col = ke + t;
    LT v[NB];
#pragma unroll
    for (int r = 0; r < NB; ++r) v[r] = FULL || r < nb ? M[(kb + r) * ld + col] : LT(0);
    l11_solve<LT, FULL>(L, ld, nb, v);
#pragma unroll
    for (int r = 0; r < NB; ++r)
      if (FULL || r < nb) M[(kb + r) * ld + col] = v[r];
  }
  // L11^{-1}: identity columns, written over L11 after everyone has read it
  const int jj = threadIdx.x;
  LT v[NB];
#pragma unroll
  for (int r = 0; r < NB; ++r) v[r] = r == jj ? LT(1) : LT(0);
  if (jj < nb) l11_solve<LT, FULL>(L, ld, nb, v);
  __syncthreads();
  if (jj < nb) {
#pragma unroll
    for (int r = 0; r < NB; ++r)
      if (r > jj && (FULL || r < nb)) M[(kb + r) * ld + kb + jj] = v[r];
  }
  __syncthreads();
}

// A22 -= L21 U12 over rows/cols [ke, S): warps take TR-row strips, lanes the
// columns ke + lane + 32 g (exactly NG groups); the inner dimension is nb.
template <typename LT, int NG, int TR>
__device__ __forceinline__ void trailing_update_ng(LT* M, int S, int ld, int kb, int nb) {
  const int ke = kb + nb, ncol = S - ke;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  bool colok[NG];
#pragma unroll
  for (int g = 0; g < NG; ++g) colok[g] = lane + 32 * g < ncol;
  for (int rs = warp; rs * TR < ncol; rs += NW) {
    const int i0 = ke + rs * TR;
    LT acc[TR][NG];
#pragma unroll
    for (int r = 0; r < TR; ++r)
#pragma unroll
      for (int g = 0; g < NG; ++g) acc[r][g] = LT(0);
    const LT* lp[TR];
#pragma unroll
    for (int r = 0; r < TR; ++r) lp[r] = M + min(i0 + r, S - 1) * ld + kb;
    const LT* up = M + kb * ld + ke + lane;
    for (int c = 0; c < nb; ++c) {
      LT lv[TR], uu[NG];
#pragma unroll
      for (int r = 0; r < TR; ++r) lv[r] = lp[r][c];
#pragma unroll
      for (int g = 0; g < NG; ++g) uu[g] = colok[g] ? up[32 * g] : LT(0);
#pragma unroll
      for (int g = 0; g < NG; ++g)
#pragma unroll
        for (int r = 0; r < TR; ++r) acc[r][g] += lv[r] * uu[g];
      up += ld;
    }
#pragma unroll
    for (int r = 0; r < TR; ++r) {
      if (i0 + r < S) {
        LT* row = M + (i0 + r) * ld + ke + lane;
#pragma unroll
        for (int g = 0; g < NG; ++g)
          if (colok[g]) row[32 * g] -= acc[r][g];
      }
    }
  }
}

// ---- tensor-core form of the FP32 trailing update (mixed path)
//
// A22 -= L21 U12 is a dense contraction with K = nb <= 32: it runs on the
// tensor cores as warp-level mma.sync m16n8k8 with TF32 operands, in the
// split form a b ~ a_hi b_hi + a_hi b_lo + a_lo b_hi (x_hi = tf32(x),
// x_lo = tf32(x - x_hi)), which keeps the products at FP32 accuracy (the
// dropped a_lo b_lo is ~2^-22 relative), so the factor is as good as the
// FP32 FMA form and the FP64 refinement needs no more sweeps. Each warp
// takes blocks of 16 rows x 8 TN columns; the A22 tile is the accumulator's
// start value and -L21 the A operand, so D = A22 - L21 U12 directly.
// Fragment layouts of m16n8k8 (g = lane / 4, q = lane % 4):
//   A (16 x 8): a0 (g, q), a1 (g + 8, q), a2 (g, q + 4), a3 (g + 8, q + 4)
//   B (8 x 8):  b0 (q, g), b1 (q + 4, g)
//   C (16 x 8): c0 (g, 2q), c1 (g, 2q + 1), c2 (g + 8, 2q), c3 (g + 8, 2q + 1)

__device__ __forceinline__ unsigned to_tf32(float x) {
  unsigned r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ void split_tf32(float x, unsigned& hi, unsigned& lo) {
  hi = to_tf32(x);
  lo = to_tf32(x - __uint_as_float(hi));
}

__device__ __forceinline__ void mma_tf32(float (&d)[4], const unsigned (&a)[4], unsigned b0, unsigned b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
      "{%0, %1, %2, %3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// A[r][c] -= sum_{k0 <= k < k0 + K} A[r][k] A[k][c] for r in [r0, r1), c in
// [c0, c1) (the L columns and U rows of the K panels, in place), K taken in
// chunks of 32 with the accumulator tiles kept in registers across chunks, so
// that every element of the rectangle is read and written once.
template <int TN>
__device__ __forceinline__ void tc_rect(float* M, int ld, int k0, int K, int r0, int r1, int c0, int c1) {
  const int m = r1 - r0, n = c1 - c0;
  if (m <= 0 || n <= 0) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, q = lane & 3;
  const int nbr = (m + 15) / 16, nbc = (n + 8 * TN - 1) / (8 * TN);
  for (int blk = warp; blk < nbr * nbc; blk += NW) {
    const int rt = r0 + (blk / nbc) * 16, ct = c0 + (blk % nbc) * 8 * TN;
    const int ra = rt + g, rb = rt + g + 8;
    const bool oka = ra < r1, okb = rb < r1;
    float d[TN][4];
#pragma unroll
    for (int t = 0; t < TN; ++t) {
      const int cc = ct + 8 * t + 2 * q;
      d[t][0] = oka && cc < c1 ? M[ra * ld + cc] : 0.0f;
      d[t][1] = oka && cc + 1 < c1 ? M[ra * ld + cc + 1] : 0.0f;
      d[t][2] = okb && cc < c1 ? M[rb * ld + cc] : 0.0f;
      d[t][3] = okb && cc + 1 < c1 ? M[rb * ld + cc + 1] : 0.0f;
    }
    for (int kc = 0; kc < K; kc += 32) {
      const int kn = min(32, K - kc), kk = k0 + kc;
      // -L rows ra, rb (columns kk .. kk + kn - 1), split into hi and lo
      unsigned ah[4][4], al[4][4];
#pragma unroll
      for (int ks = 0; ks < 4; ++ks) {
        const int e0 = 8 * ks + q, e1 = e0 + 4;
        split_tf32(oka && e0 < kn ? -M[ra * ld + kk + e0] : 0.0f, ah[ks][0], al[ks][0]);
        split_tf32(okb && e0 < kn ? -M[rb * ld + kk + e0] : 0.0f, ah[ks][1], al[ks][1]);
        split_tf32(oka && e1 < kn ? -M[ra * ld + kk + e1] : 0.0f, ah[ks][2], al[ks][2]);
        split_tf32(okb && e1 < kn ? -M[rb * ld + kk + e1] : 0.0f, ah[ks][3], al[ks][3]);
      }
#pragma unroll
      for (int t = 0; t < TN; ++t) {
        const int cg = ct + 8 * t + g;  // B operand column
#pragma unroll
        for (int ks = 0; ks < 4; ++ks) {
          if (8 * ks >= kn) break;
          const int e0 = 8 * ks + q, e1 = e0 + 4;
          unsigned bh0, bl0, bh1, bl1;
          split_tf32(cg < c1 && e0 < kn ? M[(kk + e0) * ld + cg] : 0.0f, bh0, bl0);
          split_tf32(cg < c1 && e1 < kn ? M[(kk + e1) * ld + cg] : 0.0f, bh1, bl1);
          mma_tf32(d[t], al[ks], bh0, bh1);
          mma_tf32(d[t], ah[ks], bl0, bl1);
          mma_tf32(d[t], ah[ks], bh0, bh1);
        }
      }
    }
#pragma unroll
    for (int t = 0; t < TN; ++t) {
      const int cc = ct + 8 * t + 2 * q;
      if (oka && cc < c1) M[ra * ld + cc] = d[t][0];
      if (oka && cc + 1 < c1) M[ra * ld + cc + 1] = d[t][1];
      if (okb && cc < c1) M[rb * ld + cc] = d[t][2];
      if (okb && cc + 1 < c1) M[rb * ld + cc + 1] = d[t][3];
    }
  }
}

template <typename LT, bool LARGE>
__device__ __forceinline__ void trailing_update(LT* M, int S, int ld, int kb, int nb) {
  const int ncol = S - kb - nb;
  if (ncol <= 0) return;
#if CBX_TC_LU
  // tensor cores where they pay: the global-memory matrices of large networks
  // (at 150 species, trailing blocks of <= 118 rows in shared memory, the FMA
  // form below measured 2.5 % faster over a whole solve)
  if constexpr (sizeof(LT) == 4 && LARGE) {
    tc_rect<4>((float*)M, ld, kb, nb, kb + nb, S, kb + nb, S);
    __syncthreads();
    return;
  }
#endif
  if (!LARGE) {
    switch ((ncol + 31) >> 5) {
      case 1: trailing_update_ng<LT, 1, 4>(M, S, ld, kb, nb); break;
      case 2: trailing_update_ng<LT, 2, 4>(M, S, ld, kb, nb); break;
      case 3: trailing_update_ng<LT, 3, 4>(M, S, ld, kb, nb); break;
      case 4: trailing_update_ng<LT, 4, 4>(M, S, ld, kb, nb); break;
      case 5: trailing_update_ng<LT, 5, 4>(M, S, ld, kb, nb); break;
      case 6: trailing_update_ng<LT, 6, 4>(M, S, ld, kb, nb); break;
      case 7: trailing_update_ng<LT, 7, 4>(M, S, ld, kb, nb); break;
      default: trailing_update_ng<LT, 8, 4>(M, S, ld, kb, nb); break;
    }
    __syncthreads();
    return;
  }
  switch ((ncol + 31) >> 5) {
    case 1: trailing_update_ng<LT, 1, 4>(M, S, ld, kb, nb); break;
    case 2: trailing_update_ng<LT, 2, 4>(M, S, ld, kb, nb); break;
    case 3: trailing_update_ng<LT, 3, 4>(M, S, ld, kb, nb); break;
    case 4: trailing_update_ng<LT, 4, 4>(M, S, ld, kb, nb); break;
    case 5: trailing_update_ng<LT, 5, 4>(M, S, ld, kb, nb); break;
    case 6: trailing_update_ng<LT, 6, 4>(M, S, ld, kb, nb); break;
    case 7: trailing_update_ng<LT, 7, 4>(M, S, ld, kb, nb); break;
    case 8: trailing_update_ng<LT, 8, 4>(M, S, ld, kb, nb); break;
    case 9: trailing_update_ng<LT, 9, 2>(M, S, ld, kb, nb); break;
    case 10: trailing_update_ng<LT, 10, 2>(M, S, ld, kb, nb); break;
    case 11: trailing_update_ng<LT, 11, 2>(M, S, ld, kb, nb); break;
    case 12: trailing_update_ng<LT, 12, 2>(M, S, ld, kb, nb); break;
    case 13: trailing_update_ng<LT, 13, 2>(M, S, ld, kb, nb); break;
    case 14: trailing_update_ng<LT, 14, 2>(M, S, ld, kb, nb); break;
    case 15: trailing_update_ng<LT, 15, 2>(M, S, ld, kb, nb); break;
    default: trailing_update_ng<LT, 16, 2>(M, S, ld, kb, nb); break;
  }
  __syncthreads();
}

// U_bb^{-1} of every diagonal block, in place (strict upper part; the
// diagonal reciprocals stay in invd). FP32 form: one warp per block, lane j
// solves U_bb x = e_j by back substitution in registers (the block's entries
// are broadcast loads), and the warp overwrites the block once all its lanes
// have read it.
template <typename LT, bool FULL>
__device__ __forceinline__ void invert_upper_block(LT* U, const LT* invd, int ld, int nb, int lane) {
  LT x[NB];
#pragma unroll
  for (int r = NB - 1; r >= 0; --r) {
    x[r] = LT(0);
    if (FULL || r < nb) {
      LT acc = r == lane ? LT(1) : LT(0);
#pragma unroll
      for (int c = r + 1; c < NB; ++c)
        if (FULL || c < nb) acc -= U[r * ld + c] * x[c];
      x[r] = acc * invd[r];
    }
  }
  __syncwarp();
  if (lane < nb) {
#pragma unroll
    for (int r = 0; r < NB - 1; ++r)
      if (r < lane) U[r * ld + lane] = x[r];
  }
}

// FP64 form (fewer registers than a column of NB doubles per lane): one warp
// per block, columns left to right, X[0:j, j] = -X[0:j, 0:j] U[0:j, j] / U_jj with X[0:j, 0:j] (already
// in place) and the still-original column j; lanes take the rows r < j.
template <typename LT>
__device__ void invert_upper_blocks_cols(LT* M, const LT* invd, int S, int ld) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nblk = (S + NB - 1) / NB;
  for (int b = warp; b < nblk; b += NW) {
    const int kb = b * NB, nb = min(NB, S - kb);
    LT* U = M + kb * ld + kb;
    for (int j = 1; j < nb; ++j) {
      LT acc = LT(0);
      if (lane < j) {
        LT a0 = invd[kb + lane] * U[lane * ld + j], a1 = LT(0), a2 = LT(0), a3 = LT(0);
        int c = lane + 1;
        for (; c + 4 <= j; c += 4) {
          a0 += U[lane * ld + c] * U[c * ld + j];
          a1 += U[lane * ld + c + 1] * U[(c + 1) * ld + j];
          a2 += U[lane * ld + c + 2] * U[(c + 2) * ld + j];
          a3 += U[lane * ld + c + 3] * U[(c + 3) * ld + j];
        }
        for (; c < j; ++c) a0 += U[lane * ld + c] * U[c * ld + j];
        acc = (a0 + a1) + (a2 + a3);
      }
      __syncwarp();
      if (lane < j) U[lane * ld + j] = -invd[kb + j] * acc;
      __syncwarp();
    }
  }
  __syncthreads();
}

template <typename LT>
__device__ void invert_upper_blocks(LT* M, const LT* invd, int S, int ld) {
  if constexpr (sizeof(LT) == 8) {
    invert_upper_blocks_cols<LT>(M, invd, S, ld);
    return;
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nblk = (S + NB - 1) / NB;
  for (int b = warp; b < nblk; b += NW) {
    const int kb = b * NB, nb = min(NB, S - kb);
    if (nb == NB) invert_upper_block<LT, true>(M + kb * ld + kb, invd + kb, ld, nb, lane);
    else invert_upper_block<LT, false>(M + kb * ld + kb, invd + kb, ld, nb, lane);
  }
  __syncthreads();
}

// A22 -= L21 U12 for one of the leading panels [kb, kb+NB) of a network whose
// first pivots are sparse: one thread per trailing row i; for each pivot k of
// the panel with L(i,k) != 0, the columns j >= kb+NB of U(k,:) from the
// pivot's structural list (ascending). Rows are disjoint, so no two threads
// write one element. Entries outside the pattern hold exact zeros, so the
// skipped terms are exact zeros.
template <typename LT>
__device__ void sparse_panel_update(LT* M, int S, int ld, int kb, const int* uptr, const int* ucol) {
  const int ke = kb + NB;
  for (int i = ke + threadIdx.x; i < S; i += NT) {
    LT* row = M + (size_t)i * ld;
    for (int c = 0; c < NB; ++c) {
      const LT l = row[kb + c];
      if (l == LT(0)) continue;
      const int k = kb + c;
      const LT* urow = M + (size_t)k * ld;
      const int e1 = uptr[k + 1];
      int e = uptr[k];
      while (e < e1 && ucol[e] < ke) ++e;  // columns inside the panel
      for (; e + 4 <= e1; e += 4) {
        const int j0 = ucol[e], j1 = ucol[e + 1], j2 = ucol[e + 2], j3 = ucol[e + 3];
        const LT u0 = urow[j0], u1 = urow[j1], u2 = urow[j2], u3 = urow[j3];
        const LT a0 = row[j0], a1 = row[j1], a2 = row[j2], a3 = row[j3];
        row[j0] = a0 - l * u0;
        row[j1] = a1 - l * u1;
        row[j2] = a2 - l * u2;
        row[j3] = a3 - l * u3;
      }
      for (; e < e1; ++e) {
        const int j = ucol[e];
        row[j] -= l * urow[j];
      }
    }
  }
  __syncthreads();
}

// FP32, matrix in global memory: panels in pairs, so that the trailing matrix
// is read and written once per two panels (its passes are the DRAM traffic of
// the factorisation). For panels P1 = [kb, k2) and P2 = [k2, ke): factor P1
// and form its U rows over all later columns; update only what P2 needs - its
// columns (rows >= k2) and its U rows (columns >= ke) - from P1; factor P2 and
// form its U rows; then one update of the rows and columns >= ke with K = 64
// (both panels' L columns and U rows, contiguous in place). Not inlined: its
// own register allocation keeps the kernel body free of spills (inlined, the
// kernel spilled 1.7 KB).
#ifndef CBX_PAIR_PANELS
#define CBX_PAIR_PANELS 1
#endif

__device__ __forceinline__ void panel_factor_full_rows(float* M, float* invd, int S, int ld, int kb) {
  if (S - kb > NT) panel_factor<float, true, 2>(M, invd, S, ld, kb, NB);
  else panel_factor<float, true, 1>(M, invd, S, ld, kb, NB);
}

__device__ __noinline__ void lu_blocked_pairs(float* M, float* invd, int S, int ld) {
  int kb = 0;
  for (; kb + 2 * NB < S; kb += 2 * NB) {  // pairs with a trailing matrix after them
    const int k2 = kb + NB, ke = kb + 2 * NB;
    panel_factor_full_rows(M, invd, S, ld, kb);
    panel_u12<float, true>(M, S, ld, kb, NB);
    tc_rect<4>(M, ld, kb, NB, k2, S, k2, ke);   // P2's columns
    tc_rect<4>(M, ld, kb, NB, k2, ke, ke, S);   // P2's U rows (disjoint from the above)
    __syncthreads();
    panel_factor_full_rows(M, invd, S, ld, k2);
    panel_u12<float, true>(M, S, ld, k2, NB);
    tc_rect<4>(M, ld, kb, 2 * NB, ke, S, ke, S);
    __syncthreads();
  }
  for (; kb < S; kb += NB) {  // what is left: single panels
    const int nb = min(NB, S - kb);
    if (nb == NB) {
      panel_factor_full_rows(M, invd, S, ld, kb);
      panel_u12<float, true>(M, S, ld, kb, nb);
    } else {
      panel_factor<float, false, 1>(M, invd, S, ld, kb, nb);
      panel_u12<float, false>(M, S, ld, kb, nb);
    }
    tc_rect<4>(M, ld, kb, nb, kb + nb, S, kb + nb, S);
    __syncthreads();
  }
  invert_upper_blocks<float>(M, invd, S, ld);
}

// LARGE: networks of 257..512 species (matrix in global memory): two panel
// rows per thread and up to 16 column groups in the trailing update; in FP64
// the first nsp panels take their trailing update from the pivots' U lists
// (uptr, ucol). In FP32 the dense tensor-core update of those panels costs
// less than the listed one: 500 species mixed measured 626 cell-solves/s
// dense and 506 listed, FP64 194 dense and 220 listed.
template <typename LT, bool LARGE>
__device__ void lu_blocked(LT* M, LT* invd, int S, int ld, int nsp = 0, const int* uptr = nullptr,
                           const int* ucol = nullptr) {
#if CBX_PAIR_PANELS && CBX_TC_LU
  if constexpr (sizeof(LT) == 4 && LARGE) {
    lu_blocked_pairs((float*)M, (float*)invd, S, ld);
    return;
  }
#endif
  for (int kb = 0; kb < S; kb += NB) {
    const int nb = min(NB, S - kb);
    const bool two = LARGE && S - kb > NT;  // more panel rows than threads
    if (nb == NB) {
      if (two) panel_factor<LT, true, LARGE ? 2 : 1>(M, invd, S, ld, kb, nb);
      else panel_factor<LT, true, 1>(M, invd, S, ld, kb, nb);
      panel_u12<LT, true>(M, S, ld, kb, nb);
    } else {
      panel_factor<LT, false, 1>(M, invd, S, ld, kb, nb);
      panel_u12<LT, false>(M, S, ld, kb, nb);
    }
    if (LARGE && sizeof(LT) == 8 && kb < nsp * NB) sparse_panel_update<LT>(M, S, ld, kb, uptr, ucol);
    else trailing_update<LT, LARGE>(M, S, ld, kb, nb);
  }
  invert_upper_blocks<LT>(M, invd, S, ld);
}

template <typename LT, bool FULL>
__device__ __forceinline__ void rows_minus_block(const LT* M, int ld, const LT* vb, int nb, LT* v, int i0, int i1) {
  // v[i] -= sum_c M[i][c] vb[c] for rows i in [i0, i1); M points at column kb
  for (int i = i0 + threadIdx.x; i < i1; i += NT) {
    const LT* row = M + i * ld;
    LT p0 = v[i], p1 = LT(0), p2 = LT(0), p3 = LT(0);
#pragma unroll
    for (int c = 0; c < NB; c += 4) {
      if (FULL || c < nb) p0 -= row[c] * vb[c];
      if (FULL || c + 1 < nb) p1 -= row[c + 1] * vb[c + 1];
      if (FULL || c + 2 < nb) p2 -= row[c + 2] * vb[c + 2];
      if (FULL || c + 3 < nb) p3 -= row[c + 3] * vb[c + 3];
    }
    v[i] = (p0 + p1) + (p2 + p3);
  }
}

template <typename LT>
__device__ void solve_blocked(const LT* M, const LT* invd, int S, int ld, LT* v) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  for (int kb = 0; kb < S; kb += NB) {
    const int nb = min(NB, S - kb), ke = kb + nb;
    if (warp == 0) {
      LT acc = LT(0);
      const LT* row = M + (kb + min(lane, nb - 1)) * ld + kb;
      if (lane < nb) {
        acc = v[kb + lane];
#pragma unroll
        for (int c = 0; c < NB - 1; ++c)
          if (c < lane) acc += row[c] * v[kb + c];
      }
      __syncwarp();
      if (lane < nb) v[kb + lane] = acc;
    }
    __syncthreads();
    if (nb == NB)
      rows_minus_block<LT, true>(M + kb, ld, v + kb, nb, v, ke, S);
    else
      rows_minus_block<LT, false>(M + kb, ld, v + kb, nb, v, ke, S);
    __syncthreads();
  }
  for (int kb = ((S - 1) / NB) * NB; kb >= 0; kb -= NB) {
    const int nb = min(NB, S - kb);
    if (warp == 0) {
      LT acc = LT(0);
      const LT* row = M + (kb + min(lane, nb - 1)) * ld + kb;
      if (lane < nb) {
        acc = invd[kb + lane] * v[kb + lane];
#pragma unroll
        for (int c = 1; c < NB; ++c)
          if (c > lane && c < nb) acc += row[c] * v[kb + c];
      }
      __syncwarp();
      if (lane < nb) v[kb + lane] = acc;
    }
    __syncthreads();
    if (nb == NB)
      rows_minus_block<LT, true>(M + kb, ld, v + kb, nb, v, 0, kb);
    else
      rows_minus_block<LT, false>(M + kb, ld, v + kb, nb, v, 0, kb);
    __syncthreads();
  }
}

// ---------------------------------------------------------------- shared layout

struct Smem {
  void* M;
  void* invd;
  double *D, *y, *yp, *dv, *f, *wsc, *psi, *dy, *w, *tmp, *r, *part, *red, *Tm;
  float* v32;
  int* pstage;   // staged pivot lists (FP64 shared-memory solver), or none
  PivLists piv;  // the lists the LU reads
};

__host__ __device__ inline size_t align16(size_t b) { return (b + 15) & ~size_t(15); }

__host__ __device__ inline size_t layout(int S, int R, int nseg, bool mixed, bool gm, unsigned char* base, Smem* s,
                                         int piv_ints = 0) {
  const size_t lt = mixed ? sizeof(float) : sizeof(double);
  size_t off = 0;
  auto take = [&](size_t bytes) {
    unsigned char* p = base ? base + off : nullptr;
    off += align16(bytes);
    return p;
  };
  Smem t;
  t.M = take(gm ? 0 : (size_t)S * lead_dim(S) * lt);
  t.invd = take((size_t)S * lt);
  t.D = (double*)take((size_t)kDiffRows * S * 8);
  t.y = (double*)take(S * 8);
  t.yp = (double*)take(S * 8);
  t.dv = (double*)take(S * 8);
  t.f = (double*)take(S * 8);
  t.wsc = (double*)take(S * 8);
  t.psi = (double*)take(S * 8);
  t.dy = (double*)take(S * 8);
  t.w = (double*)take(S * 8);
  t.tmp = (double*)take(S * 8);
  t.r = (double*)take((size_t)R * 8);
  t.part = (double*)take((size_t)nseg * 8);
  t.red = (double*)take(128 * 8);  // block sums; the solves' look-ahead partials
  t.Tm = (double*)take(kMaxOrder * kMaxOrder * 8);
  t.v32 = (float*)take(mixed ? S * 4 : 0);
  t.pstage = (int*)take((size_t)piv_ints * 4);
  if (s) *s = t;
  return off;
}


// Copy the index lists of the sparse pivots (k < kd: pointers and entries)
// into shared memory once per CTA, so that the LU's per-pivot index loads
// are shared-memory loads rather than L2 round trips on its critical path.
__device__ void stage_pivots(const DevNet& n, Smem& s) {
  const int kd = n.kdense;
  const int nl = n.piv_lptr[kd], nu = n.piv_uptr[kd];
  int* lp = s.pstage;
  int* up = lp + (kd + 1);
  int* l = up + (kd + 1);
  int* u = l + nl;
  for (int i = threadIdx.x; i <= kd; i += NT) {
    lp[i] = n.piv_lptr[i];
    up[i] = n.piv_uptr[i];
  }
  for (int i = threadIdx.x; i < nl; i += NT) l[i] = n.piv_l[i];
  for (int i = threadIdx.x; i < nu; i += NT) u[i] = n.piv_u[i];
  __syncthreads();
  s.piv = PivLists{n.S, kd, lp, l, up, u};
}


// ---------------------------------------------------------------- BDF pieces

// T[k][j](rho) = sum_{i=0..k} (-1)^i C(k,i) C(-i rho + j - 1, j), with
// C(s + j - 1, j) = s (s+1) ... (s+j-1) / j!. Binomials and 1/j! come from
// constant tables: no FP64 division (each costs ~10 FP64 instructions, and
// this runs on one warp).
static __constant__ double c_inv_fact[kMaxOrder + 1] = {1.0, 1.0, 0.5, 1.0 / 6.0, 1.0 / 24.0, 1.0 / 120.0};
static __constant__ double c_binom[kMaxOrder + 1][kMaxOrder + 1] = {{1, 0, 0, 0, 0, 0}, {1, 1, 0, 0, 0, 0},
                                                             {1, 2, 1, 0, 0, 0}, {1, 3, 3, 1, 0, 0},
                                                             {1, 4, 6, 4, 1, 0}, {1, 5, 10, 10, 5, 1}};

__device__ __forceinline__ double rescale_entry(int k, int j, double rho) {
  double acc = 0.0;
  for (int i = 0; i <= k; ++i) {
    const double s = -i * rho;
    double p = 1.0;
    for (int m = 0; m < j; ++m) p *= s + m;
    acc = fma((i & 1) ? -c_binom[k][i] : c_binom[k][i], p, acc);
  }
  return acc * c_inv_fact[j];
}

// D[1..q] <- T(rho) D[1..q], T[k][j] = sum_i (-1)^i C(k,i) C(-i rho + j - 1, j):
// the differences of the interpolating polynomial on the new spacing. The
// q x q matrix is computed by one warp (lane = (k, j)).
__device__ void rescale(double* D, int S, int q, double rho, double* Tm) {
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    if (lane < q * q) {
      const int k = lane / q + 1, j = lane % q + 1;
      Tm[(k - 1) * kMaxOrder + (j - 1)] = rescale_entry(k, j, rho);
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < S; i += NT) {
    double old[kMaxOrder];
#pragma unroll
    for (int j = 0; j < kMaxOrder; ++j) old[j] = j < q ? D[(j + 1) * S + i] : 0.0;
    for (int k = 0; k < q; ++k) {
      double acc = 0.0;
#pragma unroll
      for (int j = 0; j < kMaxOrder; ++j)
        if (j < q) acc = fma(Tm[k * kMaxOrder + j], old[j], acc);
      D[(k + 1) * S + i] = acc;
    }
  }
  __syncthreads();
}

template <typename LT, bool GM>
struct Cell {
  static constexpr bool gm = GM;  // M in global memory (blocked LU and solves for both precisions)
  const SolveArgs& a;
  const DevNet& n;
  Smem& s;
  LT* M;     // Newton matrix: shared memory, or the CTA's global workspace
  double* kap;
  double* g;
  double* Jv;
  cbx_cell_stats* st;  // shared-memory counters, updated by thread 0 only
};

// Solve (I - cJ) dy = w with the factored matrix in shared memory.
template <bool GM>
__device__ void linear_solve(Cell<double, GM>& c, double cc, const double* w, double* dy) {
  const int S = c.n.S;
  for (int i = threadIdx.x; i < S; i += NT) dy[i] = w[i];
  __syncthreads();
  if constexpr (GM) {
    solve_blocked<double>(c.M, (const double*)c.s.invd, S, lead_dim(S), dy);
  } else {
    forward_crout64(c.M, (const double*)c.s.invd, S, dy, c.s.red);
    backward_crout64(c.M, S, dy, c.s.red);
  }
}

// FP32 LU solve, then FP64 residual w - (dy - c J dy) against the FP64
// Jacobian and FP32 correction solves until the weighted RMS of the
// correction is <= refine_tol or max_refine sweeps.
template <bool GM>
__device__ void linear_solve(Cell<float, GM>& c, double cc, const double* w, double* dy) {
  const int S = c.n.S;
  const float* M = c.M;
  const float* invd = (const float*)c.s.invd;
  float* v = c.s.v32;
  const int ld = lead_dim(S);
  for (int i = threadIdx.x; i < S; i += NT) v[i] = (float)w[i];
  __syncthreads();
  solve_blocked<float>(M, invd, S, ld, v);
  for (int i = threadIdx.x; i < S; i += NT) dy[i] = (double)v[i];
  __syncthreads();
  for (int sweep = 0; sweep < c.a.max_refine; ++sweep) {
    for (int i = threadIdx.x; i < S; i += NT) {
      double acc = 0.0;
      const int e1 = c.n.jrow_ptr[i + 1];
      for (int e = c.n.jrow_ptr[i]; e < e1; ++e) acc = fma(c.Jv[e], dy[c.n.jcol[e]], acc);
      const double res = w[i] - (dy[i] - cc * acc);
      v[i] = (float)res;
    }
    __syncthreads();
    solve_blocked<float>(M, invd, S, ld, v);
    double sq = 0.0;
    for (int i = threadIdx.x; i < S; i += NT) {
      const double corr = (double)v[i];
      dy[i] += corr;
      const double t = corr * c.s.wsc[i];
      sq = fma(t, t, sq);
    }
    if (threadIdx.x == 0) c.st->refine_sweeps++;
    const double nrm = sqrt(block_sum(sq, c.s.red) / S);
    if (!(nrm > c.a.refine_tol)) break;
  }
}

template <typename LT, bool GM>
__device__ void factor(Cell<LT, GM>& c, double cc) {
  build_matrix<LT>(c.n, c.Jv, cc, c.M);
  if constexpr (GM) {
    lu_blocked<LT, true>(c.M, (LT*)c.s.invd, c.n.S, lead_dim(c.n.S), c.n.sparse_panels, c.n.piv_uptr, c.n.piv_u);
  } else {
    if constexpr (sizeof(LT) == 4)
      lu_blocked<LT, false>(c.M, (LT*)c.s.invd, c.n.S, lead_dim(c.n.S));
    else
      lu_crout64(c.s.piv, c.M, (double*)c.s.invd);
  }
  if (threadIdx.x == 0) c.st->lu_factors++;
}

// Simplified Newton on d - c f(yp + d) + psi = 0. Leaves y = yp + d, dv = d.
template <typename LT, bool GM>
__device__ bool newton(Cell<LT, GM>& c, double cc, int* iters) {
  const int S = c.n.S;
  Smem& s = c.s;
  for (int i = threadIdx.x; i < S; i += NT) {
    s.y[i] = s.yp[i];
    s.dv[i] = 0.0;
  }
  __syncthreads();
  double dy_old = 0.0, rate = 0.0;
  bool conv = false;
  for (int k = 0; k < kNewtonMaxIter; ++k) {
    *iters = k + 1;
    rhs(c.n, c.kap, s.y, s.f, s.r, s.part);
    if (threadIdx.x == 0) c.st->rhs_evals++;
    int bad = 0;
    for (int i = threadIdx.x; i < S; i += NT) bad |= !isfinite(s.f[i]);
    if (__syncthreads_or(bad)) break;
    for (int i = threadIdx.x; i < S; i += NT) s.w[i] = cc * s.f[i] - s.psi[i] - s.dv[i];
    __syncthreads();
    linear_solve(c, cc, s.w, s.dy);
    const double dyn = wrms(s.dy, s.wsc, 1.0, S, s.red);
    if (k > 0) {
      rate = dyn / dy_old;
      double rp = 1.0;
      for (int m = 0; m < kNewtonMaxIter - k; ++m) rp *= rate;
      if (rate >= 1.0 || rp / (1.0 - rate) * dyn > c.a.newton_tol) break;
    }
    for (int i = threadIdx.x; i < S; i += NT) {
      s.y[i] += s.dy[i];
      s.dv[i] += s.dy[i];
    }
    __syncthreads();
    if (dyn == 0.0 || (k > 0 && rate / (1.0 - rate) * dyn < c.a.newton_tol)) {
      conv = true;
      break;
    }
    dy_old = dyn;
  }
  return conv;
}

// Trajectory recorder (all threads keep identical counters; thread 0 writes ops).
struct Recorder {
  bool on = false, full = false;
  int nops = 0, nsteps = 0;
};

__device__ void rec_op(const SolveArgs& a, int cell, Recorder& r, int kind, int q, double v) {
  if (!r.on || r.full) return;
  if (r.nops >= a.tape.cap_ops) {
    r.full = true;
    return;
  }
  if (threadIdx.x == 0) {
    const size_t o = (size_t)cell * a.tape.cap_ops + r.nops;
    a.tape.ops_kq[o] = (kind << 8) | q;
    a.tape.ops_v[o] = v;
  }
  r.nops++;
}

__device__ void rec_step(const SolveArgs& a, int cell, Recorder& r, int q, double h, double t_new, const double* y,
                         int S) {
  if (!r.on || r.full) return;
  if (r.nops >= a.tape.cap_ops || r.nsteps >= a.tape.cap_steps) {
    r.full = true;
    return;
  }
  double* dst = a.tape.ys + ((size_t)cell * a.tape.cap_steps + r.nsteps) * S;
  for (int i = threadIdx.x; i < S; i += NT) dst[i] = y[i];
  if (threadIdx.x == 0) a.tape.ts[(size_t)cell * a.tape.cap_steps + r.nsteps] = t_new;
  rec_op(a, cell, r, kOpStep, q, h);
  r.nsteps++;
}

// Environment of a cell at time t from its track (t_k, n_H, T, A_V, G0, zeta),
// k = 0..K-1: linear between knots, the end values outside [t_0, t_{K-1}]
// (the phi(t) of the generalised system of Sec. 2; x is per n_H, so a
// changing n_H enters only the two-body coefficients).
__device__ cbx_cell_params track_params(const double* track, int K, int cell, double t) {
  const double* k0 = track + (size_t)cell * K * 6;
  int k = 0;
  while (k + 1 < K && k0[(k + 1) * 6] <= t) ++k;
  const double* A = k0 + k * 6;
  if (k + 1 >= K || t <= A[0]) return cbx_cell_params{A[1], A[2], A[3], A[4], A[5]};
  const double* B = A + 6;
  const double w = (t - A[0]) / (B[0] - A[0]);
  return cbx_cell_params{fma(w, B[1] - A[1], A[1]), fma(w, B[2] - A[2], A[2]), fma(w, B[3] - A[3], A[3]),
                         fma(w, B[4] - A[4], A[4]), fma(w, B[5] - A[5], A[5])};
}

// The cell's end time: its own (merged requests of different spans in one
// launch) or the launch's.
__device__ __forceinline__ double cell_t_end(const SolveArgs& a, int cell) {
  return a.t_end_cell ? a.t_end_cell[cell] : a.t_end;
}

// Every knot finite with n_H, T > 0, and the knot times strictly increasing.
__device__ bool track_valid(const double* track, int K, int cell) {
  const double* k0 = track + (size_t)cell * K * 6;
  for (int k = 0; k < K; ++k) {
    const double* A = k0 + k * 6;
    for (int f = 0; f < 6; ++f)
      if (!isfinite(A[f])) return false;
    if (!(A[1] > 0.0) || !(A[2] > 0.0)) return false;
    if (k > 0 && !(A[0] > A[-6])) return false;
  }
  return true;
}

template <typename LT, bool GM>
__device__ void solve_cell(const SolveArgs& a, int cell, Smem& s, double* ws) {
  const DevNet& n = a.net;
  const int S = n.S;
  // workspace: kappa [R], partials [2R], J values [nnzJ], then (GM) the matrix
  LT* M = GM ? (LT*)(ws + (3LL * n.R + n.nnzJ + 31) / 32 * 32) : (LT*)s.M;
  __shared__ cbx_cell_stats s_stats;
  Cell<LT, GM> c{a, n, s, M, ws, ws + n.R, ws + 3 * n.R, &s_stats};
  if (threadIdx.x == 0) {
    *c.st = cbx_cell_stats{};
    c.st->t_begin_ns = (long long)globaltimer();
  }
  int attempts = 0;
  const cbx_cell_params p = a.track ? track_params(a.track, a.K, cell, a.t0) : a.phi[cell];
  int status = CBX_CELL_OK;
  Recorder rec;
  rec.on = a.tape.nops != nullptr;
  for (int i = threadIdx.x; i < S; i += NT) s.y[i] = a.x0[(size_t)__ldg(n.perm + i) * a.C + cell];
  if (!(p.n_H > 0.0) || !(p.T > 0.0) || !isfinite(p.n_H) || !isfinite(p.T) || !isfinite(p.A_V) ||
      !isfinite(p.G0) || !isfinite(p.zeta) || (a.track && !track_valid(a.track, a.K, cell)) ||
      !(cell_t_end(a, cell) >= a.t0) || !isfinite(cell_t_end(a, cell))) {
    status = CBX_CELL_BAD_INPUT;
    __syncthreads();
    for (int i = threadIdx.x; i < S; i += NT) a.x_out[(size_t)__ldg(n.perm + i) * a.C + cell] = s.y[i];
  } else {
    rate_coefficients(n, a.alpha, p, c.kap);
    __syncthreads();
    // with a track, the coefficients follow phi(t) to every time f or J is evaluated at
    double t_rates = a.t0;
    auto rates_at = [&](double tt) {
      if (a.track && tt != t_rates) {
        rate_coefficients(n, a.alpha, track_params(a.track, a.K, cell, tt), c.kap);
        __syncthreads();
        t_rates = tt;
      }
    };
    const double rtol = a.rtol, atol = a.atol, t_end = cell_t_end(a, cell);
    double* D = s.D;
    // f0 and the initial step (Hairer, Norsett & Wanner I, II.4, p = 1)
    rhs(n, c.kap, s.y, s.f, s.r, s.part);
    if (threadIdx.x == 0) c.st->rhs_evals++;
    for (int i = threadIdx.x; i < S; i += NT) s.wsc[i] = 1.0 / (atol + rtol * fabs(s.y[i]));
    __syncthreads();
    const double d0 = wrms(s.y, s.wsc, 1.0, S, s.red);
    const double d1 = wrms(s.f, s.wsc, 1.0, S, s.red);
    const double h0 = (d0 < 1e-5 || d1 < 1e-5) ? 1e-6 : 0.01 * d0 / d1;
    for (int i = threadIdx.x; i < S; i += NT) s.tmp[i] = s.y[i] + h0 * s.f[i];
    __syncthreads();
    rates_at(a.t0 + h0);
    rhs(n, c.kap, s.tmp, s.dy, s.r, s.part);
    if (threadIdx.x == 0) c.st->rhs_evals++;
    for (int i = threadIdx.x; i < S; i += NT) s.tmp[i] = s.dy[i] - s.f[i];
    __syncthreads();
    const double d2 = wrms(s.tmp, s.wsc, 1.0, S, s.red) / h0;
    const double dm = fmax(d1, d2);
    const double h1 = dm <= 1e-15 ? fmax(1e-6, h0 * 1e-3) : sqrt(0.01 / dm);
    double t = a.t0;
    double h = fmin(fmin(100.0 * h0, h1), t_end - t);
    for (int i = threadIdx.x; i < S; i += NT) {
      D[i] = s.y[i];
      D[S + i] = h * s.f[i];
      for (int r = 2; r < kDiffRows; ++r) D[r * S + i] = 0.0;
    }
    rec_op(a, cell, rec, kOpInit, 1, h);
    rates_at(a.t0);
    jacobian(n, c.kap, s.y, c.g, c.Jv);
    if (threadIdx.x == 0) c.st->jac_evals++;
    int q = 1, n_equal = 0;
    bool jac_current = true, lu_valid = false;
    double* slot = s.red + 40;
    while (t < t_end) {
      bool accepted = false;
      double t_new = t, err = 0.0;
      while (!accepted) {
        if (attempts >= a.max_steps) {
          status = CBX_CELL_MAX_STEPS;
          break;
        }
        attempts++;
        if (h < 10.0 * (::nextafter(t, __longlong_as_double(0x7ff0000000000000LL)) - t)) {
          status = CBX_CELL_H_UNDERFLOW;
          break;
        }
        t_new = t + h;
        if (t_new > t_end) {
          t_new = t_end;
          rescale(D, S, q, (t_end - t) / h, s.Tm);
          rec_op(a, cell, rec, kOpRescale, q, (t_end - t) / h);
          n_equal = 0;
          lu_valid = false;
          h = t_end - t;
        }
        const double gq = a.gam[q];
        for (int i = threadIdx.x; i < S; i += NT) {
          double yp = 0.0;
          for (int j = 0; j <= q; ++j) yp += D[j * S + i];
          double ps = 0.0;
          for (int j = 1; j <= q; ++j) ps = fma(a.gam[j], D[j * S + i], ps);
          s.yp[i] = yp;
          s.psi[i] = ps / gq;
          s.wsc[i] = 1.0 / (atol + rtol * fabs(yp));
        }
        __syncthreads();
        const double cc = h / gq;
        bool conv = false;
        int iters = 0;
        rates_at(t_new);
        for (;;) {
          if (!lu_valid) {
            factor(c, cc);
            lu_valid = true;
          }
          conv = newton(c, cc, &iters);
          if (threadIdx.x == 0) c.st->newton_iters += iters;
          if (conv || jac_current) break;
          jacobian(n, c.kap, s.yp, c.g, c.Jv);
          if (threadIdx.x == 0) c.st->jac_evals++;
          jac_current = true;
          lu_valid = false;
        }
        if (!conv) {
          if (threadIdx.x == 0) c.st->newton_fails++;
          rescale(D, S, q, 0.5, s.Tm);
          rec_op(a, cell, rec, kOpRescale, q, 0.5);
          h *= 0.5;
          n_equal = 0;
          lu_valid = false;
          continue;
        }
        for (int i = threadIdx.x; i < S; i += NT) s.wsc[i] = 1.0 / (atol + rtol * fabs(s.y[i]));
        __syncthreads();
        err = wrms(s.dv, s.wsc, 1.0 / (q + 1), S, s.red);
        if (err > 1.0) {
          if (threadIdx.x == 0) c.st->error_fails++;
          const double fac = fmax(0.2, 0.9 * uniform_pow(err, -1.0 / (q + 1), slot));
          rescale(D, S, q, fac, s.Tm);
          rec_op(a, cell, rec, kOpRescale, q, fac);
          h *= fac;
          n_equal = 0;
          lu_valid = false;
          continue;
        }
        accepted = true;
      }
      if (!accepted) break;
      rec_step(a, cell, rec, q, h, t_new, s.y, S);
      if (threadIdx.x == 0) c.st->steps++;
      t = t_new;
      jac_current = false;
      n_equal++;
      for (int i = threadIdx.x; i < S; i += NT) {
        const double d = s.dv[i];
        D[(q + 2) * S + i] = d - D[(q + 1) * S + i];
        D[(q + 1) * S + i] = d;
        for (int j = q; j >= 0; --j) D[j * S + i] += D[(j + 1) * S + i];
      }
      __syncthreads();
      if (n_equal < q + 1) continue;
      const double em = q > 1 ? wrms(D + q * S, s.wsc, 1.0 / q, S, s.red) : INFINITY;
      const double ep = q < kMaxOrder ? wrms(D + (q + 2) * S, s.wsc, 1.0 / (q + 2), S, s.red) : INFINITY;
      double fc[3];
      fc[0] = growth(em, q, slot);
      fc[1] = growth(err, q + 1, slot);
      fc[2] = growth(ep, q + 2, slot);
      int best = 0;
      if (fc[1] > fc[best]) best = 1;
      if (fc[2] > fc[best]) best = 2;
      q += best - 1;
      const double fac = fmin(10.0, 0.9 * fc[best]);
      rescale(D, S, q, fac, s.Tm);
      rec_op(a, cell, rec, kOpRescale, q, fac);
      h *= fac;
      n_equal = 0;
      lu_valid = false;
    }
    for (int i = threadIdx.x; i < S; i += NT) a.x_out[(size_t)__ldg(n.perm + i) * a.C + cell] = D[i];
  }
  if (rec.on && rec.full && status == CBX_CELL_OK) status = CBX_CELL_TAPE_FULL;
  if (threadIdx.x == 0) {
    if (rec.on) a.tape.nops[cell] = rec.nops;
    a.status[cell] = status;
    c.st->attempts = attempts;
    c.st->t_end_ns = (long long)globaltimer();
    if (a.stats) a.stats[cell] = *c.st;
  }
  __syncthreads();
}
// ---------------------------------------------------------------- ESDIRK
//
// The stiff integrator of the paper's own code is an ESDIRK of Kvaerno's
// family (Sec. 4). One step of size h from (t_n, y_n), with f_1 = f(t_n, y_n)
// (the previous step's f_5):
//   stage i = 2..5:  Y_i = y_n + h sum_{j<i} a_ij f_j + h gamma f(t_n + c_i h, Y_i)
//   y_{n+1} = Y_5, embedded Y_4 (both at c = 1), error estimate Y_5 - Y_4.
// Each stage is the corrector d - hgamma f(Y_{i-1} + d) + (Y_{i-1} - known) = 0
// solved by the same simplified Newton as the BDF (guess Y_{i-1}, matrix
// I - h gamma J, one LU for the four stages). Controller: err = |Y_5 - Y_4|
// (weights from |Y_5|) <= 1; h *= min(10, max(0.2, 0.9 err^(-1/4))) after an
// accepted step, max(0.2, 0.9 err^(-1/4)) after a rejected one; Newton
// failure: new J at (t_n, y_n) if stale, else h / 2; J at the start and after
// such failures; LU whenever h or J changed; initial step of Hairer, Norsett &
// Wanner I, II.4 with p = 3; last step shortened to t_end.
// Shared memory: the stage derivatives f_1..f_5 take rows 0..4 of the BDF's
// difference array, y_n row 5, the previous stage value row 6.
template <typename LT, bool GM>
__device__ void solve_cell_rk(const SolveArgs& a, int cell, Smem& s, double* ws) {
  const DevNet& n = a.net;
  const int S = n.S;
  LT* M = GM ? (LT*)(ws + (3LL * n.R + n.nnzJ + 31) / 32 * 32) : (LT*)s.M;
  __shared__ cbx_cell_stats s_stats;
  Cell<LT, GM> c{a, n, s, M, ws, ws + n.R, ws + 3 * n.R, &s_stats};
  if (threadIdx.x == 0) {
    *c.st = cbx_cell_stats{};
    c.st->t_begin_ns = (long long)globaltimer();
  }
  int attempts = 0;
  const cbx_cell_params p = a.track ? track_params(a.track, a.K, cell, a.t0) : a.phi[cell];
  int status = CBX_CELL_OK;
  double* F = s.D;           // f_1..f_5, rows 0..4
  double* yn = s.D + 5 * S;  // y_n
  double* yprev = s.D + 6 * S;
  for (int i = threadIdx.x; i < S; i += NT) yn[i] = a.x0[(size_t)__ldg(n.perm + i) * a.C + cell];
  if (!(p.n_H > 0.0) || !(p.T > 0.0) || !isfinite(p.n_H) || !isfinite(p.T) || !isfinite(p.A_V) ||
      !isfinite(p.G0) || !isfinite(p.zeta) || (a.track && !track_valid(a.track, a.K, cell)) ||
      !(cell_t_end(a, cell) >= a.t0) || !isfinite(cell_t_end(a, cell))) {
    status = CBX_CELL_BAD_INPUT;
    __syncthreads();
    for (int i = threadIdx.x; i < S; i += NT) a.x_out[(size_t)__ldg(n.perm + i) * a.C + cell] = yn[i];
  } else {
    rate_coefficients(n, a.alpha, p, c.kap);
    __syncthreads();
    double t_rates = a.t0;
    auto rates_at = [&](double tt) {
      if (a.track && tt != t_rates) {
        rate_coefficients(n, a.alpha, track_params(a.track, a.K, cell, tt), c.kap);
        __syncthreads();
        t_rates = tt;
      }
    };
    const double rtol = a.rtol, atol = a.atol, t_end = cell_t_end(a, cell);
    const double gamma = a.rk_a[1][1];
    double* slot = s.red + 40;
    // f_1 and the initial step (Hairer, Norsett & Wanner I, II.4, p = 3)
    rhs(n, c.kap, yn, F, s.r, s.part);
    if (threadIdx.x == 0) c.st->rhs_evals++;
    for (int i = threadIdx.x; i < S; i += NT) s.wsc[i] = 1.0 / (atol + rtol * fabs(yn[i]));
    __syncthreads();
    const double d0 = wrms(yn, s.wsc, 1.0, S, s.red);
    const double d1 = wrms(F, s.wsc, 1.0, S, s.red);
    const double h0 = (d0 < 1e-5 || d1 < 1e-5) ? 1e-6 : 0.01 * d0 / d1;
    for (int i = threadIdx.x; i < S; i += NT) s.tmp[i] = yn[i] + h0 * F[i];
    __syncthreads();
    rates_at(a.t0 + h0);
    rhs(n, c.kap, s.tmp, s.dy, s.r, s.part);
    if (threadIdx.x == 0) c.st->rhs_evals++;
    for (int i = threadIdx.x; i < S; i += NT) s.tmp[i] = s.dy[i] - F[i];
    __syncthreads();
    const double d2 = wrms(s.tmp, s.wsc, 1.0, S, s.red) / h0;
    const double dm = fmax(d1, d2);
    const double h1 = dm <= 1e-15 ? fmax(1e-6, h0 * 1e-3) : uniform_pow(0.01 / dm, 0.25, slot);
    double t = a.t0;
    double h = fmin(fmin(100.0 * h0, h1), t_end - t);
    rates_at(a.t0);
    jacobian(n, c.kap, yn, c.g, c.Jv);
    if (threadIdx.x == 0) c.st->jac_evals++;
    bool jac_current = true, lu_valid = false;
    double lu_h = 0.0, err = 0.0;
    while (t < t_end) {
      bool accepted = false;
      while (!accepted) {
        if (attempts >= a.max_steps) {
          status = CBX_CELL_MAX_STEPS;
          break;
        }
        attempts++;
        if (h < 10.0 * (::nextafter(t, __longlong_as_double(0x7ff0000000000000LL)) - t)) {
          status = CBX_CELL_H_UNDERFLOW;
          break;
        }
        if (t + h > t_end) h = t_end - t;
        const double hg = h * gamma;
        bool failed;
        for (;;) {
          if (!lu_valid || lu_h != h) {
            factor(c, hg);
            lu_valid = true;
            lu_h = h;
          }
          failed = false;
          for (int i = threadIdx.x; i < S; i += NT) {
            yprev[i] = yn[i];
            s.wsc[i] = 1.0 / (atol + rtol * fabs(yn[i]));
          }
          __syncthreads();
          for (int st = 1; st < 5; ++st) {
            const double ti = t + a.rk_c[st] * h;
            // guess Y_{i-1}; psi = guess - known, known = y_n + h sum_{j<i} a_ij f_j
            for (int i = threadIdx.x; i < S; i += NT) {
              double known = 0.0;
              for (int j = 0; j < st; ++j) known = fma(a.rk_a[st][j], F[j * S + i], known);
              known = fma(h, known, yn[i]);
              s.yp[i] = yprev[i];
              s.psi[i] = yprev[i] - known;
            }
            __syncthreads();
            rates_at(ti);
            int iters = 0;
            const bool conv = newton(c, hg, &iters);
            if (threadIdx.x == 0) c.st->newton_iters += iters;
            if (!conv) {
              failed = true;
              break;
            }
            rhs(n, c.kap, s.y, F + st * S, s.r, s.part);
            if (threadIdx.x == 0) c.st->rhs_evals++;
            if (st < 4) {  // after the last stage yprev keeps the embedded solution Y_4
              for (int i = threadIdx.x; i < S; i += NT) yprev[i] = s.y[i];
              __syncthreads();
            }
          }
          if (!failed || jac_current) break;
          rates_at(t);
          jacobian(n, c.kap, yn, c.g, c.Jv);
          if (threadIdx.x == 0) c.st->jac_evals++;
          jac_current = true;
          lu_valid = false;
        }
        if (failed) {
          if (threadIdx.x == 0) c.st->newton_fails++;
          h *= 0.5;
          continue;
        }
        // error estimate Y_5 - Y_4 (s.y = Y_5, yprev = Y_4), weights from |Y_5|
        for (int i = threadIdx.x; i < S; i += NT) {
          s.wsc[i] = 1.0 / (atol + rtol * fabs(s.y[i]));
          s.tmp[i] = s.y[i] - yprev[i];
        }
        __syncthreads();
        err = wrms(s.tmp, s.wsc, 1.0, S, s.red);
        if (err > 1.0) {
          if (threadIdx.x == 0) c.st->error_fails++;
          h *= fmax(0.2, 0.9 * uniform_pow(err, -0.25, slot));
          continue;
        }
        accepted = true;
      }
      if (!accepted) break;
      if (threadIdx.x == 0) c.st->steps++;
      t = t + h;
      for (int i = threadIdx.x; i < S; i += NT) {
        yn[i] = s.y[i];
        F[i] = F[4 * S + i];
      }
      __syncthreads();
      jac_current = false;
      const double fac = err == 0.0 ? 10.0 : 0.9 * uniform_pow(err, -0.25, slot);
      h *= fmin(10.0, fmax(0.2, fac));
    }
    for (int i = threadIdx.x; i < S; i += NT) a.x_out[(size_t)__ldg(n.perm + i) * a.C + cell] = yn[i];
  }
  if (threadIdx.x == 0) {
    a.status[cell] = status;
    c.st->attempts = attempts;
    c.st->t_end_ns = (long long)globaltimer();
    if (a.stats) a.stats[cell] = *c.st;
  }
  __syncthreads();
}

template <typename LT, bool GM, bool RK = false>
__global__ void __launch_bounds__(NT, 1) solve_kernel(const SolveArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_cell;
  Smem s;
  layout(a.net.S, a.net.R, a.net.nseg, sizeof(LT) == 4, GM, smem_raw, &s, a.piv_ints);
  s.piv = global_pivots(a.net);
  if constexpr (!GM && sizeof(LT) == 8) {
    if (a.piv_ints > 0) stage_pivots(a.net, s);
  }
  double* ws = a.ws + (size_t)blockIdx.x * a.ws_stride;
  for (;;) {
    if (threadIdx.x == 0) s_cell = atomicAdd(a.counter, 1);
    __syncthreads();
    const int cell = s_cell;
    __syncthreads();
    if (cell >= a.C) break;
    if constexpr (RK)
      solve_cell_rk<LT, GM>(a, cell, s, ws);
    else
      solve_cell<LT, GM>(a, cell, s, ws);
  }
}

template <typename LT, bool GM, bool RK = false>
static int launch_t(const SolveArgs& a, size_t sm, int grid, cudaStream_t st) {
  cudaError_t e = cudaFuncSetAttribute(solve_kernel<LT, GM, RK>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  solve_kernel<LT, GM, RK><<<grid, NT, sm, st>>>(a);
  return cudaGetLastError();
}

template <typename LT, bool GM>
static int occupancy_t(size_t sm) {
  int blocks = 0;
  cudaError_t e = cudaFuncSetAttribute(solve_kernel<LT, GM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, solve_kernel<LT, GM>, NT, sm);
  return e == cudaSuccess ? blocks : 0;
}

}  // namespace
}  // namespace cbx
