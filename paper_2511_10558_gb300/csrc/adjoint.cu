// Discrete adjoint of the recorded BDF solve, and the per-cell reductions of
// its gradients.
#include "solver_dev.cuh"

namespace cbx {
namespace {
// ---------------------------------------------------------------- adjoint
//
// Discrete adjoint of the BDF map recorded on a tape (Sec. 3: sensitivities of
// model outputs to chemical and physical inputs). For the frozen program
// (init, rescales, accepted steps with their results y) and each corrector
// differentiated as if solved exactly, the reverse sweep carries the cotangent
// Lam of the difference array:
//   step (q, h):  lam_d = sum_{i<=q+2} Lam'[i];  mu = (I - cJ(y))^{-T} lam_d
//                 Lam[k] = sum_{i<=k} Lam'[i] + mu - lam_d - [k>=1] gamma_k/gamma_q mu  (k<=q)
//                 Lam[q+1] = -Lam'[q+2], Lam[q+2] = 0
//                 dL/d ln alpha_j += c (nu^T mu)_j r_j(y)   (c = h/gamma_q)
//   rescale:      Lam[1..q] <- T(rho)^T Lam[1..q]
//   init (h0):    dL/d ln alpha_j += h0 (nu^T Lam[1])_j r_j(y0)
// ln n_H enters through the two-body coefficients (d ln kappa_j / d ln n_H = 1)
// and T through the two-body and cosmic-ray-induced photo forms:
// d ln kappa_j / dT = beta_j/T + gamma_j/T^2 (two-body), beta_j/T (CR photo).

// v <- U^{-T} v (U unit upper, so U^T is unit lower), blocks of 32.
__device__ void forwardT_crout64(const double* M, int S, double* v) {
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, ld = lead_dim(S);
  for (int kb = 0; kb < S; kb += 32) {
    const int nb = min(32, S - kb), ke = kb + nb;
    if (w == 0) {
      double val = lane < nb ? v[kb + lane] : 0.0;
#pragma unroll
      for (int c = 0; c < 32; ++c) {
        if (c < nb) {
          const double yc = __shfl_sync(FULL, val, c);
          if (lane > c && lane < nb) val = fma(-M[(kb + c) * ld + kb + lane], yc, val);
        }
      }
      if (lane < nb) v[kb + lane] = val;
    }
    __syncthreads();
    for (int i = ke + threadIdx.x; i < S; i += NT) {
      double p0 = v[i], p1 = 0.0;
      int c = 0;
      for (; c + 2 <= nb; c += 2) {
        p0 = fma(-M[(kb + c) * ld + i], v[kb + c], p0);
        p1 = fma(-M[(kb + c + 1) * ld + i], v[kb + c + 1], p1);
      }
      if (c < nb) p0 = fma(-M[(kb + c) * ld + i], v[kb + c], p0);
      v[i] = p0 + p1;
    }
    __syncthreads();
  }
}

// v <- L^{-T} v (L unit lower, so L^T is unit upper), blocks of 32 from the bottom.
__device__ void backwardT_crout64(const double* M, int S, double* v) {
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, ld = lead_dim(S);
  for (int kb = ((S - 1) / 32) * 32; kb >= 0; kb -= 32) {
    const int nb = min(32, S - kb);
    if (w == 0) {
      double val = lane < nb ? v[kb + lane] : 0.0;
#pragma unroll
      for (int c = 31; c >= 0; --c) {
        if (c < nb) {
          const double xc = __shfl_sync(FULL, val, c);
          if (lane < c) val = fma(-M[(kb + c) * ld + kb + lane], xc, val);
        }
      }
      if (lane < nb) v[kb + lane] = val;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kb; i += NT) {
      double p0 = v[i], p1 = 0.0;
      int c = 0;
      for (; c + 2 <= nb; c += 2) {
        p0 = fma(-M[(kb + c) * ld + i], v[kb + c], p0);
        p1 = fma(-M[(kb + c + 1) * ld + i], v[kb + c + 1], p1);
      }
      if (c < nb) p0 = fma(-M[(kb + c) * ld + i], v[kb + c], p0);
      v[i] = p0 + p1;
    }
    __syncthreads();
  }
}

// w_j = (nu^T u)_j = sum over products of u - sum over reactants of u
__device__ void nu_transpose(const DevNet& n, const double* u, double* w) {
  for (int j = threadIdx.x; j < n.R; j += NT) {
    const int b = n.rb[j];
    double v = -u[n.ra[j]];
    if (b >= 0) v -= u[b];
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      const int pr = n.rprod[4 * j + p];
      if (pr >= 0) v += u[pr];
    }
    w[j] = v;
  }
  __syncthreads();
}

// grow[j] += scale w_j r_j(y); returns the n_H and T contributions (block sums).
__device__ void grad_accumulate(const DevNet& n, const double* kap, const double* dlnk_dT, const double* y,
                                const double* w, double scale, double* grow, double* red, double* out_nH,
                                double* out_T) {
  double pn = 0.0, pt = 0.0;
  for (int j = threadIdx.x; j < n.R; j += NT) {
    const int b = n.rb[j];
    double r = kap[j] * y[n.ra[j]];
    if (b >= 0) r *= y[b];
    const double c = scale * w[j] * r;
    grow[j] += c;
    if (n.rtype[j] == CBX_TWO_BODY) pn += c;
    pt = fma(c, dlnk_dT[j], pt);  // zero for the forms without T
  }
  *out_nH += block_sum(pn, red);
  *out_T += block_sum(pt, red);
}

__global__ void __launch_bounds__(NT, 1) grad_kernel(const GradArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_cell;
  const DevNet& n = a.net;
  const int S = n.S, R = n.R;
  Smem s;
  layout(S, R, n.nseg, false, false, smem_raw, &s);
  double* M = (double*)s.M;
  double* invd = (double*)s.invd;
  double* Lam = s.D;
  double* ws = a.ws + (size_t)blockIdx.x * a.ws_stride;
  double* kap = ws;            // [R]
  double* g = ws + R;          // [2R] partials, then nu^T mu
  double* Jv = ws + 3 * R;     // [nnzJ]
  double* dT = Jv + n.nnzJ;    // [R]
  for (;;) {
    if (threadIdx.x == 0) s_cell = atomicAdd(a.counter, 1);
    __syncthreads();
    const int cell = s_cell;
    __syncthreads();
    if (cell >= a.C) break;
    double* grow = a.gcell + (size_t)cell * R;
    for (int j = threadIdx.x; j < R; j += NT) grow[j] = 0.0;
    double gnH = 0.0, gT = 0.0;
    const int nops = a.tape.nops[cell];
    if (a.status[cell] == CBX_CELL_OK && nops > 0) {
      // rate coefficients and d ln k_j / dT of the environment p: two-body
      // (T/300)^beta exp(-gamma/T); CR-induced photo (T/300)^beta
      auto rates_for = [&](const cbx_cell_params& p) {
        rate_coefficients(n, a.alpha, p, kap);
        for (int j = threadIdx.x; j < R; j += NT) {
          const int t = n.rtype[j];
          dT[j] = t == CBX_TWO_BODY ? n.beta[j] / p.T + n.gamma[j] / (p.T * p.T)
                                    : (t == CBX_CR_PHOTO ? n.beta[j] / p.T : 0.0);
        }
        __syncthreads();
      };
      // with a track, the step at t_new used the coefficients of phi(t_new),
      // the initial difference D[1] = h0 f(y0) those of phi(t0)
      if (!a.track) rates_for(a.phi[cell]);
      for (int i = threadIdx.x; i < S; i += NT) {
        const int u = __ldg(n.perm + i);
        Lam[i] = a.cot[(size_t)u * a.C + cell];
        for (int r = 1; r < kDiffRows; ++r) Lam[r * S + i] = 0.0;
        s.tmp[i] = a.x0[(size_t)u * a.C + cell];  // y0, internal order
      }
      __syncthreads();
      const int* kq = a.tape.ops_kq + (size_t)cell * a.tape.cap_ops;
      const double* vv = a.tape.ops_v + (size_t)cell * a.tape.cap_ops;
      int sidx = 0;
      for (int o = 0; o < nops; ++o) sidx += (kq[o] >> 8) == kOpStep;
      for (int o = nops - 1; o >= 0; --o) {
        const int kind = kq[o] >> 8, q = kq[o] & 255;
        const double v = vv[o];
        if (kind == kOpStep) {
          --sidx;
          if (a.track) rates_for(track_params(a.track, a.K, cell, a.tape.ts[(size_t)cell * a.tape.cap_steps + sidx]));
          const double* y = a.tape.ys + ((size_t)cell * a.tape.cap_steps + sidx) * S;
          for (int i = threadIdx.x; i < S; i += NT) {
            s.y[i] = y[i];
            double L[kDiffRows];
#pragma unroll
            for (int r = 0; r < kDiffRows; ++r) L[r] = Lam[r * S + i];
            double lam_d = 0.0;
#pragma unroll
            for (int r = 0; r < kDiffRows; ++r)
              if (r <= q + 2) lam_d += L[r];
            s.dv[i] = lam_d;
            double pre = 0.0;
#pragma unroll
            for (int r = 0; r <= kMaxOrder; ++r) {
              if (r <= q) {
                pre += L[r];
                Lam[r * S + i] = pre;
              }
            }
            Lam[(q + 1) * S + i] = -L[q + 2 < kDiffRows ? q + 2 : kDiffRows - 1];
            if (q + 2 < kDiffRows) Lam[(q + 2) * S + i] = 0.0;
            s.dy[i] = lam_d;
          }
          __syncthreads();
          const double c = v / a.gam[q];
          jacobian(n, kap, s.y, g, Jv);
          build_matrix<double>(n, Jv, c, M);
          lu_crout64(global_pivots(n), M, invd);
          forwardT_crout64(M, S, s.dy);
          for (int i = threadIdx.x; i < S; i += NT) s.dy[i] *= invd[i];
          __syncthreads();
          backwardT_crout64(M, S, s.dy);
          const double gq = a.gam[q];
          for (int i = threadIdx.x; i < S; i += NT) {
            const double mu = s.dy[i], md = mu - s.dv[i];
            for (int r = 0; r <= q; ++r) {
              double x = Lam[r * S + i] + md;
              if (r >= 1) x -= a.gam[r] / gq * mu;
              Lam[r * S + i] = x;
            }
          }
          nu_transpose(n, s.dy, g);
          grad_accumulate(n, kap, dT, s.y, g, c, grow, s.red, &gnH, &gT);
        } else if (kind == kOpRescale) {
          // Lam[1..q] <- T(rho)^T Lam[1..q]
          if (threadIdx.x < 32) {
            const int lane = threadIdx.x;
            if (lane < q * q) {
              const int k = lane / q + 1, j = lane % q + 1;
              s.Tm[(k - 1) * kMaxOrder + (j - 1)] = rescale_entry(k, j, v);
            }
          }
          __syncthreads();
          for (int i = threadIdx.x; i < S; i += NT) {
            double old[kMaxOrder];
#pragma unroll
            for (int k = 0; k < kMaxOrder; ++k) old[k] = k < q ? Lam[(k + 1) * S + i] : 0.0;
            for (int j = 0; j < q; ++j) {
              double acc = 0.0;
#pragma unroll
              for (int k = 0; k < kMaxOrder; ++k)
                if (k < q) acc = fma(s.Tm[k * kMaxOrder + j], old[k], acc);
              Lam[(j + 1) * S + i] = acc;
            }
          }
          __syncthreads();
        } else {  // init
          if (a.track) rates_for(track_params(a.track, a.K, cell, a.t0));
          nu_transpose(n, Lam + S, g);
          grad_accumulate(n, kap, dT, s.tmp, g, v, grow, s.red, &gnH, &gT);
        }
      }
    }
    if (threadIdx.x == 0) {
      if (a.g_lognH) a.g_lognH[cell] = gnH;
      if (a.g_T) a.g_T[cell] = gT;
    }
    __syncthreads();
  }
}

__global__ void reduce_cells_kernel(const double* gcell, int C, int R, double* out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= R) return;
  double acc = 0.0;
  for (int c = 0; c < C; ++c) acc += gcell[(size_t)c * R + j];
  out[j] = acc;
}

// Environment gradients of each cell from its per-reaction gradients
// dL/d ln k_j (k_j is proportional to alpha_j, so these are the per-cell
// dL/d ln alpha_j): cosmic-ray coefficients carry the factor zeta (Sec. 2), as
// do those of secondary photons induced by cosmic rays (App. B.1), and photo
// coefficients G0 exp(-gamma_j A_V) (App. B.1), hence
//   dL/d ln zeta = sum over both cosmic-ray forms,  dL/d ln G0 = sum over photo j,
//   dL/dA_V = -sum over photo j of gamma_j dL/d ln k_j.
// One warp per cell: lanes take reactions lane, lane + 32, ..., and lane 0
// ends with a fixed shuffle-tree sum (deterministic).
__global__ void env_grad_kernel(const double* gcell, int C, int R, const int* rtype, const double* gamma,
                                double* g_lnzeta, double* g_lnG0, double* g_AV) {
  const int cell = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (cell >= C) return;  // whole warps leave together
  const double* row = gcell + (size_t)cell * R;
  double z = 0.0, g = 0.0, av = 0.0;
  for (int j = lane; j < R; j += 32) {
    const int t = rtype[j];
    const double v = row[j];
    if (t == CBX_COSMIC_RAY || t == CBX_CR_PHOTO) {
      z += v;
    } else if (t == CBX_PHOTO) {
      g += v;
      av -= gamma[j] * v;
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    z += __shfl_xor_sync(FULL, z, o);
    g += __shfl_xor_sync(FULL, g, o);
    av += __shfl_xor_sync(FULL, av, o);
  }
  if (lane == 0) {
    if (g_lnzeta) g_lnzeta[cell] = z;
    if (g_lnG0) g_lnG0[cell] = g;
    if (g_AV) g_AV[cell] = av;
  }
}

}  // namespace

int launch_env_grad(const double* gcell, int C, const DevNet& n, double* g_lnzeta, double* g_lnG0, double* g_AV,
                    void* stream) {
  if (C <= 0) return cudaSuccess;
  constexpr int kCellsPerBlock = 8;
  env_grad_kernel<<<(C + kCellsPerBlock - 1) / kCellsPerBlock, 32 * kCellsPerBlock, 0, (cudaStream_t)stream>>>(
      gcell, C, n.R, n.rtype, n.gamma, g_lnzeta, g_lnG0, g_AV);
  return cudaGetLastError();
}

long long grad_workspace_doubles(int S, int R, int nnzJ) {
  (void)S;
  return (4LL * R + nnzJ + 31) / 32 * 32;
}

int grad_occupancy(int S, int R, int nseg) {
  const size_t sm = smem_bytes(S, R, nseg, false, false);
  if (S > 32 * kMaxColRegs || sm > device_smem_optin()) return 0;
  int blocks = 0;
  cudaError_t e = cudaFuncSetAttribute(grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, grad_kernel, NT, sm);
  return e == cudaSuccess ? blocks : 0;
}

int launch_grad(const GradArgs& a, int grid, void* stream) {
  const size_t sm = smem_bytes(a.net.S, a.net.R, a.net.nseg, false, false);
  cudaError_t e = cudaFuncSetAttribute(grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  grad_kernel<<<grid, NT, sm, (cudaStream_t)stream>>>(a);
  return cudaGetLastError();
}

int launch_reduce_cells(const double* gcell, int C, int R, double* out, void* stream) {
  if (R <= 0) return cudaSuccess;
  reduce_cells_kernel<<<(R + 255) / 256, 256, 0, (cudaStream_t)stream>>>(gcell, C, R, out);
  return cudaGetLastError();
}

}  // namespace cbx
