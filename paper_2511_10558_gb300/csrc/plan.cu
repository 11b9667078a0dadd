// Launch planning of the solver kernel (host code): shared-memory and
// workspace sizes, the matrix placement, occupancy, and the dispatch to the
// translation unit holding each kernel instantiation.
#include "solver_dev.cuh"

namespace cbx {

size_t smem_bytes(int S, int R, int nseg, bool mixed, bool gm, int piv_ints) {
  return layout(S, R, nseg, mixed, gm, nullptr, nullptr, piv_ints);
}

long long workspace_doubles(int S, int R, int nnzJ, bool mixed, bool gm) {
  long long n = 3LL * R + nnzJ;
  n = (n + 31) / 32 * 32;
  if (gm) n += ((long long)S * lead_dim(S) * (mixed ? 4 : 8) / 8 + 31) / 32 * 32;
  return n;
}

SolverPlan plan_solver(int S, int R, int nseg, int nnzJ, bool mixed, int head_ints) {
  SolverPlan p;
  p.mixed = mixed;
  const size_t optin = device_smem_optin();
  // shared-memory matrix when it fits and the FP64 LU's register tiling allows (S <= 256)
  p.gm = !(S <= 32 * kMaxColRegs && smem_bytes(S, R, nseg, mixed, false) <= optin);
  p.smem = smem_bytes(S, R, nseg, mixed, p.gm);
  // FP64 shared-memory solver: stage the sparse pivots' lists when they fit
  if (!mixed && !p.gm && smem_bytes(S, R, nseg, false, false, head_ints) <= optin) {
    p.piv_ints = head_ints;
    p.smem = smem_bytes(S, R, nseg, false, false, head_ints);
  }
  p.ws_stride = workspace_doubles(S, R, nnzJ, mixed, p.gm);
  p.occupancy = 0;
  if (S > 2 * NT || p.smem > optin) return p;
  if (mixed)
    p.occupancy = p.gm ? occupancy_solve_mixed_gm(p.smem) : occupancy_solve_mixed(p.smem);
  else
    p.occupancy = p.gm ? occupancy_solve_fp64_gm(p.smem) : occupancy_solve_fp64(p.smem);
  return p;
}

int launch_solver(const SolveArgs& a0, const SolverPlan& p, int grid, void* stream) {
  SolveArgs a = a0;
  a.piv_ints = p.piv_ints;
  if (p.mixed)
    return p.gm ? launch_solve_mixed_gm(a, p.smem, grid, stream) : launch_solve_mixed(a, p.smem, grid, stream);
  return p.gm ? launch_solve_fp64_gm(a, p.smem, grid, stream) : launch_solve_fp64(a, p.smem, grid, stream);
}

int device_sm_count() {
  int dev = 0, v = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
  return v;
}

size_t device_smem_optin() {
  int dev = 0, v = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  return (size_t)v;
}

int launch_solver_rk(const SolveArgs& a0, const SolverPlan& p, int grid, void* stream) {
  SolveArgs a = a0;
  a.piv_ints = p.piv_ints;
  if (p.gm)
    return p.mixed ? launch_solve_mixed_gm_rk(a, p.smem, grid, stream) : launch_solve_fp64_gm_rk(a, p.smem, grid, stream);
  return p.mixed ? launch_solve_mixed_rk(a, p.smem, grid, stream) : launch_solve_fp64_rk(a, p.smem, grid, stream);
}

}  // namespace cbx
