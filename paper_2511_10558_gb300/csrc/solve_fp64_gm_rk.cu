// Instantiation of the ESDIRK solver kernel for LT = double, matrix in the CTA's global workspace.
#include "solver_dev.cuh"

namespace cbx {

int launch_solve_fp64_gm_rk(const SolveArgs& a, size_t smem, int grid, void* stream) {
  return launch_t<double, true, true>(a, smem, grid, (cudaStream_t)stream);
}

}  // namespace cbx
