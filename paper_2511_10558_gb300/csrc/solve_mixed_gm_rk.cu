// Instantiation of the ESDIRK solver kernel for LT = float, matrix in the CTA's global workspace.
#include "solver_dev.cuh"

namespace cbx {

int launch_solve_mixed_gm_rk(const SolveArgs& a, size_t smem, int grid, void* stream) {
  return launch_t<float, true, true>(a, smem, grid, (cudaStream_t)stream);
}

}  // namespace cbx
