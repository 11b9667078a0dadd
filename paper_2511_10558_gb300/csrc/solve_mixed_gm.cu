// Instantiation of the solver kernel for LT = float, matrix in the CTA's global workspace.
#include "solver_dev.cuh"

namespace cbx {

int launch_solve_mixed_gm(const SolveArgs& a, size_t smem, int grid, void* stream) {
  return launch_t<float, true>(a, smem, grid, (cudaStream_t)stream);
}

int occupancy_solve_mixed_gm(size_t smem) { return occupancy_t<float, true>(smem); }

}  // namespace cbx
