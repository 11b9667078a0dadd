// Instantiation of the solver kernel for LT = double, matrix in the CTA's global workspace.
#include "solver_dev.cuh"

namespace cbx {

int launch_solve_fp64_gm(const SolveArgs& a, size_t smem, int grid, void* stream) {
  return launch_t<double, true>(a, smem, grid, (cudaStream_t)stream);
}

int occupancy_solve_fp64_gm(size_t smem) { return occupancy_t<double, true>(smem); }

}  // namespace cbx
