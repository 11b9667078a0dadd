// Instantiation of the solver kernel for LT = float, matrix in shared memory.
#include "solver_dev.cuh"

namespace cbx {

int launch_solve_mixed(const SolveArgs& a, size_t smem, int grid, void* stream) {
  return launch_t<float, false>(a, smem, grid, (cudaStream_t)stream);
}

int occupancy_solve_mixed(size_t smem) { return occupancy_t<float, false>(smem); }

}  // namespace cbx
