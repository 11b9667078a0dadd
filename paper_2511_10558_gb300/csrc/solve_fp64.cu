// Instantiation of the solver kernel for LT = double, matrix in shared memory.
#include "solver_dev.cuh"

namespace cbx {

int launch_solve_fp64(const SolveArgs& a, size_t smem, int grid, void* stream) {
  return launch_t<double, false>(a, smem, grid, (cudaStream_t)stream);
}

int occupancy_solve_fp64(size_t smem) { return occupancy_t<double, false>(smem); }

}  // namespace cbx
