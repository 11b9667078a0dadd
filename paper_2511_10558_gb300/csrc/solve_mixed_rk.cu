// Instantiation of the ESDIRK solver kernel for LT = float, matrix in shared memory.
#include "solver_dev.cuh"

namespace cbx {

int launch_solve_mixed_rk(const SolveArgs& a, size_t smem, int grid, void* stream) {
  return launch_t<float, false, true>(a, smem, grid, (cudaStream_t)stream);
}

}  // namespace cbx
