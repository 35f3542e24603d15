// Fused sweep kernels: float state, 1D grids (all scalar counts and Riemann solvers).
#include "sweep.cuh"

namespace hydro {
HYDRO_SWEEP_DISPATCH(float, 1)
}  // namespace hydro
