// Fused sweep kernels: float state, 2D grids (all scalar counts and Riemann solvers).
#include "sweep.cuh"

namespace hydro {
HYDRO_SWEEP_DISPATCH(float, 2)
}  // namespace hydro
