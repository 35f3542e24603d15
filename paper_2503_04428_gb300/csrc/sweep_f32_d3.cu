// Fused sweep kernels: float state, 3D grids (all scalar counts and Riemann solvers).
#include "sweep.cuh"

namespace hydro {
HYDRO_SWEEP_DISPATCH(float, 3)
}  // namespace hydro
