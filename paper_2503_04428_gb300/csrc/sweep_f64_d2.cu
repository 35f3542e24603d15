// Fused sweep kernels: double state, 2D grids (all scalar counts and Riemann solvers).
#include "sweep.cuh"

namespace hydro {
HYDRO_SWEEP_DISPATCH(double, 2)
}  // namespace hydro
