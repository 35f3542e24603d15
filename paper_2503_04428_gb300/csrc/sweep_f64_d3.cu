// Fused sweep kernels: double state, 3D grids (all scalar counts and Riemann solvers).
#include "sweep.cuh"

namespace hydro {
HYDRO_SWEEP_DISPATCH(double, 3)
}  // namespace hydro
