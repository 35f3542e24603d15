// Fused sweep kernels: double state, 1D grids (all scalar counts and Riemann solvers).
#include "sweep.cuh"

namespace hydro {
HYDRO_SWEEP_DISPATCH(double, 1)
}  // namespace hydro
