// Fused sweep kernels with the dual-energy correction (Sect. 2.5): float state, 2D grids, ideal gas.
#include "sweep.cuh"

namespace hydro {
HYDRO_SWEEP_DISPATCH_DUAL(float, 2)
}  // namespace hydro
