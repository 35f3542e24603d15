// Fused sweep kernels with the dual-energy correction (Sect. 2.5): float state, 3D grids, ideal gas.
#include "sweep.cuh"

namespace hydro {
HYDRO_SWEEP_DISPATCH_DUAL(float, 3)
}  // namespace hydro
