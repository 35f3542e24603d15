// Fused sweep kernels with the gas + radiation EoS (Eq. 6-7): float state, 3D grids, HLL and HLLC, with and without dual energy.
#include "sweep.cuh"

namespace hydro {
HYDRO_SWEEP_DISPATCH_RAD(float, 3)
}  // namespace hydro
