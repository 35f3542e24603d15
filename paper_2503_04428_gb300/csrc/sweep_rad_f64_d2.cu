// Fused sweep kernels with the gas + radiation EoS (Eq. 6-7): double state, 2D grids, HLL and HLLC, with and without dual energy.
#include "sweep.cuh"

namespace hydro {
HYDRO_SWEEP_DISPATCH_RAD(double, 2)
}  // namespace hydro
