// Fused sweep kernels of a slab of a decomposed grid or of a moving grid (Sect. 3.1.1, 3.3.1):
// double state, 1D grids, ideal gas.
#include "sweep.cuh"

namespace hydro {
HYDRO_SWEEP_DISPATCH_XM(double, 1)
}  // namespace hydro
