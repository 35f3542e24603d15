// Fused sweep kernels of a slab of a decomposed grid or of a moving grid (Sect. 3.1.1, 3.3.1):
// double state, 3D grids, ideal gas.
#include "sweep.cuh"

namespace hydro {
HYDRO_SWEEP_DISPATCH_XM(double, 3)
}  // namespace hydro
