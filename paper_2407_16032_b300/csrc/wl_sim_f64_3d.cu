// wl_sim_f64_3d.cu -- Sim<double, 3>: the FP64 3D time step.
#include "wl_sim.cuh"

namespace wl {
SimBase *new_sim_f64_3d() { return new Sim<double, 3>(); }
}  // namespace wl
