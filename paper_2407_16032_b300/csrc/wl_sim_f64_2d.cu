// wl_sim_f64_2d.cu -- Sim<double, 2>: the FP64 2D time step.
#include "wl_sim.cuh"

namespace wl {
SimBase *new_sim_f64_2d() { return new Sim<double, 2>(); }
}  // namespace wl
