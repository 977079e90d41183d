// wl_sim_f32_2d.cu -- Sim<float, 2>: the FP32 2D time step.
#include "wl_sim.cuh"

namespace wl {
SimBase *new_sim_f32_2d() { return new Sim<float, 2>(); }
}  // namespace wl
