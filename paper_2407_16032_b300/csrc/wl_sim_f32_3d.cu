// wl_sim_f32_3d.cu -- Sim<float, 3>: the FP32 3D time step.
#include "wl_sim.cuh"

namespace wl {
SimBase *new_sim_f32_3d() { return new Sim<float, 3>(); }
}  // namespace wl
